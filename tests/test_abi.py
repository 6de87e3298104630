"""The C-ABI library loads and exports every function include/wd.h declares (no GPU needed)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fname in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fname.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fname)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M):
            if m.group(1) not in ("defined",):
                names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2111_14958_gb300 import build
    build.build()
    import ctypes
    return ctypes.CDLL(os.path.join(ROOT, "paper_2111_14958_gb300", "libwdcg.so"))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("wd_create", "wd_load_gauge", "wd_apply", "cg_solve", "wd_destroy", "wd_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_names_match_header(lib):
    from paper_2111_14958_gb300 import wd
    assert set(_declared()) == set(wd.EXPORTED)


def test_version_and_no_device_error(lib):
    import torch
    from paper_2111_14958_gb300 import wd
    assert "sm_103a" in wd.wd_version()
    if not torch.cuda.is_available():
        with pytest.raises(wd.WdError) as e:
            wd.wd_create((4, 4, 4, 4), 0.12, stream=0)
        assert e.value.status == wd.WD_ECUDA


def test_argument_validation_without_device(lib):
    import ctypes
    from paper_2111_14958_gb300 import wd
    out = ctypes.c_void_p()
    bad = (ctypes.c_int * 4)(4, 4, 1, 4)
    assert lib.wd_create(bad, ctypes.c_double(0.12), None, 64, None, ctypes.byref(out)) == wd.WD_EINVAL
    good = (ctypes.c_int * 4)(4, 4, 4, 4)
    assert lib.wd_create(good, ctypes.c_double(0.12), None, 7, None, ctypes.byref(out)) == wd.WD_EINVAL
    assert lib.wd_create(good, ctypes.c_double(1.5), None, 64, None, ctypes.byref(out)) == wd.WD_EINVAL
    bc = (ctypes.c_int * 4)(1, 1, 1, 0)
    assert lib.wd_create(good, ctypes.c_double(0.12), bc, 64, None, ctypes.byref(out)) == wd.WD_EINVAL
    assert lib.wd_create(good, ctypes.c_double(0.12), None, 64, None, None) == wd.WD_EINVAL


def test_noalloc_rejects_bad_sizes_and_overlap_before_any_device_call(lib):
    """wd_dslash_noalloc validates on the host first: extents whose product would overflow, a volume
    beyond its fixed scratch, and overlapping in/out ranges are rejected before any CUDA call (the
    addresses below are never dereferenced)."""
    import ctypes
    from paper_2111_14958_gb300 import wd

    def call(dims, U, a, b):
        d = (ctypes.c_int * 4)(*dims)
        return lib.wd_dslash_noalloc(d, ctypes.c_double(0.12), None, ctypes.c_void_p(U), ctypes.c_void_p(a),
                                     ctypes.c_void_p(b), 0, None, None)

    big = 1 << 30
    assert call((big, big, big, big), 0x100000, 0x200000, 0x300000) == wd.WD_EINVAL
    assert "2^20" in wd.wd_last_error()
    assert call((32, 32, 32, 33), 0x100000, 0x200000, 0x300000) == wd.WD_EINVAL
    n = 4 ** 4 * 12 * 16  # bytes of one 4^4 complex128 spinor field
    base = 1 << 40
    assert call((4, 4, 4, 4), 0x100000, base, base + 16) == wd.WD_EINVAL
    assert "overlap" in wd.wd_last_error()
    assert call((4, 4, 4, 4), 0x100000, base + 16, base) == wd.WD_EINVAL
    assert call((4, 4, 4, 4), 0x100000, base, base) == wd.WD_EINVAL


def test_binding_rejects_mistyped_fields_before_the_library(lib):
    """The binding refuses fields the library would read or write past their end: cg_solve takes
    complex128 for every precision, wd_apply one complex dtype and size on both sides (CPU tensors
    are refused too, before any device call)."""
    import torch
    from paper_2111_14958_gb300 import wd
    c128 = torch.zeros((2, 2, 2, 2, 4, 3), dtype=torch.complex128)
    c64 = torch.zeros((2, 2, 2, 2, 4, 3), dtype=torch.complex64)
    for src, x in ((c64, c64), (c128, c64), (c64, c128), (c128, c128)):   # the last: not on a device
        with pytest.raises(ValueError):
            wd.cg_solve(None, src, x, 1e-6, 10)
    for inp, out in ((c64, c128), (c128, c128[:1]), (c128, c128.clone())):
        with pytest.raises(ValueError):
            wd.wd_apply(None, inp, out)


def test_checkpoint_calls_validate_before_any_device_call(lib):
    """wd_cg_state_size / wd_cg_save_state / cg_resume refuse a null context (and the binding a
    mistyped field) without touching a device."""
    import ctypes
    import torch
    from paper_2111_14958_gb300 import wd
    n = ctypes.c_size_t()
    assert lib.wd_cg_state_size(None, ctypes.byref(n)) == wd.WD_EINVAL
    buf = ctypes.create_string_buffer(64)
    assert lib.wd_cg_save_state(None, buf, 64) == wd.WD_EINVAL
    assert lib.cg_resume(None, buf, 64, None, None, ctypes.c_double(1e-10), 10, None, None) == wd.WD_EINVAL
    assert "null context" in wd.wd_last_error()
    c128 = torch.zeros((2, 2, 2, 2, 4, 3), dtype=torch.complex128)
    with pytest.raises(ValueError):
        wd.cg_resume(None, bytes(64), c128, c128.to(torch.complex64), 1e-10, 10)
