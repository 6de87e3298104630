"""wd_dslash_noalloc: the dslash with fused norm for callers that cannot allocate device memory.

Such callers (code under an allocator that must own every device allocation, plug-ins handed
fixed buffers) cannot create a context, so this entry point takes all inputs and outputs from
the caller and keeps its reduction scratch in a fixed array inside the library. The test calls it
through the C ABI twice in a row and checks both results against the context-based wd_apply and
against the CPU oracle's operator of Eq. (1). This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import wilson
from tests.gpu_util import fields, rel, require_gpu, to_dev

pytestmark = pytest.mark.gpu

BC = (1, 1, 1, -1)


def _call(lib, dims, kappa, U, psi, out, dagger, norm, stream):
    d = (ctypes.c_int * 4)(*dims)
    b = (ctypes.c_int * 4)(*BC)
    return lib.wd_dslash_noalloc(d, ctypes.c_double(kappa), b, ctypes.c_void_p(U.data_ptr()),
                                 ctypes.c_void_p(psi.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                 int(dagger), ctypes.c_void_p(norm.data_ptr()) if norm is not None else None,
                                 ctypes.c_void_p(stream))


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 5, 4, 7), (16, 16, 16, 16)])
def test_noalloc_matches_wd_apply_on_two_calls(dims):
    wd = require_gpu()
    lib = wd._lib
    U, psi = fields(dims)
    Ud, psid = to_dev(U), to_dev(psi)
    stream = torch.cuda.current_stream().cuda_stream
    op = wd.WilsonDirac(dims, 0.12, BC, wd.WD_PREC_F64)
    op.load_gauge(Ud)
    for dagger in (False, True):
        ref = op.apply(psid, dagger=dagger)
        ref_norm = float((ref.abs() ** 2).sum())
        orc = wilson.apply_D(U, psi, 0.12, BC, dagger=dagger)
        orc_norm = wilson.norm2(orc)
        for _ in range(2):  # the shared scratch keeps the previous call's contents
            out = torch.full_like(psid, float("nan"))
            norm = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            assert _call(lib, dims, 0.12, Ud, psid, out, dagger, norm, stream) == wd.WD_OK
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            assert rel(got, ref.cpu().numpy()) < 1e-13
            assert abs(float(norm.item()) - ref_norm) <= 1e-12 * ref_norm
            assert wilson.rel_diff(got, orc) < 1e-13
            assert abs(float(norm.item()) - orc_norm) <= 1e-12 * orc_norm
    op.close()


def test_noalloc_rejects_volume_beyond_scratch():
    wd = require_gpu()
    small = torch.zeros(16, dtype=torch.complex128, device="cuda")
    other = torch.zeros(16, dtype=torch.complex128, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    # 32^3 x 33 > 2^20 sites: rejected before any pointer is used
    st = _call(wd._lib, (32, 32, 32, 33), 0.12, small, small, other, False, None, stream)
    assert st == wd.WD_EINVAL
    assert "2^20" in wd.wd_last_error()


def test_noalloc_without_norm_and_through_binding():
    wd = require_gpu()
    dims = (4, 2, 6, 4)
    U, psi = fields(dims)
    Ud, psid = to_dev(U), to_dev(psi)
    op = wd.WilsonDirac(dims, 0.13, BC, wd.WD_PREC_F64)
    op.load_gauge(Ud)
    ref = op.apply(psid).cpu().numpy()
    out = torch.empty_like(psid)
    wd.wd_dslash_noalloc(dims, 0.13, Ud, psid, out)
    torch.cuda.synchronize()
    assert rel(out.cpu().numpy(), ref) < 1e-13
    assert wilson.rel_diff(out.cpu().numpy(), wilson.apply_D(U, psi, 0.13, BC)) < 1e-13
    op.close()
    assert np.isfinite(ref).all()
