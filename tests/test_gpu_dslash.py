"""Parity of the CUDA dslash (wd_apply through the C ABI) with the FP64 CPU oracle.

Tolerances (relative 2-norm over the field): 1e-13 for FP64, 1e-6 for FP32 (18- and 12-real
links). Sizes span ragged tails (V not a multiple of the block size), L = 2 extents, mixed
boundaries, the paper's largest volume (14^4) and sampled sites of a 32^4 lattice.
"""
import numpy as np
import pytest
import torch

import synthetic
from oracle import freefield, wilson
from oracle.gamma import GAMMA5
from tests.gpu_util import fields, rel, require_gpu, to_dev, to_np

pytestmark = pytest.mark.gpu

BC = (1, 1, 1, -1)
SIZES = [(2, 2, 2, 2), (4, 4, 4, 4), (2, 3, 4, 5), (6, 4, 4, 8), (3, 5, 7, 2), (8, 8, 8, 8), (14, 14, 14, 14)]


@pytest.mark.parametrize("dims", SIZES)
@pytest.mark.parametrize("dagger", [False, True])
def test_fp64_dslash_matches_oracle(dims, dagger):
    wd = require_gpu()
    U, psi = fields(dims)
    op = wd.WilsonDirac(dims, 0.12, BC, wd.WD_PREC_F64)
    dev = op.load_gauge(to_dev(U))
    assert dev < 1e-13
    out = to_np(op.apply(to_dev(psi), dagger=dagger))
    ref = wilson.apply_D(U, psi, 0.12, BC, dagger)
    assert rel(out, ref) < 1e-13
    op.close()


@pytest.mark.parametrize("bc", [(-1, 1, -1, 1), (1, 1, 1, 1), (-1, -1, -1, -1)])
def test_fp64_dslash_boundaries(bc):
    wd = require_gpu()
    dims = (4, 2, 3, 6)
    U, psi = fields(dims)
    op = wd.WilsonDirac(dims, 0.137, bc, wd.WD_PREC_F64)
    op.load_gauge(to_dev(U))
    for dagger in (False, True):
        out = to_np(op.apply(to_dev(psi), dagger=dagger))
        assert rel(out, wilson.apply_D(U, psi, 0.137, bc, dagger)) < 1e-13
    op.close()


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 3, 4, 5), (8, 8, 8, 8), (14, 14, 14, 14)])
@pytest.mark.parametrize("c12", [False, True])
def test_fp32_dslash_matches_oracle(dims, c12):
    wd = require_gpu()
    U, psi = fields(dims)
    op = wd.WilsonDirac(dims, 0.12, BC, wd.WD_PREC_F32)
    op.load_gauge(to_dev(U), compress12=c12)
    for dagger in (False, True):
        out = to_np(op.apply(to_dev(psi, torch.complex64), dagger=dagger))
        ref = wilson.apply_D(U, psi.astype(np.complex64).astype(np.complex128), 0.12, BC, dagger)
        assert rel(out, ref) < 1e-6
    op.close()


def test_gamma5_hermiticity_on_gpu_outputs():
    wd = require_gpu()
    dims = (4, 6, 4, 4)
    U, psi = fields(dims)
    op = wd.WilsonDirac(dims, 0.125, BC, wd.WD_PREC_F64)
    op.load_gauge(to_dev(U))
    g5psi = wilson.apply_gamma5(psi)
    lhs = wilson.apply_gamma5(to_np(op.apply(to_dev(g5psi))))
    rhs = to_np(op.apply(to_dev(psi), dagger=True))
    assert rel(lhs, rhs) < 1e-14
    op.close()


def test_free_field_plane_wave_on_gpu():
    wd = require_gpu()
    dims = (8, 4, 6, 10)
    op = wd.WilsonDirac(dims, 0.11, BC, wd.WD_PREC_F64)
    op.load_gauge(to_dev(synthetic.unit_gauge(dims)))
    rng = np.random.default_rng(3)
    chi = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
    psi, p = freefield.plane_wave(dims, (1, 2, 3, 4), chi, BC)
    expect, _ = freefield.plane_wave(dims, (1, 2, 3, 4), freefield.symbol(p, 0.11) @ chi, BC)
    assert rel(to_np(op.apply(to_dev(psi))), expect) < 1e-13
    op.close()


def test_gauge_covariance_on_gpu_outputs():
    wd = require_gpu()
    dims = (4, 4, 2, 6)
    U, psi = fields(dims)
    om = synthetic.random_gauge_transform(dims, 11)
    Up = np.empty_like(U)
    for mu in range(4):
        of = np.roll(om, -1, axis=3 - mu)
        Up[..., mu, :, :] = om @ U[..., mu, :, :] @ np.conj(np.swapaxes(of, -1, -2))
    op = wd.WilsonDirac(dims, 0.12, BC, wd.WD_PREC_F64)
    op.load_gauge(to_dev(U))
    a = np.einsum("...ab,...sb->...sa", om, to_np(op.apply(to_dev(psi))))
    op.load_gauge(to_dev(Up))
    b = to_np(op.apply(to_dev(np.einsum("...ab,...sb->...sa", om, psi))))
    assert rel(b, a) < 1e-13
    op.close()


def test_host_gauge_and_twelve_real_unitarity_check():
    wd = require_gpu()
    dims = (4, 4, 4, 4)
    U, psi = fields(dims)
    op = wd.WilsonDirac(dims, 0.12, BC, wd.WD_PREC_F32)
    dev = op.load_gauge(torch.from_numpy(U), compress12=True)  # host pointer path
    assert dev < 1e-13
    bad = U.copy()
    bad[0, 0, 0, 0, 0] *= 1.01
    with pytest.raises(wd.WdError) as e:
        op.load_gauge(torch.from_numpy(bad), compress12=True)
    assert e.value.status == wd.WD_ENOTUNITARY
    op.close()


@pytest.mark.parametrize("dims", [(32, 32, 32, 32)])
def test_full_size_sampled_sites(dims):
    wd = require_gpu()
    U, psi = fields(dims)
    op = wd.WilsonDirac(dims, 0.124, BC, wd.WD_PREC_F64)
    op.load_gauge(to_dev(U))
    rng = np.random.default_rng(7)
    lx, ly, lz, lt = dims
    sites = [(0, 0, 0, 0), (lx - 1, ly - 1, lz - 1, lt - 1), (0, ly - 1, 0, lt - 1)]
    sites += [tuple(int(v) for v in rng.integers(0, (lx, ly, lz, lt))) for _ in range(40)]
    for dagger in (False, True):
        out = to_np(op.apply(to_dev(psi), dagger=dagger))
        ref = wilson.apply_D_sites(U, psi, 0.124, sites, BC, dagger)
        got = np.stack([out[t, z, y, x] for (x, y, z, t) in sites])
        assert rel(got, ref) < 1e-13
    op.close()


def test_api_errors_on_gpu():
    wd = require_gpu()
    op = wd.WilsonDirac((4, 4, 4, 4), 0.12, BC, wd.WD_PREC_F64)
    psi = to_dev(synthetic.gaussian_source((4, 4, 4, 4), 1))
    with pytest.raises(wd.WdError) as e:
        op.apply(psi)
    assert e.value.status == wd.WD_ENOGAUGE
    with pytest.raises(wd.WdError) as e:
        wd.wd_apply(op.ctx, psi, psi)
    assert e.value.status == wd.WD_EINVAL
    with pytest.raises(wd.WdError) as e:
        wd.wd_set_option(op.ctx, wd.WD_OPT_BLOCK_DSLASH, 33)
    assert e.value.status == wd.WD_EINVAL
    op.close()


@pytest.mark.parametrize("dims", SIZES)
@pytest.mark.parametrize("dagger", [False, True])
def test_fp64_two_threads_per_site_matches_oracle(dims, dagger):
    """The FP64 variant in which lanes 2i and 2i+1 share a site (forced)."""
    wd = require_gpu()
    U, psi = fields(dims)
    op = wd.WilsonDirac(dims, 0.12, BC, wd.WD_PREC_F64)
    op.load_gauge(to_dev(U))
    op.set_option(wd.WD_OPT_DSLASH_VARIANT, 2)
    for block in (64, 256):
        op.set_option(wd.WD_OPT_BLOCK_DSLASH, block)
        out = to_np(op.apply(to_dev(psi), dagger=dagger))
        assert rel(out, wilson.apply_D(U, psi, 0.12, BC, dagger)) < 1e-13, block
    op.close()


@pytest.mark.parametrize("bc", [(-1, 1, -1, 1), (1, 1, 1, 1), (-1, -1, -1, -1), (1, -1, 1, 1)])
def test_fp64_two_threads_per_site_boundaries(bc):
    wd = require_gpu()
    dims = (4, 2, 3, 6)
    U, psi = fields(dims)
    op = wd.WilsonDirac(dims, 0.137, bc, wd.WD_PREC_F64)
    op.load_gauge(to_dev(U))
    op.set_option(wd.WD_OPT_DSLASH_VARIANT, 2)
    for dagger in (False, True):
        out = to_np(op.apply(to_dev(psi), dagger=dagger))
        assert rel(out, wilson.apply_D(U, psi, 0.137, bc, dagger)) < 1e-13
    op.close()


def test_fp64_two_threads_per_site_in_solves_and_its_errors():
    wd = require_gpu()
    from oracle import cg as ocg
    dims = (6, 4, 4, 10)
    U, eta = fields(dims)
    for prec, c12 in ((wd.WD_PREC_F64, False), (wd.WD_PREC_MIXED_F16, True)):
        op = wd.WilsonDirac(dims, 0.12, BC, prec)
        op.load_gauge(to_dev(U), compress12=c12)
        op.set_option(wd.WD_OPT_DSLASH_VARIANT, 2)
        x, iters, res, st = op.solve(to_dev(eta), tol=1e-10)
        assert st == wd.WD_OK and ocg.true_residual(U, eta, to_np(x), 0.12) <= 1e-10
        assert abs(res - ocg.true_residual(U, eta, to_np(x), 0.12)) < 1e-12
        op.close()
    op = wd.WilsonDirac(dims, 0.12, BC, wd.WD_PREC_F32)
    with pytest.raises(wd.WdError) as e:
        op.set_option(wd.WD_OPT_DSLASH_VARIANT, 2)
    assert e.value.status == wd.WD_EINVAL
    with pytest.raises(wd.WdError):
        op.set_option(wd.WD_OPT_DSLASH_VARIANT, 3)
    op.close()
