"""The FP64 dslash with 4, 8 or 16 lanes per site (WD_OPT_DSLASH_VARIANT 3, 4, 5) against the oracle.

These kernels split each site of Eq. (1) over several lanes (one direction, one hop, or one hop and
one half-spinor row each) and sum the lanes' spinors by shuffles before applying -kappa. Checked:
the operator and its dagger element by element at 1e-13 over the sizes of the other dslash tests
(L = 2 extents, ragged volumes, several blocks per launch), every boundary pattern, and the CG built
on them in all three loop modes (host loop, graph, and the persistent kernel, whose iteration with
4 or more lanes is fused into two passes that form p = s + beta p and r = r - alpha q on the fly at
the neighbours): true residual from the oracle, the oracle's CGLS iterate after exactly 10
iterations (which pins alpha, beta and every update), an initial guess (the b - D x epilogue), and
the reliable updates of a mixed-precision solve in native FP64.
"""
import numpy as np
import pytest

from oracle import cg as ocg
from oracle import wilson
from tests.gpu_util import fields, rel, require_gpu, to_dev, to_np

pytestmark = pytest.mark.gpu

BC = (1, 1, 1, -1)
SIZES = [(2, 2, 2, 2), (4, 4, 4, 4), (2, 3, 4, 5), (6, 4, 4, 8), (3, 5, 7, 2), (8, 8, 8, 8), (14, 14, 14, 14)]
VARIANTS = {4: 3, 8: 4, 16: 5}   # lanes per site -> option value


@pytest.mark.parametrize("dims", SIZES)
@pytest.mark.parametrize("lanes", [4, 8, 16])
def test_lanes_dslash_matches_oracle(dims, lanes):
    wd = require_gpu()
    U, psi = fields(dims)
    op = wd.WilsonDirac(dims, 0.12, BC, wd.WD_PREC_F64)
    op.load_gauge(to_dev(U))
    op.set_option(wd.WD_OPT_DSLASH_VARIANT, VARIANTS[lanes])
    for block in (32, 64, 128, 256):
        op.set_option(wd.WD_OPT_BLOCK_DSLASH, block)
        for dagger in (False, True):
            out = to_np(op.apply(to_dev(psi), dagger=dagger))
            assert rel(out, wilson.apply_D(U, psi, 0.12, BC, dagger)) < 1e-13, (block, dagger)
    op.close()


@pytest.mark.parametrize("bc", [(-1, 1, -1, 1), (1, 1, 1, 1), (-1, -1, -1, -1), (1, -1, 1, 1)])
@pytest.mark.parametrize("lanes", [4, 8, 16])
def test_lanes_dslash_boundaries(bc, lanes):
    wd = require_gpu()
    dims = (4, 2, 3, 6)
    U, psi = fields(dims)
    op = wd.WilsonDirac(dims, 0.137, bc, wd.WD_PREC_F64)
    op.load_gauge(to_dev(U))
    op.set_option(wd.WD_OPT_DSLASH_VARIANT, VARIANTS[lanes])
    for dagger in (False, True):
        out = to_np(op.apply(to_dev(psi), dagger=dagger))
        assert rel(out, wilson.apply_D(U, psi, 0.137, bc, dagger)) < 1e-13
    op.close()


def _solve(wd, dims, lanes, mode, U, eta, tol=1e-10, maxit=4000, x0=None, block=0):
    op = wd.WilsonDirac(dims, 0.12, BC, wd.WD_PREC_F64)
    op.load_gauge(to_dev(U))
    op.set_option(wd.WD_OPT_DSLASH_VARIANT, VARIANTS[lanes])
    if block:
        op.set_option(wd.WD_OPT_BLOCK_DSLASH, block)
    op.set_option(wd.WD_OPT_USE_GRAPH, mode)
    x, iters, res, st = op.solve(to_dev(eta), x0=None if x0 is None else to_dev(x0), tol=tol, maxit=maxit)
    stats = op.stats()
    op.close()
    return to_np(x), iters, res, st, stats


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 4, 5), (8, 8, 8, 8)])
@pytest.mark.parametrize("lanes", [4, 8, 16])
def test_lanes_cg_in_every_loop_mode(dims, lanes):
    wd = require_gpu()
    U, eta = fields(dims)
    _, k_or, _, _ = ocg.cgls(U, eta, 0.12, 1e-10, 4000)
    for mode in (0, 1, 2):
        x, iters, res, st, stats = _solve(wd, dims, lanes, mode, U, eta)
        assert st == wd.WD_OK, mode
        true = ocg.true_residual(U, eta, x, 0.12)
        assert true <= 1e-10 * 1.01 and abs(res - true) < 1e-12, mode
        assert abs(iters - k_or) <= 2, (mode, iters, k_or)
        if mode == 2:
            assert stats["loop_mode"] == 2 and stats["loop_lanes"] == lanes


@pytest.mark.parametrize("lanes", [4, 8, 16])
@pytest.mark.parametrize("block", [64, 256])
def test_lanes_persistent_loop_ten_iterations_match_oracle(lanes, block):
    wd = require_gpu()
    dims = (4, 4, 4, 6)
    U, eta = fields(dims)
    x, iters, res, st, _ = _solve(wd, dims, lanes, 2, U, eta, maxit=10, block=block)
    assert st == wd.WD_NOT_CONVERGED and iters == 10
    xo, _, ro, _ = ocg.cgls(U, eta, 0.12, 0.0, 10)
    assert rel(x, xo) < 1e-10 and abs(res - ro) < 1e-10


@pytest.mark.parametrize("lanes", [4, 8, 16])
def test_lanes_initial_guess_and_repeatability(lanes):
    wd = require_gpu()
    dims = (6, 4, 4, 4)
    U, eta = fields(dims)
    rng = np.random.default_rng(3)
    x0 = 0.1 * (rng.standard_normal(eta.shape) + 1j * rng.standard_normal(eta.shape))
    a = _solve(wd, dims, lanes, 2, U, eta, maxit=7, x0=x0)
    xo, _, ro, _ = ocg.cgls(U, eta, 0.12, 0.0, 7, x0=x0)
    assert rel(a[0], xo) < 1e-10 and abs(a[2] - ro) < 1e-10
    b = _solve(wd, dims, lanes, 2, U, eta, maxit=7, x0=x0)
    assert np.array_equal(a[0], b[0]) and a[2] == b[2]   # fixed reduction order: same bits


def test_lanes_in_fp64_reliable_updates():
    wd = require_gpu()
    dims = (6, 4, 4, 10)
    U, eta = fields(dims)
    for lanes in (4, 8, 16):
        op = wd.WilsonDirac(dims, 0.12, BC, wd.WD_PREC_MIXED_F32)
        op.set_option(wd.WD_OPT_DF_UPDATES, 0)
        op.load_gauge(to_dev(U), compress12=True)
        op.set_option(wd.WD_OPT_DSLASH_VARIANT, VARIANTS[lanes])
        x, iters, res, st = op.solve(to_dev(eta), tol=1e-10)
        s = op.stats()
        op.close()
        assert st == wd.WD_OK and s["reliable_updates"] > 0
        assert ocg.true_residual(U, eta, to_np(x), 0.12) <= 1e-10 * 1.01


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (8, 8, 8, 8)])
def test_loop_tuner_choice_solves_and_repeats(dims):
    """The default path: the loop's launch shape is timed on the loop itself on the first solve;
    the solve is still correct, the tuner's runs leave no trace in it, and later solves (another
    context of the same shape included) give the same bits."""
    wd = require_gpu()
    U, eta = fields(dims)
    res = []
    for _ in range(2):
        op = wd.WilsonDirac(dims, 0.12, BC, wd.WD_PREC_F64)
        op.load_gauge(to_dev(U))
        x, iters, r, st = op.solve(to_dev(eta), tol=1e-10)
        s = op.stats()
        op.close()
        assert st == wd.WD_OK and s["loop_mode"] == 2 and s["loop_lanes"] in (1, 2, 4, 8, 16)
        assert ocg.true_residual(U, eta, to_np(x), 0.12) <= 1e-10 * 1.01
        res.append((to_np(x), iters, r))
    assert np.array_equal(res[0][0], res[1][0]) and res[0][1:] == res[1][1:]


@pytest.mark.parametrize("lanes", [4, 8, 16])
def test_lanes_with_32_thread_blocks_solve(lanes):
    """The widest grids (16 lanes per site, 32 threads per block: V / 2 blocks, each with a reduction
    partial) in the prologue's fused-norm dslash and in the loop: the solve meets the oracle."""
    wd = require_gpu()
    dims = (8, 8, 8, 8)
    U, eta = fields(dims)
    for mode in (1, 2):
        x, iters, res, st, stats = _solve(wd, dims, lanes, mode, U, eta, block=32)
        assert st == wd.WD_OK and 60 < iters < 120, (mode, iters)
        assert ocg.true_residual(U, eta, x, 0.12) <= 1e-10 * 1.01
