"""The persistent FP64 CG loop in the spin basis where gamma_t is diagonal (WD_OPT_LOOP_TIME_BASIS).

With T = [[1, 1], [-1, 1]] on the (upper, lower) spins, T gamma_k T^-1 = gamma_k for the spatial
gammas of the chiral basis and T gamma_t T^-1 = diag(1, 1, -1, -1), so the loop can run CGLS on
T D T^-1 (Eq. (1) with those gammas) with x, r, p, s held as T times the chiral vectors: a time hop
then needs no spin projection. The solve's inputs and outputs stay in the chiral basis. Checked
against the FP64 CPU oracle: the CGLS iterate after exactly 10 iterations from an initial guess
(which pins the entry and exit transforms, alpha, beta and every update), the recursive residual
history (the loop's norms are twice the chiral ones inside and must be reported halved), converged
solves (true residual from the oracle) over L = 2 and ragged extents and every time boundary, and
the same loop in the chiral basis (same iterations within one).
"""
import numpy as np
import pytest
import torch

from oracle import cg as ocg
from tests.gpu_util import fields, rel, require_gpu, to_dev, to_np

pytestmark = pytest.mark.gpu

SIZES = [(4, 4, 4, 4), (6, 4, 4, 5), (3, 5, 4, 2), (2, 2, 2, 2), (14, 14, 14, 14)]
BOUNDARIES = [(1, 1, 1, -1), (1, 1, 1, 1), (-1, 1, -1, -1)]


def _solve(wd, dims, bc, basis, U, eta, tol=1e-10, maxit=4000, x0=None, history=0):
    op = wd.WilsonDirac(dims, 0.12, bc, wd.WD_PREC_F64)
    op.load_gauge(to_dev(U))
    op.set_option(wd.WD_OPT_USE_GRAPH, 2)        # the persistent loop
    op.set_option(wd.WD_OPT_DSLASH_VARIANT, 1)   # one thread per site (the loop the basis serves)
    op.set_option(wd.WD_OPT_LOOP_TIME_BASIS, basis)
    if history:
        op.set_option(wd.WD_OPT_RESIDUAL_HISTORY, history)
    x, iters, res, st = op.solve(to_dev(eta), x0=None if x0 is None else to_dev(x0), tol=tol, maxit=maxit)
    stats = op.stats()
    h = np.array(op.residual_history()) if history else None
    op.close()
    return to_np(x), iters, res, st, stats, h


@pytest.mark.parametrize("dims", SIZES)
@pytest.mark.parametrize("bc", BOUNDARIES)
def test_ten_iterations_from_a_guess_match_the_oracle(dims, bc):
    wd = require_gpu()
    U, eta = fields(dims)
    rng = np.random.default_rng(5)
    x0 = 0.1 * (rng.standard_normal(eta.shape) + 1j * rng.standard_normal(eta.shape))
    xo, _, ro, _ = ocg.cgls(U, eta, 0.12, 0.0, 10, x0=x0, boundary=bc)
    for basis in (1, 0):
        x, iters, res, st, stats, _ = _solve(wd, dims, bc, basis, U, eta, maxit=10, x0=x0)
        assert st == wd.WD_NOT_CONVERGED and iters == 10, basis
        assert stats["loop_mode"] == 2 and stats["loop_lanes"] == 1
        assert rel(x, xo) < 1e-10 and abs(res - ro) < 1e-10, basis


@pytest.mark.parametrize("dims", SIZES)
@pytest.mark.parametrize("bc", BOUNDARIES)
def test_converged_solves_match_the_oracle_and_the_chiral_loop(dims, bc):
    wd = require_gpu()
    U, eta = fields(dims)
    got = {}
    for basis in (1, 0):
        x, iters, res, st, _, _ = _solve(wd, dims, bc, basis, U, eta)
        assert st == wd.WD_OK, basis
        true = ocg.true_residual(U, eta, x, 0.12, bc)
        assert true <= 1e-10 and abs(res - true) < 1e-12, basis
        got[basis] = (x, iters)
    assert abs(got[1][1] - got[0][1]) <= 1
    assert rel(got[1][0], got[0][0]) < 1e-8


def test_residual_history_is_reported_in_the_chiral_norm():
    wd = require_gpu()
    dims = (4, 4, 4, 6)
    bc = (1, 1, 1, -1)
    U, eta = fields(dims)
    _, io, _, ho = ocg.cgls(U, eta, 0.12, 1e-10, 2000)
    x, iters, res, st, _, h = _solve(wd, dims, bc, 1, U, eta, history=500)
    assert st == wd.WD_OK and len(h) == iters and abs(iters - io) <= 1
    assert np.max(np.abs(h[:20] / ho[1:21] - 1)) < 1e-9   # a factor 2 would show as 0.41
    n = min(len(h), len(ho) - 1)
    assert np.max(np.abs(h[:n] / ho[1:n + 1] - 1)) < 1e-3


def test_basis_solves_repeat_bitwise_and_the_option_is_checked():
    wd = require_gpu()
    dims = (6, 4, 4, 8)
    bc = (1, 1, 1, -1)
    U, eta = fields(dims)
    a = _solve(wd, dims, bc, 1, U, eta)
    b = _solve(wd, dims, bc, 1, U, eta)
    assert np.array_equal(a[0], b[0]) and a[1:3] == b[1:3]
    op = wd.WilsonDirac(dims, 0.12, bc, wd.WD_PREC_F64)
    for bad in (-1, 2, 0.5):
        with pytest.raises(wd.WdError):
            op.set_option(wd.WD_OPT_LOOP_TIME_BASIS, bad)
    op.close()


def test_batched_loops_in_the_basis_equal_solves_alone_bitwise():
    """cg_solve_batch runs each problem's loop on its own blocks of one launch: with the basis on,
    every result equals its solve alone bit for bit, and meets the tolerance by the oracle."""
    wd = require_gpu()
    dims = (6, 4, 4, 8)
    bc = (1, 1, 1, -1)
    probs = [fields(dims, gseed=10 + i, sseed=20 + i) for i in range(3)]

    def make(U):
        op = wd.WilsonDirac(dims, 0.12, bc, wd.WD_PREC_F64)
        op.load_gauge(to_dev(U))
        op.set_option(wd.WD_OPT_DSLASH_VARIANT, 1)
        op.set_option(wd.WD_OPT_LOOP_TIME_BASIS, 1)
        return op

    ops = [make(U) for U, _ in probs]
    srcs = [to_dev(eta) for _, eta in probs]
    xs = [torch.zeros_like(s) for s in srcs]
    st, iters, res, sts = wd.cg_solve_batch([o.ctx for o in ops], srcs, xs, [1e-10] * 3, 4000)
    modes = [(o.stats()["loop_mode"], o.stats()["loop_lanes"]) for o in ops]
    for o in ops:
        o.close()
    assert st == wd.WD_OK and all(s == wd.WD_OK for s in sts) and all(m == (2, 1) for m in modes)
    for i, (U, eta) in enumerate(probs):
        op = make(U)
        xa, ia, ra, sa = op.solve(to_dev(eta), tol=1e-10)
        op.close()
        assert sa == wd.WD_OK and ia == iters[i] and ra == res[i]
        assert np.array_equal(to_np(xs[i]), to_np(xa)), i
        assert ocg.true_residual(U, eta, to_np(xa), 0.12, bc) <= 1e-10
