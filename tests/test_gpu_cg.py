"""CG solves through the C ABI, checked against the FP64 CPU oracle.

Every solve's true relative residual is recomputed by the oracle in FP64 from the returned x and
must meet the tolerance; solutions are compared with the oracle's CGLS and, at 4^4, with a dense
direct solve.
"""
import json
import os

import numpy as np
import pytest
import torch

import synthetic
from oracle import cg as ocg
from oracle import freefield, wilson
from tests.gpu_util import fields, rel, require_gpu, to_dev, to_np

pytestmark = pytest.mark.gpu

BC = (1, 1, 1, -1)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "cgls_oracle.json")


def _solve(wd, dims, kappa, prec, tol, maxit=4000, U=None, eta=None, graph=True, c12=False, options=None):
    if U is None:
        U, eta = fields(dims)
    op = wd.WilsonDirac(dims, kappa, BC, prec)
    op.load_gauge(to_dev(U), compress12=c12)
    if not graph:
        op.set_option(wd.WD_OPT_USE_GRAPH, 0)
    for k, v in (options or {}).items():
        op.set_option(k, v)
    x, iters, res, status = op.solve(to_dev(eta), tol=tol, maxit=maxit)
    stats = op.stats()
    op.close()
    return to_np(x), iters, res, status, stats, U, eta


def test_c1_fp64_matches_oracle_and_direct_solve():
    wd = require_gpu()
    with open(GOLDEN) as f:
        golden = json.load(f)["solves"][0]
    dims = tuple(golden["dims"])
    x, iters, res, status, stats, U, eta = _solve(wd, dims, 0.12, wd.WD_PREC_F64, 1e-10)
    assert status == wd.WD_OK
    assert ocg.true_residual(U, eta, x, 0.12) <= 1e-10
    assert abs(res - ocg.true_residual(U, eta, x, 0.12)) < 1e-12
    assert abs(iters - golden["iterations"]) <= 2
    dense = wilson.dense_D(U, 0.12, BC)
    x_direct = np.linalg.solve(dense, eta.reshape(-1))
    assert rel(x, x_direct) < 1e-8


@pytest.mark.parametrize("idx", [1, 2])
def test_golden_cases_fp64(idx):
    wd = require_gpu()
    with open(GOLDEN) as f:
        g = json.load(f)["solves"][idx]
    dims = tuple(g["dims"])
    U = synthetic.gauge_field(dims, g["eps"], g["gauge_seed"])
    eta = synthetic.gaussian_source(dims, g["source_seed"])
    x, iters, res, status, _, _, _ = _solve(wd, dims, g["kappa"], wd.WD_PREC_F64, g["tol"], U=U, eta=eta)
    assert status == wd.WD_OK
    assert ocg.true_residual(U, eta, x, g["kappa"]) <= g["tol"]
    assert abs(iters - g["iterations"]) <= 2


def test_c2_fp64_and_fp32_14x4():
    wd = require_gpu()
    dims = (14, 14, 14, 14)
    U, eta = fields(dims)
    x64, it64, res64, st64, _, _, _ = _solve(wd, dims, 0.12, wd.WD_PREC_F64, 1e-10, U=U, eta=eta)
    assert st64 == wd.WD_OK
    assert ocg.true_residual(U, eta, x64, 0.12) <= 1e-10
    x32, it32, res32, st32, _, _, _ = _solve(wd, dims, 0.12, wd.WD_PREC_F32, 1e-6, U=U, eta=eta, c12=True)
    assert st32 == wd.WD_OK
    assert ocg.true_residual(U, eta, x32, 0.12) <= 1.05e-6
    assert rel(x32, x64) < 1e-4


@pytest.mark.parametrize("prec", ["mixed32", "mixed16"])
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (14, 14, 14, 14)])
def test_mixed_precision_reaches_fp64_accuracy(prec, dims):
    wd = require_gpu()
    p = wd.WD_PREC_MIXED_F32 if prec == "mixed32" else wd.WD_PREC_MIXED_F16
    U, eta = fields(dims)
    x, iters, res, status, stats, _, _ = _solve(wd, dims, 0.12, p, 1e-10, U=U, eta=eta, c12=True)
    assert status == wd.WD_OK, stats
    assert ocg.true_residual(U, eta, x, 0.12) <= 1e-10
    assert stats["reliable_updates"] >= 1


def test_graph_and_host_loop_agree_bitwise():
    wd = require_gpu()
    dims = (6, 4, 4, 8)
    U, eta = fields(dims)
    # a fixed block size: the reduction tree (hence the last bits of every scalar) depends on it;
    # the chiral basis in the persistent loop (the time-diagonal basis rounds differently)
    fix = {wd.WD_OPT_BLOCK_DSLASH: 128, wd.WD_OPT_LOOP_TIME_BASIS: 0}
    xa, ia, _, _, _, _, _ = _solve(wd, dims, 0.124, wd.WD_PREC_F64, 1e-10, U=U, eta=eta, graph=True, options=fix)
    xb, ib, _, _, _, _, _ = _solve(wd, dims, 0.124, wd.WD_PREC_F64, 1e-10, U=U, eta=eta, graph=False, options=fix)
    xc, ic, _, _, _, _, _ = _solve(wd, dims, 0.124, wd.WD_PREC_F64, 1e-10, U=U, eta=eta, graph=True, options=fix)
    assert ia == ib == ic
    assert np.array_equal(xa, xb) and np.array_equal(xa, xc)
    xd, id_, _, _, _, _, _ = _solve(wd, dims, 0.124, wd.WD_PREC_F64, 1e-10, U=U, eta=eta, graph=True,
                                    options={wd.WD_OPT_BLOCK_DSLASH: 128})
    assert abs(id_ - ia) <= 1 and rel(xd, xa) < 1e-8


def test_mixed_graph_and_host_loop_agree():
    wd = require_gpu()
    dims = (6, 4, 4, 8)
    U, eta = fields(dims)
    fix = {wd.WD_OPT_BLOCK_DSLASH: 128}
    xa, ia, _, _, sa, _, _ = _solve(wd, dims, 0.124, wd.WD_PREC_MIXED_F32, 1e-10, U=U, eta=eta, graph=True, options=fix)
    xb, ib, _, _, sb, _, _ = _solve(wd, dims, 0.124, wd.WD_PREC_MIXED_F32, 1e-10, U=U, eta=eta, graph=False, options=fix)
    assert ia == ib and sa["reliable_updates"] == sb["reliable_updates"]
    assert np.array_equal(xa, xb)


def test_free_field_solve_matches_fft():
    wd = require_gpu()
    dims = (8, 8, 8, 8)
    U = synthetic.unit_gauge(dims)
    eta = synthetic.gaussian_source(dims, 4)
    x, _, _, status, _, _, _ = _solve(wd, dims, 0.124, wd.WD_PREC_F64, 1e-12, U=U, eta=eta)
    assert status == wd.WD_OK
    assert rel(x, freefield.solve(eta, 0.124, BC)) < 1e-10


def test_kappa_zero_is_one_iteration():
    wd = require_gpu()
    dims = (4, 2, 2, 4)
    U, eta = fields(dims)
    x, iters, res, status, _, _, _ = _solve(wd, dims, 0.0, wd.WD_PREC_F64, 1e-12, U=U, eta=eta)
    assert status == wd.WD_OK and iters == 1
    assert rel(x, eta) < 1e-15


def test_maxit_returns_not_converged_with_iterate():
    wd = require_gpu()
    dims = (4, 4, 4, 4)
    U, eta = fields(dims)
    x, iters, res, status, _, _, _ = _solve(wd, dims, 0.12, wd.WD_PREC_F64, 1e-10, maxit=10, U=U, eta=eta)
    assert status == wd.WD_NOT_CONVERGED and iters == 10
    xo, _, ro, _ = ocg.cgls(U, eta, 0.12, 0.0, 10)
    assert rel(x, xo) < 1e-10 and abs(res - ro) < 1e-10


def test_zero_source_and_exact_guess():
    wd = require_gpu()
    dims = (4, 4, 2, 2)
    U, eta = fields(dims)
    op = wd.WilsonDirac(dims, 0.12, BC, wd.WD_PREC_F64)
    op.load_gauge(to_dev(U))
    zero = torch.zeros(op.spinor_shape, dtype=torch.complex128, device="cuda")
    x, iters, res, status = op.solve(zero, tol=1e-10)
    assert status == wd.WD_OK and iters == 0 and float(x.abs().max()) == 0.0
    # an exact initial guess needs no iteration
    xs = to_dev(np.linalg.solve(wilson.dense_D(U, 0.12, BC), eta.reshape(-1)).reshape(eta.shape))
    x, iters, res, status = op.solve(to_dev(eta), x0=xs, tol=1e-10)
    assert status == wd.WD_OK and iters == 0
    op.close()


def test_nan_source_is_breakdown():
    wd = require_gpu()
    dims = (4, 4, 2, 2)
    U, eta = fields(dims)
    eta = eta.copy()
    eta[0, 0, 0, 1, 2, 1] = np.nan
    x, iters, res, status, _, _, _ = _solve(wd, dims, 0.12, wd.WD_PREC_F64, 1e-10, U=U, eta=eta)
    assert status == wd.WD_BREAKDOWN


def test_repeated_solves_are_bitwise_identical():
    wd = require_gpu()
    dims = (8, 8, 8, 8)
    U, eta = fields(dims)
    op = wd.WilsonDirac(dims, 0.12, BC, wd.WD_PREC_MIXED_F32)
    op.load_gauge(to_dev(U), compress12=True)
    a = op.solve(to_dev(eta), tol=1e-10)[0]
    b = op.solve(to_dev(eta), tol=1e-10)[0]
    assert torch.equal(a, b)
    op.close()


@pytest.mark.parametrize("prec", ["f64", "mixed16"])
def test_separate_contexts_agree_bitwise(prec):
    """Launch shapes are tuned once per problem shape, so a second context repeats the first."""
    wd = require_gpu()
    dims = (8, 8, 8, 12)
    U, eta = fields(dims)
    p = wd.WD_PREC_F64 if prec == "f64" else wd.WD_PREC_MIXED_F16
    xs = []
    for _ in range(2):
        op = wd.WilsonDirac(dims, 0.12, BC, p)
        op.load_gauge(to_dev(U), compress12=prec != "f64")
        x, iters, res, st = op.solve(to_dev(eta), tol=1e-10)
        assert st == wd.WD_OK
        xs.append((x, iters, res))
        op.close()
    assert xs[0][1] == xs[1][1] and xs[0][2] == xs[1][2]
    assert torch.equal(xs[0][0], xs[1][0])


# ---------------------------------------------------------------- the paper's CG form (Sec. 2)

@pytest.mark.parametrize("dims,kappa", [((4, 4, 4, 4), 0.12), ((6, 4, 4, 8), 0.124)])
def test_paper_form_fp64_matches_the_oracle_paper_cg(dims, kappa):
    wd = require_gpu()
    x, iters, res, status, stats, U, eta = _solve(wd, dims, kappa, wd.WD_PREC_F64, 1e-10,
                                                  options={wd.WD_OPT_CG_FORM: 1})
    assert status == wd.WD_OK
    xo, io, ro, hist = ocg.cg_paper(U, eta, kappa, 1e-10, 4000)
    assert ocg.true_residual(U, eta, x, kappa) <= 1e-10
    assert abs(res - ocg.true_residual(U, eta, x, kappa)) < 1e-12
    assert abs(iters - io) <= 2
    # both meet 1e-10 on the same non-singular system: they agree to its conditioning
    assert rel(x, xo) < 1e-8


def test_paper_form_fp32_and_even_odd():
    wd = require_gpu()
    dims = (8, 8, 8, 8)
    U, eta = fields(dims)
    x, iters, res, status, _, _, _ = _solve(wd, dims, 0.12, wd.WD_PREC_F32, 1e-6, U=U, eta=eta, c12=True,
                                            options={wd.WD_OPT_CG_FORM: 1})
    assert status == wd.WD_OK and ocg.true_residual(U, eta, x, 0.12) <= 1e-6 * 1.05
    xe, ie, re_, se, _, _, _ = _solve(wd, dims, 0.12, wd.WD_PREC_F64 | wd.WD_EVEN_ODD, 1e-10, U=U, eta=eta,
                                      options={wd.WD_OPT_CG_FORM: 1})
    assert se == wd.WD_OK and ocg.true_residual(U, eta, xe, 0.12) <= 1e-10
    _, ifull, _, _, _, _, _ = _solve(wd, dims, 0.12, wd.WD_PREC_F64, 1e-10, U=U, eta=eta,
                                     options={wd.WD_OPT_CG_FORM: 1})
    assert ie < 0.75 * ifull


def test_paper_form_graph_and_host_loop_agree_bitwise():
    wd = require_gpu()
    dims = (4, 4, 4, 8)
    U, eta = fields(dims)
    a = _solve(wd, dims, 0.12, wd.WD_PREC_F64, 1e-10, U=U, eta=eta,
               options={wd.WD_OPT_CG_FORM: 1, wd.WD_OPT_USE_GRAPH: 1})
    b = _solve(wd, dims, 0.12, wd.WD_PREC_F64, 1e-10, U=U, eta=eta, graph=False, options={wd.WD_OPT_CG_FORM: 1})
    assert a[4]["loop_mode"] == 1 and b[4]["loop_mode"] == 0
    assert a[1] == b[1] and np.array_equal(a[0], b[0])


@pytest.mark.parametrize("prec,tol,basis", [("f64", 1e-10, 1), ("f64", 1e-10, 0), ("f32", 1e-6, 0)])
def test_paper_form_persistent_loop_matches_the_graph_and_the_oracle(prec, tol, basis):
    """The paper's CG as one persistent launch (three grid barriers per iteration): the same
    iterations as its graph within one, both solutions within the system's conditioning of each
    other and of the oracle's paper CG, the tolerance met by the oracle's residual."""
    wd = require_gpu()
    dims = (6, 4, 4, 8)
    U, eta = fields(dims, gseed=61, sseed=62)
    p = wd.WD_PREC_F64 if prec == "f64" else wd.WD_PREC_F32
    opts = {wd.WD_OPT_CG_FORM: 1}
    if prec == "f64":
        opts[wd.WD_OPT_LOOP_TIME_BASIS] = basis
    a = _solve(wd, dims, 0.12, p, tol, U=U, eta=eta, options=dict(opts))
    b = _solve(wd, dims, 0.12, p, tol, U=U, eta=eta, options={**opts, wd.WD_OPT_USE_GRAPH: 1})
    assert a[3] == wd.WD_OK and b[3] == wd.WD_OK
    assert a[4]["loop_mode"] == 2 and a[4]["loop_lanes"] == 1 and b[4]["loop_mode"] == 1
    assert abs(a[1] - b[1]) <= 1
    margin = 1.05 if prec == "f32" else 1.0 + 1e-6
    assert ocg.true_residual(U, eta, a[0], 0.12) <= tol * margin
    assert abs(a[2] - ocg.true_residual(U, eta, a[0], 0.12)) < max(1e-12, 0.05 * tol)
    assert rel(a[0], b[0]) < 1e3 * tol
    if prec == "f64":
        xo, io, _, _ = ocg.cg_paper(U, eta, 0.12, tol, 4000)
        assert abs(a[1] - io) <= 2 and rel(a[0], xo) < 1e-8


def test_paper_form_uses_the_initial_guess_and_is_rejected_where_unsupported():
    wd = require_gpu()
    dims = (4, 4, 4, 4)
    U, eta = fields(dims)
    op = wd.WilsonDirac(dims, 0.12, BC, wd.WD_PREC_F64)
    op.load_gauge(to_dev(U))
    op.set_option(wd.WD_OPT_CG_FORM, 1)
    x1, it1, _, st1 = op.solve(to_dev(eta), tol=1e-5)
    x2, it2, r2, st2 = op.solve(to_dev(eta), x0=x1, tol=1e-10)
    x3, it3, _, st3 = op.solve(to_dev(eta), tol=1e-10)
    assert st1 == st2 == st3 == wd.WD_OK
    assert it2 < it3 and ocg.true_residual(U, eta, to_np(x2), 0.12) <= 1e-10
    with pytest.raises(wd.WdError) as e:
        op.solve_multi(to_dev(np.stack([eta, eta])), tol=1e-8)
    assert e.value.status == wd.WD_EINVAL
    with pytest.raises(wd.WdError):
        op.set_option(wd.WD_OPT_CG_FORM, 2)
    op.close()
    mixed = wd.WilsonDirac(dims, 0.12, BC, wd.WD_PREC_MIXED_F32)
    with pytest.raises(wd.WdError) as e:
        mixed.set_option(wd.WD_OPT_CG_FORM, 1)
    assert e.value.status == wd.WD_EINVAL
    mixed.close()


# ---------------------------------------------------------------- persistent (cooperative) CG loop

@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 4, 5), (14, 14, 14, 14)])
@pytest.mark.parametrize("prec", ["f64", "f32c12", "f32"])
def test_persistent_loop_matches_oracle_and_graph(dims, prec):
    wd = require_gpu()
    U, eta = fields(dims)
    p, tol, c12 = {"f64": (wd.WD_PREC_F64, 1e-10, False), "f32c12": (wd.WD_PREC_F32, 1e-6, True),
                   "f32": (wd.WD_PREC_F32, 1e-6, False)}[prec]
    got = {}
    for mode in (1, 2):
        x, iters, res, status, stats, _, _ = _solve(wd, dims, 0.12, p, tol, U=U, eta=eta, c12=c12,
                                                    options={wd.WD_OPT_USE_GRAPH: mode})
        assert status == wd.WD_OK
        assert ocg.true_residual(U, eta, x, 0.12) <= tol * 1.05
        assert abs(res - ocg.true_residual(U, eta, x, 0.12)) < max(1e-12, 0.05 * tol)
        got[mode] = (x, iters)
    # same algorithm, reductions summed in another fixed order: same iterations within one
    assert abs(got[1][1] - got[2][1]) <= 1
    assert rel(got[2][0], got[1][0]) < 1e3 * tol


def test_persistent_loop_edge_cases():
    wd = require_gpu()
    dims = (4, 4, 4, 8)
    U, eta = fields(dims)
    op = wd.WilsonDirac(dims, 0.12, BC, wd.WD_PREC_F64)
    op.load_gauge(to_dev(U))
    op.set_option(wd.WD_OPT_USE_GRAPH, 2)
    x, iters, res, st = op.solve(to_dev(eta), tol=1e-10, maxit=5)       # iteration limit
    assert st == wd.WD_NOT_CONVERGED and iters == 5
    x, iters, res, st = op.solve(to_dev(np.zeros_like(eta)), tol=1e-10)  # zero source
    assert st == wd.WD_OK and iters == 0 and float(torch.abs(x).max()) == 0.0
    x1, _, _, _ = op.solve(to_dev(eta), tol=1e-5)
    x2, it2, r2, st2 = op.solve(to_dev(eta), x0=x1, tol=1e-10)           # initial guess
    assert st2 == wd.WD_OK and ocg.true_residual(U, eta, to_np(x2), 0.12) <= 1e-10
    bad = eta.copy()
    bad[0, 0, 0, 0, 0, 0] = np.nan
    x, iters, res, st = op.solve(to_dev(bad), tol=1e-10)                 # breakdown
    assert st == wd.WD_BREAKDOWN
    x3, it3, r3, st3 = op.solve(to_dev(eta), tol=1e-10)                  # the context still works
    assert st3 == wd.WD_OK and ocg.true_residual(U, eta, to_np(x3), 0.12) <= 1e-10
    with pytest.raises(wd.WdError):
        op.set_option(wd.WD_OPT_USE_GRAPH, 4)
    op.close()
    # contexts the persistent loop does not serve fall back to the graph solver
    for prec, flag in ((wd.WD_PREC_MIXED_F32, 0), (wd.WD_PREC_F64, wd.WD_EVEN_ODD)):
        op = wd.WilsonDirac(dims, 0.12, BC, prec | flag)
        op.load_gauge(to_dev(U), compress12=prec != wd.WD_PREC_F64)
        op.set_option(wd.WD_OPT_USE_GRAPH, 2)
        x, iters, res, st = op.solve(to_dev(eta), tol=1e-10)
        assert st == wd.WD_OK and ocg.true_residual(U, eta, to_np(x), 0.12) <= 1e-10
        op.close()


@pytest.mark.parametrize("prec", ["mixed32", "mixed16"])
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 4, 5), (14, 14, 14, 14)])
def test_persistent_mixed_loop_matches_oracle_and_graph(prec, dims):
    wd = require_gpu()
    U, eta = fields(dims)
    p = wd.WD_PREC_MIXED_F32 if prec == "mixed32" else wd.WD_PREC_MIXED_F16
    got = {}
    for mode in (1, 2):
        x, iters, res, status, stats, _, _ = _solve(wd, dims, 0.12, p, 1e-10, U=U, eta=eta, c12=True,
                                                    options={wd.WD_OPT_USE_GRAPH: mode})
        assert status == wd.WD_OK
        assert ocg.true_residual(U, eta, x, 0.12) <= 1e-10
        assert abs(res - ocg.true_residual(U, eta, x, 0.12)) < 1e-12
        assert stats["reliable_updates"] >= 1
        got[mode] = (x, iters, stats)
    assert got[2][2]["loop_mode"] == 2 and got[1][2]["loop_mode"] == 1
    assert abs(got[1][1] - got[2][1]) <= 1
    assert rel(got[2][0], got[1][0]) < 1e-7


def test_persistent_mixed_loop_edge_cases():
    wd = require_gpu()
    dims = (4, 4, 4, 8)
    U, eta = fields(dims)
    op = wd.WilsonDirac(dims, 0.12, BC, wd.WD_PREC_MIXED_F16)
    op.load_gauge(to_dev(U), compress12=True)
    op.set_option(wd.WD_OPT_USE_GRAPH, 2)
    x, iters, res, st = op.solve(to_dev(eta), tol=1e-10, maxit=7)       # iteration limit
    assert st == wd.WD_NOT_CONVERGED and iters == 7
    x, iters, res, st = op.solve(to_dev(np.zeros_like(eta)), tol=1e-10)  # zero source
    assert st == wd.WD_OK and iters == 0
    bad = eta.copy()
    bad[1, 0, 0, 0, 2, 1] = np.inf
    x, iters, res, st = op.solve(to_dev(bad), tol=1e-10)                 # breakdown
    assert st == wd.WD_BREAKDOWN
    x, iters, res, st = op.solve(to_dev(eta), tol=1e-10)                 # the context still works
    assert st == wd.WD_OK and ocg.true_residual(U, eta, to_np(x), 0.12) <= 1e-10
    op.set_option(wd.WD_OPT_DF_UPDATES, 0)                               # FP64 reliable updates
    op.load_gauge(to_dev(U), compress12=True)
    x, iters, res, st = op.solve(to_dev(eta), tol=1e-10)
    assert st == wd.WD_OK and ocg.true_residual(U, eta, to_np(x), 0.12) <= 1e-10
    op.close()


@pytest.mark.parametrize("prec", ["f64", "mixed16"])
def test_persistent_loop_wait_limit_reports_and_recovers(prec):
    """Failure detection without a GPU fault: with a grid-barrier wait limit of a single poll the
    persistent loop's waits run out, the kernel stops and cg_solve reports WD_ECUDA; with the
    limit restored the same context solves again."""
    wd = require_gpu()
    dims = (8, 8, 8, 8)
    U, eta = fields(dims)
    p = wd.WD_PREC_F64 if prec == "f64" else wd.WD_PREC_MIXED_F16
    op = wd.WilsonDirac(dims, 0.12, BC, p)
    op.load_gauge(to_dev(U), compress12=prec != "f64")
    op.set_option(wd.WD_OPT_USE_GRAPH, 2)
    op.set_option(wd.WD_OPT_LOOP_WAIT_LIMIT, 1)
    with pytest.raises(wd.WdError) as e:
        op.solve(to_dev(eta), tol=1e-10)
    assert e.value.status == wd.WD_ECUDA
    assert "barrier" in wd.wd_last_error()
    op.set_option(wd.WD_OPT_LOOP_WAIT_LIMIT, 0)          # back to the default limit
    x, iters, res, st = op.solve(to_dev(eta), tol=1e-10)
    assert st == wd.WD_OK and ocg.true_residual(U, eta, to_np(x), 0.12) <= 1e-10
    with pytest.raises(wd.WdError):
        op.set_option(wd.WD_OPT_LOOP_WAIT_LIMIT, -1)
    op.close()


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_residual_history_matches_the_oracle(mode):
    """The recursive residual after every iteration, for the host loop, the graph and the
    persistent loop, against the oracle's CGLS history (entry k + 1 there: it starts with the
    initial residual)."""
    wd = require_gpu()
    dims = (4, 4, 4, 6)
    U, eta = fields(dims)
    op = wd.WilsonDirac(dims, 0.12, BC, wd.WD_PREC_F64)
    op.load_gauge(to_dev(U))
    op.set_option(wd.WD_OPT_USE_GRAPH, mode)
    op.set_option(wd.WD_OPT_RESIDUAL_HISTORY, 500)
    x, iters, res, st = op.solve(to_dev(eta), tol=1e-10)
    assert st == wd.WD_OK
    h = np.array(op.residual_history())
    assert len(h) == iters and h[-1] <= 1e-10 < h[-2]
    assert np.all(h[1:] <= h[:-1] * (1 + 1e-9))           # CGLS: ||eta - D x_k|| does not grow
    _, io, _, ho = ocg.cgls(U, eta, 0.12, 1e-10, 2000)
    n = min(len(h), len(ho) - 1)
    assert abs(len(h) - io) <= 1
    assert np.max(np.abs(h[:20] / ho[1:21] - 1)) < 1e-9     # rounding-order differences only
    assert np.max(np.abs(h[:n] / ho[1:n + 1] - 1)) < 1e-3
    op.set_option(wd.WD_OPT_RESIDUAL_HISTORY, 10)           # shorter history: the first entries
    x, iters, res, st = op.solve(to_dev(eta), tol=1e-10)
    h10 = np.array(op.residual_history())
    assert len(h10) == 10 and np.allclose(h10, h[:10], rtol=1e-12)
    op.close()


def test_residual_history_mixed_and_off():
    wd = require_gpu()
    dims = (6, 4, 4, 8)
    U, eta = fields(dims)
    op = wd.WilsonDirac(dims, 0.12, BC, wd.WD_PREC_MIXED_F16)
    op.load_gauge(to_dev(U), compress12=True)
    assert op.residual_history() == []                      # no solve yet, history off
    op.set_option(wd.WD_OPT_RESIDUAL_HISTORY, 1000)
    x, iters, res, st = op.solve(to_dev(eta), tol=1e-10)
    h = op.residual_history()
    assert st == wd.WD_OK and len(h) == iters and h[-1] <= 1e-9 and res <= 1e-10
    op.set_option(wd.WD_OPT_RESIDUAL_HISTORY, 0)
    op.solve(to_dev(eta), tol=1e-10)
    assert op.residual_history() == []
    with pytest.raises(wd.WdError):
        op.set_option(wd.WD_OPT_RESIDUAL_HISTORY, -2)
    op.close()
