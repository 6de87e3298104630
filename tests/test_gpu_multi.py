"""Multi right-hand-side dslash and CG through the C ABI, against the FP64 CPU oracle."""
import numpy as np
import pytest
import torch

import synthetic
from oracle import cg as ocg
from oracle import wilson
from tests.gpu_util import rel, require_gpu, to_dev, to_np

pytestmark = pytest.mark.gpu

BC = (1, 1, 1, -1)


def _sources(dims, n, seed0=10):
    return np.stack([synthetic.gaussian_source(dims, seed0 + i) for i in range(n)])


def _point_sources(dims):
    return np.stack([synthetic.point_source(dims, s, c) for s in range(4) for c in range(3)])


@pytest.mark.parametrize("dims,n", [((4, 4, 4, 4), 1), ((6, 4, 4, 8), 3), ((2, 3, 4, 5), 12), ((8, 8, 8, 8), 5)])
@pytest.mark.parametrize("dagger", [False, True])
def test_apply_multi_fp64_matches_oracle(dims, n, dagger):
    wd = require_gpu()
    U = synthetic.gauge_field(dims, 0.4, 1)
    psi = _sources(dims, n)
    op = wd.WilsonDirac(dims, 0.12, BC, wd.WD_PREC_F64)
    op.load_gauge(to_dev(U))
    out = to_np(op.apply_multi(to_dev(psi), dagger=dagger))
    for r in range(n):
        assert rel(out[r], wilson.apply_D(U, psi[r], 0.12, BC, dagger)) < 1e-13
    op.close()


def test_apply_multi_fp32_matches_oracle():
    wd = require_gpu()
    dims = (6, 4, 4, 8)
    U = synthetic.gauge_field(dims, 0.4, 1)
    psi = _sources(dims, 4)
    op = wd.WilsonDirac(dims, 0.12, BC, wd.WD_PREC_F32)
    op.load_gauge(to_dev(U), compress12=True)
    out = to_np(op.apply_multi(to_dev(psi)))
    for r in range(4):
        ref = wilson.apply_D(U, psi[r].astype(np.complex64).astype(np.complex128), 0.12, BC)
        assert rel(out[r], ref) < 1e-6
    op.close()


def test_every_group_shape_gives_the_same_bits():
    wd = require_gpu()
    dims = (4, 4, 4, 6)
    n = 12
    U = synthetic.gauge_field(dims, 0.4, 1)
    psi = to_dev(_sources(dims, n))
    op = wd.WilsonDirac(dims, 0.12, BC, wd.WD_PREC_F64)
    op.load_gauge(to_dev(U))
    ref = None
    for K in (1, 2, 3, 4, 6, 12):
        op.set_option(wd.WD_OPT_MULTI_GROUP, K)
        out = op.apply_multi(psi)
        assert op.multi_stats()["group"] == K
        if ref is None:
            ref = out.clone()
        assert torch.equal(out, ref), K
    op.close()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_solve_multi_plain(prec):
    wd = require_gpu()
    dims = (4, 4, 4, 4)
    U = synthetic.gauge_field(dims, 0.4, 1)
    eta = _sources(dims, 3)
    p, tol = (wd.WD_PREC_F64, 1e-10) if prec == "f64" else (wd.WD_PREC_F32, 1e-6)
    op = wd.WilsonDirac(dims, 0.12, BC, p)
    op.load_gauge(to_dev(U), compress12=(prec == "f32"))
    x, iters, res, status = op.solve_multi(to_dev(eta), tol=tol)
    assert status == wd.WD_OK
    x = to_np(x)
    for r in range(3):
        assert ocg.true_residual(U, eta[r], x[r], 0.12) <= tol * 1.05
        assert abs(res[r] - ocg.true_residual(U, eta[r], x[r], 0.12)) < max(1e-12, 0.05 * tol)
        xs, its, _, _ = ocg.cgls(U, eta[r], 0.12, tol, 2000)
        assert abs(iters[r] - its) <= 2
    op.close()


@pytest.mark.parametrize("prec", ["mixed32", "mixed16"])
def test_solve_multi_mixed_point_sources(prec):
    wd = require_gpu()
    dims = (8, 8, 8, 8)
    U = synthetic.gauge_field(dims, 0.4, 1)
    eta = _point_sources(dims)
    p = wd.WD_PREC_MIXED_F32 if prec == "mixed32" else wd.WD_PREC_MIXED_F16
    op = wd.WilsonDirac(dims, 0.12, BC, p)
    op.load_gauge(to_dev(U), compress12=True)
    x, iters, res, status = op.solve_multi(to_dev(eta), tol=1e-10, maxit=4000)
    st = op.multi_stats()
    assert status == wd.WD_OK, st
    x = to_np(x)
    for r in range(12):
        assert ocg.true_residual(U, eta[r], x[r], 0.12) <= 1e-10
    assert st["reliable_updates"] >= 1 and st["group"] >= 1
    op.close()


def test_solve_multi_independent_rhs():
    wd = require_gpu()
    dims = (4, 4, 4, 4)
    U = synthetic.gauge_field(dims, 0.4, 1)
    eta = _sources(dims, 4)
    eta[1] = 0.0                       # zero source: converged before the first iteration
    op = wd.WilsonDirac(dims, 0.12, BC, wd.WD_PREC_MIXED_F32)
    op.load_gauge(to_dev(U), compress12=True)
    x, iters, res, status = op.solve_multi(to_dev(eta), tol=1e-10)
    assert status == wd.WD_OK
    assert iters[1] == 0 and float(np.abs(to_np(x)[1]).max()) == 0.0
    for r in (0, 2, 3):
        assert iters[r] > 10 and res[r] <= 1e-10
    # a NaN source breaks down alone; the others still converge
    eta[2, 0, 0, 0, 0, 0, 0] = np.nan
    x, iters, res, status = op.solve_multi(to_dev(eta), tol=1e-10)
    assert status == wd.WD_BREAKDOWN
    x = to_np(x)
    for r in (0, 3):
        assert ocg.true_residual(U, eta[r], x[r], 0.12) <= 1e-10
    op.close()


def test_solve_multi_matches_single_within_tolerance():
    wd = require_gpu()
    dims = (6, 4, 4, 8)
    U = synthetic.gauge_field(dims, 0.4, 1)
    eta = _sources(dims, 4)
    op = wd.WilsonDirac(dims, 0.124, BC, wd.WD_PREC_MIXED_F32)
    op.load_gauge(to_dev(U), compress12=True)
    xb, _, resb, st = op.solve_multi(to_dev(eta), tol=1e-10)
    assert st == wd.WD_OK
    xb = to_np(xb)
    for r in range(4):
        xs, _, ress, sts = op.solve(to_dev(eta[r]), tol=1e-10)
        assert sts == wd.WD_OK
        # both solutions solve the system to 1e-10; they agree to the conditioning of D
        assert rel(xb[r], to_np(xs)) < 1e-8
    op.close()


def test_graph_and_host_loop_agree_multi():
    wd = require_gpu()
    dims = (4, 4, 4, 6)
    U = synthetic.gauge_field(dims, 0.4, 1)
    eta = to_dev(_sources(dims, 3))
    outs = []
    for graph in (1, 0):
        op = wd.WilsonDirac(dims, 0.12, BC, wd.WD_PREC_MIXED_F32)
        op.load_gauge(to_dev(U), compress12=True)
        op.set_option(wd.WD_OPT_MULTI_GROUP, 3)
        op.set_option(wd.WD_OPT_MULTI_SITES, 32)
        op.set_option(wd.WD_OPT_USE_GRAPH, graph)
        x, iters, res, st = op.solve_multi(eta, tol=1e-10)
        assert st == wd.WD_OK
        outs.append((x, iters))
        op.close()
    assert outs[0][1] == outs[1][1]
    assert torch.equal(outs[0][0], outs[1][0])


def test_solve_multi_mixed_with_fp64_updates():
    wd = require_gpu()
    dims = (6, 4, 4, 8)
    U = synthetic.gauge_field(dims, 0.4, 1)
    eta = _sources(dims, 3)
    for df in (0, 1):
        op = wd.WilsonDirac(dims, 0.124, BC, wd.WD_PREC_MIXED_F16)
        op.set_option(wd.WD_OPT_DF_UPDATES, df)
        op.load_gauge(to_dev(U), compress12=True)
        x, iters, res, status = op.solve_multi(to_dev(eta), tol=1e-10)
        assert status == wd.WD_OK
        x = to_np(x)
        for r in range(3):
            assert ocg.true_residual(U, eta[r], x[r], 0.124) <= 1e-10
        op.close()


# ---------------------------------------------------------------- several right-hand sides per thread

@pytest.mark.parametrize("prec", ["f32", "f32c12", "f16_inner"])
@pytest.mark.parametrize("kt", [2, 4])
def test_rhs_per_thread_matches_one_per_thread_and_the_oracle(prec, kt):
    """KT right-hand sides per thread share each link load; the arithmetic per right-hand side is
    that of one per thread, so the outputs agree bit for bit, and with the oracle within the
    working-precision bound."""
    wd = require_gpu()
    dims = (6, 5, 4, 8)
    n = 12
    U = synthetic.gauge_field(dims, 0.4, 1)
    psi = _sources(dims, n)
    p, c12 = {"f32": (wd.WD_PREC_F32, False), "f32c12": (wd.WD_PREC_F32, True),
              "f16_inner": (wd.WD_PREC_MIXED_F16, True)}[prec]
    op = wd.WilsonDirac(dims, 0.12, BC, p)
    op.load_gauge(to_dev(U), compress12=c12)
    if p == wd.WD_PREC_MIXED_F16:
        op.set_option(wd.WD_OPT_APPLY_INNER, 1)
    out = {}
    for k in (1, kt):
        op.set_option(wd.WD_OPT_MULTI_RHS_PER_THREAD, k)
        op.set_option(wd.WD_OPT_MULTI_GROUP, 12)
        op.set_option(wd.WD_OPT_MULTI_SITES, 8)
        for dagger in (False, True):
            out[(k, dagger)] = to_np(op.apply_multi(to_dev(psi), dagger=dagger))
        assert op.multi_stats()["rhs_per_thread"] == k
    op.close()
    for dagger in (False, True):
        assert np.array_equal(out[(1, dagger)], out[(kt, dagger)]), dagger
        for r in range(n):
            ref = wilson.apply_D(U, psi[r].astype(np.complex64).astype(np.complex128), 0.12, BC, dagger)
            bound = 1e-6 if prec != "f16_inner" else 2.0 ** -9
            assert rel(out[(kt, dagger)][r], ref) < bound, (r, dagger)


@pytest.mark.parametrize("kt", [2, 4])
@pytest.mark.parametrize("prec", ["mixed_f32", "mixed_f16", "f32"])
def test_multi_solve_with_rhs_per_thread(kt, prec):
    wd = require_gpu()
    dims = (6, 4, 4, 8)
    n = 8
    U = synthetic.gauge_field(dims, 0.4, 1)
    eta = _sources(dims, n, seed0=40)
    p, tol = {"mixed_f32": (wd.WD_PREC_MIXED_F32, 1e-10), "mixed_f16": (wd.WD_PREC_MIXED_F16, 1e-10),
              "f32": (wd.WD_PREC_F32, 1e-6)}[prec]
    op = wd.WilsonDirac(dims, 0.12, BC, p)
    op.load_gauge(to_dev(U), compress12=True)
    op.set_option(wd.WD_OPT_MULTI_RHS_PER_THREAD, kt)
    x, iters, res, st = op.solve_multi(to_dev(eta), tol=tol, maxit=4000)
    s = op.multi_stats()
    op.close()
    assert st == wd.WD_OK and s["rhs_per_thread"] == kt
    xs = to_np(x)
    for r in range(n):
        true = ocg.true_residual(U, eta[r], xs[r], 0.12)
        assert true <= tol * 1.05, (r, true)
        assert abs(res[r] - true) <= max(1e-12, 0.05 * tol)


def test_rhs_per_thread_option_checks():
    wd = require_gpu()
    dims = (4, 4, 4, 4)
    op = wd.WilsonDirac(dims, 0.12, BC, wd.WD_PREC_MIXED_F32)
    for bad in (3, 5, -1, 8):
        with pytest.raises(wd.WdError) as e:
            op.set_option(wd.WD_OPT_MULTI_RHS_PER_THREAD, bad)
        assert e.value.status == wd.WD_EINVAL
    op.close()
