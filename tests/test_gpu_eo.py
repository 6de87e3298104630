"""Even-odd (Schur) preconditioned contexts against the FP64 CPU oracle of the full operator."""
import numpy as np
import pytest
import torch

import synthetic
from oracle import cg as ocg
from oracle import wilson
from tests.gpu_util import fields, rel, require_gpu, to_dev, to_np

pytestmark = pytest.mark.gpu

BC = (1, 1, 1, -1)


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4), (6, 4, 2, 8), (8, 8, 8, 8)])
@pytest.mark.parametrize("dagger", [False, True])
def test_eo_context_applies_the_full_operator(dims, dagger):
    wd = require_gpu()
    U, psi = fields(dims)
    op = wd.WilsonDirac(dims, 0.12, BC, wd.WD_PREC_F64 | wd.WD_EVEN_ODD)
    op.load_gauge(to_dev(U))
    out = to_np(op.apply(to_dev(psi), dagger=dagger))
    assert rel(out, wilson.apply_D(U, psi, 0.12, BC, dagger)) < 1e-13
    op.close()


@pytest.mark.parametrize("bc", [(-1, 1, -1, 1), (-1, -1, -1, -1), (1, -1, 1, 1)])
def test_eo_fp64_boundaries(bc):
    """Antiperiodic directions of extent 2 and 6: one of the two hops of a direction wraps."""
    wd = require_gpu()
    dims = (4, 2, 2, 6)
    U, psi = fields(dims)
    op = wd.WilsonDirac(dims, 0.137, bc, wd.WD_PREC_F64 | wd.WD_EVEN_ODD)
    op.load_gauge(to_dev(U))
    for dagger in (False, True):
        out = to_np(op.apply(to_dev(psi), dagger=dagger))
        assert rel(out, wilson.apply_D(U, psi, 0.137, bc, dagger)) < 1e-13
    op.close()


def test_eo_fp32_apply_and_generated_links():
    wd = require_gpu()
    dims = (4, 6, 4, 4)
    op = wd.WilsonDirac(dims, 0.12, BC, wd.WD_PREC_F32 | wd.WD_EVEN_ODD)
    op.generate_gauge(0.4, 5, compress12=True)
    U = synthetic.gauge_field_philox(dims, 0.4, 5)
    psi = synthetic.gaussian_source(dims, 2)
    out = to_np(op.apply(to_dev(psi, torch.complex64)))
    ref = wilson.apply_D(U, psi.astype(np.complex64).astype(np.complex128), 0.12, BC)
    assert rel(out, ref) < 1e-6
    op.close()


@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("f32", 1e-6), ("mixed32", 1e-10), ("mixed16", 1e-10)])
def test_eo_solves_reach_tolerance_in_fewer_iterations(prec, tol):
    wd = require_gpu()
    dims = (8, 8, 8, 8)
    U, eta = fields(dims)
    base = {"f64": wd.WD_PREC_F64, "f32": wd.WD_PREC_F32, "mixed32": wd.WD_PREC_MIXED_F32,
            "mixed16": wd.WD_PREC_MIXED_F16}[prec]
    c12 = prec != "f64"
    res = {}
    for flag in (0, wd.WD_EVEN_ODD):
        op = wd.WilsonDirac(dims, 0.124, BC, base | flag)
        op.load_gauge(to_dev(U), compress12=c12)
        x, iters, r, st = op.solve(to_dev(eta), tol=tol, maxit=5000)
        assert st == wd.WD_OK
        xs = to_np(x)
        assert ocg.true_residual(U, eta, xs, 0.124) <= tol * 1.05
        assert abs(r - ocg.true_residual(U, eta, xs, 0.124)) < max(1e-12, 0.05 * tol)
        res[flag] = (iters, xs)
        op.close()
    assert res[wd.WD_EVEN_ODD][0] < 0.75 * res[0][0]
    assert rel(res[wd.WD_EVEN_ODD][1], res[0][1]) < 1e4 * tol


def test_eo_rejects_odd_extents_and_multi_rhs():
    wd = require_gpu()
    with pytest.raises(wd.WdError) as e:
        wd.WilsonDirac((4, 4, 3, 4), 0.12, BC, wd.WD_PREC_F64 | wd.WD_EVEN_ODD)
    assert e.value.status == wd.WD_EINVAL
    dims = (4, 4, 4, 4)
    U, eta = fields(dims)
    op = wd.WilsonDirac(dims, 0.12, BC, wd.WD_PREC_F64 | wd.WD_EVEN_ODD)
    op.load_gauge(to_dev(U))
    with pytest.raises(wd.WdError) as e:
        op.apply_multi(to_dev(np.stack([eta, eta])))
    assert e.value.status == wd.WD_EINVAL
    op.close()


def test_eo_restart_keeps_the_schur_source():
    wd = require_gpu()
    dims = (4, 4, 4, 8)
    U, eta = fields(dims)
    op = wd.WilsonDirac(dims, 0.12, BC, wd.WD_PREC_F64 | wd.WD_EVEN_ODD)
    op.load_gauge(to_dev(U))
    x1, it1, r1, st1 = op.solve(to_dev(eta), tol=1e-6)
    x2, it2, r2, st2 = op.solve(to_dev(eta), x0=x1, tol=1e-11)   # restart from a previous solution
    assert st1 == st2 == wd.WD_OK
    assert ocg.true_residual(U, eta, to_np(x2), 0.12) <= 1e-11
    op.close()


@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("f32", 1e-6)])
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 8), (14, 14, 14, 14)])
def test_eo_persistent_loop_matches_graph_and_oracle(prec, tol, dims):
    wd = require_gpu()
    U, eta = fields(dims)
    base = wd.WD_PREC_F64 if prec == "f64" else wd.WD_PREC_F32
    got = {}
    for mode in (1, 2):
        op = wd.WilsonDirac(dims, 0.124, BC, base | wd.WD_EVEN_ODD)
        op.load_gauge(to_dev(U), compress12=prec != "f64")
        op.set_option(wd.WD_OPT_USE_GRAPH, mode)
        x, iters, r, st = op.solve(to_dev(eta), tol=tol, maxit=5000)
        assert st == wd.WD_OK
        xs = to_np(x)
        assert ocg.true_residual(U, eta, xs, 0.124) <= tol * 1.05
        assert abs(r - ocg.true_residual(U, eta, xs, 0.124)) < max(1e-12, 0.05 * tol)
        assert op.stats()["loop_mode"] == mode
        got[mode] = (iters, xs)
        op.close()
    assert abs(got[1][0] - got[2][0]) <= 1
    assert rel(got[2][1], got[1][1]) < 1e3 * tol
