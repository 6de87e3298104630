"""Checkpoint and resume of a CG solve (wd_cg_save_state / cg_resume).

A solve stopped at maxit leaves x, r, p, gamma and the iteration count of the CG iteration (Sec. 2)
in the context; saved to host memory and resumed, it must reach what the uninterrupted solve
reaches: bit for bit on the same launch shape (the four-phase persistent loop, the loop with 8
lanes per site, the graph, FP32, even-odd, the paper's CG form, a fresh context), to rounding in
the FP64 loop's time-diagonal basis. Every result meets the tolerance by the oracle's residual.
"""
import numpy as np
import pytest
import torch

from oracle import cg as ocg
from tests.gpu_util import fields, rel, require_gpu, to_dev, to_np

pytestmark = pytest.mark.gpu

DIMS = (6, 4, 4, 8)
BC = (1, 1, 1, -1)
KAPPA = 0.12


def _case(wd, name):
    """(precision, options, tolerance, bitwise) of a named configuration."""
    return {
        "f64_one_thread_chiral": (wd.WD_PREC_F64, {wd.WD_OPT_DSLASH_VARIANT: 1, wd.WD_OPT_LOOP_TIME_BASIS: 0}, 1e-10, True),
        "f64_eight_lanes": (wd.WD_PREC_F64, {wd.WD_OPT_DSLASH_VARIANT: 4}, 1e-10, True),
        "f64_graph": (wd.WD_PREC_F64, {wd.WD_OPT_USE_GRAPH: 1}, 1e-10, True),
        "f64_host_loop": (wd.WD_PREC_F64, {wd.WD_OPT_USE_GRAPH: 0}, 1e-10, True),
        "f64_even_odd": (wd.WD_PREC_F64 | wd.WD_EVEN_ODD, {}, 1e-10, True),
        "f32": (wd.WD_PREC_F32, {}, 1e-6, True),
        "f64_time_basis": (wd.WD_PREC_F64, {wd.WD_OPT_DSLASH_VARIANT: 1, wd.WD_OPT_LOOP_TIME_BASIS: 1}, 1e-10, False),
        "f64_paper_form": (wd.WD_PREC_F64, {wd.WD_OPT_CG_FORM: 1, wd.WD_OPT_LOOP_TIME_BASIS: 0}, 1e-10, True),
    }[name]


def _make(wd, U, prec, opts):
    op = wd.WilsonDirac(DIMS, KAPPA, BC, prec)
    op.load_gauge(to_dev(U))
    for k, v in opts.items():
        op.set_option(k, v)
    return op


@pytest.mark.parametrize("name", ["f64_one_thread_chiral", "f64_eight_lanes", "f64_graph", "f64_host_loop",
                                  "f64_even_odd", "f32", "f64_time_basis", "f64_paper_form"])
def test_resumed_solve_equals_the_uninterrupted_one(name):
    wd = require_gpu()
    prec, opts, tol, bitwise = _case(wd, name)
    U, eta = fields(DIMS, gseed=31, sseed=32)
    src = to_dev(eta)
    op = _make(wd, U, prec, opts)
    x_full, it_full, res_full, st_full = op.solve(src, tol=tol, maxit=4000)
    assert st_full == wd.WD_OK and it_full >= 12
    # stop after a third of the iterations, save, resume to two thirds (stops again), save, resume
    # to the end
    k1, k2 = it_full // 3, (2 * it_full) // 3
    _, it1, _, st1 = op.solve(src, tol=tol, maxit=k1)
    assert st1 == wd.WD_NOT_CONVERGED and it1 == k1
    s1 = op.save_state()
    assert len(s1) == wd.wd_cg_state_size(op.ctx)
    _, it2, _, st2 = op.resume(s1, src, tol=tol, maxit=k2)
    assert st2 == wd.WD_NOT_CONVERGED and it2 == k2
    s2 = op.save_state()
    x_res, it_res, res_res, st_res = op.resume(s2, src, tol=tol, maxit=4000)
    op.close()
    assert st_res == wd.WD_OK
    true = ocg.true_residual(U, eta, to_np(x_res), KAPPA, BC)
    assert true <= tol * (1.05 if prec == wd.WD_PREC_F32 else 1.0 + 1e-6), true
    if bitwise:
        assert it_res == it_full and res_res == res_full
        assert torch.equal(x_res, x_full)
    else:
        assert abs(it_res - it_full) <= 1
        assert rel(to_np(x_res), to_np(x_full)) < 1e-8


def test_state_moves_to_a_fresh_context():
    """A state saved on one context resumes on another of the same lattice, boundary, precision and
    kappa with the same links (the serving case: the first context was freed)."""
    wd = require_gpu()
    prec, opts, tol, _ = _case(wd, "f64_one_thread_chiral")
    U, eta = fields(DIMS, gseed=41, sseed=42)
    src = to_dev(eta)
    a = _make(wd, U, prec, opts)
    x_full, it_full, res_full, _ = a.solve(src, tol=tol, maxit=4000)
    a.solve(src, tol=tol, maxit=12)
    state = a.save_state()
    a.close()
    b = _make(wd, U, prec, opts)
    x_res, it_res, res_res, st = b.resume(state, src, tol=tol, maxit=4000)
    b.close()
    assert st == wd.WD_OK and it_res == it_full and res_res == res_full
    assert torch.equal(x_res, x_full)


def test_save_and_resume_refuse_what_they_cannot_continue():
    wd = require_gpu()
    U, eta = fields(DIMS, gseed=51, sseed=52)
    src = to_dev(eta)
    op = _make(wd, U, wd.WD_PREC_F64, {})
    op.solve(src, tol=1e-10, maxit=4000)  # converged: nothing to continue
    with pytest.raises(wd.WdError) as e:
        op.save_state()
    assert e.value.status == wd.WD_EINVAL
    op.solve(src, tol=1e-10, maxit=7)
    state = op.save_state()
    op.apply(src)  # a later call that uses the context's fields ends the saved state's validity
    with pytest.raises(wd.WdError):
        op.save_state()
    # a corrupted header, another kappa, another lattice
    bad = bytearray(state)
    bad[0] ^= 0xFF
    with pytest.raises(wd.WdError):
        op.resume(bad, src)
    op.set_kappa(0.121)
    with pytest.raises(wd.WdError):
        op.resume(state, src)
    op.close()
    dims2 = (4, 4, 4, 8)
    other = wd.WilsonDirac(dims2, KAPPA, BC, wd.WD_PREC_F64)
    U2, eta2 = fields(dims2, gseed=53, sseed=54)
    other.load_gauge(to_dev(U2))
    with pytest.raises(wd.WdError):
        other.resume(state, to_dev(eta2))
    other.close()
    mixed = wd.WilsonDirac(DIMS, KAPPA, BC, wd.WD_PREC_MIXED_F32)
    with pytest.raises(wd.WdError):
        wd.wd_cg_state_size(mixed.ctx)
    mixed.close()
