"""The FP32 / FP16 dslash under its other load schedules (WD_OPT_DSLASH_SCHEDULE 2 and 3).

Schedule 2: each thread takes two sites of a grid-stride step and issues both sites' loads of a
hop before either site's arithmetic. Schedule 3: one site per thread, both hops of each direction
loaded before their arithmetic. The per-site arithmetic and its order are those of the hop-by-hop
kernel (schedule 1), so the operator's output must be the same bits. Checked on ragged volumes,
both boundaries' phases, every block size, both daggers, 18- and 12-real links, the FP16 inner
operator, against the oracle's Eq. (1) at the FP32 tolerance, and through the solvers that launch
it (graph and host loop): the same iterations to one, and the oracle's true residual.
"""
import numpy as np
import pytest
import torch

from oracle import cg as ocg
from oracle import wilson
from tests.gpu_util import fields, rel, require_gpu, to_dev, to_np

pytestmark = pytest.mark.gpu

BC = (1, 1, 1, -1)
SIZES = [(2, 2, 2, 2), (3, 5, 7, 2), (8, 6, 4, 10), (16, 8, 8, 9)]


def _op(wd, dims, prec, c12, U, sched, kappa=0.12, bc=BC):
    op = wd.WilsonDirac(dims, kappa, bc, prec)
    op.load_gauge(to_dev(U), compress12=c12)
    if prec != wd.WD_PREC_F32:
        op.set_option(wd.WD_OPT_APPLY_INNER, 1)
    op.set_option(wd.WD_OPT_DSLASH_SCHEDULE, sched)
    return op


@pytest.mark.parametrize("dims", SIZES)
@pytest.mark.parametrize("prec,c12", [("f32", False), ("f32", True), ("f16", True)])
def test_schedules_same_bits_and_oracle(dims, prec, c12):
    wd = require_gpu()
    p = wd.WD_PREC_F32 if prec == "f32" else wd.WD_PREC_MIXED_F16
    U, psi = fields(dims)
    x = to_dev(psi, torch.complex64) if prec == "f32" else to_dev(psi)
    outs = {}
    for sched in (1, 2, 3):
        op = _op(wd, dims, p, c12, U, sched)
        for block in (32, 64, 128, 256):
            op.set_option(wd.WD_OPT_BLOCK_DSLASH, block)
            for dagger in (False, True):
                outs[(sched, block, dagger)] = to_np(op.apply(x, dagger=dagger))
        op.close()
    for sched in (2, 3):
        for block in (32, 64, 128, 256):
            for dagger in (False, True):
                assert np.array_equal(outs[(1, block, dagger)], outs[(sched, block, dagger)]), (sched, block, dagger)
    if prec == "f32":
        xin = psi.astype(np.complex64).astype(np.complex128)
        for dagger in (False, True):
            ref = wilson.apply_D(U, xin, 0.12, BC, dagger)
            assert rel(outs[(2, 256, dagger)], ref) < 1e-6 and rel(outs[(3, 64, dagger)], ref) < 1e-6


@pytest.mark.parametrize("bc", [(-1, 1, -1, 1), (1, 1, 1, 1)])
@pytest.mark.parametrize("sched", [2, 3])
def test_schedules_boundaries(bc, sched):
    wd = require_gpu()
    dims = (4, 2, 3, 6)
    U, psi = fields(dims)
    op = _op(wd, dims, wd.WD_PREC_F32, True, U, sched, kappa=0.137, bc=bc)
    xin = psi.astype(np.complex64).astype(np.complex128)
    for dagger in (False, True):
        out = to_np(op.apply(to_dev(psi, torch.complex64), dagger=dagger))
        assert rel(out, wilson.apply_D(U, xin, 0.137, bc, dagger)) < 1e-6
    op.close()


@pytest.mark.parametrize("prec", ["f32", "mixed_f16"])
@pytest.mark.parametrize("mode", [0, 1])
def test_schedules_in_the_solvers(prec, mode):
    """The graph (1) and host-loop (0) solvers launch the stand-alone dslash: under schedules 2 and
    3 they take the same iterations (to one: the fused norm may sum its sites in another order)
    and meet the oracle's true residual."""
    wd = require_gpu()
    dims = (8, 6, 4, 10)
    U, eta = fields(dims)
    p = wd.WD_PREC_F32 if prec == "f32" else wd.WD_PREC_MIXED_F16
    tol = 1e-6 if prec == "f32" else 1e-10
    res = {}
    for sched in (1, 2, 3):
        op = wd.WilsonDirac(dims, 0.12, BC, p)
        op.load_gauge(to_dev(U), compress12=True)
        op.set_option(wd.WD_OPT_DSLASH_SCHEDULE, sched)
        op.set_option(wd.WD_OPT_USE_GRAPH, mode)
        x, iters, r, st = op.solve(to_dev(eta), tol=tol, maxit=4000)   # complex128 for every precision
        op.close()
        assert st == wd.WD_OK
        res[sched] = (to_np(x), iters)
    for sched in (2, 3):
        assert abs(res[1][1] - res[sched][1]) <= 1   # the fused norms may sum the sites in another order
        assert ocg.true_residual(U, eta, res[sched][0], 0.12) <= tol * 1.01


def test_schedule_option_checks():
    wd = require_gpu()
    dims = (4, 4, 4, 4)
    U, _ = fields(dims)
    op = wd.WilsonDirac(dims, 0.12, BC, wd.WD_PREC_F64)
    op.load_gauge(to_dev(U))
    op.set_option(wd.WD_OPT_DSLASH_SCHEDULE, 1)
    for bad in (2, 3, 4, -1):
        with pytest.raises(wd.WdError):
            op.set_option(wd.WD_OPT_DSLASH_SCHEDULE, bad)
    op.close()
    op = wd.WilsonDirac(dims, 0.12, BC, wd.WD_PREC_F32 | wd.WD_EVEN_ODD)
    op.load_gauge(to_dev(U))
    for bad in (2, 3):
        with pytest.raises(wd.WdError):
            op.set_option(wd.WD_OPT_DSLASH_SCHEDULE, bad)
    op.close()
