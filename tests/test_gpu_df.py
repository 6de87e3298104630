"""Double-float (FP32-pair) operator and reliable updates against the FP64 oracle."""
import numpy as np
import pytest
import torch

from oracle import cg as ocg
from oracle import wilson
from tests.gpu_util import fields, rel, require_gpu, to_dev, to_np

pytestmark = pytest.mark.gpu

BC = (1, 1, 1, -1)


@pytest.mark.parametrize("dims,eo", [((4, 4, 4, 4), 0), ((2, 3, 4, 5), 0), ((8, 8, 8, 8), 0), ((6, 4, 4, 8), 1)])
@pytest.mark.parametrize("dagger", [False, True])
def test_double_float_operator_meets_the_fp64_tolerance(dims, eo, dagger):
    wd = require_gpu()
    U, psi = fields(dims)
    flag = wd.WD_EVEN_ODD if eo else 0
    op = wd.WilsonDirac(dims, 0.12, BC, wd.WD_PREC_MIXED_F32 | flag)
    op.load_gauge(to_dev(U), compress12=True)
    op.set_option(wd.WD_OPT_APPLY_DF, 1)
    out = to_np(op.apply(to_dev(psi), dagger=dagger))
    assert rel(out, wilson.apply_D(U, psi, 0.12, BC, dagger)) < 1e-13
    op.close()


@pytest.mark.parametrize("prec", ["mixed32", "mixed16"])
@pytest.mark.parametrize("eo", [0, 1])
def test_double_float_and_fp64_updates_agree(prec, eo):
    wd = require_gpu()
    dims = (8, 8, 8, 8)
    U, eta = fields(dims)
    base = wd.WD_PREC_MIXED_F32 if prec == "mixed32" else wd.WD_PREC_MIXED_F16
    res = {}
    for df in (1, 0):
        op = wd.WilsonDirac(dims, 0.124, BC, base | (wd.WD_EVEN_ODD if eo else 0))
        op.set_option(wd.WD_OPT_DF_UPDATES, df)
        op.load_gauge(to_dev(U), compress12=True)
        x, iters, r, st = op.solve(to_dev(eta), tol=1e-10)
        assert st == wd.WD_OK
        xs = to_np(x)
        assert ocg.true_residual(U, eta, xs, 0.124) <= 1e-10
        res[df] = (iters, xs, op.stats()["reliable_updates"])
        op.close()
    assert abs(res[1][0] - res[0][0]) <= 3
    assert rel(res[1][1], res[0][1]) < 1e-8
