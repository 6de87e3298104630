"""The mixed-precision and multi-RHS workloads at their full sizes, in the launch configuration the
benchmark times (device-generated fields, autotuned launch shapes, CUDA-graph solver).

A CPU oracle solve at these sizes would take hours, so parity is checked through properties that
hold at any size: every solve's true residual, recomputed from the returned x with the FP64
operator, is below the tolerance, and that FP64 operator matches the oracle's literal per-site loop
at sampled sites of the same fields (both ends of every extent included).
"""
import numpy as np
import pytest
import torch

from oracle import wilson
from tests.gpu_util import rel, require_gpu

pytestmark = pytest.mark.gpu

BC = (1, 1, 1, -1)


def _sites(dims, n, seed):
    lx, ly, lz, lt = dims
    rng = np.random.default_rng(seed)
    s = [(0, 0, 0, 0), (lx - 1, ly - 1, lz - 1, lt - 1), (lx - 1, 0, lz - 1, 0), (0, ly - 1, 0, lt - 1)]
    return s + [tuple(int(v) for v in rng.integers(0, (lx, ly, lz, lt))) for _ in range(n)]


def _check_operator(U, x, Dx, kappa, dims, seed):
    sites = _sites(dims, 30, seed)
    ref = wilson.apply_D_sites(U, x, kappa, sites, BC)
    got = np.stack([Dx[t, z, y, x_] for (x_, y, z, t) in sites])
    assert rel(got, ref) < 1e-13


def _true_residual(eta, Dx):
    e = eta.reshape(-1)
    return float(np.linalg.norm(e - Dx.reshape(-1)) / np.linalg.norm(e))


@pytest.mark.parametrize("prec", ["mixed32", "mixed16"])
def test_mixed_32x64_full_size(prec):
    wd = require_gpu()
    dims, kappa = (32, 32, 32, 64), 0.124
    p = wd.WD_PREC_MIXED_F32 if prec == "mixed32" else wd.WD_PREC_MIXED_F16
    op = wd.WilsonDirac(dims, kappa, BC, p)
    U = op.generate_gauge(0.4, 1, compress12=True, return_field=True)
    eta = op.generate_source(2)
    x, iters, res, st = op.solve(eta, tol=1e-10, maxit=4000)
    assert st == wd.WD_OK and iters > 50
    Dx = op.apply(x).cpu().numpy()          # the FP64 operator of the reliable updates
    eta_h, x_h = eta.cpu().numpy(), x.cpu().numpy()
    true = _true_residual(eta_h, Dx)
    assert true <= 1e-10 and abs(true - res) < 1e-12
    _check_operator(U.cpu().numpy(), x_h, Dx, kappa, dims, 11)
    op.close()


def test_multi_rhs_24x48_full_size():
    wd = require_gpu()
    dims, kappa = (24, 24, 24, 48), 0.12
    lx, ly, lz, lt = dims
    op = wd.WilsonDirac(dims, kappa, BC, wd.WD_PREC_MIXED_F32)
    U = op.generate_gauge(0.4, 1, compress12=True, return_field=True)
    point = torch.zeros((12, lt, lz, ly, lx, 4, 3), dtype=torch.complex128, device="cuda")
    for k in range(12):
        point[k, 0, 0, 0, 0, k // 3, k % 3] = 1.0
    x, iters, res, st = op.solve_multi(point, tol=1e-10, maxit=4000)
    assert st == wd.WD_OK
    Dx = op.apply_multi(x).cpu().numpy()    # FP64 multi-RHS operator
    eta_h, x_h = point.cpu().numpy(), x.cpu().numpy()
    Uh = U.cpu().numpy()
    for k in range(12):
        true = _true_residual(eta_h[k], Dx[k])
        assert true <= 1e-10, k
        assert abs(true - res[k]) < 1e-12, k
    for k in (0, 7, 11):
        _check_operator(Uh, x_h[k], Dx[k], kappa, dims, 20 + k)
    op.close()
