"""Pins of the oracle's two checking helpers (no GPU).

Every GPU assertion on a solve reads ``oracle.cg.true_residual`` (the relative residual
||eta - D x|| / ||eta|| that the stopping rule of Sec. 2 tests, in its relative reading) and every
field comparison reads ``oracle.wilson.rel_diff`` (||a - b|| / ||b||). Both are tied here to
``numpy.linalg.norm`` of the residual against the dense matrix of Eq. (1) (built from the COO
entries, itself pinned against the stencil and the free-field spectrum), and to closed forms:
||eta - D 0|| / ||eta|| = 1, the exact solution gives a residual at rounding level, rel_diff(2b, b)
= 1. The residual cases are sized so that a residual with its square root dropped, or D^dagger in
place of D, lands orders of magnitude away from the numpy value.
"""
import numpy as np
import pytest

import synthetic
from oracle import cg, wilson

BC = (1, 1, 1, -1)


def _problem(dims, kappa=0.12):
    U = synthetic.gauge_field(dims, 0.4, 1)
    eta = synthetic.gaussian_source(dims, 2)
    dense = wilson.dense_D(U, kappa, BC)
    x_exact = np.linalg.solve(dense, eta.reshape(-1)).reshape(eta.shape)
    return U, eta, dense, x_exact


def _numpy_residual(dense, eta, x):
    return np.linalg.norm(eta.reshape(-1) - dense @ x.reshape(-1)) / np.linalg.norm(eta.reshape(-1))


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4)])
def test_true_residual_matches_numpy_norm_of_dense_residual(dims):
    U, eta, dense, x_exact = _problem(dims)
    rng = np.random.default_rng(5)
    noise = rng.standard_normal(eta.shape) + 1j * rng.standard_normal(eta.shape)
    for scale in (1e-7, 1e-3, 1.0):
        x = x_exact + scale * noise
        ref = _numpy_residual(dense, eta, x)
        got = cg.true_residual(U, eta, x, 0.12, BC)
        # eta - D x cancels to ~1e-16 ||eta|| absolute: the bound is that plus 1e-10 relative
        assert abs(got - ref) <= 1e-14 + 1e-10 * ref, (scale, got, ref)
    # at scale 1e-7 the residual is ~1e-7: a squared ratio (no square root) would be ~1e-14
    small = _numpy_residual(dense, eta, x_exact + 1e-7 * noise)
    assert 1e-9 < small < 1e-5


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4)])
def test_true_residual_closed_forms(dims):
    U, eta, _, x_exact = _problem(dims)
    assert cg.true_residual(U, eta, np.zeros_like(eta), 0.12, BC) == pytest.approx(1.0, abs=1e-15)
    assert cg.true_residual(U, eta, x_exact, 0.12, BC) < 1e-13
    # kappa = 0: D = 1, so the residual of x = eta / 2 is exactly 1/2
    assert cg.true_residual(U, eta, 0.5 * eta, 0.0, BC) == pytest.approx(0.5, abs=1e-15)


def test_true_residual_uses_D_not_D_dagger():
    U, eta, dense, x_exact = _problem((2, 2, 2, 2))
    # the exact solution of the dagger system is not a solution of D x = eta
    x_dag = np.linalg.solve(dense.conj().T, eta.reshape(-1)).reshape(eta.shape)
    assert cg.true_residual(U, eta, x_dag, 0.12, BC) > 1e-3
    assert cg.true_residual(U, eta, x_exact, 0.12, BC) < 1e-13


def test_rel_diff_matches_numpy_norm():
    rng = np.random.default_rng(9)
    for shape in [(3, 4, 3), (2, 2, 2, 2, 4, 3)]:
        b = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
        a = 10.0 * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))
        ref = np.linalg.norm((a - b).reshape(-1)) / np.linalg.norm(b.reshape(-1))
        assert abs(wilson.rel_diff(a, b) - ref) <= 1e-14 * ref
        # normalised by the second argument: swapping them changes the value by ~10x
        ref_swapped = np.linalg.norm((a - b).reshape(-1)) / np.linalg.norm(a.reshape(-1))
        assert abs(wilson.rel_diff(b, a) - ref_swapped) <= 1e-14 * ref_swapped
        assert ref > 5 * ref_swapped


def test_rel_diff_closed_forms():
    rng = np.random.default_rng(10)
    b = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
    assert wilson.rel_diff(b, b) == 0.0
    assert wilson.rel_diff(2 * b, b) == pytest.approx(1.0, abs=1e-15)
    assert wilson.rel_diff(np.zeros_like(b), b) == pytest.approx(1.0, abs=1e-15)
    # a small difference: 1e-8 relative, where a squared ratio would give 1e-16
    d = b.copy()
    d[0, 0] += 1e-8 * np.linalg.norm(b)
    assert wilson.rel_diff(d, b) == pytest.approx(1e-8, rel=1e-6)
