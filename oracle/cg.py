"""Conjugate gradient for D psi = eta (test infrastructure only).

Sec. 2 of the paper uses gamma_5-hermiticity to turn the non-Hermitian system into a Hermitian
one, solves it with standard CG and multiplies by D^dagger. Its printed algorithm is garbled
(norms appear without squares); the readings taken here:

* ``|r|`` in the assignments to r_old and beta is the squared norm ||r||^2, and the denominator of
  alpha is ||D^dagger p||^2 -- without the squares the recurrence is not CG;
* the initial residual is eta - D D^dagger psi_0 (identical to the printed eta - D psi_0 when
  psi_0 = 0, the only guess the paper's text implies);
* the stopping test ``|r| >= r_min`` is an absolute threshold on ||r||; the library and these
  functions use a relative one, ||r|| / ||eta|| <= tol.

Two solvers follow:

* :func:`cg_paper` -- the paper's algorithm step by step (CG on D D^dagger y = eta, x = D^dagger y).
* :func:`cgls` -- CG on the normal equations D^dagger D x = D^dagger eta in the CGLS arrangement,
  which tracks the true-system residual r = eta - D x and needs the same two operator
  applications per iteration. This is the form the CUDA library implements.

Both return the exact solution x = D^{-1} eta up to the tolerance; the tests check both against a
dense direct solve.
"""
from __future__ import annotations

import numpy as np

from .wilson import DEFAULT_BOUNDARY, apply_D, norm2


def _dot(a, b) -> complex:
    return complex(np.vdot(a.reshape(-1), b.reshape(-1)))


def cgls(U, eta, kappa, tol, maxit, x0=None, boundary=DEFAULT_BOUNDARY):
    """CG on D^dagger D x = D^dagger eta (CGLS form), FP64 throughout.

    Steps: r = eta - D x; s = D^dagger r; p = s; gamma = ||s||^2; then per iteration
    q = D p; alpha = gamma / ||q||^2; x += alpha p; r -= alpha q; s = D^dagger r;
    gamma' = ||s||^2; p = s + (gamma' / gamma) p. Stops when ||r|| / ||eta|| <= tol.

    Returns (x, iterations, true relative residual ||eta - D x|| / ||eta||, history of the
    recursive relative residual, one entry per iteration plus the initial one).
    """
    D = lambda v: apply_D(U, v, kappa, boundary)                  # noqa: E731
    Dd = lambda v: apply_D(U, v, kappa, boundary, dagger=True)    # noqa: E731
    x = np.zeros_like(eta) if x0 is None else np.array(x0, dtype=np.complex128)
    eta_norm = np.sqrt(norm2(eta))
    r = eta - D(x)
    s = Dd(r)
    p = s.copy()
    gamma = norm2(s)
    history = [np.sqrt(norm2(r)) / eta_norm]
    k = 0
    while history[-1] > tol and k < maxit:
        q = D(p)
        alpha = gamma / norm2(q)
        x = x + alpha * p
        r = r - alpha * q
        s = Dd(r)
        gamma_new = norm2(s)
        p = s + (gamma_new / gamma) * p
        gamma = gamma_new
        k += 1
        history.append(np.sqrt(norm2(r)) / eta_norm)
    true_res = np.sqrt(norm2(eta - D(x))) / eta_norm
    return x, k, float(true_res), np.array(history)


def cg_paper(U, eta, kappa, tol, maxit, psi0=None, boundary=DEFAULT_BOUNDARY):
    """The paper's CG (Sec. 2 algorithm) on D D^dagger psi = eta, then x = D^dagger psi.

    psi <- psi_0; r <- eta - D D^dagger psi; p <- r; while ||r|| >= r_min: r_old <- ||r||^2;
    alpha <- r_old / ||D^dagger p||^2; psi <- psi + alpha p; r <- r - alpha D D^dagger p;
    beta <- ||r||^2 / r_old; p <- r + beta p. Here r_min = tol * ||eta||.

    Returns (x, iterations, true relative residual of x, history of ||r|| / ||eta||).
    """
    D = lambda v: apply_D(U, v, kappa, boundary)                  # noqa: E731
    Dd = lambda v: apply_D(U, v, kappa, boundary, dagger=True)    # noqa: E731
    psi = np.zeros_like(eta) if psi0 is None else np.array(psi0, dtype=np.complex128)
    eta_norm = np.sqrt(norm2(eta))
    r_min = tol * eta_norm
    r = eta - D(Dd(psi))
    p = r.copy()
    history = [np.sqrt(norm2(r)) / eta_norm]
    k = 0
    while np.sqrt(norm2(r)) >= r_min and k < maxit:
        r_old = norm2(r)
        ddp = Dd(p)
        alpha = r_old / norm2(ddp)
        psi = psi + alpha * p
        r = r - alpha * D(ddp)
        beta = norm2(r) / r_old
        p = r + beta * p
        k += 1
        history.append(np.sqrt(norm2(r)) / eta_norm)
    x = Dd(psi)
    true_res = np.sqrt(norm2(eta - D(x))) / eta_norm
    return x, k, float(true_res), np.array(history)


def true_residual(U, eta, x, kappa, boundary=DEFAULT_BOUNDARY) -> float:
    """||eta - D x|| / ||eta|| recomputed in FP64."""
    return float(np.sqrt(norm2(eta - apply_D(U, x, kappa, boundary)) / norm2(eta)))
