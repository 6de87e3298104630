"""Planted mistakes in the oracle (on the CPU) must each fail at least one pin.

This shows the pins are not vacuous: a dropped boundary phase, swapped projectors, transposed
links, a flipped kappa sign or an undaggered backward link all change some checked fact, and so
do mistakes in the two CG solvers (norms without their squares, D in place of D^dagger, a search
direction restarted, or a beta lagging by one iteration, which still converges) and in the
two checking helpers every GPU test reads (a residual without its square root or with D^dagger,
a relative difference normalised by the wrong argument or left squared).
"""
import functools

import numpy as np
import pytest

import synthetic
from oracle import cg as ocg
from oracle import freefield, wilson
from oracle.gamma import GAMMA5

BC = (1, 1, 1, -1)


def check_fft_solve():
    dims = (4, 2, 2, 4)
    eta = synthetic.gaussian_source(dims, 5)
    x = freefield.solve(eta, 0.124, BC)
    assert wilson.rel_diff(wilson.apply_D(synthetic.unit_gauge(dims), x, 0.124, BC), eta) < 1e-12


def check_gauge_covariance():
    dims = (2, 3, 2, 3)
    U = synthetic.gauge_field(dims, 0.4, 1)
    psi = synthetic.gaussian_source(dims, 2)
    om = synthetic.random_gauge_transform(dims, 11)
    Up = np.empty_like(U)
    for mu in range(4):
        of = np.roll(om, -1, axis=3 - mu)
        Up[..., mu, :, :] = om @ U[..., mu, :, :] @ np.conj(np.swapaxes(of, -1, -2))
    lhs = wilson.apply_D(Up, np.einsum("...ab,...sb->...sa", om, psi), 0.12, BC)
    rhs = np.einsum("...ab,...sb->...sa", om, wilson.apply_D(U, psi, 0.12, BC))
    assert np.abs(lhs - rhs).max() < 1e-12


def check_gamma5_hermiticity_dense():
    dims = (2, 2, 2, 2)
    U = synthetic.gauge_field(dims, 0.4, 1)
    d = wilson.dense_D(U, 0.12, BC)
    g5 = np.kron(np.eye(16), np.kron(GAMMA5, np.eye(3)))
    assert np.abs(g5 @ d @ g5 - d.conj().T).max() < 1e-12


def check_stencil_vs_coo():
    dims = (2, 3, 2, 3)
    U = synthetic.gauge_field(dims, 0.4, 1)
    psi = synthetic.gaussian_source(dims, 2)
    r, c, v = wilson.assemble_coo(U, 0.12, BC)
    a = wilson.coo_spmv(r, c, v, psi.reshape(-1))
    assert np.abs(a - wilson.apply_D(U, psi, 0.12, BC).reshape(-1)).max() < 1e-12


def check_plane_wave():
    dims = (4, 3, 2, 4)
    chi = np.arange(12).reshape(4, 3) * (1 + 0.5j)
    psi, p = freefield.plane_wave(dims, (1, 2, 1, 3), chi, BC)
    out = wilson.apply_D(synthetic.unit_gauge(dims), psi, 0.11, BC)
    ref, _ = freefield.plane_wave(dims, (1, 2, 1, 3), freefield.symbol(p, 0.11) @ chi, BC)
    assert np.abs(out - ref).max() < 1e-12


def _dense_solution(dims, kappa):
    U = synthetic.gauge_field(dims, 0.4, 1)
    eta = synthetic.gaussian_source(dims, 2)
    x = np.linalg.solve(wilson.dense_D(U, kappa, BC), eta.reshape(-1))
    return U, eta, x


def check_cgls_against_dense_solve():
    dims = (2, 2, 2, 2)
    U, eta, xd = _dense_solution(dims, 0.12)
    x, k, res, hist = ocg.cgls(U, eta, 0.12, 1e-12, 150, boundary=BC)
    assert wilson.rel_diff(x.reshape(-1), xd) < 1e-9
    assert k < 150 and np.all(np.diff(hist) <= 1e-12 * hist[:-1])  # CGLS: monotone residual


def check_cg_paper_against_dense_solve():
    dims = (2, 2, 2, 2)
    U, eta, xd = _dense_solution(dims, 0.12)
    x, k, res, _ = ocg.cg_paper(U, eta, 0.12, 1e-12, 150, boundary=BC)
    assert wilson.rel_diff(x.reshape(-1), xd) < 1e-9 and k < 150


def check_true_residual_against_dense():
    dims = (2, 2, 2, 2)
    U, eta, xd = _dense_solution(dims, 0.12)
    d = wilson.dense_D(U, 0.12, BC)
    rng = np.random.default_rng(3)
    x = xd + 1e-7 * (rng.standard_normal(xd.shape) + 1j * rng.standard_normal(xd.shape))
    ref = np.linalg.norm(eta.reshape(-1) - d @ x) / np.linalg.norm(eta.reshape(-1))
    got = ocg.true_residual(U, eta, x.reshape(eta.shape), 0.12, BC)
    assert abs(got - ref) <= 1e-14 + 1e-10 * ref


def check_rel_diff_against_numpy():
    rng = np.random.default_rng(4)
    b = rng.standard_normal((6, 4, 3)) + 1j * rng.standard_normal((6, 4, 3))
    a = b + 1e-6 * (rng.standard_normal(b.shape) + 1j * rng.standard_normal(b.shape))
    for u, v in ((a, b), (3 * b, b), (b, 3 * b)):
        ref = np.linalg.norm((u - v).reshape(-1)) / np.linalg.norm(v.reshape(-1))
        assert abs(wilson.rel_diff(u, v) - ref) <= 1e-14 * ref


def _krylov_basis(A, b, k):
    V = np.zeros((b.size, k), dtype=np.complex128)
    v = b / np.linalg.norm(b)
    for j in range(k):
        for _ in range(2):
            v = v - V[:, :j] @ (V[:, :j].conj().T @ v)
        V[:, j] = v / np.linalg.norm(v)
        v = A @ V[:, j]
    return V


def check_cg_iterates_are_krylov_minimisers():
    # after 3 iterations from zero: CGLS minimises ||eta - D x||, the paper's CG the error of
    # x = D^dag psi, both over K_3(D^dag D, D^dag eta)
    dims = (2, 2, 2, 2)
    U, eta, xd = _dense_solution(dims, 0.12)
    d = wilson.dense_D(U, 0.12, BC)
    b = eta.reshape(-1)
    V = _krylov_basis(d.conj().T @ d, d.conj().T @ b, 3)
    y, *_ = np.linalg.lstsq(d @ V, b, rcond=None)
    x, _, _, _ = ocg.cgls(U, eta, 0.12, 0.0, 3, boundary=BC)
    assert wilson.rel_diff(x.reshape(-1), V @ y) < 1e-9
    x, _, _, _ = ocg.cg_paper(U, eta, 0.12, 0.0, 3, boundary=BC)
    assert wilson.rel_diff(x.reshape(-1), V @ (V.conj().T @ xd)) < 1e-9


CHECKS = [check_fft_solve, check_gauge_covariance, check_gamma5_hermiticity_dense,
          check_stencil_vs_coo, check_plane_wave, check_cgls_against_dense_solve,
          check_cg_paper_against_dense_solve, check_true_residual_against_dense,
          check_rel_diff_against_numpy, check_cg_iterates_are_krylov_minimisers]


def _wrap_both(monkeypatch, transform_args):
    """Apply the same planted mistake to the stencil and to the COO assembly."""
    orig_apply, orig_coo = wilson.apply_D, wilson.assemble_coo

    def apply(U, psi, kappa, boundary=BC, dagger=False):
        U, kappa, boundary = transform_args(U, kappa, boundary)
        return orig_apply(U, psi, kappa, boundary, dagger)

    def coo(U, kappa, boundary=BC):
        U, kappa, boundary = transform_args(U, kappa, boundary)
        return orig_coo(U, kappa, boundary)

    monkeypatch.setattr(wilson, "apply_D", apply)
    monkeypatch.setattr(wilson, "assemble_coo", coo)


def _mut_drop_phase(mp):
    _wrap_both(mp, lambda U, k, b: (U, k, (1, 1, 1, 1)))


def _mut_transpose_links(mp):
    _wrap_both(mp, lambda U, k, b: (np.swapaxes(U, -1, -2), k, b))


def _mut_kappa_sign(mp):
    _wrap_both(mp, lambda U, k, b: (U, -k, b))


def _mut_swap_projectors(mp):
    pm, pp = wilson.projector_minus, wilson.projector_plus
    mp.setattr(wilson, "projector_minus", pp)
    mp.setattr(wilson, "projector_plus", pm)


def _mut_gamma_t_sign(mp):
    pm, pp = wilson.projector_minus, wilson.projector_plus
    mp.setattr(wilson, "projector_minus", lambda mu: pp(mu) if mu == 3 else pm(mu))
    mp.setattr(wilson, "projector_plus", lambda mu: pm(mu) if mu == 3 else pp(mu))


def _mut_undaggered_backward_link(mp):
    # the stencil's backward hop uses U(n - mu) instead of U(n - mu)^dagger
    orig = wilson.apply_D

    def apply(U, psi, kappa, boundary=BC, dagger=False):
        hop = np.zeros_like(psi)
        for mu in range(4):
            ax = 3 - mu
            u = U[..., mu, :, :]
            L = psi.shape[ax]
            pf = wilson._edge_phase(np.roll(psi, -1, axis=ax), mu, L - 1, boundary[mu])
            pb = wilson._edge_phase(np.roll(psi, 1, axis=ax), mu, 0, boundary[mu])
            fwd = np.einsum("...ab,...sb->...sa", u, pf)
            bwd = np.einsum("...ab,...sb->...sa", np.roll(u, 1, axis=ax), pb)
            hop += wilson._spin(wilson.projector_minus(mu), fwd)
            hop += wilson._spin(wilson.projector_plus(mu), bwd)
        return psi - kappa * hop

    mp.setattr(wilson, "apply_D", apply)
    assert orig is not apply


def _mut_unsquared_cg_norms(mp):
    # the printed algorithm's literal reading: norms where squared norms belong
    orig = ocg.norm2
    mp.setattr(ocg, "norm2", lambda v: float(np.sqrt(orig(v))))


def _mut_cg_without_dagger(mp):
    # both solvers apply D where D^dagger belongs
    orig = ocg.apply_D
    mp.setattr(ocg, "apply_D", lambda U, v, kappa, boundary=BC, dagger=False: orig(U, v, kappa, boundary, False))


def _mut_true_residual_squared(mp):
    # the squared ratio ||eta - D x||^2 / ||eta||^2 (square root dropped)
    mp.setattr(ocg, "true_residual", lambda U, eta, x, kappa, boundary=BC: float(
        wilson.norm2(eta - wilson.apply_D(U, x, kappa, boundary)) / wilson.norm2(eta)))


def _mut_true_residual_dagger(mp):
    mp.setattr(ocg, "true_residual", lambda U, eta, x, kappa, boundary=BC: float(np.sqrt(
        wilson.norm2(eta - wilson.apply_D(U, x, kappa, boundary, dagger=True)) / wilson.norm2(eta))))


def _mut_rel_diff_wrong_norm(mp):
    # normalised by the first argument instead of the second
    mp.setattr(wilson, "rel_diff", lambda a, b: float(
        np.sqrt(wilson.norm2(np.asarray(a) - np.asarray(b)) / wilson.norm2(a))))


def _mut_rel_diff_squared(mp):
    mp.setattr(wilson, "rel_diff", lambda a, b: float(
        wilson.norm2(np.asarray(a) - np.asarray(b)) / wilson.norm2(b)))


def _mut_cgls_periodic_restart(mp):
    # CGLS that drops the search direction's history every other iteration (p = s): the third
    # iterate already leaves the Krylov minimiser
    def cgls(U, eta, kappa, tol, maxit, x0=None, boundary=BC):
        D = lambda v: wilson.apply_D(U, v, kappa, boundary)                  # noqa: E731
        Dd = lambda v: wilson.apply_D(U, v, kappa, boundary, dagger=True)    # noqa: E731
        x = np.zeros_like(eta) if x0 is None else np.array(x0, dtype=np.complex128)
        en = np.sqrt(wilson.norm2(eta))
        r = eta - D(x)
        s = Dd(r)
        p, gamma, hist, k = s.copy(), wilson.norm2(s), [np.sqrt(wilson.norm2(r)) / en], 0
        while hist[-1] > tol and k < maxit:
            q = D(p)
            alpha = gamma / wilson.norm2(q)
            x, r = x + alpha * p, r - alpha * q
            s = Dd(r)
            gnew = wilson.norm2(s)
            p = s if (k + 1) % 2 == 0 else s + (gnew / gamma) * p
            gamma, k = gnew, k + 1
            hist.append(np.sqrt(wilson.norm2(r)) / en)
        return x, k, float(np.sqrt(wilson.norm2(eta - D(x))) / en), np.array(hist)

    mp.setattr(ocg, "cgls", cgls)


def _mut_paper_cg_lagged_beta(mp):
    # the paper's CG with beta taken from the previous iteration's ratio: it still reaches
    # D^-1 eta within the dense-solve check's budget, so only the iterate check sees it
    def cg_paper(U, eta, kappa, tol, maxit, psi0=None, boundary=BC):
        D = lambda v: wilson.apply_D(U, v, kappa, boundary)                  # noqa: E731
        Dd = lambda v: wilson.apply_D(U, v, kappa, boundary, dagger=True)    # noqa: E731
        psi = np.zeros_like(eta) if psi0 is None else np.array(psi0, dtype=np.complex128)
        en = np.sqrt(wilson.norm2(eta))
        r = eta - D(Dd(psi))
        p, k, beta_prev, hist = r.copy(), 0, 0.0, [np.sqrt(wilson.norm2(r)) / en]
        while np.sqrt(wilson.norm2(r)) >= tol * en and k < maxit:
            r_old = wilson.norm2(r)
            ddp = Dd(p)
            alpha = r_old / wilson.norm2(ddp)
            psi, r = psi + alpha * p, r - alpha * D(ddp)
            beta = wilson.norm2(r) / r_old
            p = r + (beta_prev if k > 0 else beta) * p
            beta_prev, k = beta, k + 1
            hist.append(np.sqrt(wilson.norm2(r)) / en)
        x = Dd(psi)
        return x, k, float(np.sqrt(wilson.norm2(eta - D(x))) / en), np.array(hist)

    mp.setattr(ocg, "cg_paper", cg_paper)


MUTATIONS = {
    "cgls_periodic_restart": _mut_cgls_periodic_restart,
    "paper_cg_lagged_beta": _mut_paper_cg_lagged_beta,
    "drop_boundary_phase": _mut_drop_phase,
    "transpose_links": _mut_transpose_links,
    "flip_kappa_sign": _mut_kappa_sign,
    "swap_projectors": _mut_swap_projectors,
    "flip_gamma_t": _mut_gamma_t_sign,
    "undaggered_backward_link": _mut_undaggered_backward_link,
    "unsquared_cg_norms": _mut_unsquared_cg_norms,
    "cg_without_dagger": _mut_cg_without_dagger,
    "true_residual_squared": _mut_true_residual_squared,
    "true_residual_dagger": _mut_true_residual_dagger,
    "rel_diff_wrong_norm": _mut_rel_diff_wrong_norm,
    "rel_diff_squared": _mut_rel_diff_squared,
}


def test_unmutated_oracle_passes_all_checks():
    for check in CHECKS:
        check()


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, monkeypatch):
    MUTATIONS[name](monkeypatch)
    failed = []
    for check in CHECKS:
        try:
            check()
        except AssertionError:
            failed.append(check.__name__)
    assert failed, f"planted mistake {name} passed every pin"
