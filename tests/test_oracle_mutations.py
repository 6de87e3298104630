"""Planted mistakes in the oracle (on the CPU) must each fail at least one pin.

This shows the pins are not vacuous: a dropped boundary phase, swapped projectors, transposed
links, a flipped kappa sign or an undaggered backward link all change some checked fact.
"""
import functools

import numpy as np
import pytest

import synthetic
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


CHECKS = [check_fft_solve, check_gauge_covariance, check_gamma5_hermiticity_dense,
          check_stencil_vs_coo, check_plane_wave]


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


MUTATIONS = {
    "drop_boundary_phase": _mut_drop_phase,
    "transpose_links": _mut_transpose_links,
    "flip_kappa_sign": _mut_kappa_sign,
    "swap_projectors": _mut_swap_projectors,
    "flip_gamma_t": _mut_gamma_t_sign,
    "undaggered_backward_link": _mut_undaggered_backward_link,
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
