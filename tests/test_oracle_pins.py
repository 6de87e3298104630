"""Pins of the CPU oracle against facts fixed by the paper and by mathematics (no GPU).

Each check ties the oracle to something other than itself: hand-written gamma entries, the
Clifford algebra, gamma_5-hermiticity (Sec. 2), the free-field closed form of Eq. (1), a dense
direct solve (brute force), gauge and translation covariance, and CG's monotone residual.
``test_oracle_mutations.py`` plants plausible mistakes in the oracle and shows these pins catch them.
"""
import json
import os

import numpy as np
import pytest

import synthetic
from oracle import cg, freefield, wilson
from oracle.gamma import GAMMA, GAMMA5

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
BC = (1, 1, 1, -1)


def _parse(entry):
    return {"0": 0, "1": 1, "-1": -1, "i": 1j, "-i": -1j}[entry]


def _fields(dims, eps=0.4, gseed=1, sseed=2):
    return synthetic.gauge_field(dims, eps, gseed), synthetic.gaussian_source(dims, sseed)


# ---------------------------------------------------------------- gamma matrices

def test_gamma_matches_handwritten_fixture():
    with open(os.path.join(GOLDEN, "gamma_chiral.json")) as f:
        g = json.load(f)
    for mu, key in enumerate(["gamma_x", "gamma_y", "gamma_z", "gamma_t"]):
        ref = np.array([[_parse(e) for e in row] for row in g[key]], dtype=np.complex128)
        assert np.array_equal(GAMMA[mu], ref), key
    ref5 = np.array([[_parse(e) for e in row] for row in g["gamma_5"]], dtype=np.complex128)
    assert np.allclose(GAMMA5, ref5, atol=0)


def test_clifford_algebra_and_hermiticity():
    for mu in range(4):
        assert np.allclose(GAMMA[mu], GAMMA[mu].conj().T)
        for nu in range(4):
            anti = GAMMA[mu] @ GAMMA[nu] + GAMMA[nu] @ GAMMA[mu]
            assert np.allclose(anti, 2 * (mu == nu) * np.eye(4))
        assert np.allclose(GAMMA5 @ GAMMA[mu], -GAMMA[mu] @ GAMMA5)


# ---------------------------------------------------------------- gauge generator

@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4)])
def test_links_are_su3(dims):
    U = synthetic.gauge_field(dims, 0.4, 1)
    eye = np.eye(3)
    dev = np.abs(np.conj(np.swapaxes(U, -1, -2)) @ U - eye).max()
    det = np.abs(np.linalg.det(U) - 1).max()
    assert dev < 1e-14 and det < 1e-14
    # not trivially close to the identity: eps = 0.4 moves links well away from 1
    assert np.abs(U - eye).max() > 0.3


# ---------------------------------------------------------------- three constructions of D

@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (3, 3, 3, 3), (2, 3, 4, 5)])
@pytest.mark.parametrize("dagger", [False, True])
def test_stencil_equals_literal_loop(dims, dagger):
    U, psi = _fields(dims)
    full = wilson.apply_D(U, psi, 0.12, BC, dagger)
    lx, ly, lz, lt = dims
    sites = [(x, y, z, t) for t in range(lt) for z in range(lz) for y in range(ly) for x in range(lx)]
    loop = wilson.apply_D_sites(U, psi, 0.12, sites, BC, dagger)
    assert np.abs(full.reshape(-1, 4, 3) - loop).max() < 1e-14


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (3, 3, 3, 3), (2, 3, 4, 5), (4, 4, 4, 4)])
def test_stencil_equals_coo_equals_dense(dims):
    U, psi = _fields(dims)
    kappa = 0.13
    stencil = wilson.apply_D(U, psi, kappa, BC).reshape(-1)
    row, col, val = wilson.assemble_coo(U, kappa, BC)
    coo = wilson.coo_spmv(row, col, val, psi.reshape(-1))
    assert np.abs(stencil - coo).max() < 1e-14
    if synthetic.volume(dims) <= 256:
        dense = wilson.dense_D(U, kappa, BC)
        assert np.abs(dense @ psi.reshape(-1) - stencil).max() < 1e-13


def test_coo_has_49_nonzeros_per_row():
    # 1 diagonal + 8 hops x 2 spin entries x 3 colours, for every extent >= 3
    U, _ = _fields((3, 3, 4, 3))
    row, _, _ = wilson.assemble_coo(U, 0.12, BC)
    counts = np.bincount(row)
    assert counts.min() == 49 and counts.max() == 49


def test_two_site_extent_adds_both_hops():
    # L = 2: n + mu and n - mu coincide; Eq. (1) sums both terms (the COO keeps duplicates)
    U, psi = _fields((2, 2, 2, 2))
    row, col, val = wilson.assemble_coo(U, 0.12, BC)
    pairs = row.astype(np.int64) * (12 * 16) + col
    assert len(np.unique(pairs)) < len(pairs)
    dense = wilson.dense_D(U, 0.12, BC)
    stencil = wilson.apply_D(U, psi, 0.12, BC).reshape(-1)
    assert np.abs(dense @ psi.reshape(-1) - stencil).max() < 1e-14


# ---------------------------------------------------------------- hermiticity (Sec. 2)

@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 3, 4, 5)])
def test_dagger_is_conjugate_transpose(dims):
    U, psi = _fields(dims)
    dense = wilson.dense_D(U, 0.12, BC)
    dag = wilson.apply_D(U, psi, 0.12, BC, dagger=True).reshape(-1)
    assert np.abs(dense.conj().T @ psi.reshape(-1) - dag).max() < 1e-14


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (3, 2, 4, 3)])
def test_gamma5_hermiticity(dims):
    # gamma_5 D gamma_5 = D^dagger, as a matrix identity and on random fields
    U, psi = _fields(dims)
    dense = wilson.dense_D(U, 0.12, BC)
    V = synthetic.volume(dims)
    g5 = np.kron(np.eye(V), np.kron(GAMMA5, np.eye(3)))
    assert np.abs(g5 @ dense @ g5 - dense.conj().T).max() < 1e-14
    lhs = wilson.apply_gamma5(wilson.apply_D(U, wilson.apply_gamma5(psi), 0.12, BC))
    rhs = wilson.apply_D(U, psi, 0.12, BC, dagger=True)
    assert np.abs(lhs - rhs).max() < 1e-14


def test_adjoint_inner_product():
    # <chi, D psi> = <D^dagger chi, psi>
    U, psi = _fields((4, 3, 2, 5))
    chi = synthetic.gaussian_source((4, 3, 2, 5), 7)
    a = np.vdot(chi, wilson.apply_D(U, psi, 0.12, BC))
    b = np.vdot(wilson.apply_D(U, chi, 0.12, BC, dagger=True), psi)
    assert abs(a - b) < 1e-11 * abs(a)


# ---------------------------------------------------------------- free-field closed form

def test_free_field_spectrum_4444():
    dims = (4, 4, 4, 4)
    U = synthetic.unit_gauge(dims)
    dense = wilson.dense_D(U, 0.12, BC)
    ev = np.linalg.eigvalsh(dense.conj().T @ dense)
    ref = freefield.DdagD_eigenvalues(dims, 0.12, BC)
    assert np.abs(np.sort(ev) - ref).max() < 1e-12
    # smallest value by hand: p = (0, 0, 0, pi/4): a = 1 - 0.24 (3 + cos(pi/4)), |b|^2 = 4 k^2 / 2
    a = 1 - 0.24 * (3 + np.cos(np.pi / 4))
    assert abs(ref[0] - (a * a + 4 * 0.12 ** 2 * 0.5)) < 1e-15


def test_free_field_spectrum_mixed_boundaries():
    dims = (2, 3, 2, 4)
    bc = (1, -1, 1, -1)
    U = synthetic.unit_gauge(dims)
    dense = wilson.dense_D(U, 0.2, bc)
    ev = np.linalg.eigvalsh(dense.conj().T @ dense)
    assert np.abs(np.sort(ev) - freefield.DdagD_eigenvalues(dims, 0.2, bc)).max() < 1e-12


@pytest.mark.parametrize("k", [(0, 0, 0, 0), (1, 2, 0, 3), (3, 1, 2, 5)])
def test_plane_wave_eigenvectors(k):
    dims = (4, 3, 5, 6)
    U = synthetic.unit_gauge(dims)
    rng = np.random.default_rng(3)
    chi = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
    psi, p = freefield.plane_wave(dims, k, chi, BC)
    out = wilson.apply_D(U, psi, 0.11, BC)
    expect, _ = freefield.plane_wave(dims, k, freefield.symbol(p, 0.11) @ chi, BC)
    assert np.abs(out - expect).max() < 1e-13


def test_free_field_fft_solve():
    dims = (6, 4, 4, 8)
    U = synthetic.unit_gauge(dims)
    eta = synthetic.gaussian_source(dims, 5)
    x = freefield.solve(eta, 0.124, BC)
    assert wilson.rel_diff(wilson.apply_D(U, x, 0.124, BC), eta) < 1e-13


# ---------------------------------------------------------------- covariance

@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 3, 3, 4)])
def test_gauge_covariance(dims):
    U, psi = _fields(dims)
    omega = synthetic.random_gauge_transform(dims, 11)
    Up = np.empty_like(U)
    for mu in range(4):
        ax = 3 - mu
        omega_fwd = np.roll(omega, -1, axis=ax)          # Omega(n + mu)
        Up[..., mu, :, :] = omega @ U[..., mu, :, :] @ np.conj(np.swapaxes(omega_fwd, -1, -2))
    psip = np.einsum("...ab,...sb->...sa", omega, psi)
    for dagger in (False, True):
        lhs = wilson.apply_D(Up, psip, 0.12, BC, dagger)
        rhs = np.einsum("...ab,...sb->...sa", omega, wilson.apply_D(U, psi, 0.12, BC, dagger))
        assert np.abs(lhs - rhs).max() < 1e-13


def test_translation_covariance():
    dims = (3, 4, 2, 5)
    U, psi = _fields(dims)
    # periodic x: shift everything by one site
    lhs = wilson.apply_D(np.roll(U, 1, axis=3), np.roll(psi, 1, axis=3), 0.12, BC)
    assert np.abs(lhs - np.roll(wilson.apply_D(U, psi, 0.12, BC), 1, axis=3)).max() < 1e-14

    # antiperiodic t: a twisted shift, psi'(t) = psi(t - 1) with psi(-1) = -psi(Lt - 1)
    def tshift(f):
        g = np.roll(f, 1, axis=0)
        g[0] *= -1
        return g

    lhs = wilson.apply_D(np.roll(U, 1, axis=0), tshift(psi), 0.12, BC)
    assert np.abs(lhs - tshift(wilson.apply_D(U, psi, 0.12, BC))).max() < 1e-14


def test_linearity_and_kappa_zero():
    U, psi = _fields((2, 3, 2, 3))
    chi = synthetic.gaussian_source((2, 3, 2, 3), 9)
    a, b = 0.7 - 0.2j, -1.3 + 0.5j
    lhs = wilson.apply_D(U, a * psi + b * chi, 0.12, BC)
    rhs = a * wilson.apply_D(U, psi, 0.12, BC) + b * wilson.apply_D(U, chi, 0.12, BC)
    assert np.abs(lhs - rhs).max() < 1e-13
    assert np.array_equal(wilson.apply_D(U, psi, 0.0, BC), psi)


# ---------------------------------------------------------------- CG against brute force

def test_cgls_matches_direct_solve_4444():
    dims = (4, 4, 4, 4)
    U, eta = _fields(dims)
    dense = wilson.dense_D(U, 0.12, BC)
    x_direct = np.linalg.solve(dense, eta.reshape(-1))
    x, iters, true_res, hist = cg.cgls(U, eta, 0.12, 1e-10, 2000)
    assert true_res <= 1e-10
    assert 20 < iters < 300
    assert wilson.rel_diff(x.reshape(-1), x_direct) < 1e-8
    # recursive and true residual agree at the end (FP64 drift is tiny at this size)
    assert abs(hist[-1] - true_res) < 1e-12


def test_cg_paper_form_matches_direct_solve():
    dims = (2, 2, 4, 4)
    U, eta = _fields(dims)
    dense = wilson.dense_D(U, 0.12, BC)
    x_direct = np.linalg.solve(dense, eta.reshape(-1))
    x, iters, true_res, _ = cg.cg_paper(U, eta, 0.12, 1e-10, 2000)
    assert true_res <= 2e-10          # the paper's test is on the DD^dagger residual
    assert wilson.rel_diff(x.reshape(-1), x_direct) < 1e-8


def test_cgls_true_residual_is_monotone():
    # CGLS minimises ||eta - D x_k|| over a growing Krylov space: non-increasing up to rounding
    dims = (4, 4, 2, 4)
    U, eta = _fields(dims, eps=0.5)
    dense = wilson.dense_D(U, 0.124, BC)
    prev = np.inf
    for k in range(0, 60, 3):
        x, _, res, _ = cg.cgls(U, eta, 0.124, 0.0, k)
        true = np.linalg.norm(eta.reshape(-1) - dense @ x.reshape(-1)) / np.linalg.norm(eta)
        assert abs(true - res) < 1e-12
        assert res <= prev * (1 + 1e-12)
        prev = res


def test_cgls_kappa_zero_one_iteration():
    U, eta = _fields((2, 2, 2, 4))
    x, iters, res, _ = cg.cgls(U, eta, 0.0, 1e-12, 10)
    assert iters == 1 and res < 1e-15 and np.allclose(x, eta, atol=1e-15)


def test_cgls_free_field_matches_fft_solve():
    dims = (4, 4, 4, 6)
    U = synthetic.unit_gauge(dims)
    eta = synthetic.gaussian_source(dims, 4)
    x, _, res, _ = cg.cgls(U, eta, 0.12, 1e-11, 2000)
    assert res <= 1e-11
    assert wilson.rel_diff(x, freefield.solve(eta, 0.12, BC)) < 1e-9


def _krylov_basis(A, b, k):
    """Orthonormal basis of K_k(A, b) = span{b, A b, ..., A^(k-1) b} (Gram-Schmidt, twice)."""
    V = np.zeros((b.size, k), dtype=np.complex128)
    v = b / np.linalg.norm(b)
    for j in range(k):
        for _ in range(2):
            v = v - V[:, :j] @ (V[:, :j].conj().T @ v)
        V[:, j] = v / np.linalg.norm(v)
        v = A @ V[:, j]
    return V


@pytest.mark.parametrize("k", [1, 2, 3, 5, 7])
def test_cgls_iterate_is_the_krylov_least_squares_minimiser(k):
    """From x0 = 0, the k-th CGLS iterate minimises ||eta - D x|| over K_k(D^dag D, D^dag eta):
    checked against a least-squares solve on an explicit Krylov basis of the dense D, so a wrong
    alpha, beta or update order fails here even where the iteration would still converge."""
    dims = (2, 2, 2, 4)
    U, eta = _fields(dims, eps=0.5, gseed=7, sseed=8)
    D = wilson.dense_D(U, 0.124, BC)
    b = eta.reshape(-1)
    V = _krylov_basis(D.conj().T @ D, D.conj().T @ b, k)
    y, *_ = np.linalg.lstsq(D @ V, b, rcond=None)
    x, iters, _, _ = cg.cgls(U, eta, 0.124, 0.0, k)
    assert iters == k
    assert wilson.rel_diff(x.reshape(-1), V @ y) < 1e-9


@pytest.mark.parametrize("k", [1, 2, 4, 6])
def test_paper_cg_iterate_minimises_the_error_norm(k):
    """CG on D D^dag psi = eta from psi0 = 0 minimises the D D^dag-energy norm of the error of psi,
    which is the 2-norm of the error of x = D^dag psi; x_k therefore is the orthogonal projection of
    the exact solution D^-1 eta onto K_k(D^dag D, D^dag eta) (dense solve, explicit basis)."""
    dims = (2, 2, 2, 4)
    U, eta = _fields(dims, eps=0.5, gseed=9, sseed=10)
    D = wilson.dense_D(U, 0.124, BC)
    b = eta.reshape(-1)
    xstar = np.linalg.solve(D, b)
    V = _krylov_basis(D.conj().T @ D, D.conj().T @ b, k)
    x, iters, _, _ = cg.cg_paper(U, eta, 0.124, 0.0, k)
    assert iters == k
    assert wilson.rel_diff(x.reshape(-1), V @ (V.conj().T @ xstar)) < 1e-9
