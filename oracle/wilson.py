"""The Wilson-Dirac operator D of Eq. (1), computed three independent ways (test infrastructure).

Eq. (1) (Sec. 1) poses D^{AB}_{alpha beta}(n, m) psi^B_beta(m) = eta^A_alpha(n) with colour indices
A, B in {0,1,2} and spin indices alpha, beta in {0..3}, D being the Wilson-Dirac operator. The paper
does not write D out. This oracle uses the hopping (kappa) form with Wilson parameter r = 1:

    (D psi)(n) = psi(n) - kappa * sum_mu [ (1 - gamma_mu) U_mu(n)            b_mu^+(n) psi(n + mu)
                                         + (1 + gamma_mu) U_mu(n - mu)^dag   b_mu^-(n) psi(n - mu) ]

with mu = 0..3 = x, y, z, t, neighbours taken modulo the lattice extent, and b_mu^{+/-}(n) the
boundary phase ``boundary[mu]`` (+1 periodic, -1 antiperiodic) for a hop that wraps around the
lattice edge in direction mu, else 1. For L_mu = 2 both hops land on the same site and both terms
are added. D^dagger swaps the two projectors (the conjugate transpose of the hopping matrix),
which equals gamma_5 D gamma_5 (Sec. 2).

Array layout: spinors complex128 [Lt, Lz, Ly, Lx, 4, 3]; links complex128 [Lt, Lz, Ly, Lx, 4, 3, 3]
with U[t,z,y,x,mu] = U_mu(n). Flattened vectors use the C order of that layout:
index = 12 * site + 3 * spin + colour, site = x + Lx * (y + Ly * (z + Lz * t)).
"""
from __future__ import annotations

import numpy as np

from .gamma import GAMMA, GAMMA5, projector_minus, projector_plus

DEFAULT_BOUNDARY = (1, 1, 1, -1)


def lattice_dims(field) -> tuple:
    """(Lx, Ly, Lz, Lt) of a spinor or gauge array."""
    lt, lz, ly, lx = field.shape[:4]
    return (lx, ly, lz, lt)


def _axis(mu: int) -> int:
    # array axis of direction mu: x is axis 3, t is axis 0
    return 3 - mu


def _edge_phase(field, mu: int, index: int, phase: float):
    """Multiply the slab at coordinate `index` along direction mu by `phase` (in a copy)."""
    if phase == 1:
        return field
    out = field.copy()
    sl = [slice(None)] * out.ndim
    sl[_axis(mu)] = index
    out[tuple(sl)] *= phase
    return out


def _spin(matrix, chi):
    # apply a 4x4 spin matrix to a field [..., 4, 3]
    return np.einsum("st,...tc->...sc", matrix, chi)


def apply_D(U, psi, kappa: float, boundary=DEFAULT_BOUNDARY, dagger: bool = False):
    """R1: the stencil form of Eq. (1), vectorised over sites with periodic shifts.

    ``dagger=True`` applies D^dagger: the forward hop takes (1 + gamma_mu), the backward hop
    (1 - gamma_mu).
    """
    hop = np.zeros_like(psi)
    for mu in range(4):
        ax = _axis(mu)
        L = psi.shape[ax]
        u = U[..., mu, :, :]
        # forward: psi(n + mu); the site at coordinate L-1 wraps around to 0
        psi_f = _edge_phase(np.roll(psi, -1, axis=ax), mu, L - 1, boundary[mu])
        fwd = np.einsum("...ab,...sb->...sa", u, psi_f)
        # backward: U_mu(n - mu)^dagger psi(n - mu); the site at coordinate 0 wraps to L-1
        u_b = np.roll(u, 1, axis=ax)
        psi_b = _edge_phase(np.roll(psi, 1, axis=ax), mu, 0, boundary[mu])
        bwd = np.einsum("...ba,...sb->...sa", np.conj(u_b), psi_b)
        if dagger:
            hop += _spin(projector_plus(mu), fwd) + _spin(projector_minus(mu), bwd)
        else:
            hop += _spin(projector_minus(mu), fwd) + _spin(projector_plus(mu), bwd)
    return psi - kappa * hop


def apply_D_sites(U, psi, kappa: float, sites, boundary=DEFAULT_BOUNDARY, dagger: bool = False):
    """R1': a literal per-site loop of Eq. (1) for the listed sites (x, y, z, t).

    Slow pure-Python control flow with explicit neighbour coordinates and edge tests; used to
    cross-check R1 and to check sampled outputs of large lattices. Returns [len(sites), 4, 3].
    """
    lx, ly, lz, lt = lattice_dims(psi)
    ext = (lx, ly, lz, lt)
    out = np.empty((len(sites), 4, 3), dtype=np.complex128)
    for k, site in enumerate(sites):
        n = list(site)
        acc = np.zeros((4, 3), dtype=np.complex128)
        for mu in range(4):
            fwd_site = list(n)
            fwd_site[mu] += 1
            phase_f = 1.0
            if fwd_site[mu] == ext[mu]:
                fwd_site[mu] = 0
                phase_f = boundary[mu]
            bwd_site = list(n)
            bwd_site[mu] -= 1
            phase_b = 1.0
            if bwd_site[mu] < 0:
                bwd_site[mu] = ext[mu] - 1
                phase_b = boundary[mu]
            x, y, z, t = n
            xf, yf, zf, tf = fwd_site
            xb, yb, zb, tb = bwd_site
            u_here = U[t, z, y, x, mu]
            u_back = U[tb, zb, yb, xb, mu]
            chi_f = phase_f * (psi[tf, zf, yf, xf] @ u_here.T)            # U psi, per spin row
            chi_b = phase_b * (psi[tb, zb, yb, xb] @ np.conj(u_back))     # U^dag psi, per spin row
            p_f = projector_plus(mu) if dagger else projector_minus(mu)
            p_b = projector_minus(mu) if dagger else projector_plus(mu)
            acc += p_f @ chi_f + p_b @ chi_b
        x, y, z, t = n
        out[k] = psi[t, z, y, x] - kappa * acc
    return out


def site_index(x, y, z, t, dims):
    lx, ly, lz, lt = dims
    return x + lx * (y + ly * (z + lz * t))


def assemble_coo(U, kappa: float, boundary=DEFAULT_BOUNDARY):
    """R2: D in the paper's coordinate format (Sec. 2): arrays Row, Col, Val of its non-zeros.

    One entry per structurally non-zero element of each term of Eq. (1): the unit diagonal, then
    for every site, direction, hop sign, spin pair with a non-zero projector entry and colour pair,
    the value -kappa * phase * P[alpha, beta] * (U or U^dagger)[A, B]. Entries are not merged, so
    on an L_mu = 2 lattice two entries can share a (Row, Col) pair and accumulate in the product.
    """
    lx, ly, lz, lt = dims = lattice_dims(U)
    vol = lx * ly * lz * lt
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx),
                             indexing="ij")
    coords = [c.reshape(-1) for c in (x, y, z, t)]
    here = site_index(*coords, dims)
    ext = dims
    rows, cols, vals = [np.arange(12 * vol)], [np.arange(12 * vol)], [np.ones(12 * vol, np.complex128)]
    Uflat = U.reshape(vol, 4, 3, 3)
    for mu in range(4):
        for sign in (+1, -1):
            nb = [c.copy() for c in coords]
            nb[mu] = nb[mu] + sign
            wrapped = (nb[mu] == ext[mu]) | (nb[mu] < 0)
            nb[mu] = nb[mu] % ext[mu]
            phase = np.where(wrapped, float(boundary[mu]), 1.0)
            there = site_index(*nb, dims)
            if sign > 0:
                spin = projector_minus(mu)
                link = Uflat[here, mu]                                   # U_mu(n)[A, B]
            else:
                spin = projector_plus(mu)
                link = np.conj(np.swapaxes(Uflat[there, mu], -1, -2))  # U_mu(n - mu)^dagger[A, B]
            for alpha in range(4):
                for beta in range(4):
                    if spin[alpha, beta] == 0:
                        continue
                    for A in range(3):
                        for B in range(3):
                            rows.append(12 * here + 3 * alpha + A)
                            cols.append(12 * there + 3 * beta + B)
                            vals.append(-kappa * phase * spin[alpha, beta] * link[:, A, B])
    return np.concatenate(rows), np.concatenate(cols), np.concatenate(vals)


def coo_spmv(row, col, val, vec):
    """The paper's COO product (Sec. 2): out[Row[k]] += Val[k] * in[Col[k]] for every k.

    ``np.add.at`` is unbuffered, so repeated Row entries accumulate exactly as the loop does.
    """
    out = np.zeros(vec.shape[0], dtype=np.result_type(val, vec))
    np.add.at(out, row, val * vec[col])
    return out


def dense_D(U, kappa: float, boundary=DEFAULT_BOUNDARY):
    """R3: D as a dense (12V x 12V) matrix, summed from the COO entries. For V <= 4^4 only."""
    row, col, val = assemble_coo(U, kappa, boundary)
    n = 12 * int(np.prod(U.shape[:4]))
    dense = np.zeros((n, n), dtype=np.complex128)
    np.add.at(dense, (row, col), val)
    return dense


def apply_gamma5(psi):
    """gamma_5 acting on the spin index of a spinor field."""
    return np.einsum("st,...tc->...sc", GAMMA5, psi)


def gamma_matrices():
    return GAMMA


def norm2(v) -> float:
    """Squared 2-norm of a complex field, in FP64."""
    v = np.asarray(v)
    return float(np.vdot(v.reshape(-1), v.reshape(-1)).real)


def rel_diff(a, b) -> float:
    """||a - b|| / ||b|| over the whole field."""
    nb = np.sqrt(norm2(b))
    return float(np.sqrt(norm2(np.asarray(a) - np.asarray(b))) / (nb if nb > 0 else 1.0))
