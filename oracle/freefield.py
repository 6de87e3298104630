"""Closed forms of the Wilson-Dirac operator with unit links (test infrastructure only).

With U = 1 the operator of Eq. (1) is diagonal in momentum space. A plane wave
psi(n) = exp(i p.n) chi with p_mu = (2 pi k_mu + theta_mu) / L_mu, theta_mu = 0 for a periodic
and pi for an antiperiodic direction, obeys psi(n + mu) = exp(i p_mu) psi(n) including the
boundary phase, so

    D(p) = 1 - 2 kappa sum_mu cos p_mu + 2 i kappa sum_mu gamma_mu sin p_mu,

and, by the Clifford algebra, D(p)^dagger D(p) = (1 - 2 kappa sum cos p)^2 + 4 kappa^2 sum sin^2 p,
times the identity in spin (and colour): every momentum contributes that value 12 times to the
spectrum of D^dagger D. These derive from Eq. (1) and the gamma algebra, not from the stencil code,
so they pin the stencil, the COO assembly and the dense matrix independently.
"""
from __future__ import annotations

import numpy as np

from .gamma import GAMMA, IDENTITY4


def momenta(dims, boundary):
    """Per-direction momentum arrays p_mu (length L_mu), mu = 0..3 = x, y, z, t."""
    out = []
    for L, b in zip(dims, boundary):
        theta = np.pi if b == -1 else 0.0
        out.append((2 * np.pi * np.arange(L) + theta) / L)
    return out


def symbol(p, kappa):
    """D(p) as a 4x4 spin matrix for one momentum p = (p_x, p_y, p_z, p_t)."""
    m = (1 - 2 * kappa * sum(np.cos(pm) for pm in p)) * IDENTITY4
    for mu in range(4):
        m = m + 2j * kappa * np.sin(p[mu]) * GAMMA[mu]
    return m


def DdagD_eigenvalues(dims, kappa, boundary):
    """Sorted spectrum of D^dagger D for unit links (12V values, each momentum 12 times)."""
    px, py, pz, pt = momenta(dims, boundary)
    PT, PZ, PY, PX = np.meshgrid(pt, pz, py, px, indexing="ij")
    cos_sum = np.cos(PX) + np.cos(PY) + np.cos(PZ) + np.cos(PT)
    sin2_sum = np.sin(PX) ** 2 + np.sin(PY) ** 2 + np.sin(PZ) ** 2 + np.sin(PT) ** 2
    lam = (1 - 2 * kappa * cos_sum) ** 2 + 4 * kappa ** 2 * sin2_sum
    return np.sort(np.repeat(lam.reshape(-1), 12))


def plane_wave(dims, k, chi, boundary):
    """psi(n) = exp(i p.n) chi for integer wave numbers k = (kx, ky, kz, kt); chi is [4, 3]."""
    lx, ly, lz, lt = dims
    p = [m[ki] for m, ki in zip(momenta(dims, boundary), k)]
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx),
                             indexing="ij")
    phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    return phase[..., None, None] * chi[None, None, None, None], p


def solve(eta, kappa, boundary):
    """x = D^{-1} eta for unit links, exactly (FFT to momentum space, invert D(p), back).

    D(p)^{-1} = (a - i b.gamma) / (a^2 + |b|^2) with a = 1 - 2 kappa sum cos p,
    b_mu = 2 kappa sin p_mu. Antiperiodic directions are handled by twisting the field with
    exp(-i theta n / L) before a standard FFT.
    """
    lt, lz, ly, lx = eta.shape[:4]
    dims = (lx, ly, lz, lt)
    px, py, pz, pt = momenta(dims, boundary)
    thetas = [(np.pi if b == -1 else 0.0) for b in boundary]
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx),
                             indexing="ij")
    twist = np.exp(1j * (thetas[0] * x / lx + thetas[1] * y / ly + thetas[2] * z / lz
                         + thetas[3] * t / lt))
    eta_k = np.fft.fftn(np.conj(twist)[..., None, None] * eta, axes=(0, 1, 2, 3))
    PT, PZ, PY, PX = np.meshgrid(pt, pz, py, px, indexing="ij")
    P = (PX, PY, PZ, PT)
    a = 1 - 2 * kappa * (np.cos(PX) + np.cos(PY) + np.cos(PZ) + np.cos(PT))
    b = [2 * kappa * np.sin(Pm) for Pm in P]
    den = a ** 2 + sum(bm ** 2 for bm in b)
    inv = a[..., None, None] * IDENTITY4
    for mu in range(4):
        inv = inv - 1j * b[mu][..., None, None] * GAMMA[mu]
    inv = inv / den[..., None, None]
    psi_k = np.einsum("...st,...tc->...sc", inv, eta_k)
    psi = np.fft.ifftn(psi_k, axes=(0, 1, 2, 3))
    return twist[..., None, None] * psi
