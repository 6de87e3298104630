"""Euclidean Dirac matrices in the chiral basis (test infrastructure only).

Eq. (1) of the paper carries spin indices alpha, beta in {0,1,2,3} but prints no gamma basis.
This oracle takes the chiral basis (the library's stated reading):

    gamma_k = [[0, -i sigma_k], [i sigma_k, 0]]   for k = 1, 2, 3  (mu = 0, 1, 2 = x, y, z)
    gamma_4 = [[0, 1], [1, 0]]                                      (mu = 3 = t)
    gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 = diag(1, 1, -1, -1)

written with 2x2 blocks in spin space. All four are Hermitian and obey
{gamma_mu, gamma_nu} = 2 delta_mu_nu; the tests check this, gamma_5's form, and the
gamma_5-hermiticity gamma_5 D gamma_5 = D^dagger that Sec. 2 relies on.
"""
from __future__ import annotations

import numpy as np

SIGMA = (
    np.array([[0, 1], [1, 0]], dtype=np.complex128),
    np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    np.array([[1, 0], [0, -1]], dtype=np.complex128),
)

_Z2 = np.zeros((2, 2), dtype=np.complex128)
_I2 = np.eye(2, dtype=np.complex128)


def _block(a, b, c, d):
    return np.block([[a, b], [c, d]])


GAMMA = tuple(
    [_block(_Z2, -1j * s, 1j * s, _Z2) for s in SIGMA] + [_block(_Z2, _I2, _I2, _Z2)]
)
"""gamma_mu for mu = 0, 1, 2, 3 (x, y, z, t); each a 4x4 complex128 matrix."""

GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]

IDENTITY4 = np.eye(4, dtype=np.complex128)


def projector_minus(mu: int) -> np.ndarray:
    """(1 - gamma_mu): the spin factor of the forward hop n -> n + mu in D (Eq. (1), Wilson r = 1)."""
    return IDENTITY4 - GAMMA[mu]


def projector_plus(mu: int) -> np.ndarray:
    """(1 + gamma_mu): the spin factor of the backward hop n -> n - mu in D."""
    return IDENTITY4 + GAMMA[mu]
