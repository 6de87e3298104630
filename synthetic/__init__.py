"""Seeded synthetic inputs for the Wilson-Dirac solver: gauge links, sources, gauge transforms.

This module only draws inputs. It holds none of the operator or solver arithmetic, so both the
CPU oracle and the CUDA path can take their inputs from it without sharing any of the method.

Conventions (the paper fixes none of them; they are this library's stated readings):

* Lattice ``dims = (Lx, Ly, Lz, Lt)``; arrays are indexed ``[t, z, y, x, ...]`` so the site index
  ``x + Lx*(y + Ly*(z + Lz*t))`` runs with x fastest.
* Gauge field: complex128 ``[Lt, Lz, Ly, Lx, 4, 3, 3]``; ``U[t,z,y,x,mu]`` is the link from site n
  to n + mu-hat (mu = 0,1,2,3 = x,y,z,t), stored row-major (row = colour index a, column = b).
* Spinor field: complex128 ``[Lt, Lz, Ly, Lx, 4, 3]`` (spin, colour).
* Gauge links: U = exp(i*eps*H) with H the traceless Hermitian part of a matrix M whose real and
  imaginary entries are i.i.d. N(0, 1); all real parts of the whole field are drawn first, then
  all imaginary parts, each in C order of the array above. The links are then re-unitarised to
  SU(3) in FP64 (Gram-Schmidt on rows 0 and 1, row 2 = conj(row0 x row1), so det U = 1).
* Gaussian source: real and imaginary parts i.i.d. N(0, 1) per component (real parts first).

Counter-based variants (``gauge_field_philox``, ``gaussian_source_philox``) draw the same kind of
fields from Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC11) so that a GPU can generate them
independently and bit-for-bit in its random numbers: key = the 64-bit seed, counter = (object
index low 32 bits, high 32 bits, stream, block), uniforms (x + 1/2) 2^-32, Gaussians by
Box-Muller (r = sqrt(-2 ln u1); r cos 2 pi u2, r sin 2 pi u2). A link (object index 4 n + mu,
stream 0) takes 18 Gaussians: Re of its 9 entries of M (row-major), then Im; a source site
(object index n, stream 1) takes 24: Re of its 12 components, then Im.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "philox4x32_10",
    "gauge_field_philox",
    "gaussian_source_philox",
    "volume",
    "gauge_field",
    "unit_gauge",
    "gaussian_source",
    "point_source",
    "random_su3",
    "random_gauge_transform",
]


def volume(dims) -> int:
    lx, ly, lz, lt = (int(d) for d in dims)
    return lx * ly * lz * lt


def _shape(dims):
    lx, ly, lz, lt = (int(d) for d in dims)
    return (lt, lz, ly, lx)


def _dagger(m):
    return np.conj(np.swapaxes(m, -1, -2))


def _reunitarise(u):
    """Project near-unitary 3x3 matrices onto SU(3): Gram-Schmidt rows 0, 1; row 2 from them."""
    r0 = u[..., 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=-1, keepdims=True)
    r1 = u[..., 1, :]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=-2)


def _su3_from_normal(re, im, eps):
    m = re + 1j * im
    h = 0.5 * (m + _dagger(m))
    tr = np.trace(h, axis1=-2, axis2=-1).real / 3.0
    h = h - tr[..., None, None] * np.eye(3)
    w, v = np.linalg.eigh(h)
    u = (v * np.exp(1j * eps * w)[..., None, :]) @ _dagger(v)
    return _reunitarise(u)


def gauge_field(dims, eps: float, seed: int, chunk: int = 1 << 20) -> np.ndarray:
    """Random SU(3) gauge field U = exp(i*eps*H), complex128 [Lt,Lz,Ly,Lx,4,3,3]."""
    shape = _shape(dims) + (4, 3, 3)
    rng = np.random.default_rng(seed)
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    re = re.reshape(-1, 3, 3)
    im = im.reshape(-1, 3, 3)
    out = np.empty(re.shape, dtype=np.complex128)
    for s in range(0, re.shape[0], chunk):
        out[s:s + chunk] = _su3_from_normal(re[s:s + chunk], im[s:s + chunk], eps)
    return out.reshape(shape)


def unit_gauge(dims) -> np.ndarray:
    """Free field: every link is the 3x3 identity."""
    shape = _shape(dims) + (4, 3, 3)
    out = np.zeros(shape, dtype=np.complex128)
    out[..., :, :] = np.eye(3)
    return out


def gaussian_source(dims, seed: int) -> np.ndarray:
    """Complex Gaussian spinor field, Re and Im i.i.d. N(0, 1), complex128 [Lt,Lz,Ly,Lx,4,3]."""
    shape = _shape(dims) + (4, 3)
    rng = np.random.default_rng(seed)
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return re + 1j * im


def point_source(dims, spin: int, colour: int, site=(0, 0, 0, 0)) -> np.ndarray:
    """Unit point source at site (x, y, z, t) in one spin-colour component."""
    shape = _shape(dims) + (4, 3)
    out = np.zeros(shape, dtype=np.complex128)
    x, y, z, t = site
    out[t, z, y, x, spin, colour] = 1.0
    return out


def random_su3(n: int, seed: int, eps: float = 1.0) -> np.ndarray:
    """n independent random SU(3) matrices (same recipe as the gauge links)."""
    rng = np.random.default_rng(seed)
    re = rng.standard_normal((n, 3, 3))
    im = rng.standard_normal((n, 3, 3))
    return _su3_from_normal(re, im, eps)


def random_gauge_transform(dims, seed: int) -> np.ndarray:
    """One SU(3) matrix per site, complex128 [Lt,Lz,Ly,Lx,3,3]."""
    return random_su3(volume(dims), seed, eps=2.0).reshape(_shape(dims) + (3, 3))


# ---------------------------------------------------------------------------- counter-based

_PHILOX_M0, _PHILOX_M1 = 0xD2511F53, 0xCD9E8D57
_PHILOX_W0, _PHILOX_W1 = 0x9E3779B9, 0xBB67AE85
_MASK32 = 0xFFFFFFFF


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds on arrays of 32-bit counters; returns four uint64 arrays < 2^32."""
    c = [np.asarray(v, dtype=np.uint64) & _MASK32 for v in (c0, c1, c2, c3)]
    k0 = np.uint64(int(k0) & _MASK32)
    k1 = np.uint64(int(k1) & _MASK32)
    m0, m1 = np.uint64(_PHILOX_M0), np.uint64(_PHILOX_M1)
    mask = np.uint64(_MASK32)
    for r in range(10):
        if r > 0:
            k0 = np.uint64((int(k0) + _PHILOX_W0) & _MASK32)
            k1 = np.uint64((int(k1) + _PHILOX_W1) & _MASK32)
        p0 = m0 * c[0]          # < 2^64: exact in uint64
        p1 = m1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & mask
        hi1, lo1 = p1 >> np.uint64(32), p1 & mask
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return c


def gauge_field_philox(dims, eps: float, seed: int, chunk: int = 1 << 20) -> np.ndarray:
    """SU(3) field U = exp(i eps H) from the counter-based stream (same recipe as gauge_field)."""
    shape = _shape(dims) + (4, 3, 3)
    n = volume(dims) * 4
    out = np.empty((n, 3, 3), dtype=np.complex128)
    for s in range(0, n, chunk):
        m = min(chunk, n - s)
        g = _philox_gaussians_range(s, m, 18, 0, seed)
        out[s:s + m] = _su3_from_normal(g[:, :9].reshape(m, 3, 3), g[:, 9:].reshape(m, 3, 3), eps)
    return out.reshape(shape)


def _philox_gaussians_range(start, count, n_gauss, stream, seed):
    g = _philox_gaussians_from(np.arange(start, start + count, dtype=np.uint64), n_gauss, stream, seed)
    return g


def _philox_gaussians_from(idx, n_gauss, stream, seed):
    lo = idx & np.uint64(_MASK32)
    hi = idx >> np.uint64(32)
    seed = int(seed)
    k0, k1 = seed & _MASK32, (seed >> 32) & _MASK32
    n = idx.shape[0]
    blocks = []
    for j in range((n_gauss + 3) // 4):
        blocks.extend(philox4x32_10(lo, hi, np.full(n, stream, np.uint64), np.full(n, j, np.uint64), k0, k1))
    u = (np.stack(blocks[:n_gauss], axis=1).astype(np.float64) + 0.5) * (1.0 / 4294967296.0)
    r = np.sqrt(-2.0 * np.log(u[:, 0::2]))
    ang = 2.0 * np.pi * u[:, 1::2]
    g = np.empty((n, n_gauss))
    g[:, 0::2] = r * np.cos(ang)
    g[:, 1::2] = r * np.sin(ang)
    return g


def gaussian_source_philox(dims, seed: int) -> np.ndarray:
    """Complex Gaussian spinor field from the counter-based stream, complex128 [Lt,Lz,Ly,Lx,4,3]."""
    n = volume(dims)
    g = _philox_gaussians_from(np.arange(n, dtype=np.uint64), 24, 1, seed)
    return (g[:, :12] + 1j * g[:, 12:]).reshape(_shape(dims) + (4, 3))
