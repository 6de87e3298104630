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
"""
from __future__ import annotations

import numpy as np

__all__ = [
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
