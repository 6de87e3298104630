"""Device-side seeded generators against the CPU implementation of the same counter-based streams."""
import numpy as np
import pytest
import torch

import synthetic
from oracle import wilson
from tests.gpu_util import rel, require_gpu, to_dev, to_np

pytestmark = pytest.mark.gpu

BC = (1, 1, 1, -1)


@pytest.mark.parametrize("dims,eps,seed", [((4, 4, 4, 4), 0.4, 1), ((6, 2, 4, 5), 0.3, 12345678901),
                                           ((8, 8, 8, 8), 0.5, 2**63 + 17)])
def test_gauge_generator_matches_cpu_stream(dims, eps, seed):
    wd = require_gpu()
    op = wd.WilsonDirac(dims, 0.12, BC, wd.WD_PREC_F64)
    U = to_np(op.generate_gauge(eps, seed, return_field=True))
    ref = synthetic.gauge_field_philox(dims, eps, seed)
    assert np.abs(U - ref).max() < 1e-13
    dev = np.abs(np.conj(np.swapaxes(U, -1, -2)) @ U - np.eye(3)).max()
    assert dev < 1e-14 and np.abs(np.linalg.det(U) - 1).max() < 1e-14
    op.close()


def test_source_generator_matches_cpu_stream():
    wd = require_gpu()
    dims = (6, 4, 4, 8)
    op = wd.WilsonDirac(dims, 0.12, BC, wd.WD_PREC_F64)
    src = to_np(op.generate_source(99))
    assert np.abs(src - synthetic.gaussian_source_philox(dims, 99)).max() < 1e-13
    op.close()


@pytest.mark.parametrize("prec,c12,tol", [("f64", False, 1e-13), ("f32", True, 1e-6)])
def test_generated_field_in_the_operator(prec, c12, tol):
    wd = require_gpu()
    dims = (4, 6, 4, 4)
    p = wd.WD_PREC_F64 if prec == "f64" else wd.WD_PREC_F32
    op = wd.WilsonDirac(dims, 0.12, BC, p)
    op.generate_gauge(0.4, 5, compress12=c12)
    U = synthetic.gauge_field_philox(dims, 0.4, 5)
    psi = synthetic.gaussian_source_philox(dims, 6)
    dt = torch.complex128 if prec == "f64" else torch.complex64
    out = to_np(op.apply(to_dev(psi, dt)))
    src = psi if prec == "f64" else psi.astype(np.complex64).astype(np.complex128)
    assert rel(out, wilson.apply_D(U, src, 0.12, BC)) < tol
    op.close()
