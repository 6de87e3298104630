"""The mixed-precision solvers' inner operators against the oracle, element by element.

Reliable updates make a mixed solve converge to the FP64 answer even with a poor inner operator
(a wrong inner dslash costs iterations, not accuracy), so the solve tests cannot vouch for the FP32
and FP16+norm kernels. Here ``WD_OPT_APPLY_INNER`` makes ``wd_apply`` / ``wd_apply_multi`` run the
inner operator of Eq. (1) itself, and the result is compared with ``oracle.wilson.apply_D`` applied
to the same quantised input:

* FP32 (FP32 links, 18 or 12 reals): the input is rounded to complex64 first, so both sides see
  the same numbers; the bound is the FP32 tolerance, 1e-6 relative over the field.
* FP16 spinors with a per-site FP32 norm: the input is built exactly representable (per site a
  power-of-two norm 2^k and components j * 2^(k-10), |j| <= 1024, one of them +-2^k), so the only
  rounding is the output's: per element at most 2^-12 of the site's norm, hence per site at most
  sqrt(24) * 2^-12 relative (plus FP32 arithmetic, ~1e-6), and over the field the test asks for
  2^-11. A Gaussian input (rounded on the way in too) must stay within 2^-9.
"""
import numpy as np
import pytest
import torch

import synthetic
from oracle import wilson
from tests.gpu_util import require_gpu, to_dev

pytestmark = pytest.mark.gpu

BC = (1, 1, 1, -1)
SITE_BOUND_F16 = np.sqrt(24.0) * 2.0 ** -12 + 5e-6


def _exact_f16_field(dims, seed, nrhs=None):
    """A spinor field (or nrhs of them) that FP16 storage with a power-of-two per-site norm holds
    exactly."""
    rng = np.random.default_rng(seed)
    lx, ly, lz, lt = dims
    shape = ((nrhs,) if nrhs else ()) + (lt, lz, ly, lx)
    k = rng.integers(-3, 4, size=shape).astype(np.float64)
    j = rng.integers(-1024, 1025, size=shape + (4, 3, 2)).astype(np.float64)
    # one component per site carries the site's maximum, +-2^k
    j[..., 0, 0, 0] = np.where(rng.random(shape) < 0.5, -1024.0, 1024.0)
    v = j * np.exp2(k - 10.0)[..., None, None, None]
    return (v[..., 0] + 1j * v[..., 1]).astype(np.complex128)


def _per_site_rel(got, ref):
    g = got.reshape(-1, 12)
    r = ref.reshape(-1, 12)
    return np.linalg.norm(g - r, axis=1) / np.maximum(np.linalg.norm(r, axis=1), 1e-300)


def _op(wd, dims, prec, kappa, c12, U):
    op = wd.WilsonDirac(dims, kappa, BC, prec)
    op.load_gauge(to_dev(U), compress12=c12)
    op.set_option(wd.WD_OPT_APPLY_INNER, 1)
    return op


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 5, 4, 7), (16, 16, 16, 16)])
@pytest.mark.parametrize("c12", [False, True])
def test_fp32_inner_operator_matches_oracle(dims, c12):
    wd = require_gpu()
    U = synthetic.gauge_field(dims, 0.4, 1)
    psi = synthetic.gaussian_source(dims, 2).astype(np.complex64).astype(np.complex128)
    op = _op(wd, dims, wd.WD_PREC_MIXED_F32, 0.124, c12, U)
    for dagger in (False, True):
        got = op.apply(to_dev(psi), dagger=dagger).cpu().numpy()
        ref = wilson.apply_D(U, psi, 0.124, BC, dagger=dagger)
        assert wilson.rel_diff(got, ref) < 1e-6, (dims, c12, dagger)
    # switching the option off returns to the FP64 operator
    op.set_option(wd.WD_OPT_APPLY_INNER, 0)
    got = op.apply(to_dev(psi)).cpu().numpy()
    assert wilson.rel_diff(got, wilson.apply_D(U, psi, 0.124, BC)) < 1e-13
    op.close()


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 5, 4, 7), (16, 16, 16, 16)])
def test_fp16_inner_operator_matches_oracle_on_exact_input(dims):
    wd = require_gpu()
    U = synthetic.gauge_field(dims, 0.4, 1)
    psi = _exact_f16_field(dims, 3)
    op = _op(wd, dims, wd.WD_PREC_MIXED_F16, 0.124, True, U)
    for dagger in (False, True):
        got = op.apply(to_dev(psi), dagger=dagger).cpu().numpy()
        ref = wilson.apply_D(U, psi, 0.124, BC, dagger=dagger)
        site = _per_site_rel(got, ref)
        assert site.max() <= SITE_BOUND_F16, (dims, dagger, site.max())
        assert wilson.rel_diff(got, ref) <= 2.0 ** -11, (dims, dagger)
        # the FP16 result really is rounded (not an FP32 operator in disguise)
        assert wilson.rel_diff(got, ref) > 1e-6
    op.close()


def test_fp16_inner_operator_on_gaussian_input():
    wd = require_gpu()
    dims = (8, 6, 4, 6)
    U = synthetic.gauge_field(dims, 0.4, 1)
    psi = synthetic.gaussian_source(dims, 2)
    op = _op(wd, dims, wd.WD_PREC_MIXED_F16, 0.12, True, U)
    for dagger in (False, True):
        got = op.apply(to_dev(psi), dagger=dagger).cpu().numpy()
        ref = wilson.apply_D(U, psi, 0.12, BC, dagger=dagger)
        assert wilson.rel_diff(got, ref) <= 2.0 ** -9, dagger
    op.close()


@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_inner_operator_of_even_odd_contexts(prec):
    wd = require_gpu()
    dims = (6, 4, 4, 8)
    U = synthetic.gauge_field(dims, 0.4, 1)
    base = wd.WD_PREC_MIXED_F32 if prec == "f32" else wd.WD_PREC_MIXED_F16
    if prec == "f32":
        psi = synthetic.gaussian_source(dims, 2).astype(np.complex64).astype(np.complex128)
    else:
        psi = _exact_f16_field(dims, 4)
    op = _op(wd, dims, base | wd.WD_EVEN_ODD, 0.12, True, U)
    for dagger in (False, True):
        got = op.apply(to_dev(psi), dagger=dagger).cpu().numpy()
        ref = wilson.apply_D(U, psi, 0.12, BC, dagger=dagger)
        if prec == "f32":
            assert wilson.rel_diff(got, ref) < 1e-6
        else:
            assert _per_site_rel(got, ref).max() <= SITE_BOUND_F16
            assert wilson.rel_diff(got, ref) <= 2.0 ** -11
    op.close()


@pytest.mark.parametrize("prec", ["f32", "f16"])
@pytest.mark.parametrize("nrhs", [3, 12])
def test_multi_rhs_inner_operator_matches_oracle(prec, nrhs):
    wd = require_gpu()
    dims = (6, 5, 4, 8)
    U = synthetic.gauge_field(dims, 0.4, 1)
    if prec == "f32":
        base = wd.WD_PREC_MIXED_F32
        psi = np.stack([synthetic.gaussian_source(dims, 10 + r) for r in range(nrhs)])
        psi = psi.astype(np.complex64).astype(np.complex128)
    else:
        base = wd.WD_PREC_MIXED_F16
        psi = _exact_f16_field(dims, 5, nrhs=nrhs)
    op = _op(wd, dims, base, 0.124, True, U)
    for dagger in (False, True):
        got = op.apply_multi(torch.from_numpy(psi).cuda(), dagger=dagger).cpu().numpy()
        for r in range(nrhs):
            ref = wilson.apply_D(U, psi[r], 0.124, BC, dagger=dagger)
            if prec == "f32":
                assert wilson.rel_diff(got[r], ref) < 1e-6, (r, dagger)
            else:
                assert _per_site_rel(got[r], ref).max() <= SITE_BOUND_F16, (r, dagger)
                assert wilson.rel_diff(got[r], ref) <= 2.0 ** -11, (r, dagger)
    op.close()


def test_apply_inner_rejected_outside_mixed_precision():
    wd = require_gpu()
    op = wd.WilsonDirac((4, 4, 4, 4), 0.12, BC, wd.WD_PREC_F64)
    with pytest.raises(wd.WdError) as e:
        op.set_option(wd.WD_OPT_APPLY_INNER, 1)
    assert e.value.status == wd.WD_EINVAL
    op.close()
