"""The FP32 dslash with TMA-staged neighbour spinors (WD_OPT_DSLASH_TMA) against the oracle.

The staged kernel reads every neighbour from shared memory filled by bulk tensor copies (tile, and
six face slabs taken across the periodic boundary), so it must give exactly the per-thread-load
kernel's result (same arithmetic per site) and agree with the FP64 oracle of Eq. (1) within the FP32
bound on the same rounded input. Lattices span one and several tiles per direction, L = 2 extents
and every boundary pattern.
"""
import numpy as np
import pytest
import torch

import synthetic
from oracle import wilson
from tests.gpu_util import require_gpu, to_dev

pytestmark = pytest.mark.gpu

CASES = [((8, 4, 4, 6), 1), ((8, 4, 4, 6), 2), ((16, 2, 4, 2), 1), ((4, 4, 4, 4), 1), ((4, 4, 4, 4), 2),
         ((32, 4, 2, 4), 1), ((32, 4, 2, 4), 2), ((12, 8, 6, 4), 2), ((16, 16, 16, 16), 2)]


@pytest.mark.parametrize("dims,tile", CASES)
@pytest.mark.parametrize("bc", [(1, 1, 1, -1), (-1, 1, -1, -1)])
def test_tma_dslash_matches_oracle_and_the_load_kernel(dims, tile, bc):
    wd = require_gpu()
    U = synthetic.gauge_field(dims, 0.4, 1)
    psi = synthetic.gaussian_source(dims, 2).astype(np.complex64)
    op = wd.WilsonDirac(dims, 0.124, bc, wd.WD_PREC_F32)
    op.load_gauge(to_dev(U), compress12=True)
    for dagger in (False, True):
        plain = op.apply(to_dev(psi, dtype=torch.complex64), dagger=dagger).cpu().numpy()
        op.set_option(wd.WD_OPT_DSLASH_TMA, tile)
        staged = op.apply(to_dev(psi, dtype=torch.complex64), dagger=dagger).cpu().numpy()
        op.set_option(wd.WD_OPT_DSLASH_TMA, 0)
        assert np.array_equal(staged, plain), (dims, tile, dagger)
        ref = wilson.apply_D(U, psi.astype(np.complex128), 0.124, bc, dagger=dagger)
        assert wilson.rel_diff(staged.astype(np.complex128), ref) < 1e-6
    op.close()


def test_tma_timing_and_option_checks():
    wd = require_gpu()
    dims = (16, 8, 8, 8)
    op = wd.WilsonDirac(dims, 0.12, (1, 1, 1, -1), wd.WD_PREC_F32)
    op.generate_gauge(0.4, 1, compress12=True)
    op.set_option(wd.WD_OPT_DSLASH_TMA, 1)
    assert op.time_dslash(False, 5) > 0
    op.close()
    bad = wd.WilsonDirac((6, 4, 4, 4), 0.12, (1, 1, 1, -1), wd.WD_PREC_F32)   # Lx not a multiple of 4
    with pytest.raises(wd.WdError) as e:
        bad.set_option(wd.WD_OPT_DSLASH_TMA, 1)
    assert e.value.status == wd.WD_EINVAL
    bad.close()
    f64 = wd.WilsonDirac((8, 4, 4, 4), 0.12, (1, 1, 1, -1), wd.WD_PREC_F64)
    with pytest.raises(wd.WdError):
        f64.set_option(wd.WD_OPT_DSLASH_TMA, 1)
    f64.close()
