"""The paper's COO representation and SpMV (Sec. 2) on the GPU, against the oracle's COO and D."""
import numpy as np
import pytest
import torch

from oracle import wilson
from tests.gpu_util import fields, rel, require_gpu, to_dev, to_np

pytestmark = pytest.mark.gpu

BC = (1, 1, 1, -1)


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4), (2, 3, 4, 6)])
def test_coo_spmv_matches_oracle(dims):
    wd = require_gpu()
    U, psi = fields(dims)
    op = wd.WilsonDirac(dims, 0.12, BC, wd.WD_PREC_F64)
    Ud = to_dev(U)
    row, col, val = wd.wd_coo_build(op.ctx, Ud)
    V = int(np.prod(dims))
    assert row.numel() == 49 * 12 * V
    counts = torch.bincount(row.long(), minlength=12 * V)
    assert int(counts.min()) == 49 and int(counts.max()) == 49
    out = torch.empty_like(to_dev(psi))
    wd.wd_coo_spmv(op.ctx, row, col, val, to_dev(psi), out)
    assert rel(to_np(out), wilson.apply_D(U, psi, 0.12, BC)) < 1e-13
    # the same matrix as the oracle's COO assembly, entry by entry once both are summed densely
    if V <= 16:
        r, c, v = wilson.assemble_coo(U, 0.12, BC)
        dense_ref = np.zeros((12 * V, 12 * V), complex)
        np.add.at(dense_ref, (r, c), v)
        dense = np.zeros_like(dense_ref)
        np.add.at(dense, (row.cpu().numpy(), col.cpu().numpy()), to_np(val))
        assert np.abs(dense - dense_ref).max() < 1e-15
    op.close()
