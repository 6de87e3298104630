"""Batched solves (cg_solve_batch, and the serving runtime's batches) against solves alone and the oracle.

A batch runs each problem's persistent CG loop on its own blocks of one shared cooperative launch,
with the grid, fields and scalars of its solve alone, so every result must equal the solve alone bit
for bit; the true residual of each is recomputed by the oracle in FP64 (Eq. (1)). Shapes the
persistent loop does not serve, or mixed shapes, are solved one after another by the same call.
"""
import numpy as np
import pytest
import torch

import synthetic
from oracle import cg as ocg
from tests.gpu_util import require_gpu, to_np

pytestmark = pytest.mark.gpu

BC = (1, 1, 1, -1)


def _problems(wd, dims, prec, n, tols=(1e-10,), c12=True):
    ops, srcs, fields = [], [], []
    for i in range(n):
        kappa = (0.115, 0.12, 0.124)[i % 3]
        op = wd.WilsonDirac(dims, kappa, BC, prec)
        eps = 0.3 + 0.05 * (i % 4)
        op.generate_gauge(eps, 300 + i, compress12=c12 and prec != wd.WD_PREC_F64)
        srcs.append(op.generate_source(400 + i))
        ops.append(op)
        fields.append((eps, 300 + i, 400 + i, kappa, tols[i % len(tols)]))
    return ops, srcs, fields


def _alone(wd, dims, prec, f, c12=True):
    eps, gs, ss, kappa, tol = f
    op = wd.WilsonDirac(dims, kappa, BC, prec)
    op.generate_gauge(eps, gs, compress12=c12 and prec != wd.WD_PREC_F64)
    src = op.generate_source(ss)
    x = torch.zeros_like(src)
    st, it, res = wd.cg_solve(op.ctx, src, x, tol, 20000)
    op.close()
    return st, it, res, to_np(x)


CASES = [((8, 8, 8, 8), "mixed_f32"), ((8, 8, 8, 8), "mixed_f16"), ((12, 12, 12, 12), "mixed_f32"),
         ((4, 4, 4, 4), "f64"), ((8, 8, 8, 8), "f64"), ((6, 6, 6, 6), "f32")]


@pytest.mark.parametrize("dims,prec", CASES)
def test_batch_equals_solves_alone_bitwise(dims, prec):
    wd = require_gpu()
    p = {"mixed_f32": wd.WD_PREC_MIXED_F32, "mixed_f16": wd.WD_PREC_MIXED_F16, "f64": wd.WD_PREC_F64,
         "f32": wd.WD_PREC_F32}[prec]
    tols = (1e-6,) if prec == "f32" else (1e-10, 1e-8)
    n = 5
    ops, srcs, fields = _problems(wd, dims, p, n, tols)
    xs = [torch.zeros_like(s) for s in srcs]
    st, iters, res, sts = wd.cg_solve_batch([o.ctx for o in ops], srcs, xs, [f[4] for f in fields], 20000)
    loop_modes = [o.stats()["loop_mode"] for o in ops]
    for o in ops:
        o.close()
    assert st == wd.WD_OK and all(s == wd.WD_OK for s in sts)
    assert all(m == 2 for m in loop_modes)          # the persistent loop, shared
    for i, f in enumerate(fields):
        sa, ia, ra, xa = _alone(wd, dims, p, f)
        assert sa == wd.WD_OK
        assert ia == iters[i] and ra == res[i], (i, ia, iters[i], ra, res[i])
        assert np.array_equal(to_np(xs[i]), xa), i
    # the oracle's residual of one problem of each tolerance
    for i in (0, 1):
        eps, gs, ss, kappa, tol = fields[i]
        U = synthetic.gauge_field_philox(dims, eps, gs)
        eta = synthetic.gaussian_source_philox(dims, ss)
        assert ocg.true_residual(U, eta, to_np(xs[i]), kappa) <= tol * 1.01


def test_batch_of_unbatchable_or_mixed_shapes_runs_one_after_another():
    wd = require_gpu()
    a_ops, a_src, a_f = _problems(wd, (16, 16, 16, 16), wd.WD_PREC_MIXED_F32, 2)   # graph path
    b_ops, b_src, b_f = _problems(wd, (4, 4, 4, 6), wd.WD_PREC_F64, 1)
    ops, srcs, fields = a_ops + b_ops, a_src + b_src, a_f + b_f
    xs = [torch.zeros_like(s) for s in srcs]
    st, iters, res, sts = wd.cg_solve_batch([o.ctx for o in ops], srcs, xs, [f[4] for f in fields], 20000)
    for o in ops:
        o.close()
    assert st == wd.WD_OK
    for i, (dims, p) in enumerate([((16, 16, 16, 16), wd.WD_PREC_MIXED_F32)] * 2 + [((4, 4, 4, 6), wd.WD_PREC_F64)]):
        sa, ia, ra, xa = _alone(wd, dims, p, fields[i])
        assert ia == iters[i] and ra == res[i] and np.array_equal(to_np(xs[i]), xa), i


def test_batch_statuses_and_errors():
    wd = require_gpu()
    dims = (6, 4, 4, 8)
    ops, srcs, fields = _problems(wd, dims, wd.WD_PREC_MIXED_F32, 3)
    srcs[1] = srcs[1].clone()
    srcs[1][0, 0, 0, 0, 0, 0] = float("nan")       # one problem breaks down, the others solve
    xs = [torch.zeros_like(s) for s in srcs]
    st, iters, res, sts = wd.cg_solve_batch([o.ctx for o in ops], srcs, xs, [1e-10] * 3, 20000)
    assert st == wd.WD_BREAKDOWN
    assert sts[0] == wd.WD_OK and sts[1] == wd.WD_BREAKDOWN and sts[2] == wd.WD_OK
    # maxit reached by every problem
    x2 = [torch.zeros_like(srcs[0]), torch.zeros_like(srcs[2])]   # from zero, not the solutions above
    st, iters, res, sts = wd.cg_solve_batch([ops[0].ctx, ops[2].ctx], [srcs[0], srcs[2]], x2, [1e-10] * 2, 3)
    assert st == wd.WD_NOT_CONVERGED and all(s == wd.WD_NOT_CONVERGED for s in sts) and all(i == 3 for i in iters)
    with pytest.raises(wd.WdError) as e:
        wd.cg_solve_batch([ops[0].ctx, ops[0].ctx], srcs[:2], xs[:2], [1e-10] * 2, 100)
    assert e.value.status == wd.WD_EINVAL
    for o in ops:
        o.close()


def test_server_batches_same_operator_requests():
    wd = require_gpu()
    dims = (8, 8, 8, 8)
    srv = wd.Server(budget_bytes=8e9, slots=1, max_batch=8)
    blocker = srv.submit(dims=(16, 16, 16, 16), kappa=0.12, eps=0.4, gauge_seed=1, source_seed=1, tol=1e-10)
    reqs = []
    for i in range(10):   # queued behind the first request, then admitted in batches
        q = dict(dims=dims, kappa=(0.115, 0.12, 0.124)[i % 3], eps=0.3 + 0.02 * i, gauge_seed=700 + i,
                 source_seed=800 + i, tol=(1e-10, 1e-8)[i % 2], precision=wd.WD_PREC_MIXED_F32)
        x = torch.empty((8, 8, 8, 8, 4, 3), dtype=torch.complex128)
        reqs.append((q, x, srv.submit(x_host=x, **q)))
    assert srv.wait(blocker)["status"] == wd.WD_OK
    results = [srv.wait(rid) for _, _, rid in reqs]
    st = srv.stats()
    srv.close()
    assert st["batches"] >= 1 and st["batched_requests"] >= 2
    assert max(r["batch"] for r in results) > 1
    for (q, x, _), r in zip(reqs, results):
        assert r["status"] == wd.WD_OK
        f = (q["eps"], q["gauge_seed"], q["source_seed"], q["kappa"], q["tol"])
        sa, ia, ra, xa = _alone(wd, dims, q["precision"], f)
        assert ia == r["iterations"] and ra == r["true_rel_residual"] and np.array_equal(x.numpy(), xa)
        U = synthetic.gauge_field_philox(dims, q["eps"], q["gauge_seed"])
        eta = synthetic.gaussian_source_philox(dims, q["source_seed"])
        assert ocg.true_residual(U, eta, x.numpy(), q["kappa"]) <= q["tol"] * 1.01


def test_server_without_batching_and_option_checks():
    wd = require_gpu()
    srv = wd.Server(budget_bytes=4e9, slots=2, max_batch=1)
    ids = [srv.submit(dims=(8, 8, 8, 8), kappa=0.12, eps=0.4, gauge_seed=50 + i, source_seed=60 + i, tol=1e-8)
           for i in range(6)]
    res = [srv.wait(i) for i in ids]
    st = srv.stats()
    assert all(r["status"] == wd.WD_OK and r["batch"] == 1 for r in res) and st["batches"] == 0
    for bad in (0, 17, -1):
        with pytest.raises(wd.WdError):
            srv.set_max_batch(bad)
    srv.close()


@pytest.mark.parametrize("policy,max_wait,small_first", [(1, 1e7, True), (1, 0.0, False), (0, 1e7, False)])
def test_server_admission_policy(policy, max_wait, small_first):
    """Shortest-first admission (policy 1) starts queued small requests before an older large one;
    with no waiting allowed (max_wait 0) or the default policy the oldest goes first."""
    import time
    wd = require_gpu()
    srv = wd.Server(budget_bytes=8e9, slots=1, max_batch=1)
    srv.set_policy(policy, max_wait)
    q = dict(kappa=0.12, eps=0.4, source_seed=3, tol=1e-10, precision=wd.WD_PREC_MIXED_F32)
    t0 = time.perf_counter()
    ids, ts = [], []
    for i, dims in enumerate([(16, 16, 16, 16), (16, 16, 16, 32), (4, 4, 4, 4), (6, 6, 6, 6)]):
        ts.append(time.perf_counter() - t0)
        ids.append(srv.submit(dims=dims, gauge_seed=40 + i, **q))
    res = [srv.wait(i) for i in ids]
    srv.close()
    assert all(r["status"] == wd.WD_OK for r in res)
    start = [1e-3 * r["queue_ms"] + t for r, t in zip(res, ts)]
    big, small = start[1], min(start[2], start[3])
    assert (small < big) == small_first, (policy, max_wait, start)
    with pytest.raises(wd.WdError):
        wd.Server(budget_bytes=1e9, slots=1).set_policy(2, 0.0)
