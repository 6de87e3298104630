"""Small, self-contained workloads for profiling one kernel under ncu.

Examples:
  python -m paper_2111_14958_gb300.profile_case --prec 64 --dims 14,14,14,14 --launches 5
  python -m paper_2111_14958_gb300.profile_case --prec 32 --c12 --dims 32,32,32,32 --launches 3
  python -m paper_2111_14958_gb300.profile_case --prec 64 --dims 14,14,14,14 --solve
  python -m paper_2111_14958_gb300.profile_case --prec 6432 --c12 --dims 16,16,16,16 --launches 0 \
      --apply 3 --apply-df        # the double-float dslash (through wd_apply)
  python -m paper_2111_14958_gb300.profile_case --prec 6432 --c12 --dims 16,16,16,32 --launches 0 \
      --multi 12                  # the multi-RHS dslash (through wd_apply_multi)
  python -m paper_2111_14958_gb300.profile_case --prec 6432 --c12 --dims 24,24,24,48 --launches 0 \
      --device-fields --msolve 12 # one multi-RHS mixed-precision solve of 12 Gaussian sources

Fields come from the seeded generators (links exp(i 0.4 H), Gaussian source; on the host, or with
--device-fields from the library's own generators on the device); the program prints
the timing of the dslash as the solver launches it (CUDA events) and, with --solve, one CG solve.
"""
from __future__ import annotations

import argparse
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--prec", type=int, default=64, help="64, 32, 6432 or 6416")
    ap.add_argument("--dims", default="14,14,14,14")
    ap.add_argument("--c12", action="store_true")
    ap.add_argument("--launches", type=int, default=5)
    ap.add_argument("--dagger", action="store_true")
    ap.add_argument("--solve", action="store_true")
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--kappa", type=float, default=0.12)
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--apply", type=int, default=0, help="wd_apply calls on a Gaussian field")
    ap.add_argument("--apply-df", action="store_true",
                    help="mixed-precision contexts: wd_apply through the double-float operator")
    ap.add_argument("--even-odd", action="store_true")
    ap.add_argument("--multi", type=int, default=0, help="wd_apply_multi calls on this many Gaussian fields")
    ap.add_argument("--mgroup", type=int, default=0, help="multi-RHS group size K (0 = tuned)")
    ap.add_argument("--msites", type=int, default=0, help="multi-RHS sites per block (0 = tuned)")
    ap.add_argument("--msolve", type=int, default=0, help="one cg_solve_multi on this many Gaussian sources")
    ap.add_argument("--device-fields", action="store_true", help="generate links and sources on the device")
    ap.add_argument("--graph", type=int, default=-1,
                    help="WD_OPT_USE_GRAPH for the solves (0 = plain launches, which ncu lists one by one)")
    args = ap.parse_args(argv)

    import torch

    import synthetic
    from paper_2111_14958_gb300 import wd

    dims = tuple(int(v) for v in args.dims.split(","))
    prec = args.prec | (wd.WD_EVEN_ODD if args.even_odd else 0)
    op = wd.WilsonDirac(dims, args.kappa, (1, 1, 1, -1), prec)
    if args.device_fields:
        op.generate_gauge(0.4, 1, compress12=args.c12)
    else:
        op.load_gauge(torch.from_numpy(synthetic.gauge_field(dims, 0.4, 1)).cuda(), compress12=args.c12)

    def source(seed):
        if args.device_fields:
            return op.generate_source(seed)
        return torch.from_numpy(synthetic.gaussian_source(dims, seed)).cuda()
    if args.block:
        op.set_option(wd.WD_OPT_BLOCK_DSLASH, args.block)
    if args.graph >= 0:
        op.set_option(wd.WD_OPT_USE_GRAPH, args.graph)
    if args.launches:
        ms = op.time_dslash(args.dagger, args.launches)
        print(f"dslash dims={dims} prec={args.prec} c12={args.c12}: {ms * 1e3:.2f} us per launch")
    if args.apply:
        if args.apply_df:
            op.set_option(wd.WD_OPT_APPLY_DF, 1)
        psi = source(3)
        if args.prec == wd.WD_PREC_F32:
            psi = psi.to(torch.complex64)
        out = torch.empty_like(psi)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(args.apply):
            op.apply(psi, out=out)
        b.record()
        torch.cuda.synchronize()
        print(f"wd_apply x{args.apply}: {a.elapsed_time(b) / args.apply * 1e3:.2f} us per call (with packing)")
    if args.multi:
        if args.mgroup:
            op.set_option(wd.WD_OPT_MULTI_GROUP, args.mgroup)
        if args.msites:
            op.set_option(wd.WD_OPT_MULTI_SITES, args.msites)
        psi = torch.stack([source(10 + i) for i in range(args.multi)])
        out = op.apply_multi(psi)  # tunes the launch shape
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(3):
            out = op.apply_multi(psi)
        b.record()
        torch.cuda.synchronize()
        st = op.multi_stats()
        print(f"wd_apply_multi x3 ({args.multi} RHS): {a.elapsed_time(b) / 3 * 1e3:.1f} us per call with packing; "
              f"tuned group {st['group']} sites/block {st['sites_per_block']} dslash {st['dslash_ms'] * 1e3:.1f} us")
    if args.msolve:
        eta = torch.stack([source(100 + i) for i in range(args.msolve)])
        x = torch.zeros_like(eta)
        wd.cg_solve_multi(op.ctx, eta, x, args.tol, 20000)  # tunes the launch shapes
        x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, iters, res = wd.cg_solve_multi(op.ctx, eta, x, args.tol, 20000)
        t1 = time.perf_counter()
        ms = wd.wd_get_multi_stats(op.ctx)
        print(f"cg_solve_multi ({args.msolve} RHS): status {st} iterations {max(iters)} "
              f"max true residual {max(res):.3e} reliable updates {ms['reliable_updates']} "
              f"group {ms['group']} sites/block {ms['sites_per_block']} ms {1e3 * (t1 - t0):.1f}")
    if args.solve:
        eta = source(2)
        x, iters, res, status = op.solve(eta, tol=args.tol, maxit=4000)
        s = op.stats()
        print(f"solve: status {status} iterations {iters} true residual {res:.3e} "
              f"reliable updates {s['reliable_updates']} host ms {s['solve_ms']:.3f}")
    op.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
