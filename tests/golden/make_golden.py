"""Write the stored expected values under tests/golden/ by calling only the CPU oracle.

Run from the repository root: ``python tests/golden/make_golden.py``. The GPU tests read these
files; no stored value comes from the CUDA path.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import synthetic  # noqa: E402
from oracle import cg  # noqa: E402


def cgls_record(dims, kappa, eps, gseed, sseed, tol, maxit):
    U = synthetic.gauge_field(dims, eps, gseed)
    eta = synthetic.gaussian_source(dims, sseed)
    x, iters, true_res, hist = cg.cgls(U, eta, kappa, tol, maxit)
    return {
        "dims": list(dims), "kappa": kappa, "eps": eps, "gauge_seed": gseed, "source_seed": sseed,
        "tol": tol, "maxit": maxit, "iterations": int(iters), "true_rel_residual": true_res,
        "x_norm2": float(np.vdot(x, x).real),
        "history_every_10": [float(h) for h in hist[::10]],
    }


def main():
    out = {
        "what": "CGLS (CG on D^dagger D x = D^dagger eta) solves by the FP64 CPU oracle",
        "citation": "Sec. 2 CG algorithm (normal-equation reading); operator of Eq. (1) with "
                    "kappa form, r = 1, chiral gamma basis, antiperiodic time",
        "generator": "tests/golden/make_golden.py (calls oracle/ and synthetic/ only)",
        "solves": [
            cgls_record((4, 4, 4, 4), 0.12, 0.4, 1, 2, 1e-10, 2000),
            cgls_record((2, 3, 4, 5), 0.12, 0.4, 1, 2, 1e-10, 2000),
            cgls_record((6, 6, 6, 8), 0.124, 0.4, 3, 4, 1e-10, 2000),
        ],
    }
    with open(os.path.join(HERE, "cgls_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)
    # the benchmark workload: 14^4, kappa 0.12, eps 0.4, seeds 1/2, tol 1e-10
    rec = cgls_record((14, 14, 14, 14), 0.12, 0.4, 1, 2, 1e-10, 4000)
    rec["what"] = "oracle CGLS solve of the benchmark workload (iteration count for extrapolation)"
    with open(os.path.join(HERE, "bench_workload.json"), "w") as f:
        json.dump(rec, f, indent=1)


if __name__ == "__main__":
    main()
