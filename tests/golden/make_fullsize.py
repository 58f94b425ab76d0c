"""Write tests/golden/fullsize_c2.json from the CPU oracle only.

Runs the oracle's CG on the full 128^3 7-point Poisson workload (b = 2U-1,
tol 1e-14) in the mirrored summation order of plan (V=1, T=256, G=456) --
the plan the solver picks for this matrix on a 152-SM GB300, three blocks per
SM -- and records the iteration count, status, the bits of the final FP64
relative residual, the SHA-256 of the solution's bits and a few sampled
solution words.  The GPU tests compare the CUDA solver against these values
at full size.

Usage: python tests/golden/make_fullsize.py [arith ...]   (about 15 min for qtw, 8 for dw)
"""
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2510_13536_gb300 import problems as P  # noqa: E402

PLAN = (1, 256, 456)
OUT = os.path.join(HERE, "fullsize_c2.json")


def main(ariths):
    A, b, tol, maxit = P.workload("c2")
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    if tuple(data.get("plan", PLAN)) != PLAN:
        data = {}                                    # values of another plan: start afresh
    data["_source"] = ("CPU oracle (oracle/mwcg_oracle.cpp), mirrored order, written by "
                       "tests/golden/make_fullsize.py; workload c2: " + P.WORKLOADS["c2"])
    data["plan"] = list(PLAN)
    for ar in ariths:
        t = time.time()
        x, it, rr, st = oracle.cg(ar, A, b, tol=tol, maxit=maxit, plan=PLAN)
        xb = np.ascontiguousarray(x).view(np.uint64)
        idx = [0, 1, 12345, A.n // 2, A.n - 1]
        data[ar] = {
            "iters": int(it), "status": int(st), "relres_hex": float(rr).hex(),
            "x_sha256": hashlib.sha256(xb.tobytes()).hexdigest(),
            "samples": {str(i): [float(x[k, i]).hex() for k in range(x.shape[0])] for i in idx},
            "oracle_seconds": round(time.time() - t, 1),
        }
        print(ar, it, st, rr, round(time.time() - t, 1), "s", flush=True)
        json.dump(data, open(OUT, "w"), indent=1)


if __name__ == "__main__":
    main(sys.argv[1:] or ["qtw", "dw", "fp64"])
