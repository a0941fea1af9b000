"""Writes oracle_cycles.json: how many defect-correction cycles the FP64 oracle needs for the
first CN step of the uniform 256^3 resistive-bump workload (and smaller sizes of the same
family) to reach ||R||/||S|| <= 1e-9 with V(2,2) cycles and 16 coarsest sweeps.

Calls only oracle/ and the seeded input generators.  Used by bench.py's CPU-baseline leg to
turn the oracle's time per cycle into cell-steps/s.  Run: python tests/golden/make_oracle_cycles.py [n ...]
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.oracle import Oracle  # noqa: E402
from paper_1009_0798_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_cycles.json")


def main(sizes):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for n in sizes:
        wl = W.resistive_bump_256(n=n)
        o = Oracle(wl.hier, wl.lam, wl.eta)
        t = time.time()
        _, info = o.cn_step(wl.B, wl.dt, wl.tol, nu_pre=2, nu_post=2, n_coarse=16, max_outer=200)
        data[f"resistive_bump_{n}"] = {"cycles": info["cycles"], "converged": info["converged"],
                                       "history": [float(v) for v in info["history"]],
                                       "tol": wl.tol, "nu": [2, 2], "n_coarse": 16,
                                       "seconds": round(time.time() - t, 1)}
        json.dump(data, open(OUT, "w"), indent=1)
        print(n, info["cycles"], time.time() - t, flush=True)


if __name__ == "__main__":
    main([int(a) for a in sys.argv[1:]] or [32, 64, 128, 256])
