"""Calibrate the scale c of the N = 10^6 Pareto fitness workload.

Writes tests/golden/pareto_scale.json: the c for which the oracle's mean
degree 2M/N of one Miller-Hagberg sample (Sec. 2.4) equals 20, found by
bisection on log c with common random numbers (seed 0, sample 0).  The
expected number of edges sum_{i<j} p_ij (Eq. 1) is what the sample estimates;
its sampling noise at M ~ 10^7 is about 3e-4 relative.

Run:  python oracle/calibrate_scale.py
"""
import json
import math
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import oracle  # noqa: E402
from paper_2509_13230_gb300 import workloads  # noqa: E402

TARGET = 20.0
N = 1_000_000


def mean_degree(c: float) -> float:
    net = workloads.pareto_ubcm(N, c, seed=3)
    _, _, _, counts, _ = oracle.mh_sample(oracle.UBCM, net.x, seed=0, num_samples=1, seg_target=1 << 30)
    return 2.0 * float(counts[0]) / N


def main():
    lo, hi = math.log(1e-4), math.log(1e-2)
    for _ in range(18):
        mid = 0.5 * (lo + hi)
        k = mean_degree(math.exp(mid))
        print(f"c={math.exp(mid):.6e} mean degree={k:.4f}", flush=True)
        if k < TARGET:
            lo = mid
        else:
            hi = mid
    c = float(f"{math.exp(0.5 * (lo + hi)):.4g}")
    k = mean_degree(c)
    out = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden",
                       "pareto_scale.json")
    with open(out, "w") as f:
        json.dump({"scale": c, "n": N, "mean_degree": k, "target": TARGET,
                   "how": "oracle/calibrate_scale.py: bisection on the oracle's one-sample mean degree"}, f,
                  indent=1)
        f.write("\n")
    print("scale", c, "mean degree", k)


if __name__ == "__main__":
    main()
