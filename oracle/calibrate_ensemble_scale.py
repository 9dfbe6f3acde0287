"""Calibrate the Pareto fitness scale c over network sizes N in [10^3, 10^6].

Writes tests/golden/pareto_scale_grid.json: for each N of a grid with four
points per decade, the c for which the oracle's mean degree 2M/N of one
Miller-Hagberg sample (Sec. 2.4) is 20, by bisection on log c with common
random numbers (fitness seed 3, sampler seed 0, sample 0), as
oracle/calibrate_scale.py does for N = 10^6 alone.  Sizes between grid points
interpolate log c linearly in log N.

Run:  python oracle/calibrate_ensemble_scale.py
"""
import json
import math
import multiprocessing as mp
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

TARGET = 20.0
GRID = [int(round(10 ** (3 + k / 4))) for k in range(13)]


def mean_degree(n: int, c: float) -> float:
    import oracle
    from paper_2509_13230_gb300 import workloads
    net = workloads.pareto_ubcm(n, c, seed=3)
    _, _, _, counts, _ = oracle.mh_sample(oracle.UBCM, net.x, seed=0, num_samples=1, seg_target=1 << 30)
    return 2.0 * float(counts[0]) / n


def calibrate(n: int):
    lo, hi = math.log(1e-5), math.log(1.0)
    for _ in range(18):
        mid = 0.5 * (lo + hi)
        if mean_degree(n, math.exp(mid)) < TARGET:
            lo = mid
        else:
            hi = mid
    c = float(f"{math.exp(0.5 * (lo + hi)):.4g}")
    return n, c, mean_degree(n, c)


def main():
    with mp.get_context("spawn").Pool(min(len(GRID), os.cpu_count() or 1)) as pool:
        rows = pool.map(calibrate, GRID)
    out = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden",
                       "pareto_scale_grid.json")
    with open(out, "w") as f:
        json.dump({"n": [r[0] for r in rows], "scale": [r[1] for r in rows],
                   "mean_degree": [round(r[2], 4) for r in rows], "target": TARGET,
                   "how": "oracle/calibrate_ensemble_scale.py: bisection on the oracle's one-sample mean degree"},
                  f, indent=1)
        f.write("\n")
    for r in rows:
        print(r)


if __name__ == "__main__":
    main()
