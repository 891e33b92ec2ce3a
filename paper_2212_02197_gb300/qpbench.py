"""Batched QP subproblems, Eq. (QP-subproblem): the three solvers of
mc_qp_solve_batch on the same seeded random QPs (box-constrained, positive
definite 2x2 stage blocks, bounds active at the start on every fifth stage).

    python -m paper_2212_02197_gb300.qpbench [--n 30000] [--N 20,60]

Each line gives the wall time of one blocking call (host-device copies
included), the mean active-set iterations and the largest difference of du
from the serial active-set solution.  The kernels' own device times come
from running this under ncu's launch list (gpu__time_duration.sum):
k_qp_batch is one QP per thread, k_qp_batch_warp one QP per warp.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def random_qps(n, N, rng):
    A = rng.uniform(0.6, 1.2, (n, N))
    B = rng.uniform(-2.0, 2.0, (n, N))
    b = rng.normal(0.0, 0.5, (n, N))
    L = rng.normal(size=(n, N + 1, 2, 2)) + 1.5 * np.eye(2)
    Wk = L @ np.swapaxes(L, -1, -2) + 0.1 * np.eye(2)
    Wxx, Wxu, Wuu = Wk[..., 0, 0].copy(), Wk[..., 0, 1].copy(), Wk[..., 1, 1].copy()
    Wxx[:, 0] = Wxu[:, 0] = 0.0
    Wxu[:, N] = Wuu[:, N] = 0.0
    q = rng.normal(0.0, 2.0, (n, N + 1))
    q[:, 0] = 0.0
    r = rng.normal(0.0, 2.0, (n, N))
    lb = -rng.uniform(0.0, 0.3, (n, N))
    ub = rng.uniform(0.0, 0.3, (n, N))
    lb[:, ::5] = 0.0
    return A, B, b, Wxx, Wxu, Wuu, q, r, lb, ub


def main():
    from . import mc

    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=30000)
    ap.add_argument("--N", default="20,60")
    args = ap.parse_args()
    for N in [int(v) for v in args.N.split(",")]:
        qp = random_qps(args.n, N, np.random.default_rng(N))
        ref = None
        for solver in ("active_set", "active_set_warp", "ipm"):
            mc.qp_solve_batch(*qp, solver=solver)          # warm-up
            t = time.perf_counter()
            out = mc.qp_solve_batch(*qp, solver=solver)
            wall = time.perf_counter() - t
            if ref is None:
                ref = out
            print(json.dumps({"N": N, "n": args.n, "solver": solver, "wall_ms": wall * 1e3,
                              "mean_iters": float(out["iters"].mean()),
                              "solved": int((out["status"] == 0).sum()),
                              "max_du_diff_vs_active_set": float(np.abs(out["du"] - ref["du"]).max())}),
                  flush=True)


if __name__ == "__main__":
    main()
