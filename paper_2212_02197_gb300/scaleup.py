"""Scale-up of the Monte Carlo study with the number of SMs: the GPU
counterpart of the paper's scale-up over CPU cores (Sec. VII-B, Fig. 2).

    python -m paper_2212_02197_gb300.scaleup [--workload W] [--n-steps K]
                                             [--sms 8,16,32,64,128,0]

For each SM count the NMPC study of the workload runs on an SM partition of
that size (a green context, ``mc_set_sm_partition``; 0 = the whole GPU).
One JSON line per point gives the SMs used, the device time of the run, the
trajectories/s, and the speed-up and parallel efficiency relative to the
smallest partition.  Every point must reproduce the whole-GPU Phi bit for bit
(the partition changes where trajectories run, not what they compute).
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def main():
    import torch

    from . import mc, workloads as W

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="cstr_30k_x240_N20_fp64")
    ap.add_argument("--n-steps", type=int, default=24)
    ap.add_argument("--n-traj", type=int, default=None)
    ap.add_argument("--sms", default="8,16,32,64,128,0")
    ap.add_argument("--reps", type=int, default=2)
    args = ap.parse_args()

    w = W.get(args.workload)
    w["model"]["n_steps"] = args.n_steps
    n = args.n_traj or w["n_traj"]
    stream = torch.cuda.current_stream()
    h = mc.MonteCarlo(w["model"], w["nmpc"], n, w["seed"])
    ref = None
    base = None
    for req in [int(v) for v in args.sms.split(",")]:
        got = h.set_sm_partition(req)
        h.run(stream)                      # warm-up
        h.sync()
        ms = []
        for _ in range(args.reps):
            h.run(stream)
            ms.append(h.stats()["gpu_ms"])
        phi = h.phi()
        t = min(ms)
        if base is None:
            base = (got, t)
        speedup = base[1] / t
        line = {"sms": got, "requested": req, "ms": t, "trajectories_per_s": n / (t / 1e3),
                "speedup_vs_first": speedup, "efficiency": speedup / (got / base[0]),
                "workload": args.workload, "n_traj": n, "n_steps": args.n_steps}
        if ref is None:
            ref = phi
        line["phi_identical_to_first"] = bool(np.array_equal(phi, ref))
        print(json.dumps(line), flush=True)
    h.set_sm_partition(0)
    h.close()


if __name__ == "__main__":
    main()
