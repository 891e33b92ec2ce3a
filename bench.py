"""Benchmark: the paper-scale Monte Carlo closed-loop study on GB300.

One step = the whole hot path on one batch: 30,000 NMPC closed-loop
trajectories (CD-EKF + SQP per sample) and the 30,000 PI reference
trajectories on the same noise, 240 control steps each, N = 20, inlet-
temperature step disturbance, followed by the on-device reduction of Phi and
the OCP statistics.  value = NMPC closed-loop trajectories per second (the PI
companion runs inside the same timed step and is not counted).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME]

--impl reference times the FP64 CPU oracle (the plain C implementation of the
paper's method) on the host cores, one trajectory per thread at a time, on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2212_02197_gb300 import shards, workloads as W  # noqa: E402

METRIC = "closed-loop trajectories/sec (NMPC CSTR, 30k sims) mixed vs FP64, at stated tol"
DEFAULT_WORKLOAD = "cstr_30k_x240_N20_fp64"


# ------------------------------------------------------------------ algorithmic work
#
# The NMPC kernel is bound by GB300's FP64 pipe (nominally 2 fused
# multiply-adds per SM per clock).  Two measures of its work per launch, both
# multiplied by the launch's own counters (trajectories, OCPs, SQP iterations,
# line-search trials, QP iterations):
#
# * algorithmic flops, counted by the oracle's operation-counting build
#   (oracle/opcount.py writes oracle/opcounts.json): per shooting interval,
#   per Euler-Maruyama substep with its normals, per sample (measurement,
#   filter, set-points, Phi), per NLP evaluation and per SQP iteration, in the
#   oracle's own formulation; +, -, x, /, sqrt, compare and min/max count one
#   flop each, exp, log, sin and cos the cost of the library function measured
#   on the device (peaks.py), in FP64 fused multiply-adds, times two.  The QP
#   subproblem is counted as the structured method solves it, a Riccati
#   recursion of 24 fused operations and one division per stage and active-set
#   iteration (the oracle condenses it densely instead, for independence).
#   Shooting intervals are counted as the method needs them: all N at a
#   trajectory's first OCP and at every line-search trial, and 2 at a later
#   OCP's start (the shifted warm start reuses the other N - 2, evaluated at
#   the same points); the CD-EKF prediction rides on the final iterate's
#   interval 0, so it adds nothing beyond its covariance.
# * FP64 pipe operations of the kernel's own formulation (the operation model
#   below, from the kernel source), elementary functions at their measured
#   cost: how busy the pipe is kept.

# per unit of the kernel's formulation, in FP64 pipe operations besides the
# elementary functions (one state, one input):
OPS_MODEL1 = 15                               # f, df/dx, df/dF (+ exp + reciprocal)
OPS_RK4_STAGE = 29                            # one RK4 step's stage algebra with sensitivities
OPS_INTERVAL_EXTRA = 12                       # F/V, (F sigma_T)^2, B = Fconv b, g_k, q_k, objective
OPS_COV_STEP = 15                             # CD-EKF covariance on an RK4 step of interval 0
OPS_QP_STAGE = 24                             # active-set iteration, per stage (+ 1 division)
OPS_SQP_STAGE = 45                            # gradient, KKT test, block BFGS, merit (+ 2 div)
OPS_ACCEPT_STAGE = 15                         # multiplier step, gradients, copy (+ 1 div)
OPS_TRIAL_STAGE = 6                           # trial point and its merit sum
OPS_EKF = 12                                  # filter (+ 1 div)
OPS_EM = 50                                   # EM substep (+ exp + div + 2 x (log + sqrt + sincospi + 8))
PEAK_NOMINAL_TFLOPS = 2 * 2 * 152 * 2.07e9 / 1e12   # 2 DFMA/clk/SM x 152 SMs x 2.07 GHz x 2
RICCATI_FLOPS_STAGE = 2 * 24 + 1              # the QP's structured solve, per stage and iteration
OPCOUNTS = os.path.join(ROOT, "oracle", "opcounts.json")

# DRAM bytes (read + write) of k_nmpc_persist<double> per control step of the
# 30,000-trajectory FP64 study, from one ncu capture of a 60-step case of it
# (dram__bytes_read.sum 59.48 GB + dram__bytes_write.sum 76.15 GB).  A full
# launch is scaled by its steps and trajectories.
TRAFFIC_WORKLOAD = "cstr_30k_x240_N20_fp64"
TRAFFIC_BYTES_PER_STEP_30K = (59476805000 + 76153419000) / 60


def nmpc_pipe_ops(cfg_model, cfg_ctrl, n_traj, st, w):
    """FP64 pipe operations of one NMPC launch in the kernel's formulation,
    elementary functions weighted by w (DFMA equivalents)."""
    N, nrk = cfg_ctrl["N"], cfg_ctrl["n_rk4"]
    K, nem = cfg_model["n_steps"], cfg_model["n_em"]
    model1 = OPS_MODEL1 + w["exp_table"] + w.get("rcp", w["div"])
    per_interval = nrk * (4 * model1 + OPS_RK4_STAGE) + OPS_INTERVAL_EXTRA
    first_evals = n_traj * N + (st["n_ocp"] - n_traj) * min(N, 2)   # warm starts reuse N-2
    ops = (first_evals + st["ls_trials"] * N) * per_interval
    ops += (st["n_ocp"] + st["ls_trials"]) * nrk * OPS_COV_STEP   # interval 0 of each evaluation
    ops += st["qp_iters"] * N * (OPS_QP_STAGE + w.get("rcp", w["div"]))   # the pivot's reciprocal
    ops += st["sqp_iters"] * N * (OPS_SQP_STAGE + OPS_ACCEPT_STAGE + 3 * w["div"])
    ops += st["ls_trials"] * N * OPS_TRIAL_STAGE
    em = OPS_EM + w["exp_table"] + w["div"] + 2 * (8 + w["log"] + w["sqrt"] + w["sincospi"])
    ops += n_traj * K * (OPS_EKF + w["div"] + nem * em)
    return ops


def _flops(ops: dict, w: dict) -> float:
    """Algorithmic flops of one event from the oracle's counts by kind."""
    plain = sum(ops.get(k, 0.0) for k in ("add", "mul", "div", "sqrt", "cmp", "minmax"))
    special = (ops.get("exp", 0.0) * w["exp_lib"] + ops.get("log", 0.0) * w["log"] +
               (ops.get("sin", 0.0) + ops.get("cos", 0.0)) * 0.5 * w["sincospi"])
    return plain + 2.0 * special


def nmpc_algorithmic_flops(cfg_model, cfg_ctrl, n_traj, st, w, opc):
    """Algorithmic flops of one one-state NMPC launch from the oracle's
    per-event operation counts and the launch's counters."""
    ev = opc["events"]
    N = cfg_ctrl["N"]
    K, nem = cfg_model["n_steps"], cfg_model["n_em"]
    f = {k: _flops(v["ops"], w) for k, v in ev.items()}
    rest = opc["sqp_rest"]
    intervals = n_traj * N + (st["n_ocp"] - n_traj) * min(N, 2) + st["ls_trials"] * N
    flops = intervals * f["rk4_interval"]
    flops += n_traj * K * (nem * (f["em_step"] + f["process_noise"]) + f["meas_noise"] +
                           f["ekf_filter"] + f["closed_loop_sample"])
    flops += (st["n_ocp"] + st["ls_trials"]) * f["evaluate"]
    flops += st["n_ocp"] * _flops(rest["per_ocp"], w)
    flops += st["sqp_iters"] * _flops(rest["per_sqp_iteration"], w)
    flops += st["qp_iters"] * N * RICCATI_FLOPS_STAGE
    return flops


def warp_trace_summary(h, n_steps=None):
    """Where the last persistent launch's time went, from its per-warp record
    (mc_copy_warp_trace): the SMs' busy share of the launch (last warp end
    minus first warp start on each SM, over the launch's span), the warps'
    pool rounds, and the lanes holding a trajectory per round."""
    import numpy as np

    tr = h.warp_trace()
    t0, t1, sm = tr["t_start_ns"], tr["t_end_ns"], tr["sm"]
    span = float(t1.max() - t0.min())
    busy = [float(t1[sm == q].max() - t0[sm == q].min()) for q in np.unique(sm)]
    r = tr["rounds"].astype(float)
    dur = (t1 - t0).astype(float)
    slow = int(np.argmax(t1))
    out = {"warps": int(len(r)), "sms": int(len(busy)), "span_ms": span / 1e6,
           "sm_busy_frac": float(np.mean(busy) / span),
           "rounds_mean": float(r.mean()), "rounds_max": int(r.max()),
           "lanes_per_round": float(tr["lane_rounds"].sum() / r.sum()),
           "warp_ms_mean": float(dur.mean() / 1e6), "warp_ms_max": float(dur.max() / 1e6),
           "last_warp": {"rounds": int(r[slow]), "ms": float(dur[slow] / 1e6),
                         "us_per_round": float(dur[slow] / r[slow] / 1e3)},
           "us_per_round_mean": float(np.mean(dur / r) / 1e3),
           "corr_rounds_ms": float(np.corrcoef(r, dur)[0, 1])}
    if n_steps is not None:
        # a trajectory's own trials: one per OCP start and one per line-search
        # trial (a backtracking line search shoots several in one round, so
        # this bounds the trajectory's rounds from above)
        cnt = h.counters()
        tr_r = n_steps + cnt["ls_trials"].astype(np.int64)
        jm = int(np.argmax(tr_r))
        out["trajectory_starts_and_trials"] = {
            "mean": float(tr_r.mean()), "max": int(tr_r[jm]),
            "slowest": {"j": jm, "ocps_at_iteration_limit": int(cnt["n_ocp_failed"][jm]),
                        "sqp_iters": int(cnt["sqp_iters"][jm])},
            "trajectories_with_an_ocp_at_the_limit": int((cnt["n_ocp_failed"] > 0).sum())}
    return out


def measured_peaks():
    """FP64/FP32 peaks and elementary-function costs measured on this device;
    falls back to the nominal FP64 peak and fixed weights if the probe fails."""
    from paper_2212_02197_gb300 import peaks

    try:
        return peaks.measure(), "measured"
    except Exception as e:  # pragma: no cover
        return {"fp64_tflops": PEAK_NOMINAL_TFLOPS, "fp32_tflops": None,
                "weights_dfma": {k: 1.0 for k in ("exp_table", "exp_lib", "div", "rcp", "log",
                                                  "sqrt", "sincospi")},
                "error": str(e)}, "nominal (the probe failed; functions weighted 1)"


# ------------------------------------------------------------------ clocks

class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = str(gpu_index)
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu, f"--query-gpu={self.Q}", "--format=csv,noheader",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([t.strip() for t in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            if self.thread:
                self.thread.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1].split()[0]))
                mx = float(r[2].split()[0])
            except Exception:
                continue
            for name, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ reference arm

def run_reference(args, workload):
    """Oracle on the host cores: bounded sample of the workload per step."""
    import oracle

    oracle.build()
    w = W.get(workload)
    cores = os.cpu_count() or 1
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    # sample size: about 10 s of host time per step at most
    n = 16 * cores
    t0 = time.perf_counter()
    oracle.run(w["model"], w["nmpc"], w["seed"], 0, n, threads=cores)
    if w["pi"] is not None:
        oracle.run(w["model"], w["pi"], w["seed"], 0, n, threads=cores)
    dt = time.perf_counter() - t0
    n = max(cores, min(w["n_traj"], int(n * 8.0 / max(dt, 1e-3))))
    times = []
    for s in range(args.warmup + args.steps):
        j0 = (s * n) % max(1, w["n_traj"] - n)
        t0 = time.perf_counter()
        oracle.run(w["model"], w["nmpc"], w["seed"], j0, j0 + n, threads=cores)
        if w["pi"] is not None:
            oracle.run(w["model"], w["pi"], w["seed"], j0, j0 + n, threads=cores)
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = n * len(times) / tot
    sample = (f"{n} NMPC + {n} PI trajectories of {workload} per step "
              f"({'pthreads, one trajectory per thread at a time'})")
    return {"metric": METRIC, "value": value, "unit": "trajectories/s", "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload, "n_traj": n, "oracle": "oracle/ (C, FP64)"},
            "cpu_baseline": {"value": value, "unit": "trajectories/s", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "trajectories/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def cpu_baseline(workload, budget_s=15.0):
    import oracle

    oracle.build()
    w = W.get(workload)
    cores = os.cpu_count() or 1
    n = 8 * cores
    t0 = time.perf_counter()
    done = 0
    while True:
        oracle.run(w["model"], w["nmpc"], w["seed"], done, done + n, threads=cores)
        if w["pi"] is not None:
            oracle.run(w["model"], w["pi"], w["seed"], done, done + n, threads=cores)
        done += n
        if time.perf_counter() - t0 > budget_s or done + n > w["n_traj"]:
            break
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": "trajectories/s", "cores": cores, "kind": "oracle",
            "sample": f"trajectories 0..{done - 1} of {workload}, NMPC and PI each, "
                      f"{cores} host threads, {dt:.1f} s"}


def cpu_baseline_nmpc(workload, budget_s=12.0):
    """The oracle's NMPC trajectories/s on the host cores, on a prefix of the
    workload (trajectories are i.i.d.)."""
    import oracle

    oracle.build()
    w = W.get(workload)
    cores = os.cpu_count() or 1
    n = 2 * cores
    t0 = time.perf_counter()
    done = 0
    while True:
        oracle.run(w["model"], w["nmpc"], w["seed"], done, done + n, threads=cores)
        done += n
        if time.perf_counter() - t0 > budget_s or done + n > w["n_traj"]:
            break
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": "NMPC trajectories/s", "cores": cores, "kind": "oracle",
            "sample": f"NMPC trajectories 0..{done - 1} of {workload}, {cores} host threads, "
                      f"{dt:.1f} s"}


# ------------------------------------------------------------------ our arm

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-grad", action="store_true")
    # smaller cases of the same workload, for profiling captures
    ap.add_argument("--n-traj", type=int, default=None)
    ap.add_argument("--n-steps", type=int, default=None)
    args = ap.parse_args()

    if args.impl == "reference":
        line = run_reference(args, args.workload)
        if line is not None:
            print(json.dumps(line), flush=True)
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2212_02197_gb300 import mc

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    w = W.get(args.workload)
    if args.n_traj:
        w["n_traj"] = args.n_traj
    if args.n_steps:
        w["model"]["n_steps"] = args.n_steps
    T = w["n_traj"]
    # weak scaling: rank r simulates trajectories r*T .. (r+1)*T-1
    j0, j1 = rank * T, (rank + 1) * T
    h_n = mc.MonteCarlo(w["model"], w["nmpc"], j1, w["seed"])
    h_p = mc.MonteCarlo(w["model"], w["pi"], j1, w["seed"]) if w["pi"] is not None else None
    tuned_tps = None
    if w["nmpc"].get("schedule") == "persistent" and not args.no_autotune:
        tuned_tps = h_n.autotune(probe_steps=24, stream=stream)   # set-up, untimed
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    pk, pk_src = measured_peaks()          # set-up, untimed

    def step():
        h_n.run(stream, j0, j1)
        if h_p is not None:
            h_p.run(stream, j0, j1)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    nmpc_ms = []
    barrier()
    clocks.start()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()                       # L2 flush between timed steps (untimed)
        a, b, c = ev[i]
        a.record(stream)
        h_n.run(stream, j0, j1)
        b.record(stream)
        if h_p is not None:
            h_p.run(stream, j0, j1)
        c.record(stream)
    barrier()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    step_ms = [a.elapsed_time(c) for a, b, c in ev]
    nmpc_ms = [a.elapsed_time(b) for a, b, c in ev]
    st_n = h_n.stats()
    # the study's statistics over all ranks (only the reduced numbers travel)
    st_all = shards.allgather_stats(st_n, dist if world > 1 else None)
    my_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([my_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        my_ms = float(t.item())
    ms_per_step = my_ms / args.steps
    value = world * T / (ms_per_step / 1e3)

    # dominant kernel: the NMPC closed loop; its device time per launch
    # (mc_run = k_nmpc + two small reduction kernels)
    wts = pk["weights_dfma"]
    k_ms = statistics.mean(nmpc_ms)
    traffic = None
    if (args.workload == TRAFFIC_WORKLOAD and w["nmpc"].get("schedule") == "persistent"
            and w["nmpc"]["precision"] == "fp64"):
        traffic = TRAFFIC_BYTES_PER_STEP_30K * w["model"]["n_steps"] * T / 30000.0
    peak = pk["fp64_tflops"]
    pipe_tf = 2.0 * nmpc_pipe_ops(w["model"], w["nmpc"], T, st_n, wts) / (k_ms / 1e3) / 1e12
    roofline = {"bound": "alu", "achieved": None, "peak": peak, "unit": "TFLOP/s",
                "frac": None, "traffic": traffic,
                "traffic_note": "DRAM bytes per launch, scaled from a 60-step ncu capture; "
                                "structure-of-arrays scratch, not algorithmic bytes",
                "kernel": "k_nmpc_persist<double> (FP64 pipe)",
                "peak_source": f"{pk_src}: FP64 fma chains on this device (paper_2212_02197_gb300"
                               f".peaks, 2 flops per fma); nominal {PEAK_NOMINAL_TFLOPS:.3f}",
                "pipe": {"achieved": pipe_tf, "frac": pipe_tf / peak,
                         "frac_of_nominal": pipe_tf / PEAK_NOMINAL_TFLOPS,
                         "work": "FP64 pipe operations of the kernel's formulation x 2, "
                                 "elementary functions at their measured cost"},
                "weights_dfma": wts}
    opc = None
    if os.path.exists(OPCOUNTS) and w["nmpc"].get("nx_model", 1) != 3:
        with open(OPCOUNTS) as fh:
            opc = json.load(fh)["nmpc"]
        alg = nmpc_algorithmic_flops(w["model"], w["nmpc"], T, st_n, wts, opc)
        roofline["achieved"] = alg / (k_ms / 1e3) / 1e12
        roofline["frac"] = roofline["achieved"] / peak
        roofline["work"] = ("algorithmic flops: the oracle's operation counts per event "
                            "(oracle/opcounts.json) x this launch's counters; QP as a "
                            "Riccati recursion")
    else:
        roofline["achieved"], roofline["frac"] = pipe_tf, pipe_tf / peak
        roofline["work"] = roofline["pipe"]["work"]
    if w["nmpc"].get("schedule") == "persistent" and w["nmpc"].get("nx_model", 1) != 3:
        roofline["warp_trace"] = warp_trace_summary(h_n, w["model"]["n_steps"])

    def timed(handles, n, label_ranges=True):
        """Mean device ms of n timed runs of the handles (in order, one stream),
        after one warm-up; L2 flushed before each."""
        for h in handles:
            h.run(stream, j0, j1)
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(len(handles) + 1)]
               for _ in range(n)]
        barrier()
        for e in evs:
            flush.zero_()
            e[0].record(stream)
            for h, ee in zip(handles, e[1:]):
                h.run(stream, j0, j1)
                ee.record(stream)
        barrier()
        per = [statistics.mean(e[q].elapsed_time(e[q + 1]) for e in evs)
               for q in range(len(handles))]
        if world > 1:
            t = torch.tensor(per, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            per = t.tolist()
        return per

    def ks_stat(a, b):
        try:
            from scipy import stats as sps
            return float(sps.ks_2samp(a, b).statistic)
        except Exception:
            return None

    def accept(st_x, phi_x, st_ref, phi_ref):
        mean_rel = st_x["phi_mean"] / st_ref["phi_mean"] - 1.0
        ks = ks_stat(phi_x, phi_ref)
        return {"phi_mean_rel_vs_fp64": mean_rel, "ks_vs_fp64": ks,
                "median_rel_err_vs_fp64": float(np.median(np.abs(phi_x - phi_ref) /
                                                          np.abs(phi_ref))),
                "accepted": bool(abs(mean_rel) < 5e-3 and ks is not None and ks < 1e-2)}

    def ocp_stats(st):
        return {k: st[k] for k in ("n_ocp", "n_ocp_failed", "n_ls_fail", "sqp_iters",
                                   "ls_trials", "qp_iters")}

    # the same study in mixed precision, timed the same way and accepted
    # against this FP64 run (mean of Phi within 0.5 %, KS statistic < 0.01);
    # beside it the FP64 path under the mixed path's SQP stopping rule, so that
    # the precision's share of the speed-up is separate from the rule's
    mixed = None
    wl32 = args.workload.replace("_fp64", "_mixed")
    steps2 = max(1, min(args.steps, 5))
    if not args.no_mixed and wl32 in W.WORKLOADS and wl32 != args.workload:
        w32 = W.get(wl32)
        w32["model"] = w["model"]
        h32 = mc.MonteCarlo(w32["model"], w32["nmpc"], j1, w32["seed"])
        h32p = mc.MonteCarlo(w32["model"], w32["pi"], j1, w32["seed"])
        c_rule = dict(w["nmpc"], sqp_tol=w32["nmpc"]["sqp_tol"], ls_max=w32["nmpc"]["ls_max"])
        h64r = mc.MonteCarlo(w["model"], c_rule, j1, w["seed"])
        if c_rule.get("schedule") == "persistent" and tuned_tps:
            h64r.autotune(probe_steps=24, stream=stream)
        m_nmpc_ms, m_pi_ms = timed([h32, h32p], args.steps)
        m_ms = m_nmpc_ms + m_pi_ms
        (r_nmpc_ms,) = timed([h64r], steps2)
        st32, st64r = h32.stats(), h64r.stats()
        phi64, phi32, phi64r = h_n.phi(j0, T), h32.phi(j0, T), h64r.phi(j0, T)
        alg32 = (nmpc_algorithmic_flops(w32["model"], w32["nmpc"], T, st32, wts, opc)
                 if opc else None)
        mixed = {"workload": wl32, "schedule": w32["nmpc"].get("schedule", "static"),
                 "value": world * T / (m_ms / 1e3), "unit": "trajectories/s",
                 "ms_per_step": m_ms, "nmpc_ms_per_step": m_nmpc_ms,
                 "speedup_vs_fp64": ms_per_step / m_ms,
                 "speedup_note": "mixed precision with its own SQP stopping rule against "
                                 "FP64 at tolerance 1e-5: precision and rule together",
                 "dtype": "f32 shooting/plant/EKF-predict + f64 Joseph/QP/merit/BFGS/KKT",
                 "sqp_tol": w32["nmpc"]["sqp_tol"], "ls_max": w32["nmpc"]["ls_max"],
                 **accept(st32, phi32, st_n, phi64),
                 "ocp_stats": ocp_stats(st32),
                 "algorithmic_tflops": (alg32 / (m_nmpc_ms / 1e3) / 1e12) if alg32 else None,
                 "frac_of_fp64_peak": (alg32 / (m_nmpc_ms / 1e3) / 1e12 / peak)
                 if alg32 else None,
                 "frac_of_fp32_peak": (alg32 / (m_nmpc_ms / 1e3) / 1e12 / pk["fp32_tflops"])
                 if alg32 and pk.get("fp32_tflops") else None,
                 "fp64_same_rule": {
                     "what": "the FP64 path (NMPC kernel only) under the mixed path's SQP "
                             "stopping rule",
                     "schedule": c_rule.get("schedule", "static"),
                     "nmpc_ms_per_step": r_nmpc_ms,
                     "speedup_mixed_vs_fp64_same_rule": r_nmpc_ms / m_nmpc_ms,
                     "speedup_fp64_same_rule_vs_fp64": k_ms / r_nmpc_ms,
                     **accept(st64r, phi64r, st_n, phi64),
                     "ocp_stats": ocp_stats(st64r)}}
        h32.close()
        h32p.close()
        h64r.close()

    # the mixed-precision study of the workload list: 100,000 NMPC trajectories,
    # N = 30, E_a/R lognormal 2 %, 240 steps; timed in mixed precision and
    # accepted against an FP64 run of all 100,000 trajectories (once, untimed
    # beyond its own launch), with the FP64 path at the mixed rule beside it
    cfg3 = None
    if not args.no_mixed and args.workload == DEFAULT_WORKLOAD and not args.n_traj \
            and not args.n_steps:
        w3 = W.get("cstr_100k_x240_N30_mixed")
        n3 = w3["n_traj"]
        jj0, jj1 = rank * n3, (rank + 1) * n3
        c64 = dict(w3["nmpc"], precision="fp64", sqp_tol=1e-5, ls_max=30,
                   schedule="persistent")
        c64r = dict(c64, sqp_tol=w3["nmpc"]["sqp_tol"], ls_max=w3["nmpc"]["ls_max"])
        h3 = mc.MonteCarlo(w3["model"], w3["nmpc"], jj1, w3["seed"])
        h3_64 = mc.MonteCarlo(w3["model"], c64, jj1, w3["seed"])
        h3_64r = mc.MonteCarlo(w3["model"], c64r, jj1, w3["seed"])
        # one resident thread per trajectory (the autotuner's choice in every
        # run measured; its 24-step probes of this study cost a minute)
        tps3 = None
        saved = (j0, j1)
        j0, j1 = jj0, jj1
        (ms3,) = timed([h3], max(1, min(args.steps, 3)))
        (ms3_64r,) = timed([h3_64r], 1)
        ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        ea.record(stream)
        h3_64.run(stream, j0, j1)
        eb.record(stream)
        barrier()
        ms3_64 = ea.elapsed_time(eb)
        j0, j1 = saved
        s3, s3_64, s3_64r = h3.stats(), h3_64.stats(), h3_64r.stats()
        p3, p3_64, p3_64r = h3.phi(jj0, n3), h3_64.phi(jj0, n3), h3_64r.phi(jj0, n3)
        cfg3 = {"workload": "cstr_100k_x240_N30_mixed", "n_traj": n3, "N": 30,
                "precision": "mixed", "schedule": w3["nmpc"].get("schedule", "static"),
                "value": world * n3 / (ms3 / 1e3), "unit": "trajectories/s", "ms": ms3,
                "sqp_tol": w3["nmpc"]["sqp_tol"], "ls_max": w3["nmpc"]["ls_max"],
                **accept(s3, p3, s3_64, p3_64), "ocp_stats": ocp_stats(s3),
                "fp64": {"ms": ms3_64, "value": world * n3 / (ms3_64 / 1e3),
                         "schedule": "persistent", "threads_per_sm": tps3,
                         "sqp_tol": 1e-5, "ocp_stats": ocp_stats(s3_64)},
                "fp64_same_rule": {"ms": ms3_64r, "value": world * n3 / (ms3_64r / 1e3),
                                   "speedup_mixed_vs_fp64_same_rule": ms3_64r / ms3,
                                   **accept(s3_64r, p3_64r, s3_64, p3_64),
                                   "ocp_stats": ocp_stats(s3_64r)}}
        for h in (h3, h3_64, h3_64r):
            h.close()

    # the paper's own setting (Sec. VII-A: T_s = 1 s, N_s = 20, N = 60, 600
    # steps, u_max = 1000 mL/min), FP64, one run of each controller: the only
    # workload directly comparable with the paper's 55 min for 30,000 NMPC
    # simulations on 32 Xeon cores (Table II)
    paper_ctx = None
    if not args.no_mixed and args.workload == DEFAULT_WORKLOAD and not args.n_traj \
            and not args.n_steps:
        wp = W.get("cstr_paper_30k_x600_N60")
        npp = wp["n_traj"]
        hp_n = mc.MonteCarlo(wp["model"], wp["nmpc"], (rank + 1) * npp, wp["seed"])
        hp_p = mc.MonteCarlo(wp["model"], wp["pi"], (rank + 1) * npp, wp["seed"])
        tpsp = None   # one resident thread per trajectory, as for the 100k study
        saved = (j0, j1)
        j0, j1 = rank * npp, (rank + 1) * npp
        ea, eb, ec = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        barrier()
        ea.record(stream)
        hp_n.run(stream, j0, j1)
        eb.record(stream)
        hp_p.run(stream, j0, j1)
        ec.record(stream)
        barrier()
        j0, j1 = saved
        sp = hp_n.stats()
        paper_ctx = {"workload": "cstr_paper_30k_x600_N60", "n_traj": npp, "n_steps": 600,
                     "N": 60, "precision": "fp64", "schedule": "persistent",
                     "threads_per_sm": tpsp,
                     "nmpc_s": ea.elapsed_time(eb) / 1e3, "pi_s": eb.elapsed_time(ec) / 1e3,
                     "nmpc_value": world * npp / (ea.elapsed_time(eb) / 1e3),
                     "unit": "NMPC trajectories/s", "ocp_stats": ocp_stats(sp),
                     "paper": "about 55 min (3,300 s) for 30,000 NMPC simulations on 32 "
                              "Xeon Gold 6226R cores, 9.1 trajectories/s; 424 of 18,000,000 "
                              "OCPs at the iteration limit (Table II)"}
        hp_n.close()
        hp_p.close()

    # gradient of mean Phi of the PI study with respect to (k_P, k_I, k_aw):
    # forward sweep with checkpoints every 20 samples and the discrete adjoint,
    # timed like the study; checked against central differences (h = 1e-5 of
    # each gain) of the GPU's own mean Phi
    grad = None
    if not args.no_grad and h_p is not None and w["pi"]["precision"] == "fp64":
        ck = 20
        for _ in range(max(1, args.warmup)):
            h_p.pi_grad(ck, stream, j0, j1)
        evg = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        barrier()
        for a, b in evg:
            flush.zero_()
            a.record(stream)
            h_p.pi_grad(ck, stream, j0, j1)
            b.record(stream)
        barrier()
        g_ms = statistics.mean(a.elapsed_time(b) for a, b in evg)
        gm = h_p.grad_mean()
        g_phi = h_p.stats()["phi_mean"]
        cp = w["pi"]
        fd = []
        for q, k in enumerate(("kP", "kI", "kaw")):
            dk = 1e-5 * abs(cp[k])
            m2 = []
            for sgn in (1, -1):
                g = {kk: cp[kk] for kk in ("kP", "kI", "kaw")}
                g[k] += sgn * dk
                h_p.set_pi_gains(g["kP"], g["kI"], g["kaw"])
                h_p.run(stream, j0, j1)
                m2.append(h_p.stats()["phi_mean"])
            fd.append((m2[0] - m2[1]) / (2 * dk))
        h_p.set_pi_gains(cp["kP"], cp["kI"], cp["kaw"])
        h_p.run(stream, j0, j1)
        if world > 1:
            t = torch.tensor([g_ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            g_ms = float(t.item())
        grad = {"what": "d mean Phi / d(k_P, k_I, k_aw) of the PI study, discrete adjoint",
                "checkpoint_every": ck, "value": world * T / (g_ms / 1e3),
                "unit": "trajectories/s (forward + adjoint)", "ms_per_step": g_ms,
                "phi_mean": g_phi, "grad_mean": gm.tolist(), "fd_h_rel": 1e-5,
                "fd_grad_mean": fd,
                "fd_rel_err": [abs(f / g - 1.0) if g != 0 else None for f, g in zip(fd, gm)]}

    # gradient of mean Phi of the NMPC study with respect to the objective
    # weights (Q_z, R_u, Q_n) at R_u = 0.2, Q_n = 1.0 (with the paper's
    # objective, R_u = Q_n = 0, the Q_z direction vanishes): implicit
    # derivatives of the OCPs' KKT points, forward-mode tangents of plant and
    # CD-EKF, on the study's schedule (persistent: the closed loop records each
    # sample, then all lanes propagate the tangents through the records in
    # step).  Checked by central differences where that is
    # meaningful: OCPs solved to 1e-7 (a looser SQP lags the exact solution
    # map), steps 1e-2 of each weight, 2,000 trajectories x 24 samples, over
    # the trajectories whose OCPs all converged.
    ngrad = None
    if (not args.no_grad and w["nmpc"]["precision"] == "fp64" and
            w["nmpc"].get("nx_model", 1) != 3):
        cw = dict(w["nmpc"], Ru=0.2, Qn=1.0)
        if cw.get("schedule") == "persistent" and tuned_tps:
            cw["threads_per_sm"] = tuned_tps
        hg = mc.MonteCarlo(dict(w["model"], n_steps=min(24, w["model"]["n_steps"])), cw, j1,
                           w["seed"])
        for _ in range(max(1, args.warmup)):
            hg.nmpc_grad(stream, j0, j1)
        hg.sync()
        hg.close()
        hg = mc.MonteCarlo(w["model"], cw, j1, w["seed"])
        a_ev, b_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        flush.zero_()
        a_ev.record(stream)
        hg.nmpc_grad(stream, j0, j1)
        b_ev.record(stream)
        barrier()
        ng_ms = a_ev.elapsed_time(b_ev)
        ng_mean = hg.grad_mean()
        ng_st = hg.stats()
        hg.close()
        nf = min(2000, T)
        # the persistent schedule keeps the warps busy past OCPs that need
        # hundreds of iterations at this tolerance
        cf = dict(cw, sqp_tol=1e-7, sqp_max_it=100, schedule="persistent")
        cf.pop("threads_per_sm", None)
        hf = mc.MonteCarlo(dict(w["model"], n_steps=min(24, w["model"]["n_steps"])), cf, nf,
                           w["seed"])
        hf.nmpc_grad(stream)
        hf.sync()
        gf = hf.grad()
        okf = hf.counters()["n_ocp_failed"] == 0
        fdr = {}
        for kk in ("Qz", "Ru", "Qn"):
            hk = 1e-2 * cf[kk]
            for sgn in (1, -1):
                ww = {q: cf[q] for q in ("Qz", "Ru", "Qn")}
                ww[kk] += sgn * hk
                hf.set_nmpc_weights(ww["Qz"], ww["Ru"], ww["Qn"])
                hf.run(stream)
                hf.sync()
                fdr[(kk, sgn)] = hf.phi()
                okf &= hf.counters()["n_ocp_failed"] == 0
        hf.close()
        # per trajectory: Phi_j is piecewise smooth in the weights and a
        # difference that straddles an active-set change is no derivative
        fd_med, fd_frac, fd_med_all, fd_frac_all = [], [], [], []
        fin = np.isfinite(gf).all(axis=1)
        for q, kk in enumerate(("Qz", "Ru", "Qn")):
            hk = 1e-2 * cf[kk]
            fd_all = (fdr[(kk, 1)] - fdr[(kk, -1)]) / (2 * hk)
            t_all = gf[:, q]
            rel_all = np.abs(fd_all - t_all) / (np.abs(t_all) + 1e-2 * np.abs(t_all[fin]).max())
            rel = rel_all[okf]
            fd_med.append(float(np.median(rel)))
            fd_frac.append(float(np.mean(rel <= 5e-2)))
            fd_med_all.append(float(np.median(rel_all[fin])))
            fd_frac_all.append(float(np.mean(rel_all[fin] <= 5e-2)))
        if world > 1:
            t = torch.tensor([ng_ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ng_ms = float(t.item())
        ngrad = {"what": "d mean Phi / d(Q_z, R_u, Q_n) of the NMPC study (R_u = 0.2, "
                         "Q_n = 1), implicit OCP derivatives + forward-mode tangents",
                 "value": world * T / (ng_ms / 1e3), "unit": "trajectories/s (with tangents)",
                 "ms_per_step": ng_ms, "phi_mean": ng_st["phi_mean"],
                 "schedule": cw.get("schedule", "static"),
                 "threads_per_sm": cw.get("threads_per_sm"),
                 "grad_mean": ng_mean.tolist(),
                 "ocps_without_sensitivity": ng_st["qp_fail"],
                 "fd_check": {"trajectories": int(okf.sum()), "of": nf, "n_steps": 24,
                              "sqp_tol": 1e-7, "h_rel": 1e-2, "median_rel_err": fd_med,
                              "frac_within_5e-2": fd_frac,
                              "all_trajectories": {
                                  "trajectories": int(fin.sum()),
                                  "note": "every trajectory, including those with an OCP "
                                          "at the iteration limit in one of the seven runs",
                                  "median_rel_err": fd_med_all,
                                  "frac_within_5e-2": fd_frac_all}}}

    # end to end through the C ABI with host buffers: create (config h2d),
    # run, stats and Phi copied back to host, destroy
    e2e_ms = []
    for _ in range(0 if args.no_e2e else max(1, min(args.steps, 2))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hn = mc.MonteCarlo(w["model"], w["nmpc"], j1, w["seed"])
        hn.run(stream, j0, j1)
        hp = None
        if w["pi"] is not None:
            hp = mc.MonteCarlo(w["model"], w["pi"], j1, w["seed"])
            hp.run(stream, j0, j1)
        phi_n = hn.phi(j0, T)
        sn = hn.stats()
        if hp is not None:
            phi_p = hp.phi(j0, T)
            hp.stats()
            hp.close()
        hn.close()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_ms_step = statistics.mean(e2e_ms) if e2e_ms else float("nan")
    if world > 1:
        t = torch.tensor([e2e_ms_step], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms_step = float(t.item())
    h2d = 2 * (8 * len(w["model"]["sp_time"]) * 2 + 400)
    d2h = 8 * T * (2 if w["pi"] is not None else 1) + 2 * 2400

    st_pall = shards.allgather_stats(h_p.stats(), dist if world > 1 else None) \
        if h_p is not None else None
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "trajectories/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic",
                "config": {"workload": args.workload, "n_traj_nmpc": T,
                           "n_traj_pi": T if w["pi"] is not None else 0,
                           "n_steps": w["model"]["n_steps"], "N": w["nmpc"]["N"],
                           "precision": w["nmpc"]["precision"],
                           "qp_solver": w["nmpc"]["qp_solver"],
                           "schedule": w["nmpc"].get("schedule", "static"),
                           "threads_per_sm": tuned_tps,
                           "l2": "512 MB buffer written between timed steps",
                           "parallelism": f"trajectory shards x{world}"},
                "nmpc_ms_per_step": statistics.mean(nmpc_ms),
                "ocp_stats": {k: st_all[k] for k in ("n_ocp", "n_ocp_failed", "n_ls_fail",
                                                     "sqp_iters", "ls_trials", "qp_iters",
                                                     "n_hess_reset")},
                "phi": {"nmpc_mean": st_all["phi_mean"], "nmpc_var": st_all["phi_var"],
                        "n_traj": st_all["n_traj"]},
                "gpu_launches": args.steps * (3 + (3 if h_p is not None else 0)),
                "roofline": roofline,
                "clocks": clk, "wall_s_timed": wall,
                "e2e": {"value": world * T / (e2e_ms_step / 1e3), "unit": "trajectories/s",
                        "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}}
        if h_p is not None:
            line["phi"].update(pi_mean=st_pall["phi_mean"], pi_var=st_pall["phi_var"])
        if mixed is not None:
            line["mixed"] = mixed
        if cfg3 is not None:
            line["mixed_100k_N30"] = cfg3
        if paper_ctx is not None:
            line["paper_setting"] = paper_ctx
        line["peaks"] = {k: pk[k] for k in ("fp64_tflops", "fp32_tflops")} | {"source": pk_src}
        if grad is not None:
            line["pi_grad"] = grad
        if ngrad is not None:
            line["nmpc_grad"] = ngrad
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args.workload)
            if paper_ctx is not None:
                line["paper_setting"]["oracle"] = cpu_baseline_nmpc("cstr_paper_30k_x600_N60")
        print(json.dumps(line), flush=True)
    h_n.close()
    if h_p is not None:
        h_p.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
