"""The benchmark's bookkeeping, on the host: the algorithmic work of an NMPC
launch from the oracle's per-event operation counts scales with the launch's
counters, and the per-warp record's summary (SM busy share, rounds, the
slowest trajectory) is computed as its definition says."""
import json
import os

import numpy as np
import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

W = {"exp_table": 9.4, "exp_lib": 18.0, "div": 5.4, "rcp": 4.4, "log": 34.8, "sqrt": 9.1,
     "sincospi": 32.3}
MODEL = {"n_steps": 240, "n_em": 10}
CTRL = {"N": 20, "n_rk4": 5}


def _stats(scale):
    return {"n_ocp": 7_200_000 * scale, "ls_trials": 35_759_051 * scale,
            "sqp_iters": 35_706_023 * scale, "qp_iters": 38_975_494 * scale}


def test_algorithmic_flops_scale_with_the_counters():
    with open(os.path.join(ROOT, "oracle", "opcounts.json")) as fh:
        opc = json.load(fh)["nmpc"]
    f1 = bench.nmpc_algorithmic_flops(MODEL, CTRL, 30_000, _stats(1), W, opc)
    f2 = bench.nmpc_algorithmic_flops(MODEL, CTRL, 60_000, _stats(2), W, opc)
    assert f1 > 0 and f2 == pytest.approx(2 * f1, rel=1e-12)
    # the shooting dominates: at least the intervals times the oracle's
    # per-interval flops; with these counters (the bench's 30k x 240 study)
    # about 1.4e12 flops, 0.83 TFLOP/s over its 1.72 s launch
    per_interval = bench._flops(opc["events"]["rk4_interval"]["ops"], W)
    intervals = 30_000 * 20 + (7_200_000 - 30_000) * 2 + 35_759_051 * 20
    assert f1 > intervals * per_interval
    assert 1e12 < f1 < 2e12
    p1 = bench.nmpc_pipe_ops(MODEL, CTRL, 30_000, _stats(1), W)
    assert 0.5 < 2 * p1 / f1 < 1.5   # the kernel's formulation and the oracle's agree roughly


class _FakeHandle:
    def __init__(self):
        # 4 warps on 2 SMs: SM 0 busy 0..100 ns, SM 1 busy 10..60 ns
        self.tr = {"rounds": np.array([10, 20, 5, 8]), "lane_rounds": np.array([300, 600, 100, 200]),
                   "t_start_ns": np.array([0, 0, 10, 20]), "t_end_ns": np.array([50, 100, 60, 40]),
                   "sm": np.array([0, 0, 1, 1])}

    def warp_trace(self):
        return self.tr

    def counters(self):
        return {"ls_trials": np.array([3, 9, 4], dtype=np.int32),
                "n_ocp_failed": np.array([0, 1, 0], dtype=np.int32),
                "sqp_iters": np.array([3, 7, 4], dtype=np.int32)}


def test_warp_trace_summary():
    s = bench.warp_trace_summary(_FakeHandle(), n_steps=2)
    assert s["warps"] == 4 and s["sms"] == 2
    assert s["span_ms"] == pytest.approx(100e-6)
    assert s["sm_busy_frac"] == pytest.approx((100 + 50) / 2 / 100)
    assert s["rounds_max"] == 20 and s["rounds_mean"] == pytest.approx(10.75)
    assert s["lanes_per_round"] == pytest.approx(1200 / 43)
    assert s["last_warp"]["rounds"] == 20 and s["last_warp"]["ms"] == pytest.approx(100e-6)
    t = s["trajectory_starts_and_trials"]
    assert t["max"] == 11 and t["slowest"]["j"] == 1
    assert t["slowest"]["ocps_at_iteration_limit"] == 1
    assert t["trajectories_with_an_ocp_at_the_limit"] == 1
