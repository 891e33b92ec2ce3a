"""Measured throughput of the arithmetic pipes the closed loop runs on.

The FP64 path is bound by the FP64 pipe, which GB300 gives far fewer units
than FP32 (nominally 2 fused multiply-adds per SM per clock).  Its roofline
therefore needs a measured FP64 peak and the cost, in FP64 fused
multiply-adds, of each elementary operation the method evaluates (exp of the
rate law, division, the rate law's reciprocal, and log, sqrt and sincospi of
the Box-Muller transform).
All of them come from ``mc_pipe_probe`` (include/mc.h), timed on the device.

    python -m paper_2212_02197_gb300.peaks     # prints the JSON record
"""
from __future__ import annotations

import json

from . import mc

KINDS = {"dfma": 0, "none": 1, "exp_table": 2, "exp_lib": 3, "div": 4, "log": 5,
         "sqrt": 6, "sincospi": 7, "ffma": 8, "expf": 9, "none_f32": 10, "rcp": 11}


def probe(kind: str, iters: int) -> float:
    """Seconds per chain step of the probe ``kind``."""
    ms, steps = mc.pipe_probe(KINDS[kind], iters)
    return ms * 1e-3 / steps


def measure(iters: int = 1 << 14, repeats: int = 3) -> dict:
    """FP64 and FP32 fused-multiply-add peaks (TFLOP/s, 2 flops per fma) and
    the cost of each elementary operation in FP64 fma equivalents (FP32 expf
    in FP32 fma equivalents).  The best of `repeats` launches per probe."""
    t = {}
    for k in KINDS:
        n = iters if k in ("dfma", "none", "ffma", "none_f32", "expf") else iters // 4
        t[k] = min(probe(k, n) for _ in range(repeats))
    w = {k: (t[k] - t["none"]) / t["dfma"]
         for k in ("exp_table", "exp_lib", "div", "rcp", "log", "sqrt", "sincospi")}
    w["expf_ffma"] = (t["expf"] - t["none_f32"]) / t["ffma"]
    return {"fp64_fma_per_s": 1.0 / t["dfma"], "fp64_tflops": 2.0 / t["dfma"] / 1e12,
            "fp32_fma_per_s": 1.0 / t["ffma"], "fp32_tflops": 2.0 / t["ffma"] / 1e12,
            "weights_dfma": w,
            "how": "mc_pipe_probe: 16 four-warp blocks per SM, 8 independent chains per "
                   "thread; op cost = (t(fma + op) - t(fma + add)) / t(fma)"}


if __name__ == "__main__":
    print(json.dumps(measure()))
