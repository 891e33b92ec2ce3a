"""Operation counts of the oracle's closed loop, for the roofline's
algorithmic work.

TEST AND MEASUREMENT INFRASTRUCTURE ONLY (see oracle.h).  The oracle's C
sources are compiled a second time, as C++ with ``or_count.hpp`` forced in
first, so that every floating-point operation of the oracle is counted in the
category of the function it runs in (a marker is inserted at the top of the
shooting interval, the Euler-Maruyama substep, the two noise draws, the
CD-EKF prediction and filter, and the QP subproblem).  The arithmetic is the
oracle's own, unchanged.

Running it writes ``oracle/opcounts.json``: per-event operation counts of the
paper's method on the one-state CSTR closed loop --

* one shooting interval with forward sensitivities (N_c RK4 steps),
* one Euler-Maruyama substep of the plant and its three normals,
* one measurement normal, one CD-EKF prediction and one filter step,
* one NLP evaluation besides its shooting (objective, its gradient and the
  constraint residuals), which every OCP start and every line-search trial
  runs,
* the SQP's own work besides evaluations and QPs (Lagrangian gradients,
  damped block BFGS, convergence test, penalty update, merit, step) as a
  least-squares fit per OCP and per SQP iteration over the trajectories of
  the 100-trajectory workload,
* and the closed loop's own bookkeeping (set-points, Phi) per sample;

the QP subproblem is reported separately: the oracle condenses it into a
dense problem, which is not the structured (Riccati) work the method calls
for.

    python -m oracle.opcount      # writes oracle/opcounts.json
"""
from __future__ import annotations

import ctypes as C
import json
import os
import re
import shutil
import subprocess
import tempfile

import numpy as np

from . import Ctrl, Model, TrajOut, _SRC, make_ctrl, make_model

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle_count.so")
OUT = os.path.join(_HERE, "opcounts.json")
KINDS = ["add", "mul", "div", "sqrt", "exp", "log", "sin", "cos", "cmp", "minmax"]
CATS = ["other", "rk4_interval", "em_step", "process_noise", "meas_noise", "ekf_predict",
        "ekf_filter", "qp_solve", "evaluate", "sqp"]
# category markers: (source file, function definition prefix, category)
MARKERS = [("or_model.c", "void or_rk4_interval(", "ORC_RK4_INTERVAL"),
           ("or_model.c", "void or_em_step(", "ORC_EM_STEP"),
           ("or_model.c", "void or_ekf_predict(", "ORC_EKF_PREDICT"),
           ("or_model.c", "void or_ekf_filter(", "ORC_EKF_FILTER"),
           ("or_random.c", "void or_process_noise(", "ORC_PROCESS_NOISE"),
           ("or_random.c", "double or_meas_noise(", "ORC_MEAS_NOISE"),
           ("or_sqp.c", "int or_qp_solve(", "ORC_QP_SOLVE"),
           ("or_sqp.c", "static void evaluate(", "ORC_EVALUATE"),
           ("or_sqp.c", "static int sqp_impl(", "ORC_SQP")]
_COUNT_SRC = ["or_random.c", "or_model.c", "or_sqp.c", "or_closedloop.c", "or_nmpc3.c"]


def _insert_markers(text: str, fn: str) -> str:
    for f, head, cat in MARKERS:
        if f != fn:
            continue
        i = text.index("\n" + head) + 1
        j = text.index("{", i)
        text = text[: j + 1] + f"\n  OrcCat orc_guard_({cat});" + text[j + 1:]
    return text


def build(force: bool = False) -> str:
    srcs = [os.path.join(_HERE, s) for s in _COUNT_SRC] + [
        os.path.join(_HERE, "oracle.h"), os.path.join(_HERE, "or_count.hpp"),
        os.path.abspath(__file__)]
    if not force and os.path.exists(_SO):
        t = os.path.getmtime(_SO)
        if all(os.path.getmtime(s) <= t for s in srcs):
            return _SO
    d = tempfile.mkdtemp(prefix="orcount")
    try:
        shutil.copy(os.path.join(_HERE, "oracle.h"), d)
        shutil.copy(os.path.join(_HERE, "or_count.hpp"), d)
        for s in _COUNT_SRC:
            with open(os.path.join(_HERE, s)) as fh:
                text = fh.read()
            with open(os.path.join(d, s), "w") as fh:
                fh.write(_insert_markers(text, s))
        with open(os.path.join(d, "or_count_data.cpp"), "w") as fh:
            fh.write('#include "or_count.hpp"\n'
                     'extern "C" {\nuint64_t orc_ops[ORC_NCAT][ORC_NKIND];\n'
                     'uint64_t orc_calls[ORC_NCAT];\n'
                     'void orc_reset(void) { memset(orc_ops, 0, sizeof(orc_ops)); '
                     'memset(orc_calls, 0, sizeof(orc_calls)); }\n}\n'
                     'int orc_cat = ORC_OTHER;\n')
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["g++", "-O1", "-std=gnu++17", "-fPIC", "-shared", "-ffp-contract=off", "-w",
               "-include", os.path.join(d, "or_count.hpp"), "-x", "c++", "-o", tmp]
        cmd += [os.path.join(d, s) for s in _COUNT_SRC + ["or_count_data.cpp"]]
        cmd += ["-lm", "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    finally:
        shutil.rmtree(d, ignore_errors=True)
    return _SO


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.or_traj.argtypes = [C.POINTER(Model), C.POINTER(Ctrl), C.c_uint64, C.c_int64,
                              C.POINTER(TrajOut), C.POINTER(C.c_double)]
        L.orc_reset.argtypes = []
        _lib = L
    return _lib


def _read():
    L = lib()
    ops = np.ctypeslib.as_array((C.c_uint64 * (len(CATS) * len(KINDS))).in_dll(L, "orc_ops"))
    calls = np.ctypeslib.as_array((C.c_uint64 * len(CATS)).in_dll(L, "orc_calls"))
    return ops.reshape(len(CATS), len(KINDS)).astype(np.int64).copy(), calls.astype(np.int64).copy()


def count_traj(model: dict, ctrl: dict, seed: int, j: int):
    """(ops per category and kind, calls per category, TrajOut) of trajectory j,
    run by the counting build of the oracle (single thread)."""
    L = lib()
    m, c = make_model(model), make_ctrl(ctrl)
    out = TrajOut()
    L.orc_reset()
    L.or_traj(C.byref(m), C.byref(c), seed, j, C.byref(out), None)
    ops, calls = _read()
    return ops, calls, out


def per_event(model: dict, ctrl: dict, seed: int, n: int) -> dict:
    """Per-event operation counts (by kind) over trajectories 0..n-1."""
    tot = np.zeros((len(CATS), len(KINDS)), dtype=np.int64)
    calls = np.zeros(len(CATS), dtype=np.int64)
    rows, other = [], []
    for j in range(n):
        ops, cl, out = count_traj(model, ctrl, seed, j)
        tot += ops
        calls += cl
        rows.append([out.n_ocp, out.sqp_iters])
        other.append(ops[CATS.index("sqp")])
    res = {"trajectories": n, "kinds": KINDS, "events": {}}
    for ci, cat in enumerate(CATS):
        if cat == "sqp":
            continue
        if cat == "other":
            res["events"]["closed_loop_sample"] = {
                "calls": int(calls[CATS.index("ekf_filter")]),
                "ops": dict(zip(KINDS, (tot[0] / calls[CATS.index("ekf_filter")]).tolist()))}
            continue
        if calls[ci]:
            res["events"][cat] = {"calls": int(calls[ci]),
                                  "ops": dict(zip(KINDS, (tot[ci] / calls[ci]).tolist()))}
    # the SQP's own work per OCP and per SQP iteration
    X = np.array(rows, dtype=np.float64)
    Y = np.array(other, dtype=np.float64)
    coef, *_ = np.linalg.lstsq(X, Y, rcond=None)
    fit = X @ coef
    resid = np.max(np.abs(fit - Y).sum(axis=1) / np.maximum(1.0, Y.sum(axis=1)))
    res["sqp_rest"] = {"per_ocp": dict(zip(KINDS, coef[0].tolist())),
                       "per_sqp_iteration": dict(zip(KINDS, coef[1].tolist())),
                       "max_relative_residual": float(resid)}
    return res


def main():
    from paper_2212_02197_gb300 import workloads as W

    w = W.get("cstr_100x120_N20_fp64")
    res = {"workload": "cstr_100x120_N20_fp64 (100 NMPC trajectories, 120 steps, N = 20)",
           "nmpc": per_event(w["model"], w["nmpc"], w["seed"], w["n_traj"]),
           "note": "operations of the oracle's own formulation (or_count.hpp); the "
                   "qp_solve event is the oracle's condensed dense QP"}
    with open(OUT, "w") as fh:
        json.dump(res, fh, indent=1)
    print(json.dumps(res, indent=1))


if __name__ == "__main__":
    main()
