"""The operation-counting build of the oracle (oracle/opcount.py), whose
per-event counts give the roofline's algorithmic work.  It must compute
exactly what the oracle computes, count what the method evaluates per event,
and the stored counts must be the ones it produces."""
import json

import numpy as np
import pytest

import oracle
from oracle import opcount
from paper_2212_02197_gb300 import workloads as W

W1 = W.get("cstr_100x120_N20_fp64")


@pytest.mark.parametrize("kind", ["nmpc", "pi"])
def test_counting_build_computes_what_the_oracle_computes(kind):
    m = dict(W1["model"], n_steps=30)
    ref = oracle.run(m, W1[kind], W1["seed"], 0, 6, threads=1)
    for j in range(6):
        _, _, out = opcount.count_traj(m, W1[kind], W1["seed"], j)
        assert out.phi == ref["phi"][j]                # bit for bit
        assert out.sqp_iters == ref["sqp_iters"][j]


def test_counts_per_event_follow_the_method():
    """Per shooting interval 4 N_c rate-law exponentials; per Euler-Maruyama
    substep one exponential and one square root; three normals per substep
    (two Box-Muller pairs: two logs, square roots, sines and cosines), one per
    measurement; one exponential per rate-law evaluation of the CD-EKF
    prediction; no elementary function in the filter or the QP."""
    m = dict(W1["model"], n_steps=12)
    res = opcount.per_event(m, W1["nmpc"], W1["seed"], 4)
    ev = res["events"]
    nrk = W1["nmpc"]["n_rk4"]
    assert ev["rk4_interval"]["ops"]["exp"] == 4 * nrk
    assert ev["em_step"]["ops"]["exp"] == 1 and ev["em_step"]["ops"]["sqrt"] == 1
    for k in ("log", "sqrt", "sin", "cos"):
        assert ev["process_noise"]["ops"][k] == 2
        assert ev["meas_noise"]["ops"][k] == 1
    assert ev["ekf_predict"]["ops"]["exp"] == 4 * nrk
    assert ev["ekf_filter"]["ops"]["exp"] == 0
    assert ev["qp_solve"]["ops"]["exp"] == 0
    assert ev["evaluate"]["ops"]["exp"] == 0
    # one counted call per event
    K = m["n_steps"]
    assert ev["em_step"]["calls"] == 4 * K * m["n_em"]
    assert ev["meas_noise"]["calls"] == 4 * K
    assert res["sqp_rest"]["max_relative_residual"] < 0.01


def test_stored_counts_are_the_counting_builds():
    with open(opcount.OUT) as fh:
        stored = json.load(fh)["nmpc"]
    fresh = opcount.per_event(W1["model"], W1["nmpc"], W1["seed"], 8)
    for ev in ("rk4_interval", "em_step", "process_noise", "meas_noise", "ekf_predict",
               "ekf_filter", "evaluate"):
        for k, v in fresh["events"][ev]["ops"].items():
            assert stored["events"][ev]["ops"][k] == pytest.approx(v, rel=1e-12, abs=1e-12), (ev, k)
    assert stored["trajectories"] == W1["n_traj"]
