"""Mixed precision (plant SDE, noise transform, EKF prediction and OCP shooting
in FP32; Joseph update, QP pivots, merit, BFGS and the convergence test in
FP64) against FP64.

Acceptance is statistical: the mean of Phi within 0.5 % and the two-sample
Kolmogorov-Smirnov statistic of the Phi distributions below 0.01.  Both runs
use the same trajectories and noise (common random numbers), so the
per-trajectory errors are reported too."""
import numpy as np
import pytest

import oracle
from paper_2212_02197_gb300 import mc, workloads as W

pytestmark = pytest.mark.gpu


def _ks(a, b):
    from scipy import stats

    return stats.ks_2samp(a, b).statistic


def _run(w, ctrl, n):
    h = mc.MonteCarlo(w["model"], ctrl, n, w["seed"])
    h.run()
    st = h.stats(timeout_ms=1800000)
    phi = h.phi()
    h.close()
    return phi, st


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2212_02197_gb300 import _build

    _build.build()
    oracle.build()


def test_mixed_matches_fp64_on_the_paper_scale_study():
    w64 = W.get("cstr_30k_x240_N20_fp64")
    w32 = W.get("cstr_30k_x240_N20_mixed")
    n = w64["n_traj"]
    for kind in ("nmpc", "pi"):
        ref, st64 = _run(w64, w64[kind], n)
        phi, st32 = _run(w32, w32[kind], n)
        assert st32["n_nonfinite"] == 0
        assert abs(st32["phi_mean"] / st64["phi_mean"] - 1.0) < 5e-3
        assert _ks(phi, ref) < 1e-2
        rel = np.abs(phi - ref) / np.abs(ref)
        assert np.median(rel) < 1e-3
        if kind == "nmpc":
            assert st32["n_ocp"] == n * w32["model"]["n_steps"]
            # Table II analogue: no OCP runs into the iteration limit
            assert st32["n_ocp_failed"] <= 1e-4 * st32["n_ocp"]


def test_mixed_against_the_oracle_on_a_sample_of_the_100k_study():
    """The E_a-perturbed N = 30 study: the first 800 trajectories in mixed
    precision against the FP64 oracle on the same trajectories."""
    w = W.get("cstr_100k_x240_N30_mixed")
    n = 800
    phi, st = _run(w, w["nmpc"], n)
    ref = oracle.run(w["model"], dict(w["nmpc"], precision="fp64", sqp_tol=1e-5, ls_max=30),
                     w["seed"], 0, n)["phi"]
    fin = np.isfinite(ref) & np.isfinite(phi)
    assert fin.sum() >= 0.99 * n
    assert abs(np.mean(phi[fin]) / np.mean(ref[fin]) - 1.0) < 5e-3
    assert _ks(phi[fin], ref[fin]) < 2e-2   # 800 samples: sampling noise of KS is ~0.05
    assert np.median(np.abs(phi[fin] - ref[fin]) / np.abs(ref[fin])) < 1e-3


def test_mixed_pi_small_against_oracle():
    w = W.get("cstr_100x120_N20_fp64")
    c = dict(w["pi"], precision="mixed")
    phi, _ = _run(w, c, 100)
    ref = oracle.run(w["model"], w["pi"], w["seed"], 0, 100)["phi"]
    rel = np.abs(phi - ref) / np.abs(ref)
    assert np.max(rel) < 1e-3
