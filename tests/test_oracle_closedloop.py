"""Closed-loop checks of the oracle (Sec. VII): counting identities of Table II,
the qualitative result of Sec. VII-C (NMPC beats PI in mean and variance of
Phi), common random numbers, and independence of the result from how the
trajectories are split over threads."""
import numpy as np
import pytest

import oracle
from paper_2212_02197_gb300 import workloads as W


@pytest.fixture(scope="module")
def small():
    w = W.get("cstr_100x120_N20_fp64")
    n = 32
    r_n = oracle.run(w["model"], w["nmpc"], w["seed"], 0, n)
    r_p = oracle.run(w["model"], w["pi"], w["seed"], 0, n)
    return w, r_n, r_p


def test_total_ocps_equals_trajectories_times_steps(small):
    w, r_n, r_p = small
    K = w["model"]["n_steps"]
    assert np.all(r_n["n_ocp"] == K)
    assert r_n["n_ocp"].sum() == len(r_n["phi"]) * K
    assert np.all(r_p["n_ocp"] == 0)


def test_nmpc_outperforms_pi_in_mean_and_variance(small):
    _, r_n, r_p = small
    assert r_n["phi"].mean() < r_p["phi"].mean()
    assert r_n["phi"].var() < r_p["phi"].var()
    assert np.all(np.isfinite(r_n["phi"])) and np.all(np.isfinite(r_p["phi"]))


def test_failed_ocp_fraction_is_small():
    """Table II: a tiny fraction of the OCPs hits the iteration limit."""
    w = W.get("cstr_30k_x240_N20_fp64")
    r = oracle.run(w["model"], w["nmpc"], w["seed"], 0, 24)
    frac = r["n_ocp_failed"].sum() / r["n_ocp"].sum()
    assert frac < 1e-3
    assert r["n_ls_fail"].sum() == 0


def test_split_and_thread_count_do_not_change_results():
    w = W.get("cstr_100x120_N20_fp64")
    one = oracle.run(w["model"], w["nmpc"], w["seed"], 0, 12, threads=1)
    a = oracle.run(w["model"], w["nmpc"], w["seed"], 0, 5, threads=3)
    b = oracle.run(w["model"], w["nmpc"], w["seed"], 5, 12, threads=2)
    for f in oracle.TRAJ_FIELDS:
        assert np.array_equal(one[f], np.concatenate([a[f], b[f]]))


def test_common_random_numbers_between_controllers():
    """NMPC and PI trajectories with the same seed and index see the same
    measurement noise: their first measurements coincide."""
    w = W.get("cstr_100x120_N20_fp64")
    for j in (0, 7):
        tn = oracle.traj(w["model"], w["nmpc"], w["seed"], j, with_trace=True)["trace"]
        tp = oracle.traj(w["model"], w["pi"], w["seed"], j, with_trace=True)["trace"]
        assert tn[0, 0] == tp[0, 0] and tn[0, 1] == tp[0, 1]
    a = oracle.traj(w["model"], w["pi"], w["seed"], 0)["phi"]
    b = oracle.traj(w["model"], w["pi"], w["seed"], 1)["phi"]
    assert a != b


def test_noise_free_nmpc_tracks_all_setpoints():
    """Sec. VII-A: the NMPC tracks stable and unstable steady states.  With
    negligible noise the plant settles at each reachable set-point."""
    w = W.get("cstr_30k_x240_N20_fp64")
    m = dict(w["model"])
    m["sigma"] = [1e-9, 1e-9, 1e-9]
    m["meas_sd"] = 1e-6
    m["dTin_step"] = 0.0
    tr = oracle.traj(m, w["nmpc"], w["seed"], 0, with_trace=True)["trace"]
    Tplant = tr[:, 0]
    # the unstable 290 K steady state is held from 50 s until the 340 K set-point
    # enters the 10 s horizon at 70 s; 340 K is held from 100 s to the end
    assert np.all(np.abs(Tplant[100:140] - 290.0) < 0.02)
    assert np.all(np.abs(Tplant[200:240] - 340.0) < 0.02)
    # the 282 K set-point is reached before the anticipation of 290 K begins
    assert np.min(np.abs(Tplant[60:68] - 282.0)) < 0.1


def test_trajectory_parameters():
    """Inlet-temperature step at a uniform time in [t0, tf) with a +-5 K sign,
    and a median-preserving lognormal E_a/R."""
    w = W.get("cstr_30k_x240_N20_fp64")
    m = w["model"]
    tds, signs = [], []
    for j in range(400):
        EaR, td, dT = oracle.traj_params(m, 3, j)
        assert EaR == m["EaR"]
        assert 0.0 <= td < m["n_steps"] * m["Ts"]
        assert abs(dT) == 5.0
        tds.append(td)
        signs.append(dT > 0)
    assert 0.4 < np.mean(signs) < 0.6
    assert abs(np.mean(tds) / (m["n_steps"] * m["Ts"]) - 0.5) < 0.06
    m3 = W.get("cstr_100k_x240_N30_mixed")["model"]
    logs = np.log([oracle.traj_params(m3, 3, j)[0] / m3["EaR"] for j in range(2000)])
    assert abs(np.std(logs) - 0.02) < 0.002 and abs(np.mean(logs)) < 0.002


def test_degenerate_filter_is_reported_not_hidden():
    """Without measurement and process noise the filter gain is 0/0; the
    trajectory is flagged non-finite and its Phi is NaN."""
    w = W.get("cstr_100x120_N20_fp64")
    m = dict(w["model"])
    m["sigma"] = [0.0, 0.0, 0.0]
    m["meas_sd"] = 0.0
    r = oracle.traj(m, w["nmpc"], w["seed"], 0)
    assert r["nonfinite"] == 1 and np.isnan(r["phi"])


def test_uneven_horizon_draw():
    """Uneven batches: the horizon is uniform on N_min..N and the SQP limit on
    sqp_max_it_min..sqp_max_it, independently per trajectory."""
    c = W.get("cstr_262k_x120_N10to40_uneven")["nmpc"]
    Ns, its = zip(*[oracle.traj_horizon(c, 9, j) for j in range(6200)])
    Ns, its = np.array(Ns), np.array(its)
    assert Ns.min() == 10 and Ns.max() == 40 and its.min() == 5 and its.max() == 30
    cnt = np.bincount(Ns - 10, minlength=31)
    assert np.all(np.abs(cnt - 200) < 5 * np.sqrt(200))
    assert abs(np.corrcoef(Ns, its)[0, 1]) < 0.05
    c_fixed = W.nmpc(20)
    assert oracle.traj_horizon(c_fixed, 9, 5) == (20, 100)


def test_uneven_trajectory_uses_its_horizon():
    """A trajectory's OCPs use its own iteration limit: with a limit of 5 no OCP
    takes more than 5 QPs."""
    w = W.get("cstr_262k_x120_N10to40_uneven")
    m = dict(w["model"], n_steps=20)
    c = dict(w["nmpc"], sqp_max_it=5, sqp_max_it_min=5)
    r = oracle.run(m, c, w["seed"], 0, 6)
    assert np.all(r["sqp_iters"] <= 5 * 20)


# ------------------------------------------------------------------ model mismatch

def test_mismatch_first_input_is_the_nominal_controllers():
    """With the E_a/R perturbation in the plant only, the controller sees at
    sample 0 only the initial state and the measurement, so its first input is
    the one of the unperturbed study, bit for bit; when the controller knows
    the trajectory's E_a/R (the default) the first input moves with it."""
    w = W.get("cstr_30k_x240_N20_fp64_mismatch")
    m_mis = dict(w["model"], n_steps=3)
    m_nom = dict(m_mis, Ea_logsd=0.0)
    m_known = dict(m_mis, Ea_plant_only=False)
    # the first sample's (applied input, SQP iterations of its OCP); the NMPC's
    # first inputs sit on the lower bound, its iteration counts still differ
    for kind in ("nmpc", "pi"):
        moved_known, moved_later = [], []
        for j in (0, 1, 2):
            t_mis = oracle.traj(m_mis, w[kind], w["seed"], j, with_trace=True)["trace"]
            t_nom = oracle.traj(m_nom, w[kind], w["seed"], j, with_trace=True)["trace"]
            t_kn = oracle.traj(m_known, w[kind], w["seed"], j, with_trace=True)["trace"]
            assert np.array_equal(t_mis[0, 3:5], t_nom[0, 3:5]), (kind, j)
            moved_known.append(not np.array_equal(t_kn[0, 3:5], t_nom[0, 3:5]))
            # from sample 1 on, the perturbed plant has moved the measurement
            moved_later.append(t_mis[1, 1] != t_nom[1, 1])
        assert all(moved_known) and all(moved_later), (kind, moved_known, moved_later)


def test_mismatch_flag_is_inert_without_perturbation():
    w = W.get("cstr_100x120_N20_fp64")
    m = dict(w["model"], n_steps=20)
    for kind in ("nmpc", "pi"):
        a = oracle.run(m, w[kind], w["seed"], 0, 6)["phi"]
        b = oracle.run(dict(m, Ea_plant_only=True), w[kind], w["seed"], 0, 6)["phi"]
        assert np.array_equal(a, b)
