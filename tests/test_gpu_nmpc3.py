"""The three-state NMPC (3x3 CD-EKF, three states per OCP stage, Riccati
QP with a 3x3 Riccati matrix) on the GPU against the oracle's three-state
NMPC (condensed dense QP)."""
import numpy as np
import pytest

import oracle
from paper_2212_02197_gb300 import mc, workloads as W

pytestmark = pytest.mark.gpu

WL = "cstr_30k_x240_N20_fp64_nx3"


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2212_02197_gb300 import _build

    _build.build()
    oracle.build()


def _run(m, c, n, seed):
    h = mc.MonteCarlo(m, c, n, seed)
    h.run()
    st = h.stats(timeout_ms=600000)
    phi, cnt = h.phi(), h.counters()
    h.close()
    return phi, cnt, st


def test_first_ocp_matches_oracle():
    """One control step: Phi depends on the first OCP's input only, and the
    SQP iteration counts of that OCP are compared too."""
    w = W.get(WL)
    m = dict(w["model"], n_steps=1)
    n = 200
    phi, cnt, _ = _run(m, w["nmpc"], n, w["seed"])
    ref = oracle.run(m, w["nmpc"], w["seed"], 0, n)
    np.testing.assert_allclose(phi, ref["phi"], rtol=1e-9, atol=0)
    assert np.mean(np.abs(cnt["sqp_iters"] - ref["sqp_iters"]) <= 1) >= 0.95


@pytest.mark.parametrize("sched", ["persistent", "static"])
def test_closed_loop_matches_oracle_tight(sched):
    """The parity bar of the FP64 path, 1e-6 relative in Phi: 64 trajectories
    x 60 steps with the T_in step and every OCP solved to 1e-8 on the scaled
    KKT test (200 SQP iterations at most), where both implementations end at
    the same KKT point up to the rounding floor of the merit function.

    * Every trajectory whose OCPs all converged on both sides: within 1e-6.
    * Every trajectory, with no exception: within 1e-5.  At this tolerance the
      three-state SQP often stalls at the merit's rounding floor; where one
      side's line search runs out of halvings and the other's runs on to the
      iteration limit, the two stop at different iterates of the floor.
      Trajectory 37 is the one case here: at its sample 25 the oracle's line
      search fails after 543 SQP iterations in all, the GPU's runs to the
      limit, and Phi moves by 1.26e-6.
    * At least 95 % of all within 1e-6, the median within 1e-8."""
    w = W.get(WL)
    m = dict(w["model"], n_steps=60)
    c = dict(w["nmpc"], sqp_tol=1e-8, sqp_max_it=200, schedule=sched)
    n = 64
    phi, cnt, st = _run(m, c, n, w["seed"])
    ref = oracle.run(m, c, w["seed"], 0, n)
    rel = np.abs(phi - ref["phi"]) / np.abs(ref["phi"])
    stalled = ((ref["n_ocp_failed"] > 0) | (cnt["n_ocp_failed"] > 0) |
               (ref["n_ls_fail"] > 0) | (cnt["n_ls_fail"] > 0))
    assert np.all(rel[~stalled] <= 1e-6), (rel[~stalled].max(), int(np.argmax(np.where(stalled, 0, rel))))
    assert np.all(rel <= 1e-5), (rel.max(), int(np.argmax(rel)))
    assert np.mean(rel <= 1e-6) >= 0.95, np.sort(rel)[-5:]
    assert np.median(rel) <= 1e-8
    assert st["n_nonfinite"] == 0


def test_closed_loop_matches_oracle():
    """A secondary check at the workload's own tolerance: 160 trajectories
    (5 warps), 60 steps, with the T_in step.  Each OCP stops at the scaled KKT
    tolerance 1e-5 (Sec. IV, Eq. (convergence)); two FP64 implementations that
    differ in rounding can stop at different iterates inside it, after 9.5 SQP
    iterations per OCP on average.  So: every trajectory whose OCPs all
    converged within 1e-5 relative in Phi, 95 % of them within 1e-6, and those
    with an OCP at the iteration limit within 1e-3.  The 1e-6 bar itself is
    held by the tight-tolerance test above."""
    w = W.get(WL)
    m = dict(w["model"], n_steps=60)
    n = 160
    phi, cnt, st = _run(m, w["nmpc"], n, w["seed"])
    ref = oracle.run(m, w["nmpc"], w["seed"], 0, n)
    rel = np.abs(phi - ref["phi"]) / np.abs(ref["phi"])
    hit = (ref["n_ocp_failed"] > 0) | (cnt["n_ocp_failed"] > 0)
    assert np.all(rel[~hit] <= 1e-5), (rel[~hit].max(), np.argmax(np.where(hit, 0, rel)))
    assert np.mean(rel[~hit] <= 1e-6) >= 0.95, np.sort(rel[~hit])[-10:]
    assert np.all(rel[hit] <= 1e-3)
    assert st["n_ocp"] == n * 60 and st["n_nonfinite"] == 0
    # the total SQP effort agrees closely
    assert abs(cnt["sqp_iters"].sum() / ref["sqp_iters"].sum() - 1.0) < 0.02


def test_full_study_sampled():
    """The full three-state study (30,000 trajectories, 240 steps, the
    workload's persistent schedule) in one launch; 48 trajectories spread over
    the index range against the oracle, with the tolerances of the 60-step
    test (OCPs stop at the scaled KKT tolerance 1e-5, Sec. IV)."""
    w = W.get(WL)
    n = w["n_traj"]
    phi, cnt, st = _run(w["model"], w["nmpc"], n, w["seed"])
    assert st["n_traj"] == n and st["n_nonfinite"] == 0
    assert st["n_ocp"] == n * w["model"]["n_steps"]
    assert st["n_ocp_failed"] <= 1e-3 * st["n_ocp"]
    sample = np.unique(np.linspace(0, n - 1, 48).astype(int))
    refs = [oracle.run(w["model"], w["nmpc"], w["seed"], int(j), int(j) + 1, threads=1)
            for j in sample]
    ref_phi = np.concatenate([r["phi"] for r in refs])
    ref_fail = np.concatenate([r["n_ocp_failed"] for r in refs])
    rel = np.abs(phi[sample] - ref_phi) / np.abs(ref_phi)
    hit = (ref_fail > 0) | (cnt["n_ocp_failed"][sample] > 0)
    assert np.all(rel[~hit] <= 1e-5), (rel[~hit].max(), sample[np.argmax(np.where(hit, 0, rel))])
    assert np.mean(rel[~hit] <= 1e-6) >= 0.9, np.sort(rel[~hit])[-8:]
    assert np.all(rel[hit] <= 1e-3)


def test_three_state_and_one_state_controllers_agree_roughly():
    """Both control the same plant; with the plant near the reaction-invariant
    manifold they track alike (mean Phi within 5 %)."""
    w = W.get("cstr_100x120_N20_fp64")
    m = dict(w["model"], n_steps=60)
    phi3, _, _ = _run(m, dict(w["nmpc"], nx_model=3, schedule="static"), 96, w["seed"])
    phi1, _, _ = _run(m, w["nmpc"], 96, w["seed"])
    assert abs(phi3.mean() / phi1.mean() - 1.0) < 0.05


def test_persistent_schedule_is_bit_identical_to_static():
    """The persistent schedule (per-lane phases, a shooting pool per round)
    runs the same arithmetic per trajectory as the static one; with
    threads_per_sm = 1 fewer lanes than trajectories exercise the queue."""
    w = W.get(WL)
    m = dict(w["model"], n_steps=12)
    out = {}
    for sched, tps in (("static", 0), ("persistent", 0), ("persistent", 1)):
        h = mc.MonteCarlo(m, dict(w["nmpc"], schedule=sched, threads_per_sm=tps), 200,
                          w["seed"])
        h.run()
        h.sync()
        out[(sched, tps)] = (h.phi(), h.counters())
        h.close()
    ref_phi, ref_cnt = out[("static", 0)]
    for key in (("persistent", 0), ("persistent", 1)):
        phi, cnt = out[key]
        assert np.array_equal(phi, ref_phi), key
        for k in ref_cnt:
            assert np.array_equal(cnt[k], ref_cnt[k]), (key, k)


def test_three_state_validation():
    w = W.get(WL)
    base = w["nmpc"]
    for bad in (dict(precision="mixed"), dict(qp_solver="ipm"), dict(nx_model=2)):
        with pytest.raises(mc.McError):
            mc.MonteCarlo(w["model"], dict(base, **bad), 4, w["seed"])
