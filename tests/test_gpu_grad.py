"""The discrete adjoint of the PI closed loop (mc_pi_grad) against the oracle's
complex-step derivative, finite differences of the GPU's own mean Phi, and the
invariances the checkpointing must keep."""
import numpy as np
import pytest
import torch

import oracle
from paper_2212_02197_gb300 import mc, workloads as W
from paper_2212_02197_gb300.autograd import pi_mean_phi

pytestmark = pytest.mark.gpu

WL = "cstr_30k_x240_N20_fp64"   # 240 samples, inlet step +-5 K at a random time


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2212_02197_gb300 import _build

    _build.build()
    oracle.build()


def _grad(w, n, ckpt=20, ctrl=None, model=None):
    h = mc.MonteCarlo(model or w["model"], ctrl or w["pi"], n, w["seed"])
    h.pi_grad(ckpt)
    st = h.stats(timeout_ms=600000)
    g, phi, gm = h.grad(), h.phi(), h.grad_mean()
    h.close()
    return phi, g, gm, st


def test_adjoint_matches_complex_step_per_trajectory():
    w = W.get(WL)
    n = 300   # spans 3 blocks of 128 and a ragged tail
    phi, g, _, _ = _grad(w, n)
    ref_phi, ref = oracle.pi_grad(w["model"], w["pi"], w["seed"], 0, n)
    np.testing.assert_allclose(phi, ref_phi, rtol=1e-12, atol=0)
    scale = np.abs(ref).mean(axis=0)
    err = np.abs(g - ref) / (np.abs(ref) + 1e-6 * scale)
    assert np.all(np.isfinite(g))
    assert err.max() < 1e-8, err.max()


def test_adjoint_on_a_sample_of_the_full_study():
    """The full 30k launch; trajectories sampled across it against the oracle."""
    w = W.get(WL)
    n = w["n_traj"]
    _, g, gm, st = _grad(w, n)
    assert st["n_nonfinite"] == 0
    idx = np.linspace(0, n - 1, 40).astype(int)
    for j in idx:
        _, ref = oracle.pi_grad(w["model"], w["pi"], w["seed"], int(j), int(j) + 1)
        np.testing.assert_allclose(g[j], ref[0], rtol=1e-8, atol=1e-8 * np.abs(ref).max())
    np.testing.assert_allclose(gm, g.mean(axis=0), rtol=1e-12)


def test_checkpoint_interval_does_not_change_the_result():
    w = W.get(WL)
    _, g20, _, _ = _grad(w, 64, 20)
    for ck in (1, 7, 32):
        _, g, _, _ = _grad(w, 64, ck)
        assert np.array_equal(g, g20), ck


def test_phi_equals_the_plain_run():
    w = W.get(WL)
    phi, _, _, _ = _grad(w, 256)
    h = mc.MonteCarlo(w["model"], w["pi"], 256, w["seed"])
    h.run()
    ref = h.phi()
    h.close()
    np.testing.assert_allclose(phi, ref, rtol=1e-12, atol=0)


# central differences of mean Phi over the 30k study: step (relative to the
# gain) and the relative tolerance per gain (k_P, k_I, k_aw).  A trajectory
# whose input crosses a bound of the clip between k - h and k + h has a kink
# inside the difference interval and contributes an O(1) error to its own
# difference quotient; the anti-windup derivative, which is small, feels this
# most (the oracle's own differences are 5e-4 off there at h = 1e-5).  At
# h = 1e-6 the rounding of mean Phi (~229) over 2h adds its share.
FD_CASES = [(1e-5, (1e-4, 1e-4, 2e-3)), (1e-6, (1e-5, 1e-5, 1e-4))]


@pytest.mark.parametrize("step,tols", FD_CASES)
def test_mean_gradient_matches_central_differences_of_mean_phi(step, tols):
    w = W.get(WL)
    n = w["n_traj"]
    _, _, gm, _ = _grad(w, n)
    h = mc.MonteCarlo(w["model"], w["pi"], n, w["seed"])
    c = w["pi"]
    for q, k in enumerate(("kP", "kI", "kaw")):
        dk = step * abs(c[k])
        means = []
        for sgn in (1, -1):
            g = dict(kP=c["kP"], kI=c["kI"], kaw=c["kaw"])
            g[k] += sgn * dk
            h.set_pi_gains(g["kP"], g["kI"], g["kaw"])
            h.run()
            means.append(h.stats()["phi_mean"])
        fd = (means[0] - means[1]) / (2 * dk)
        assert fd == pytest.approx(gm[q], rel=tols[q]), (k, fd, gm[q])
    h.close()


def test_autograd_function():
    w = W.get(WL)
    h = mc.MonteCarlo(w["model"], w["pi"], 512, w["seed"])
    c = w["pi"]
    x = torch.tensor([c["kP"], c["kI"], c["kaw"]], dtype=torch.float64, requires_grad=True)
    y = pi_mean_phi(x, h)
    y.backward()
    gm = h.grad_mean()
    h.close()
    assert torch.allclose(x.grad, torch.tensor(gm, dtype=torch.float64), rtol=0, atol=0)
    _, _, gm2, st = _grad(w, 512)
    assert float(y) == pytest.approx(st["phi_mean"], rel=1e-15)


def test_edge_cases_and_errors():
    w = W.get(WL)
    # no control steps: Phi = (c_T(0) - z-bar(0))^2, which no gain moves
    phi, g, _, _ = _grad(w, 40, model=dict(w["model"], n_steps=0))
    assert np.all(g == 0.0) and np.all(np.isfinite(phi))
    # one step, checkpoint interval longer than the run
    _, g1, _, _ = _grad(w, 40, 32, model=dict(w["model"], n_steps=1))
    _, r1 = oracle.pi_grad(dict(w["model"], n_steps=1), w["pi"], w["seed"], 0, 40)
    np.testing.assert_allclose(g1, r1, rtol=1e-9, atol=1e-12)
    # empty range
    h = mc.MonteCarlo(w["model"], w["pi"], 10, w["seed"])
    with pytest.raises(mc.McError):
        h.grad_mean()                       # not run yet
    h.pi_grad(20, j0=3, j1=3)
    assert np.all(h.grad_mean() == 0.0)
    for bad in (0, 33):
        with pytest.raises(mc.McError):
            h.pi_grad(bad)
    with pytest.raises(mc.McError):
        h.set_pi_gains(float("nan"), 0.0, 0.0)
    h.close()
    with pytest.raises(mc.McError):
        _grad(w, 4, model=dict(w["model"], n_em=33))
    hn = mc.MonteCarlo(w["model"], w["nmpc"], 4, w["seed"])
    with pytest.raises(mc.McError):
        hn.pi_grad(20)
    with pytest.raises(mc.McError):
        hn.set_pi_gains(-1e-3, -1e-4, -1e-1)
    hn.close()
    hm = mc.MonteCarlo(w["model"], dict(w["pi"], precision="mixed"), 4, w["seed"])
    with pytest.raises(mc.McError):
        hm.pi_grad(20)
    hm.close()


# ------------------------------------------------------------------ NMPC weights

from paper_2212_02197_gb300.autograd import nmpc_mean_phi  # noqa: E402

WN = "cstr_100x120_N20_fp64"


def _ocp_cases(n, N, rng):
    """OCPs from the oracle's SQP whose first input is interior."""
    m = W.model(240)
    c = dict(W.nmpc(N), Ru=0.3, Qn=2.0)
    out = []
    while len(out) < n:
        z = rng.choice([282.0, 290.0, 300.0, 340.0])
        x0 = z + rng.uniform(0.2, 2.0)
        zb = np.full(N + 1, z)
        u, x, lam, pil, piu, info = oracle.sqp(m, c, m["EaR"], x0, zb, np.full(N, 0.5),
                                               np.full(N + 1, x0))
        if info["status"] == 0 and 0.0 < u[0] < 1.0:
            out.append((x0, zb, u, x, lam, pil, piu))
    return m, c, out


def test_ocp_sensitivity_matches_oracle():
    """The GPU's second-order shooting sensitivities and Riccati sweep against
    the oracle's difference Hessian and dense KKT solve, on the same KKT
    points."""
    rng = np.random.default_rng(21)
    N = 20
    m, c, cases = _ocp_cases(24, N, rng)
    cols = list(zip(*cases))
    sens, st = mc.ocp_sens_batch(m, c, np.array(cols[0]), m["EaR"], np.array(cols[1]),
                                 np.array(cols[2]), np.array(cols[3]), np.array(cols[4]),
                                 np.array(cols[5]), np.array(cols[6]))
    assert np.all(st == 0)
    for i, (x0, zb, u, x, lam, pil, piu) in enumerate(cases):
        s_ok, ref = oracle.ocp_sens(m, c, m["EaR"], x0, zb, u, x, lam, pil, piu)
        assert s_ok == 0
        scale = np.abs(ref).max()
        np.testing.assert_allclose(sens[i], ref, rtol=1e-5, atol=1e-7 * scale)


def test_nmpc_grad_matches_oracle_per_trajectory():
    w = W.get(WN)
    m = dict(w["model"], n_steps=40)
    c = dict(w["nmpc"], Ru=0.2, Qn=1.0, schedule="static")
    n = 48
    h = mc.MonteCarlo(m, c, n, w["seed"])
    h.nmpc_grad()
    st = h.stats(timeout_ms=600000)
    phi, g, cnt = h.phi(), h.grad(), h.counters()
    h.close()
    rphi, rg, fails = oracle.nmpc_grad(m, c, w["seed"], 0, n)
    ok = (cnt["n_ocp_failed"] == 0) & (fails == 0)
    assert ok.sum() >= 0.9 * n
    np.testing.assert_allclose(phi[ok], rphi[ok], rtol=1e-6)
    scale = np.abs(rg[ok]).max(axis=0)
    err = np.abs(g[ok] - rg[ok]) / (np.abs(rg[ok]) + 1e-3 * scale)
    assert err.max() < 1e-3, err.max()
    assert st["n_nonfinite"] == 0


def test_nmpc_grad_full_study_sampled():
    """The NMPC-weight gradient of the full 30,000-trajectory, 240-step study
    (R_u = 0.2, Q_n = 1) on the persistent schedule, as the benchmark times
    it; 24 trajectories across the index range against the oracle's
    complex-step derivative, with the per-trajectory tolerances of the
    40-step test."""
    w = W.get(WL)
    n = w["n_traj"]
    c = dict(w["nmpc"], Ru=0.2, Qn=1.0, schedule="persistent")
    h = mc.MonteCarlo(w["model"], c, n, w["seed"])
    h.nmpc_grad()
    st = h.stats(timeout_ms=1800000)
    phi, g, cnt = h.phi(), h.grad(), h.counters()
    h.close()
    assert st["n_traj"] == n and st["n_nonfinite"] == 0
    sample = np.unique(np.linspace(0, n - 1, 24).astype(int))
    rphi, rg, fails = [], [], []
    for j in sample:
        p_, g_, f_ = oracle.nmpc_grad(w["model"], c, w["seed"], int(j), int(j) + 1)
        rphi.append(p_[0]), rg.append(g_[0]), fails.append(f_[0])
    rphi, rg, fails = np.array(rphi), np.array(rg), np.array(fails)
    ok = (cnt["n_ocp_failed"][sample] == 0) & (fails == 0)
    assert ok.sum() >= 0.75 * len(sample)
    np.testing.assert_allclose(phi[sample][ok], rphi[ok], rtol=1e-6)
    gs = g[sample][ok]
    scale = np.abs(rg[ok]).max(axis=0)
    err = np.abs(gs - rg[ok]) / (np.abs(rg[ok]) + 1e-3 * scale)
    assert err.max() < 1e-3, err.max()


def test_nmpc_grad_phi_equals_the_static_run():
    w = W.get(WN)
    m = dict(w["model"], n_steps=40)
    c = dict(w["nmpc"], Ru=0.2, Qn=1.0, schedule="static")
    h = mc.MonteCarlo(m, c, 128, w["seed"])
    h.nmpc_grad()
    h.sync()
    phi = h.phi()
    h.run()
    h.sync()
    assert np.array_equal(h.phi(), phi)
    h.close()


@pytest.mark.parametrize("horizons", ["fixed", "mixed"])
def test_nmpc_grad_persistent_is_bit_identical_to_static(horizons):
    """The persistent schedule records each sample's starting state and KKT
    point while it runs the closed loop, then propagates the tangents through
    the records; per trajectory the arithmetic is the static schedule's, so
    Phi, the tangents and the counters agree bit for bit (also with horizons
    and iteration limits that differ between trajectories, and with the
    records split into chunks)."""
    w = W.get(WN)
    m = dict(w["model"], n_steps=40)
    c = dict(w["nmpc"], Ru=0.2, Qn=1.0)
    if horizons == "mixed":
        c.update(N_min=5, sqp_max_it_min=3)
    n = 300
    out = {}
    for sched in ("static", "persistent"):
        h = mc.MonteCarlo(m, dict(c, schedule=sched), n, w["seed"])
        h.nmpc_grad()
        h.sync()
        out[sched] = (h.phi(), h.grad(), h.counters())
        if sched == "persistent":   # a sub-range: the records of a chunk start at j0
            h.nmpc_grad(j0=37, j1=250)
            h.sync()
            out["range"] = (h.phi()[37:250], h.grad()[37:250])
        h.close()
    (p0, g0, c0), (p1, g1, c1) = out["static"], out["persistent"]
    assert np.array_equal(p0, p1)
    assert np.array_equal(g0, g1)
    for k in c0:
        assert np.array_equal(c0[k], c1[k]), k
    assert np.array_equal(out["range"][0], p0[37:250])
    assert np.array_equal(out["range"][1], g0[37:250])


def test_nmpc_grad_in_record_chunks_is_bit_identical():
    """A record budget of a few trajectories' records splits the persistent
    gradient into many chunks (each a recording launch and a tangent launch,
    the chunks' records reusing one buffer); the results are those of one
    chunk and of the static schedule, bit for bit.  A budget below one
    trajectory's records is rejected."""
    w = W.get(WN)
    m = dict(w["model"], n_steps=30)
    c = dict(w["nmpc"], Ru=0.2, Qn=1.0)
    n = 200
    per_traj = 8 * (5 * (c["N"] + 1) + 8) * (m["n_steps"] + 1)
    out = {}
    for key, sched, budget in (("static", "static", 0), ("one", "persistent", 0),
                               ("chunks", "persistent", 23 * per_traj)):
        h = mc.MonteCarlo(m, dict(c, schedule=sched), n, w["seed"])
        h.set_grad_record_budget(budget)
        h.nmpc_grad()
        h.sync()
        out[key] = (h.phi(), h.grad(), h.counters())
        if key == "chunks":
            with pytest.raises(mc.McError) as e:
                h.set_grad_record_budget(per_traj - 8)
            assert e.value.status == mc.MC_EINVAL
        h.close()
    for key in ("one", "chunks"):
        assert np.array_equal(out[key][0], out["static"][0]), key
        assert np.array_equal(out[key][1], out["static"][1]), key
        for q in out["static"][2]:
            assert np.array_equal(out[key][2][q], out["static"][2][q]), (key, q)


def test_nmpc_gradient_matches_central_differences():
    """The tangent is the derivative of the closed loop whose OCPs sit exactly
    at their KKT points.  Phi_j is only piecewise smooth in the weights: where
    an OCP along the trajectory changes its active set (an input bound) inside
    [w - h, w + h], a central difference straddles the kink and says nothing
    about the local derivative.  Those trajectories are few but their
    differences are large, so they dominate a mean; the comparison is
    therefore per trajectory: most trajectories agree to a small multiple of
    the SQP tolerance's effect, and only a minority may straddle a kink
    (with the oracle, median relative error 1e-5, 90th percentile 2e-3 for
    Q_z and R_u).  OCPs solved to 1e-7, steps of 1e-2 of each weight,
    trajectories whose OCPs all converged in every run."""
    w = W.get(WN)
    m = dict(w["model"], n_steps=24)
    c = dict(w["nmpc"], Ru=0.2, Qn=1.0, sqp_tol=1e-7, sqp_max_it=100, schedule="static")
    n = 2000
    h = mc.MonteCarlo(m, c, n, w["seed"])
    h.nmpc_grad()
    h.sync()
    g = h.grad()
    ok = h.counters()["n_ocp_failed"] == 0
    h.close()
    # the perturbed runs on the persistent schedule: the same Phi bit for bit,
    # faster past the OCPs that need hundreds of iterations at this tolerance
    h = mc.MonteCarlo(m, dict(c, schedule="persistent"), n, w["seed"])
    runs = {}
    for k in ("Qz", "Ru", "Qn"):
        hk = 1e-2 * c[k]
        for sgn in (1, -1):
            ww = dict(Qz=c["Qz"], Ru=c["Ru"], Qn=c["Qn"])
            ww[k] += sgn * hk
            h.set_nmpc_weights(ww["Qz"], ww["Ru"], ww["Qn"])
            h.run()
            h.sync()
            runs[(k, sgn)] = h.phi()
            ok &= h.counters()["n_ocp_failed"] == 0
    h.close()
    assert ok.sum() >= 0.5 * n
    for q, k in enumerate(("Qz", "Ru", "Qn")):
        hk = 1e-2 * c[k]
        fd = (runs[(k, 1)][ok] - runs[(k, -1)][ok]) / (2 * hk)
        t = g[ok, q]
        rel = np.abs(fd - t) / (np.abs(t) + 1e-2 * np.abs(t).max())
        assert np.median(rel) <= 1e-3, (k, np.median(rel))
        assert np.mean(rel <= 5e-2) >= 0.85, (k, np.mean(rel <= 5e-2))


def test_nmpc_autograd_and_errors():
    w = W.get(WN)
    m = dict(w["model"], n_steps=24)
    c = dict(w["nmpc"], Ru=0.2, Qn=1.0, schedule="static")
    h = mc.MonteCarlo(m, c, 256, w["seed"])
    x = torch.tensor([1.0, 0.2, 1.0], dtype=torch.float64, requires_grad=True)
    with pytest.warns(UserWarning, match="SQP tolerance"):
        y = nmpc_mean_phi(x, h)   # the workload's 1e-5: value and tangent part ways
    y.backward()
    assert torch.allclose(x.grad, torch.tensor(h.grad_mean(), dtype=torch.float64), rtol=0, atol=0)
    with pytest.raises(mc.McError):
        h.set_nmpc_weights(-1.0, 0.0, 0.0)
    h.close()
    hp = mc.MonteCarlo(m, w["pi"], 4, w["seed"])
    with pytest.raises(mc.McError):
        hp.nmpc_grad()
    with pytest.raises(mc.McError):
        hp.set_nmpc_weights(1.0, 0.0, 0.0)
    hp.close()
    hm = mc.MonteCarlo(m, dict(c, precision="mixed", sqp_tol=1e-3, ls_max=3), 4, w["seed"])
    with pytest.raises(mc.McError):
        hm.nmpc_grad()
    hm.close()
