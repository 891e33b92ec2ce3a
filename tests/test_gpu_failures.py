"""Failure detection of the closed-loop study, driven from the host.

Nothing here faults, traps or hangs the GPU: a wait that is cut short by the
host-side limit of mc_sync / mc_stats while the kernels run to their normal
end, OCPs forced to stop at an iteration limit of 0 or 1 (Sec. VII-C counts
OCPs at the limit as failed and applies their last iterate), and states driven
out of the finite range by an extreme noise intensity or a NaN parameter,
which the closed loop detects at the next sample and reports."""
import math

import numpy as np
import pytest

import oracle
from paper_2212_02197_gb300 import mc, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2212_02197_gb300 import _build

    _build.build()
    oracle.build()


def test_host_wait_limit_returns_etimeout_then_the_result():
    """A full-size study takes about two seconds; a 1 ms wait limit returns
    MC_ETIMEOUT (the run carries on), and a wait without limit then returns
    the complete statistics."""
    w = W.get("cstr_30k_x240_N20_fp64")
    h = mc.MonteCarlo(w["model"], w["nmpc"], w["n_traj"], w["seed"])
    h.run()
    with pytest.raises(mc.McError) as e:
        h.stats(timeout_ms=1)
    assert e.value.status == mc.MC_ETIMEOUT
    with pytest.raises(mc.McError) as e:
        h.sync(timeout_ms=1)
    assert e.value.status == mc.MC_ETIMEOUT
    st = h.stats()
    assert st["status"] == mc.MC_OK and st["n_traj"] == w["n_traj"]
    assert st["n_ocp"] == w["n_traj"] * w["model"]["n_steps"]
    h.close()


def test_stats_before_any_run_is_enotrun():
    w = W.get("cstr_100x120_N20_fp64")
    h = mc.MonteCarlo(w["model"], w["pi"], 8, w["seed"])
    with pytest.raises(mc.McError) as e:
        h.stats()
    assert e.value.status == mc.MC_ENOTRUN
    h.close()


@pytest.mark.parametrize("max_it", [0, 1])
@pytest.mark.parametrize("sched", ["persistent", "static"])
def test_forced_sqp_failures_match_the_oracle(max_it, sched):
    """With an SQP iteration limit of 0 or 1 almost every OCP stops at the
    limit and applies its current iterate; the per-trajectory counts of failed
    OCPs and of SQP iterations equal the oracle's, and Phi agrees as closely as
    for converged OCPs."""
    w = W.get("cstr_100x120_N20_fp64")
    m = dict(w["model"], n_steps=30)
    c = dict(w["nmpc"], sqp_max_it=max_it, schedule=sched)
    n = 64
    h = mc.MonteCarlo(m, c, n, w["seed"])
    h.run()
    st = h.stats()
    phi, cnt = h.phi(), h.counters()
    h.close()
    ref = oracle.run(m, c, w["seed"], 0, n)
    assert np.array_equal(cnt["n_ocp_failed"], ref["n_ocp_failed"])
    assert np.array_equal(cnt["sqp_iters"], ref["sqp_iters"])
    assert st["n_ocp_failed"] == ref["n_ocp_failed"].sum() > 0.9 * n * 30
    assert np.max(np.abs(phi - ref["phi"]) / np.abs(ref["phi"])) <= 1e-9


def _nonfinite_case(kind, scale, n, steps, **model_over):
    w = W.get("cstr_100x120_N20_fp64")
    m = dict(w["model"], n_steps=steps, **model_over)
    m["sigma"] = [s * scale for s in m["sigma"]]
    c = dict(w[kind])
    h = mc.MonteCarlo(m, c, n, w["seed"])
    h.run()
    st = h.stats()
    phi, cnt = h.phi(), h.counters()
    h.close()
    ref = oracle.run(m, c, w["seed"], 0, n)
    return st, phi, cnt, ref


@pytest.mark.parametrize("kind,scale,steps", [("pi", 1000.0, 120), ("nmpc", 200.0, 30)])
def test_extreme_noise_drives_trajectories_non_finite(kind, scale, steps):
    """Process noise hundreds of times the workload's drives the reactor
    temperature through zero in some trajectories (the rate law then
    overflows).  The library reports MC_WARN_NONFINITE, flags exactly the
    trajectories the oracle flags (same noise), gives them Phi = NaN and
    leaves the others as the oracle computes them."""
    n = 128
    st, phi, cnt, ref = _nonfinite_case(kind, scale, n, steps)
    bad = ref["nonfinite"] > 0
    assert 0 < bad.sum() < n, bad.sum()          # some, not all
    assert st["status"] == mc.MC_WARN_NONFINITE
    assert st["n_nonfinite"] == bad.sum()
    assert np.array_equal(cnt["nonfinite"] > 0, bad)
    assert np.all(np.isnan(phi[bad]))
    # the finite ones: PI to rounding; NMPC, whose OCPs stop anywhere inside
    # the 1e-5 KKT tolerance, with states swinging hundreds of times wider than
    # in the workload, to 1e-3 and mostly to rounding
    tol = 1e-12 if kind == "pi" else 1e-3
    good = ~bad
    rel = np.abs(phi[good] - ref["phi"][good]) / np.abs(ref["phi"][good])
    assert np.all(rel <= tol), rel.max()
    assert np.median(rel) <= (1e-12 if kind == "pi" else 1e-9), np.median(rel)
    # the statistics cover the finite trajectories only
    assert st["n_traj"] == n
    assert st["phi_mean"] == pytest.approx(np.mean(phi[~bad]), rel=1e-12)


@pytest.mark.parametrize("kind", ["pi", "nmpc"])
@pytest.mark.parametrize("field", ["T_in", "Ea_logsd"])
def test_nan_parameter_makes_every_trajectory_non_finite(kind, field):
    """A NaN in a parameter that the library passes through unchecked (the
    inlet temperature, the E_a/R spread) makes every trajectory non-finite at
    its first sample, on the GPU and in the oracle alike; the run still ends
    normally and reports it."""
    w = W.get("cstr_100x120_N20_fp64")
    m = dict(w["model"], n_steps=10)
    m[field] = math.nan
    n = 40
    h = mc.MonteCarlo(m, w[kind], n, w["seed"])
    h.run()
    st = h.stats()
    cnt = h.counters()
    h.close()
    ref = oracle.run(m, w[kind], w["seed"], 0, n)
    assert np.all(ref["nonfinite"] == 1)
    assert st["status"] == mc.MC_WARN_NONFINITE and st["n_nonfinite"] == n
    assert np.all(cnt["nonfinite"] == 1)


@pytest.mark.parametrize("field,value", [("V", math.nan), ("meas_sd", math.nan),
                                         ("Ts", math.nan), ("EaR", -1.0)])
def test_invalid_parameters_are_rejected_before_any_launch(field, value):
    w = W.get("cstr_100x120_N20_fp64")
    m = dict(w["model"], **{field: value})
    with pytest.raises(mc.McError) as e:
        mc.MonteCarlo(m, w["nmpc"], 4, w["seed"])
    assert e.value.status == mc.MC_EINVAL


def test_nmpc_gradient_of_trajectories_that_go_non_finite():
    """The NMPC-weight gradient when extreme noise drives some trajectories
    non-finite part-way: the persistent schedule's records then end at the
    sample where the trajectory stopped.  Both schedules flag the same
    trajectories, give them Phi and tangents NaN, and agree bit for bit on
    the others."""
    w = W.get("cstr_100x120_N20_fp64")
    m = dict(w["model"], n_steps=30)
    m["sigma"] = [s * 200.0 for s in m["sigma"]]
    c = dict(w["nmpc"], Ru=0.2, Qn=1.0)
    n = 128
    out = {}
    for sched in ("static", "persistent"):
        h = mc.MonteCarlo(m, dict(c, schedule=sched), n, w["seed"])
        h.nmpc_grad()
        st = h.stats()
        out[sched] = (h.phi(), h.grad(), h.counters(), st)
        h.close()
    (p0, g0, c0, s0), (p1, g1, c1, s1) = out["static"], out["persistent"]
    bad = c0["nonfinite"] > 0
    assert 0 < bad.sum() < n, bad.sum()
    assert s1["n_nonfinite"] == bad.sum()
    assert np.all(np.isnan(p1[bad])) and np.all(np.isnan(g1[bad]))
    assert np.array_equal(p0, p1, equal_nan=True)
    assert np.array_equal(g0, g1, equal_nan=True)
    for k in c0:
        assert np.array_equal(c0[k], c1[k]), k
    assert np.all(np.isfinite(g1[~bad]))
