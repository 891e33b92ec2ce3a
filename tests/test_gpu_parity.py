"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (FP64 everywhere on this path):
  * Philox words: bit-exact.  Box-Muller normals: 1e-13 absolute (the device
    takes sin/cos of 2 pi u with an exact argument scaling).
  * QP solutions (active set): both sides reach the same KKT point exactly;
    1e-9 relative.  Interior point: stopped at 1e-14 (scaled) residual and
    complementarity, compared at 1e-6.
  * Closed loop, per trajectory: PI Phi within 1e-12 relative; NMPC Phi within
    1e-6 relative (the SQP stops at a tolerance of 1e-5 on the scaled KKT test,
    so the two implementations may stop one iteration apart); trajectories with
    an OCP at the iteration limit on either side are counted and held to 1e-3.
  * The tight-tolerance tests stop every OCP at 1e-8 or 1e-9 instead, where
    both implementations end at the same KKT point up to the merit function's
    rounding floor: every OCP's inputs within 1e-8 where both converged, and
    every trajectory's Phi within 1e-6 with no exclusion at all (an OCP that
    stalls at the floor is as close to the KKT point as the arithmetic allows).
    On the oracle alone, Phi at tolerances 1e-7 .. 1e-9 stays within 2e-7 of
    Phi at 1e-10 for every trajectory of these cases.
"""
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


# ------------------------------------------------------------------ random numbers

def test_philox_bit_exact():
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, size=(20000, 4), dtype=np.uint64).astype(np.uint32)
    key = [0x12345678, 0x9ABCDEF0]
    dev = mc.philox(ctr, key)
    for i in range(0, 20000, 97):
        assert list(dev[i]) == oracle.philox(list(map(int, ctr[i])), key)
    kat = mc.philox([[0, 0, 0, 0]], [0, 0])
    assert list(kat[0]) == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]


@pytest.mark.parametrize("j", [0, 1, 29999, 262143])
def test_noise_matches_oracle(j):
    import ctypes as C

    seed = W.SEED
    proc, meas = mc.noise(seed, j, 0, 2400)
    L = oracle.lib()
    xi = np.zeros(3)
    for k in range(0, 2400, 7):
        L.or_process_noise(seed, j, k, xi.ctypes.data_as(C.POINTER(C.c_double)))
        assert np.allclose(proc[k], xi, rtol=0, atol=1e-13)
        assert abs(meas[k] - L.or_meas_noise(seed, j, k)) <= 1e-13
    # FP32 transform of the same words: 24-bit uniforms, so |dz| grows like
    # 2^-24 / (u1 |z|) in the tails
    p32, m32 = mc.noise(seed, j, 0, 2400, "mixed")
    assert np.max(np.abs(p32 - proc)) < 1e-3 and np.max(np.abs(m32 - meas)) < 1e-3
    assert np.median(np.abs(p32 - proc)) < 1e-6


# ------------------------------------------------------------------ QP subproblem

def random_qps(n, N, rng):
    A = rng.uniform(0.6, 1.2, (n, N))
    B = rng.uniform(-2.0, 2.0, (n, N))
    b = rng.normal(0.0, 0.5, (n, N))
    L = rng.normal(size=(n, N + 1, 2, 2)) + 1.5 * np.eye(2)
    Wk = L @ np.swapaxes(L, -1, -2) + 0.1 * np.eye(2)
    Wxx, Wxu, Wuu = Wk[..., 0, 0].copy(), Wk[..., 0, 1].copy(), Wk[..., 1, 1].copy()
    Wxx[:, 0] = Wxu[:, 0] = 0.0
    Wxu[:, N] = Wuu[:, N] = 0.0
    q = rng.normal(0.0, 2.0, (n, N + 1))
    q[:, 0] = 0.0
    r = rng.normal(0.0, 2.0, (n, N))
    lb = -rng.uniform(0.0, 0.3, (n, N))
    ub = rng.uniform(0.0, 0.3, (n, N))
    lb[:, ::5] = 0.0   # some inputs start on a bound, as in the SQP
    return A, B, b, Wxx, Wxu, Wuu, q, r, lb, ub


def test_device_exp_within_two_ulp():
    """The table-driven FP64 exp of the rate law against numpy's exp: over the
    arguments the simulation meets (-(E_a/R)/T for T in 150..2000 K, so about
    -57..-4) and beyond, on a dense grid plus random points, including
    table-boundary multiples of ln2/32; large |x| falls back to the library."""
    rng = np.random.default_rng(7)
    x = np.concatenate([np.linspace(-60.0, 5.0, 200001), rng.uniform(-700.0, 700.0, 100000),
                        np.arange(-2000, 2001) * np.log(2.0) / 32.0,
                        [0.0, -0.0, 1e-300, -1e-300, 709.0, -745.0, 800.0, -800.0]])
    y = mc.exp_batch(x)
    ref = np.exp(x)
    fin = np.isfinite(ref) & (ref > 1e-300)
    ulp = np.abs(y[fin] - ref[fin]) / np.spacing(ref[fin])
    assert ulp.max() <= 2.0, ulp.max()
    assert y[-2] == np.inf and y[-1] == 0.0


def test_device_reciprocal_within_one_ulp():
    """The Newton-refined reciprocal of the one-state rate law against the
    correctly rounded 1/x: temperatures the simulation meets (150..2000 K),
    random magnitudes over the whole normal range with both signs, powers of
    two (exact), and the special values (the approximation's own, exact)."""
    rng = np.random.default_rng(11)
    x = np.concatenate([np.linspace(150.0, 2000.0, 200001),
                        rng.uniform(1.0, 2.0, 100000) * 2.0 ** rng.integers(-1000, 1000, 100000),
                        -rng.uniform(1e-3, 1e3, 10000), 2.0 ** np.arange(-1000, 1001)])
    y = mc.rcp_batch(x)
    ref = 1.0 / x
    ulp = np.abs(y - ref) / np.spacing(np.abs(ref))
    assert ulp.max() <= 1.0, ulp.max()
    assert np.all(y[-2001:] == ref[-2001:])   # powers of two are exact
    sp = mc.rcp_batch(np.array([0.0, -0.0, np.inf, -np.inf, np.nan]))
    assert sp[0] == np.inf and sp[1] == -np.inf and sp[2] == 0.0 and sp[3] == 0.0
    assert np.signbit(sp[3]) and np.isnan(sp[4])


@pytest.mark.parametrize("N", [1, 2, 5, 20, 31, 32, 33, 40, 60, 64])
@pytest.mark.parametrize("solver", ["active_set", "ipm", "active_set_warp"])
def test_qp_matches_oracle(N, solver):
    rng = np.random.default_rng(N)
    n = 300
    qp = random_qps(n, N, rng)
    dev = mc.qp_solve_batch(*qp, solver=solver)
    assert np.all(dev["status"] == 0), np.flatnonzero(dev["status"])
    tol = dict(active_set=(1e-9, 1e-10), ipm=(1e-6, 1e-6), active_set_warp=(1e-9, 1e-10))[solver]
    for i in range(n):
        ref = oracle.qp_solve(*[a[i] for a in qp])
        assert ref["status"] == 0
        for key in ("du", "dx", "mu", "nul", "nuu"):
            scale = 1.0 + np.max(np.abs(ref[key]))
            assert np.allclose(dev[key][i], ref[key], rtol=tol[0], atol=tol[1] * scale), (i, key)


@pytest.mark.parametrize("N", [3, 20, 60, 64])
def test_warp_qp_follows_the_serial_active_set(N):
    """The parallel-in-horizon solver takes the same working-set steps as the
    serial active-set method (same iteration counts) and lands on the same
    point to rounding; bounds that start active and a horizon that fills two
    stages per lane are covered."""
    rng = np.random.default_rng(100 + N)
    n = 500
    qp = random_qps(n, N, rng)
    a = mc.qp_solve_batch(*qp, solver="active_set")
    b = mc.qp_solve_batch(*qp, solver="active_set_warp")
    assert np.array_equal(a["status"], b["status"])
    assert np.array_equal(a["iters"], b["iters"])
    for key in ("du", "dx", "mu", "nul", "nuu"):
        scale = 1.0 + np.max(np.abs(a[key]), axis=1, keepdims=True)
        assert np.all(np.abs(a[key] - b[key]) <= 1e-10 * scale), key
    # active bounds are hit exactly
    lb, ub = qp[8], qp[9]
    on = (np.abs(b["du"] - lb) == 0) | (np.abs(b["du"] - ub) == 0)
    assert on.any()


# ------------------------------------------------------------------ OCPs

def ocp_cases(n, N, rng):
    m = W.model(240)
    x0 = rng.uniform(276.0, 345.0, n)
    zs = rng.choice([276.0, 282.0, 290.0, 340.0], size=(n, 2))
    ksw = rng.integers(1, N + 1, n)
    zbar = np.where(np.arange(N + 1)[None, :] < ksw[:, None], zs[:, :1], zs[:, 1:])
    u = np.clip(rng.uniform(-0.2, 1.2, (n, 1)) * np.ones((1, N)), 0.0, 1.0)
    x = np.repeat(x0[:, None], N + 1, axis=1)
    return m, x0, zbar, u, x


@pytest.mark.parametrize("N", [2, 20, 30])
def test_ocp_sqp_matches_oracle(N):
    rng = np.random.default_rng(7 + N)
    n = 96
    c = W.nmpc(N)
    m, x0, zbar, u, x = ocp_cases(n, N, rng)
    dev = mc.ocp_solve_batch(m, c, x0, m["EaR"], zbar, u, x)
    agree = 0
    for i in range(n):
        ru, rx, rl, _, _, info = oracle.sqp(m, c, m["EaR"], x0[i], zbar[i], u[i], x[i])
        assert dev["status"][i] == info["status"] or info["status"] != 0 or dev["status"][i] != 0
        if info["status"] == 0 and dev["status"][i] == 0:
            agree += abs(int(dev["iters"][i]) - info["iters"]) <= 1
            assert np.allclose(dev["u"][i], ru, rtol=0, atol=1e-5), i
            assert dev["kkt_grad"][i] <= c["sqp_tol"] and dev["kkt_eq"][i] <= c["sqp_tol"]
    # near the tolerance the two may stop an iteration or two apart
    assert agree >= 0.8 * n


@pytest.mark.parametrize("N", [2, 20, 30])
def test_ocp_sqp_matches_oracle_tight(N):
    """The same OCPs solved to 1e-9 on the scaled KKT test (200 iterations at
    most): where both sides converge the inputs agree to 1e-8, and every OCP,
    converged or stalled at the rounding floor, to 1e-6."""
    rng = np.random.default_rng(7 + N)
    n = 96
    c = dict(W.nmpc(N), sqp_tol=1e-9, sqp_max_it=200)
    m, x0, zbar, u, x = ocp_cases(n, N, rng)
    dev = mc.ocp_solve_batch(m, c, x0, m["EaR"], zbar, u, x)
    both = 0
    for i in range(n):
        ru, rx, rl, _, _, info = oracle.sqp(m, c, m["EaR"], x0[i], zbar[i], u[i], x[i])
        assert np.max(np.abs(dev["u"][i] - ru)) <= 1e-6, (i, info["status"], dev["status"][i])
        if info["status"] == 0 and dev["status"][i] == 0:
            both += 1
            assert np.max(np.abs(dev["u"][i] - ru)) <= 1e-8, i
            assert np.max(np.abs(dev["x"][i][1:] - rx[1:])) <= 1e-8 * np.max(np.abs(rx)), i
    assert both >= 0.7 * n


@pytest.mark.parametrize("Ru,Qn", [(0.5, 0.0), (0.0, 4.0), (2.0, 1.0)])
def test_weighted_ocp_matches_oracle(Ru, Qn):
    """The extended objective (input-deviation and terminal weights)."""
    rng = np.random.default_rng(11)
    N, n = 20, 64
    c = dict(W.nmpc(N), Ru=Ru, Qn=Qn)
    m, x0, zbar, u, x = ocp_cases(n, N, rng)
    dev = mc.ocp_solve_batch(m, c, x0, m["EaR"], zbar, u, x)
    agree = 0
    for i in range(n):
        ru, rx, rl, _, _, info = oracle.sqp(dict(m), c, m["EaR"], x0[i], zbar[i], u[i], x[i])
        if info["status"] == 0 and dev["status"][i] == 0:
            agree += 1
            assert np.allclose(dev["u"][i], ru, rtol=0, atol=1e-5), i
            assert dev["f"][i] == pytest.approx(info["f"], rel=1e-6, abs=1e-9)
    assert agree >= 0.9 * n


def test_weighted_closed_loop_matches_oracle():
    w = W.get("cstr_100x120_N20_fp64")
    m = dict(w["model"], n_steps=60)
    for sched in ("persistent", "static"):
        c = dict(w["nmpc"], Ru=0.5, Qn=2.0, schedule=sched)
        h = mc.MonteCarlo(m, c, 64, w["seed"])
        h.run()
        h.sync()
        phi, cnt = h.phi(), h.counters()
        h.close()
        ref = oracle.run(m, c, w["seed"], 0, 64)
        compare_phi(phi, ref, cnt, 1e-6)


# ------------------------------------------------------------------ closed loop

def compare_phi(dev_phi, ref, dev_cnt, tol):
    """Per-trajectory relative Phi error; trajectories with an OCP at the
    iteration limit on either side are allowed 1e-3 and reported."""
    rel = np.abs(dev_phi - ref["phi"]) / np.abs(ref["phi"])
    hit = (ref["n_ocp_failed"] > 0) | (dev_cnt["n_ocp_failed"] > 0)
    assert np.all(rel[~hit] <= tol), (np.max(rel[~hit]), np.argmax(np.where(hit, 0, rel)))
    assert np.all(rel[hit] <= 1e-3)
    return rel, hit


@pytest.fixture(scope="module")
def small():
    w = W.get("cstr_100x120_N20_fp64")
    n = w["n_traj"]
    out = {}
    for kind in ("nmpc", "pi"):
        h = mc.MonteCarlo(w["model"], w[kind], n, w["seed"])
        h.run()
        st = h.stats(timeout_ms=600000)
        out[kind] = (h.phi(), h.counters(), st,
                     oracle.run(w["model"], w[kind], w["seed"], 0, n))
        h.close()
    return w, out


def test_closed_loop_pi_small(small):
    _, out = small
    phi, cnt, st, ref = out["pi"]
    compare_phi(phi, ref, cnt, 1e-12)
    assert st["n_traj"] == 100 and st["n_ocp"] == 0 and st["n_nonfinite"] == 0


def test_closed_loop_nmpc_small(small):
    w, out = small
    phi, cnt, st, ref = out["nmpc"]
    rel, hit = compare_phi(phi, ref, cnt, 1e-6)
    K = w["model"]["n_steps"]
    assert st["n_ocp"] == 100 * K
    assert st["n_ocp_failed"] == cnt["n_ocp_failed"].sum()
    # the SQP work is the same up to rounding-level stopping decisions
    assert abs(cnt["sqp_iters"].sum() - ref["sqp_iters"].sum()) <= 0.01 * ref["sqp_iters"].sum()


@pytest.mark.parametrize("sched", ["persistent", "static"])
def test_closed_loop_nmpc_tight(sched):
    """64 trajectories x 60 steps with every OCP solved to 1e-8 (200 SQP
    iterations at most): every trajectory within 1e-6, with no trajectory set
    aside for an OCP at the iteration limit, and most far closer."""
    w = W.get("cstr_100x120_N20_fp64")
    m = dict(w["model"], n_steps=60)
    c = dict(w["nmpc"], sqp_tol=1e-8, sqp_max_it=200, schedule=sched)
    n = 64
    h = mc.MonteCarlo(m, c, n, w["seed"])
    h.run()
    h.sync()
    phi, cnt = h.phi(), h.counters()
    h.close()
    ref = oracle.run(m, c, w["seed"], 0, n)
    rel = np.abs(phi - ref["phi"]) / np.abs(ref["phi"])
    assert np.all(rel <= 1e-6), (rel.max(), int(np.argmax(rel)))
    assert np.median(rel) <= 1e-8


def test_stats_reduction_matches_numpy(small):
    _, out = small
    for kind in ("nmpc", "pi"):
        phi, cnt, st, _ = out[kind]
        assert st["phi_mean"] == pytest.approx(phi.mean(), rel=1e-13)
        assert st["phi_var"] == pytest.approx(phi.var(ddof=1), rel=1e-11)
        assert st["phi_min"] == phi.min() and st["phi_max"] == phi.max()
        h, _ = np.histogram(phi, bins=st["n_bins"], range=(st["bin_lo"], st["bin_hi"]))
        # the top edge is inclusive in numpy and clamped into the last bin here
        assert np.array_equal(st["hist"], h)
        for k in ("sqp_iters", "ls_trials", "qp_iters", "n_hess_reset"):
            assert st[k] == cnt[k].sum()


def test_nmpc_beats_pi_small(small):
    _, out = small
    a, b = out["nmpc"][0], out["pi"][0]
    assert a.mean() < b.mean() and a.var() < b.var()


def test_paper_scale_sampled_parity():
    """The 30,000-trajectory FP64 study in the benchmark's launch configuration;
    the oracle recomputes a sample of trajectories spread over the index range."""
    w = W.get("cstr_30k_x240_N20_fp64")
    n = w["n_traj"]
    sample = np.unique(np.concatenate([np.arange(0, 8), np.linspace(0, n - 1, 40).astype(int),
                                       [n - 1]]))
    for kind, tol in (("nmpc", 1e-6), ("pi", 1e-12)):
        h = mc.MonteCarlo(w["model"], w[kind], n, w["seed"])
        h.run()
        st = h.stats(timeout_ms=1800000)
        phi = h.phi()
        cnt = h.counters()
        h.close()
        assert st["n_traj"] == n and st["n_nonfinite"] == 0
        refs = [oracle.run(w["model"], w[kind], w["seed"], int(j), int(j) + 1, threads=1)
                for j in sample]
        ref = {k: np.concatenate([r[k] for r in refs]) for k in refs[0]}
        compare_phi(phi[sample], ref, {k: v[sample] for k, v in cnt.items()}, tol)
        if kind == "nmpc":
            # Table II: total OCPs = trajectories x steps; failures are rare
            assert st["n_ocp"] == n * w["model"]["n_steps"]
            assert st["n_ocp_failed"] <= 1e-3 * st["n_ocp"]


def test_uneven_study_full_size_sampled():
    """The 262,144-trajectory uneven study (horizons 10..40, SQP limits 5..30,
    120 steps) in one launch of the persistent schedule; three blocks of 16
    trajectories (start, middle, end of the index range) against the oracle."""
    w = W.get("cstr_262k_x120_N10to40_uneven")
    n = w["n_traj"]
    h = mc.MonteCarlo(w["model"], w["nmpc"], n, w["seed"])
    h.run()
    st = h.stats(timeout_ms=1800000)
    phi, cnt = h.phi(), h.counters()
    h.close()
    assert st["n_traj"] == n and st["n_nonfinite"] == 0
    assert st["n_ocp"] == n * w["model"]["n_steps"]
    for j0 in (0, n // 2 - 8, n - 16):
        ref = oracle.run(w["model"], w["nmpc"], w["seed"], j0, j0 + 16)
        compare_phi(phi[j0:j0 + 16], ref, {k: v[j0:j0 + 16] for k, v in cnt.items()}, 1e-6)


def test_mixed_100k_study_full_size_sampled():
    """The 100,000-trajectory mixed-precision study (N = 30, E_a/R lognormal)
    in one launch; blocks of trajectories across the range against the FP64
    oracle: mixed precision moves Phi by ~1e-4 relative (median)."""
    w = W.get("cstr_100k_x240_N30_mixed")
    n = w["n_traj"]
    h = mc.MonteCarlo(w["model"], w["nmpc"], n, w["seed"])
    h.run()
    st = h.stats(timeout_ms=1800000)
    phi = h.phi()
    h.close()
    assert st["n_traj"] == n and st["n_nonfinite"] == 0
    assert st["n_ocp"] == n * w["model"]["n_steps"]
    rels = []
    c64 = dict(w["nmpc"], precision="fp64", sqp_tol=1e-5, ls_max=30)
    for j0 in (0, n // 2 - 12, n - 24):
        ref = oracle.run(w["model"], c64, w["seed"], j0, j0 + 24)["phi"]
        rels.append(np.abs(phi[j0:j0 + 24] - ref) / np.abs(ref))
    rel = np.concatenate(rels)
    assert np.median(rel) < 1e-3 and np.max(rel) < 5e-2


# ------------------------------------------------------------------ edge cases

def test_range_split_is_bit_identical():
    w = W.get("cstr_100x120_N20_fp64")
    m = dict(w["model"], n_steps=30)
    for kind in ("nmpc", "pi"):
        full = mc.MonteCarlo(m, w[kind], 100, 5)
        full.run()
        full.sync()
        part = mc.MonteCarlo(m, w[kind], 100, 5)
        part.run(j0=0, j1=37)
        part.run(j0=37, j1=100)
        part.sync()
        assert np.array_equal(full.phi(), part.phi())
        a, b = full.counters(), part.counters()
        for k in a:
            assert np.array_equal(a[k], b[k])
        full.close()
        part.close()


@pytest.mark.parametrize("n", [0, 1, 129])
def test_sizes_empty_single_ragged(n):
    w = W.get("cstr_100x120_N20_fp64")
    m = dict(w["model"], n_steps=12)
    for kind in ("nmpc", "pi"):
        h = mc.MonteCarlo(m, w[kind], n, 11)
        h.run()
        st = h.stats(timeout_ms=600000)
        assert st["n_traj"] == n
        if n:
            ref = oracle.run(m, w[kind], 11, 0, n)
            phi = h.phi()
            assert np.allclose(phi, ref["phi"], rtol=1e-6 if kind == "nmpc" else 1e-12, atol=0)
        h.close()


@pytest.mark.parametrize("N", [1, 64])
def test_horizon_extremes(N):
    w = W.get("cstr_100x120_N20_fp64")
    m = dict(w["model"], n_steps=24)
    c = W.nmpc(N)
    h = mc.MonteCarlo(m, c, 6, 3)
    h.run()
    h.sync()
    ref = oracle.run(m, c, 3, 0, 6)
    compare_phi(h.phi(), ref, h.counters(), 1e-6)
    h.close()


def test_fixed_input_degenerate_box():
    """u_min = u_max: the OCP has no freedom; both sides apply the bound."""
    w = W.get("cstr_100x120_N20_fp64")
    m = dict(w["model"], n_steps=16)
    c = dict(w["nmpc"], u_min=400.0, u_max=400.0)
    h = mc.MonteCarlo(m, c, 4, 3)
    h.run()
    h.sync()
    ref = oracle.run(m, c, 3, 0, 4)
    assert np.allclose(h.phi(), ref["phi"], rtol=1e-10, atol=0)
    h.close()


def test_ipm_closed_loop_matches_oracle():
    """The paper's QP solver (Riccati interior point) in the closed loop."""
    w = W.get("cstr_100x120_N20_fp64")
    m = dict(w["model"], n_steps=60)
    c = dict(w["nmpc"], qp_solver="ipm")
    h = mc.MonteCarlo(m, c, 16, w["seed"])
    h.run()
    h.sync()
    ref = oracle.run(m, c, w["seed"], 0, 16)
    compare_phi(h.phi(), ref, h.counters(), 1e-6)
    h.close()


@pytest.mark.parametrize("kind", ["nmpc", "pi"])
def test_model_mismatch_matches_oracle(kind):
    """E_a/R perturbed in the plant only (the controllers keep the nominal
    model): 100 trajectories of the paper-scale mismatch study, 80 steps,
    against the oracle; the variant differs from the matched one."""
    w = W.get("cstr_30k_x240_N20_fp64_mismatch")
    m = dict(w["model"], n_steps=80)
    n = 100
    h = mc.MonteCarlo(m, w[kind], n, w["seed"])
    h.run()
    h.sync()
    phi, cnt = h.phi(), h.counters()
    h.close()
    ref = oracle.run(m, w[kind], w["seed"], 0, n)
    compare_phi(phi, ref, cnt, 1e-6 if kind == "nmpc" else 1e-12)
    hk = mc.MonteCarlo(dict(m, Ea_plant_only=False), w[kind], n, w["seed"])
    hk.run()
    hk.sync()
    assert not np.array_equal(hk.phi(), phi)
    hk.close()


def test_model_mismatch_full_study_sampled():
    """The full mismatch study (30,000 trajectories, 240 steps, lognormal
    E_a/R in the plant only) in one launch of the benchmark's schedule; 48
    trajectories across the index range against the oracle."""
    w = W.get("cstr_30k_x240_N20_fp64_mismatch")
    n = w["n_traj"]
    h = mc.MonteCarlo(w["model"], w["nmpc"], n, w["seed"])
    h.run()
    st = h.stats(timeout_ms=1800000)
    phi, cnt = h.phi(), h.counters()
    h.close()
    assert st["n_traj"] == n and st["n_nonfinite"] == 0
    assert st["n_ocp"] == n * w["model"]["n_steps"]
    sample = np.unique(np.linspace(0, n - 1, 48).astype(int))
    refs = [oracle.run(w["model"], w["nmpc"], w["seed"], int(j), int(j) + 1, threads=1)
            for j in sample]
    ref = {k: np.concatenate([r[k] for r in refs]) for k in refs[0]}
    compare_phi(phi[sample], ref, {k: v[sample] for k, v in cnt.items()}, 1e-6)


# ------------------------------------------------------------------ schedules

@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_persistent_schedule_is_bit_identical_to_static(precision):
    """The persistent per-lane state machine runs the same arithmetic per
    trajectory as the static schedule."""
    w = W.get("cstr_100x120_N20_fp64")
    m = dict(w["model"], n_steps=40)
    base = dict(w["nmpc"], precision=precision)
    if precision == "mixed":
        base.update(sqp_tol=1e-3, ls_max=3)
    out = {}
    for sched, tps in (("static", 0), ("persistent", 0), ("persistent", 1)):
        h = mc.MonteCarlo(m, dict(base, schedule=sched, threads_per_sm=tps), 200, w["seed"])
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


@pytest.mark.parametrize("precision,spec_lanes", [("fp64", 0), ("fp64", 8), ("mixed", 0)])
def test_speculative_backtracking_is_bit_identical_to_static(precision, spec_lanes):
    """The persistent schedule shoots the next halvings of a backtracking line
    search together and tests them in order; the static schedule tries one
    trial point at a time.  On the first 24 steps of the 100k study (N = 30,
    E_a lognormal 2 %), where many SQP iterations sit at the merit's rounding
    floor and backtrack, Phi and every counter (iterations, trials, iteration
    limits, line-search failures) agree bit for bit."""
    w = W.get("cstr_100k_x240_N30_mixed")
    m = dict(w["model"], n_steps=24)
    c = dict(w["nmpc"], precision="fp64", sqp_tol=1e-5, ls_max=30)
    if precision == "mixed":
        c.update(precision="mixed", sqp_tol=1e-3, ls_max=3)
    n = 256
    out = {}
    for sched in ("static", "persistent"):
        h = mc.MonteCarlo(m, dict(c, schedule=sched, ls_spec_lanes=spec_lanes), n, w["seed"])
        h.run()
        st = h.stats()
        out[sched] = (h.phi(), h.counters(), st)
        h.close()
    (p0, c0, s0), (p1, c1, s1) = out["static"], out["persistent"]
    assert s0["ls_trials"] > 1.2 * s0["sqp_iters"], (s0["ls_trials"], s0["sqp_iters"])
    assert np.array_equal(p0, p1)
    for k in c0:
        assert np.array_equal(c0[k], c1[k]), k


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_warp_trace_accounts_for_every_round(precision):
    """The per-warp record of a persistent launch: at every pool round a lane
    that still holds a trajectory has one OCP start or one line-search round
    pending (a round of a backtracking line search shoots several trials), so
    the lane-rounds of all warps lie between the launch's OCP starts plus SQP
    iterations (one trial each at least) and its OCP starts plus trials; each
    warp ran within the launch's time.  A static launch leaves no record."""
    w = W.get("cstr_100x120_N20_fp64")
    m = dict(w["model"], n_steps=40)
    c = dict(w["nmpc"], precision=precision, schedule="persistent")
    if precision == "mixed":
        c.update(sqp_tol=1e-3, ls_max=3)
    n = 200
    h = mc.MonteCarlo(m, c, n, w["seed"])
    h.run()
    st = h.stats()
    tr = h.warp_trace()
    h.close()
    assert len(tr["rounds"]) == (n + 31) // 32
    lr = tr["lane_rounds"].sum()
    assert st["n_ocp"] + st["sqp_iters"] <= lr <= st["n_ocp"] + st["ls_trials"]
    assert np.all(tr["lane_rounds"] <= 32 * tr["rounds"])
    assert np.all(tr["rounds"] >= 1) and np.all(tr["t_end_ns"] >= tr["t_start_ns"])
    import torch

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert np.all((tr["sm"] >= 0) & (tr["sm"] < sms))
    hs = mc.MonteCarlo(m, dict(c, schedule="static"), 32, w["seed"])
    hs.run()
    hs.sync()
    with pytest.raises(mc.McError) as e:
        hs.warp_trace()
    assert e.value.status == mc.MC_ENOTRUN
    hs.close()


def test_uneven_batch_matches_oracle():
    """Per-trajectory horizons 10..40 and SQP limits 5..30 (persistent
    schedule, queue ordered by horizon) against the oracle."""
    w = W.get("cstr_262k_x120_N10to40_uneven")
    m = dict(w["model"], n_steps=30)
    n = 96
    h = mc.MonteCarlo(m, w["nmpc"], n, w["seed"])
    h.run()
    st = h.stats(timeout_ms=600000)
    phi, cnt = h.phi(), h.counters()
    h.close()
    ref = oracle.run(m, w["nmpc"], w["seed"], 0, n)
    compare_phi(phi, ref, cnt, 1e-6)
    assert st["n_ocp"] == n * 30
    # the same trajectories through the static schedule, bit for bit
    hs = mc.MonteCarlo(m, dict(w["nmpc"], schedule="static"), n, w["seed"])
    hs.run()
    hs.sync()
    assert np.array_equal(hs.phi(), phi)
    hs.close()


def test_graph_replay_and_autotune_keep_results():
    """CUDA-graph replay of a captured run and an autotuned persistent
    schedule give the same per-trajectory results as a direct launch."""
    import torch

    w = W.get("cstr_262k_x120_N10to40_uneven")
    m = dict(w["model"], n_steps=16)
    n = 300
    ref = mc.MonteCarlo(m, w["nmpc"], n, w["seed"])
    ref.run()
    ref.sync()
    phi0, cnt0 = ref.phi(), ref.counters()
    ref.close()
    s = torch.cuda.Stream()
    h = mc.MonteCarlo(m, w["nmpc"], n, w["seed"])
    tps = h.autotune(probe_steps=3, stream=s)
    # a listed candidate, or one resident thread per trajectory
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert tps in (32, 64, 96, 128, 160, 192, 256, 384, 512) or tps * sms >= n
    h.set_graph(True)
    for _ in range(2):          # capture, then replay
        h.run(stream=s)
        st = h.stats(timeout_ms=600000)
        assert np.array_equal(h.phi(), phi0)
        cnt = h.counters()
        for k in cnt0:
            assert np.array_equal(cnt[k], cnt0[k])
        assert st["n_traj"] == n
    h.run(stream=s, j0=10, j1=50)   # another range gets its own graph
    h.sync()
    assert np.array_equal(h.phi()[10:50], phi0[10:50])
    h.close()


def torch_sms():
    import torch

    return torch.cuda.get_device_properties(0).multi_processor_count


def test_sm_partition_keeps_results():
    """A green-context partition of 16 SMs changes where trajectories run,
    not what they compute: Phi and the counters equal the whole-GPU run, for
    the persistent and the static schedule and for the PI gradient."""
    w = W.get("cstr_100x120_N20_fp64")
    m = dict(w["model"], n_steps=20)
    for sched in ("persistent", "static"):
        c = dict(w["nmpc"], schedule=sched)
        h = mc.MonteCarlo(m, c, 300, w["seed"])
        h.run()
        h.sync()
        phi0, cnt0 = h.phi(), h.counters()
        sms = torch_sms()
        got = h.set_sm_partition(16)
        assert 16 <= got < sms
        h.run()
        st = h.stats()
        assert np.array_equal(h.phi(), phi0)
        cnt = h.counters()
        for k in cnt0:
            assert np.array_equal(cnt[k], cnt0[k])
        assert st["n_traj"] == 300 and st["gpu_ms"] > 0
        assert h.set_sm_partition(0) == sms
        h.close()
    hp = mc.MonteCarlo(m, w["pi"], 200, w["seed"])
    hp.pi_grad(20)
    g0 = hp.grad()
    hp.set_sm_partition(8)
    hp.pi_grad(20)
    assert np.array_equal(hp.grad(), g0)
    with pytest.raises(mc.McError):
        hp.set_sm_partition(-1)
    hp.close()
