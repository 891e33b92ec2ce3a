"""Pins of the oracle's CSTR model (Sec. VI), Euler-Maruyama plant (Sec. II,
VII-A), RK4 shooting with sensitivities (Sec. III-B, VII-A), CD-EKF (Sec. III-A),
PI law (Sec. V) and performance index (Eq. Phi), each against facts that do not
come from the oracle itself: closed forms, conservation laws, steady states,
finite differences, an independent ODE integrator and hand-computed values.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2212_02197_gb300 import workloads as W

M = W.model(120)
V, beta, Tin = M["V"], M["beta"], M["T_in"]


def on_manifold(T):
    """Three-state plant state on the reaction-invariant manifold at temperature T."""
    cA = M["cA_in"] + (Tin - T) / beta
    cB = M["cB_in"] + 2.0 * (Tin - T) / beta
    return np.array([cA, cB, T]) * V


# --------------------------------------------------------------- model / drift

def test_model1_jacobians_match_finite_differences():
    for T in (275.0, 290.0, 320.0, 345.0):
        for F in (1e-3, 6e-3, 1.3e-2):
            x = T * V
            f, fx, fF = oracle.model1(M, x, F)
            hx, hF = 1e-5 * x, 1e-6 * F
            fx_fd = (oracle.model1(M, x + hx, F)[0] - oracle.model1(M, x - hx, F)[0]) / (2 * hx)
            fF_fd = (oracle.model1(M, x, F + hF)[0] - oracle.model1(M, x, F - hF)[0]) / (2 * hF)
            assert fx == pytest.approx(fx_fd, rel=1e-7, abs=1e-9)
            assert fF == pytest.approx(fF_fd, rel=1e-7)


@pytest.mark.parametrize("T", [276.0, 282.0, 290.0, 310.0, 340.0])
def test_plant_drift_vanishes_at_one_state_steady_state(T):
    """The three-state drift (Eq. CSTR with S = [-1, -2, beta]) is zero on the
    invariant manifold at the flow where the one-state model is stationary."""
    F = oracle.Fss(M, T)
    assert 0.0 < F
    f = oracle.plant_drift(M, on_manifold(T), F)
    scale = F * np.array([M["cA_in"], M["cB_in"], T]) * 1.0
    assert np.all(np.abs(f) <= 1e-12 * np.maximum(scale, 1e-3) * 10)
    # and the one-state model agrees
    f1, _, _ = oracle.model1(M, T * V, F)
    assert abs(f1) <= 1e-11 * F * T


def test_plant_reaction_invariants():
    """d/dt (beta n_A + n_T) and d/dt (beta n_B + 2 n_T) contain no reaction term:
    they equal the flow terms F (feed - reactor) exactly."""
    rng = np.random.default_rng(1)
    for _ in range(50):
        n = rng.uniform([0.01, 0.01, 26.0], [0.09, 0.13, 37.0])
        F = rng.uniform(0.0, 0.015)
        f = oracle.plant_drift(M, n, F)
        c = n / V
        lhs1 = beta * f[0] + f[2]
        rhs1 = F * (beta * M["cA_in"] + Tin) - F * (beta * c[0] + c[2])
        lhs2 = beta * f[1] + 2.0 * f[2]
        rhs2 = F * (beta * M["cB_in"] + 2.0 * Tin) - F * (beta * c[1] + 2.0 * c[2])
        assert lhs1 == pytest.approx(rhs1, rel=1e-9, abs=1e-12)
        assert lhs2 == pytest.approx(rhs2, rel=1e-9, abs=1e-12)


def test_plant_batch_rate_law():
    """With no flow only the reaction acts: the drifts are in the ratio of the
    stoichiometry S = [-1, -2, beta]; at T* with E_a/R / T* = ln k0 the rate
    constant is one, so -dn_A/dt = c_A c_B V; and the Arrhenius ratio holds."""
    Tstar = M["EaR"] / math.log(M["k0"])
    n = np.array([0.5, 0.7, Tstar]) * V
    f = oracle.plant_drift(M, n, 0.0)
    assert f[1] / f[0] == pytest.approx(2.0, rel=1e-14)
    assert f[2] / f[0] == pytest.approx(-beta, rel=1e-14)
    assert -f[0] / V == pytest.approx(0.5 * 0.7, rel=1e-12)
    n2 = np.array([0.5, 0.7, 300.0]) * V
    f2 = oracle.plant_drift(M, n2, 0.0)
    assert f2[0] / f[0] == pytest.approx(math.exp(-M["EaR"] * (1 / 300.0 - 1 / Tstar)), rel=1e-12)


def test_unstable_branch_inside_operating_window():
    """Sec. VI: the model has a branch of unstable steady states in the operating
    window [0, 800] mL/min.  Along the steady-state curve F_ss(T) the one-state
    model is unstable exactly where F_ss increases with T."""
    Ts_ = np.linspace(274.0, 353.0, 800)
    Fm = np.array([oracle.Fss(M, T) for T in Ts_]) * 60000.0
    dF = np.gradient(Fm, Ts_)
    unstable = dF > 0
    assert unstable.any()
    assert np.all((Fm[unstable] > 0.0) & (Fm[unstable] < 800.0))
    for T, d in zip(Ts_[::40], dF[::40]):
        _, fx, _ = oracle.model1(M, T * V, oracle.Fss(M, T))
        assert (fx > 0) == (d > 0)
    # the chosen set-points: 276, 282, 340 K stable; 290 K unstable
    for T, is_unstable in ((276.0, False), (282.0, False), (290.0, True), (340.0, False)):
        _, fx, _ = oracle.model1(M, T * V, oracle.Fss(M, T))
        assert (fx > 0) == is_unstable


def test_zbar_piecewise_constant():
    assert oracle.zbar(M, 0.0) == 276.0
    assert oracle.zbar(M, 19.999999) == 276.0
    assert oracle.zbar(M, 20.0) == 282.0
    assert oracle.zbar(M, 40.0) == 290.0
    assert oracle.zbar(M, 1e9) == 340.0


# --------------------------------------------------------------- Euler-Maruyama

def _no_noise(m):
    m = dict(m)
    m["sigma"] = [0.0, 0.0, 0.0]
    return m


@pytest.mark.parametrize("T", [276.0, 340.0])
def test_em_noise_free_steady_state(T):
    m = _no_noise(M)
    F = oracle.Fss(m, T)
    n0 = on_manifold(T)
    n = n0.copy()
    for _ in range(20000):  # 1000 s of 0.05 s steps
        n = oracle.em_step(m, n, F, 0.05, [0.0, 0.0, 0.0])
    assert np.allclose(n, n0, rtol=1e-10, atol=0.0)


def test_em_diffusion_term():
    """n+ = n + f h + F sigma-bar sqrt(h) xi: at a steady state (f = 0) the
    increment is exactly the diffusion term."""
    T = 282.0
    F = oracle.Fss(M, T)
    n0 = on_manifold(T)
    xi = np.array([0.3, -1.7, 2.2])
    h = 0.05
    n1 = oracle.em_step(M, n0, F, h, xi)
    f = oracle.plant_drift(M, n0, F)
    expect = F * np.array(M["sigma"]) * math.sqrt(h) * xi
    assert np.allclose(n1 - n0 - f * h, expect, rtol=1e-9, atol=1e-16)


def test_em_converges_at_order_one():
    from scipy.integrate import solve_ivp

    m = _no_noise(M)
    F = 400.0 / 60000.0
    n0 = np.array([M["cA_in"], M["cB_in"], Tin]) * V + np.array([0.0, 0.0, 20.0 * V])
    tf = 10.0
    ref = solve_ivp(lambda t, n: oracle.plant_drift(m, n, F), (0.0, tf), n0, rtol=1e-12,
                    atol=1e-14, method="DOP853").y[:, -1]
    errs = []
    for h in (0.05, 0.025, 0.0125):
        n = n0.copy()
        for _ in range(int(round(tf / h))):
            n = oracle.em_step(m, n, F, h, [0.0, 0.0, 0.0])
        errs.append(np.max(np.abs(n - ref)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 1.8 < r1 < 2.2 and 1.8 < r2 < 2.2


# --------------------------------------------------------------- RK4 shooting

def _linear(m):
    m = dict(m)
    m["k0"] = 0.0
    return m


def test_rk4_linear_closed_form():
    """With k0 = 0 the one-state model is linear, dx/dt = (F/V)(T_in V - x); n
    classical RK4 steps multiply the deviation by R(z)^n, z = -h F/V,
    R(z) = 1 + z + z^2/2 + z^3/6 + z^4/24 (and B follows by differentiation)."""
    m = _linear(M)
    Ts, n = 0.5, 5
    h = Ts / n
    Fconv = 800.0 / 60000.0
    for x0 in (280.0 * V, 330.0 * V):
        for v in (0.2, 0.9):
            F = v * Fconv
            z = -h * F / V
            R = 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24
            dR = 1 + z + z * z / 2 + z ** 3 / 6
            xs = Tin * V
            xF, A, B = oracle.rk4_interval(m, n, Ts, x0, v, Fconv)
            assert xF == pytest.approx(xs + (x0 - xs) * R ** n, rel=1e-14)
            assert A == pytest.approx(R ** n, rel=1e-13)
            Bx = (x0 - xs) * n * R ** (n - 1) * dR * (-h * Fconv / V)
            assert B == pytest.approx(Bx, rel=1e-11)


def test_rk4_sensitivities_match_finite_differences():
    Fconv = 800.0 / 60000.0
    for T in (276.0, 290.0, 335.0):
        for v in (0.05, 0.4, 0.95):
            x0 = T * V
            xF, A, B = oracle.rk4_interval(M, 5, 0.5, x0, v, Fconv)
            hx, hv = 1e-6 * x0, 1e-6
            Afd = (oracle.rk4_interval(M, 5, 0.5, x0 + hx, v, Fconv)[0]
                   - oracle.rk4_interval(M, 5, 0.5, x0 - hx, v, Fconv)[0]) / (2 * hx)
            Bfd = (oracle.rk4_interval(M, 5, 0.5, x0, v + hv, Fconv)[0]
                   - oracle.rk4_interval(M, 5, 0.5, x0, v - hv, Fconv)[0]) / (2 * hv)
            assert A == pytest.approx(Afd, rel=1e-6)
            assert B == pytest.approx(Bfd, rel=1e-6, abs=1e-9)


def test_rk4_fourth_order_against_reference_integrator():
    from scipy.integrate import solve_ivp

    Fconv = 800.0 / 60000.0
    x0, v, Ts = 300.0 * V, 0.3, 0.5
    ref = solve_ivp(lambda t, x: [oracle.model1(M, x[0], v * Fconv)[0]], (0, Ts), [x0],
                    rtol=1e-13, atol=1e-13, method="DOP853").y[0, -1]
    e = [abs(oracle.rk4_interval(M, n, Ts, x0, v, Fconv)[0] - ref) for n in (1, 2, 4)]
    assert e[0] / e[1] > 12 and e[1] / e[2] > 12
    assert abs(oracle.rk4_interval(M, 5, Ts, x0, v, Fconv)[0] - ref) < 1e-7 * x0


# --------------------------------------------------------------- CD-EKF

def test_ekf_predict_linear_closed_form():
    """k0 = 0: the CD-EKF prediction is the continuous-discrete Kalman predictor
    of dx = a (T_in V - x) dt + F sigma_T dw, a = F/V:
      x- = T_in V + (x - T_in V) e^{-a Ts},
      P- = e^{-2 a Ts} P + (F sigma_T)^2 (1 - e^{-2 a Ts}) / (2 a).
    Each linear equation y' = lam (y - y*) is integrated by n RK4 steps, which
    give exactly y* + R(lam h)^n (y - y*); that is checked to rounding, and the
    continuous solution within RK4's error, |R(z) - e^z| <= |z|^5/120 per step
    relative to |e^z - 1| for the forced part."""
    m = _linear(M)
    Ts, n = m["Ts"], 5
    h = Ts / n

    def R(z):
        return 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24

    for F in (3e-3, 1.2e-2):
        a = F / V
        q = (F * m["sigma"][2]) ** 2
        for x, P in ((280.0 * V, 1e-6), (300.0 * V, 0.3)):
            xp, Pp = oracle.ekf_predict(m, n, F, x, P)
            xs, Ps = Tin * V, q / (2 * a)
            assert xp == pytest.approx(xs + R(-a * h) ** n * (x - xs), rel=1e-14)
            assert Pp == pytest.approx(Ps + R(-2 * a * h) ** n * (P - Ps), rel=1e-12)
            xe = Tin * V + (x - Tin * V) * math.exp(-a * Ts)
            Pe = math.exp(-2 * a * Ts) * P + q * (1 - math.exp(-2 * a * Ts)) / (2 * a)
            bound = n * (2 * a * h) ** 4 / 120 * 2
            assert xp == pytest.approx(xe, rel=1e-11)
            assert Pp == pytest.approx(Pe, rel=bound)


def test_ekf_prediction_state_is_the_one_interval_shooting():
    """The state part of the CD-EKF prediction (Eq. (predictionEquations): RK4
    on x' = f(x, F) over one sample) and the OCP's shooting of one interval
    (Eq. (OCP_NLP): RK4 on the same model, the same N_c steps, from the same x
    under the same flow F = v F_conv) are one integration.  The GPU path
    therefore takes the prediction from the interval-0 shooting of the last
    OCP's final iterate; here the oracle's two routines agree to rounding,
    also far from steady state and near the unstable branch."""
    m = dict(M)
    c = W.nmpc()
    Fconv = c["u_scale"] / 60000.0
    rng = np.random.default_rng(7)
    for _ in range(40):
        x = V * rng.uniform(270.0, 360.0)
        v = rng.uniform(0.0, 1.0)
        xp, _ = oracle.ekf_predict(m, c["n_rk4"], v * Fconv, x, 1e-3)
        xF, _, _ = oracle.rk4_interval(m, c["n_rk4"], m["Ts"], x, v, Fconv)
        assert xp == pytest.approx(xF, rel=1e-14, abs=0), (x, v)


def test_ekf_filter_is_bayes_posterior_and_joseph_equals_short():
    """For a linear measurement y = x/V + v the filtered pair is the Gaussian
    posterior: precision 1/P + C^2/R, mean (x/P + C y/R) / precision, C = 1/V."""
    R = M["meas_sd"] ** 2
    C = 1.0 / V
    for x, P, y in ((29.0, 1e-6, 277.0), (31.5, 2e-3, 299.5), (35.0, 0.5, 331.0)):
        xf, Pf, Ps = oracle.ekf_filter(M, y, x, P)
        prec = 1.0 / P + C * C / R
        assert Pf == pytest.approx(1.0 / prec, rel=1e-12)
        assert xf == pytest.approx((x / P + C * y / R) / prec, rel=1e-12)
        assert Ps == pytest.approx(Pf, rel=1e-12)
        assert Pf > 0


# --------------------------------------------------------------- PI law

def test_pi_hand_computed_sequence():
    """Eq. (PI) with k_P = -1e-3, k_I = -1e-4, k_aw = -1e-1, T_s = 0.5 s,
    u-bar = 5e-3 L/s and bounds [0, 800] mL/min; values computed by hand with
    exact fractions; steps 3 and 4 saturate and wind the integrator back."""
    c = W.pi()
    Ihat = 0.0
    expect = [(-1, 0.00605, 5e-05), (-2, 0.00715, 0.00015),
              (-10, 800.0 / 60000.0, 0.0005341666666666666),
              (-10, 800.0 / 60000.0, 0.000899125), (5, 0.000649125, 0.000649125)]
    for e, u_exp, I_exp in expect:
        y = 290.0 - e
        u, Ihat = oracle.pi_step(c, 0.5, 290.0, y, 5e-3, Ihat)
        assert u == pytest.approx(u_exp, rel=1e-12)
        assert Ihat == pytest.approx(I_exp, rel=1e-12)


# --------------------------------------------------------------- performance index

@pytest.mark.parametrize("kind", ["pi", "nmpc"])
def test_phi_definition_on_a_frozen_plant(kind):
    """Eq. (Phi) with K + 1 samples: without reaction (k0 = 0) and noise the
    reactor filled with feed stays at T_in whatever the input, so
    Phi = sum_i (T_in - zbar(t_i))^2 / (K + 1); for K = 120, T_s = 0.5 s and the
    schedule 276 K | 282 K from 20 s | 290 K from 40 s this is 5588009/48400."""
    m = _no_noise(_linear(M))
    m["meas_sd"] = 1e-6   # the filter needs R > 0; the plant ignores it
    c = W.pi() if kind == "pi" else W.nmpc(4)
    r = oracle.traj(m, c, 1, 0)
    assert r["phi"] == pytest.approx(5588009.0 / 48400.0, rel=1e-12)
    assert r["n_ocp"] == (120 if kind == "nmpc" else 0)
