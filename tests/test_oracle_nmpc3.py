"""Pins of the oracle's three-state NMPC model (drift Jacobian, RK4 shooting
with sensitivities, 3x3 CD-EKF, the three-state QP, block BFGS, the SQP and
the closed loop).

Independent references: central finite differences; the one-state oracle on
the reaction-invariant manifold (RK4 preserves the two linear invariants
exactly, and on the manifold the three-state drift reduces to the one-state
model); the one-state filter when only the temperature is uncertain; the
closed form of RK4 on the linear (k0 = 0) model; the one-state QP on a
decoupled three-state QP; enumeration of active sets with the full (not
condensed) KKT system; brute force over a horizon-2 OCP."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2212_02197_gb300 import workloads as W


@pytest.fixture(scope="module")
def m():
    oracle.build()
    return W.model(120)


def on_manifold(m, T):
    """n on the invariant manifold at temperature T (feed values of the
    invariants beta c_A + c_T and beta c_B + 2 c_T)."""
    cA = m["cA_in"] + (m["T_in"] - T) / m["beta"]
    cB = m["cB_in"] + 2.0 * (m["T_in"] - T) / m["beta"]
    return np.array([cA, cB, T]) * m["V"]


def test_drift3_is_the_plant_drift_and_its_jacobian(m):
    rng = np.random.default_rng(1)
    for _ in range(5):
        n = np.array([rng.uniform(0.1, 1.0), rng.uniform(0.2, 1.5), rng.uniform(275, 345)]) * m["V"]
        F = rng.uniform(0.0, 0.013)
        f, J, fF = oracle.drift3(m, n, F)
        np.testing.assert_allclose(f, oracle.plant_drift(m, n, F), rtol=1e-15, atol=1e-17)
        for q in range(3):
            h = 1e-6 * abs(n[q])
            e = np.zeros(3)
            e[q] = h
            fd = (oracle.drift3(m, n + e, F)[0] - oracle.drift3(m, n - e, F)[0]) / (2 * h)
            np.testing.assert_allclose(J[:, q], fd, rtol=1e-6, atol=1e-9 * np.abs(J).max())
        hF = 1e-7
        fdF = (oracle.drift3(m, n, F + hF)[0] - oracle.drift3(m, n, F - hF)[0]) / (2 * hF)
        np.testing.assert_allclose(fF, fdF, rtol=1e-7, atol=1e-10)


def test_rk4_interval3_sensitivities_match_differences(m):
    rng = np.random.default_rng(2)
    for _ in range(4):
        x0 = np.array([rng.uniform(0.2, 0.8), rng.uniform(0.4, 1.2), rng.uniform(280, 340)]) * m["V"]
        v = rng.uniform(0.1, 0.9)
        Fc = 800.0 / 60000.0
        xF, A, B = oracle.rk4_interval3(m, 5, 0.5, x0, v, Fc)
        for q in range(3):
            h = 1e-6 * abs(x0[q])
            e = np.zeros(3)
            e[q] = h
            fd = (oracle.rk4_interval3(m, 5, 0.5, x0 + e, v, Fc)[0] -
                  oracle.rk4_interval3(m, 5, 0.5, x0 - e, v, Fc)[0]) / (2 * h)
            np.testing.assert_allclose(A[:, q], fd, rtol=1e-6, atol=1e-9)
        hv = 1e-6
        fdv = (oracle.rk4_interval3(m, 5, 0.5, x0, v + hv, Fc)[0] -
               oracle.rk4_interval3(m, 5, 0.5, x0, v - hv, Fc)[0]) / (2 * hv)
        np.testing.assert_allclose(B, fdv, rtol=1e-6, atol=1e-10)


@pytest.mark.parametrize("T0", [276.0, 290.0, 320.0, 340.0])
def test_rk4_interval3_reduces_to_the_one_state_model_on_the_manifold(m, T0):
    x0 = on_manifold(m, T0)
    v, Fc = 0.45, 800.0 / 60000.0
    xF, A, B = oracle.rk4_interval3(m, 5, 0.5, x0, v, Fc)
    xT, a1, b1 = oracle.rk4_interval(m, 5, 0.5, x0[2], v, Fc)
    # the invariants are kept, so the end point is on the manifold again ...
    np.testing.assert_allclose(xF, on_manifold(m, xF[2] / m["V"]), rtol=1e-12, atol=1e-14)
    # ... and its temperature is the one-state RK4 result
    assert xF[2] == pytest.approx(xT, rel=1e-12)
    # sensitivities along the manifold: the tangent (-1/beta, -2/beta, 1)
    t = np.array([-1.0 / m["beta"], -2.0 / m["beta"], 1.0])
    assert (A @ t)[2] == pytest.approx(a1, rel=1e-10)
    assert B[2] == pytest.approx(b1, rel=1e-10)


def test_ekf3_filter_reduces_to_the_one_state_filter(m):
    x = on_manifold(m, 300.0)
    p = 2.5e-4
    P = np.diag([0.0, 0.0, p])
    y = 300.4
    x3, P3, Ps = oracle.ekf3_filter(m, y, x, P)
    x1, P1 = oracle.ekf_filter(m, y, x[2], p)[:2]
    assert x3[2] == pytest.approx(x1, rel=1e-14)
    assert P3[2, 2] == pytest.approx(P1, rel=1e-13)
    np.testing.assert_array_equal(x3[:2], x[:2])
    # Joseph and short forms agree; P stays symmetric positive semidefinite
    rng = np.random.default_rng(3)
    L = rng.normal(size=(3, 3)) * 1e-3
    Pf = L @ L.T + 1e-8 * np.eye(3)
    _, PJ, PS = oracle.ekf3_filter(m, y, x, Pf)
    np.testing.assert_allclose(PJ, PS, rtol=1e-10, atol=1e-18)
    np.testing.assert_allclose(PJ, PJ.T, rtol=0, atol=1e-20)
    assert np.all(np.linalg.eigvalsh(PJ) > -1e-20)


def test_ekf3_predict_is_the_rk4_closed_form_without_reaction(m):
    """k0 = 0: f(n) = F (c_in V - n) / V, J = -(F/V) I, so every component of
    x - c_in V and of P - (its steady state) decays by the RK4 stability
    polynomial R(z) = 1 + z + z^2/2 + z^3/6 + z^4/24 per step."""
    lin = dict(m, k0=0.0)
    F, nr = 0.009, 5
    h = lin["Ts"] / nr
    a = F / lin["V"]
    R = lambda z: 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24
    cin = np.array([lin["cA_in"], lin["cB_in"], lin["T_in"]]) * lin["V"]
    x0 = cin + np.array([0.01, -0.02, 0.5])
    P0 = np.array([[1e-6, 2e-7, 0.0], [2e-7, 3e-6, 1e-7], [0.0, 1e-7, 5e-6]])
    x1, P1 = oracle.ekf3_predict(lin, nr, F, x0, P0)
    np.testing.assert_allclose(x1 - cin, (x0 - cin) * R(-a * h) ** nr, rtol=1e-12)
    Pss = np.diag([(F * s) ** 2 / (2 * a) for s in lin["sigma"]])
    np.testing.assert_allclose(P1 - Pss, (P0 - Pss) * R(-2 * a * h) ** nr, rtol=1e-9,
                               atol=1e-16)


def random_qp3(N, rng, decoupled=False):
    A = rng.uniform(-0.3, 0.3, (N, 3, 3)) + np.eye(3) * rng.uniform(0.6, 1.1, (N, 1, 1))
    B = rng.uniform(-1.5, 1.5, (N, 3))
    b = rng.normal(0, 0.3, (N, 3))
    Wxx = np.zeros((N + 1, 3, 3))
    Wxu = np.zeros((N + 1, 3))
    Wuu = np.zeros(N + 1)
    for k in range(N + 1):
        Lk = rng.normal(size=(4, 4)) + 2 * np.eye(4)
        Wk = Lk @ Lk.T + 0.1 * np.eye(4)
        Wxx[k], Wxu[k], Wuu[k] = Wk[:3, :3], Wk[:3, 3], Wk[3, 3]
    Wxx[0] = 0.0
    Wxu[0] = 0.0
    Wxu[N] = 0.0
    Wuu[N] = 0.0
    q = rng.normal(0, 1.0, (N + 1, 3))
    q[0] = 0.0
    r = rng.normal(0, 1.0, N)
    lb = -rng.uniform(0.0, 0.4, N)
    ub = rng.uniform(0.0, 0.4, N)
    if decoupled:
        A[:, :2, 2] = A[:, 2, :2] = 0.0
        A[:, 0, 1] = A[:, 1, 0] = 0.0
        B[:, :2] = 0.0
        b[:, :2] = 0.0
        Wxx[:, :2, 2] = Wxx[:, 2, :2] = 0.0
        Wxu[:, :2] = 0.0
        q[:, :2] = 0.0
    return A, B, b, Wxx, Wxu, Wuu, q, r, lb, ub


def test_qp3_on_a_decoupled_problem_is_the_one_state_qp():
    rng = np.random.default_rng(4)
    for N in (1, 3, 12):
        A, B, b, Wxx, Wxu, Wuu, q, r, lb, ub = random_qp3(N, rng, decoupled=True)
        s3 = oracle.qp3_solve(A, B, b, Wxx, Wxu, Wuu, q, r, lb, ub)
        s1 = oracle.qp_solve(A[:, 2, 2], B[:, 2], b[:, 2], Wxx[:, 2, 2], Wxu[:, 2], Wuu, q[:, 2],
                             r, lb, ub)
        assert s3["status"] == 0 and s1["status"] == 0
        np.testing.assert_allclose(s3["du"], s1["du"], rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(s3["dx"][:, 2], s1["dx"], rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(s3["mu"][:, 2], s1["mu"], rtol=1e-9, atol=1e-11)
        np.testing.assert_allclose(s3["nul"], s1["nul"], rtol=1e-9, atol=1e-11)


def full_kkt_qp(A, B, b, Wxx, Wxu, Wuu, q, r, fixed):
    """The equality-constrained QP with inputs in `fixed` held (dict k -> value),
    solved by one dense KKT system over all stage variables (not condensed)."""
    N = len(r)
    nv = N + 3 * N          # du_0..du_{N-1}, dx_1..dx_N
    iu = lambda k: k
    ix = lambda k: N + 3 * (k - 1)
    H = np.zeros((nv, nv))
    g = np.zeros(nv)
    for k in range(N):
        H[iu(k), iu(k)] += Wuu[k]
        g[iu(k)] += r[k]
        if k >= 1:
            H[ix(k):ix(k) + 3, ix(k):ix(k) + 3] += Wxx[k]
            H[ix(k):ix(k) + 3, iu(k)] += Wxu[k]
            H[iu(k), ix(k):ix(k) + 3] += Wxu[k]
            g[ix(k):ix(k) + 3] += q[k]
    H[ix(N):ix(N) + 3, ix(N):ix(N) + 3] += Wxx[N]
    g[ix(N):ix(N) + 3] += q[N]
    rows, rhs = [], []
    for k in range(N):        # dx_{k+1} - A_k dx_k - B_k du_k = b_k
        for i in range(3):
            row = np.zeros(nv)
            row[ix(k + 1) + i] = 1.0
            if k >= 1:
                row[ix(k):ix(k) + 3] -= A[k][i]
            row[iu(k)] -= B[k][i]
            rows.append(row)
            rhs.append(b[k][i])
    for k, val in fixed.items():
        row = np.zeros(nv)
        row[iu(k)] = 1.0
        rows.append(row)
        rhs.append(val)
    E = np.array(rows)
    K = np.block([[H, E.T], [E, np.zeros((len(rows), len(rows)))]])
    sol = np.linalg.solve(K, np.concatenate([-g, rhs]))
    z, y = sol[:nv], sol[nv:]
    # multipliers of the fixed inputs are the last entries (sign: H z + g + E^T y = 0)
    return z[:N], -y[3 * N:]


def test_qp3_matches_enumeration_of_active_sets_with_the_full_kkt():
    rng = np.random.default_rng(5)
    N = 2
    for _ in range(20):
        A, B, b, Wxx, Wxu, Wuu, q, r, lb, ub = random_qp3(N, rng)
        best = None
        for sides in itertools.product((0, 1, 2), repeat=N):
            fixed = {k: (lb[k] if s == 1 else ub[k]) for k, s in enumerate(sides) if s}
            du, nu = full_kkt_qp(A, B, b, Wxx, Wxu, Wuu, q, r, fixed)
            if np.any(du < lb - 1e-12) or np.any(du > ub + 1e-12):
                continue
            ok = True
            for j, (k, s) in enumerate(sorted(fixed.items())):
                side = sides[k]
                # at a lower bound the bound multiplier is >= 0, at an upper bound <= 0
                if (side == 1 and nu[j] < -1e-10) or (side == 2 and nu[j] > 1e-10):
                    ok = False
            if ok:
                best = du
                break
        assert best is not None
        s3 = oracle.qp3_solve(A, B, b, Wxx, Wxu, Wuu, q, r, lb, ub)
        assert s3["status"] == 0
        np.testing.assert_allclose(s3["du"], best, rtol=1e-9, atol=1e-11)


def test_bfgs_blockn_secant_and_the_two_by_two_case():
    rng = np.random.default_rng(6)
    for n in (1, 3, 4):
        L = rng.normal(size=(n, n)) + 2 * np.eye(n)
        W = L @ L.T
        s = rng.normal(size=n)
        y = W @ s + 0.1 * rng.normal(size=n)       # curvature s^T y > 0.2 s^T W s
        Wn = oracle.bfgs_blockn(W, s, y)
        np.testing.assert_allclose(Wn @ s, y, rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(Wn, Wn.T, rtol=0, atol=1e-13)
        assert np.all(np.linalg.eigvalsh(Wn) > 0)
    W2 = np.array([[2.0, 0.3], [0.3, 1.5]])
    s2, y2 = np.array([0.4, -0.7]), np.array([0.1, -0.9])
    packed = oracle.bfgs_block(np.array([2.0, 0.3, 1.5]), s2, y2)
    Wn2 = oracle.bfgs_blockn(W2, s2, y2)
    np.testing.assert_allclose([Wn2[0, 0], Wn2[0, 1], Wn2[1, 1]], packed, rtol=1e-14)


def test_sqp3_kkt_point_and_horizon_two_brute_force(m):
    c = dict(W.nmpc(2), sqp_tol=1e-9, nx_model=3)
    xs = c["x_scale"]
    Fc = c["u_scale"] / 60000.0
    x0 = on_manifold(m, 300.0) / xs
    zbar = np.array([0.0, 310.0, 312.0])
    u0 = np.array([0.5, 0.5])
    xi = np.repeat(x0[None, :], 3, axis=0)
    u, x, lam, pil, piu, info = oracle.sqp3(m, c, m["EaR"], x0, zbar, u0, xi)
    assert info["status"] == 0 and info["kkt_grad"] <= 1e-9 and info["kkt_eq"] <= 1e-9

    def cost(v):
        xk, f = x0 * xs, 0.0
        for k in range(2):
            xk = oracle.rk4_interval3(m, 5, m["Ts"], xk, v[k], Fc)[0]
            f += c["Qz"] * (xk[2] / m["V"] - zbar[k + 1]) ** 2 * m["Ts"]
        return f

    grid = np.linspace(0.0, 1.0, 201)
    fg = np.array([[cost((a, bb)) for bb in grid] for a in grid])
    i, j = np.unravel_index(np.argmin(fg), fg.shape)
    # golden-section refinement would only lower the grid value; the SQP
    # minimum must not be above the grid minimum
    assert cost(u) <= fg[i, j] + 1e-9 * max(1.0, fg[i, j])


def test_nmpc3_closed_loop_tracks_like_the_one_state_controller(m):
    """The plant starts on the invariant manifold and the noise moves it off
    only a little, so the three-state and the one-state NMPC give close Phi;
    both beat the PI controller."""
    w = W.get("cstr_100x120_N20_fp64")
    mm = dict(w["model"], n_steps=60)
    c3 = dict(w["nmpc"], nx_model=3)
    n = 8
    r3 = oracle.run(mm, c3, w["seed"], 0, n)
    r1 = oracle.run(mm, w["nmpc"], w["seed"], 0, n)
    rp = oracle.run(mm, w["pi"], w["seed"], 0, n)
    assert np.all(np.isfinite(r3["phi"])) and r3["n_ocp_failed"].sum() == 0
    assert np.all(r3["n_ocp"] == 60)
    np.testing.assert_allclose(r3["phi"], r1["phi"], rtol=0.05)
    assert r3["phi"].mean() < rp["phi"].mean()
