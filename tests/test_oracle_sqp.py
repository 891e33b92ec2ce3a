"""Pins of the oracle's SQP (Sec. IV): damped block BFGS (Sec. IV-C), the KKT
point it returns (Sec. IV-D), and the OCP minimum on horizon-2 problems found
by brute-force grid search over the inputs (single shooting, independent of
the multiple-shooting NLP)."""
import numpy as np
import pytest

import oracle
from paper_2212_02197_gb300 import workloads as W

EPS_M = 2.220446049250313e-16


def unpack(w):
    return np.array([[w[0], w[1]], [w[1], w[2]]]) if len(w) == 3 else np.array([[w[0]]])


@pytest.mark.parametrize("seed", range(20))
def test_bfgs_secant_and_damping(seed):
    """r = theta y + (1 - theta) W s with theta = 1 if s'y >= 0.2 s'Ws, else
    0.8 s'Ws / (s'Ws - s'y); the update satisfies W+ s = r and keeps W+ > 0."""
    rng = np.random.default_rng(seed)
    L = rng.normal(size=(2, 2)) + np.eye(2)
    W0 = L @ L.T + 0.05 * np.eye(2)
    w = [W0[0, 0], W0[0, 1], W0[1, 1]]
    s = rng.normal(size=2)
    y = rng.normal(size=2)
    sWs = s @ W0 @ s
    sy = s @ y
    theta = 1.0 if sy >= 0.2 * sWs else 0.8 * sWs / (sWs - sy)
    r = theta * y + (1 - theta) * W0 @ s
    Wn = unpack(oracle.bfgs_block(w, s, y))
    assert np.allclose(Wn @ s, r, rtol=1e-10, atol=1e-12)
    assert np.all(np.linalg.eigvalsh(Wn) > 0)
    assert s @ r >= 0.2 * sWs * (1 - 1e-12)
    if sy >= 0.2 * sWs:
        assert np.allclose(Wn @ s, y, rtol=1e-10, atol=1e-12)


def test_bfgs_scalar_block_and_safeguard():
    Wn = oracle.bfgs_block([2.0], [0.5], [3.0])  # s'y = 1.5 >= 0.2 s'Ws = 0.1
    assert Wn[0] == pytest.approx(6.0, rel=1e-14)  # secant: W+ = y/s
    # kappa = min(s'Ws, s'r) <= eps_m: the block is left unchanged
    w = [1.3, 0.2, 0.9]
    assert np.all(oracle.bfgs_block(w, [1e-9, 0.0], [5.0, 1.0]) == w)
    assert np.all(oracle.bfgs_block([1.3], [0.0], [1.0]) == [1.3])


# ---------------------------------------------------------------- OCPs

M = W.model(120)
V = M["V"]


def ctrl(N, tol):
    c = W.nmpc(N)
    c["sqp_tol"] = tol
    c["sqp_max_it"] = 200
    return c


def shoot(c, x0, u):
    """Single shooting: states of the OCP (in K) for inputs u (OCP units)."""
    Fconv = c["u_scale"] / 60000.0
    xs = [x0]
    for v in u:
        xF, _, _ = oracle.rk4_interval(M, c["n_rk4"], M["Ts"], xs[-1] * c["x_scale"], v, Fconv)
        xs.append(xF / c["x_scale"])
    return np.array(xs)


def objective(c, x, zb):
    z = x * c["x_scale"] / V
    return float(np.sum(c["Qz"] * (z[1:] - zb[1:]) ** 2 * M["Ts"]))


def kkt_residuals(c, x0, zb, u, x, lam, pil, piu):
    """Stationarity of L = f - lam^T g - pil^T (u - umin) - piu^T (umax - u)
    with the gradients of f and of g_k = F(x_k, u_k) - x_{k+1} taken by central
    differences of the single-interval map."""
    N = len(u)
    Fconv = c["u_scale"] / 60000.0
    xs_ = c["x_scale"]

    def Fk(xk, v):
        return oracle.rk4_interval(M, c["n_rk4"], M["Ts"], xk * xs_, v, Fconv)[0] / xs_

    h = 1e-6
    gu = np.zeros(N)
    gx = np.zeros(N + 1)
    for k in range(N):
        xk = x0 if k == 0 else x[k]
        dFdu = (Fk(xk, u[k] + h) - Fk(xk, u[k] - h)) / (2 * h)
        gu[k] = -lam[k] * dFdu - pil[k] + piu[k]
        if k >= 1:
            dFdx = (Fk(xk + h, u[k]) - Fk(xk - h, u[k])) / (2 * h)
            gx[k] += -lam[k] * dFdx
    for k in range(1, N + 1):
        gx[k] += 2 * c["Qz"] * (x[k] * xs_ / V - zb[k]) * M["Ts"] * xs_ / V + lam[k - 1]
    g = np.array([Fk(x0 if k == 0 else x[k], u[k]) - x[k + 1] for k in range(N)])
    return gu, gx[1:], g


@pytest.mark.parametrize("N,x0,zset", [(3, 280.0, 285.0), (5, 289.0, 290.0),
                                      (8, 330.0, 340.0), (20, 300.0, 290.0)])
def test_sqp_returns_kkt_point(N, x0, zset):
    c = ctrl(N, 1e-8)
    zb = np.full(N + 1, zset)
    v0 = 0.4
    u0 = np.full(N, v0)
    xw = np.full(N + 1, x0)
    u, x, lam, pil, piu, info = oracle.sqp(M, c, M["EaR"], x0, zb, u0, xw)
    assert info["status"] == 0
    assert info["kkt_grad"] <= 1e-8 and info["kkt_eq"] <= 1e-8
    gu, gx, g = kkt_residuals(c, x0, zb, u, x, lam, pil, piu)
    assert np.max(np.abs(g)) <= 1e-8
    assert np.max(np.abs(gu)) <= 1e-5 and np.max(np.abs(gx)) <= 1e-5  # FD accuracy
    lo, hi = c["u_min"] / c["u_scale"], c["u_max"] / c["u_scale"]
    assert np.all(u >= lo) and np.all(u <= hi)
    assert np.all(pil >= -1e-12) and np.all(piu >= -1e-12)
    assert np.all(np.abs(pil * (u - lo)) <= 1e-7) and np.all(np.abs(piu * (hi - u)) <= 1e-7)


@pytest.mark.parametrize("x0,z1,z2", [(280.0, 282.0, 282.0), (289.5, 290.0, 290.0),
                                      (300.0, 295.0, 290.0), (336.0, 340.0, 340.0),
                                      (276.0, 290.0, 300.0)])
def test_sqp_matches_grid_search_on_horizon_two(x0, z1, z2):
    """Horizon N = 2: the objective over (u0, u1) in the box is minimised by a
    201 x 201 grid and a bounded local refinement from the best grid points; the
    SQP objective must not be worse."""
    from scipy.optimize import minimize

    c = ctrl(2, 1e-8)
    zb = np.array([0.0, z1, z2])

    def fobj(uv):
        return objective(c, shoot(c, x0, uv), zb)

    g = np.linspace(0.0, 1.0, 201)
    vals = np.array([[fobj((a, b)) for b in g] for a in g])
    best = np.argsort(vals.ravel())[:5]
    fbest = np.inf
    for idx in best:
        a, b = g[idx // 201], g[idx % 201]
        r = minimize(fobj, [a, b], bounds=[(0, 1), (0, 1)], method="L-BFGS-B",
                     options=dict(ftol=1e-15, gtol=1e-12))
        fbest = min(fbest, r.fun, vals.ravel()[idx])
    u, x, lam, pil, piu, info = oracle.sqp(M, c, M["EaR"], x0, zb, [0.5, 0.5], [x0] * 3)
    assert info["status"] == 0
    fsqp = objective(c, shoot(c, x0, u), zb)
    assert fsqp <= fbest + 1e-9 * max(1.0, abs(fbest))


# ------------------------------------------------------------------ weighted objective

def weighted_objective(c, x, u, zb):
    """Extended objective: the paper's output term plus R_u (v_{k-1} - vbar_k)^2 T_s
    and Q_n (z_N - zbar_N)^2, vbar_k the steady-state input of zbar_k."""
    Fconv = c["u_scale"] / 60000.0
    z = x * c["x_scale"] / V
    f = np.sum(c["Qz"] * (z[1:] - zb[1:]) ** 2 * M["Ts"])
    vbar = np.array([oracle.Fss(M, zk) / Fconv for zk in zb[1:]])
    f += np.sum(c["Ru"] * (np.asarray(u) - vbar) ** 2 * M["Ts"])
    f += c["Qn"] * (z[-1] - zb[-1]) ** 2
    return float(f)


@pytest.mark.parametrize("Ru,Qn", [(0.5, 0.0), (0.0, 4.0), (2.0, 1.0)])
def test_weighted_objective_matches_grid_search_on_horizon_two(Ru, Qn):
    from scipy.optimize import minimize

    c = dict(ctrl(2, 1e-8), Ru=Ru, Qn=Qn)
    x0 = 300.0
    zb = np.array([0.0, 305.0, 310.0])

    def fobj(uv):
        return weighted_objective(c, shoot(c, x0, uv), uv, zb)

    g = np.linspace(0.0, 1.0, 101)
    vals = np.array([[fobj((a, b)) for b in g] for a in g])
    fbest = np.inf
    for idx in np.argsort(vals.ravel())[:5]:
        a, b = g[idx // 101], g[idx % 101]
        r = minimize(fobj, [a, b], bounds=[(0, 1), (0, 1)], method="L-BFGS-B",
                     options=dict(ftol=1e-15, gtol=1e-12))
        fbest = min(fbest, r.fun, vals.ravel()[idx])
    u, x, lam, pil, piu, info = oracle.sqp(M, c, M["EaR"], x0, zb, [0.5, 0.5], [x0] * 3)
    assert info["status"] == 0 and info["kkt_grad"] <= 1e-8
    assert fobj(u) <= fbest + 1e-9 * max(1.0, abs(fbest))
    assert info["f"] == pytest.approx(fobj(u), rel=1e-9)


def test_large_input_weight_drives_the_inputs_to_the_steady_state():
    """Q_z = 0 and R_u dominant: the minimiser is the reference input vbar_k
    itself (clipped into the bounds), whatever the set-points ask of z."""
    N = 6
    c = dict(ctrl(N, 1e-10), Qz=0.0, Ru=1.0, Qn=0.0)
    x0 = 300.0
    zb = np.array([0.0, 282.0, 282.0, 290.0, 290.0, 300.0, 300.0])
    u, x, lam, pil, piu, info = oracle.sqp(M, c, M["EaR"], x0, zb, np.full(N, 0.5),
                                           np.full(N + 1, x0))
    assert info["status"] == 0
    Fconv = c["u_scale"] / 60000.0
    vbar = np.clip([oracle.Fss(M, z) / Fconv for z in zb[1:]], 0.0, 1.0)
    np.testing.assert_allclose(u, vbar, rtol=0, atol=1e-8)


# ------------------------------------------------------------------ OCP sensitivity

def _solve(c, x0, zb, N, converged=True):
    u, x, lam, pil, piu, info = oracle.sqp(M, c, M["EaR"], x0, zb, np.full(N, 0.5),
                                           np.full(N + 1, x0))
    # near 1e-8 the merit's rounding floor can stop a solve at the iteration
    # limit with its input already accurate; only the base point must converge
    if converged:
        assert info["status"] == 0, info
    return u, x, lam, pil, piu


# cases whose first input is interior (above the set-point the reactor needs
# flow to cool; below it the input sits on its lower bound)
INTERIOR = [(290.5, 290.0), (340.5, 340.0)]


@pytest.mark.parametrize("x0,zset", INTERIOR)
def test_ocp_sensitivity_matches_differences_of_the_solution(x0, zset):
    """du_0/d(x_0, Q_z, R_u, Q_n) from the KKT system against central
    differences of OCP solutions converged to 1e-9 (the steps are sized to
    that accuracy)."""
    N = 8
    c = dict(ctrl(N, 1e-8), Ru=0.3, Qn=2.0)
    zb = np.full(N + 1, zset)
    u, x, lam, pil, piu = _solve(c, x0, zb, N)
    assert 0.0 < u[0] < 1.0
    st, s = oracle.ocp_sens(M, c, M["EaR"], x0, zb, u, x, lam, pil, piu)
    assert st == 0
    h = 1e-2
    fd = [(_solve(c, x0 + h, zb, N, False)[0][0] - _solve(c, x0 - h, zb, N, False)[0][0]) / (2 * h)]
    for key in ("Qz", "Ru", "Qn"):
        hk = 1e-3 * max(1.0, c[key])
        up = _solve(dict(c, **{key: c[key] + hk}), x0, zb, N, False)[0][0]
        dn = _solve(dict(c, **{key: c[key] - hk}), x0, zb, N, False)[0][0]
        fd.append((up - dn) / (2 * hk))
    np.testing.assert_allclose(s[0], fd[0], rtol=1e-5)
    np.testing.assert_allclose(s[1:], fd[1:], rtol=1e-4, atol=1e-7 * abs(fd[0]))


def test_ocp_sensitivity_exact_zeros():
    """With R_u = Q_n = 0 the minimiser does not depend on Q_z (the objective
    only scales), and an input held on an active bound does not move."""
    N = 8
    c = ctrl(N, 1e-8)
    x0, zs = INTERIOR[0]
    zb = np.full(N + 1, zs)
    u, x, lam, pil, piu = _solve(c, x0, zb, N)
    st, s = oracle.ocp_sens(M, c, M["EaR"], x0, zb, u, x, lam, pil, piu)
    assert st == 0 and abs(s[0]) > 0.1
    assert abs(s[1]) <= 1e-7 * abs(s[0])
    zb2 = np.full(N + 1, 306.0)          # heating: the first input on its lower bound
    u2, x2, lam2, pil2, piu2 = _solve(c, 300.0, zb2, N)
    assert u2[0] == 0.0 and pil2[0] > 1e-10
    st2, s2 = oracle.ocp_sens(M, c, M["EaR"], 300.0, zb2, u2, x2, lam2, pil2, piu2)
    assert st2 == 0 and np.all(np.abs(s2) <= 1e-12)
