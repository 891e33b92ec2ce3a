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
