"""Pins of the oracle's QP subproblem solver, Eq. (QP-subproblem)/(nlpsqp_qp):
  min sum_k 1/2 [dx_k; du_k]^T W_k [dx_k; du_k] + q_k dx_k + r_k du_k
  s.t. dx_{k+1} = A_k dx_k + B_k du_k + b_k, dx_0 = 0, lb_k <= du_k <= ub_k.

The oracle condenses and runs a primal active-set method.  The pins below do
not: small problems are solved by enumerating every active set and solving the
full (uncondensed) KKT system of each with numpy, and larger ones are checked
against the KKT optimality certificate of a convex QP.
"""
import itertools

import numpy as np
import pytest

import oracle


def random_qp(N, rng, tight=True):
    A = rng.uniform(0.6, 1.2, N)
    B = rng.uniform(-2.0, 2.0, N)
    b = rng.normal(0.0, 0.5, N)
    Wxx, Wxu, Wuu = np.zeros(N + 1), np.zeros(N + 1), np.zeros(N + 1)
    for k in range(N + 1):
        L = rng.normal(size=(2, 2)) + 1.5 * np.eye(2)
        Wk = L @ L.T + 0.1 * np.eye(2)
        Wxx[k], Wxu[k], Wuu[k] = Wk[0, 0], Wk[0, 1], Wk[1, 1]
    Wxx[0] = Wxu[0] = 0.0
    Wxu[N] = Wuu[N] = 0.0
    q = rng.normal(0.0, 2.0, N + 1)
    q[0] = 0.0
    r = rng.normal(0.0, 2.0, N)
    w = 0.3 if tight else 1e6
    lb = -rng.uniform(0.0 if tight else 0.5 * w, w, N)
    ub = rng.uniform(0.0 if tight else 0.5 * w, w, N)
    return A, B, b, Wxx, Wxu, Wuu, q, r, lb, ub


def full_kkt(A, B, b, Wxx, Wxu, Wuu, q, r, lb, ub, fixed):
    """Solve the uncondensed equality QP with du_i fixed at its bound for
    fixed[i] in {'l', 'u'}.  Unknowns z = [du_0..du_{N-1}, dx_1..dx_N], mu (N),
    one multiplier per fixed bound; returns (du, dx, mu, nul, nuu)."""
    N = len(B)
    iu = lambda k: k            # du_k
    ix = lambda k: N + k - 1    # dx_k, k >= 1
    nz = 2 * N
    H = np.zeros((nz, nz))
    g = np.zeros(nz)
    for k in range(N):
        H[iu(k), iu(k)] += Wuu[k]
        g[iu(k)] += r[k]
    for k in range(1, N + 1):
        H[ix(k), ix(k)] += Wxx[k]
        g[ix(k)] += q[k]
    for k in range(1, N):
        H[ix(k), iu(k)] += Wxu[k]
        H[iu(k), ix(k)] += Wxu[k]
    E = np.zeros((N, nz))    # dynamics: A dx_k + B du_k - dx_{k+1} = -b_k
    e = -b.copy()
    for k in range(N):
        if k >= 1:
            E[k, ix(k)] = A[k]
        E[k, iu(k)] = B[k]
        E[k, ix(k + 1)] = -1.0
    act = sorted(fixed)
    na = len(act)
    Cb = np.zeros((na, nz))  # fixed bounds: du_i = bound
    cb = np.zeros(na)
    for a, i in enumerate(act):
        Cb[a, iu(i)] = 1.0
        cb[a] = lb[i] if fixed[i] == "l" else ub[i]
    # stationarity: H z + g - E^T mu - Cb^T nu = 0 with nu = nul (lower) or -nuu (upper)
    K = np.block([[H, -E.T, -Cb.T], [E, np.zeros((N, N)), np.zeros((N, na))],
                  [Cb, np.zeros((na, N)), np.zeros((na, na))]])
    rhs = np.concatenate([-g, e, cb])
    sol = np.linalg.solve(K, rhs)
    z, mu, nu = sol[:nz], sol[nz:nz + N], sol[nz + N:]
    du = z[:N]
    dx = np.concatenate([[0.0], z[N:]])
    nul, nuu = np.zeros(N), np.zeros(N)
    for a, i in enumerate(act):
        if fixed[i] == "l":
            nul[i] = nu[a]
        else:
            nuu[i] = -nu[a]
    return du, dx, mu, nul, nuu


def brute_force(*qp):
    N = len(qp[1])
    lb, ub = qp[8], qp[9]
    found = []
    for pattern in itertools.product("fLU", repeat=N):
        fixed = {i: ("l" if p == "L" else "u") for i, p in enumerate(pattern) if p != "f"}
        du, dx, mu, nul, nuu = full_kkt(*qp, fixed)
        tol = 1e-12
        if np.any(du < lb - tol) or np.any(du > ub + tol):
            continue
        if np.any(nul < -tol) or np.any(nuu < -tol):
            continue
        found.append((du, dx, mu, nul, nuu))
    assert found, "no KKT point among the 3^N active sets"
    # strictly convex: every KKT point is the same point
    for f in found[1:]:
        assert np.allclose(f[0], found[0][0], atol=1e-10)
    return found[0]


@pytest.mark.parametrize("N", [1, 2, 3, 4])
@pytest.mark.parametrize("seed", range(12))
def test_qp_matches_active_set_enumeration(N, seed):
    rng = np.random.default_rng(100 * N + seed)
    qp = random_qp(N, rng)
    du, dx, mu, nul, nuu = brute_force(*qp)
    res = oracle.qp_solve(*qp)
    assert res["status"] == 0
    assert np.allclose(res["du"], du, rtol=1e-10, atol=1e-11)
    assert np.allclose(res["dx"], dx, rtol=1e-10, atol=1e-11)
    assert np.allclose(res["mu"], mu, rtol=1e-9, atol=1e-10)
    assert np.allclose(res["nul"], nul, rtol=1e-9, atol=1e-10)
    assert np.allclose(res["nuu"], nuu, rtol=1e-9, atol=1e-10)


@pytest.mark.parametrize("N", [5, 20, 40])
def test_qp_unconstrained_equals_dense_kkt_solve(N):
    rng = np.random.default_rng(N)
    qp = random_qp(N, rng, tight=False)
    du, dx, mu, _, _ = full_kkt(*qp, {})
    assert np.all(du > qp[8]) and np.all(du < qp[9])
    res = oracle.qp_solve(*qp)
    assert res["status"] == 0
    assert np.allclose(res["du"], du, rtol=1e-9, atol=1e-10)
    assert np.allclose(res["mu"], mu, rtol=1e-8, atol=1e-9)
    assert np.all(res["nul"] == 0.0) and np.all(res["nuu"] == 0.0)


@pytest.mark.parametrize("N", [10, 20, 30, 60])
@pytest.mark.parametrize("seed", range(4))
def test_qp_solution_satisfies_kkt_certificate(N, seed):
    """Convex QP: primal feasibility, stationarity, dual feasibility and
    complementarity together prove optimality."""
    rng = np.random.default_rng(1000 + 10 * N + seed)
    A, B, b, Wxx, Wxu, Wuu, q, r, lb, ub = qp = random_qp(N, rng)
    res = oracle.qp_solve(*qp)
    assert res["status"] == 0
    du, dx, mu, nul, nuu = (res[k] for k in ("du", "dx", "mu", "nul", "nuu"))
    scale = 1.0 + np.max(np.abs(np.concatenate([q, r, b])))
    # primal
    assert dx[0] == 0.0
    for k in range(N):
        Ak = A[k] if k >= 1 else 0.0
        assert abs(Ak * dx[k] + B[k] * du[k] + b[k] - dx[k + 1]) <= 1e-10 * scale
    assert np.all(du >= lb - 1e-12) and np.all(du <= ub + 1e-12)
    # dual feasibility and complementarity
    assert np.all(nul >= -1e-10 * scale) and np.all(nuu >= -1e-10 * scale)
    assert np.all(np.abs(nul * (du - lb)) <= 1e-9 * scale)
    assert np.all(np.abs(nuu * (ub - du)) <= 1e-9 * scale)
    # stationarity in du and dx
    for k in range(N):
        cross = Wxu[k] * dx[k] if k >= 1 else 0.0
        su = Wuu[k] * du[k] + cross + r[k] - mu[k] * B[k] - nul[k] + nuu[k]
        assert abs(su) <= 1e-9 * scale
    for k in range(1, N):
        sx = Wxx[k] * dx[k] + Wxu[k] * du[k] + q[k] - mu[k] * A[k] + mu[k - 1]
        assert abs(sx) <= 1e-9 * scale * (1 + np.max(np.abs(mu)))
    assert abs(Wxx[N] * dx[N] + q[N] + mu[N - 1]) <= 1e-9 * scale


def test_qp_degenerate_fixed_input():
    """u_min = u_max: every du is pinned at 0 and the dynamics give dx."""
    rng = np.random.default_rng(5)
    A, B, b, Wxx, Wxu, Wuu, q, r, lb, ub = random_qp(6, rng)
    lb[:] = 0.0
    ub[:] = 0.0
    res = oracle.qp_solve(A, B, b, Wxx, Wxu, Wuu, q, r, lb, ub)
    assert res["status"] == 0
    assert np.all(res["du"] == 0.0)
    dx = [0.0]
    for k in range(6):
        dx.append((A[k] if k else 0.0) * dx[-1] + b[k])
    assert np.allclose(res["dx"], dx, rtol=1e-14, atol=1e-15)
