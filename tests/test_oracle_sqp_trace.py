"""Pins of the decisions inside the oracle's SQP iterations (Sec. IV), read
from a per-iteration trace of real OCPs of the one-state CSTR model:

* the penalty weights of the l1 merit (Sec. IV-B): sigma = |mu| at the first
  iteration, then sigma = max(|mu|, (sigma_prev + |mu|) / 2);
* the merit T(0) = f + sigma^T |g| and its slope DT(0) = grad f^T dxi -
  sigma^T |g|, which must be a descent slope (it is at most
  -dxi^T W dxi - (sigma - |mu|)^T |g| for a positive definite W);
* the backtracking line search (Eq. Armijo): trial steps 1, 1/2, 1/4, ...,
  every rejected trial violates T(alpha) <= T(0) + c1 alpha DT(0) with
  c1 = 1e-4, the accepted one satisfies it;
* the scaled convergence test (Eq. convergence): s_d = max(s_max,
  (||lam||_1 + ||pi_l||_1 + ||pi_u||_1) / (m_e + m_l + m_u)) / s_max with
  s_max = 100 and m_e + m_l + m_u = 3N (N dynamics rows and N lower and N
  upper input bounds), and the stop exactly when both scaled norms are
  within the tolerance;
* the Hessian reset (Sec. IV-C): when a block is not positive definite
  after the damped update, every block is set to the identity.

The OCPs below were chosen so that the trace shows each rule where it
matters: steps that backtrack, an accepted step whose Armijo ratio lies
between 1e-4 and 0.1, penalty weights that keep part of their old value, and
multipliers whose mean exceeds s_max.  The coverage tests assert that.
"""
import numpy as np
import pytest

import oracle
from paper_2212_02197_gb300 import workloads as W

C1, BETA, S_MAX = 1e-4, 0.5, 100.0
M = W.model(120)

# (N, Q_z, x0, set-point, warm-start input, warm-start state)
CASES = [
    (8, 10000.0, 283.7441357847265, 300.6107568411557, 0.6488199317970121, 298.141151417851),
    (6, 10000.0, 287.5119800680615, 287.88688393571175, 0.9540027078139908, 289.5784444505533),
    (6, 100.0, 336.9975308585508, 321.62265310048, 0.09142453216616109, 309.34870140291423),
    (4, 100.0, 276.72880518056576, 299.0161127717473, 0.008636209165301167, 296.6335758230862),
    (3, 10000.0, 281.00292647194175, 339.96138322609625, 0.17840618099979666, 298.40208842879554),
    (8, 1.0, 329.31568442535206, 297.21999321892855, 0.9520073955698587, 343.92304836547567),
    (20, 1.0, 300.0, 290.0, 0.4, 300.0),
]


def solve(case, tol=1e-8, max_it=100):
    N, Qz, x0, zs, v0, xw = case
    c = W.nmpc(N)
    c.update(sqp_tol=tol, sqp_max_it=max_it, Qz=Qz)
    zb = np.full(N + 1, zs)
    out = oracle.sqp_traced(M, c, M["EaR"], x0, zb, np.full(N, v0), np.full(N + 1, xw))
    return c, out


@pytest.fixture(scope="module")
def traces():
    return [solve(case) for case in CASES]


def qp_rows(rows):
    return [r for r in rows if r["stop"] == -1]


def test_penalty_weights_follow_the_update_rule(traces):
    kept = 0
    for c, (_, _, _, _, _, info, rows) in traces:
        prev = None
        for r in qp_rows(rows):
            am = np.abs(r["mu"])
            want = am if r["l"] == 0 else np.maximum(am, 0.5 * (prev + am))
            assert np.array_equal(r["sigma"], want), r["l"]
            if r["l"] > 0:
                kept += int(np.sum(want > am))
            prev = r["sigma"]
    assert kept > 0   # the rule's memory term decided some weights


def test_merit_and_its_slope(traces):
    for c, (_, _, _, _, _, info, rows) in traces:
        for r in qp_rows(rows):
            pen = float(np.sum(r["sigma"] * np.abs(r["g"])))
            dfd = float(np.sum(r["r"] * r["du"]) + np.sum(r["q"][1:] * r["dx"][1:]))
            assert r["T0"] == pytest.approx(r["f"] + pen, rel=1e-13, abs=1e-13)
            assert r["DT0"] == pytest.approx(dfd - pen, rel=1e-10, abs=1e-10 * (abs(dfd) + pen))
            step = np.max(np.abs(r["du"])) + np.max(np.abs(r["dx"]))
            if step > 1e-12:
                assert r["DT0"] < 0.0   # a descent direction of the merit


def armijo_ok(r, i):
    return r["f_trial"][i] + r["pen_trial"][i] <= r["T0"] + C1 * r["alpha"][i] * r["DT0"]


def test_armijo_backtracking(traces):
    backtracks, mid_ratio = 0, 0
    for c, (_, _, _, _, _, info, rows) in traces:
        for r in qp_rows(rows):
            n = r["n_trials"]
            assert n >= 1
            assert np.array_equal(r["alpha"], BETA ** np.arange(n))
            for i in range(n - 1):
                assert not armijo_ok(r, i), (r["l"], i)
            if r["accepted"]:
                assert armijo_ok(r, n - 1)
                a = r["alpha"][-1]
                rho = (r["f_trial"][-1] + r["pen_trial"][-1] - r["T0"]) / (a * r["DT0"])
                mid_ratio += int(C1 <= rho < 0.1)
            else:
                assert n == c["ls_max"] + 1 and not armijo_ok(r, n - 1)
            backtracks += int(n > 1)
    assert backtracks > 0     # some line searches halved the step
    assert mid_ratio > 0      # some accepted step has 1e-4 <= ratio < 0.1


def test_convergence_test_scaling(traces):
    big = 0
    for c, (_, _, _, _, _, info, rows) in traces:
        N = c["N"]
        for r in rows:
            mult1 = float(np.sum(np.abs(r["lam"]) + np.abs(r["pil"]) + np.abs(r["piu"])))
            s_d = max(S_MAX, mult1 / (3 * N)) / S_MAX
            assert r["s_d"] == pytest.approx(s_d, rel=1e-14)
            big += int(mult1 / N > S_MAX)
            # gradient of the Lagrangian L = f - lam^T g - pil^T (u - umin) - piu^T (umax - u)
            lam = r["lam"]
            gu = r["r"] - lam * r["B"] - r["pil"] + r["piu"]
            gx = r["q"][1:].copy()
            gx[:-1] += -lam[1:] * r["A"][1:]
            gx += lam
            raw = max(np.max(np.abs(gu)), np.max(np.abs(gx)))
            assert r["kkt_grad_raw"] == pytest.approx(raw, rel=1e-12, abs=1e-14)
            assert r["kkt_grad"] == pytest.approx(r["kkt_grad_raw"] / s_d, rel=1e-14)
            assert r["kkt_eq"] == np.max(np.abs(r["g"]))
            converged = r["kkt_grad"] <= c["sqp_tol"] and r["kkt_eq"] <= c["sqp_tol"]
            assert converged == (r["stop"] == 0)
        assert rows[-1]["stop"] == 0 and info["status"] == 0
        assert info["iters"] == len(rows) - 1
    assert big > 0   # multipliers large enough that the 3N average matters


def test_iteration_limit_stops_before_the_qp():
    c, (_, _, _, _, _, info, rows) = solve(CASES[6], tol=1e-12, max_it=2)
    assert info["status"] == 1 and info["iters"] == 2
    assert [r["l"] for r in rows] == [0, 1, 2]
    assert rows[-1]["stop"] == 1 and rows[-1]["n_trials"] == 0


def test_hessian_reset_sets_every_block_to_the_identity():
    """One block left indefinite (its step is zero, so the damped update keeps
    it): all blocks, including the ones the update just changed, return to I."""
    rng = np.random.default_rng(7)
    N = 5
    W0 = np.tile([1.0, 0.0, 1.0], (N + 1, 1))
    for k in range(1, N):
        L = rng.normal(size=(2, 2)) + 2 * np.eye(2)
        A = L @ L.T
        W0[k] = [A[0, 0], A[0, 1], A[1, 1]]
    W0[3] = [1.0, 2.0, 1.0]                        # eigenvalues 3 and -1
    s_u, y_u = rng.normal(size=N), rng.normal(size=N)
    s_x, y_x = rng.normal(size=N + 1), rng.normal(size=N + 1)
    s_x[0] = y_x[0] = 0.0
    s_u[3] = s_x[3] = 0.0                          # block 3 is not updated
    Wn, reset = oracle.bfgs_update_blocks(W0, s_u, s_x, y_u, y_x)
    assert reset == 1
    assert np.array_equal(Wn, np.tile([1.0, 0.0, 1.0], (N + 1, 1)))
    # without the indefinite block: each block gets its damped update, no reset
    W0[3] = [2.0, 0.5, 1.5]
    s_u[3], s_x[3] = 0.3, -0.2
    Wn, reset = oracle.bfgs_update_blocks(W0, s_u, s_x, y_u, y_x)
    assert reset == 0
    for k in range(1, N):
        want = oracle.bfgs_block(W0[k], [s_x[k], s_u[k]], [y_x[k], y_u[k]])
        assert np.array_equal(Wn[k], want)
        Wk = np.array([[Wn[k][0], Wn[k][1]], [Wn[k][1], Wn[k][2]]])
        assert np.all(np.linalg.eigvalsh(Wk) > 0)
    assert Wn[0][0] == oracle.bfgs_block([W0[0][0]], [s_u[0]], [y_u[0]])[0]
    assert Wn[N][0] == oracle.bfgs_block([W0[N][0]], [s_x[N]], [y_x[N]])[0]
