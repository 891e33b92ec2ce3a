"""Pins of the oracle's derivative of Phi_j with respect to the PI gains
(complex-step differentiation of the closed loop, Sec. V and VII).

The complex-step value is pinned against things it does not share code with:
central finite differences of the plain real oracle (or_run), extrapolated
by Richardson's rule; exact zeros where the PI law fixes them (no
saturation means the anti-windup term never acts; a fixed input means no gain
matters); and the real part, which must be the real simulation's Phi."""
import numpy as np
import pytest

import oracle
from paper_2212_02197_gb300 import workloads as W

GAINS = ("kP", "kI", "kaw")


@pytest.fixture(scope="module")
def w():
    oracle.build()
    w = W.get("cstr_30k_x240_N20_fp64")
    return dict(w, model=dict(w["model"], n_steps=80))


def _phi(w, ctrl, j):
    return oracle.run(w["model"], ctrl, w["seed"], j, j + 1, threads=1)["phi"][0]


def _fd(w, j, q, rel):
    """Central difference of the real oracle's Phi_j in gain q, step rel*|k|."""
    c = w["pi"]
    h = rel * abs(c[GAINS[q]])
    up = _phi(w, dict(c, **{GAINS[q]: c[GAINS[q]] + h}), j)
    dn = _phi(w, dict(c, **{GAINS[q]: c[GAINS[q]] - h}), j)
    return (up - dn) / (2 * h)


def test_real_part_is_the_simulated_phi(w):
    phi, _ = oracle.pi_grad(w["model"], w["pi"], w["seed"], 0, 16)
    ref = oracle.run(w["model"], w["pi"], w["seed"], 0, 16)["phi"]
    np.testing.assert_allclose(phi, ref, rtol=1e-14, atol=0)


@pytest.mark.parametrize("j", [0, 3, 11])
def test_complex_step_matches_richardson_central_differences(w, j):
    _, d = oracle.pi_grad(w["model"], w["pi"], w["seed"], j, j + 1)
    for q in range(3):
        d1, d2 = _fd(w, j, q, 1e-4), _fd(w, j, q, 5e-5)
        rich = (4 * d2 - d1) / 3            # O(h^4)
        scale = max(abs(rich), 1e-6 * abs(d[0, 0]))
        # a saturation switch inside [k - h, k + h] breaks the smooth expansion;
        # the two step sizes then disagree and the point is not a pin
        if abs(d1 - d2) > 1e-3 * scale:
            continue
        assert abs(d[0, q] - rich) <= 1e-6 * scale, (q, d[0, q], rich)


def test_each_gain_moves_phi(w):
    _, d = oracle.pi_grad(w["model"], w["pi"], w["seed"], 0, 8)
    assert np.all(np.isfinite(d))
    assert np.all(np.abs(d[:, :2]).max(axis=0) > 0)


def test_anti_windup_gain_is_inert_without_saturation(w):
    wide = dict(w["pi"], u_min=-1e9, u_max=1e9)
    _, d = oracle.pi_grad(w["model"], wide, w["seed"], 0, 4)
    assert np.all(d[:, 2] == 0.0)
    assert np.all(d[:, 0] != 0.0)


def test_fixed_input_makes_every_gain_inert(w):
    fixed = dict(w["pi"], u_min=300.0, u_max=300.0)
    phi, d = oracle.pi_grad(w["model"], fixed, w["seed"], 0, 4)
    assert np.all(np.isfinite(phi))
    assert np.all(d == 0.0)


def test_complex_step_is_insensitive_to_its_step(w):
    # no subtractive cancellation: steps 1e-20 and 1e-30 of |k| agree to rounding
    c = w["pi"]
    for q in range(3):
        h = abs(c[GAINS[q]])
        _, a = oracle.pi_phi_cs(w["model"], c, w["seed"], 5, q, 1e-20 * h)
        _, b = oracle.pi_phi_cs(w["model"], c, w["seed"], 5, q, 1e-30 * h)
        assert a == pytest.approx(b, rel=1e-12)


# ------------------------------------------------------------------ NMPC weights

@pytest.fixture(scope="module")
def wn():
    oracle.build()
    w = W.get("cstr_100x120_N20_fp64")
    return dict(w, model=dict(w["model"], n_steps=12))


def test_nmpc_grad_real_part_is_the_simulated_phi(wn):
    c = dict(wn["nmpc"], Ru=0.2, Qn=1.0)
    phi, _, fails = oracle.nmpc_grad(wn["model"], c, wn["seed"], 0, 6)
    ref = oracle.run(wn["model"], c, wn["seed"], 0, 6)["phi"]
    np.testing.assert_allclose(phi, ref, rtol=1e-12, atol=0)
    assert np.all(fails == 0)


def test_nmpc_grad_matches_central_differences_with_tight_ocps(wn):
    """With the OCPs solved to 1e-8, the closed loop's Phi is the composition
    the implicit derivative describes; central differences of the plain
    oracle (steps 2e-3 of each weight) agree."""
    c = dict(wn["nmpc"], Ru=0.2, Qn=1.0, sqp_tol=1e-8, sqp_max_it=300)
    _, d, _ = oracle.nmpc_grad(wn["model"], c, wn["seed"], 0, 6)
    fd = []
    for k in ("Qz", "Ru", "Qn"):
        hk = 2e-3 * c[k]
        a = oracle.run(wn["model"], dict(c, **{k: c[k] + hk}), wn["seed"], 0, 6)["phi"]
        b = oracle.run(wn["model"], dict(c, **{k: c[k] - hk}), wn["seed"], 0, 6)["phi"]
        fd.append((a - b) / (2 * hk))
    fd = np.array(fd).T
    scale = np.abs(fd).max(axis=0)
    assert np.all(np.abs(d - fd) <= 1e-3 * np.abs(fd) + 1e-4 * scale), np.abs(d - fd) / scale


def test_nmpc_grad_paper_objective_is_invariant_to_the_output_weight(wn):
    """R_u = Q_n = 0: every KKT point is invariant to scaling Q_z, so the
    derivative along Q_z vanishes, while R_u and Q_n still move Phi."""
    m = dict(wn["model"], n_steps=60)     # past the first set-point change
    _, d, _ = oracle.nmpc_grad(m, wn["nmpc"], wn["seed"], 0, 6)
    assert np.abs(d[:, 1]).max() > 0
    # the OCPs stop at the 1e-5 KKT test, so the invariance holds to that order
    assert np.all(np.abs(d[:, 0]) <= 1e-4 * np.abs(d[:, 1:]).max())
