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
