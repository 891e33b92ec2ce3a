"""The discrete adjoint of the PI closed loop (mc_pi_grad) against the oracle's
complex-step derivative, finite differences of the GPU's own mean Phi, and the
invariances the checkpointing must keep."""
import numpy as np
import pytest
import torch

import oracle
from paper_2212_02197_gb300 import mc, workloads as W
from paper_2212_02197_gb300.autograd import pi_mean_phi

pytestmark = pytest.mark.gpu

WL = "cstr_30k_x240_N20_fp64"   # 240 samples, inlet step +-5 K at a random time


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2212_02197_gb300 import _build

    _build.build()
    oracle.build()


def _grad(w, n, ckpt=20, ctrl=None, model=None):
    h = mc.MonteCarlo(model or w["model"], ctrl or w["pi"], n, w["seed"])
    h.pi_grad(ckpt)
    st = h.stats(timeout_ms=600000)
    g, phi, gm = h.grad(), h.phi(), h.grad_mean()
    h.close()
    return phi, g, gm, st


def test_adjoint_matches_complex_step_per_trajectory():
    w = W.get(WL)
    n = 300   # spans 3 blocks of 128 and a ragged tail
    phi, g, _, _ = _grad(w, n)
    ref_phi, ref = oracle.pi_grad(w["model"], w["pi"], w["seed"], 0, n)
    np.testing.assert_allclose(phi, ref_phi, rtol=1e-12, atol=0)
    scale = np.abs(ref).mean(axis=0)
    err = np.abs(g - ref) / (np.abs(ref) + 1e-6 * scale)
    assert np.all(np.isfinite(g))
    assert err.max() < 1e-8, err.max()


def test_adjoint_on_a_sample_of_the_full_study():
    """The full 30k launch; trajectories sampled across it against the oracle."""
    w = W.get(WL)
    n = w["n_traj"]
    _, g, gm, st = _grad(w, n)
    assert st["n_nonfinite"] == 0
    idx = np.linspace(0, n - 1, 40).astype(int)
    for j in idx:
        _, ref = oracle.pi_grad(w["model"], w["pi"], w["seed"], int(j), int(j) + 1)
        np.testing.assert_allclose(g[j], ref[0], rtol=1e-8, atol=1e-8 * np.abs(ref).max())
    np.testing.assert_allclose(gm, g.mean(axis=0), rtol=1e-12)


def test_checkpoint_interval_does_not_change_the_result():
    w = W.get(WL)
    _, g20, _, _ = _grad(w, 64, 20)
    for ck in (1, 7, 32):
        _, g, _, _ = _grad(w, 64, ck)
        assert np.array_equal(g, g20), ck


def test_phi_equals_the_plain_run():
    w = W.get(WL)
    phi, _, _, _ = _grad(w, 256)
    h = mc.MonteCarlo(w["model"], w["pi"], 256, w["seed"])
    h.run()
    ref = h.phi()
    h.close()
    np.testing.assert_allclose(phi, ref, rtol=1e-12, atol=0)


# central differences of mean Phi over the 30k study: step (relative to the
# gain) and the relative tolerance per gain (k_P, k_I, k_aw).  A trajectory
# whose input crosses a bound of the clip between k - h and k + h has a kink
# inside the difference interval and contributes an O(1) error to its own
# difference quotient; the anti-windup derivative, which is small, feels this
# most (the oracle's own differences are 5e-4 off there at h = 1e-5).  At
# h = 1e-6 the rounding of mean Phi (~229) over 2h adds its share.
FD_CASES = [(1e-5, (1e-4, 1e-4, 2e-3)), (1e-6, (1e-5, 1e-5, 1e-4))]


@pytest.mark.parametrize("step,tols", FD_CASES)
def test_mean_gradient_matches_central_differences_of_mean_phi(step, tols):
    w = W.get(WL)
    n = w["n_traj"]
    _, _, gm, _ = _grad(w, n)
    h = mc.MonteCarlo(w["model"], w["pi"], n, w["seed"])
    c = w["pi"]
    for q, k in enumerate(("kP", "kI", "kaw")):
        dk = step * abs(c[k])
        means = []
        for sgn in (1, -1):
            g = dict(kP=c["kP"], kI=c["kI"], kaw=c["kaw"])
            g[k] += sgn * dk
            h.set_pi_gains(g["kP"], g["kI"], g["kaw"])
            h.run()
            means.append(h.stats()["phi_mean"])
        fd = (means[0] - means[1]) / (2 * dk)
        assert fd == pytest.approx(gm[q], rel=tols[q]), (k, fd, gm[q])
    h.close()


def test_autograd_function():
    w = W.get(WL)
    h = mc.MonteCarlo(w["model"], w["pi"], 512, w["seed"])
    c = w["pi"]
    x = torch.tensor([c["kP"], c["kI"], c["kaw"]], dtype=torch.float64, requires_grad=True)
    y = pi_mean_phi(x, h)
    y.backward()
    gm = h.grad_mean()
    h.close()
    assert torch.allclose(x.grad, torch.tensor(gm, dtype=torch.float64), rtol=0, atol=0)
    _, _, gm2, st = _grad(w, 512)
    assert float(y) == pytest.approx(st["phi_mean"], rel=1e-15)


def test_edge_cases_and_errors():
    w = W.get(WL)
    # no control steps: Phi = (c_T(0) - z-bar(0))^2, which no gain moves
    phi, g, _, _ = _grad(w, 40, model=dict(w["model"], n_steps=0))
    assert np.all(g == 0.0) and np.all(np.isfinite(phi))
    # one step, checkpoint interval longer than the run
    _, g1, _, _ = _grad(w, 40, 32, model=dict(w["model"], n_steps=1))
    _, r1 = oracle.pi_grad(dict(w["model"], n_steps=1), w["pi"], w["seed"], 0, 40)
    np.testing.assert_allclose(g1, r1, rtol=1e-9, atol=1e-12)
    # empty range
    h = mc.MonteCarlo(w["model"], w["pi"], 10, w["seed"])
    with pytest.raises(mc.McError):
        h.grad_mean()                       # not run yet
    h.pi_grad(20, j0=3, j1=3)
    assert np.all(h.grad_mean() == 0.0)
    for bad in (0, 33):
        with pytest.raises(mc.McError):
            h.pi_grad(bad)
    with pytest.raises(mc.McError):
        h.set_pi_gains(float("nan"), 0.0, 0.0)
    h.close()
    with pytest.raises(mc.McError):
        _grad(w, 4, model=dict(w["model"], n_em=33))
    hn = mc.MonteCarlo(w["model"], w["nmpc"], 4, w["seed"])
    with pytest.raises(mc.McError):
        hn.pi_grad(20)
    with pytest.raises(mc.McError):
        hn.set_pi_gains(-1e-3, -1e-4, -1e-1)
    hn.close()
    hm = mc.MonteCarlo(w["model"], dict(w["pi"], precision="mixed"), 4, w["seed"])
    with pytest.raises(mc.McError):
        hm.pi_grad(20)
    hm.close()
