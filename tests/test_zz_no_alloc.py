"""mc_reduce_noalloc: the statistics reduction for callers that cannot call
cudaMalloc (a device-memory budget fixed up front, a loop that must never
enter the allocator, or a host framework that owns all device memory).

It reduces per-trajectory Phi and counters the caller already holds on the
device, using only the library's static device scratch.  Its result must
match mc_stats of the run that produced those arrays, call after call (the
scratch keeps the previous call's contents).  Collected last on purpose.
"""
import numpy as np
import pytest

from paper_2212_02197_gb300 import mc, workloads as W

pytestmark = pytest.mark.gpu


def _same(a, b):
    assert a["n_traj"] == b["n_traj"]
    for k in ("n_ocp_failed", "sqp_iters", "ls_trials", "n_hess_reset", "n_ls_fail", "qp_iters",
              "n_nonfinite", "qp_fail"):
        assert a[k] == b[k], k
    assert a["phi_mean"] == pytest.approx(b["phi_mean"], rel=1e-13)
    assert a["phi_var"] == pytest.approx(b["phi_var"], rel=1e-11)
    assert a["phi_min"] == b["phi_min"] and a["phi_max"] == b["phi_max"]
    assert a["bin_lo"] == b["bin_lo"] and a["bin_hi"] == b["bin_hi"]
    assert np.array_equal(a["hist"], b["hist"])


@pytest.mark.parametrize("kind", ["nmpc", "pi"])
def test_reduce_noalloc_matches_mc_stats_twice(kind):
    import torch

    from paper_2212_02197_gb300 import _build

    _build.build()
    w = W.get("cstr_100x120_N20_fp64")
    m = dict(w["model"], n_steps=30)
    n = 300
    h = mc.MonteCarlo(m, w[kind], n, w["seed"])
    h.set_histogram(32)
    h.run()
    ref = h.stats(timeout_ms=600000)
    phi = torch.empty(n, dtype=torch.float64, device="cuda")
    cnt = torch.empty((n, mc.N_COUNTERS), dtype=torch.int32, device="cuda")
    h.phi(out=phi)
    h.counters_to(cnt)
    torch.cuda.synchronize()
    for _ in range(2):
        got = mc.reduce_noalloc(phi, cnt, n, n_bins=32)
        _same(got, ref)
    # a smaller reduction in between leaves nothing behind for the next call
    small = mc.reduce_noalloc(phi, cnt, 17, n_bins=32)
    assert small["n_traj"] == 17
    assert small["phi_mean"] == pytest.approx(float(phi[:17].mean()), rel=1e-13)
    _same(mc.reduce_noalloc(phi, cnt, n, n_bins=32), ref)
    h.close()


def test_reduce_noalloc_rejects_sizes_beyond_its_scratch():
    import torch

    import ctypes as C

    phi = torch.zeros(4, dtype=torch.float64, device="cuda")
    cnt = torch.zeros((4, mc.N_COUNTERS), dtype=torch.int32, device="cuda")
    # the C entry point itself refuses n beyond its scratch, before any launch
    s = mc.McStats()
    st = mc.lib().mc_reduce_noalloc(C.c_void_p(phi.data_ptr()), C.c_void_p(cnt.data_ptr()),
                                    mc.MAX_NOALLOC_TRAJ + 1, 64, 0.0, 0.0, C.c_void_p(0),
                                    C.byref(s))
    assert st == mc.MC_EINVAL
    assert "262144" in mc.lib().mc_last_error(None).decode()
    with pytest.raises(mc.McError):
        mc.reduce_noalloc(phi, cnt, 4, n_bins=0)
    # the binding refuses arrays shorter than n
    with pytest.raises(ValueError):
        mc.reduce_noalloc(phi, cnt, 5)
