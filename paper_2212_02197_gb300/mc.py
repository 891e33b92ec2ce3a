"""Python binding of the C ABI in include/mc.h (argument marshalling only).

Every step of the closed-loop path runs in the CUDA library
``libmc_gb300.so``; this module converts plain-data configurations
(``workloads`` dicts) into the C structs, passes CUDA streams and pointers, and
returns numpy arrays.  There is no CPU fallback: if the library has not been
built, or no GPU is visible, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import _build

MAX_SETPOINTS = 16
MAX_HORIZON = 64
MAX_BINS = 256
N_COUNTERS = 8
COUNTER_NAMES = ["n_ocp_failed", "sqp_iters", "ls_trials", "n_hess_reset", "n_ls_fail",
                 "qp_iters", "nonfinite", "qp_fail"]

MC_OK, MC_EINVAL, MC_ENOMEM, MC_ECUDA, MC_ETIMEOUT, MC_ENOTRUN = 0, 1, 2, 3, 4, 5
MC_WARN_NONFINITE = 100
QP_SOLVERS = {"active_set": 0, "ipm": 1, "active_set_warp": 2}
PRECISIONS = {"fp64": 0, "mixed": 1}
KINDS = {"nmpc": 0, "pi": 1}
SCHEDULES = {"static": 0, "persistent": 1}

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)


class McModel(C.Structure):
    _fields_ = [("V", C.c_double), ("k0", C.c_double), ("EaR", C.c_double),
                ("beta", C.c_double), ("cA_in", C.c_double), ("cB_in", C.c_double),
                ("T_in", C.c_double), ("sigma", C.c_double * 3), ("meas_sd", C.c_double),
                ("Ts", C.c_double), ("t0", C.c_double), ("n_steps", C.c_int32),
                ("n_em", C.c_int32), ("n_setpoints", C.c_int32), ("Ea_plant_only", C.c_int32),
                ("sp_time", _dp), ("sp_value", _dp), ("Ea_logsd", C.c_double),
                ("dT_in_step", C.c_double)]


class McController(C.Structure):
    _fields_ = [("kind", C.c_int32), ("precision", C.c_int32), ("u_min", C.c_double),
                ("u_max", C.c_double), ("kP", C.c_double), ("kI", C.c_double),
                ("kaw", C.c_double), ("N", C.c_int32), ("n_rk4", C.c_int32),
                ("Qz", C.c_double), ("P0", C.c_double), ("sqp_max_it", C.c_int32),
                ("ls_max", C.c_int32), ("sqp_tol", C.c_double), ("qp_solver", C.c_int32),
                ("ip_max_it", C.c_int32), ("ip_tol", C.c_double), ("u_scale", C.c_double),
                ("x_scale", C.c_double), ("N_min", C.c_int32), ("sqp_max_it_min", C.c_int32),
                ("schedule", C.c_int32), ("threads_per_sm", C.c_int32),
                ("nx_model", C.c_int32), ("Ru", C.c_double), ("Qn", C.c_double),
                ("ls_spec_lanes", C.c_int32)]


class McStats(C.Structure):
    _fields_ = [("n_traj", C.c_int64), ("n_ocp", C.c_int64), ("n_ocp_failed", C.c_int64),
                ("n_ls_fail", C.c_int64), ("n_hess_reset", C.c_int64),
                ("n_nonfinite", C.c_int64), ("sqp_iters", C.c_int64), ("ls_trials", C.c_int64),
                ("qp_iters", C.c_int64), ("qp_fail", C.c_int64), ("phi_mean", C.c_double),
                ("phi_var", C.c_double), ("phi_min", C.c_double), ("phi_max", C.c_double),
                ("n_bins", C.c_int32), ("reserved0", C.c_int32), ("bin_lo", C.c_double),
                ("bin_hi", C.c_double), ("hist", C.c_int64 * MAX_BINS), ("gpu_ms", C.c_double)]


class McError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


_lib = None
_lock = threading.Lock()


def lib():
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_build.LIB):
                raise RuntimeError(f"CUDA library {_build.LIB} is missing: build it with "
                                   "__graft_entry__.build() (there is no CPU fallback)")
            L = C.CDLL(_build.LIB)
            H = C.c_void_p
            L.mc_create.argtypes = [C.POINTER(McModel), C.POINTER(McController), C.c_int64,
                                    C.c_uint64, C.POINTER(H)]
            L.mc_set_histogram.argtypes = [H, C.c_int32, C.c_double, C.c_double]
            L.mc_run.argtypes = [H, C.c_void_p]
            L.mc_run_range.argtypes = [H, C.c_int64, C.c_int64, C.c_void_p]
            L.mc_stats.argtypes = [H, C.POINTER(McStats), C.c_int64]
            L.mc_copy_phi.argtypes = [H, C.c_int64, C.c_int64, C.c_void_p, C.c_int]
            L.mc_copy_counters.argtypes = [H, C.c_int64, C.c_int64, C.c_void_p, C.c_int]
            L.mc_sync.argtypes = [H, C.c_int64]
            L.mc_destroy.argtypes = [H]
            L.mc_destroy.restype = None
            L.mc_status_str.argtypes = [C.c_int]
            L.mc_status_str.restype = C.c_char_p
            L.mc_last_error.argtypes = [H]
            L.mc_last_error.restype = C.c_char_p
            u32p = C.POINTER(C.c_uint32)
            L.mc_philox.argtypes = [u32p, u32p, C.c_int64, u32p]
            L.mc_noise.argtypes = [C.c_uint64, C.c_int64, C.c_int64, C.c_int64, C.c_int32,
                                   _dp, _dp]
            L.mc_qp_solve_batch.argtypes = ([C.c_int32, C.c_int64, C.c_int32, C.c_int32,
                                             C.c_double] + [_dp] * 15 + [_ip, _ip])
            L.mc_ocp_solve_batch.argtypes = ([C.POINTER(McModel), C.POINTER(McController),
                                              C.c_int64] + [_dp] * 8 + [_ip, _dp])
            L.mc_reduce_noalloc.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32,
                                            C.c_double, C.c_double, C.c_void_p,
                                            C.POINTER(McStats)]
            L.mc_set_graph.argtypes = [H, C.c_int]
            L.mc_autotune.argtypes = [H, C.c_int32, C.c_void_p, C.POINTER(C.c_int32)]
            L.mc_set_sm_partition.argtypes = [H, C.c_int32, C.POINTER(C.c_int32)]
            L.mc_set_sm_partition.restype = C.c_int
            L.mc_set_nmpc_weights.argtypes = [H, C.c_double, C.c_double, C.c_double]
            L.mc_set_nmpc_weights.restype = C.c_int
            L.mc_nmpc_grad.argtypes = [H, C.c_int64, C.c_int64, C.c_void_p]
            L.mc_nmpc_grad.restype = C.c_int
            L.mc_ocp_sens_batch.argtypes = ([C.POINTER(McModel), C.POINTER(McController),
                                              C.c_int64] + [_dp] * 9 + [_ip])
            L.mc_ocp_sens_batch.restype = C.c_int
            L.mc_copy_warp_trace.argtypes = [H, C.POINTER(C.c_uint64), C.c_int64,
                                             C.POINTER(C.c_int64)]
            L.mc_copy_warp_trace.restype = C.c_int
            L.mc_set_grad_record_budget.argtypes = [H, C.c_int64]
            L.mc_set_grad_record_budget.restype = C.c_int
            for f in ("mc_exp_batch", "mc_rcp_batch"):
                getattr(L, f).argtypes = [_dp, C.c_int64, _dp]
                getattr(L, f).restype = C.c_int
            L.mc_pipe_probe.argtypes = [C.c_int32, C.c_int64, _dp, _dp]
            L.mc_pipe_probe.restype = C.c_int
            L.mc_set_pi_gains.argtypes = [H, C.c_double, C.c_double, C.c_double]
            L.mc_pi_grad.argtypes = [H, C.c_int64, C.c_int64, C.c_int32, C.c_void_p]
            L.mc_grad_mean.argtypes = [H, _dp, C.c_int64]
            L.mc_copy_grad.argtypes = [H, C.c_int64, C.c_int64, C.c_void_p, C.c_int]
            for f in ("mc_set_graph", "mc_autotune", "mc_set_pi_gains", "mc_pi_grad",
                      "mc_grad_mean", "mc_copy_grad"):
                getattr(L, f).restype = C.c_int
            for f in ("mc_create", "mc_set_histogram", "mc_run", "mc_run_range", "mc_stats",
                      "mc_copy_phi", "mc_copy_counters", "mc_sync", "mc_philox", "mc_noise",
                      "mc_qp_solve_batch", "mc_ocp_solve_batch", "mc_reduce_noalloc"):
                getattr(L, f).restype = C.c_int
            _lib = L
    return _lib


WARP_TRACE_WORDS = 5   # MC_WARP_TRACE_WORDS


def _check(status, handle=None, ok=(MC_OK,)):
    if status in ok:
        return status
    L = lib()
    msg = L.mc_last_error(handle).decode() or L.mc_status_str(status).decode()
    raise McError(status, msg)


def _p(a):
    return a.ctypes.data_as(_dp)


def make_model(md: dict):
    """(McModel, keep-alive arrays) from a workloads model dict."""
    sp_t = np.ascontiguousarray(md["sp_time"], dtype=np.float64)
    sp_v = np.ascontiguousarray(md["sp_value"], dtype=np.float64)
    m = McModel()
    for k in ("V", "k0", "EaR", "beta", "cA_in", "cB_in", "T_in", "meas_sd", "Ts", "t0",
              "Ea_logsd"):
        setattr(m, k, float(md[k]))
    m.dT_in_step = float(md["dTin_step"])
    for i in range(3):
        m.sigma[i] = float(md["sigma"][i])
    m.n_steps, m.n_em = int(md["n_steps"]), int(md["n_em"])
    m.n_setpoints = len(sp_t)
    m.Ea_plant_only = 1 if md.get("Ea_plant_only", False) else 0
    m.sp_time, m.sp_value = _p(sp_t), _p(sp_v)
    return m, (sp_t, sp_v)


def make_ctrl(cd: dict) -> McController:
    c = McController()
    c.kind = KINDS[cd["kind"]]
    c.precision = PRECISIONS[cd.get("precision", "fp64")]
    for k in ("u_min", "u_max", "kP", "kI", "kaw", "Qz", "P0", "sqp_tol", "u_scale", "x_scale"):
        setattr(c, k, float(cd[k]))
    for k in ("N", "n_rk4", "sqp_max_it"):
        setattr(c, k, int(cd[k]))
    c.ls_max = int(cd["ls_max"])
    c.qp_solver = QP_SOLVERS[cd.get("qp_solver", "active_set")]
    c.ip_max_it = int(cd.get("ip_max_it", 60))
    c.ip_tol = float(cd.get("ip_tol", 1e-14))
    c.N_min = int(cd.get("N_min", 0))
    c.sqp_max_it_min = int(cd.get("sqp_max_it_min", 0))
    c.schedule = SCHEDULES[cd.get("schedule", "static")]
    c.threads_per_sm = int(cd.get("threads_per_sm", 0))
    c.ls_spec_lanes = int(cd.get("ls_spec_lanes", 0))
    c.nx_model = int(cd.get("nx_model", 1))
    c.Ru = float(cd.get("Ru", 0.0))
    c.Qn = float(cd.get("Qn", 0.0))
    return c


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return C.c_void_p(0)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


class MonteCarlo:
    """A handle of the C ABI: n_sims trajectories of one controller."""

    def __init__(self, model: dict, ctrl: dict, n_sims: int, seed: int):
        L = lib()
        self._m, self._keep = make_model(model)
        self._c = make_ctrl(ctrl)
        self.n_sims = int(n_sims)
        self.sqp_tol = float(ctrl["sqp_tol"]) if ctrl.get("kind") == "nmpc" else None
        self._h = C.c_void_p()
        _check(L.mc_create(C.byref(self._m), C.byref(self._c), self.n_sims, int(seed),
                           C.byref(self._h)))

    def close(self):
        if getattr(self, "_h", None):
            lib().mc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_histogram(self, n_bins: int, lo: float = 0.0, hi: float = 0.0):
        _check(lib().mc_set_histogram(self._h, n_bins, lo, hi), self._h)

    def set_graph(self, on: bool = True):
        """Replay each range's launches from a captured CUDA graph."""
        _check(lib().mc_set_graph(self._h, 1 if on else 0), self._h)

    def set_sm_partition(self, n_sms: int) -> int:
        """Run on a partition of at least n_sms SMs (0: the whole GPU); returns
        the SM count actually used."""
        got = C.c_int32()
        _check(lib().mc_set_sm_partition(self._h, int(n_sms), C.byref(got)), self._h)
        return got.value

    def autotune(self, probe_steps: int = 8, stream=None) -> int:
        """Resident threads per SM of the persistent schedule, chosen by timing."""
        tps = C.c_int32()
        _check(lib().mc_autotune(self._h, probe_steps, _stream_ptr(stream), C.byref(tps)),
               self._h)
        return tps.value

    def run(self, stream=None, j0: int = 0, j1: int | None = None):
        j1 = self.n_sims if j1 is None else j1
        _check(lib().mc_run_range(self._h, j0, j1, _stream_ptr(stream)), self._h)

    def sync(self, timeout_ms: int = 0):
        _check(lib().mc_sync(self._h, timeout_ms), self._h)

    def stats(self, timeout_ms: int = 0) -> dict:
        s = McStats()
        st = _check(lib().mc_stats(self._h, C.byref(s), timeout_ms), self._h,
                    ok=(MC_OK, MC_WARN_NONFINITE))
        d = {f: getattr(s, f) for f, _ in McStats._fields_ if f not in ("hist", "reserved0")}
        d["hist"] = np.array(s.hist[: s.n_bins], dtype=np.int64)
        d["status"] = st
        return d

    def phi(self, j0: int = 0, n: int | None = None, out=None):
        """Phi of trajectories j0..j0+n-1: a numpy array, or into `out` (a CUDA
        torch tensor of float64, copied device to device)."""
        n = self.n_sims - j0 if n is None else n
        if out is not None:
            _check(lib().mc_copy_phi(self._h, j0, n, C.c_void_p(out.data_ptr()), 1), self._h)
            return out
        a = np.empty(n, dtype=np.float64)
        _check(lib().mc_copy_phi(self._h, j0, n, a.ctypes.data_as(C.c_void_p), 0), self._h)
        return a

    def counters_to(self, out, j0: int = 0, n: int | None = None):
        """Per-trajectory counters copied device to device into `out` (a CUDA
        torch tensor of n x N_COUNTERS int32)."""
        n = self.n_sims - j0 if n is None else n
        _check(lib().mc_copy_counters(self._h, j0, n, C.c_void_p(out.data_ptr()), 1), self._h)
        return out

    def counters(self, j0: int = 0, n: int | None = None) -> dict:
        n = self.n_sims - j0 if n is None else n
        a = np.empty((n, N_COUNTERS), dtype=np.int32)
        _check(lib().mc_copy_counters(self._h, j0, n, a.ctypes.data_as(C.c_void_p), 0), self._h)
        return {k: a[:, i].copy() for i, k in enumerate(COUNTER_NAMES)}

    def warp_trace(self) -> dict:
        """Per-warp record of the last one-state persistent NMPC launch
        (mc_copy_warp_trace): pool rounds, lane-rounds, start and end on the
        GPU's global timer (ns), and the SM, one entry per warp."""
        nw = C.c_int64()
        _check(lib().mc_copy_warp_trace(self._h, None, 0, C.byref(nw)), self._h)
        a = np.zeros((max(nw.value, 1), WARP_TRACE_WORDS), dtype=np.uint64)
        _check(lib().mc_copy_warp_trace(self._h, a.ctypes.data_as(C.POINTER(C.c_uint64)),
                                        nw.value, C.byref(nw)), self._h)
        a = a[:nw.value]
        return {"rounds": a[:, 0].astype(np.int64), "lane_rounds": a[:, 1].astype(np.int64),
                "t_start_ns": a[:, 2].astype(np.int64), "t_end_ns": a[:, 3].astype(np.int64),
                "sm": a[:, 4].astype(np.int64)}

    # -- gradients of the PI study

    def set_pi_gains(self, kP: float, kI: float, kaw: float):
        _check(lib().mc_set_pi_gains(self._h, float(kP), float(kI), float(kaw)), self._h)

    def pi_grad(self, checkpoint_every: int = 20, stream=None, j0: int = 0,
                j1: int | None = None):
        """Forward and adjoint sweeps of trajectories j0..j1-1 (asynchronous)."""
        j1 = self.n_sims if j1 is None else j1
        _check(lib().mc_pi_grad(self._h, j0, j1, int(checkpoint_every), _stream_ptr(stream)),
               self._h)

    def set_nmpc_weights(self, Qz: float, Ru: float, Qn: float):
        _check(lib().mc_set_nmpc_weights(self._h, float(Qz), float(Ru), float(Qn)), self._h)

    def set_grad_record_budget(self, nbytes: int):
        """Device memory the persistent gradient's sample records may take (0: 8 GB)."""
        _check(lib().mc_set_grad_record_budget(self._h, int(nbytes)), self._h)

    def nmpc_grad(self, stream=None, j0: int = 0, j1: int | None = None):
        """Closed loop with the tangents of Phi in (Q_z, R_u, Q_n) (asynchronous)."""
        j1 = self.n_sims if j1 is None else j1
        _check(lib().mc_nmpc_grad(self._h, j0, j1, _stream_ptr(stream)), self._h)

    def grad_mean(self, timeout_ms: int = 0) -> np.ndarray:
        """Mean dPhi/d(k_P, k_I, k_aw) over the finite trajectories of the last pi_grad."""
        g = np.zeros(3)
        _check(lib().mc_grad_mean(self._h, _p(g), timeout_ms), self._h,
               ok=(MC_OK, MC_WARN_NONFINITE))
        return g

    def grad(self, j0: int = 0, n: int | None = None, out=None):
        """Per-trajectory dPhi_j/d(k_P, k_I, k_aw), n x 3: a numpy array, or into
        `out` (a CUDA torch tensor of float64, copied device to device)."""
        n = self.n_sims - j0 if n is None else n
        if out is not None:
            _check(lib().mc_copy_grad(self._h, j0, n, C.c_void_p(out.data_ptr()), 1), self._h)
            return out
        a = np.empty((n, 3), dtype=np.float64)
        _check(lib().mc_copy_grad(self._h, j0, n, a.ctypes.data_as(C.c_void_p), 0), self._h)
        return a


# ------------------------------------------------------------------ building blocks

def ocp_sens_batch(model: dict, ctrl: dict, x0, EaR, zbar, u, x, lam, pil, piu):
    """du_0/d(x_0, Q_z, R_u, Q_n) at given OCP solutions; returns (sens n x 4, status)."""
    L = lib()
    m, keep = make_model(model)
    c = make_ctrl(ctrl)
    u = np.ascontiguousarray(u, dtype=np.float64)
    n = u.shape[0]
    arrs = [np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.float64), shp))
            for a, shp in ((x0, (n,)), (EaR, (n,)), (zbar, (n, c.N + 1)), (u, (n, c.N)),
                           (x, (n, c.N + 1)), (lam, (n, c.N)), (pil, (n, c.N)), (piu, (n, c.N)))]
    sens = np.zeros((n, 4))
    st = np.zeros(n, dtype=np.int32)
    _check(L.mc_ocp_sens_batch(C.byref(m), C.byref(c), n, *[_p(a) for a in arrs], _p(sens),
                               st.ctypes.data_as(_ip)))
    return sens, st


def exp_batch(x):
    """The device FP64 exponential of the rate law, elementwise on x."""
    x = np.ascontiguousarray(x, dtype=np.float64).ravel()
    y = np.empty_like(x)
    _check(lib().mc_exp_batch(_p(x), len(x), _p(y)))
    return y


def rcp_batch(x):
    """The device FP64 reciprocal of the one-state rate law, elementwise on x."""
    x = np.ascontiguousarray(x, dtype=np.float64).ravel()
    y = np.empty_like(x)
    _check(lib().mc_rcp_batch(_p(x), len(x), _p(y)))
    return y


def pipe_probe(kind: int, iters: int):
    """(device ms, chain steps) of one throughput-probe launch (mc_pipe_probe)."""
    ms, steps = C.c_double(), C.c_double()
    _check(lib().mc_pipe_probe(int(kind), int(iters), C.byref(ms), C.byref(steps)))
    return ms.value, steps.value


def philox(ctr, key):
    """Device Philox4x32-10 of counters ctr (n x 4 uint32) under key (2 words)."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    out = np.empty_like(ctr)
    k = (C.c_uint32 * 2)(*[int(v) for v in key])
    u32p = C.POINTER(C.c_uint32)
    _check(lib().mc_philox(ctr.ctypes.data_as(u32p), k, len(ctr), out.ctypes.data_as(u32p)))
    return out


def noise(seed: int, j: int, k0: int, nk: int, precision: str = "fp64"):
    """(process noise nk x 3, measurement noise nk) of trajectory j as drawn on the GPU."""
    out = np.empty((nk, 3))
    meas = np.empty(nk)
    _check(lib().mc_noise(seed, j, k0, nk, PRECISIONS[precision], _p(out), _p(meas)))
    return out, meas


def qp_solve_batch(A, B, b, Wxx, Wxu, Wuu, q, r, lb, ub, solver="active_set", max_it=None,
                   tol=1e-14):
    """Solve a batch of structured QPs on the GPU; arrays are (n, N) or (n, N+1)."""
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (A, B, b, Wxx, Wxu, Wuu, q, r,
                                                                 lb, ub)]
    n, N = arrs[1].shape
    if max_it is None:
        max_it = 10 * N + 20 if solver in ("active_set", "active_set_warp") else 60
    du, mu, nul, nuu = (np.empty((n, N)) for _ in range(4))
    dx = np.empty((n, N + 1))
    it = np.empty(n, dtype=np.int32)
    st = np.empty(n, dtype=np.int32)
    _check(lib().mc_qp_solve_batch(N, n, QP_SOLVERS[solver], max_it, tol, *[_p(a) for a in arrs],
                                   _p(du), _p(dx), _p(mu), _p(nul), _p(nuu),
                                   it.ctypes.data_as(_ip), st.ctypes.data_as(_ip)))
    return dict(du=du, dx=dx, mu=mu, nul=nul, nuu=nuu, iters=it, status=st)


def ocp_solve_batch(model: dict, ctrl: dict, x0, EaR, zbar, u, x, lam=None, pil=None, piu=None):
    """Solve a batch of NMPC OCPs by the GPU SQP from warm starts; returns the
    updated (u, x, lam, pil, piu) and per-OCP info/kkt arrays."""
    m, keep = make_model(model)
    c = make_ctrl(ctrl)
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    n, N = len(x0), c.N
    EaR = np.ascontiguousarray(np.broadcast_to(EaR, (n,)), dtype=np.float64)
    zbar = np.ascontiguousarray(zbar, dtype=np.float64).reshape(n, N + 1)
    u = np.array(u, dtype=np.float64).reshape(n, N)
    x = np.array(x, dtype=np.float64).reshape(n, N + 1)
    lam = np.zeros((n, N)) if lam is None else np.array(lam, dtype=np.float64).reshape(n, N)
    pil = np.zeros((n, N)) if pil is None else np.array(pil, dtype=np.float64).reshape(n, N)
    piu = np.zeros((n, N)) if piu is None else np.array(piu, dtype=np.float64).reshape(n, N)
    info = np.empty((n, 4), dtype=np.int32)
    kkt = np.empty((n, 3))
    _check(lib().mc_ocp_solve_batch(C.byref(m), C.byref(c), n, _p(x0), _p(EaR), _p(zbar), _p(u),
                                    _p(x), _p(lam), _p(pil), _p(piu), info.ctypes.data_as(_ip),
                                    _p(kkt)))
    del keep
    return dict(u=u, x=x, lam=lam, pil=pil, piu=piu, iters=info[:, 0], status=info[:, 1],
                ls_trials=info[:, 2], qp_iters=info[:, 3], kkt_grad=kkt[:, 0], kkt_eq=kkt[:, 1],
                f=kkt[:, 2])


MAX_NOALLOC_TRAJ = 262144


def _stats_dict(s: McStats, st: int) -> dict:
    d = {f: getattr(s, f) for f, _ in McStats._fields_ if f not in ("hist", "reserved0")}
    d["hist"] = np.array(s.hist[: s.n_bins], dtype=np.int64)
    d["status"] = st
    return d


def _check_device_array(t, name: str, dtype_name: str, n: int, cols: int | None):
    """Reject anything the reduction's kernels could read past: the tensor must
    be a contiguous CUDA tensor of the right dtype on the current device with
    at least n rows (of `cols` columns)."""
    import torch

    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name} must be a CUDA torch tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (got device {t.device})")
    if t.dtype != getattr(torch, dtype_name):
        raise ValueError(f"{name} must be {dtype_name} (got {t.dtype})")
    if t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name} is on cuda:{t.device.index}, not on the current device "
                         f"cuda:{torch.cuda.current_device()}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if cols is None:
        if t.numel() < n:
            raise ValueError(f"{name} holds {t.numel()} values, fewer than n = {n}")
    elif t.dim() != 2 or t.shape[1] != cols or t.shape[0] < n:
        raise ValueError(f"{name} must have shape (>= {n}, {cols}), not {tuple(t.shape)}")


def reduce_noalloc(phi_dev, counters_dev, n: int, n_bins: int = 64, lo: float = 0.0,
                   hi: float = 0.0, stream=None) -> dict:
    """Statistics of per-trajectory results already on the device (CUDA torch
    tensors on the current device: n float64 and n x N_COUNTERS int32),
    reduced without any device allocation (see mc_reduce_noalloc in
    include/mc.h).  Tensors of the wrong kind, device or size raise ValueError
    before anything is launched."""
    n = int(n)
    if n < 0:
        raise ValueError("n must be >= 0")
    _check_device_array(phi_dev, "phi_dev", "float64", n, None)
    _check_device_array(counters_dev, "counters_dev", "int32", n, N_COUNTERS)
    s = McStats()
    st = _check(lib().mc_reduce_noalloc(C.c_void_p(phi_dev.data_ptr()),
                                        C.c_void_p(counters_dev.data_ptr()), n, n_bins, lo, hi,
                                        _stream_ptr(stream), C.byref(s)),
                ok=(MC_OK, MC_WARN_NONFINITE))
    return _stats_dict(s, st)
