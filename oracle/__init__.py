"""Plain FP64 CPU oracle for the Monte Carlo closed-loop NMPC/PI study
(Kaysfeld, Zanon, Joergensen, arXiv 2212.02197).

TEST INFRASTRUCTURE ONLY.  The test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only users.  It shares no code with the
CUDA path; configurations reach it as plain data (dicts from
``paper_2212_02197_gb300.workloads``).

The C sources in this directory follow the paper section by section (see
``oracle.h``); this module only builds them with gcc and marshals arguments.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = ["or_random.c", "or_model.c", "or_sqp.c", "or_closedloop.c", "or_grad.c",
        "or_nmpc3.c"]
MAX_SP = 16
MAX_N = 64


def compile_sources(src_dir: str, out: str) -> str:
    """Compile the oracle's C sources found in ``src_dir`` into the shared
    library ``out`` (the flags of ``build``)."""
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared",
           "-Wall", "-Wno-unused-function", "-o", tmp]
    cmd += [os.path.join(src_dir, s) for s in _SRC] + ["-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` with gcc.

    FP contraction is disabled so that x86-64 and aarch64 builds round alike.
    """
    srcs = [os.path.join(_HERE, s) for s in _SRC] + [os.path.join(_HERE, "oracle.h")]
    if not force and os.path.exists(_SO):
        so_t = os.path.getmtime(_SO)
        if all(os.path.getmtime(s) <= so_t for s in srcs):
            return _SO
    return compile_sources(_HERE, _SO)


def sources() -> list[str]:
    """Paths of the oracle's C sources and header."""
    return [os.path.join(_HERE, s) for s in _SRC] + [os.path.join(_HERE, "oracle.h")]


class Model(C.Structure):
    _fields_ = [("V", C.c_double), ("k0", C.c_double), ("EaR", C.c_double),
                ("beta", C.c_double), ("cA_in", C.c_double), ("cB_in", C.c_double),
                ("T_in", C.c_double), ("sigma", C.c_double * 3), ("meas_sd", C.c_double),
                ("Ts", C.c_double), ("t0", C.c_double), ("n_steps", C.c_int32),
                ("n_em", C.c_int32), ("n_sp", C.c_int32), ("Ea_plant_only", C.c_int32),
                ("sp_time", C.c_double * MAX_SP), ("sp_value", C.c_double * MAX_SP),
                ("Ea_logsd", C.c_double), ("dTin_step", C.c_double)]


class Ctrl(C.Structure):
    _fields_ = [("kind", C.c_int32), ("N", C.c_int32), ("n_rk4", C.c_int32),
                ("sqp_max_it", C.c_int32), ("ls_max", C.c_int32), ("nx_model", C.c_int32),
                ("u_min", C.c_double), ("u_max", C.c_double), ("kP", C.c_double),
                ("kI", C.c_double), ("kaw", C.c_double), ("Qz", C.c_double),
                ("P0", C.c_double), ("sqp_tol", C.c_double), ("u_scale", C.c_double),
                ("x_scale", C.c_double), ("N_min", C.c_int32), ("it_min", C.c_int32),
                ("Ru", C.c_double), ("Qn", C.c_double)]


class TrajOut(C.Structure):
    _fields_ = [("phi", C.c_double), ("n_ocp", C.c_int32), ("n_ocp_failed", C.c_int32),
                ("sqp_iters", C.c_int32), ("ls_trials", C.c_int32),
                ("n_hess_reset", C.c_int32), ("n_ls_fail", C.c_int32),
                ("qp_iters", C.c_int32), ("nonfinite", C.c_int32)]


class SqpInfo(C.Structure):
    _fields_ = [("iters", C.c_int32), ("status", C.c_int32), ("ls_trials", C.c_int32),
                ("n_hess_reset", C.c_int32), ("qp_iters", C.c_int32), ("pad0", C.c_int32),
                ("kkt_grad", C.c_double), ("kkt_eq", C.c_double), ("f", C.c_double)]


TRACE_MAX_TRIALS = 64


class SqpTraceRow(C.Structure):
    _fields_ = [("l", C.c_int32), ("reset", C.c_int32), ("n_trials", C.c_int32),
                ("accepted", C.c_int32), ("stop", C.c_int32), ("pad0", C.c_int32),
                ("s_d", C.c_double), ("kkt_grad_raw", C.c_double), ("kkt_grad", C.c_double),
                ("kkt_eq", C.c_double), ("f", C.c_double), ("T0", C.c_double),
                ("DT0", C.c_double), ("lam", C.c_double * MAX_N), ("pil", C.c_double * MAX_N),
                ("piu", C.c_double * MAX_N), ("g", C.c_double * MAX_N),
                ("q", C.c_double * (MAX_N + 1)), ("r", C.c_double * MAX_N),
                ("A", C.c_double * MAX_N), ("B", C.c_double * MAX_N),
                ("du", C.c_double * MAX_N), ("dx", C.c_double * (MAX_N + 1)),
                ("mu", C.c_double * MAX_N), ("sigma", C.c_double * MAX_N),
                ("alpha", C.c_double * TRACE_MAX_TRIALS),
                ("f_trial", C.c_double * TRACE_MAX_TRIALS),
                ("pen_trial", C.c_double * TRACE_MAX_TRIALS)]


_lib = None
_lock = threading.Lock()
_dp = C.POINTER(C.c_double)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # MC_ORACLE_LIB: a library built from altered sources, for the
            # tests that check the pins fail on planted mistakes
            path = os.environ.get("MC_ORACLE_LIB")
            if not path:
                build()
                path = _SO
            L = C.CDLL(path)
            u32p = C.POINTER(C.c_uint32)
            L.or_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.or_uniform52.argtypes = [C.c_uint32, C.c_uint32]
            L.or_uniform52.restype = C.c_double
            L.or_normal_pair.argtypes = [u32p, _dp]
            L.or_process_noise.argtypes = [C.c_uint64, C.c_int64, C.c_int64, _dp]
            L.or_meas_noise.argtypes = [C.c_uint64, C.c_int64, C.c_int64]
            L.or_meas_noise.restype = C.c_double
            L.or_traj_params.argtypes = [C.POINTER(Model), C.c_uint64, C.c_int64, _dp, _dp, _dp]
            L.or_plant_drift.argtypes = [C.POINTER(Model), C.c_double, C.c_double, _dp,
                                         C.c_double, _dp]
            L.or_model1.argtypes = [C.POINTER(Model), C.c_double, C.c_double, C.c_double,
                                    _dp, _dp, _dp]
            L.or_zbar.argtypes = [C.POINTER(Model), C.c_double]
            L.or_zbar.restype = C.c_double
            L.or_Fss.argtypes = [C.POINTER(Model), C.c_double, C.c_double]
            L.or_Fss.restype = C.c_double
            L.or_em_step.argtypes = [C.POINTER(Model), C.c_double, C.c_double, _dp,
                                     C.c_double, C.c_double, _dp]
            L.or_rk4_interval.argtypes = [C.POINTER(Model), C.c_double, C.c_int, C.c_double,
                                          C.c_double, C.c_double, C.c_double, _dp, _dp, _dp]
            L.or_ekf_predict.argtypes = [C.POINTER(Model), C.c_double, C.c_int, C.c_double,
                                         _dp, _dp]
            L.or_ekf_filter.argtypes = [C.POINTER(Model), C.c_double, _dp, _dp, _dp]
            L.or_qp_solve.argtypes = [C.c_int] + [_dp] * 15 + [C.POINTER(C.c_int)]
            L.or_qp_solve.restype = C.c_int
            L.or_sqp.argtypes = [C.POINTER(Model), C.POINTER(Ctrl), C.c_double, C.c_double,
                                 _dp, _dp, _dp, _dp, _dp, _dp, C.POINTER(SqpInfo)]
            L.or_sqp.restype = C.c_int
            L.or_sqp_traced.argtypes = ([C.POINTER(Model), C.POINTER(Ctrl), C.c_double,
                                         C.c_double] + [_dp] * 6 +
                                        [C.POINTER(SqpInfo), C.POINTER(SqpTraceRow), C.c_int,
                                         C.POINTER(C.c_int)])
            L.or_sqp_traced.restype = C.c_int
            L.or_bfgs_update_blocks.argtypes = [C.c_int] + [_dp] * 5
            L.or_bfgs_update_blocks.restype = C.c_int
            L.or_bfgs_block.argtypes = [C.c_int, _dp, _dp, _dp]
            L.or_traj_horizon.argtypes = [C.POINTER(Ctrl), C.c_uint64, C.c_int64,
                                          C.POINTER(C.c_int), C.POINTER(C.c_int)]
            L.or_pi_step.argtypes = [C.POINTER(Ctrl), C.c_double, C.c_double, C.c_double,
                                     C.c_double, _dp]
            L.or_pi_step.restype = C.c_double
            L.or_traj.argtypes = [C.POINTER(Model), C.POINTER(Ctrl), C.c_uint64, C.c_int64,
                                  C.POINTER(TrajOut), _dp]
            L.or_run.argtypes = [C.POINTER(Model), C.POINTER(Ctrl), C.c_uint64, C.c_int64,
                                 C.c_int64, C.c_int, C.POINTER(TrajOut)]
            L.or_drift3.argtypes = [C.POINTER(Model), C.c_double, C.c_double, _dp, C.c_double,
                                    _dp, _dp, _dp]
            L.or_rk4_interval3.argtypes = [C.POINTER(Model), C.c_double, C.c_int, C.c_double,
                                           _dp, C.c_double, C.c_double, _dp, _dp, _dp]
            L.or_ekf3_predict.argtypes = [C.POINTER(Model), C.c_double, C.c_int, C.c_double,
                                          _dp, _dp]
            L.or_ekf3_filter.argtypes = [C.POINTER(Model), C.c_double, _dp, _dp, _dp]
            L.or_qp3_solve.argtypes = [C.c_int] + [_dp] * 15 + [C.POINTER(C.c_int)]
            L.or_qp3_solve.restype = C.c_int
            L.or_bfgs_blockn.argtypes = [C.c_int, _dp, _dp, _dp]
            L.or_sqp3.argtypes = [C.POINTER(Model), C.POINTER(Ctrl), C.c_double, _dp, _dp, _dp,
                                  _dp, _dp, _dp, _dp, C.POINTER(SqpInfo)]
            L.or_sqp3.restype = C.c_int
            L.or_ocp_sens.argtypes = [C.POINTER(Model), C.POINTER(Ctrl), C.c_double, C.c_double,
                                      _dp, _dp, _dp, _dp, _dp, _dp, _dp]
            L.or_ocp_sens.restype = C.c_int
            L.or_nmpc_grad_run.argtypes = [C.POINTER(Model), C.POINTER(Ctrl), C.c_uint64,
                                           C.c_int64, C.c_int64, C.c_int, _dp, _dp,
                                           C.POINTER(C.c_int)]
            L.or_pi_phi_cs.argtypes = [C.POINTER(Model), C.POINTER(Ctrl), C.c_uint64,
                                       C.c_int64, C.c_int, C.c_double, _dp]
            L.or_pi_phi_cs.restype = C.c_double
            L.or_pi_grad_run.argtypes = [C.POINTER(Model), C.POINTER(Ctrl), C.c_uint64,
                                         C.c_int64, C.c_int64, C.c_int, _dp, _dp]
            _lib = L
    return _lib


# ----------------------------------------------------------------------------
# marshalling of plain-data configurations


def make_model(md: dict) -> Model:
    m = Model()
    for k in ("V", "k0", "EaR", "beta", "cA_in", "cB_in", "T_in", "meas_sd", "Ts", "t0",
              "Ea_logsd", "dTin_step"):
        setattr(m, k, float(md[k]))
    for i in range(3):
        m.sigma[i] = float(md["sigma"][i])
    m.n_steps = int(md["n_steps"])
    m.n_em = int(md["n_em"])
    m.Ea_plant_only = 1 if md.get("Ea_plant_only", False) else 0
    sp_t, sp_v = md["sp_time"], md["sp_value"]
    assert len(sp_t) == len(sp_v) and 1 <= len(sp_t) <= MAX_SP
    m.n_sp = len(sp_t)
    for i, (t, v) in enumerate(zip(sp_t, sp_v)):
        m.sp_time[i] = float(t)
        m.sp_value[i] = float(v)
    return m


def make_ctrl(cd: dict) -> Ctrl:
    c = Ctrl()
    c.kind = {"nmpc": 0, "pi": 1}[cd["kind"]]
    for k in ("N", "n_rk4", "sqp_max_it", "ls_max"):
        setattr(c, k, int(cd[k]))
    for k in ("u_min", "u_max", "kP", "kI", "kaw", "Qz", "P0", "sqp_tol", "u_scale",
              "x_scale"):
        setattr(c, k, float(cd[k]))
    c.nx_model = int(cd.get("nx_model", 1))
    c.Ru = float(cd.get("Ru", 0.0))
    c.Qn = float(cd.get("Qn", 0.0))
    c.N_min = int(cd.get("N_min", 0))
    c.it_min = int(cd.get("sqp_max_it_min", 0))
    assert 1 <= c.N <= MAX_N
    return c


def _p(a):
    return a.ctypes.data_as(_dp)


TRAJ_FIELDS = ["phi", "n_ocp", "n_ocp_failed", "sqp_iters", "ls_trials", "n_hess_reset",
               "n_ls_fail", "qp_iters", "nonfinite"]


def run(model: dict, ctrl: dict, seed: int, j0: int, j1: int, threads: int | None = None):
    """Run trajectories j0..j1-1; returns a dict of numpy arrays (one entry per field)."""
    L = lib()
    m, c = make_model(model), make_ctrl(ctrl)
    n = j1 - j0
    out = (TrajOut * max(n, 1))()
    if threads is None:
        threads = os.cpu_count() or 1
    if n > 0:
        L.or_run(C.byref(m), C.byref(c), seed, j0, j1, int(threads), out)
    res = {}
    for f in TRAJ_FIELDS:
        res[f] = np.array([getattr(out[i], f) for i in range(n)])
    return res


def pi_grad(model: dict, ctrl: dict, seed: int, j0: int, j1: int, threads: int | None = None):
    """Phi_j and dPhi_j/d(k_P, k_I, k_aw) of PI trajectories j0..j1-1 by complex-step
    differentiation; returns (phi[n], dphi[n, 3])."""
    L = lib()
    m, c = make_model(model), make_ctrl(dict(ctrl, kind="pi"))
    n = j1 - j0
    phi = np.zeros(max(n, 1))
    dphi = np.zeros((max(n, 1), 3))
    if threads is None:
        threads = os.cpu_count() or 1
    if n > 0:
        L.or_pi_grad_run(C.byref(m), C.byref(c), seed, j0, j1, int(threads), _p(phi), _p(dphi))
    return phi[:n], dphi[:n]


def pi_phi_cs(model: dict, ctrl: dict, seed: int, j: int, which: int, h: float):
    """(Phi_j, Im Phi_j(k + i h) / h) for gain `which` (0 k_P, 1 k_I, 2 k_aw)."""
    L = lib()
    m, c = make_model(model), make_ctrl(dict(ctrl, kind="pi"))
    d = C.c_double()
    phi = L.or_pi_phi_cs(C.byref(m), C.byref(c), seed, j, which, h, C.byref(d))
    return phi, d.value


def traj(model: dict, ctrl: dict, seed: int, j: int, with_trace: bool = False):
    L = lib()
    m, c = make_model(model), make_ctrl(ctrl)
    out = TrajOut()
    tr = np.zeros((model["n_steps"], 5)) if with_trace else None
    L.or_traj(C.byref(m), C.byref(c), seed, j, C.byref(out), _p(tr) if with_trace else None)
    d = {f: getattr(out, f) for f in TRAJ_FIELDS}
    if with_trace:
        d["trace"] = tr
    return d


def sqp(model: dict, ctrl: dict, EaR: float, x0: float, zbar, u, x, lam=None, pil=None,
        piu=None):
    """One OCP.  zbar has N+1 entries (index 0 unused); u, x (N, N+1) are the
    warm start; returns (u, x, lam, pil, piu, info-dict)."""
    L = lib()
    m, c = make_model(model), make_ctrl(ctrl)
    N = c.N
    zb = np.ascontiguousarray(zbar, dtype=np.float64)
    u = np.array(u, dtype=np.float64)
    x = np.array(x, dtype=np.float64)
    lam = np.zeros(N) if lam is None else np.array(lam, dtype=np.float64)
    pil = np.zeros(N) if pil is None else np.array(pil, dtype=np.float64)
    piu = np.zeros(N) if piu is None else np.array(piu, dtype=np.float64)
    info = SqpInfo()
    L.or_sqp(C.byref(m), C.byref(c), EaR, x0, _p(zb), _p(u), _p(x), _p(lam), _p(pil),
             _p(piu), C.byref(info))
    d = {f: getattr(info, f) for f, _ in SqpInfo._fields_ if f != "pad0"}
    return u, x, lam, pil, piu, d


def sqp_traced(model: dict, ctrl: dict, EaR: float, x0: float, zbar, u, x, lam=None,
               pil=None, piu=None, max_rows: int = 256):
    """One OCP as ``sqp``, plus one trace row per SQP iteration: a list of dicts
    with the quantities each step of Sec. IV saw (arrays cut to N or N + 1)."""
    L = lib()
    m, c = make_model(model), make_ctrl(ctrl)
    N = c.N
    zb = np.ascontiguousarray(zbar, dtype=np.float64)
    u = np.array(u, dtype=np.float64)
    x = np.array(x, dtype=np.float64)
    lam = np.zeros(N) if lam is None else np.array(lam, dtype=np.float64)
    pil = np.zeros(N) if pil is None else np.array(pil, dtype=np.float64)
    piu = np.zeros(N) if piu is None else np.array(piu, dtype=np.float64)
    info = SqpInfo()
    rows = (SqpTraceRow * max_rows)()
    nr = C.c_int(0)
    L.or_sqp_traced(C.byref(m), C.byref(c), EaR, x0, _p(zb), _p(u), _p(x), _p(lam), _p(pil),
                    _p(piu), C.byref(info), rows, max_rows, C.byref(nr))
    d = {f: getattr(info, f) for f, _ in SqpInfo._fields_ if f != "pad0"}
    out = []
    for i in range(nr.value):
        r = rows[i]
        row = {}
        for f, t in SqpTraceRow._fields_:
            v = getattr(r, f)
            if f == "pad0":
                continue
            if f in ("alpha", "f_trial", "pen_trial"):
                row[f] = np.array(v[: r.n_trials])
            elif f in ("q", "dx"):
                row[f] = np.array(v[: N + 1])
            elif hasattr(v, "__len__"):
                row[f] = np.array(v[:N])
            else:
                row[f] = v
        out.append(row)
    return u, x, lam, pil, piu, d, out


def bfgs_update_blocks(W, s_u, s_x, y_u, y_x):
    """The block-BFGS step with the reset rule on N + 1 packed blocks W
    ((N + 1) x 3); returns (updated W, reset flag)."""
    W = np.array(W, dtype=np.float64).reshape(-1, 3).copy()
    N = W.shape[0] - 1
    s_u, y_u = (np.ascontiguousarray(a, dtype=np.float64) for a in (s_u, y_u))
    s_x, y_x = (np.ascontiguousarray(a, dtype=np.float64) for a in (s_x, y_x))
    assert len(s_u) == N and len(y_u) == N and len(s_x) == N + 1 and len(y_x) == N + 1
    reset = lib().or_bfgs_update_blocks(N, _p(W), _p(s_u), _p(s_x), _p(y_u), _p(y_x))
    return W, reset


def qp_solve(A, B, b, Wxx, Wxu, Wuu, q, r, lb, ub):
    L = lib()
    N = len(B)
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (A, B, b, Wxx, Wxu, Wuu, q, r, lb, ub)]
    du, mu, nul, nuu = (np.zeros(N) for _ in range(4))
    dx = np.zeros(N + 1)
    it = C.c_int(0)
    st = L.or_qp_solve(N, *[_p(a) for a in arrs], _p(du), _p(dx), _p(mu), _p(nul), _p(nuu),
                       C.byref(it))
    return dict(status=st, iters=it.value, du=du, dx=dx, mu=mu, nul=nul, nuu=nuu)


def bfgs_block(w, s, y):
    """Damped BFGS update of a packed block (w = [W11] or [W11, W12, W22])."""
    L = lib()
    w = np.array(w, dtype=np.float64)
    s = np.ascontiguousarray(s, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    L.or_bfgs_block(len(s), _p(w), _p(s), _p(y))
    return w


def philox(ctr, key):
    L = lib()
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    L.or_philox4x32_10(c, k, o)
    return list(o)


def plant_drift(model: dict, n, F, EaR=None, T_in=None):
    L = lib()
    m = make_model(model)
    n = np.ascontiguousarray(n, dtype=np.float64)
    f = np.zeros(3)
    L.or_plant_drift(C.byref(m), model["EaR"] if EaR is None else EaR,
                     model["T_in"] if T_in is None else T_in, _p(n), F, _p(f))
    return f


def model1(model: dict, x, F, EaR=None):
    L = lib()
    m = make_model(model)
    f, fx, fF = C.c_double(), C.c_double(), C.c_double()
    L.or_model1(C.byref(m), model["EaR"] if EaR is None else EaR, x, F, C.byref(f),
                C.byref(fx), C.byref(fF))
    return f.value, fx.value, fF.value


def Fss(model: dict, Tbar, EaR=None):
    return lib().or_Fss(C.byref(make_model(model)), model["EaR"] if EaR is None else EaR,
                        Tbar)


def zbar(model: dict, t):
    return lib().or_zbar(C.byref(make_model(model)), t)


def em_step(model: dict, n, F, h, xi, EaR=None, T_in=None):
    L = lib()
    m = make_model(model)
    n = np.array(n, dtype=np.float64)
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    L.or_em_step(C.byref(m), model["EaR"] if EaR is None else EaR,
                 model["T_in"] if T_in is None else T_in, _p(n), F, h, _p(xi))
    return n


def rk4_interval(model: dict, n_rk4, Ts, x0, v, Fconv, EaR=None):
    L = lib()
    m = make_model(model)
    xF, A, B = C.c_double(), C.c_double(), C.c_double()
    L.or_rk4_interval(C.byref(m), model["EaR"] if EaR is None else EaR, n_rk4, Ts, x0, v,
                      Fconv, C.byref(xF), C.byref(A), C.byref(B))
    return xF.value, A.value, B.value


def ekf_predict(model: dict, n_rk4, F, x, P, EaR=None):
    L = lib()
    m = make_model(model)
    xx, PP = C.c_double(x), C.c_double(P)
    L.or_ekf_predict(C.byref(m), model["EaR"] if EaR is None else EaR, n_rk4, F,
                     C.byref(xx), C.byref(PP))
    return xx.value, PP.value


def ekf_filter(model: dict, y, x, P):
    L = lib()
    m = make_model(model)
    xx, PP, Ps = C.c_double(x), C.c_double(P), C.c_double()
    L.or_ekf_filter(C.byref(m), y, C.byref(xx), C.byref(PP), C.byref(Ps))
    return xx.value, PP.value, Ps.value


def pi_step(ctrl: dict, Ts, ybar, y, ubar, Ihat):
    L = lib()
    c = make_ctrl(ctrl)
    I = C.c_double(Ihat)
    u = L.or_pi_step(C.byref(c), Ts, ybar, y, ubar, C.byref(I))
    return u, I.value


def traj_params(model: dict, seed, j):
    L = lib()
    m = make_model(model)
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    L.or_traj_params(C.byref(m), seed, j, C.byref(a), C.byref(b), C.byref(c))
    return a.value, b.value, c.value


def traj_horizon(ctrl: dict, seed, j):
    L = lib()
    c = make_ctrl(ctrl)
    N, it = C.c_int(), C.c_int()
    L.or_traj_horizon(C.byref(c), seed, j, C.byref(N), C.byref(it))
    return N.value, it.value


# ---------------------------------------------------------------- three-state NMPC model

def _arr(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a if n is None else a.reshape(n)


def drift3(model: dict, n, F, EaR=None, T_in=None):
    L = lib()
    m = make_model(model)
    n = _arr(n).copy()
    f, J, fF = np.zeros(3), np.zeros(9), np.zeros(3)
    L.or_drift3(C.byref(m), model["EaR"] if EaR is None else EaR,
                model["T_in"] if T_in is None else T_in, _p(n), F, _p(f), _p(J), _p(fF))
    return f, J.reshape(3, 3), fF


def rk4_interval3(model: dict, n_rk4, Ts, x0, v, Fconv, EaR=None):
    L = lib()
    m = make_model(model)
    x0 = _arr(x0).copy()
    xF, A, B = np.zeros(3), np.zeros(9), np.zeros(3)
    L.or_rk4_interval3(C.byref(m), model["EaR"] if EaR is None else EaR, n_rk4, Ts, _p(x0), v,
                       Fconv, _p(xF), _p(A), _p(B))
    return xF, A.reshape(3, 3), B


def ekf3_predict(model: dict, n_rk4, F, x, P, EaR=None):
    L = lib()
    m = make_model(model)
    x = _arr(x).copy()
    P = _arr(P).reshape(9).copy()
    L.or_ekf3_predict(C.byref(m), model["EaR"] if EaR is None else EaR, n_rk4, F, _p(x), _p(P))
    return x, P.reshape(3, 3)


def ekf3_filter(model: dict, y, x, P):
    L = lib()
    m = make_model(model)
    x = _arr(x).copy()
    P = _arr(P).reshape(9).copy()
    Ps = np.zeros(9)
    L.or_ekf3_filter(C.byref(m), y, _p(x), _p(P), _p(Ps))
    return x, P.reshape(3, 3), Ps.reshape(3, 3)


def qp3_solve(A, B, b, Wxx, Wxu, Wuu, q, r, lb, ub):
    """Three-state QP: A (N,3,3), B, b (N,3), Wxx (N+1,3,3), Wxu (N+1,3), Wuu (N+1),
    q (N+1,3), r, lb, ub (N)."""
    L = lib()
    N = len(r)
    ins = [_arr(a).copy() for a in (A, B, b, Wxx, Wxu, Wuu, q, r, lb, ub)]
    du, dx, mu = np.zeros(N), np.zeros((N + 1) * 3), np.zeros(N * 3)
    nul, nuu = np.zeros(N), np.zeros(N)
    it = C.c_int()
    st = L.or_qp3_solve(N, *[_p(a) for a in ins], _p(du), _p(dx), _p(mu), _p(nul), _p(nuu),
                        C.byref(it))
    return dict(status=st, iters=it.value, du=du, dx=dx.reshape(N + 1, 3), mu=mu.reshape(N, 3),
                nul=nul, nuu=nuu)


def bfgs_blockn(W, s, y):
    L = lib()
    W = _arr(W).copy()
    n = W.shape[0]
    Wf = W.reshape(n * n).copy()
    L.or_bfgs_blockn(n, _p(Wf), _p(_arr(s).copy()), _p(_arr(y).copy()))
    return Wf.reshape(n, n)


def sqp3(model: dict, ctrl: dict, EaR: float, x0, zbar, u, x, lam=None, pil=None, piu=None):
    """One three-state OCP.  x0 (3), zbar (N+1), u (N), x ((N+1) x 3) scaled."""
    L = lib()
    m, c = make_model(model), make_ctrl(dict(ctrl, nx_model=3))
    N = c.N
    u = _arr(u).copy()
    x = _arr(x).reshape((N + 1) * 3).copy()
    lam = np.zeros(N * 3) if lam is None else _arr(lam).reshape(N * 3).copy()
    pil = np.zeros(N) if pil is None else _arr(pil).copy()
    piu = np.zeros(N) if piu is None else _arr(piu).copy()
    zb = _arr(zbar).copy()
    x0 = _arr(x0).copy()
    info = SqpInfo()
    L.or_sqp3(C.byref(m), C.byref(c), EaR, _p(x0), _p(zb), _p(u), _p(x), _p(lam), _p(pil),
              _p(piu), C.byref(info))
    d = {f: getattr(info, f) for f, _ in SqpInfo._fields_ if f != "pad0"}
    return u, x.reshape(N + 1, 3), lam.reshape(N, 3), pil, piu, d


def ocp_sens(model: dict, ctrl: dict, EaR: float, x0: float, zbar, u, x, lam, pil, piu):
    """du_0/d(x_0, Q_z, R_u, Q_n) at an OCP solution (implicit differentiation)."""
    L = lib()
    m, c = make_model(model), make_ctrl(ctrl)
    arrs = [_arr(a).copy() for a in (zbar, u, x, lam, pil, piu)]
    out = np.zeros(4)
    st = L.or_ocp_sens(C.byref(m), C.byref(c), EaR, x0, *[_p(a) for a in arrs], _p(out))
    return st, out


def nmpc_grad(model: dict, ctrl: dict, seed: int, j0: int, j1: int, threads: int | None = None):
    """Phi_j and dPhi_j/d(Q_z, R_u, Q_n) of NMPC trajectories j0..j1-1 (complex step
    with implicit OCP derivatives); returns (phi[n], dphi[n, 3], sens_fail[n])."""
    L = lib()
    m, c = make_model(model), make_ctrl(dict(ctrl, kind="nmpc"))
    n = j1 - j0
    phi = np.zeros(max(n, 1))
    dphi = np.zeros((max(n, 1), 3))
    fails = np.zeros(max(n, 1), dtype=np.int32)
    if threads is None:
        threads = os.cpu_count() or 1
    if n > 0:
        L.or_nmpc_grad_run(C.byref(m), C.byref(c), seed, j0, j1, int(threads), _p(phi),
                           _p(dphi), fails.ctypes.data_as(C.POINTER(C.c_int)))
    return phi[:n], dphi[:n], fails[:n]
