"""Synthetic workloads of the Monte Carlo closed-loop study (arXiv 2212.02197).

Plain data only: model parameters, controller settings, set-point schedules,
sizes and seeds.  Nothing here evaluates the method; the CUDA path and the
oracle each consume these dicts on their own.

The paper's case study (Sec. VI-VII) is a synthetic model, so these presets
are the workload itself.  Values the paper does not print are the readings
recorded with the design notes:

* CSTR parameters (Sec. VI defers them to its reference [wahlgreen:2020a]):
  V = 0.105 L, k0 = exp(24.6) L/(mol s), E_a/R = 8500 K,
  beta = -dH_r/(rho c_P) = 560/4.186 K L/mol, c_A,in = 0.8 mol/L,
  c_B,in = 1.2 mol/L, T_in = 273.65 K.  With them the steady-state flow has a
  minimum of about 293 mL/min at 286.5 K and a maximum of about 637 mL/min at
  329.8 K; between the two lies the branch of unstable steady states.
* sigma-bar = 1e-2 diag(c_A,in, c_B,in, T_in); measurement sd 0.1 K.
* T_s = 0.5 s with N_s = 10 Euler-Maruyama substeps (0.05 s, the paper's own
  EM step of 1 s / 20).
* Set-point z-bar(t): piecewise constant in absolute time, 276 K from 0 s and
  282 K from 20 s (low stable branch), 290 K from 40 s (unstable branch) and
  340 K from 80 s (high stable branch).  Every target can be reached from the
  paper's initial state, the reactor filled with feed at T_in.
* NMPC scaling: the OCP state is the temperature (n_T / V, in K) and the OCP
  input is F / u_max; the SQP tolerance is 1e-5 on the scaled KKT test.
"""
from __future__ import annotations

import copy
import math

SEED = 20221205

CSTR = dict(
    V=0.105,
    k0=math.exp(24.6),
    EaR=8500.0,
    beta=560.0 / 4.186,
    cA_in=0.8,
    cB_in=1.2,
    T_in=273.65,
)

# set-point schedule: (segment start time in s, set-point in K)
SCHEDULE = ((0.0, 276.0), (20.0, 282.0), (40.0, 290.0), (80.0, 340.0))
SCHEDULE_PAPER = ((0.0, 276.0), (20.0, 282.0), (40.0, 290.0), (80.0, 340.0),
                  (300.0, 310.0), (450.0, 280.0))


def model(n_steps: int, Ts: float = 0.5, n_em: int = 10, Ea_logsd: float = 0.0,
          dTin_step: float = 0.0, schedule=SCHEDULE, Ea_plant_only: bool = False) -> dict:
    """Plant/model/closed-loop dict.  Ea_plant_only: the E_a/R perturbation acts
    on the plant alone (the controller's model keeps the nominal value)."""
    m = dict(CSTR)
    m["sigma"] = [1e-2 * m["cA_in"], 1e-2 * m["cB_in"], 1e-2 * m["T_in"]]
    m["meas_sd"] = 0.1
    m["Ts"] = float(Ts)
    m["t0"] = 0.0
    m["n_steps"] = int(n_steps)
    m["n_em"] = int(n_em)
    m["sp_time"] = [float(t) for t, _ in schedule]
    m["sp_value"] = [float(v) for _, v in schedule]
    m["Ea_logsd"] = float(Ea_logsd)
    m["dTin_step"] = float(dTin_step)
    m["Ea_plant_only"] = bool(Ea_plant_only)
    return m


def nmpc(N: int = 20, u_max: float = 800.0, precision: str = "fp64") -> dict:
    """NMPC settings of Sec. VII-A (N_c = 5 RK4 steps, Q_z = 1, P_{-1|-1} = 1e-6).

    FP64 runs the persistent schedule (lanes share the line-search shooting
    while each advances its own SQP); mixed precision, where the FP64 phases
    dominate, runs the static one.  Mixed precision shoots in FP32, whose rounding (about 1e-7 of the RK4
    increments) sets a floor under the merit function; its SQP stops at
    1e-3 on the scaled KKT test or after 3 step halvings that find no
    decrease, and is accepted statistically against FP64."""
    mixed = precision == "mixed"
    return dict(kind="nmpc", precision=precision, N=int(N), n_rk4=5, sqp_max_it=100,
                ls_max=3 if mixed else 30, u_min=0.0, u_max=float(u_max), kP=-1e-3, kI=-1e-4,
                kaw=-1e-1, Qz=1.0, Ru=0.0, Qn=0.0, P0=1e-6, sqp_tol=1e-3 if mixed else 1e-5,
                u_scale=float(u_max), x_scale=CSTR["V"], qp_solver="active_set", ip_max_it=60,
                ip_tol=1e-14, schedule="static" if mixed else "persistent")


def pi(u_max: float = 800.0, precision: str = "fp64") -> dict:
    """PI settings of Sec. VII-A: k_P = -1e-3, k_I = -1e-4, k_aw = -1e-1."""
    c = nmpc(u_max=u_max, precision=precision)
    c["kind"] = "pi"
    return c


WORKLOADS = {
    # small case: 100 NMPC + 100 PI trajectories, 120 steps, N = 20 (parity)
    "cstr_100x120_N20_fp64": dict(model=model(120), nmpc=nmpc(20), pi=pi(), n_traj=100,
                                  seed=SEED),
    # paper-scale FP64 study: 30k NMPC + 30k PI, 240 steps, N = 20, T_in step +-5 K
    "cstr_30k_x240_N20_fp64": dict(model=model(240, dTin_step=5.0), nmpc=nmpc(20), pi=pi(),
                                   n_traj=30000, seed=SEED),
    # the paper-scale study in mixed precision (same trajectories and noise)
    "cstr_30k_x240_N20_mixed": dict(model=model(240, dTin_step=5.0),
                                    nmpc=nmpc(20, precision="mixed"),
                                    pi=pi(precision="mixed"), n_traj=30000, seed=SEED),
    # mixed precision: 100k NMPC, 240 steps, N = 30, E_a/R lognormal sd 2 %
    "cstr_100k_x240_N30_mixed": dict(model=model(240, Ea_logsd=0.02),
                                     nmpc=nmpc(30, precision="mixed"), pi=None,
                                     n_traj=100000, seed=SEED),
    # model mismatch: the paper-scale FP64 study with E_a/R lognormal sd 2 % in the
    # plant only; the controllers' models (EKF, OCP, steady-state input) keep the
    # nominal E_a/R
    "cstr_30k_x240_N20_fp64_mismatch": dict(
        model=model(240, dTin_step=5.0, Ea_logsd=0.02, Ea_plant_only=True), nmpc=nmpc(20),
        pi=pi(), n_traj=30000, seed=SEED),
    # the three-state NMPC model (3x3 CD-EKF, three states per OCP stage): the
    # paper-scale FP64 study with the controller on the plant's own model
    "cstr_30k_x240_N20_fp64_nx3": dict(
        model=model(240, dTin_step=5.0),
        nmpc=dict(nmpc(20), nx_model=3, schedule="persistent"), pi=pi(), n_traj=30000,
        seed=SEED),
    # uneven batches: 262,144 trajectories, 120 steps, horizon uniform on 10..40 and
    # SQP iteration limit uniform on 5..30 per trajectory, persistent schedule
    "cstr_262k_x120_N10to40_uneven": dict(
        model=model(120),
        nmpc=dict(nmpc(40), N_min=10, sqp_max_it=30, sqp_max_it_min=5, schedule="persistent"),
        pi=None, n_traj=262144, seed=SEED),
    # the paper's own setting (Sec. VII-A): T_s = 1 s, N_s = 20, N = 60, 600 steps
    "cstr_paper_30k_x600_N60": dict(model=model(600, Ts=1.0, n_em=20,
                                                schedule=SCHEDULE_PAPER),
                                    nmpc=nmpc(60, u_max=1000.0), pi=pi(u_max=1000.0),
                                    n_traj=30000, seed=SEED),
}


def get(name: str, **overrides) -> dict:
    w = copy.deepcopy(WORKLOADS[name])
    w.update(overrides)
    return w
