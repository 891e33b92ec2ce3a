"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's C sources -- a dropped
term, a wrong sign, a wrong index or operand, a wrong constant -- builds that
copy, and runs the pins that should catch it against it (the oracle loads the
library named by MC_ORACLE_LIB).  The pins must fail; against the unaltered
oracle the same selections pass.  Nothing here touches the CUDA path.
"""
import os
import shutil
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (case, file, original text, planted text, pin file, pytest -k selection)
MUTANTS = [
    ("rate law: dropped product-rule term", "or_model.c",
     "const double dr = dk * cA * cB + k * dcA * cB + k * cA * dcB;",
     "const double dr = dk * cA * cB + k * cA * dcB;",
     "test_oracle_model.py", "model1_jacobians"),
    ("rate law: sign of the reaction heat", "or_model.c",
     "*f = F * (m->T_in - cT) + m->beta * r * m->V;",
     "*f = F * (m->T_in - cT) - m->beta * r * m->V;",
     "test_oracle_model.py", "model1_jacobians or shooting"),
    ("RK4: a stage weight", "or_model.c",
     "    x = x + h / 6.0 * (f1 + 2.0 * f2 + 2.0 * f3 + f4);\n    a = a + h / 6.0",
     "    x = x + h / 6.0 * (f1 + 2.0 * f2 + f3 + f4);\n    a = a + h / 6.0",
     "test_oracle_model.py", "rk4"),
    ("CD-EKF: covariance stage uses the wrong slope", "or_model.c",
     "const double p3 = 2.0 * A3 * (Ps + 0.5 * h * p2) + q;",
     "const double p3 = 2.0 * A3 * (Ps + 0.5 * h * p1) + q;",
     "test_oracle_model.py", "ekf_predict"),
    ("Joseph form: dropped measurement-noise term", "or_model.c",
     "const double Pj = ImKC * (*P) * ImKC + K * R * K;",
     "const double Pj = ImKC * (*P) * ImKC;",
     "test_oracle_model.py", "ekf_filter"),
    ("Euler-Maruyama: h instead of sqrt(h) in the diffusion", "or_model.c",
     "n[i] = n[i] + f[i] * h + F * m->sigma[i] * sq * xi[i];",
     "n[i] = n[i] + f[i] * h + F * m->sigma[i] * h * xi[i];",
     "test_oracle_model.py", "em_"),
    ("plant: stoichiometric coefficient of B", "or_model.c",
     "f[1] = m->cB_in * F - cB * F + (-2.0) * r * m->V;",
     "f[1] = m->cB_in * F - cB * F + (-1.0) * r * m->V;",
     "test_oracle_model.py", "invariants"),
    ("PI: sign of the anti-windup term", "or_closedloop.c",
     "const double Iaw = Ts * c->kaw * (uhat - u);",
     "const double Iaw = Ts * c->kaw * (u - uhat);",
     "test_oracle_model.py", "pi_hand"),
    ("Phi: divided by K instead of K + 1", "or_closedloop.c",
     "out->phi = phi / (double)(K + 1);",
     "out->phi = phi / (double)K;",
     "test_oracle_model.py", "phi_definition"),
    ("Philox: a multiplier constant", "or_random.c",
     "0xD2511F53u", "0xD2511F35u",
     "test_oracle_random.py", "known_answers"),
    ("QP: sign of q in the multiplier recursion", "or_sqp.c",
     "mu[k - 1] = mu[k] * A[k] - (Wxx[k] * dx[k] + Wxu[k] * du[k] + q[k]);",
     "mu[k - 1] = mu[k] * A[k] - (Wxx[k] * dx[k] + Wxu[k] * du[k] - q[k]);",
     "test_oracle_qp.py", "kkt_certificate"),
    ("SQP: multiplier index in the Lagrangian gradient", "or_sqp.c",
     "gx[k] = e->q[k] - lam[k] * e->A[k] + lam[k - 1];",
     "gx[k] = e->q[k] - lam[k - 1] * e->A[k] + lam[k];",
     "test_oracle_sqp.py", "kkt_point or grid_search"),
    ("BFGS: damping threshold", "or_sqp.c",
     "(sy >= 0.2 * sWs)", "(sy >= 0.02 * sWs)",
     "test_oracle_sqp.py", "bfgs"),
    ("OCP sensitivity: dropped Hessian cross term", "or_sqp.c",
     "K[IU(k) * n + IX(k)] += -lam[k] * Fxu[k];",
     "K[IU(k) * n + IX(k)] += 0.0 * Fxu[k];",
     "test_oracle_sqp.py", "ocp_sensitivity"),
    ("Box-Muller: angle of pi instead of 2 pi", "or_random.c",
     "const double ang = 2.0 * M_PI * u2;",
     "const double ang = M_PI * u2;",
     "test_oracle_random.py", "box_muller"),
    ("set-point schedule: strict comparison", "or_model.c",
     "if (t >= m->sp_time[s]) z = m->sp_value[s];",
     "if (t > m->sp_time[s]) z = m->sp_value[s];",
     "test_oracle_model.py", "zbar"),
    ("trajectory parameters: lognormal E_a/R without its spread", "or_random.c",
     "*EaR_j = (m->Ea_logsd != 0.0) ? m->EaR * exp(m->Ea_logsd * z[0]) : m->EaR;",
     "*EaR_j = (m->Ea_logsd != 0.0) ? m->EaR * exp(0.5 * m->Ea_logsd * z[0]) : m->EaR;",
     "test_oracle_closedloop.py", "trajectory_parameters"),
    ("three-state drift: Jacobian misses the dilution term", "or_nmpc3.c",
     "for (int q = 0; q < 3; ++q) J[p * 3 + q] = (p == q ? -F / V : 0.0) + S[p] * drv[q];",
     "for (int q = 0; q < 3; ++q) J[p * 3 + q] = S[p] * drv[q];",
     "test_oracle_nmpc3.py", "drift3_is_the_plant_drift"),
    ("PI gradient: complex-step path with the anti-windup sign flipped", "or_grad.c",
     "Ihat = Ii + m->Ts * kaw * (uhat - u);",
     "Ihat = Ii + m->Ts * kaw * (u - uhat);",
     "test_oracle_grad.py", "real_part or richardson"),
    ("SQP: penalty weights set to |mu| at every iteration", "or_sqp.c",
     "sigma[k] = (l == 0) ? fabs(mu[k]) : fmax(fabs(mu[k]), 0.5 * (sigma[k] + fabs(mu[k])));",
     "sigma[k] = fabs(mu[k]);",
     "test_oracle_sqp_trace.py", "penalty"),
    ("SQP: s_d averages the multipliers over N instead of 3N", "or_sqp.c",
     "mult1 / (double)(3 * N)", "mult1 / (double)N",
     "test_oracle_sqp_trace.py", "scaling"),
    ("SQP: Armijo constant 0.1 instead of 1e-4", "or_sqp.c",
     "c1 = 1e-4, beta_ls", "c1 = 0.1, beta_ls",
     "test_oracle_sqp_trace.py", "armijo"),
    ("SQP: step quartered instead of halved", "or_sqp.c",
     "beta_ls = 0.5", "beta_ls = 0.25",
     "test_oracle_sqp_trace.py", "armijo"),
    ("SQP: Hessian reset disabled", "or_sqp.c",
     "  if (!pd) {\n    for (int k = 0; k <= N; ++k) { Wb[k][0] = 1.0;",
     "  if (0) {\n    for (int k = 0; k <= N; ++k) { Wb[k][0] = 1.0;",
     "test_oracle_sqp_trace.py", "reset"),
    ("SQP: reset of the offending block only", "or_sqp.c",
     "    for (int k = 0; k <= N; ++k) { Wb[k][0] = 1.0; Wb[k][1] = 0.0; Wb[k][2] = 1.0; }\n    return 1;",
     "    for (int k = 0; k <= N; ++k) if (!block_pd(k == 0 || k == N ? 1 : 2, Wb[k])) "
     "{ Wb[k][0] = 1.0; Wb[k][1] = 0.0; Wb[k][2] = 1.0; }\n    return 1;",
     "test_oracle_sqp_trace.py", "reset"),
    ("SQP: convergence test ignores the state part of grad L", "or_sqp.c",
     "for (int k = 1; k <= N; ++k) kg = fmax(kg, fabs(gx[k]));",
     "for (int k = 1; k <= N; ++k) kg = fmax(kg, 0.0 * fabs(gx[k]));",
     "test_oracle_sqp_trace.py", "scaling"),
]


def _run_pins(pin_file, selection, lib_path):
    env = dict(os.environ)
    if lib_path:
        env["MC_ORACLE_LIB"] = lib_path
    else:
        env.pop("MC_ORACLE_LIB", None)
    cmd = [sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", pin_file), "-q", "-x",
           "-m", "not gpu", "-k", selection, "-p", "no:cacheprovider"]
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


@pytest.mark.parametrize("pin_file", sorted({m[4] for m in MUTANTS}))
def test_pin_selections_pass_on_the_oracle(pin_file):
    oracle.build()
    selection = " or ".join(sorted({f"({m[5]})" for m in MUTANTS if m[4] == pin_file}))
    r = _run_pins(pin_file, selection, None)
    assert r.returncode == 0, r.stdout[-2000:]
    assert " passed" in r.stdout


@pytest.mark.parametrize("case,src,old,new,pin_file,selection", MUTANTS,
                         ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(tmp_path, case, src, old, new, pin_file, selection):
    for path in oracle.sources():
        shutil.copy(path, tmp_path)
    target = tmp_path / src
    text = target.read_text()
    assert text.count(old) == 1, case
    target.write_text(text.replace(old, new))
    lib = oracle.compile_sources(str(tmp_path), str(tmp_path / "libmutant.so"))
    r = _run_pins(pin_file, selection, lib)
    assert r.returncode == 1, (case, r.returncode, r.stdout[-1500:])
    assert " failed" in r.stdout, (case, r.stdout[-1500:])
