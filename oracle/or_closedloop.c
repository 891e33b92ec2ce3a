/*
 * or_closedloop.c -- one stochastic closed-loop simulation (Sec. VII) with the
 * NMPC (Sec. III-IV) or the PI controller (Sec. V), and a thread pool that runs
 * independent trajectories on the host cores, one trajectory per thread at a
 * time, as the paper's Monte Carlo toolbox does (Sec. I, VII-B).
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

/* PI controller with input bounds and anti-windup, Eq. (PI):
 *   e = ybar - y, P = kP e, I = Ihat + Ts kI e, uhat = ubar + P + I,
 *   u = max(u_min, min(u_max, uhat)), I_aw = Ts kaw (uhat - u), Ihat = I + I_aw.
 * Flows in L/s; the bounds are given in mL/min. */
double or_pi_step(const or_ctrl* c, double Ts, double ybar, double y, double ubar,
                  double* Ihat) {
  const double umin = c->u_min / 60000.0, umax = c->u_max / 60000.0;
  const double e = ybar - y;
  const double P = c->kP * e;
  const double I = *Ihat + Ts * c->kI * e;
  const double uhat = ubar + P + I;
  const double u = fmax(umin, fmin(umax, uhat));
  const double Iaw = Ts * c->kaw * (uhat - u);
  *Ihat = I + Iaw;
  return u;
}

static void trace_row(double* trace, int i, double T, double y, double xhat, double u,
                      double it) {
  if (!trace) return;
  double* r = trace + 5 * (size_t)i;
  r[0] = T; r[1] = y; r[2] = xhat; r[3] = u; r[4] = it;
}

void or_traj(const or_model* m, const or_ctrl* c_in, uint64_t seed, int64_t j,
             or_traj_out* out, double* trace) {
  double EaR, t_d, dTin;
  or_traj_params(m, seed, j, &EaR, &t_d, &dTin);
  /* the controller's model (EKF, OCP, steady-state input): the trajectory's
   * E_a/R, or the nominal one when the perturbation is the plant's alone */
  const double EaR_c = m->Ea_plant_only ? m->EaR : EaR;
  /* this trajectory's horizon and SQP iteration limit (uneven batches) */
  or_ctrl cj = *c_in;
  or_traj_horizon(c_in, seed, j, &cj.N, &cj.sqp_max_it);
  const or_ctrl* c = &cj;
  memset(out, 0, sizeof(*out));

  /* plant initialised with the feed, x_0 = n_0 = C_in V (Sec. VII-A) */
  double n[3] = {m->cA_in * m->V, m->cB_in * m->V, m->T_in * m->V};
  const int K = m->n_steps;
  const double h = m->Ts / (double)m->n_em;
  double phi = 0.0;

  /* NMPC state: CD-EKF estimate and the SQP warm start */
  const int N = c->N;
  const double Fconv = c->u_scale / 60000.0;
  double xhat = m->T_in * m->V, P = c->P0;
  double u[OR_MAX_N], x[OR_MAX_N + 1], lam[OR_MAX_N], pil[OR_MAX_N], piu[OR_MAX_N];
  double zb[OR_MAX_N + 1];
  double F_prev = 0.0;
  double Ihat = 0.0;
  /* three-state NMPC model: estimate of n, its 3x3 covariance, and the
   * warm start with three states and three multipliers per stage */
  const int nx3 = (c->kind == 0 && c->nx_model == 3);
  double xh3[3] = {m->cA_in * m->V, m->cB_in * m->V, m->T_in * m->V};
  double P3[9] = {c->P0, 0.0, 0.0, 0.0, c->P0, 0.0, 0.0, 0.0, c->P0};
  static __thread double x3[(OR_MAX_N + 1) * 3], lam3[OR_MAX_N * 3];

  if (nx3) {
    double v0 = or_Fss(m, EaR_c, or_zbar(m, m->t0)) / Fconv;
    v0 = fmin(fmax(v0, c->u_min / c->u_scale), c->u_max / c->u_scale);
    for (int k = 0; k < N; ++k) {
      u[k] = v0;
      pil[k] = piu[k] = 0.0;
      for (int q = 0; q < 3; ++q) lam3[k * 3 + q] = 0.0;
    }
    for (int k = 0; k <= N; ++k)
      for (int q = 0; q < 3; ++q) x3[k * 3 + q] = xh3[q] / c->x_scale;
  } else if (c->kind == 0) {
    /* first OCP guess: steady-state input of the first set-point (clipped),
     * states at the initial estimate, multipliers zero */
    double v0 = or_Fss(m, EaR_c, or_zbar(m, m->t0)) / Fconv;
    v0 = fmin(fmax(v0, c->u_min / c->u_scale), c->u_max / c->u_scale);
    x[0] = xhat / c->x_scale;
    for (int k = 0; k < N; ++k) {
      u[k] = v0;
      x[k + 1] = xhat / c->x_scale;
      lam[k] = pil[k] = piu[k] = 0.0;
    }
  }

  for (int i = 0; i <= K; ++i) {
    const double t_i = m->t0 + (double)i * m->Ts;
    const double cT = n[2] / m->V;
    int bad3 = 0;
    for (int q = 0; q < 3 && nx3; ++q) bad3 |= !isfinite(xh3[q]);
    for (int q = 0; q < 9 && nx3; ++q) bad3 |= !isfinite(P3[q]);
    if (!isfinite(cT) || !isfinite(xhat) || !isfinite(P) || bad3) {
      out->nonfinite = 1;
      phi = NAN;
      break;
    }
    /* performance index, Eq. (Phi), on the true plant output z = c_T */
    const double ez = cT - or_zbar(m, t_i);
    phi += ez * ez;
    if (i == K) break;

    /* measurement y_i = c_T(t_i) + v_i */
    const double y = cT + m->meas_sd * or_meas_noise(seed, j, i);
    const double zbar_i = or_zbar(m, t_i);
    double F;
    double its = 0.0;
    if (nx3) {
      /* three-state CD-EKF and OCP, as below */
      if (i > 0) or_ekf3_predict(m, EaR_c, c->n_rk4, F_prev, xh3, P3);
      or_ekf3_filter(m, y, xh3, P3, NULL);
      for (int k = 1; k <= N; ++k) zb[k] = or_zbar(m, m->t0 + (double)(i + k) * m->Ts);
      double x0s[3] = {xh3[0] / c->x_scale, xh3[1] / c->x_scale, xh3[2] / c->x_scale};
      or_sqp_info info;
      or_sqp3(m, c, EaR_c, x0s, zb, u, x3, lam3, pil, piu, &info);
      out->n_ocp++;
      out->sqp_iters += info.iters;
      out->ls_trials += info.ls_trials;
      out->n_hess_reset += info.n_hess_reset;
      out->qp_iters += info.qp_iters;
      if (info.status == 1) out->n_ocp_failed++;
      if (info.status == 2) out->n_ls_fail++;
      its = info.iters;
      F = u[0] * Fconv;
      for (int k = 0; k < N - 1; ++k) {
        u[k] = u[k + 1];
        pil[k] = pil[k + 1];
        piu[k] = piu[k + 1];
        for (int q = 0; q < 3; ++q) {
          x3[(k + 1) * 3 + q] = x3[(k + 2) * 3 + q];
          lam3[k * 3 + q] = lam3[(k + 1) * 3 + q];
        }
      }
      xhat = xh3[2];
    } else if (c->kind == 0) {
      /* CD-EKF: prediction from t_{i-1} (none before the first sample), filtering */
      if (i > 0) or_ekf_predict(m, EaR_c, c->n_rk4, F_prev, &xhat, &P);
      or_ekf_filter(m, y, &xhat, &P, NULL);
      /* regulator: OCP over the horizon t_{i+1} .. t_{i+N} */
      for (int k = 1; k <= N; ++k) zb[k] = or_zbar(m, m->t0 + (double)(i + k) * m->Ts);
      or_sqp_info info;
      or_sqp(m, c, EaR_c, xhat / c->x_scale, zb, u, x, lam, pil, piu, &info);
      out->n_ocp++;
      out->sqp_iters += info.iters;
      out->ls_trials += info.ls_trials;
      out->n_hess_reset += info.n_hess_reset;
      out->qp_iters += info.qp_iters;
      if (info.status == 1) out->n_ocp_failed++;
      if (info.status == 2) out->n_ls_fail++;
      its = info.iters;
      F = u[0] * Fconv;
      /* receding horizon: shift the solution one interval for the next OCP,
       * duplicating the last interval */
      for (int k = 0; k < N - 1; ++k) {
        u[k] = u[k + 1];
        x[k + 1] = x[k + 2];
        lam[k] = lam[k + 1];
        pil[k] = pil[k + 1];
        piu[k] = piu[k + 1];
      }
    } else {
      const double ubar = or_Fss(m, EaR_c, zbar_i);
      F = or_pi_step(c, m->Ts, zbar_i, y, ubar, &Ihat);
    }
    trace_row(trace, i, cT, y, (c->kind == 0) ? xhat / m->V : NAN, F * 60000.0, its);

    /* plant: N_s Euler-Maruyama substeps with zero-order hold on F and T_in */
    for (int s = 0; s < m->n_em; ++s) {
      const int64_t ks = (int64_t)i * m->n_em + s;
      const double tau = m->t0 + (double)ks * h;
      const double T_in = (m->dTin_step != 0.0 && tau >= t_d) ? m->T_in + dTin : m->T_in;
      double xi[3];
      or_process_noise(seed, j, ks, xi);
      or_em_step(m, EaR, T_in, n, F, h, xi);
    }
    F_prev = F;
  }
  out->phi = phi / (double)(K + 1);
}

typedef struct {
  const or_model* m;
  const or_ctrl* c;
  uint64_t seed;
  int64_t j0, j1;
  int tid, nt;
  or_traj_out* out;
} job_t;

static void* worker(void* arg) {
  job_t* jb = (job_t*)arg;
  for (int64_t j = jb->j0 + jb->tid; j < jb->j1; j += jb->nt)
    or_traj(jb->m, jb->c, jb->seed, j, &jb->out[j - jb->j0], NULL);
  return NULL;
}

/* Monte Carlo driver: trajectories j0 .. j1-1 on n_threads host threads. */
void or_run(const or_model* m, const or_ctrl* c, uint64_t seed, int64_t j0,
            int64_t j1, int n_threads, or_traj_out* out) {
  if (n_threads < 1) n_threads = 1;
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)n_threads);
  job_t* jobs = (job_t*)malloc(sizeof(job_t) * (size_t)n_threads);
  for (int t = 0; t < n_threads; ++t) {
    jobs[t] = (job_t){m, c, seed, j0, j1, t, n_threads, out};
    pthread_create(&th[t], NULL, worker, &jobs[t]);
  }
  for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
  free(th);
  free(jobs);
}
