/*
 * or_grad.c -- derivative of one trajectory's performance index Phi_j with
 * respect to a gain of the PI controller (Sec. V, Eq. (PI)): k_P, k_I or k_aw.
 *
 * Method: complex-step differentiation (Squire and Trapp, SIAM Review 40,
 * 1998; Martins, Sturdza and Alonso, ACM TOMS 29, 2003).  The closed loop of
 * Sec. VII with the PI controller is run once in complex arithmetic with the
 * chosen gain set to k + i h; then dPhi/dk = Im Phi(k + i h) / h with an error
 * of order h^2 and no subtractive cancellation, so h = 1e-20 |k| returns the
 * derivative of the discrete closed loop to rounding.  Comparisons (the input
 * clip of Eq. (PI), the inlet step time) act on real parts, which yields the
 * derivative of the branch the real simulation takes.  Noise is drawn exactly
 * as in or_traj and does not depend on the gains.
 *
 * The clip u = max(u_min, min(u_max, u-hat)) passes u-hat through only when
 * u_min < u-hat < u_max strictly; at equality it counts as saturated (zero
 * derivative).  The real parts follow or_traj's PI trajectory operation by
 * operation; they differ from it only by terms of order h^2.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 */
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

typedef double complex cplx;

/* three-state CSTR drift, Eq. (CSTR), in complex arithmetic */
static void drift_c(const or_model* m, double EaR, double T_in, const cplx n[3], cplx F,
                    cplx f[3]) {
  const cplx cA = n[0] / m->V;
  const cplx cB = n[1] / m->V;
  const cplx cT = n[2] / m->V;
  const cplx k = m->k0 * cexp(-EaR / cT);
  const cplx r = k * cA * cB;
  f[0] = m->cA_in * F - cA * F + (-1.0) * r * m->V;
  f[1] = m->cB_in * F - cB * F + (-2.0) * r * m->V;
  f[2] = T_in * F - cT * F + m->beta * r * m->V;
}

double or_pi_phi_cs(const or_model* m, const or_ctrl* c, uint64_t seed, int64_t j,
                    int which, double h_cs, double* dphi) {
  double EaR, t_d, dTin;
  or_traj_params(m, seed, j, &EaR, &t_d, &dTin);
  cplx kP = c->kP, kI = c->kI, kaw = c->kaw;
  if (which == 0) kP += I * h_cs;
  if (which == 1) kI += I * h_cs;
  if (which == 2) kaw += I * h_cs;
  const double umin = c->u_min / 60000.0, umax = c->u_max / 60000.0;
  cplx n[3] = {m->cA_in * m->V, m->cB_in * m->V, m->T_in * m->V};
  const int K = m->n_steps;
  const double h = m->Ts / (double)m->n_em;
  const double sq = sqrt(h);
  cplx phi = 0.0, Ihat = 0.0;
  for (int i = 0; i <= K; ++i) {
    const double t_i = m->t0 + (double)i * m->Ts;
    const cplx cT = n[2] / m->V;
    if (!isfinite(creal(cT))) {
      *dphi = NAN;
      return NAN;
    }
    const cplx ez = cT - or_zbar(m, t_i);
    phi += ez * ez;
    if (i == K) break;
    const cplx y = cT + m->meas_sd * or_meas_noise(seed, j, i);
    const double zbar_i = or_zbar(m, t_i);
    const double ubar = or_Fss(m, m->Ea_plant_only ? m->EaR : EaR, zbar_i);
    /* Eq. (PI) */
    const cplx e = zbar_i - y;
    const cplx P = kP * e;
    const cplx Ii = Ihat + m->Ts * kI * e;
    const cplx uhat = ubar + P + Ii;
    cplx u;
    if (creal(uhat) > umin && creal(uhat) < umax) u = uhat;
    else u = (creal(uhat) >= umax) ? umax : umin;
    Ihat = Ii + m->Ts * kaw * (uhat - u);
    /* plant: N_s Euler-Maruyama substeps, Eq. (CDS) */
    for (int s = 0; s < m->n_em; ++s) {
      const int64_t ks = (int64_t)i * m->n_em + s;
      const double tau = m->t0 + (double)ks * h;
      const double T_in = (m->dTin_step != 0.0 && tau >= t_d) ? m->T_in + dTin : m->T_in;
      double xi[3];
      or_process_noise(seed, j, ks, xi);
      cplx f[3];
      drift_c(m, EaR, T_in, n, u, f);
      for (int q = 0; q < 3; ++q) n[q] = n[q] + f[q] * h + u * m->sigma[q] * sq * xi[q];
    }
  }
  phi = phi / (double)(K + 1);
  *dphi = cimag(phi) / h_cs;
  return creal(phi);
}

typedef struct {
  const or_model* m;
  const or_ctrl* c;
  uint64_t seed;
  int64_t j0, j1;
  int tid, nt;
  double *phi, *dphi;
} gjob_t;

static void* gworker(void* arg) {
  gjob_t* g = (gjob_t*)arg;
  const double gains[3] = {g->c->kP, g->c->kI, g->c->kaw};
  for (int64_t j = g->j0 + g->tid; j < g->j1; j += g->nt) {
    const int64_t r = j - g->j0;
    for (int q = 0; q < 3; ++q) {
      const double hq = 1e-20 * (gains[q] != 0.0 ? fabs(gains[q]) : 1.0);
      g->phi[r] = or_pi_phi_cs(g->m, g->c, g->seed, j, q, hq, &g->dphi[3 * r + q]);
    }
  }
  return NULL;
}

void or_pi_grad_run(const or_model* m, const or_ctrl* c, uint64_t seed, int64_t j0,
                    int64_t j1, int n_threads, double* phi, double* dphi) {
  if (n_threads < 1) n_threads = 1;
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)n_threads);
  gjob_t* jobs = (gjob_t*)malloc(sizeof(gjob_t) * (size_t)n_threads);
  for (int t = 0; t < n_threads; ++t) {
    jobs[t] = (gjob_t){m, c, seed, j0, j1, t, n_threads, phi, dphi};
    pthread_create(&th[t], NULL, gworker, &jobs[t]);
  }
  for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
  free(th);
  free(jobs);
}

/* ------------------------------------------------------------------------ */
/* Derivative of Phi_j with respect to a weight of the extended NMPC objective
 * (which = 0: Q_z, 1: R_u, 2: Q_n), one-state NMPC.  The derivative is that
 * of the closed loop in which every OCP is represented by its solution map
 * u_0 = U(x-hat, theta) at the KKT point the SQP returns: the plant, the
 * measurement and the CD-EKF are run in complex arithmetic (complex step,
 * h_cs), each OCP is solved on the real parts by or_sqp, and the imaginary
 * part of its input is the implicit derivative or_ocp_sens applied to the
 * imaginary parts of x-hat and of the weight.  Returns Phi_j; *dphi. */

/* one-state model in complex arithmetic: f and df/dx (or_model1's formulas) */
static void model1_c(const or_model* m, double EaR, cplx x, cplx F, cplx* f, cplx* fx) {
  const cplx cT = x / m->V;
  const cplx cA = m->cA_in + (m->T_in - cT) / m->beta;
  const cplx cB = m->cB_in + 2.0 * (m->T_in - cT) / m->beta;
  const cplx k = m->k0 * cexp(-EaR / cT);
  const cplx r = k * cA * cB;
  *f = F * (m->T_in - cT) + m->beta * r * m->V;
  const cplx dk = k * EaR / (cT * cT);
  const double dcA = -1.0 / m->beta, dcB = -2.0 / m->beta;
  const cplx dr = dk * cA * cB + k * dcA * cB + k * cA * dcB;
  *fx = (-F + m->beta * dr * m->V) / m->V;
}

/* CD-EKF prediction (RK4 on x and P) and Joseph filter, complex */
static void ekf_predict_c(const or_model* m, double EaR, int n_rk4, cplx F, cplx* x, cplx* P) {
  const double h = m->Ts / (double)n_rk4;
  const cplx q = (F * m->sigma[2]) * (F * m->sigma[2]);
  cplx xs = *x, Ps = *P;
  for (int s = 0; s < n_rk4; ++s) {
    cplx f1, A1, f2, A2, f3, A3, f4, A4;
    model1_c(m, EaR, xs, F, &f1, &A1);
    const cplx p1 = 2.0 * A1 * Ps + q;
    model1_c(m, EaR, xs + 0.5 * h * f1, F, &f2, &A2);
    const cplx p2 = 2.0 * A2 * (Ps + 0.5 * h * p1) + q;
    model1_c(m, EaR, xs + 0.5 * h * f2, F, &f3, &A3);
    const cplx p3 = 2.0 * A3 * (Ps + 0.5 * h * p2) + q;
    model1_c(m, EaR, xs + h * f3, F, &f4, &A4);
    const cplx p4 = 2.0 * A4 * (Ps + h * p3) + q;
    xs = xs + h / 6.0 * (f1 + 2.0 * f2 + 2.0 * f3 + f4);
    Ps = Ps + h / 6.0 * (p1 + 2.0 * p2 + 2.0 * p3 + p4);
  }
  *x = xs;
  *P = Ps;
}

static void ekf_filter_c(const or_model* m, cplx y, cplx* x, cplx* P) {
  const double R = m->meas_sd * m->meas_sd, C = 1.0 / m->V;
  const cplx e = y - C * (*x);
  const cplx Re = R + C * (*P) * C;
  const cplx K = (*P) * C / Re;
  const cplx M = 1.0 - K * C;
  *P = M * (*P) * M + K * R * K;
  *x = *x + K * e;
}

double or_nmpc_phi_cs(const or_model* m, const or_ctrl* c, uint64_t seed, int64_t j, int which,
                      double h_cs, double* dphi, int* n_sens_fail) {
  double EaR, t_d, dTin;
  or_traj_params(m, seed, j, &EaR, &t_d, &dTin);
  const double EaR_c = m->Ea_plant_only ? m->EaR : EaR;
  const int N = c->N, K = m->n_steps;
  const double h = m->Ts / (double)m->n_em, sq = sqrt(h);
  const double Fconv = c->u_scale / 60000.0;
  double u[OR_MAX_N], x[OR_MAX_N + 1], lam[OR_MAX_N], pil[OR_MAX_N], piu[OR_MAX_N];
  double zb[OR_MAX_N + 1];
  cplx n[3] = {m->cA_in * m->V, m->cB_in * m->V, m->T_in * m->V};
  cplx xhat = m->T_in * m->V, P = c->P0, F_prev = 0.0, phi = 0.0;
  *n_sens_fail = 0;
  double v0 = or_Fss(m, EaR_c, or_zbar(m, m->t0)) / Fconv;
  v0 = fmin(fmax(v0, c->u_min / c->u_scale), c->u_max / c->u_scale);
  x[0] = creal(xhat) / c->x_scale;
  for (int k = 0; k < N; ++k) {
    u[k] = v0;
    x[k + 1] = creal(xhat) / c->x_scale;
    lam[k] = pil[k] = piu[k] = 0.0;
  }
  for (int i = 0; i <= K; ++i) {
    const double t_i = m->t0 + (double)i * m->Ts;
    const cplx cT = n[2] / m->V;
    if (!isfinite(creal(cT)) || !isfinite(creal(xhat)) || !isfinite(creal(P))) {
      *dphi = NAN;
      return NAN;
    }
    const cplx ez = cT - or_zbar(m, t_i);
    phi += ez * ez;
    if (i == K) break;
    const cplx y = cT + m->meas_sd * or_meas_noise(seed, j, i);
    if (i > 0) ekf_predict_c(m, EaR_c, c->n_rk4, F_prev, &xhat, &P);
    ekf_filter_c(m, y, &xhat, &P);
    for (int k = 1; k <= N; ++k) zb[k] = or_zbar(m, m->t0 + (double)(i + k) * m->Ts);
    or_sqp_info info;
    or_sqp(m, c, EaR_c, creal(xhat) / c->x_scale, zb, u, x, lam, pil, piu, &info);
    double S[4] = {0.0, 0.0, 0.0, 0.0};
    if (or_ocp_sens(m, c, EaR_c, creal(xhat) / c->x_scale, zb, u, x, lam, pil, piu, S) != 0) {
      S[0] = S[1] = S[2] = S[3] = 0.0;
      ++*n_sens_fail;
    }
    const double du_im = S[0] * cimag(xhat) / c->x_scale + S[1 + which] * h_cs;
    const cplx F = (u[0] + I * du_im) * Fconv;
    for (int k = 0; k < N - 1; ++k) {
      u[k] = u[k + 1];
      x[k + 1] = x[k + 2];
      lam[k] = lam[k + 1];
      pil[k] = pil[k + 1];
      piu[k] = piu[k + 1];
    }
    for (int s = 0; s < m->n_em; ++s) {
      const int64_t ks = (int64_t)i * m->n_em + s;
      const double tau = m->t0 + (double)ks * h;
      const double T_in = (m->dTin_step != 0.0 && tau >= t_d) ? m->T_in + dTin : m->T_in;
      double xi[3];
      or_process_noise(seed, j, ks, xi);
      cplx f[3];
      drift_c(m, EaR, T_in, n, F, f);
      for (int q = 0; q < 3; ++q) n[q] = n[q] + f[q] * h + F * m->sigma[q] * sq * xi[q];
    }
    F_prev = F;
  }
  phi = phi / (double)(K + 1);
  *dphi = cimag(phi) / h_cs;
  return creal(phi);
}

typedef struct {
  const or_model* m;
  const or_ctrl* c;
  uint64_t seed;
  int64_t j0, j1;
  int tid, nt;
  double *phi, *dphi;
  int* fails;
} njob_t;

static void* nworker(void* arg) {
  njob_t* g = (njob_t*)arg;
  const double gains[3] = {g->c->Qz, g->c->Ru, g->c->Qn};
  for (int64_t j = g->j0 + g->tid; j < g->j1; j += g->nt) {
    const int64_t r = j - g->j0;
    int f = 0, ft = 0;
    for (int q = 0; q < 3; ++q) {
      const double hq = 1e-20 * (gains[q] != 0.0 ? fabs(gains[q]) : 1.0);
      g->phi[r] = or_nmpc_phi_cs(g->m, g->c, g->seed, j, q, hq, &g->dphi[3 * r + q], &f);
      ft = f;
    }
    g->fails[r] = ft;
  }
  return NULL;
}

void or_nmpc_grad_run(const or_model* m, const or_ctrl* c, uint64_t seed, int64_t j0,
                      int64_t j1, int n_threads, double* phi, double* dphi, int* fails) {
  if (n_threads < 1) n_threads = 1;
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)n_threads);
  njob_t* jobs = (njob_t*)malloc(sizeof(njob_t) * (size_t)n_threads);
  for (int t = 0; t < n_threads; ++t) {
    jobs[t] = (njob_t){m, c, seed, j0, j1, t, n_threads, phi, dphi, fails};
    pthread_create(&th[t], NULL, nworker, &jobs[t]);
  }
  for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
  free(th);
  free(jobs);
}
