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
