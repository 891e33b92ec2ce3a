/*
 * or_model.c -- CSTR model, Euler-Maruyama, RK4 shooting with sensitivities
 * and the continuous-discrete EKF, in plain FP64.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 */
#include <math.h>
#include "oracle.h"

/* Drift of the three-state plant, Eq. (CSTR) of Sec. VI:
 *   dn/dt = C_in F - c F + S^T r(c) V,  c = n / V,
 *   r = k(c_T) c_A c_B,  k(c_T) = k0 exp(-(E_a/R) / c_T),  S = [-1, -2, beta].
 * T_in is passed separately so that an inlet-temperature disturbance can act
 * on the plant only.  F is the flow in L/s. */
void or_plant_drift(const or_model* m, double EaR, double T_in, const double n[3],
                    double F, double f[3]) {
  const double cA = n[0] / m->V;
  const double cB = n[1] / m->V;
  const double cT = n[2] / m->V;
  const double k = m->k0 * exp(-EaR / cT);
  const double r = k * cA * cB;
  f[0] = m->cA_in * F - cA * F + (-1.0) * r * m->V;
  f[1] = m->cB_in * F - cB * F + (-2.0) * r * m->V;
  f[2] = T_in * F - cT * F + m->beta * r * m->V;
}

/* One-state model used by the NMPC (Sec. VI): state x = n_T = c_T V.  The
 * paper leaves c_A and c_B of the rate law implicit; they follow from the two
 * reaction invariants of the three-state drift: beta c_A + c_T and
 * beta c_B + 2 c_T both relax to their feed values, so on the invariant
 * manifold c_A = c_A,in + (T_in - c_T)/beta and c_B = c_B,in + 2 (T_in - c_T)/beta.
 * Returns f, df/dx and df/dF. */
void or_model1(const or_model* m, double EaR, double x, double F, double* f,
               double* fx, double* fF) {
  const double cT = x / m->V;
  const double cA = m->cA_in + (m->T_in - cT) / m->beta;
  const double cB = m->cB_in + 2.0 * (m->T_in - cT) / m->beta;
  const double k = m->k0 * exp(-EaR / cT);
  const double r = k * cA * cB;
  *f = F * (m->T_in - cT) + m->beta * r * m->V;
  /* dr/dc_T by the product rule; dk/dc_T = k (E_a/R) / c_T^2 */
  const double dk = k * EaR / (cT * cT);
  const double dcA = -1.0 / m->beta;
  const double dcB = -2.0 / m->beta;
  const double dr = dk * cA * cB + k * dcA * cB + k * cA * dcB;
  *fx = (-F + m->beta * dr * m->V) / m->V;
  *fF = m->T_in - cT;
}

/* Piecewise-constant set-point z-bar(t), held beyond the last segment start. */
double or_zbar(const or_model* m, double t) {
  double z = m->sp_value[0];
  for (int s = 1; s < m->n_sp; ++s)
    if (t >= m->sp_time[s]) z = m->sp_value[s];
  return z;
}

/* Steady-state flow (L/s) of the one-state model at temperature Tbar:
 * 0 = F (T_in - Tbar) + beta r(Tbar) V  solved for F. */
double or_Fss(const or_model* m, double EaR, double Tbar) {
  const double cA = m->cA_in + (m->T_in - Tbar) / m->beta;
  const double cB = m->cB_in + 2.0 * (m->T_in - Tbar) / m->beta;
  const double r = m->k0 * exp(-EaR / Tbar) * cA * cB;
  return m->beta * r * m->V / (Tbar - m->T_in);
}

/* One Euler-Maruyama substep of Eq. (CDS) for the plant:
 *   n <- n + f(n, F) h + F sigma-bar sqrt(h) xi,  xi ~ N(0, I). */
void or_em_step(const or_model* m, double EaR, double T_in, double n[3], double F,
                double h, const double xi[3]) {
  double f[3];
  or_plant_drift(m, EaR, T_in, n, F, f);
  const double sq = sqrt(h);
  for (int i = 0; i < 3; ++i) n[i] = n[i] + f[i] * h + F * m->sigma[i] * sq * xi[i];
}

/* F(x0, v) over one control interval Ts with n_rk4 classical RK4 steps
 * (Sec. VII-A, N_c), and its sensitivities A = dF/dx0, B = dF/dv obtained by
 * differentiating every RK4 stage (forward mode).  The input variable v is in
 * OCP units; the flow is F = v * Fconv (L/s). */
void or_rk4_interval(const or_model* m, double EaR, int n_rk4, double Ts, double x0,
                     double v, double Fconv, double* xF, double* A, double* B) {
  const double h = Ts / (double)n_rk4;
  const double F = v * Fconv;
  double x = x0, a = 1.0, b = 0.0;
  for (int s = 0; s < n_rk4; ++s) {
    double f1, fx1, fF1, f2, fx2, fF2, f3, fx3, fF3, f4, fx4, fF4;
    or_model1(m, EaR, x, F, &f1, &fx1, &fF1);
    const double a1 = fx1 * a, b1 = fx1 * b + fF1 * Fconv;
    const double x2 = x + 0.5 * h * f1;
    const double a2s = a + 0.5 * h * a1, b2s = b + 0.5 * h * b1;
    or_model1(m, EaR, x2, F, &f2, &fx2, &fF2);
    const double a2 = fx2 * a2s, b2 = fx2 * b2s + fF2 * Fconv;
    const double x3 = x + 0.5 * h * f2;
    const double a3s = a + 0.5 * h * a2, b3s = b + 0.5 * h * b2;
    or_model1(m, EaR, x3, F, &f3, &fx3, &fF3);
    const double a3 = fx3 * a3s, b3 = fx3 * b3s + fF3 * Fconv;
    const double x4 = x + h * f3;
    const double a4s = a + h * a3, b4s = b + h * b3;
    or_model1(m, EaR, x4, F, &f4, &fx4, &fF4);
    const double a4 = fx4 * a4s, b4 = fx4 * b4s + fF4 * Fconv;
    x = x + h / 6.0 * (f1 + 2.0 * f2 + 2.0 * f3 + f4);
    a = a + h / 6.0 * (a1 + 2.0 * a2 + 2.0 * a3 + a4);
    b = b + h / 6.0 * (b1 + 2.0 * b2 + 2.0 * b3 + b4);
  }
  *xF = x;
  if (A) *A = a;
  if (B) *B = b;
}

/* CD-EKF prediction, Eq. (predictionEquations): integrate
 *   dx/dt = f(x, F),  dP/dt = A P + P A^T + sigma sigma^T,
 * with A = df/dx along x(t) and sigma = F sigma_T for the one-state model,
 * over one sample time by n_rk4 classical RK4 steps of the joint system. */
void or_ekf_predict(const or_model* m, double EaR, int n_rk4, double F, double* x,
                    double* P) {
  const double h = m->Ts / (double)n_rk4;
  const double q = (F * m->sigma[2]) * (F * m->sigma[2]);
  double xs = *x, Ps = *P;
  for (int s = 0; s < n_rk4; ++s) {
    double f1, A1, f2, A2, f3, A3, f4, A4, dummy;
    or_model1(m, EaR, xs, F, &f1, &A1, &dummy);
    const double p1 = 2.0 * A1 * Ps + q;
    or_model1(m, EaR, xs + 0.5 * h * f1, F, &f2, &A2, &dummy);
    const double p2 = 2.0 * A2 * (Ps + 0.5 * h * p1) + q;
    or_model1(m, EaR, xs + 0.5 * h * f2, F, &f3, &A3, &dummy);
    const double p3 = 2.0 * A3 * (Ps + 0.5 * h * p2) + q;
    or_model1(m, EaR, xs + h * f3, F, &f4, &A4, &dummy);
    const double p4 = 2.0 * A4 * (Ps + h * p3) + q;
    xs = xs + h / 6.0 * (f1 + 2.0 * f2 + 2.0 * f3 + f4);
    Ps = Ps + h / 6.0 * (p1 + 2.0 * p2 + 2.0 * p3 + p4);
  }
  *x = xs;
  *P = Ps;
}

/* CD-EKF filtering (Sec. III-A): y-hat = g(x) = x / V, C = 1/V,
 * e = y - y-hat, R_e = R + C P C^T, K = P C^T / R_e, x += K e, and the
 * covariance in the Joseph form (Josph).  P_short returns the short form
 * P - K R_e K^T for comparison. */
void or_ekf_filter(const or_model* m, double y, double* x, double* P, double* P_short) {
  const double R = m->meas_sd * m->meas_sd;
  const double C = 1.0 / m->V;
  const double yhat = *x / m->V;
  const double e = y - yhat;
  const double Re = R + C * (*P) * C;
  const double K = (*P) * C / Re;
  const double ImKC = 1.0 - K * C;
  const double Pj = ImKC * (*P) * ImKC + K * R * K;
  if (P_short) *P_short = *P - K * Re * K;
  *x = *x + K * e;
  *P = Pj;
}
