/*
 * or_nmpc3.c -- the NMPC with the three-state model of Eq. (CSTR) (Sec. VI
 * gives it; the paper's controller uses the one-state reduction): CD-EKF on
 * n = (n_A, n_B, n_T) with a 3x3 covariance, and the multiple-shooting OCP
 * with three states and one input per stage, solved by the same SQP as
 * or_sqp.c (QP subproblem, l1-merit backtracking, damped block BFGS, scaled
 * convergence test), in plain FP64.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Notation: NX = 3 states, one input.  Decision vector
 * xi = [u_0, x_1, u_1, ..., u_{N-1}, x_N] with x_k in R^3 the scaled state
 * n / x_scale; constraints g_k = F_k - x_{k+1} in R^3; Lagrangian
 *   L = f - sum_k lam_k^T g_k - pil^T (u - u_min) - piu^T (u_max - u).
 * The objective is that of Sec. VII-A on the temperature component,
 *   f = sum_{k=1..N} Q_z (z_k - zbar_k)^2 T_s,  z_k = x_k[2] x_scale / V.
 */
#include <math.h>
#include <string.h>
#include "oracle.h"

#define NX 3
#define NB 4   /* variables of a stage block: x (3) and u */

/* ------------------------------------------------------------------ model */

/* Drift f(n, F) of Eq. (CSTR) with inlet temperature T_in, its Jacobian
 * J = df/dn (row-major 3x3) and df/dF. */
void or_drift3(const or_model* m, double EaR, double T_in, const double n[3], double F,
               double f[3], double J[9], double fF[3]) {
  const double V = m->V;
  const double cA = n[0] / V, cB = n[1] / V, cT = n[2] / V;
  const double k = m->k0 * exp(-EaR / cT);
  const double rV = k * cA * cB * V;
  const double S[3] = {-1.0, -2.0, m->beta};
  const double cin[3] = {m->cA_in, m->cB_in, T_in};
  const double c[3] = {cA, cB, cT};
  /* d(rV)/dn: k c_B, k c_A, rV (E_a/R) / c_T^2 / V */
  const double drv[3] = {k * cB, k * cA, rV * EaR / (cT * cT) / V};
  for (int p = 0; p < 3; ++p) {
    f[p] = cin[p] * F - c[p] * F + S[p] * rV;
    fF[p] = cin[p] - c[p];
    for (int q = 0; q < 3; ++q) J[p * 3 + q] = (p == q ? -F / V : 0.0) + S[p] * drv[q];
  }
}

/* F(x0, v) over T_s by n_rk4 classical RK4 steps of the drift (nominal T_in),
 * and its sensitivities A = dF/dx0 (3x3) and B = dF/dv (3), obtained by
 * applying the same RK4 steps to the variational equations
 * Phi' = J Phi, psi' = J psi + f_F Fconv.  States in moles; v in OCP units. */
void or_rk4_interval3(const or_model* m, double EaR, int n_rk4, double Ts, const double x0[3],
                      double v, double Fconv, double xF[3], double A[9], double B[3]) {
  const double h = Ts / (double)n_rk4;
  const double F = v * Fconv;
  double x[3], Phi[9], psi[3];
  for (int i = 0; i < 3; ++i) {
    x[i] = x0[i];
    psi[i] = 0.0;
    for (int j = 0; j < 3; ++j) Phi[i * 3 + j] = (i == j) ? 1.0 : 0.0;
  }
  for (int s = 0; s < n_rk4; ++s) {
    double kx[4][3], kP[4][9], kp[4][3];
    double xs[3], Ps[9], ps[3];
    for (int st = 0; st < 4; ++st) {
      const double a = (st == 0) ? 0.0 : ((st == 3) ? h : 0.5 * h);
      for (int i = 0; i < 3; ++i) {
        xs[i] = x[i] + (st ? a * kx[st - 1][i] : 0.0);
        ps[i] = psi[i] + (st ? a * kp[st - 1][i] : 0.0);
        for (int j = 0; j < 3; ++j)
          Ps[i * 3 + j] = Phi[i * 3 + j] + (st ? a * kP[st - 1][i * 3 + j] : 0.0);
      }
      double f[3], J[9], fF[3];
      or_drift3(m, EaR, m->T_in, xs, F, f, J, fF);
      for (int i = 0; i < 3; ++i) {
        kx[st][i] = f[i];
        double sp = fF[i] * Fconv;
        for (int q = 0; q < 3; ++q) sp += J[i * 3 + q] * ps[q];
        kp[st][i] = sp;
        for (int j = 0; j < 3; ++j) {
          double sP = 0.0;
          for (int q = 0; q < 3; ++q) sP += J[i * 3 + q] * Ps[q * 3 + j];
          kP[st][i * 3 + j] = sP;
        }
      }
    }
    for (int i = 0; i < 3; ++i) {
      x[i] = x[i] + h / 6.0 * (kx[0][i] + 2.0 * kx[1][i] + 2.0 * kx[2][i] + kx[3][i]);
      psi[i] = psi[i] + h / 6.0 * (kp[0][i] + 2.0 * kp[1][i] + 2.0 * kp[2][i] + kp[3][i]);
      for (int j = 0; j < 3; ++j)
        Phi[i * 3 + j] = Phi[i * 3 + j] + h / 6.0 * (kP[0][i * 3 + j] + 2.0 * kP[1][i * 3 + j] +
                                                     2.0 * kP[2][i * 3 + j] + kP[3][i * 3 + j]);
    }
  }
  for (int i = 0; i < 3; ++i) {
    xF[i] = x[i];
    B[i] = psi[i];
    for (int j = 0; j < 3; ++j) A[i * 3 + j] = Phi[i * 3 + j];
  }
}

/* ------------------------------------------------------------------ CD-EKF */

/* Prediction over one sample, Eq. (predictionEquations) for three states:
 * RK4 (n_rk4 steps) on x' = f(x, F), P' = J P + P J^T + F^2 diag(sigma^2),
 * with the nominal T_in.  P is row-major 3x3, kept symmetric. */
void or_ekf3_predict(const or_model* m, double EaR, int n_rk4, double F, double x[3],
                     double P[9]) {
  const double h = m->Ts / (double)n_rk4;
  double Qc[9] = {0};
  for (int i = 0; i < 3; ++i) Qc[i * 3 + i] = F * F * m->sigma[i] * m->sigma[i];
  for (int s = 0; s < n_rk4; ++s) {
    double kx[4][3], kP[4][9];
    for (int st = 0; st < 4; ++st) {
      const double a = (st == 0) ? 0.0 : ((st == 3) ? h : 0.5 * h);
      double xs[3], Ps[9];
      for (int i = 0; i < 3; ++i) xs[i] = x[i] + (st ? a * kx[st - 1][i] : 0.0);
      for (int i = 0; i < 9; ++i) Ps[i] = P[i] + (st ? a * kP[st - 1][i] : 0.0);
      double f[3], J[9], fF[3];
      or_drift3(m, EaR, m->T_in, xs, F, f, J, fF);
      for (int i = 0; i < 3; ++i) {
        kx[st][i] = f[i];
        for (int j = 0; j < 3; ++j) {
          double s1 = 0.0, s2 = 0.0;
          for (int q = 0; q < 3; ++q) {
            s1 += J[i * 3 + q] * Ps[q * 3 + j];
            s2 += Ps[i * 3 + q] * J[j * 3 + q];
          }
          kP[st][i * 3 + j] = s1 + s2 + Qc[i * 3 + j];
        }
      }
    }
    for (int i = 0; i < 3; ++i)
      x[i] = x[i] + h / 6.0 * (kx[0][i] + 2.0 * kx[1][i] + 2.0 * kx[2][i] + kx[3][i]);
    for (int i = 0; i < 9; ++i)
      P[i] = P[i] + h / 6.0 * (kP[0][i] + 2.0 * kP[1][i] + 2.0 * kP[2][i] + kP[3][i]);
  }
}

/* Filtering, Eq. (Josph), with the output c_T = n_T / V: C = [0, 0, 1/V].
 * K = P C^T / (C P C^T + R), x += K (y - C x),
 * P = (I - K C) P (I - K C)^T + K R K^T.  Optionally the short form
 * (I - K C) P for comparison. */
void or_ekf3_filter(const or_model* m, double y, double x[3], double P[9], double* P_short) {
  const double R = m->meas_sd * m->meas_sd;
  const double C[3] = {0.0, 0.0, 1.0 / m->V};
  double PC[3];
  for (int i = 0; i < 3; ++i) PC[i] = P[i * 3 + 0] * C[0] + P[i * 3 + 1] * C[1] + P[i * 3 + 2] * C[2];
  const double Re = R + C[0] * PC[0] + C[1] * PC[1] + C[2] * PC[2];
  double K[3];
  for (int i = 0; i < 3; ++i) K[i] = PC[i] / Re;
  const double e = y - (C[0] * x[0] + C[1] * x[1] + C[2] * x[2]);
  for (int i = 0; i < 3; ++i) x[i] = x[i] + K[i] * e;
  double M[9], MP[9], Pn[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) M[i * 3 + j] = (i == j ? 1.0 : 0.0) - K[i] * C[j];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int q = 0; q < 3; ++q) s += M[i * 3 + q] * P[q * 3 + j];
      MP[i * 3 + j] = s;
    }
  if (P_short) memcpy(P_short, MP, sizeof(MP));
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int q = 0; q < 3; ++q) s += MP[i * 3 + q] * M[j * 3 + q];
      Pn[i * 3 + j] = s + K[i] * R * K[j];
    }
  memcpy(P, Pn, sizeof(Pn));
}

/* --------------------------------------------------------- QP subproblem */

/* Dense Cholesky (row-major, leading dimension ld); 0 or -1 (pivot <= 0). */
static int chol3(int n, double* a, int ld) {
  for (int j = 0; j < n; ++j) {
    double d = a[j * ld + j];
    for (int k = 0; k < j; ++k) d -= a[j * ld + k] * a[j * ld + k];
    if (!(d > 0.0)) return -1;
    d = sqrt(d);
    a[j * ld + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double s = a[i * ld + j];
      for (int k = 0; k < j; ++k) s -= a[i * ld + k] * a[j * ld + k];
      a[i * ld + j] = s / d;
    }
  }
  return 0;
}

static void chol3_solve(int n, const double* l, int ld, double* z) {
  for (int i = 0; i < n; ++i) {
    double s = z[i];
    for (int k = 0; k < i; ++k) s -= l[i * ld + k] * z[k];
    z[i] = s / l[i * ld + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = z[i];
    for (int k = i + 1; k < n; ++k) s -= l[k * ld + i] * z[k];
    z[i] = s / l[i * ld + i];
  }
}

/*
 * QP subproblem for three states and one input per stage:
 *   min  sum_k 1/2 [dx_k; du_k]^T W_k [dx_k; du_k] + q_k^T dx_k + r_k du_k
 *   s.t. dx_{k+1} = A_k dx_k + B_k du_k + b_k, dx_0 = 0, lb_k <= du_k <= ub_k.
 * Arrays: A (N x 9), B, b (N x 3), Wxx ((N+1) x 9), Wxu ((N+1) x 3),
 * Wuu (N+1), q ((N+1) x 3), r, lb, ub (N); outputs du (N), dx ((N+1) x 3),
 * mu (N x 3), nul, nuu (N).  W_0 uses only Wuu[0], W_N only Wxx[N].
 *
 * Method: condense dx_k = G_k du + c_k (G_k 3 x N) into a dense box QP in du
 * and solve it by the primal active-set method of or_qp_solve (start at
 * du = 0 with the bounds active there in the working set, cut a step at the
 * first blocking bound, release the most negative multiplier); then dx from
 * the dynamics, mu from stationarity in dx (backwards), and the bound
 * multipliers from stationarity in du.  0, -1 (not positive definite) or -2.
 */
int or_qp3_solve(int N, const double* A, const double* B, const double* b, const double* Wxx,
                 const double* Wxu, const double* Wuu, const double* q, const double* r,
                 const double* lb, const double* ub, double* du, double* dx, double* mu,
                 double* nul, double* nuu, int* iters) {
  enum { FREE = 0, LOWER = 1, UPPER = 2 };
  static __thread double G[OR_MAX_N + 1][3][OR_MAX_N];
  double c[OR_MAX_N + 1][3];
  static __thread double H[OR_MAX_N * OR_MAX_N], L[OR_MAX_N * OR_MAX_N];
  double h[OR_MAX_N];
  int ws[OR_MAX_N];
  for (int i = 0; i < 3; ++i) {
    c[0][i] = 0.0;
    for (int j = 0; j < N; ++j) G[0][i][j] = 0.0;
  }
  for (int k = 0; k < N; ++k) {
    for (int i = 0; i < 3; ++i) {
      double cs = b[k * 3 + i];
      for (int q2 = 0; q2 < 3; ++q2) cs += (k == 0 ? 0.0 : A[k * 9 + i * 3 + q2]) * c[k][q2];
      c[k + 1][i] = cs;
      for (int j = 0; j < N; ++j) {
        double s = 0.0;
        for (int q2 = 0; q2 < 3; ++q2) s += (k == 0 ? 0.0 : A[k * 9 + i * 3 + q2]) * G[k][q2][j];
        G[k + 1][i][j] = s;
      }
      G[k + 1][i][k] += B[k * 3 + i];
    }
  }
  /* H = sum_k G_k^T Wxx_k G_k + diag(Wuu) + cross terms; h likewise */
  for (int i = 0; i < N; ++i) {
    for (int j = 0; j < N; ++j) {
      double s = (i == j) ? Wuu[i] : 0.0;
      for (int k = 1; k <= N; ++k)
        for (int a = 0; a < 3; ++a)
          for (int bb = 0; bb < 3; ++bb) s += G[k][a][i] * Wxx[k * 9 + a * 3 + bb] * G[k][bb][j];
      if (j >= 1 && j <= N - 1)
        for (int a = 0; a < 3; ++a) s += Wxu[j * 3 + a] * G[j][a][i];
      if (i >= 1 && i <= N - 1)
        for (int a = 0; a < 3; ++a) s += Wxu[i * 3 + a] * G[i][a][j];
      H[i * N + j] = s;
    }
    double s = r[i];
    for (int k = 1; k <= N; ++k)
      for (int a = 0; a < 3; ++a) {
        double wc = q[k * 3 + a];
        for (int bb = 0; bb < 3; ++bb) wc += Wxx[k * 9 + a * 3 + bb] * c[k][bb];
        s += G[k][a][i] * wc;
      }
    if (i >= 1 && i <= N - 1)
      for (int a = 0; a < 3; ++a) s += Wxu[i * 3 + a] * c[i][a];
    h[i] = s;
  }

  double hscale = 1.0;
  for (int i = 0; i < N; ++i) hscale = fmax(hscale, fabs(h[i]));
  const double mult_tol = 1e-13 * hscale;
  for (int i = 0; i < N; ++i) {
    du[i] = 0.0;
    ws[i] = (lb[i] >= 0.0) ? LOWER : ((ub[i] <= 0.0) ? UPPER : FREE);
    if (ws[i] == LOWER) du[i] = lb[i];
    if (ws[i] == UPPER) du[i] = ub[i];
  }
  int it = 0, status = -2;
  const int max_it = 10 * N + 20;
  for (; it < max_it; ++it) {
    int idx[OR_MAX_N], nf = 0;
    for (int i = 0; i < N; ++i)
      if (ws[i] == FREE) idx[nf++] = i;
    double z[OR_MAX_N];
    for (int a = 0; a < nf; ++a) {
      const int i = idx[a];
      double s = h[i];
      for (int j = 0; j < N; ++j)
        if (ws[j] != FREE) s += H[i * N + j] * du[j];
      z[a] = -s;
      for (int bb = 0; bb < nf; ++bb) L[a * OR_MAX_N + bb] = H[i * N + idx[bb]];
    }
    if (nf > 0) {
      if (chol3(nf, L, OR_MAX_N) != 0) {
        status = -1;
        break;
      }
      chol3_solve(nf, L, OR_MAX_N, z);
    }
    double alpha = 1.0;
    int block = -1, side = FREE;
    for (int a = 0; a < nf; ++a) {
      const int i = idx[a];
      const double p = z[a] - du[i];
      if (p < 0.0 && z[a] < lb[i]) {
        const double t = (lb[i] - du[i]) / p;
        if (t < alpha) { alpha = t; block = i; side = LOWER; }
      } else if (p > 0.0 && z[a] > ub[i]) {
        const double t = (ub[i] - du[i]) / p;
        if (t < alpha) { alpha = t; block = i; side = UPPER; }
      }
    }
    if (block >= 0) {
      if (alpha < 0.0) alpha = 0.0;
      for (int a = 0; a < nf; ++a) du[idx[a]] = du[idx[a]] + alpha * (z[a] - du[idx[a]]);
      ws[block] = side;
      du[block] = (side == LOWER) ? lb[block] : ub[block];
      continue;
    }
    for (int a = 0; a < nf; ++a) du[idx[a]] = z[a];
    int worst = -1;
    double worst_val = -mult_tol;
    for (int i = 0; i < N; ++i) {
      if (ws[i] == FREE) continue;
      double gi = h[i];
      for (int j = 0; j < N; ++j) gi += H[i * N + j] * du[j];
      const double lam = (ws[i] == LOWER) ? gi : -gi;
      if (lam < worst_val) { worst_val = lam; worst = i; }
    }
    if (worst < 0) {
      status = 0;
      ++it;
      break;
    }
    ws[worst] = FREE;
  }
  if (iters) *iters = it;

  for (int i = 0; i < 3; ++i) dx[i] = 0.0;
  for (int k = 0; k < N; ++k)
    for (int i = 0; i < 3; ++i) {
      double s = B[k * 3 + i] * du[k] + b[k * 3 + i];
      for (int q2 = 0; q2 < 3; ++q2) s += (k == 0 ? 0.0 : A[k * 9 + i * 3 + q2]) * dx[k * 3 + q2];
      dx[(k + 1) * 3 + i] = s;
    }
  /* mu_{N-1} = -(Wxx_N dx_N + q_N);
   * mu_{k-1} = A_k^T mu_k - (Wxx_k dx_k + Wxu_k du_k + q_k), k = N-1..1 */
  for (int i = 0; i < 3; ++i) {
    double s = q[N * 3 + i];
    for (int bb = 0; bb < 3; ++bb) s += Wxx[N * 9 + i * 3 + bb] * dx[N * 3 + bb];
    mu[(N - 1) * 3 + i] = -s;
  }
  for (int k = N - 1; k >= 1; --k)
    for (int i = 0; i < 3; ++i) {
      double s = 0.0;
      for (int a = 0; a < 3; ++a) s += A[k * 9 + a * 3 + i] * mu[k * 3 + a];
      double w = q[k * 3 + i] + Wxu[k * 3 + i] * du[k];
      for (int bb = 0; bb < 3; ++bb) w += Wxx[k * 9 + i * 3 + bb] * dx[k * 3 + bb];
      mu[(k - 1) * 3 + i] = s - w;
    }
  /* Wuu_k du_k + Wxu_k^T dx_k + r_k - mu_k^T B_k - nul_k + nuu_k = 0 */
  for (int k = 0; k < N; ++k) {
    double v = Wuu[k] * du[k] + r[k];
    for (int a = 0; a < 3; ++a) {
      if (k >= 1) v += Wxu[k * 3 + a] * dx[k * 3 + a];
      v -= mu[k * 3 + a] * B[k * 3 + a];
    }
    nul[k] = (ws[k] == LOWER) ? v : 0.0;
    nuu[k] = (ws[k] == UPPER) ? -v : 0.0;
  }
  return status;
}

/* ------------------------------------------------------------------ SQP */

/* Damped BFGS update (Sec. IV-C) of one symmetric n x n block (row-major,
 * n <= 4): theta-damped secant r = theta y + (1 - theta) W s, skipped when
 * min(s^T W s, s^T r) <= eps_m. */
void or_bfgs_blockn(int n, double* W, const double* s, const double* y) {
  const double eps_m = 2.220446049250313e-16;
  double Ws[NB], rr[NB];
  double sWs = 0.0, sy = 0.0, sr = 0.0;
  for (int i = 0; i < n; ++i) {
    double t = 0.0;
    for (int j = 0; j < n; ++j) t += W[i * n + j] * s[j];
    Ws[i] = t;
    sWs += s[i] * t;
    sy += s[i] * y[i];
  }
  const double theta = (sy >= 0.2 * sWs) ? 1.0 : (0.8 * sWs) / (sWs - sy);
  for (int i = 0; i < n; ++i) {
    rr[i] = theta * y[i] + (1.0 - theta) * Ws[i];
    sr += s[i] * rr[i];
  }
  if (!(fmin(sWs, sr) > eps_m)) return;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) W[i * n + j] = W[i * n + j] - Ws[i] * Ws[j] / sWs + rr[i] * rr[j] / sr;
}

static int block_pd_n(int n, const double* W) {
  double a[NB * NB];
  memcpy(a, W, sizeof(double) * (size_t)(n * n));
  return chol3(n, a, n) == 0;
}

typedef struct {
  double F[OR_MAX_N][3], A[OR_MAX_N][9], B[OR_MAX_N][3], g[OR_MAX_N][3];
  double q[OR_MAX_N + 1][3], r[OR_MAX_N];
  double f;
} eval3_t;

static void evaluate3(const or_model* m, const or_ctrl* c, double EaR, double Fconv,
                      const double x0[3], const double* zbar, const double* u,
                      const double* x, eval3_t* e) {
  const int N = c->N;
  const double xs = c->x_scale;
  for (int k = 0; k < N; ++k) {
    double n0[3], Fn[3], Ak[9], Bk[3];
    for (int i = 0; i < 3; ++i) n0[i] = ((k == 0) ? x0[i] : x[k * 3 + i]) * xs;
    or_rk4_interval3(m, EaR, c->n_rk4, m->Ts, n0, u[k], Fconv, Fn, Ak, Bk);
    for (int i = 0; i < 3; ++i) {
      e->F[k][i] = Fn[i] / xs;
      e->B[k][i] = Bk[i] / xs;
      e->g[k][i] = e->F[k][i] - x[(k + 1) * 3 + i];
    }
    for (int i = 0; i < 9; ++i) e->A[k][i] = Ak[i];
    e->r[k] = 0.0;
  }
  double f = 0.0;
  for (int i = 0; i < 3; ++i) e->q[0][i] = 0.0;
  for (int k = 1; k <= N; ++k) {
    const double dz = x[k * 3 + 2] * xs / m->V - zbar[k];
    f += c->Qz * dz * dz * m->Ts;
    e->q[k][0] = 0.0;
    e->q[k][1] = 0.0;
    e->q[k][2] = 2.0 * c->Qz * dz * m->Ts * xs / m->V;
  }
  e->f = f;
}

/* d/du_k L = r_k - lam_k^T B_k - pil_k + piu_k;
 * d/dx_k L = q_k - A_k^T lam_k + lam_{k-1} (k = 1..N-1); d/dx_N L = q_N + lam_{N-1} */
static void grad_lagrangian3(int N, const eval3_t* e, const double* lam, const double* pil,
                             const double* piu, double* gu, double* gx) {
  for (int k = 0; k < N; ++k) {
    double s = e->r[k] - pil[k] + piu[k];
    for (int i = 0; i < 3; ++i) s -= lam[k * 3 + i] * e->B[k][i];
    gu[k] = s;
  }
  for (int i = 0; i < 3; ++i) gx[i] = 0.0;
  for (int k = 1; k < N; ++k)
    for (int i = 0; i < 3; ++i) {
      double s = e->q[k][i] + lam[(k - 1) * 3 + i];
      for (int a = 0; a < 3; ++a) s -= e->A[k][a * 3 + i] * lam[k * 3 + a];
      gx[k * 3 + i] = s;
    }
  for (int i = 0; i < 3; ++i) gx[N * 3 + i] = e->q[N][i] + lam[(N - 1) * 3 + i];
}

/* The SQP of or_sqp for three states.  Blocks: W_0 = [u_0] (1x1),
 * W_k = [x_k; u_k] (4x4, k = 1..N-1), W_N = [x_N] (3x3).  x0 and x are
 * scaled states (x has (N+1) x 3 entries, row 0 = x0); lam (N x 3). */
int or_sqp3(const or_model* m, const or_ctrl* c, double EaR, const double x0[3],
            const double* zbar, double* u, double* x, double* lam, double* pil, double* piu,
            or_sqp_info* info) {
  const int N = c->N;
  const double Fconv = c->u_scale / 60000.0;
  const double umin = c->u_min / c->u_scale, umax = c->u_max / c->u_scale;
  const double c1 = 1e-4, beta_ls = 0.5, s_max = 100.0;
  static __thread double W0, Wk[OR_MAX_N][NB * NB], WN[9];
  static __thread eval3_t ev, evt;
  double du[OR_MAX_N], dx[(OR_MAX_N + 1) * 3], mu[OR_MAX_N * 3], nul[OR_MAX_N], nuu[OR_MAX_N];
  double sigma[OR_MAX_N * 3];
  double gu[OR_MAX_N], gx[(OR_MAX_N + 1) * 3], gu_old[OR_MAX_N], gx_old[(OR_MAX_N + 1) * 3];
  double s_u[OR_MAX_N], s_x[(OR_MAX_N + 1) * 3];
  double ut[OR_MAX_N], xt[(OR_MAX_N + 1) * 3];
  static __thread double Aq[OR_MAX_N * 9], Bq[OR_MAX_N * 3], bq[OR_MAX_N * 3];
  static __thread double Wxx[(OR_MAX_N + 1) * 9], Wxu[(OR_MAX_N + 1) * 3], Wuu[OR_MAX_N + 1];
  static __thread double qq[(OR_MAX_N + 1) * 3];
  double lb[OR_MAX_N], ub[OR_MAX_N];

  W0 = 1.0;
  for (int k = 1; k < N; ++k)
    for (int i = 0; i < NB * NB; ++i) Wk[k][i] = (i % (NB + 1) == 0) ? 1.0 : 0.0;
  for (int i = 0; i < 9; ++i) WN[i] = (i % 4 == 0) ? 1.0 : 0.0;
  memset(info, 0, sizeof(*info));
  for (int i = 0; i < 3; ++i) x[i] = x0[i];
  evaluate3(m, c, EaR, Fconv, x0, zbar, u, x, &ev);

  int l = 0, nqp = 0;
  for (;; ++l) {
    if (l > 0) {
      grad_lagrangian3(N, &ev, lam, pil, piu, gu, gx);
      double s4[NB], y4[NB];
      s4[0] = s_u[0];
      y4[0] = gu[0] - gu_old[0];
      or_bfgs_blockn(1, &W0, s4, y4);
      for (int k = 1; k < N; ++k) {
        for (int i = 0; i < 3; ++i) {
          s4[i] = s_x[k * 3 + i];
          y4[i] = gx[k * 3 + i] - gx_old[k * 3 + i];
        }
        s4[3] = s_u[k];
        y4[3] = gu[k] - gu_old[k];
        or_bfgs_blockn(NB, Wk[k], s4, y4);
      }
      for (int i = 0; i < 3; ++i) {
        s4[i] = s_x[N * 3 + i];
        y4[i] = gx[N * 3 + i] - gx_old[N * 3 + i];
      }
      or_bfgs_blockn(3, WN, s4, y4);
      int pd = (W0 > 0.0) && block_pd_n(3, WN);
      for (int k = 1; k < N; ++k) pd = pd && block_pd_n(NB, Wk[k]);
      if (!pd) {
        W0 = 1.0;
        for (int k = 1; k < N; ++k)
          for (int i = 0; i < NB * NB; ++i) Wk[k][i] = (i % (NB + 1) == 0) ? 1.0 : 0.0;
        for (int i = 0; i < 9; ++i) WN[i] = (i % 4 == 0) ? 1.0 : 0.0;
        info->n_hess_reset++;
      }
    }

    grad_lagrangian3(N, &ev, lam, pil, piu, gu, gx);
    double mult1 = 0.0;
    for (int k = 0; k < N; ++k) {
      mult1 += fabs(pil[k]) + fabs(piu[k]);
      for (int i = 0; i < 3; ++i) mult1 += fabs(lam[k * 3 + i]);
    }
    const double s_d = fmax(s_max, mult1 / (double)(5 * N)) / s_max;
    double kg = 0.0, ke = 0.0;
    for (int k = 0; k < N; ++k) kg = fmax(kg, fabs(gu[k]));
    for (int k = 1; k <= N; ++k)
      for (int i = 0; i < 3; ++i) kg = fmax(kg, fabs(gx[k * 3 + i]));
    kg /= s_d;
    for (int k = 0; k < N; ++k)
      for (int i = 0; i < 3; ++i) ke = fmax(ke, fabs(ev.g[k][i]));
    info->kkt_grad = kg;
    info->kkt_eq = ke;
    info->f = ev.f;
    if (kg <= c->sqp_tol && ke <= c->sqp_tol) {
      info->status = 0;
      break;
    }
    if (l >= c->sqp_max_it) {
      info->status = 1;
      break;
    }

    /* QP at xi^[l] */
    for (int k = 0; k <= N; ++k) {
      for (int i = 0; i < 9; ++i) Wxx[k * 9 + i] = 0.0;
      for (int i = 0; i < 3; ++i) Wxu[k * 3 + i] = 0.0;
      Wuu[k] = 0.0;
      for (int i = 0; i < 3; ++i) qq[k * 3 + i] = ev.q[k][i];
    }
    Wuu[0] = W0;
    for (int k = 1; k < N; ++k) {
      for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) Wxx[k * 9 + i * 3 + j] = Wk[k][i * NB + j];
        Wxu[k * 3 + i] = Wk[k][i * NB + 3];
      }
      Wuu[k] = Wk[k][3 * NB + 3];
    }
    for (int i = 0; i < 9; ++i) Wxx[N * 9 + i] = WN[i];
    for (int k = 0; k < N; ++k) {
      for (int i = 0; i < 9; ++i) Aq[k * 9 + i] = ev.A[k][i];
      for (int i = 0; i < 3; ++i) {
        Bq[k * 3 + i] = ev.B[k][i];
        bq[k * 3 + i] = ev.g[k][i];
      }
      lb[k] = umin - u[k];
      ub[k] = umax - u[k];
    }
    int qp_it = 0;
    or_qp3_solve(N, Aq, Bq, bq, Wxx, Wxu, Wuu, qq, ev.r, lb, ub, du, dx, mu, nul, nuu, &qp_it);
    info->qp_iters += qp_it;
    ++nqp;

    for (int k = 0; k < N * 3; ++k)
      sigma[k] = (l == 0) ? fabs(mu[k]) : fmax(fabs(mu[k]), 0.5 * (sigma[k] + fabs(mu[k])));
    double pen = 0.0, dfd = 0.0;
    for (int k = 0; k < N; ++k)
      for (int i = 0; i < 3; ++i) pen += sigma[k * 3 + i] * fabs(ev.g[k][i]);
    for (int k = 0; k < N; ++k) dfd += ev.r[k] * du[k];
    for (int k = 1; k <= N; ++k)
      for (int i = 0; i < 3; ++i) dfd += ev.q[k][i] * dx[k * 3 + i];
    const double T0 = ev.f + pen;
    const double DT0 = dfd - pen;

    double alpha = 1.0;
    int accepted = 0;
    for (int hv = 0; hv <= c->ls_max; ++hv) {
      for (int i = 0; i < 3; ++i) xt[i] = x0[i];
      for (int k = 0; k < N; ++k) {
        ut[k] = fmin(fmax(u[k] + alpha * du[k], umin), umax);
        for (int i = 0; i < 3; ++i) xt[(k + 1) * 3 + i] = x[(k + 1) * 3 + i] + alpha * dx[(k + 1) * 3 + i];
      }
      evaluate3(m, c, EaR, Fconv, x0, zbar, ut, xt, &evt);
      info->ls_trials++;
      double pt = 0.0;
      for (int k = 0; k < N; ++k)
        for (int i = 0; i < 3; ++i) pt += sigma[k * 3 + i] * fabs(evt.g[k][i]);
      if (evt.f + pt <= T0 + c1 * alpha * DT0) {
        accepted = 1;
        break;
      }
      alpha *= beta_ls;
    }
    if (!accepted) {
      info->status = 2;
      break;
    }
    for (int k = 0; k < N; ++k) {
      for (int i = 0; i < 3; ++i) lam[k * 3 + i] = lam[k * 3 + i] + alpha * (mu[k * 3 + i] - lam[k * 3 + i]);
      pil[k] = pil[k] + alpha * (nul[k] - pil[k]);
      piu[k] = piu[k] + alpha * (nuu[k] - piu[k]);
    }
    grad_lagrangian3(N, &ev, lam, pil, piu, gu_old, gx_old);
    for (int k = 0; k < N; ++k) {
      s_u[k] = ut[k] - u[k];
      u[k] = ut[k];
      for (int i = 0; i < 3; ++i) {
        s_x[(k + 1) * 3 + i] = xt[(k + 1) * 3 + i] - x[(k + 1) * 3 + i];
        x[(k + 1) * 3 + i] = xt[(k + 1) * 3 + i];
      }
    }
    ev = evt;
  }
  info->iters = nqp;
  return info->status;
}
