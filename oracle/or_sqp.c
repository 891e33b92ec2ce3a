/*
 * or_sqp.c -- the NMPC regulator: multiple-shooting NLP (OCP_NLP) solved by
 * SQP with a Powell l1-merit backtracking line search and a damped block BFGS
 * Hessian approximation (Sec. III-B and IV), in plain FP64.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Decision vector (Sec. III-B): xi = [u_0, x_1, u_1, x_2, ..., u_{N-1}, x_N],
 * with x_0 = x-hat_{i|i} a parameter.  Constraints g_k = F_k - x_{k+1}
 * (k = 0..N-1) and u_min <= u_k <= u_max.  Lagrangian
 *   L = f - lam^T g - pil^T (u - u_min) - piu^T (u_max - u),  pil, piu >= 0.
 */
#include <math.h>
#include <string.h>
#include "oracle.h"

#define QP_MAXN OR_MAX_N

/* Dense Cholesky of the n x n symmetric matrix in a (row-major, leading
 * dimension ld); returns 0 on success, -1 if a pivot is not positive. */
static int chol(int n, double* a, int ld) {
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

/* Solve L L^T z = rhs in place. */
static void chol_solve(int n, const double* l, int ld, double* z) {
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
 * QP subproblem, Eq. (QP-subproblem) with the stage costs (nlpsqp_qp):
 *   min  sum_k 1/2 [dx_k; du_k]^T W_k [dx_k; du_k] + q_k dx_k + r_k du_k
 *   s.t. dx_{k+1} = A_k dx_k + B_k du_k + b_k,  dx_0 = 0,  lb_k <= du_k <= ub_k.
 * W_0 has only its du-part (Wuu[0]), W_N only its dx-part (Wxx[N]).
 * (The paper prints the dynamics with transposed A_k, B_k in the gradient
 * convention; for one state and one input this is the same number.)
 *
 * Method: condense dx = G du + c (G lower-triangular state sensitivities,
 * c the free response to b) into a dense box-constrained QP in du,
 *   min 1/2 du^T H du + h^T du,  lb <= du <= ub,
 * and solve it with a primal active-set method started at the feasible point
 * du = 0: each iteration minimises over the free variables with the working
 * set fixed at its bounds; a step that leaves the box is cut at the first
 * blocking bound, which joins the working set; at a subspace minimiser the
 * working-set bound with the most negative multiplier is released.  Then
 * dx follows from the dynamics, the dynamics multipliers mu from the
 * stationarity conditions in dx (backwards), and the bound multipliers from
 * the stationarity conditions in du.  Returns 0, or -1 if H is not positive
 * definite on a subspace, -2 if the iteration limit is hit.
 */
int or_qp_solve(int N, const double* A, const double* B, const double* b,
                const double* Wxx, const double* Wxu, const double* Wuu,
                const double* q, const double* r, const double* lb, const double* ub,
                double* du, double* dx, double* mu, double* nul, double* nuu,
                int* iters) {
  static const int FREE = 0, LOWER = 1, UPPER = 2;
  double G[QP_MAXN + 1][QP_MAXN];
  double c[QP_MAXN + 1];
  double H[QP_MAXN * QP_MAXN], h[QP_MAXN], L[QP_MAXN * QP_MAXN];
  int ws[QP_MAXN];

  /* condensing: c_{k+1} = A_k c_k + b_k, G_{k+1,j} = A_k G_{k,j}, G_{k+1,k} = B_k */
  for (int j = 0; j < N; ++j) G[0][j] = 0.0;
  c[0] = 0.0;
  for (int k = 0; k < N; ++k) {
    const double Ak = (k == 0) ? 0.0 : A[k];
    for (int j = 0; j < N; ++j) G[k + 1][j] = Ak * G[k][j];
    G[k + 1][k] = B[k];
    c[k + 1] = Ak * c[k] + b[k];
  }
  for (int i = 0; i < N; ++i) {
    for (int j = 0; j < N; ++j) {
      double s = 0.0;
      for (int k = 1; k <= N; ++k) s += Wxx[k] * G[k][i] * G[k][j];
      if (i == j) s += Wuu[i];
      if (j >= 1 && j <= N - 1) s += Wxu[j] * G[j][i];
      if (i >= 1 && i <= N - 1) s += Wxu[i] * G[i][j];
      H[i * N + j] = s;
    }
    double s = r[i];
    for (int k = 1; k <= N; ++k) s += G[k][i] * (Wxx[k] * c[k] + q[k]);
    if (i >= 1 && i <= N - 1) s += Wxu[i] * c[i];
    h[i] = s;
  }

  /* primal active set on the box, started at du = 0 */
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
    /* subspace minimiser: H_FF z_F = -(h_F + H_FX du_X) */
    int idx[QP_MAXN], nf = 0;
    for (int i = 0; i < N; ++i)
      if (ws[i] == FREE) idx[nf++] = i;
    double z[QP_MAXN];
    for (int a = 0; a < nf; ++a) {
      const int i = idx[a];
      double s = h[i];
      for (int j = 0; j < N; ++j)
        if (ws[j] != FREE) s += H[i * N + j] * du[j];
      z[a] = -s;
      for (int bb = 0; bb < nf; ++bb) L[a * QP_MAXN + bb] = H[i * N + idx[bb]];
    }
    if (nf > 0) {
      if (chol(nf, L, QP_MAXN) != 0) {
        status = -1;
        break;
      }
      chol_solve(nf, L, QP_MAXN, z);
    }
    /* ratio test along du -> z */
    double alpha = 1.0;
    int block = -1, block_side = FREE;
    for (int a = 0; a < nf; ++a) {
      const int i = idx[a];
      const double p = z[a] - du[i];
      if (p < 0.0 && z[a] < lb[i]) {
        const double t = (lb[i] - du[i]) / p;
        if (t < alpha) { alpha = t; block = i; block_side = LOWER; }
      } else if (p > 0.0 && z[a] > ub[i]) {
        const double t = (ub[i] - du[i]) / p;
        if (t < alpha) { alpha = t; block = i; block_side = UPPER; }
      }
    }
    if (block >= 0) {
      if (alpha < 0.0) alpha = 0.0;
      for (int a = 0; a < nf; ++a) {
        const int i = idx[a];
        du[i] = du[i] + alpha * (z[a] - du[i]);
      }
      ws[block] = block_side;
      du[block] = (block_side == LOWER) ? lb[block] : ub[block];
      continue;
    }
    for (int a = 0; a < nf; ++a) du[idx[a]] = z[a];
    /* multipliers of the working set: gradient of the condensed objective */
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

  /* states from the dynamics */
  dx[0] = 0.0;
  for (int k = 0; k < N; ++k) {
    const double Ak = (k == 0) ? 0.0 : A[k];
    dx[k + 1] = Ak * dx[k] + B[k] * du[k] + b[k];
  }
  /* dynamics multipliers from stationarity in dx_k:
   *   k = N:       Wxx_N dx_N + q_N + mu_{N-1} = 0
   *   1<=k<=N-1:   Wxx_k dx_k + Wxu_k du_k + q_k - mu_k A_k + mu_{k-1} = 0 */
  mu[N - 1] = -(Wxx[N] * dx[N] + q[N]);
  for (int k = N - 1; k >= 1; --k)
    mu[k - 1] = mu[k] * A[k] - (Wxx[k] * dx[k] + Wxu[k] * du[k] + q[k]);
  /* bound multipliers from stationarity in du_k:
   *   Wuu_k du_k + Wxu_k dx_k + r_k - mu_k B_k - nul_k + nuu_k = 0 */
  for (int k = 0; k < N; ++k) {
    const double cross = (k >= 1) ? Wxu[k] * dx[k] : 0.0;
    const double v = Wuu[k] * du[k] + cross + r[k] - mu[k] * B[k];
    nul[k] = 0.0;
    nuu[k] = 0.0;
    if (ws[k] == LOWER) nul[k] = v;
    if (ws[k] == UPPER) nuu[k] = -v;
  }
  return status;
}

/* ------------------------------------------------------------------------ */

typedef struct {
  double F[OR_MAX_N], A[OR_MAX_N], B[OR_MAX_N], g[OR_MAX_N];
  double q[OR_MAX_N + 1], r[OR_MAX_N];
  double f;
} eval_t;

/* Objective of Sec. VII-A, phi = sum_{k=1..N} Q_z (z_k - zbar_k)^2 T_s, with
 * the optional weights of the extended objective
 *   + sum_{k=1..N} R_u (v_{k-1} - vbar_k)^2 T_s + Q_n (z_N - zbar_N)^2,
 * vbar_k the steady-state input F_ss(zbar_k) in OCP units (both weights are
 * 0 in the paper's objective); its gradient; and the shooting constraints
 * g_k = F_k - x_{k+1} with the sensitivities A_k, B_k of F_k.  The NLP
 * variables are scaled: the OCP state is x = n_T / x_scale (so
 * z = x x_scale / V) and the OCP input is v, with flow F = v Fconv in L/s. */
static void evaluate(const or_model* m, const or_ctrl* c, double EaR, double Fconv,
                     double x0, const double* zbar, const double* u, const double* x,
                     eval_t* e) {
  const int N = c->N;
  const double xs = c->x_scale;
  double f = 0.0;
  for (int k = 0; k < N; ++k) {
    const double xk = (k == 0) ? x0 : x[k];
    double Fn, a, b;
    or_rk4_interval(m, EaR, c->n_rk4, m->Ts, xk * xs, u[k], Fconv, &Fn, &a, &b);
    e->F[k] = Fn / xs;
    e->A[k] = a;
    e->B[k] = b / xs;
    e->g[k] = e->F[k] - x[k + 1];
    e->r[k] = 0.0;
  }
  e->q[0] = 0.0;
  for (int k = 1; k <= N; ++k) {
    const double dz = x[k] * xs / m->V - zbar[k];
    f += c->Qz * dz * dz * m->Ts;
    e->q[k] = 2.0 * c->Qz * dz * m->Ts * xs / m->V;
  }
  if (c->Ru != 0.0) {
    for (int k = 0; k < N; ++k) {
      const double dv = u[k] - or_Fss(m, EaR, zbar[k + 1]) / Fconv;
      f += c->Ru * dv * dv * m->Ts;
      e->r[k] = 2.0 * c->Ru * dv * m->Ts;
    }
  }
  if (c->Qn != 0.0) {
    const double dz = x[N] * xs / m->V - zbar[N];
    f += c->Qn * dz * dz;
    e->q[N] += 2.0 * c->Qn * dz * xs / m->V;
  }
  e->f = f;
}

/* Gradient of the Lagrangian w.r.t. xi, split into u- and x-parts:
 *   d/du_k L = r_k - lam_k B_k - pil_k + piu_k
 *   d/dx_k L = q_k - lam_k A_k + lam_{k-1}   (k = 1..N-1)
 *   d/dx_N L = q_N + lam_{N-1}                                         */
static void grad_lagrangian(int N, const eval_t* e, const double* lam, const double* pil,
                            const double* piu, double* gu, double* gx) {
  for (int k = 0; k < N; ++k) gu[k] = e->r[k] - lam[k] * e->B[k] - pil[k] + piu[k];
  gx[0] = 0.0;
  for (int k = 1; k < N; ++k) gx[k] = e->q[k] - lam[k] * e->A[k] + lam[k - 1];
  gx[N] = e->q[N] + lam[N - 1];
}

/* One damped BFGS update of a 1x1 or 2x2 block (Sec. IV-C).  w is the packed
 * symmetric block (w[0] = W11, w[1] = W12, w[2] = W22), n its size. */
static void bfgs_block(int n, double* w, const double* s, const double* y) {
  const double eps_m = 2.220446049250313e-16;
  double Ws[2];
  if (n == 1) {
    Ws[0] = w[0] * s[0];
  } else {
    Ws[0] = w[0] * s[0] + w[1] * s[1];
    Ws[1] = w[1] * s[0] + w[2] * s[1];
  }
  double sWs = 0.0, sy = 0.0;
  for (int i = 0; i < n; ++i) {
    sWs += s[i] * Ws[i];
    sy += s[i] * y[i];
  }
  const double theta = (sy >= 0.2 * sWs) ? 1.0 : (0.8 * sWs) / (sWs - sy);
  double rr[2], sr = 0.0;
  for (int i = 0; i < n; ++i) {
    rr[i] = theta * y[i] + (1.0 - theta) * Ws[i];
    sr += s[i] * rr[i];
  }
  const double kappa = fmin(sWs, sr);
  if (!(kappa > eps_m)) return;
  if (n == 1) {
    w[0] = w[0] - Ws[0] * Ws[0] / sWs + rr[0] * rr[0] / sr;
  } else {
    w[0] = w[0] - Ws[0] * Ws[0] / sWs + rr[0] * rr[0] / sr;
    w[1] = w[1] - Ws[0] * Ws[1] / sWs + rr[0] * rr[1] / sr;
    w[2] = w[2] - Ws[1] * Ws[1] / sWs + rr[1] * rr[1] / sr;
  }
}

/* exported for the tests: one damped block update, W packed as above */
void or_bfgs_block(int n, double* w, const double* s, const double* y) {
  bfgs_block(n, w, s, y);
}

/* positive definiteness of a packed block by its Cholesky pivots */
static int block_pd(int n, const double* w) {
  if (!(w[0] > 0.0)) return 0;
  if (n == 1) return 1;
  return (w[2] - w[1] * w[1] / w[0]) > 0.0;
}

/* The block-BFGS step of Sec. IV-C on all N + 1 blocks (W[k] packed as above;
 * block 0 = [u_0], block k = [x_k u_k], block N = [x_N]): the damped update of
 * every block, then the reset of all blocks to the identity when any of them
 * is not positive definite.  Returns 1 after a reset. */
static int bfgs_update_blocks(int N, double (*Wb)[3], const double* s_u, const double* s_x,
                              const double* y_u, const double* y_x) {
  double s2[2], y2[2];
  s2[0] = s_u[0]; y2[0] = y_u[0];
  bfgs_block(1, Wb[0], s2, y2);
  for (int k = 1; k < N; ++k) {
    s2[0] = s_x[k]; s2[1] = s_u[k];
    y2[0] = y_x[k]; y2[1] = y_u[k];
    bfgs_block(2, Wb[k], s2, y2);
  }
  s2[0] = s_x[N]; y2[0] = y_x[N];
  bfgs_block(1, Wb[N], s2, y2);
  int pd = block_pd(1, Wb[0]) && block_pd(1, Wb[N]);
  for (int k = 1; k < N; ++k) pd = pd && block_pd(2, Wb[k]);
  if (!pd) {
    for (int k = 0; k <= N; ++k) { Wb[k][0] = 1.0; Wb[k][1] = 0.0; Wb[k][2] = 1.0; }
    return 1;
  }
  return 0;
}

/* exported for the tests: W holds the N + 1 packed blocks, 3 doubles each */
int or_bfgs_update_blocks(int N, double* W, const double* s_u, const double* s_x,
                          const double* y_u, const double* y_x) {
  return bfgs_update_blocks(N, (double (*)[3])W, s_u, s_x, y_u, y_x);
}

/* The SQP; with rows != NULL each iteration that reaches the QP also writes
 * one trace row (at most max_rows). */
static int sqp_impl(const or_model* m, const or_ctrl* c, double EaR, double x0,
                    const double* zbar, double* u, double* x, double* lam, double* pil,
                    double* piu, or_sqp_info* info, or_sqp_trace_row* rows, int max_rows,
                    int* n_rows) {
  const int N = c->N;
  const double Fconv = c->u_scale / 60000.0;      /* OCP unit -> L/s */
  const double umin = c->u_min / c->u_scale;      /* bounds in OCP units */
  const double umax = c->u_max / c->u_scale;
  const double c1 = 1e-4, beta_ls = 0.5, s_max = 100.0;

  /* packed Hessian blocks: block 0 = [u_0], block k = [x_k u_k], block N = [x_N] */
  double Wb[OR_MAX_N + 1][3];
  eval_t ev, ev_trial;
  double du[OR_MAX_N], dx[OR_MAX_N + 1], mu[OR_MAX_N], nul[OR_MAX_N], nuu[OR_MAX_N];
  double sigma[OR_MAX_N];
  double gu[OR_MAX_N], gx[OR_MAX_N + 1], gu_old[OR_MAX_N], gx_old[OR_MAX_N + 1];
  double s_u[OR_MAX_N], s_x[OR_MAX_N + 1];
  double ut[OR_MAX_N], xt[OR_MAX_N + 1];
  double A_qp[OR_MAX_N], Wxx[OR_MAX_N + 1], Wxu[OR_MAX_N + 1], Wuu[OR_MAX_N + 1];
  double lb[OR_MAX_N], ub[OR_MAX_N];

  for (int k = 0; k <= N; ++k) {           /* W^[0] = I */
    Wb[k][0] = 1.0; Wb[k][1] = 0.0; Wb[k][2] = 1.0;
  }
  memset(info, 0, sizeof(*info));
  x[0] = x0;
  evaluate(m, c, EaR, Fconv, x0, zbar, u, x, &ev);

  int l = 0, nqp = 0;
  if (n_rows) *n_rows = 0;
  for (;; ++l) {
    int reset = 0;
    if (l > 0) {
      /* damped block BFGS with s = xi^[l] - xi^[l-1],
       * y = grad L(xi^[l], .) - grad L(xi^[l-1], .), both at the new multipliers */
      grad_lagrangian(N, &ev, lam, pil, piu, gu, gx);
      double y_u[OR_MAX_N], y_x[OR_MAX_N + 1];
      for (int k = 0; k < N; ++k) y_u[k] = gu[k] - gu_old[k];
      y_x[0] = 0.0;
      for (int k = 1; k <= N; ++k) y_x[k] = gx[k] - gx_old[k];
      reset = bfgs_update_blocks(N, Wb, s_u, s_x, y_u, y_x);
      info->n_hess_reset += reset;
    }

    /* scaled convergence test, Eq. (convergence) */
    grad_lagrangian(N, &ev, lam, pil, piu, gu, gx);
    double mult1 = 0.0;
    for (int k = 0; k < N; ++k) mult1 += fabs(lam[k]) + fabs(pil[k]) + fabs(piu[k]);
    const double s_d = fmax(s_max, mult1 / (double)(3 * N)) / s_max;
    double kg = 0.0, ke = 0.0;
    for (int k = 0; k < N; ++k) kg = fmax(kg, fabs(gu[k]));
    for (int k = 1; k <= N; ++k) kg = fmax(kg, fabs(gx[k]));
    const double kg_raw = kg;
    kg /= s_d;
    for (int k = 0; k < N; ++k) ke = fmax(ke, fabs(ev.g[k]));
    info->kkt_grad = kg;
    info->kkt_eq = ke;
    info->f = ev.f;
    or_sqp_trace_row* tr = NULL;
    if (rows && *n_rows < max_rows) {
      tr = &rows[(*n_rows)++];
      memset(tr, 0, sizeof(*tr));
      tr->stop = -1;
      tr->l = l;
      tr->reset = reset;
      tr->s_d = s_d;
      tr->kkt_grad_raw = kg_raw;
      tr->kkt_grad = kg;
      tr->kkt_eq = ke;
      tr->f = ev.f;
      for (int k = 0; k < N; ++k) {
        tr->lam[k] = lam[k];
        tr->pil[k] = pil[k];
        tr->piu[k] = piu[k];
        tr->g[k] = ev.g[k];
        tr->r[k] = ev.r[k];
        tr->A[k] = ev.A[k];
        tr->B[k] = ev.B[k];
      }
      for (int k = 0; k <= N; ++k) tr->q[k] = ev.q[k];
    }
    if (kg <= c->sqp_tol && ke <= c->sqp_tol) {
      info->status = 0;
      if (tr) tr->stop = 0;
      break;
    }
    if (l >= c->sqp_max_it) {
      info->status = 1;
      if (tr) tr->stop = 1;
      break;
    }

    /* QP subproblem at xi^[l] */
    for (int k = 0; k <= N; ++k) {
      Wxx[k] = (k >= 1) ? ((k == N) ? Wb[N][0] : Wb[k][0]) : 0.0;
      Wxu[k] = (k >= 1 && k < N) ? Wb[k][1] : 0.0;
      Wuu[k] = (k == 0) ? Wb[0][0] : ((k < N) ? Wb[k][2] : 0.0);
    }
    for (int k = 0; k < N; ++k) {
      A_qp[k] = ev.A[k];
      lb[k] = umin - u[k];
      ub[k] = umax - u[k];
    }
    int qp_it = 0;
    or_qp_solve(N, A_qp, ev.B, ev.g, Wxx, Wxu, Wuu, ev.q, ev.r, lb, ub, du, dx, mu, nul,
                nuu, &qp_it);
    info->qp_iters += qp_it;
    ++nqp;

    /* penalty update and the merit slope */
    for (int k = 0; k < N; ++k)
      sigma[k] = (l == 0) ? fabs(mu[k]) : fmax(fabs(mu[k]), 0.5 * (sigma[k] + fabs(mu[k])));
    double pen = 0.0, dfd = 0.0;
    for (int k = 0; k < N; ++k) pen += sigma[k] * fabs(ev.g[k]);
    for (int k = 0; k < N; ++k) dfd += ev.r[k] * du[k];
    for (int k = 1; k <= N; ++k) dfd += ev.q[k] * dx[k];
    const double T0 = ev.f + pen;
    const double DT0 = dfd - pen;
    if (tr) {
      tr->T0 = T0;
      tr->DT0 = DT0;
      for (int k = 0; k < N; ++k) {
        tr->du[k] = du[k];
        tr->mu[k] = mu[k];
        tr->sigma[k] = sigma[k];
      }
      for (int k = 0; k <= N; ++k) tr->dx[k] = dx[k];
    }

    /* backtracking on the Armijo condition */
    double alpha = 1.0;
    int accepted = 0;
    for (int hv = 0; hv <= c->ls_max; ++hv) {
      ut[0] = 0.0;
      xt[0] = x0;
      for (int k = 0; k < N; ++k) {
        /* the step keeps u inside its bounds (Sec. IV-A); the clip only
         * removes the last-bit rounding of u + (bound - u) */
        ut[k] = fmin(fmax(u[k] + alpha * du[k], umin), umax);
        xt[k + 1] = x[k + 1] + alpha * dx[k + 1];
      }
      evaluate(m, c, EaR, Fconv, x0, zbar, ut, xt, &ev_trial);
      info->ls_trials++;
      double pt = 0.0;
      for (int k = 0; k < N; ++k) pt += sigma[k] * fabs(ev_trial.g[k]);
      if (tr && tr->n_trials < OR_TRACE_MAX_TRIALS) {
        tr->alpha[tr->n_trials] = alpha;
        tr->f_trial[tr->n_trials] = ev_trial.f;
        tr->pen_trial[tr->n_trials] = pt;
        tr->n_trials++;
      }
      if (ev_trial.f + pt <= T0 + c1 * alpha * DT0) {
        accepted = 1;
        break;
      }
      alpha *= beta_ls;
    }
    if (tr) tr->accepted = accepted;
    if (!accepted) {
      info->status = 2;
      break;
    }

    /* step in the primal and dual variables */
    for (int k = 0; k < N; ++k) {
      lam[k] = lam[k] + alpha * (mu[k] - lam[k]);
      pil[k] = pil[k] + alpha * (nul[k] - pil[k]);
      piu[k] = piu[k] + alpha * (nuu[k] - piu[k]);
    }
    grad_lagrangian(N, &ev, lam, pil, piu, gu_old, gx_old);
    for (int k = 0; k < N; ++k) {
      s_u[k] = ut[k] - u[k];
      s_x[k + 1] = xt[k + 1] - x[k + 1];
      u[k] = ut[k];
      x[k + 1] = xt[k + 1];
    }
    ev = ev_trial;
  }
  info->iters = nqp;
  return info->status;
}

int or_sqp(const or_model* m, const or_ctrl* c, double EaR, double x0,
           const double* zbar, double* u, double* x, double* lam, double* pil,
           double* piu, or_sqp_info* info) {
  return sqp_impl(m, c, EaR, x0, zbar, u, x, lam, pil, piu, info, NULL, 0, NULL);
}

int or_sqp_traced(const or_model* m, const or_ctrl* c, double EaR, double x0,
                  const double* zbar, double* u, double* x, double* lam, double* pil,
                  double* piu, or_sqp_info* info, or_sqp_trace_row* rows, int max_rows,
                  int* n_rows) {
  int dummy = 0;
  return sqp_impl(m, c, EaR, x0, zbar, u, x, lam, pil, piu, info, rows, max_rows,
                  n_rows ? n_rows : &dummy);
}

/* ------------------------------------------------------------------------ */
/* Sensitivity of the OCP solution's first input u_0 to the initial state x_0
 * (scaled) and to the objective weights (Q_z, R_u, Q_n), by implicit
 * differentiation of the KKT conditions at a solution (u, x, lam, pil, piu)
 * of or_sqp: the tangent (dx, du) solves the equality-constrained QP whose
 * Hessian is that of the Lagrangian, whose linear term is the derivative of
 * the Lagrangian gradient with respect to the parameter, and whose
 * constraints are the linearised dynamics (dx_1 = A_0 dx_0 + B_0 du_0) with
 * the active bounds held (du_k = 0).  The second derivatives of the shooting
 * map come from central differences of its analytic first derivatives; the
 * QP is solved through its full KKT matrix by Gaussian elimination with
 * partial pivoting.  A bound is active when u_k lies on it and its
 * multiplier exceeds 1e-10.  out[0..3] = du_0/dx_0, du_0/dQ_z, du_0/dR_u,
 * du_0/dQ_n; returns 0, or -1 if the KKT matrix is singular. */

static int dense_solve(int n, double* a, double* b) {
  for (int j = 0; j < n; ++j) {
    int piv = j;
    for (int i = j + 1; i < n; ++i)
      if (fabs(a[i * n + j]) > fabs(a[piv * n + j])) piv = i;
    if (!(fabs(a[piv * n + j]) > 0.0)) return -1;
    if (piv != j) {
      for (int k = 0; k < n; ++k) {
        const double t = a[j * n + k];
        a[j * n + k] = a[piv * n + k];
        a[piv * n + k] = t;
      }
      const double t = b[j];
      b[j] = b[piv];
      b[piv] = t;
    }
    for (int i = j + 1; i < n; ++i) {
      const double f = a[i * n + j] / a[j * n + j];
      if (f == 0.0) continue;
      for (int k = j; k < n; ++k) a[i * n + k] -= f * a[j * n + k];
      b[i] -= f * b[j];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int k = i + 1; k < n; ++k) s -= a[i * n + k] * b[k];
    b[i] = s / a[i * n + i];
  }
  return 0;
}

int or_ocp_sens(const or_model* m, const or_ctrl* c, double EaR, double x0, const double* zbar,
                const double* u, const double* x, const double* lam, const double* pil,
                const double* piu, double* out) {
  const int N = c->N;
  const double xs = c->x_scale, Ts = m->Ts;
  const double Fconv = c->u_scale / 60000.0;
  const double umin = c->u_min / c->u_scale, umax = c->u_max / c->u_scale;
  const double sz = xs / m->V;                       /* dz/dx */
  static __thread double Fxx[OR_MAX_N], Fxu[OR_MAX_N], Fuu[OR_MAX_N], Ak[OR_MAX_N], Bk[OR_MAX_N];
  int act[OR_MAX_N];
  for (int k = 0; k < N; ++k) {
    const double xk = (k == 0) ? x0 : x[k];
    double Fn, a, b, ap, bp, am, bm;
    or_rk4_interval(m, EaR, c->n_rk4, Ts, xk * xs, u[k], Fconv, &Fn, &a, &b);
    Ak[k] = a;
    Bk[k] = b / xs;
    /* second derivatives of the scaled map F(x, v) = F_n(x xs, v) / xs */
    const double hx = 1e-5 * fabs(xk), hv = 1e-5;
    or_rk4_interval(m, EaR, c->n_rk4, Ts, (xk + hx) * xs, u[k], Fconv, &Fn, &ap, &bp);
    or_rk4_interval(m, EaR, c->n_rk4, Ts, (xk - hx) * xs, u[k], Fconv, &Fn, &am, &bm);
    Fxx[k] = (ap - am) / (2.0 * hx);
    Fxu[k] = (bp - bm) / (2.0 * hx) / xs;
    or_rk4_interval(m, EaR, c->n_rk4, Ts, xk * xs, u[k] + hv, Fconv, &Fn, &ap, &bp);
    or_rk4_interval(m, EaR, c->n_rk4, Ts, xk * xs, u[k] - hv, Fconv, &Fn, &am, &bm);
    Fuu[k] = (bp - bm) / (2.0 * hv) / xs;
    act[k] = ((u[k] - umin <= 1e-12 && pil[k] > 1e-10) || (umax - u[k] <= 1e-12 && piu[k] > 1e-10));
  }
  /* unknowns: du_0..du_{N-1}, dx_1..dx_N, then multipliers of the N dynamics
   * rows and of the active bounds */
  int na = 0;
  for (int k = 0; k < N; ++k) na += act[k];
  const int nv = 2 * N, n = nv + N + na;
  static __thread double K[(4 * OR_MAX_N) * (4 * OR_MAX_N)], rhs[4 * OR_MAX_N];
#define IU(k) (k)
#define IX(k) (N + (k) - 1)
  for (int dir = 0; dir < 4; ++dir) {
    for (int i = 0; i < n * n; ++i) K[i] = 0.0;
    for (int i = 0; i < n; ++i) rhs[i] = 0.0;
    const double dx0 = (dir == 0) ? 1.0 : 0.0;
    const double dQz = (dir == 1), dRu = (dir == 2), dQn = (dir == 3);
    /* Hessian of the Lagrangian and the linear terms */
    for (int k = 0; k < N; ++k) {
      K[IU(k) * n + IU(k)] += 2.0 * Ts * c->Ru - lam[k] * Fuu[k];
      if (k >= 1) {
        K[IX(k) * n + IX(k)] += 2.0 * Ts * c->Qz * sz * sz - lam[k] * Fxx[k];
        K[IX(k) * n + IU(k)] += -lam[k] * Fxu[k];
        K[IU(k) * n + IX(k)] += -lam[k] * Fxu[k];
      } else {
        rhs[IU(0)] -= -lam[0] * Fxu[0] * dx0;              /* x_0 cross term */
      }
      const double vb = or_Fss(m, EaR, zbar[k + 1]) / Fconv;
      rhs[IU(k)] -= 2.0 * Ts * dRu * (u[k] - vb);
    }
    K[IX(N) * n + IX(N)] += (2.0 * Ts * c->Qz + 2.0 * c->Qn) * sz * sz;
    for (int k = 1; k <= N; ++k) {
      const double dz = x[k] * sz - zbar[k];
      rhs[IX(k)] -= 2.0 * Ts * dQz * dz * sz;
      if (k == N) rhs[IX(k)] -= 2.0 * dQn * dz * sz;
    }
    /* dynamics rows: dx_{k+1} - A_k dx_k - B_k du_k = (k == 0 ? A_0 dx_0 : 0) */
    for (int k = 0; k < N; ++k) {
      const int row = nv + k;
      K[row * n + IX(k + 1)] = 1.0;
      K[IX(k + 1) * n + row] = 1.0;
      K[row * n + IU(k)] = -Bk[k];
      K[IU(k) * n + row] = -Bk[k];
      if (k >= 1) {
        K[row * n + IX(k)] = -Ak[k];
        K[IX(k) * n + row] = -Ak[k];
      }
      rhs[row] = (k == 0) ? Ak[0] * dx0 : 0.0;
    }
    int r = nv + N;
    for (int k = 0; k < N; ++k)
      if (act[k]) {
        K[r * n + IU(k)] = 1.0;
        K[IU(k) * n + r] = 1.0;
        rhs[r] = 0.0;
        ++r;
      }
    if (dense_solve(n, K, rhs) != 0) return -1;
    out[dir] = rhs[IU(0)];
  }
#undef IU
#undef IX
  return 0;
}
