// mc_sqp.cuh -- the NMPC regulator of Sec. III-B solved by the SQP of Sec. IV,
// per thread.
//
// NLP (Eq. OCP_NLP) in scaled variables: OCP state x = n_T / x_scale, OCP
// input v with flow F = v Fconv; decision vector [v_0, x_1, ..., v_{N-1}, x_N];
// constraints g_k = F_k - x_{k+1}; Lagrangian
//   L = f - lam^T g - pil^T (v - v_min) - piu^T (v_max - v).
//
// The SQP is written as resumable phases so that a persistent kernel can run
// each lane's SQP at its own pace while the warp's lanes share the expensive
// shooting evaluations (see mc_closedloop.cuh):
//   sqp_start          W = I, first evaluation at the warm start
//   sqp_check          block BFGS, the scaled KKT test, the QP, the merit
//                      slope, and the first trial point
//   sqp_eval_trial     shooting at the trial point (the dominant cost)
//   sqp_trial_result   Armijo test; accept and step, or halve the step
// sqp_solve chains them for one OCP.
#pragma once

#include "mc_qp.cuh"

namespace mc {

struct SqpInfo {
  int iters, status, ls_trials, qp_iters, n_hess_reset, qp_fail;
  double kkt_grad, kkt_eq, f;
};

// Resumable SQP state of one OCP.
struct SqpState {
  int N, max_it;      // horizon and iteration limit of this OCP
  int l;              // iteration counter
  int hv;             // halvings in the current line search
  int nc;             // line-search candidates set up for the next evaluation (1
                      // unless the persistent schedule backtracks speculatively)
  bool pt_ready;      // pt holds the trial point's penalty sigma^T |g|
  double f, ft, pt, alpha, T0, DT0;
  SqpInfo info;
};

// One shooting interval with sensitivities: F_k = RK4^{N_c}(x_k, u_k) and
// A_k = dF_k/dx_k, B_k = dF_k/du_k in the scaled variables, and the residual
// g_k = F_k - x_{k+1}.  Not inlined: the loop of evaluate and the persistent
// schedule's shooting pool (any lane integrating any lane's interval) run this
// one compiled body, so both give the same bits.
// With cov (interval 0), the same RK4 stages also give the CD-EKF prediction
// of the next sample from (x_0, P0) under this input: xpr = F_0 in K L and Ppr.
// The results come back by value: a non-inlined function that wrote them
// through references would force the caller's variables into local memory.
struct Shot {
  double A, B, g, xpr, Ppr;
};

template <class R>
__device__ __noinline__ Shot shoot_interval(const DevModel& m, const DevCtrl& c, double EaR,
                                            double xk, double uk, double xn, double xs,
                                            double ixs, bool cov, double P0) {
  R Fn, a, b, P1 = 0;
  rk4_interval<R, true>(m, (R)EaR, c.n_rk4, (R)m.Ts, (R)(xk * xs), (R)uk, (R)c.Fconv, Fn, a,
                        b, cov, (R)P0, &P1);
  Shot r;
  r.A = (double)a;
  r.B = (double)b * ixs;
  r.g = fma((double)Fn, ixs, -xn);
  r.xpr = (double)Fn;
  r.Ppr = (double)P1;
  return r;
}

// The objective's stage terms Q_z (z_k - zbar_k)^2 T_s, k = 1..N, and their
// gradients q_k at the states x (columns as in the SQP passes).
__device__ __forceinline__ double objective_pass(int N, int64_t ld, double Qz, double Ts,
                                                 double xs, double iV, double qf,
                                                 const double* __restrict__ x_,
                                                 const double* __restrict__ zb_,
                                                 double* __restrict__ q_) {
  double f = 0.0;
#pragma unroll 2
  for (int k = 1; k <= N; ++k) {
    const int64_t o = k * ld;
    const double dz = x_[o] * xs * iV - zb_[o];
    f += Qz * dz * dz * Ts;
    q_[o] = qf * dz;
  }
  return f;
}

// The same interval without the covariance: the static schedule's intervals
// 1 .. N-1, which need no runtime test of the covariance flag in their RK4
// steps.  Same operations on x, A and B as shoot_interval, and the same
// bits: the model and the RK4 steps write out every rounding, so the two
// compiled bodies leave the compiler no contraction to choose differently.
template <class R>
__device__ __noinline__ Shot shoot_interval_plain(const DevModel& m, const DevCtrl& c,
                                                  double EaR, double xk, double uk, double xn,
                                                  double xs, double ixs) {
  R Fn, a, b;
  rk4_interval<R, true>(m, (R)EaR, c.n_rk4, (R)m.Ts, (R)(xk * xs), (R)uk, (R)c.Fconv, Fn, a,
                        b);
  Shot r;
  r.A = (double)a;
  r.B = (double)b * ixs;
  r.g = fma((double)Fn, ixs, -xn);
  r.xpr = 0.0;
  r.Ppr = 0.0;
  return r;
}

// Which intervals evaluate integrates.
enum RkMode : int {
  kRkAll = 0,   // every interval
  kRkEnds = 1,  // only 0 and N-1: after the receding-horizon shift the
                // intervals 1 .. N-2 hold the previous OCP's A_k, B_k, g_k at
                // the same (x_k, u_k)
  kRkNone = 2   // none: the arrays were filled by the shooting pool
};

// The extended objective's terms, R_u (v_k - vbar_{k+1})^2 T_s and
// Q_n (z_N - zbar_N)^2 (zero in the paper's objective), and Q_n's gradient.
__device__ __forceinline__ double objective_extra(const DevModel& m, const DevCtrl& c, int N,
                                                  const Ws& w, int u_arr, int x_arr,
                                                  int q_arr) {
  double f = 0.0;
  const double xs = c.x_scale;
  if (c.Ru != 0.0) {
    for (int k = 0; k < N; ++k) {
      const double dv = w(u_arr, k) - w(VB, k + 1);
      f += c.Ru * dv * dv * m.Ts;
    }
  }
  if (c.Qn != 0.0) {
    const double dz = w(x_arr, N) * xs * m.iV - w(ZB, N);
    f += c.Qn * dz * dz;
    w(q_arr, N) += 2.0 * c.Qn * dz * xs * m.iV;
  }
  return f;
}

// Shooting of the intervals selected by rk_mode at the point (u_arr, x_arr),
// writing A_k, B_k, g_k into (a_arr, b_arr, g_arr) and q_k = df/dx_k into
// q_arr; returns the objective f = sum_k Q_z (z_k - zbar_k)^2 T_s, which
// depends on the states only.
// R is the arithmetic of the RK4 integration (FP32 on the mixed-precision
// path); the constraint residual g_k, the objective and its gradient are FP64.
// Not inlined: the shooting loop is the hot spot, and as a function of its own
// it gets the full register file instead of sharing it with the SQP state.
template <class R>
__device__ __noinline__ double evaluate(const DevModel& m, const DevCtrl& c, double EaR,
                                           int N, const Ws& w, int u_arr, int x_arr,
                                           int a_arr, int b_arr, int g_arr, int q_arr,
                                           int rk_mode) {
  const double xs = c.x_scale, ixs = 1.0 / c.x_scale;
  const double qf = 2.0 * c.Qz * m.Ts * xs * m.iV;
  if (rk_mode == kRkNone)  // the pool shot the intervals: the objective pass only
    return objective_pass(N, w.ld, c.Qz, m.Ts, xs, m.iV, qf, ws_col(w, x_arr), ws_col(w, ZB),
                          ws_col(w, q_arr)) +
           objective_extra(m, c, N, w, u_arr, x_arr, q_arr);
  double f = 0.0;
  double xk = w(X, 0);
  const int pr_arr = (a_arr == TA) ? TPR : EPR;
  for (int k = 0; k < N; ++k) {
    const double xn = w(x_arr, k + 1);
    if (rk_mode == kRkAll || (rk_mode == kRkEnds && (k == 0 || k == N - 1))) {
      Shot r;
      if (k == 0) {
        r = shoot_interval<R>(m, c, EaR, xk, w(u_arr, k), xn, xs, ixs, true, w(PIN, 0));
        w(pr_arr, 0) = r.xpr;
        w(pr_arr, 1) = r.Ppr;
      } else {
        r = shoot_interval_plain<R>(m, c, EaR, xk, w(u_arr, k), xn, xs, ixs);
      }
      w(a_arr, k) = r.A;
      w(b_arr, k) = r.B;
      w(g_arr, k) = r.g;
    }
    const double dz = xn * xs * m.iV - w(ZB, k + 1);
    f += c.Qz * dz * dz * m.Ts;
    w(q_arr, k + 1) = qf * dz;
    xk = xn;
  }
  return f + objective_extra(m, c, N, w, u_arr, x_arr, q_arr);
}

// Damped BFGS update of one packed block (Sec. IV-C); n = 1 or 2.
__device__ __forceinline__ void bfgs_block(int n, double& w11, double& w12, double& w22,
                                           double s1, double s2, double y1, double y2) {
  const double eps_m = 2.220446049250313e-16;
  double Ws1, Ws2 = 0.0, sWs, sy;
  if (n == 1) {
    Ws1 = w11 * s1;
    sWs = s1 * Ws1;
    sy = s1 * y1;
  } else {
    Ws1 = w11 * s1 + w12 * s2;
    Ws2 = w12 * s1 + w22 * s2;
    sWs = s1 * Ws1 + s2 * Ws2;
    sy = s1 * y1 + s2 * y2;
  }
  const double theta = (sy >= 0.2 * sWs) ? 1.0 : (0.8 * sWs) / (sWs - sy);
  const double r1 = theta * y1 + (1.0 - theta) * Ws1;
  const double r2 = theta * y2 + (1.0 - theta) * Ws2;
  const double sr = (n == 1) ? s1 * r1 : s1 * r1 + s2 * r2;
  const double kappa = fmin(sWs, sr);
  if (!(kappa > eps_m)) return;
  // both reciprocals from one division (both factors exceed eps_m here)
  const double inv = rcp_newton(sWs * sr);
  const double isWs = sr * inv, isr = sWs * inv;
  w11 = w11 - Ws1 * Ws1 * isWs + r1 * r1 * isr;
  if (n == 2) {
    w12 = w12 - Ws1 * Ws2 * isWs + r1 * r2 * isr;
    w22 = w22 - Ws2 * Ws2 * isWs + r2 * r2 * isr;
  }
}

// Trial point xi + alpha dxi (u clipped into its bounds against rounding).
// The per-lane passes below take the scratch rows as separate columns through
// restrict-qualified pointers (element k at c[k * ld]; the rows are disjoint),
// so that the compiler may issue the next stages' loads while the current
// stage's stores are pending: these passes are bound by memory latency, not by
// their arithmetic.
__device__ __forceinline__ void trial_point_pass(int N, int64_t ld, double alpha, double vmin,
                                                 double vmax, const double* __restrict__ u_,
                                                 const double* __restrict__ du_,
                                                 const double* __restrict__ x_,
                                                 const double* __restrict__ dx_,
                                                 double* __restrict__ ut_,
                                                 double* __restrict__ xt_) {
#pragma unroll 2
  for (int k = 0; k < N; ++k) {
    const int64_t o = k * ld;
    ut_[o] = fmin(fmax(u_[o] + alpha * du_[o], vmin), vmax);
    xt_[o + ld] = x_[o + ld] + alpha * dx_[o + ld];
  }
}

__device__ __forceinline__ void sqp_trial_point(const DevCtrl& c, const Ws& w,
                                                const SqpState& s) {
  trial_point_pass(s.N, w.ld, s.alpha, c.vmin, c.vmax, ws_col(w, U), ws_col(w, DU),
                   ws_col(w, X), ws_col(w, DX), ws_col(w, UT), ws_col(w, XT));
}

// Speculative backtracking (persistent schedule): after a failed trial, the
// trial points of the next nc halvings, alpha, alpha/2, ..., alpha/2^(nc-1)
// (exact: powers of two), each in its candidate's columns, so that the pool
// shoots them in one round.  nc doubles with every round the line search
// keeps failing (2, then kLsCand), and never passes the halving limit.  The
// candidates are then tested in order with the same Armijo rule, so the
// accepted step, the iterates and the trial count are those of the
// sequential line search; the shot candidates after the accepted one are
// the price, which only pays while the warp has idle lanes: with more than
// c.spec_lanes of its lanes busy (nbusy) there is one trial point.
__device__ __forceinline__ void sqp_trial_points_spec(const DevCtrl& c, const Ws& w,
                                                      SqpState& s, int nbusy) {
  int nc = (nbusy > c.spec_lanes) ? 1 : (s.hv <= 1) ? 2 : kLsCand;
  const int left = c.ls_max - s.hv + 1;  // trials the halving limit still allows
  nc = nc < left ? nc : left;
  nc = nc < 1 ? 1 : nc;
  double a = s.alpha;
  for (int q = 0; q < nc; ++q) {
    trial_point_pass(s.N, w.ld, a, c.vmin, c.vmax, ws_col(w, U), ws_col(w, DU), ws_col(w, X),
                     ws_col(w, DX), ws_col(w, lsc_col(UT, q)), ws_col(w, lsc_col(XT, q)));
    a *= 0.5;
  }
  s.nc = nc;
}

// Start an OCP from the warm start in (U, X, LAM, PIL, PIU) with x0 and the
// set-points z-bar(t_{i+k}) in ZB[1..N]; W^[0] = I.  With shifted_eval the
// evaluation arrays hold the previous OCP's final evaluation shifted by one
// interval (see evaluate).
// With shoot = false the first evaluation is left to the caller: the
// persistent schedule shoots the intervals kRkEnds or kRkAll names in its pool
// and then calls sqp_start_eval.
template <class R>
__device__ __forceinline__ void sqp_start(const DevModel& m, const DevCtrl& c, double EaR,
                                          double x0, const Ws& w, int N, int max_it,
                                          bool shifted_eval, SqpState& s, bool shoot = true) {
  s.N = N;
  s.max_it = max_it;
  s.l = 0;
  s.hv = 0;
  s.nc = 1;
  s.pt_ready = false;
  s.alpha = 0.0;
  s.info = SqpInfo{};
  for (int k = 0; k <= N; ++k) {
    w(WXX, k) = 1.0;
    w(WXU, k) = 0.0;
    w(WUU, k) = 1.0;
  }
  w(X, 0) = x0;
  s.f = shoot ? evaluate<R>(m, c, EaR, N, w, U, X, EA, EB, EG, EQ,
                            shifted_eval ? kRkEnds : kRkAll)
              : 0.0;
}

// The first evaluation after its intervals were shot elsewhere.
template <class R>
__device__ __forceinline__ void sqp_start_eval(const DevModel& m, const DevCtrl& c, double EaR,
                                               const Ws& w, SqpState& s) {
  s.f = evaluate<R>(m, c, EaR, s.N, w, U, X, EA, EB, EG, EQ, kRkNone);
}

// Top of an SQP iteration at xi^[l] (evaluated): damped block BFGS for l > 0,
// the scaled KKT test of Eq. (convergence) and the iteration limit.  Returns
// true when the OCP is finished (s.info.status set).  Otherwise solves the QP,
// updates the l1 penalty weights, forms T(0) and its slope and prepares the
// first trial point (alpha = 1).
// First pass of an SQP iteration: Lagrangian gradient at the current point
// (its infinity norm kg and the multipliers' 1-norm), for l > 0 the damped
// block BFGS of every block with the positive-definiteness test of the
// updated blocks, max |g_k| and the QP bounds.  GLX(k) holds, on entry, the
// new-point x-gradient of stage k minus its old-point value (written by the
// previous stage of this pass), the s-y pair's x part of block k.
__device__ __forceinline__ void check_pass(
    int N, int64_t ld, bool bfgs, double alpha, bool has_r, double vmin, double vmax,
    const double* __restrict__ lam_, const double* __restrict__ pil_,
    const double* __restrict__ piu_, const double* __restrict__ A_,
    const double* __restrict__ B_, const double* __restrict__ g_, const double* __restrict__ q_,
    const double* __restrict__ r_, double* __restrict__ du_,
    const double* __restrict__ dx_, const double* __restrict__ glu_,
    double* __restrict__ glx_, double* __restrict__ wxx_, double* __restrict__ wxu_,
    double* __restrict__ wuu_, const double* __restrict__ u_, double* __restrict__ lb_,
    double* __restrict__ ub_, double& kg, double& ke, double& mult1, bool& pd, uint64_t& lo,
    uint64_t& up, double& gscale) {
  kg = 0.0;
  ke = 0.0;
  mult1 = 0.0;
  pd = true;
  lo = 0;
  up = 0;
  gscale = 1.0;
  double lam = lam_[0];
#pragma unroll 2
  for (int k = 0; k < N; ++k) {
    const int64_t o = k * ld;
    const double pil = pil_[o], piu = piu_[o];
    mult1 += fabs(lam) + fabs(pil) + fabs(piu);
    double gu = -lam * B_[o] - pil + piu;
    if (has_r) gu += r_[o];
    double gx, lam_n = 0.0;
    if (k + 1 < N) {
      lam_n = lam_[o + ld];
      gx = q_[o + ld] - lam_n * A_[o + ld] + lam;
    } else {
      gx = q_[o + ld] + lam;
    }
    if (bfgs) {
      // damped block BFGS with s = alpha (du, dx) and
      // y = grad L(xi^[l], .) - grad L(xi^[l-1], .) at the new multipliers
      const double su = alpha * du_[o], sx = alpha * dx_[o];
      const double yu = gu - glu_[o], yx = (k > 0) ? glx_[o] : 0.0;
      if (k == 0) {
        double w11 = wuu_[0], w12 = 0.0, w22 = 0.0;
        bfgs_block(1, w11, w12, w22, su, 0.0, yu, 0.0);
        wuu_[0] = w11;
        pd = pd && (w11 > 0.0);
      } else {
        double w11 = wxx_[o], w12 = wxu_[o], w22 = wuu_[o];
        bfgs_block(2, w11, w12, w22, sx, su, yx, yu);
        wxx_[o] = w11;
        wxu_[o] = w12;
        wuu_[o] = w22;
        // Cholesky pivots a and d - b^2/a, the second tested as a d - b^2 > 0
        pd = pd && (w11 > 0.0) && (w11 * w22 - w12 * w12 > 0.0);
      }
      const double glx_n = glx_[o + ld];
      if (k == N - 1) {
        double wn = wxx_[o + ld], d0 = 0.0, d1 = 0.0;
        bfgs_block(1, wn, d0, d1, alpha * dx_[o + ld], 0.0, gx - glx_n, 0.0);
        wxx_[o + ld] = wn;
        pd = pd && (wn > 0.0);
      }
      // keep the new-point x-gradient of stage k+1 for its block
      glx_[o + ld] = gx - glx_n;
    }
    kg = fmax(kg, fmax(fabs(gu), fabs(gx)));
    ke = fmax(ke, fabs(g_[o]));
    // the QP's bounds and starting working set (the bounds active at the
    // current iterate, du on them), read after the BFGS step read du
    const double u = u_[o];
    const double lb = vmin - u, ub = vmax - u;
    lb_[o] = lb;
    ub_[o] = ub;
    double du0 = 0.0;
    if (lb >= 0.0) {
      lo |= 1ull << k;
      du0 = lb;
    } else if (ub <= 0.0) {
      up |= 1ull << k;
      du0 = ub;
    }
    du_[o] = du0;
    gscale = fmax(gscale, fabs(q_[o + ld]));
    if (has_r) gscale = fmax(gscale, fabs(r_[o]));
    lam = lam_n;
  }
}

// The sigma update of the l1 penalty weights (Sec. IV-B), the penalty and the
// merit slope's objective part, fused with the first trial point (alpha = 1).
__device__ __forceinline__ void penalty_pass(
    int N, int64_t ld, bool first, bool has_r, double vmin, double vmax,
    const double* __restrict__ mu_, double* __restrict__ sig_, const double* __restrict__ g_,
    const double* __restrict__ q_, const double* __restrict__ r_,
    const double* __restrict__ du_, const double* __restrict__ dx_,
    const double* __restrict__ u_, const double* __restrict__ x_, double* __restrict__ ut_,
    double* __restrict__ xt_, double& pen, double& dfd) {
  pen = 0.0;
  dfd = 0.0;
#pragma unroll 2
  for (int k = 0; k < N; ++k) {
    const int64_t o = k * ld;
    const double am = fabs(mu_[o]);
    const double sg = first ? am : fmax(am, 0.5 * (sig_[o] + am));
    sig_[o] = sg;
    pen += sg * fabs(g_[o]);
    const double dxn = dx_[o + ld];
    dfd += q_[o + ld] * dxn;
    const double du = du_[o];
    if (has_r) dfd += r_[o] * du;
    ut_[o] = fmin(fmax(u_[o] + 1.0 * du, vmin), vmax);
    xt_[o + ld] = x_[o + ld] + 1.0 * dxn;
  }
}

// Top of an SQP iteration at xi^[l] (evaluated): damped block BFGS for l > 0,
// the scaled KKT test of Eq. (convergence) and the iteration limit.  Returns
// true when the OCP is finished (s.info.status set).  Otherwise solves the QP,
// updates the l1 penalty weights, forms T(0) and its slope and prepares the
// first trial point (alpha = 1).
__device__ __forceinline__ bool sqp_check_body(const DevCtrl& c, const Ws& w, SqpState& s) {
  const int N = s.N;
  const int64_t ld = w.ld;
  const double s_max = 100.0;
  const bool has_r = (c.Ru != 0.0);
  if (has_r)  // input gradient r_k = 2 R_u (v_k - vbar_{k+1}) T_s at the current point
    for (int k = 0; k < N; ++k) w(QR, k) = c.r_scale * (w(U, k) - w(VB, k + 1));
  double kg, ke, mult1, gscale;
  bool pd;
  uint64_t lo, up;
  check_pass(N, ld, s.l > 0, s.alpha, has_r, c.vmin, c.vmax, ws_col(w, LAM), ws_col(w, PIL),
             ws_col(w, PIU), ws_col(w, EA), ws_col(w, EB), ws_col(w, EG), ws_col(w, EQ),
             ws_col(w, QR), ws_col(w, DU), ws_col(w, DX), ws_col(w, GLU), ws_col(w, GLX),
             ws_col(w, WXX), ws_col(w, WXU), ws_col(w, WUU), ws_col(w, U), ws_col(w, LB),
             ws_col(w, UB), kg, ke, mult1, pd, lo, up, gscale);
  if (s.l > 0 && !pd) {
    // a block is not positive definite: reset all of them to the identity
    for (int k = 0; k <= N; ++k) {
      w(WXX, k) = 1.0;
      w(WXU, k) = 0.0;
      w(WUU, k) = 1.0;
    }
    s.info.n_hess_reset++;
  }
  const double s_d = fmax(s_max, mult1 / (3.0 * N)) / s_max;
  kg /= s_d;
  s.info.kkt_grad = kg;
  s.info.kkt_eq = ke;
  s.info.f = s.f;
  if (kg <= c.sqp_tol && ke <= c.sqp_tol) {
    s.info.status = 0;
    return true;
  }
  if (s.l >= s.max_it) {
    s.info.status = 1;
    return true;
  }

  // QP subproblem at xi^[l] (bounds LB, UB and the starting working set from
  // the first pass)
  const QpResult qr = (c.qp_solver == 1)
                          ? qp_ipm(w, N, has_r, c.ip_max_it, c.ip_tol)
                          : qp_active_set_from(w, N, has_r, 10 * N + 20, lo, up, gscale);
  s.info.qp_iters += qr.iters;
  if (qr.status != 0) s.info.qp_fail++;
  s.info.iters++;

  // penalty weights (sigma update), the merit slope and the first trial point
  double pen, dfd;
  penalty_pass(N, ld, s.l == 0, has_r, c.vmin, c.vmax, ws_col(w, MU), ws_col(w, SIG),
               ws_col(w, EG), ws_col(w, EQ), ws_col(w, QR), ws_col(w, DU), ws_col(w, DX),
               ws_col(w, U), ws_col(w, X), ws_col(w, UT), ws_col(w, XT), pen, dfd);
  s.T0 = s.f + pen;
  s.DT0 = dfd - pen;
  s.alpha = 1.0;
  s.hv = 0;
  s.nc = 1;
  return false;
}

template <class R>
__device__ __forceinline__ void sqp_eval_trial(const DevModel& m, const DevCtrl& c, double EaR,
                                               const Ws& w, SqpState& s) {
  s.ft = evaluate<R>(m, c, EaR, s.N, w, UT, XT, TA, TB, TG, TQ, kRkAll);
  s.pt_ready = false;
  s.info.ls_trials++;
}

// The trial point's objective terms and q_k, and its penalty sigma^T |g| (the
// same sums, in the same order, as the objective pass and the Armijo test).
__device__ __forceinline__ void trial_objective_pass(
    int N, int64_t ld, double Qz, double Ts, double xs, double iV, double qf,
    const double* __restrict__ x_, const double* __restrict__ zb_, double* __restrict__ q_,
    const double* __restrict__ sig_, const double* __restrict__ g_, double& f, double& pt) {
  f = 0.0;
  pt = 0.0;
#pragma unroll 2
  for (int k = 0; k < N; ++k) {
    const int64_t o = k * ld;
    const double dz = x_[o + ld] * xs * iV - zb_[o + ld];
    f += Qz * dz * dz * Ts;
    q_[o + ld] = qf * dz;
    pt += sig_[o] * fabs(g_[o]);
  }
}

// The same trial evaluation after the warp has shot the intervals (the
// persistent schedule's pool): only the objective, q_k and the penalty, of
// line-search candidate q.
template <class R>
__device__ __forceinline__ void sqp_eval_trial_shot(const DevModel& m, const DevCtrl& c,
                                                    double EaR, const Ws& w, SqpState& s,
                                                    int q = 0) {
  const double xs = c.x_scale;
  const double qf = 2.0 * c.Qz * m.Ts * xs * m.iV;
  double f, pt;
  trial_objective_pass(s.N, w.ld, c.Qz, m.Ts, xs, m.iV, qf, ws_col(w, lsc_col(XT, q)),
                       ws_col(w, ZB), ws_col(w, lsc_col(TQ, q)), ws_col(w, SIG),
                       ws_col(w, lsc_col(TG, q)), f, pt);
  s.ft = f + objective_extra(m, c, s.N, w, lsc_col(UT, q), lsc_col(XT, q), lsc_col(TQ, q));
  s.pt = pt;
  s.pt_ready = true;
  s.info.ls_trials++;
}

// An accepted step, one pass over the stages: the multipliers step by alpha
// towards the QP's, the old-point Lagrangian gradient at the new multipliers
// (GLU, GLX; r at the old point) is kept for BFGS, and the trial point and its
// evaluation become current; the step actually taken (after the bound clip)
// is what BFGS sees.  lam of stage k+1 is stepped one stage ahead, since the
// x-gradient of stage k+1 needs it, and each old-point value is read before
// its stage's copy overwrites it.
__device__ __forceinline__ void accept_pass(
    int N, int64_t ld, double alpha, bool has_r, const double* __restrict__ mu_,
    const double* __restrict__ nul_, const double* __restrict__ nuu_,
    double* __restrict__ lam_, double* __restrict__ pil_, double* __restrict__ piu_,
    const double* __restrict__ r_, double* __restrict__ glu_, double* __restrict__ glx_,
    const double* __restrict__ ut_, double* __restrict__ u_, double* __restrict__ du_,
    const double* __restrict__ xt_, double* __restrict__ x_, const double* __restrict__ ta_,
    double* __restrict__ ea_, const double* __restrict__ tb_, double* __restrict__ eb_,
    const double* __restrict__ tg_, double* __restrict__ eg_, const double* __restrict__ tq_,
    double* __restrict__ eq_) {
  const double ialpha = 1.0 / alpha;  // alpha is a power of two: exact
  double lam = lam_[0] + alpha * (mu_[0] - lam_[0]);
#pragma unroll 2
  for (int k = 0; k < N; ++k) {
    const int64_t o = k * ld;
    lam_[o] = lam;
    const double pil = pil_[o] + alpha * (nul_[o] - pil_[o]);
    const double piu = piu_[o] + alpha * (nuu_[o] - piu_[o]);
    pil_[o] = pil;
    piu_[o] = piu;
    double glu = -lam * eb_[o] - pil + piu;
    if (has_r) glu += r_[o];
    double gx, lam_n = 0.0;
    if (k + 1 < N) {
      lam_n = lam_[o + ld] + alpha * (mu_[o + ld] - lam_[o + ld]);
      gx = eq_[o + ld] - lam_n * ea_[o + ld] + lam;
    } else {
      gx = eq_[o + ld] + lam;
    }
    glu_[o] = glu;
    glx_[o + ld] = gx;
    const double un = ut_[o];
    du_[o] = (un - u_[o]) * ialpha;
    u_[o] = un;
    x_[o + ld] = xt_[o + ld];
    ea_[o] = ta_[o];
    eb_[o] = tb_[o];
    eg_[o] = tg_[o];
    eq_[o + ld] = tq_[o + ld];
    lam = lam_n;
  }
}

// Armijo test of the evaluated trial point (line-search candidate q).  Returns
// 0 when the step was accepted (xi^[l+1] is current and evaluated; continue
// with sqp_check), 1 when the line search ran out of halvings (status 2; the
// OCP is finished at the current iterate), 2 when the step was halved
// (evaluate the new trial; its trial point is set up here when next_point).
__device__ __forceinline__ int sqp_trial_result_body(const DevCtrl& c, const Ws& w,
                                                     SqpState& s, int q = 0,
                                                     bool next_point = true) {
  const int N = s.N;
  const double c1 = 1e-4;
  double pt = 0.0;
  if (s.pt_ready) {
    pt = s.pt;
  } else {
    for (int k = 0; k < N; ++k) pt += w(SIG, k) * fabs(w(TG, k));
  }
  if (!(s.ft + pt <= s.T0 + c1 * s.alpha * s.DT0)) {
    if (s.hv >= c.ls_max) {
      s.info.status = 2;
      return 1;
    }
    s.hv++;
    s.alpha *= 0.5;
    if (next_point) sqp_trial_point(c, w, s);
    return 2;
  }
  const double alpha = s.alpha;
  accept_pass(N, w.ld, alpha, c.Ru != 0.0, ws_col(w, MU), ws_col(w, NUL), ws_col(w, NUU),
              ws_col(w, LAM), ws_col(w, PIL), ws_col(w, PIU), ws_col(w, QR), ws_col(w, GLU),
              ws_col(w, GLX), ws_col(w, lsc_col(UT, q)), ws_col(w, U), ws_col(w, DU),
              ws_col(w, lsc_col(XT, q)), ws_col(w, X), ws_col(w, lsc_col(TA, q)),
              ws_col(w, EA), ws_col(w, lsc_col(TB, q)), ws_col(w, EB),
              ws_col(w, lsc_col(TG, q)), ws_col(w, EG), ws_col(w, lsc_col(TQ, q)),
              ws_col(w, EQ));
  w(EPR, 0) = w(lsc_col(TPR, q), 0);
  w(EPR, 1) = w(lsc_col(TPR, q), 1);
  s.f = s.ft;
  s.l++;
  return 0;
}

// Code placement.  On the mixed-precision path the FP32 shooting is cheap and
// the FP64 phases dominate; compiled as separate functions they keep their
// own register allocation (measured 2.2x faster on the 30k study).  On the
// FP64 path inlining them is as fast or faster.
__device__ __noinline__ bool sqp_check_call(const DevCtrl& c, const Ws& w, SqpState& s) {
  return sqp_check_body(c, w, s);
}
__device__ __noinline__ int sqp_trial_result_call(const DevCtrl& c, const Ws& w, SqpState& s,
                                                  int q, bool next_point) {
  return sqp_trial_result_body(c, w, s, q, next_point);
}
template <class R>
__device__ __forceinline__ bool sqp_check(const DevCtrl& c, const Ws& w, SqpState& s) {
  if constexpr (sizeof(R) == 4) return sqp_check_call(c, w, s);
  else return sqp_check_body(c, w, s);
}
template <class R>
__device__ __forceinline__ int sqp_trial_result(const DevCtrl& c, const Ws& w, SqpState& s,
                                                int q = 0, bool next_point = true) {
  if constexpr (sizeof(R) == 4) return sqp_trial_result_call(c, w, s, q, next_point);
  else return sqp_trial_result_body(c, w, s, q, next_point);
}

// SQP of Sec. IV for one OCP, all phases in sequence.  Returns diagnostics;
// the solution (or the last iterate on failure) is left in U, X and the
// multipliers.  N and max_it default to the controller's.
template <class R>
__device__ __noinline__ SqpInfo sqp_solve(const DevModel& m, const DevCtrl& c, double EaR,
                                          double x0, const Ws& w, bool shifted_eval = false,
                                          int N = 0, int max_it = -1) {
  SqpState s;
  w(PIN, 0) = 0.0;  // no filter here: the prediction the shooting carries is unused
  sqp_start<R>(m, c, EaR, x0, w, N > 0 ? N : c.N, max_it >= 0 ? max_it : c.sqp_max_it,
               shifted_eval, s);
  while (!sqp_check<R>(c, w, s)) {
    int r;
    do {
      sqp_eval_trial<R>(m, c, EaR, w, s);
      r = sqp_trial_result<R>(c, w, s);
    } while (r == 2);
    if (r == 1) break;
  }
  return s.info;
}

}  // namespace mc
