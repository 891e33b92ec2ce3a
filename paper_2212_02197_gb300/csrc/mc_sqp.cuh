// mc_sqp.cuh -- the NMPC regulator of Sec. III-B solved by the SQP of Sec. IV,
// and one whole NMPC closed-loop trajectory (Sec. VII), per thread.
//
// NLP (Eq. OCP_NLP) in scaled variables: OCP state x = n_T / x_scale, OCP
// input v with flow F = v Fconv; decision vector [v_0, x_1, ..., v_{N-1}, x_N];
// constraints g_k = F_k - x_{k+1}; Lagrangian
//   L = f - lam^T g - pil^T (v - v_min) - piu^T (v_max - v).
#pragma once

#include "mc_qp.cuh"

namespace mc {

struct SqpInfo {
  int iters, status, ls_trials, qp_iters, n_hess_reset, qp_fail;
  double kkt_grad, kkt_eq, f;
};

// Shooting of all N intervals at the point (u_arr, x_arr) with sensitivities,
// writing A_k, B_k, g_k and q_k into (a_arr, b_arr, g_arr, q_arr); returns the
// objective f = sum_k Q_z (z_k - zbar_k)^2 T_s.  With reuse_mid the intervals
// 1 .. N-2 keep the A_k, B_k, g_k already in the arrays: after the receding-
// horizon shift they are the previous OCP's values at the same (x_k, u_k), so
// only the first and the last interval are integrated again.
// R is the arithmetic of the RK4 integration (FP32 on the mixed-precision
// path); the constraint residual g_k, the objective and its gradient are FP64.
template <class R>
__device__ __forceinline__ double evaluate(const DevModel& m, const DevCtrl& c, double EaR,
                                           double x0, const Ws& w, int u_arr, int x_arr,
                                           int a_arr, int b_arr, int g_arr, int q_arr,
                                           bool reuse_mid = false) {
  const int N = c.N;
  const double xs = c.x_scale, ixs = 1.0 / c.x_scale;
  const double qf = 2.0 * c.Qz * m.Ts * xs * m.iV;
  double f = 0.0;
  double xk = x0;
  for (int k = 0; k < N; ++k) {
    const double xn = w(x_arr, k + 1);
    if (!(reuse_mid && k >= 1 && k <= N - 2)) {
      R Fn, a, b;
      rk4_interval<R, true>(m, (R)EaR, c.n_rk4, (R)m.Ts, (R)(xk * xs), (R)w(u_arr, k),
                            (R)c.Fconv, Fn, a, b);
      w(a_arr, k) = (double)a;
      w(b_arr, k) = (double)b * ixs;
      w(g_arr, k) = (double)Fn * ixs - xn;
    }
    const double dz = xn * xs * m.iV - w(ZB, k + 1);
    f += c.Qz * dz * dz * m.Ts;
    w(q_arr, k + 1) = qf * dz;
    xk = xn;
  }
  return f;
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
  const double isWs = 1.0 / sWs, isr = 1.0 / sr;
  w11 = w11 - Ws1 * Ws1 * isWs + r1 * r1 * isr;
  if (n == 2) {
    w12 = w12 - Ws1 * Ws2 * isWs + r1 * r2 * isr;
    w22 = w22 - Ws2 * Ws2 * isWs + r2 * r2 * isr;
  }
}

// SQP of Sec. IV for one OCP from the warm start in (U, X, LAM, PIL, PIU); the
// set-points z-bar(t_{i+k}) are in ZB[1..N].  Returns diagnostics; the
// solution (or the last iterate on failure) is left in U, X and the multipliers.
// With shifted_eval the evaluation arrays hold the previous OCP's final
// evaluation shifted by one interval (see evaluate).  R is the shooting
// arithmetic; everything else (QP, merit, BFGS, convergence test) is FP64.
template <class R>
__device__ __noinline__ SqpInfo sqp_solve(const DevModel& m, const DevCtrl& c, double EaR,
                                          double x0, const Ws& w, bool shifted_eval = false) {
  const int N = c.N;
  const double c1 = 1e-4, s_max = 100.0;
  SqpInfo info{};
  for (int k = 0; k <= N; ++k) {
    w(WXX, k) = 1.0;
    w(WXU, k) = 0.0;
    w(WUU, k) = 1.0;
  }
  w(X, 0) = x0;
  double f = evaluate<R>(m, c, EaR, x0, w, U, X, EA, EB, EG, EQ, shifted_eval);
  double alpha = 0.0;
  int nqp = 0;
  for (int l = 0;; ++l) {
    // gradient of the Lagrangian at the current iterate and multipliers
    double kg = 0.0, ke = 0.0, mult1 = 0.0;
    for (int k = 0; k < N; ++k) {
      const double lam = w(LAM, k), pil = w(PIL, k), piu = w(PIU, k);
      mult1 += fabs(lam) + fabs(pil) + fabs(piu);
      const double gu = -lam * w(EB, k) - pil + piu;
      double gx;
      if (k + 1 < N)
        gx = w(EQ, k + 1) - w(LAM, k + 1) * w(EA, k + 1) + lam;
      else
        gx = w(EQ, N) + lam;
      if (l > 0) {
        // damped block BFGS with s = alpha (du, dx) and
        // y = grad L(xi^[l], .) - grad L(xi^[l-1], .) at the new multipliers
        const double su = alpha * w(DU, k), sx = alpha * w(DX, k);
        const double yu = gu - w(GLU, k), yx = (k > 0) ? w(GLX, k) : 0.0;
        double w11, w12, w22;
        if (k == 0) {
          w11 = w(WUU, 0);
          w12 = 0.0;
          w22 = 0.0;
          bfgs_block(1, w11, w12, w22, su, 0.0, yu, 0.0);
          w(WUU, 0) = w11;
        } else {
          w11 = w(WXX, k);
          w12 = w(WXU, k);
          w22 = w(WUU, k);
          bfgs_block(2, w11, w12, w22, sx, su, yx, yu);
          w(WXX, k) = w11;
          w(WXU, k) = w12;
          w(WUU, k) = w22;
        }
        if (k == N - 1) {
          double wn = w(WXX, N), d0 = 0.0, d1 = 0.0;
          bfgs_block(1, wn, d0, d1, alpha * w(DX, N), 0.0, gx - w(GLX, N), 0.0);
          w(WXX, N) = wn;
        }
        // keep the new-point x-gradient of stage k+1 for its block
        w(GLX, k + 1) = gx - w(GLX, k + 1);
      }
      kg = fmax(kg, fmax(fabs(gu), fabs(gx)));
    }
    if (l > 0) {
      // positive definiteness of every block, else reset all to the identity
      bool pd = w(WUU, 0) > 0.0 && w(WXX, N) > 0.0;
      for (int k = 1; k < N; ++k) {
        const double a = w(WXX, k), b = w(WXU, k), d = w(WUU, k);
        pd = pd && (a > 0.0) && (d - b * b / a > 0.0);
      }
      if (!pd) {
        for (int k = 0; k <= N; ++k) {
          w(WXX, k) = 1.0;
          w(WXU, k) = 0.0;
          w(WUU, k) = 1.0;
        }
        info.n_hess_reset++;
      }
    }
    const double s_d = fmax(s_max, mult1 / (3.0 * N)) / s_max;
    kg /= s_d;
    for (int k = 0; k < N; ++k) ke = fmax(ke, fabs(w(EG, k)));
    info.kkt_grad = kg;
    info.kkt_eq = ke;
    info.f = f;
    if (kg <= c.sqp_tol && ke <= c.sqp_tol) {
      info.status = 0;
      break;
    }
    if (l >= c.sqp_max_it) {
      info.status = 1;
      break;
    }

    // QP subproblem at xi^[l]
    for (int k = 0; k < N; ++k) {
      const double u = w(U, k);
      w(LB, k) = c.vmin - u;
      w(UB, k) = c.vmax - u;
    }
    QpResult qr = (c.qp_solver == 1) ? qp_ipm(w, N, false, c.ip_max_it, c.ip_tol)
                                     : qp_active_set(w, N, false, 10 * N + 20);
    info.qp_iters += qr.iters;
    if (qr.status != 0) info.qp_fail++;
    ++nqp;

    // penalty weights (sigma update) and the merit slope
    double pen = 0.0, dfd = 0.0;
    for (int k = 0; k < N; ++k) {
      const double am = fabs(w(MU, k));
      const double sg = (l == 0) ? am : fmax(am, 0.5 * (w(SIG, k) + am));
      w(SIG, k) = sg;
      pen += sg * fabs(w(EG, k));
      dfd += w(EQ, k + 1) * w(DX, k + 1);
    }
    const double T0 = f + pen;
    const double DT0 = dfd - pen;

    // backtracking line search on the Armijo condition
    alpha = 1.0;
    bool accepted = false;
    double ft = 0.0;
    for (int hv = 0; hv <= c.ls_max; ++hv) {
      for (int k = 0; k < N; ++k) {
        w(UT, k) = fmin(fmax(w(U, k) + alpha * w(DU, k), c.vmin), c.vmax);
        w(XT, k + 1) = w(X, k + 1) + alpha * w(DX, k + 1);
      }
      ft = evaluate<R>(m, c, EaR, x0, w, UT, XT, TA, TB, TG, TQ);
      info.ls_trials++;
      double pt = 0.0;
      for (int k = 0; k < N; ++k) pt += w(SIG, k) * fabs(w(TG, k));
      if (ft + pt <= T0 + c1 * alpha * DT0) {
        accepted = true;
        break;
      }
      alpha *= 0.5;
    }
    if (!accepted) {
      info.status = 2;
      break;
    }

    // step in the multipliers; old-point Lagrangian gradient at the new multipliers
    for (int k = 0; k < N; ++k) {
      const double lam = w(LAM, k) + alpha * (w(MU, k) - w(LAM, k));
      const double pil = w(PIL, k) + alpha * (w(NUL, k) - w(PIL, k));
      const double piu = w(PIU, k) + alpha * (w(NUU, k) - w(PIU, k));
      w(LAM, k) = lam;
      w(PIL, k) = pil;
      w(PIU, k) = piu;
    }
    for (int k = 0; k < N; ++k) {
      const double lam = w(LAM, k);
      w(GLU, k) = -lam * w(EB, k) - w(PIL, k) + w(PIU, k);
      double gx;
      if (k + 1 < N)
        gx = w(EQ, k + 1) - w(LAM, k + 1) * w(EA, k + 1) + lam;
      else
        gx = w(EQ, N) + lam;
      w(GLX, k + 1) = gx;
    }
    // accept the trial point and its evaluation; the step actually taken
    // (after the bound clip) is what BFGS sees
    for (int k = 0; k < N; ++k) {
      const double un = w(UT, k);
      w(DU, k) = (un - w(U, k)) / alpha;
      w(U, k) = un;
      w(X, k + 1) = w(XT, k + 1);
      w(EA, k) = w(TA, k);
      w(EB, k) = w(TB, k);
      w(EG, k) = w(TG, k);
      w(EQ, k + 1) = w(TQ, k + 1);
    }
    f = ft;
  }
  info.iters = nqp;
  return info;
}

}  // namespace mc
