// mc_qp.cuh -- the structured QP subproblem of the SQP, Eq. (QP-subproblem)
// with the stage costs of Eq. (nlpsqp_qp), for one state and one input:
//
//   min  sum_k 1/2 [dx_k; du_k]^T W_k [dx_k; du_k] + q_k dx_k + r_k du_k
//   s.t. dx_{k+1} = A_k dx_k + B_k du_k + b_k,  dx_0 = 0,  lb_k <= du_k <= ub_k,
//
// solved per thread by a Riccati recursion over the horizon.  Two solvers:
//
//   qp_active_set  primal active-set method; each iteration solves the
//                  equality-constrained LQ problem with the working-set inputs
//                  fixed at their bounds by one backward Riccati sweep and one
//                  forward sweep (dx, du, mu).  Exact finite termination.
//   qp_ipm         the paper's choice (Sec. IV-A): primal-dual interior point
//                  (Mehrotra predictor-corrector) whose Newton systems are the
//                  same Riccati sweeps with barrier-augmented input weights.
//
// Per-thread arrays live in the structure-of-arrays scratch `Ws`: element k of
// array a of the thread's trajectory is at p[(a * (N+1) + k) * ld], so the 32
// lanes of a warp touch 32 consecutive doubles for every access.
#pragma once

#include "mc_device.cuh"

namespace mc {

// Line-search candidates the persistent schedule may shoot in one round when
// it backtracks (candidate 0 is the trial point itself).
constexpr int kLsCand = 4;

enum Arr : int {
  U, X, LAM, PIL, PIU,            // SQP iterate and warm start
  WXX, WXU, WUU,                  // block-BFGS Hessian blocks
  EA, EB, EG, EQ,                 // A_k, B_k, g_k = F_k - x_{k+1}, q_k = df/dx_k
  TA, TB, TG, TQ, UT, XT,         // line-search trial point and its evaluation
  DU, DX, MU, NUL, NUU,           // QP solution
  SIG, GLU, GLX, ZB,              // merit weights, old Lagrangian gradient, set-points
  LB, UB, QR,                     // QP bounds and input gradient r_k
  RP, RPP, RK, RKF, RZ,           // Riccati factors P_{k+1}, p_{k+1}, K_k, k_k; trial du
  TL, TU, ZL, ZU, DUA, RIR, RSB,  // IPM slacks, duals, affine du, 1/Rbar, Sbar
  DXS, DMS,                       // IPM step in dx and mu
  VB,                             // steady-state inputs vbar_k of the set-points (R_u term)
  PIN, TPR, EPR,                  // P_{i|i} (row 0); the CD-EKF prediction (x, P in rows 0,
                                  // 1) carried by the interval-0 shooting: trial, current
  LSC,                            // line-search candidates 1 .. kLsCand-1: 7 columns each,
                                  // as UT, XT, TA, TB, TG, TQ, TPR
  kNArr = LSC + 7 * (kLsCand - 1)
};

// Column a (one of UT, XT, TA, TB, TG, TQ, TPR) of line-search candidate q.
__host__ __device__ constexpr int lsc_col(int a, int q) {
  return q == 0 ? a
                : LSC + 7 * (q - 1) +
                      (a == UT ? 0 : a == XT ? 1 : a == TA ? 2 : a == TB ? 3 : a == TG ? 4
                                                  : a == TQ ? 5 : 6);
}

struct Ws {
  double* p;
  int64_t ld;
  int N1;
  MC_HD double& operator()(int a, int k) const {
    return p[(int64_t)(a * N1 + k) * ld];
  }
};

// 1/x for the recursions below: on the device the Newton-refined hardware
// reciprocal (rcp_newton: four dependent operations on the pipe instead of a
// division's longer sequence, on the Riccati recursion's critical path), on
// the host the division.
MC_HD double recip(double x) {
#ifdef __CUDA_ARCH__
  return rcp_newton(x);
#else
  return 1.0 / x;
#endif
}

struct QpResult {
  int iters;
  int status;  // 0 solved, 1 iteration limit, 2 not positive definite
};

// Backward Riccati sweep for the LQ problem with stage input weight
// Rt_k = Wuu_k + extra_k, linear terms (qk, rk) and dynamics offset bk, with
// the inputs in `fixed` held at the value w(DU, k).  Stores P_{k+1}, p_{k+1},
// K_k, k_k; returns false on a non-positive pivot.
// The three functors give rk (input gradient), bk (dynamics offset) and the
// extra diagonal input weight of stage k.
template <class RkF, class BkF, class QkF, class ExtraF>
MC_HD bool riccati_backward(const Ws& w, int N, uint64_t fixed, RkF rk_of,
                                                 BkF bk_of, QkF qk_of, ExtraF extra_of,
                                                 bool store_factors) {
  double P = w(WXX, N), p = qk_of(N);
  for (int k = N - 1; k >= 0; --k) {
    const double A = (k > 0) ? w(EA, k) : 0.0;
    const double B = w(EB, k);
    const double b = bk_of(k);
    const double Pbp = P * b + p;
    w(RP, k + 1) = P;
    w(RPP, k + 1) = p;
    double Pn = 0.0, pn = 0.0;
    if ((fixed >> k) & 1ull) {
      const double c = w(DU, k);
      w(RK, k) = 0.0;
      w(RKF, k) = c;
      if (k > 0) {
        Pn = w(WXX, k) + A * A * P;
        pn = qk_of(k) + w(WXU, k) * c + A * (P * (B * c) + Pbp);
      }
    } else {
      const double Rb = w(WUU, k) + extra_of(k) + B * B * P;
      if (!(Rb > 0.0)) return false;
      const double iR = recip(Rb);
      const double Sb = (k > 0) ? w(WXU, k) + A * P * B : 0.0;
      const double sb = rk_of(k) + B * Pbp;
      w(RK, k) = -Sb * iR;
      w(RKF, k) = -sb * iR;
      if (store_factors) {
        w(RIR, k) = iR;
        w(RSB, k) = Sb;
      }
      if (k > 0) {
        Pn = w(WXX, k) + A * A * P - Sb * Sb * iR;
        pn = qk_of(k) + A * Pbp - Sb * sb * iR;
      }
    }
    P = Pn;
    p = pn;
  }
  return true;
}

// ---------------------------------------------------------------------------
// Primal active-set method.  Reads EA, EB, EG (= b), WXX, WXU, WUU, EQ (= q),
// QR (= r, if has_r), LB, UB; writes DU, DX, MU, NUL, NUU.
//
// The arrays are handed to the solver as separate columns (element k of a
// column at c[k * ld]) through restrict-qualified pointers: they are disjoint
// rows of the scratch, and saying so lets the compiler issue the loads of the
// next stages while the stores of the current one are pending.  The recursions
// are latency-bound per lane, so this overlap, not the arithmetic, sets their
// speed.  Same operations as the plain formulation, stage by stage.
MC_HD double* ws_col(const Ws& w, int a) { return w.p + (int64_t)a * w.N1 * w.ld; }

// Backward Riccati sweep of the active-set method (input weight Wuu, inputs in
// `fixed` held at du): stores P_{k+1}, p_{k+1}, K_k, k_k; false on a pivot <= 0.
MC_HD bool as_backward(int N, int64_t ld, uint64_t fixed, bool has_r,
                       const double* __restrict__ A_, const double* __restrict__ B_,
                       const double* __restrict__ b_, const double* __restrict__ q_,
                       const double* __restrict__ r_, const double* __restrict__ Wxx,
                       const double* __restrict__ Wxu, const double* __restrict__ Wuu,
                       const double* __restrict__ du_, double* __restrict__ P_,
                       double* __restrict__ p_, double* __restrict__ K_,
                       double* __restrict__ kf_) {
  double P = Wxx[N * ld], p = q_[N * ld];
#pragma unroll 2
  for (int k = N - 1; k >= 0; --k) {
    const int64_t o = k * ld;
    const double A = (k > 0) ? A_[o] : 0.0;
    const double B = B_[o];
    const double b = b_[o];
    const double Pbp = P * b + p;
    P_[o + ld] = P;
    p_[o + ld] = p;
    double Pn = 0.0, pn = 0.0;
    if ((fixed >> k) & 1ull) {
      const double c = du_[o];
      K_[o] = 0.0;
      kf_[o] = c;
      if (k > 0) {
        Pn = Wxx[o] + A * A * P;
        pn = q_[o] + Wxu[o] * c + A * (P * (B * c) + Pbp);
      }
    } else {
      const double Rb = Wuu[o] + B * B * P;
      if (!(Rb > 0.0)) return false;
      const double iR = recip(Rb);
      const double Sb = (k > 0) ? Wxu[o] + A * P * B : 0.0;
      const double sb = (has_r ? r_[o] : 0.0) + B * Pbp;
      K_[o] = -Sb * iR;
      kf_[o] = -sb * iR;
      if (k > 0) {
        Pn = Wxx[o] + A * A * P - Sb * Sb * iR;
        pn = q_[o] + A * Pbp - Sb * sb * iR;
      }
    }
    P = Pn;
    p = pn;
  }
  return true;
}

// Forward sweep (subspace minimiser z, states, dynamics multipliers) fused with
// the ratio test over the free inputs and with the working set's bound
// multipliers: returns the blocking stage (-1 if none), its side and the step
// length alpha.  On the free stages du becomes z and the previous du is kept
// in z_ (the caller steps from it by alpha when a bound blocks).  On the fixed
// stages the multiplier of the active bound comes from stationarity in du_k
// at (dx_k, mu_k), all at hand in the sweep; nul, nuu receive them (0 on free
// stages) and worst the stage with the most negative one below -mult_tol (-1:
// none).  They are the QP's when nothing blocks and none is negative.
MC_HD int as_forward(int N, int64_t ld, uint64_t fixed, uint64_t lo, bool has_r,
                     double mult_tol, const double* __restrict__ A_,
                     const double* __restrict__ B_, const double* __restrict__ b_,
                     const double* __restrict__ P_, const double* __restrict__ p_,
                     const double* __restrict__ K_, const double* __restrict__ kf_,
                     const double* __restrict__ lb_, const double* __restrict__ ub_,
                     const double* __restrict__ r_, const double* __restrict__ Wxu,
                     const double* __restrict__ Wuu, double* __restrict__ du_,
                     double* __restrict__ z_, double* __restrict__ dx_,
                     double* __restrict__ mu_, double* __restrict__ nul_,
                     double* __restrict__ nuu_, double& alpha, bool& block_lo, int& worst) {
  double dx = 0.0;
  alpha = 1.0;
  int block = -1;
  block_lo = false;
  worst = -1;
  double worst_val = -mult_tol;
#pragma unroll 2
  for (int k = 0; k < N; ++k) {
    const int64_t o = k * ld;
    const double A = (k > 0) ? A_[o] : 0.0;
    const double B = B_[o];
    const double z = K_[o] * dx + kf_[o];
    const double dxn = A * dx + B * z + b_[o];
    const double mu = -(P_[o + ld] * dxn + p_[o + ld]);
    dx_[o + ld] = dxn;
    mu_[o] = mu;
    const double du = du_[o];
    double nl = 0.0, nu = 0.0;
    if ((fixed >> k) & 1ull) {
      const double cross = (k > 0) ? Wxu[o] * dx : 0.0;
      const double v = Wuu[o] * du + cross + (has_r ? r_[o] : 0.0) - mu * B;
      const bool at_lo = (lo >> k) & 1ull;
      const double lam = at_lo ? v : -v;
      if (lam < worst_val) { worst_val = lam; worst = k; }
      if (at_lo) nl = v; else nu = -v;
    } else {
      z_[o] = du;
      du_[o] = z;
      const double lb = lb_[o], ub = ub_[o];
      const double pk = z - du;
      if (pk < 0.0 && z < lb) {
        const double t = (lb - du) / pk;
        if (t < alpha) { alpha = t; block = k; block_lo = true; }
      } else if (pk > 0.0 && z > ub) {
        const double t = (ub - du) / pk;
        if (t < alpha) { alpha = t; block = k; block_lo = false; }
      }
    }
    nul_[o] = nl;
    nuu_[o] = nu;
    dx = dxn;
  }
  return block;
}

// Working set at the start (bounds active at the current iterate, du on them)
// and the scale of the multiplier test.
MC_HD double as_init(int N, int64_t ld, bool has_r, const double* __restrict__ lb_,
                     const double* __restrict__ ub_, const double* __restrict__ q_,
                     const double* __restrict__ r_, double* __restrict__ du_, uint64_t& lo,
                     uint64_t& up) {
  lo = 0;
  up = 0;
  double gscale = 1.0;
#pragma unroll 2
  for (int k = 0; k < N; ++k) {
    const int64_t o = k * ld;
    const double lb = lb_[o], ub = ub_[o];
    double du = 0.0;
    if (lb >= 0.0) {
      lo |= 1ull << k;
      du = lb;
    } else if (ub <= 0.0) {
      up |= 1ull << k;
      du = ub;
    }
    du_[o] = du;
    gscale = fmax(gscale, fabs(q_[o + ld]));
    if (has_r) gscale = fmax(gscale, fabs(r_[o]));
  }
  return gscale;
}

// Bound multipliers from stationarity in du at the final working set.
MC_HD void as_bound_multipliers(int N, int64_t ld, uint64_t lo, uint64_t up, bool has_r,
                                const double* __restrict__ B_, const double* __restrict__ r_,
                                const double* __restrict__ Wxu, const double* __restrict__ Wuu,
                                const double* __restrict__ du_, const double* __restrict__ dx_,
                                const double* __restrict__ mu_, double* __restrict__ nul_,
                                double* __restrict__ nuu_) {
#pragma unroll 2
  for (int k = 0; k < N; ++k) {
    const int64_t o = k * ld;
    double nl = 0.0, nu = 0.0;
    if (((lo | up) >> k) & 1ull) {
      const double cross = (k > 0) ? Wxu[o] * dx_[o] : 0.0;
      const double v = Wuu[o] * du_[o] + cross + (has_r ? r_[o] : 0.0) - mu_[o] * B_[o];
      if ((lo >> k) & 1ull) nl = v; else nu = -v;
    }
    nul_[o] = nl;
    nuu_[o] = nu;
  }
}

// The active-set method from a given starting working set (lo, up), with du
// already on the active bounds and gscale the scale of the multiplier test.
MC_HD QpResult qp_active_set_from(const Ws& w, int N, bool has_r, int max_it, uint64_t lo,
                                  uint64_t up, double gscale) {
  const int64_t ld = w.ld;
  const double *A_ = ws_col(w, EA), *B_ = ws_col(w, EB), *b_ = ws_col(w, EG),
               *q_ = ws_col(w, EQ), *r_ = ws_col(w, QR), *Wxx = ws_col(w, WXX),
               *Wxu = ws_col(w, WXU), *Wuu = ws_col(w, WUU), *lb_ = ws_col(w, LB),
               *ub_ = ws_col(w, UB);
  double *du_ = ws_col(w, DU), *dx_ = ws_col(w, DX), *mu_ = ws_col(w, MU),
         *nul_ = ws_col(w, NUL), *nuu_ = ws_col(w, NUU), *P_ = ws_col(w, RP),
         *p_ = ws_col(w, RPP), *K_ = ws_col(w, RK), *kf_ = ws_col(w, RKF), *z_ = ws_col(w, RZ);
  const double mult_tol = 1e-13 * gscale;

  QpResult res{0, 1};
  for (int it = 0; it < max_it; ++it) {
    res.iters = it + 1;
    const uint64_t fixed = lo | up;
    if (!as_backward(N, ld, fixed, has_r, A_, B_, b_, q_, r_, Wxx, Wxu, Wuu, du_, P_, p_, K_,
                     kf_)) {
      res.status = 2;
      return res;
    }
    double alpha;
    bool block_lo;
    int worst;
    const int block = as_forward(N, ld, fixed, lo, has_r, mult_tol, A_, B_, b_, P_, p_, K_,
                                 kf_, lb_, ub_, r_, Wxu, Wuu, du_, z_, dx_, mu_, nul_, nuu_,
                                 alpha, block_lo, worst);
    if (block >= 0) {
      // step from the previous du (kept in z_) towards z (now in du_)
      if (alpha < 0.0) alpha = 0.0;
      for (int k = 0; k < N; ++k) {
        if ((fixed >> k) & 1ull) continue;
        const int64_t o = k * ld;
        const double du = z_[o];
        du_[o] = du + alpha * (du_[o] - du);
      }
      if (block_lo) {
        lo |= 1ull << block;
        du_[block * ld] = lb_[block * ld];
      } else {
        up |= 1ull << block;
        du_[block * ld] = ub_[block * ld];
      }
      continue;
    }
    if (worst < 0) {
      res.status = 0;
      break;
    }
    lo &= ~(1ull << worst);
    up &= ~(1ull << worst);
  }
  // the forward sweep wrote the bound multipliers of an optimal working set;
  // at the iteration limit they follow from the last one
  if (res.status != 0)
    as_bound_multipliers(N, ld, lo, up, has_r, B_, r_, Wxu, Wuu, du_, dx_, mu_, nul_, nuu_);
  dx_[0] = 0.0;
  return res;
}

// The active-set method started at the bounds active at the current iterate.
MC_HD QpResult qp_active_set(const Ws& w, int N, bool has_r, int max_it) {
  uint64_t lo, up;
  const double gscale = as_init(N, w.ld, has_r, ws_col(w, LB), ws_col(w, UB), ws_col(w, EQ),
                                ws_col(w, QR), ws_col(w, DU), lo, up);
  return qp_active_set_from(w, N, has_r, max_it, lo, up, gscale);
}

// ---------------------------------------------------------------------------
// Primal-dual interior point (Mehrotra predictor-corrector).  Slacks
// tl = du - lb, tu = ub - du and their duals zl, zu; each Newton system reduces
// to the LQ problem with input weight Wuu + zl/tl + zu/tu, solved by the same
// Riccati sweeps.  Same inputs/outputs as qp_active_set.
MC_HD QpResult qp_ipm(const Ws& w, int N, bool has_r, int max_it,
                                           double tol) {
  auto rk_of = [&](int k) { return has_r ? w(QR, k) : 0.0; };
  double scale = 1.0;
  for (int k = 0; k < N; ++k) {
    const double lb = w(LB, k), ub = w(UB, k);
    // start at the centre of the box with unit duals
    const double wid = fmax(ub - lb, 1e-8);
    const double du0 = 0.5 * (lb + ub);
    w(DU, k) = du0;
    w(TL, k) = fmax(du0 - lb, 0.5 * wid);
    w(TU, k) = fmax(ub - du0, 0.5 * wid);
    w(ZL, k) = 1.0;
    w(ZU, k) = 1.0;
    w(MU, k) = 0.0;
    scale = fmax(scale, fabs(w(EQ, k + 1)));
    scale = fmax(scale, fabs(rk_of(k)));
  }
  // states consistent with the initial du
  {
    double dx = 0.0;
    w(DX, 0) = 0.0;
    for (int k = 0; k < N; ++k) {
      const double A = (k > 0) ? w(EA, k) : 0.0;
      dx = A * dx + w(EB, k) * w(DU, k) + w(EG, k);
      w(DX, k + 1) = dx;
    }
  }
  // residuals of the KKT conditions at stage k (see the derivation above)
  auto r_u = [&](int k) {
    const double cross = (k > 0) ? w(WXU, k) * w(DX, k) : 0.0;
    return w(WUU, k) * w(DU, k) + cross + rk_of(k) - w(MU, k) * w(EB, k) - w(ZL, k) + w(ZU, k);
  };
  auto r_x = [&](int k) {  // k = 1..N
    if (k == N) return w(WXX, N) * w(DX, N) + w(EQ, N) + w(MU, N - 1);
    return w(WXX, k) * w(DX, k) + w(WXU, k) * w(DU, k) + w(EQ, k) - w(MU, k) * w(EA, k) +
           w(MU, k - 1);
  };
  auto r_d = [&](int k) {
    const double A = (k > 0) ? w(EA, k) : 0.0;
    return A * w(DX, k) + w(EB, k) * w(DU, k) + w(EG, k) - w(DX, k + 1);
  };
  auto r_l = [&](int k) { return w(DU, k) - w(LB, k) - w(TL, k); };
  auto r_r = [&](int k) { return w(UB, k) - w(DU, k) - w(TU, k); };
  auto extra = [&](int k) { return w(ZL, k) / w(TL, k) + w(ZU, k) / w(TU, k); };

  QpResult res{0, 1};
  const double inv2N = 1.0 / (2.0 * N);
  for (int it = 0; it <= max_it; ++it) {
    double gap = 0.0, rmax = 0.0;
    for (int k = 0; k < N; ++k) {
      gap += w(TL, k) * w(ZL, k) + w(TU, k) * w(ZU, k);
      rmax = fmax(rmax, fmax(fabs(r_u(k)), fabs(r_d(k))));
      rmax = fmax(rmax, fmax(fabs(r_l(k)), fabs(r_r(k))));
      rmax = fmax(rmax, fabs(r_x(k + 1)));
    }
    const double mu_c = gap * inv2N;
    if (rmax <= tol * scale && mu_c <= tol * scale) {
      res.status = 0;
      break;
    }
    if (it == max_it) break;
    res.iters = it + 1;

    // predictor: complementarity target 0
    auto rho_u_aff = [&](int k) {
      const double tl = w(TL, k), tu = w(TU, k), zl = w(ZL, k), zu = w(ZU, k);
      return r_u(k) + (tl * zl + zl * r_l(k)) / tl - (tu * zu + zu * r_r(k)) / tu;
    };
    auto rx_of = [&](int k) { return r_x(k); };
    if (!riccati_backward(w, N, 0ull, rho_u_aff, r_d, rx_of, extra, true)) {
      res.status = 2;
      return res;
    }
    double dx = 0.0;
    double a_aff = 1.0;
    for (int k = 0; k < N; ++k) {
      const double A = (k > 0) ? w(EA, k) : 0.0;
      const double du = w(RK, k) * dx + w(RKF, k);
      dx = A * dx + w(EB, k) * du + r_d(k);
      w(DUA, k) = du;
      const double tl = w(TL, k), tu = w(TU, k), zl = w(ZL, k), zu = w(ZU, k);
      const double dtl = du + r_l(k), dtu = r_r(k) - du;
      const double dzl = (-tl * zl - zl * dtl) / tl, dzu = (-tu * zu - zu * dtu) / tu;
      if (dtl < 0.0) a_aff = fmin(a_aff, -tl / dtl);
      if (dtu < 0.0) a_aff = fmin(a_aff, -tu / dtu);
      if (dzl < 0.0) a_aff = fmin(a_aff, -zl / dzl);
      if (dzu < 0.0) a_aff = fmin(a_aff, -zu / dzu);
    }
    double gap_aff = 0.0;
    for (int k = 0; k < N; ++k) {
      const double du = w(DUA, k);
      const double tl = w(TL, k), tu = w(TU, k), zl = w(ZL, k), zu = w(ZU, k);
      const double dtl = du + r_l(k), dtu = r_r(k) - du;
      const double dzl = (-tl * zl - zl * dtl) / tl, dzu = (-tu * zu - zu * dtu) / tu;
      gap_aff += (tl + a_aff * dtl) * (zl + a_aff * dzl) + (tu + a_aff * dtu) * (zu + a_aff * dzu);
    }
    const double ratio = gap_aff / gap;
    const double smu = ratio * ratio * ratio * mu_c;

    // corrector: rho_c = t z + dt_aff dz_aff - sigma mu
    auto rho_c = [&](int k, double& rcl, double& rcu) {
      const double du = w(DUA, k);
      const double tl = w(TL, k), tu = w(TU, k), zl = w(ZL, k), zu = w(ZU, k);
      const double dtl = du + r_l(k), dtu = r_r(k) - du;
      const double dzl = (-tl * zl - zl * dtl) / tl, dzu = (-tu * zu - zu * dtu) / tu;
      rcl = tl * zl + dtl * dzl - smu;
      rcu = tu * zu + dtu * dzu - smu;
    };
    // vector-only backward sweep reusing the stored factors (RIR, RSB, RP)
    {
      double p = r_x(N);
      for (int k = N - 1; k >= 0; --k) {
        const double A = (k > 0) ? w(EA, k) : 0.0;
        const double B = w(EB, k);
        const double P = w(RP, k + 1);
        w(RPP, k + 1) = p;
        const double Pbp = P * r_d(k) + p;
        double rcl, rcu;
        rho_c(k, rcl, rcu);
        const double tl = w(TL, k), tu = w(TU, k), zl = w(ZL, k), zu = w(ZU, k);
        const double ru = r_u(k) + (rcl + zl * r_l(k)) / tl - (rcu + zu * r_r(k)) / tu;
        const double sb = ru + B * Pbp;
        const double iR = w(RIR, k);
        w(RKF, k) = -sb * iR;
        // keep the corrector rhs of the complementarity for the recovery below
        w(RZ, k) = rcl;
        w(DXS, k) = rcu;
        if (k > 0) p = r_x(k) + A * Pbp - w(RSB, k) * sb * iR;
      }
    }
    // forward sweep, then one common step length
    dx = 0.0;
    double amax = 1.0;
    for (int k = 0; k < N; ++k) {
      const double A = (k > 0) ? w(EA, k) : 0.0;
      const double du = w(RK, k) * dx + w(RKF, k);
      const double dxn = A * dx + w(EB, k) * du + r_d(k);
      const double dmu = -(w(RP, k + 1) * dxn + w(RPP, k + 1));
      const double tl = w(TL, k), tu = w(TU, k), zl = w(ZL, k), zu = w(ZU, k);
      const double rcl = w(RZ, k), rcu = w(DXS, k);
      const double dtl = du + r_l(k), dtu = r_r(k) - du;
      const double dzl = (-rcl - zl * dtl) / tl, dzu = (-rcu - zu * dtu) / tu;
      if (dtl < 0.0) amax = fmin(amax, -tl / dtl);
      if (dtu < 0.0) amax = fmin(amax, -tu / dtu);
      if (dzl < 0.0) amax = fmin(amax, -zl / dzl);
      if (dzu < 0.0) amax = fmin(amax, -zu / dzu);
      w(DUA, k) = du;
      w(DXS, k) = dxn;   // (rcu no longer needed)
      w(DMS, k) = dmu;
      w(RZ, k) = dtl;
      w(RP, k) = dzl;    // stage k's factor P_k is not needed any more this iteration
      w(RIR, k) = dzu;
      dx = dxn;
    }
    double alpha = fmin(1.0, 0.995 * amax);
    // keep the iterate in the wide neighbourhood t_i z_i >= 1e-3 mu of the
    // central path (without it Mehrotra steps can bounce between the bounds of
    // a narrow box)
    for (int bt = 0; bt < 30; ++bt) {
      double g = 0.0, pmin = INFINITY;
      for (int k = 0; k < N; ++k) {
        const double tl = w(TL, k) + alpha * w(RZ, k);
        const double tu = w(TU, k) + alpha * (r_r(k) - w(DUA, k));
        const double zl = w(ZL, k) + alpha * w(RP, k);
        const double zu = w(ZU, k) + alpha * w(RIR, k);
        g += tl * zl + tu * zu;
        pmin = fmin(pmin, fmin(tl * zl, tu * zu));
      }
      if (pmin >= 1e-3 * g * inv2N) break;
      alpha *= 0.8;
    }
    for (int k = 0; k < N; ++k) {
      const double du = w(DUA, k);
      const double dtu = r_r(k) - du;  // uses the old du and tu
      w(TL, k) = w(TL, k) + alpha * w(RZ, k);
      w(TU, k) = w(TU, k) + alpha * dtu;
      w(ZL, k) = w(ZL, k) + alpha * w(RP, k);
      w(ZU, k) = w(ZU, k) + alpha * w(RIR, k);
      w(DU, k) = w(DU, k) + alpha * du;
      w(DX, k + 1) = w(DX, k + 1) + alpha * w(DXS, k);
      w(MU, k) = w(MU, k) + alpha * w(DMS, k);
    }
  }
  for (int k = 0; k < N; ++k) {
    w(NUL, k) = w(ZL, k);
    w(NUU, k) = w(ZU, k);
  }
  return res;
}

}  // namespace mc
