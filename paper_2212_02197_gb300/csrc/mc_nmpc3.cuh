// mc_nmpc3.cuh -- the NMPC with the three-state model of Eq. (CSTR): CD-EKF
// on n = (n_A, n_B, n_T) with a 3x3 covariance, multiple-shooting OCP with
// three states and one input per stage, the SQP of Sec. IV (Riccati active-
// set QP with a 3x3 Riccati matrix, l1-merit line search, damped BFGS on
// 1/4/3-dimensional blocks, scaled convergence test).  FP64, one thread per
// trajectory.
//
// Scratch: structure of arrays as for the one-state NMPC, one array per
// component: w(X0 + i, k) is component i of x_k, symmetric 3x3 matrices keep
// their six entries (00, 01, 02, 11, 12, 22), A_k its nine (row-major).
#pragma once

#include "mc_closedloop.cuh"

namespace mc {

enum Arr3 : int {
  U3 = 0, X3 = 1 /* 3 */, LAM3 = 4 /* 3 */, PIL3 = 7, PIU3 = 8,
  WXX3 = 9 /* 6 */, WXU3 = 15 /* 3 */, WUU3 = 18,
  EA3 = 19 /* 9 */, EB3 = 28 /* 3 */, EG3 = 31 /* 3 */, EQ3 = 34,  // q_k: temperature part
  TA3 = 35 /* 9 */, TB3 = 44 /* 3 */, TG3 = 47 /* 3 */, TQ3 = 50, UT3 = 51, XT3 = 52 /* 3 */,
  DU3 = 55, DX3 = 56 /* 3 */, MU3 = 59 /* 3 */, NUL3 = 62, NUU3 = 63,
  SIG3 = 64 /* 3 */, GLU3 = 67, GLX3 = 68 /* 3 */, ZB3 = 71, LB3 = 72, UB3 = 73,
  RP3 = 74 /* 6 */, RPP3 = 80 /* 3 */, RK3 = 83 /* 3 */, RKF3 = 86, RZ3 = 87,
  kNArr3 = 88
};

// index of entry (i, j) of a symmetric 3x3 matrix stored as 00 01 02 11 12 22
__host__ __device__ constexpr int s3(int i, int j) {
  return (i <= j) ? (i == 0 ? j : (i == 1 ? 2 + j : 5)) : (j == 0 ? i : (j == 1 ? 2 + i : 5));
}

// ---------------------------------------------------------------------------
// Model: drift of Eq. (CSTR), its Jacobian J = df/dn and df/dF.  With
// r = k c_A c_B, k = k_0 exp(-g), g = (E_a/R) / c_T, the reaction term is
// S_p r V (S = (-1, -2, beta)) and its partials in n are (k c_B, k c_A,
// r g / c_T); one reciprocal, 1 / c_T, serves the whole evaluation.
__device__ __forceinline__ void drift3(const DevModel& m, double EaR, double T_in,
                                       const double n[3], double F, double f[3], double J[9],
                                       double fF[3]) {
  const double iV = m.iV;
  const double cA = n[0] * iV, cB = n[1] * iV, cT = n[2] * iV;
  const double iT = 1.0 / cT;
  const double g = EaR * iT;
  const double k = m.k0 * expr(-g);
  const double kcB = k * cB;
  const double r = kcB * cA;
  const double rV = r * m.V;
  const double S[3] = {-1.0, -2.0, m.beta};
  const double cin[3] = {m.cA_in, m.cB_in, T_in};
  const double c[3] = {cA, cB, cT};
  const double drv[3] = {kcB, k * cA, r * (g * iT)};
  const double nFiV = -(F * iV);
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    fF[p] = cin[p] - c[p];
    f[p] = fma(fF[p], F, S[p] * rV);
#pragma unroll
    for (int q = 0; q < 3; ++q) J[p * 3 + q] = (p == q) ? fma(S[p], drv[q], nFiV) : S[p] * drv[q];
  }
}

// F(x0, v) over Ts by n_rk4 RK4 steps of the drift (nominal T_in) and the
// sensitivities A = dF/dx0, B = dF/dv from the same RK4 steps applied to the
// variational equations.  States in moles, v in OCP units.
__device__ __noinline__ void rk4_interval3(const DevModel& m, double EaR, int n_rk4, double Ts,
                                           const double* x0, double v, double Fconv,
                                           double* xF, double* A, double* B) {
  const double h = Ts / (double)n_rk4;
  const double F = v * Fconv;
  double x[3], Phi[9], psi[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    x[i] = x0[i];
    psi[i] = 0.0;
#pragma unroll
    for (int j = 0; j < 3; ++j) Phi[i * 3 + j] = (i == j) ? 1.0 : 0.0;
  }
  for (int s = 0; s < n_rk4; ++s) {
    double ax[3] = {0, 0, 0}, aP[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, ap[3] = {0, 0, 0};
    double kx[3], kP[9], kp[3];
#pragma unroll
    for (int st = 0; st < 4; ++st) {
      const double a = (st == 0) ? 0.0 : ((st == 3) ? h : 0.5 * h);
      double xs[3], Ps[9], ps[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        xs[i] = x[i] + (st ? a * kx[i] : 0.0);
        ps[i] = psi[i] + (st ? a * kp[i] : 0.0);
#pragma unroll
        for (int j = 0; j < 3; ++j) Ps[i * 3 + j] = Phi[i * 3 + j] + (st ? a * kP[i * 3 + j] : 0.0);
      }
      double f[3], J[9], fF[3];
      drift3(m, EaR, m.T_in, xs, F, f, J, fF);
      const double wgt = (st == 0 || st == 3) ? 1.0 : 2.0;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        kx[i] = f[i];
        double sp = fF[i] * Fconv;
#pragma unroll
        for (int q = 0; q < 3; ++q) sp += J[i * 3 + q] * ps[q];
        kp[i] = sp;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          double sP = 0.0;
#pragma unroll
          for (int q = 0; q < 3; ++q) sP += J[i * 3 + q] * Ps[q * 3 + j];
          kP[i * 3 + j] = sP;
        }
      }
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        ax[i] += wgt * kx[i];
        ap[i] += wgt * kp[i];
      }
#pragma unroll
      for (int i = 0; i < 9; ++i) aP[i] += wgt * kP[i];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      x[i] = x[i] + h / 6.0 * ax[i];
      psi[i] = psi[i] + h / 6.0 * ap[i];
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) Phi[i] = Phi[i] + h / 6.0 * aP[i];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    xF[i] = x[i];
    B[i] = psi[i];
  }
#pragma unroll
  for (int i = 0; i < 9; ++i) A[i] = Phi[i];
}

// CD-EKF prediction for three states (P symmetric, six entries).
__device__ __noinline__ void ekf3_predict(const DevModel& m, double EaR, int n_rk4, double F, double x[3],
                             double P[6]) {
  const double h = m.Ts / (double)n_rk4;
  double Qd[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) Qd[i] = F * F * m.sigma[i] * m.sigma[i];
  for (int s = 0; s < n_rk4; ++s) {
    double ax[3] = {0, 0, 0}, aP[6] = {0, 0, 0, 0, 0, 0};
    double kx[3], kP[6];
#pragma unroll
    for (int st = 0; st < 4; ++st) {
      const double a = (st == 0) ? 0.0 : ((st == 3) ? h : 0.5 * h);
      double xs[3], Ps[6];
#pragma unroll
      for (int i = 0; i < 3; ++i) xs[i] = x[i] + (st ? a * kx[i] : 0.0);
#pragma unroll
      for (int i = 0; i < 6; ++i) Ps[i] = P[i] + (st ? a * kP[i] : 0.0);
      double f[3], J[9], fF[3];
      drift3(m, EaR, m.T_in, xs, F, f, J, fF);
#pragma unroll
      for (int i = 0; i < 3; ++i) kx[i] = f[i];
      // J P + P J^T + Q, entry (i, j), i <= j
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
          double v = (i == j) ? Qd[i] : 0.0;
#pragma unroll
          for (int q = 0; q < 3; ++q) v += J[i * 3 + q] * Ps[s3(q, j)] + Ps[s3(i, q)] * J[j * 3 + q];
          kP[s3(i, j)] = v;
        }
      const double wgt = (st == 0 || st == 3) ? 1.0 : 2.0;
#pragma unroll
      for (int i = 0; i < 3; ++i) ax[i] += wgt * kx[i];
#pragma unroll
      for (int i = 0; i < 6; ++i) aP[i] += wgt * kP[i];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) x[i] = x[i] + h / 6.0 * ax[i];
#pragma unroll
    for (int i = 0; i < 6; ++i) P[i] = P[i] + h / 6.0 * aP[i];
  }
}

// Filtering with y = n_T / V + v, Joseph form.
__device__ __noinline__ void ekf3_filter(const DevModel& m, double y, double x[3], double P[6]) {
  const double R = m.meas_sd * m.meas_sd;
  const double iV = 1.0 / m.V;
  double PC[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) PC[i] = P[s3(i, 2)] * iV;
  const double Re = R + iV * PC[2];
  double K[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) K[i] = PC[i] / Re;
  const double e = y - x[2] * iV;
#pragma unroll
  for (int i = 0; i < 3; ++i) x[i] = x[i] + K[i] * e;
  // M = I - K C (C = [0 0 1/V]); P = M P M^T + K R K^T
  double M[9], MP[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) M[i * 3 + j] = (i == j ? 1.0 : 0.0) - (j == 2 ? K[i] * iV : 0.0);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
#pragma unroll
      for (int q = 0; q < 3; ++q) s += M[i * 3 + q] * P[s3(q, j)];
      MP[i * 3 + j] = s;
    }
  double Pn[6];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      double s = 0.0;
#pragma unroll
      for (int q = 0; q < 3; ++q) s += MP[i * 3 + q] * M[j * 3 + q];
      Pn[s3(i, j)] = s + K[i] * R * K[j];
    }
#pragma unroll
  for (int i = 0; i < 6; ++i) P[i] = Pn[i];
}

// ---------------------------------------------------------------------------
// QP subproblem with three states per stage: Riccati recursion with P_{k+1}
// (3x3), p_{k+1}, K_k (1x3), k_k inside the primal active-set method of
// qp_active_set (same working-set rules).  Reads EA3, EB3, EG3 (b_k), WXX3,
// WXU3, WUU3, EQ3 (temperature part of q_k), LB3, UB3; writes DU3, DX3, MU3,
// NUL3, NUU3.  q_k and r_k are zero except the temperature part of q_k.

__device__ __noinline__ bool riccati3(const Ws& w, int N, uint64_t fixed) {
  double P[6], p[3];
#pragma unroll
  for (int i = 0; i < 6; ++i) P[i] = w(WXX3 + i, N);
  p[0] = 0.0;
  p[1] = 0.0;
  p[2] = w(EQ3, N);
  for (int k = N - 1; k >= 0; --k) {
    double A[9], B[3], b[3];
#pragma unroll
    for (int i = 0; i < 9; ++i) A[i] = (k > 0) ? w(EA3 + i, k) : 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      B[i] = w(EB3 + i, k);
      b[i] = w(EG3 + i, k);
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) w(RP3 + i, k + 1) = P[i];
#pragma unroll
    for (int i = 0; i < 3; ++i) w(RPP3 + i, k + 1) = p[i];
    // Pbp = P b + p, PB = P B
    double Pbp[3], PB[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      double s1 = p[i], s2 = 0.0;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        s1 += P[s3(i, q)] * b[q];
        s2 += P[s3(i, q)] * B[q];
      }
      Pbp[i] = s1;
      PB[i] = s2;
    }
    // A^T P A (symmetric)
    double AtPA[6];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i; j < 3; ++j) {
        double s = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int c2 = 0; c2 < 3; ++c2) s += A[a * 3 + i] * P[s3(a, c2)] * A[c2 * 3 + j];
        AtPA[s3(i, j)] = s;
      }
    double Pn[6], pn[3];
    const double q2 = (k > 0) ? w(EQ3, k) : 0.0;
    if ((fixed >> k) & 1ull) {
      const double c = w(DU3, k);
#pragma unroll
      for (int i = 0; i < 3; ++i) w(RK3 + i, k) = 0.0;
      w(RKF3, k) = c;
      // p_k = q_k + Wxu c + A^T (P (B c + b) + p)
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        double s = (i == 2 ? q2 : 0.0) + ((k > 0) ? w(WXU3 + i, k) * c : 0.0);
#pragma unroll
        for (int a = 0; a < 3; ++a) s += A[a * 3 + i] * (PB[a] * c + Pbp[a]);
        pn[i] = s;
      }
#pragma unroll
      for (int i = 0; i < 6; ++i) Pn[i] = ((k > 0) ? w(WXX3 + i, k) : 0.0) + AtPA[i];
    } else {
      double Rb = w(WUU3, k);
#pragma unroll
      for (int q = 0; q < 3; ++q) Rb += B[q] * PB[q];
      if (!(Rb > 0.0)) return false;
      const double iR = 1.0 / Rb;
      double Sb[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        double s = (k > 0) ? w(WXU3 + i, k) : 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a) s += A[a * 3 + i] * PB[a];
        Sb[i] = (k > 0) ? s : 0.0;
      }
      double sb = 0.0;
#pragma unroll
      for (int q = 0; q < 3; ++q) sb += B[q] * Pbp[q];
#pragma unroll
      for (int i = 0; i < 3; ++i) w(RK3 + i, k) = -Sb[i] * iR;
      w(RKF3, k) = -sb * iR;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        double s = (i == 2 ? q2 : 0.0) - Sb[i] * sb * iR;
#pragma unroll
        for (int a = 0; a < 3; ++a) s += A[a * 3 + i] * Pbp[a];
        pn[i] = s;
      }
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j)
          Pn[s3(i, j)] = ((k > 0) ? w(WXX3 + s3(i, j), k) : 0.0) + AtPA[s3(i, j)] -
                         Sb[i] * Sb[j] * iR;
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) P[i] = Pn[i];
#pragma unroll
    for (int i = 0; i < 3; ++i) p[i] = pn[i];
  }
  return true;
}

__device__ __noinline__ QpResult qp3_active_set(const Ws& w, int N, int max_it) {
  uint64_t lo = 0, up = 0;
  double gscale = 1.0;
  for (int k = 0; k < N; ++k) {
    const double lb = w(LB3, k), ub = w(UB3, k);
    double du = 0.0;
    if (lb >= 0.0) {
      lo |= 1ull << k;
      du = lb;
    } else if (ub <= 0.0) {
      up |= 1ull << k;
      du = ub;
    }
    w(DU3, k) = du;
    gscale = fmax(gscale, fabs(w(EQ3, k + 1)));
  }
  const double mult_tol = 1e-13 * gscale;
  QpResult res{0, 1};
  for (int it = 0; it < max_it; ++it) {
    res.iters = it + 1;
    const uint64_t fixed = lo | up;
    if (!riccati3(w, N, fixed)) {
      res.status = 2;
      return res;
    }
    double dx[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < N; ++k) {
      double z = w(RKF3, k);
#pragma unroll
      for (int i = 0; i < 3; ++i) z += w(RK3 + i, k) * dx[i];
      double dxn[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        double s = w(EB3 + i, k) * z + w(EG3 + i, k);
        if (k > 0)
#pragma unroll
          for (int q = 0; q < 3; ++q) s += w(EA3 + i * 3 + q, k) * dx[q];
        dxn[i] = s;
      }
      w(RZ3, k) = z;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        w(DX3 + i, k + 1) = dxn[i];
        double s = w(RPP3 + i, k + 1);
#pragma unroll
        for (int q = 0; q < 3; ++q) s += w(RP3 + s3(i, q), k + 1) * dxn[q];
        w(MU3 + i, k) = -s;
        dx[i] = dxn[i];
      }
    }
    double alpha = 1.0;
    int block = -1;
    bool block_lo = false;
    for (int k = 0; k < N; ++k) {
      if ((fixed >> k) & 1ull) continue;
      const double z = w(RZ3, k), du = w(DU3, k);
      const double lb = w(LB3, k), ub = w(UB3, k);
      const double pk = z - du;
      if (pk < 0.0 && z < lb) {
        const double t = (lb - du) / pk;
        if (t < alpha) { alpha = t; block = k; block_lo = true; }
      } else if (pk > 0.0 && z > ub) {
        const double t = (ub - du) / pk;
        if (t < alpha) { alpha = t; block = k; block_lo = false; }
      }
    }
    if (block >= 0) {
      if (alpha < 0.0) alpha = 0.0;
      for (int k = 0; k < N; ++k) {
        if ((fixed >> k) & 1ull) continue;
        const double du = w(DU3, k);
        w(DU3, k) = du + alpha * (w(RZ3, k) - du);
      }
      if (block_lo) {
        lo |= 1ull << block;
        w(DU3, block) = w(LB3, block);
      } else {
        up |= 1ull << block;
        w(DU3, block) = w(UB3, block);
      }
      continue;
    }
    int worst = -1;
    double worst_val = -mult_tol;
    for (int k = 0; k < N; ++k) {
      const bool f = (fixed >> k) & 1ull;
      const double du = f ? w(DU3, k) : w(RZ3, k);
      w(DU3, k) = du;
      if (!f) continue;
      double v = w(WUU3, k) * du;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        if (k > 0) v += w(WXU3 + i, k) * w(DX3 + i, k);
        v -= w(MU3 + i, k) * w(EB3 + i, k);
      }
      const double lam = ((lo >> k) & 1ull) ? v : -v;
      if (lam < worst_val) { worst_val = lam; worst = k; }
    }
    if (worst < 0) {
      res.status = 0;
      break;
    }
    lo &= ~(1ull << worst);
    up &= ~(1ull << worst);
  }
  for (int k = 0; k < N; ++k) {
    double nl = 0.0, nu = 0.0;
    if (((lo | up) >> k) & 1ull) {
      double v = w(WUU3, k) * w(DU3, k);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        if (k > 0) v += w(WXU3 + i, k) * w(DX3 + i, k);
        v -= w(MU3 + i, k) * w(EB3 + i, k);
      }
      if ((lo >> k) & 1ull) nl = v; else nu = -v;
    }
    w(NUL3, k) = nl;
    w(NUU3, k) = nu;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) w(DX3 + i, 0) = 0.0;
  return res;
}

// ---------------------------------------------------------------------------
// SQP for the three-state OCP.

// Shooting of interval k at (u_arr, x_arr) with sensitivities into (a_arr,
// b_arr, g_arr).  Not inlined: evaluate3 and the persistent schedule's pool
// (any lane shooting any lane's interval) run this one compiled body, so both
// give the same bits.
__device__ __noinline__ void shoot3_interval(const DevModel& m, const DevCtrl& c, double EaR,
                                             const Ws& w, int k, int u_arr, int x_arr,
                                             int a_arr, int b_arr, int g_arr) {
  const double xs = c.x_scale, ixs = 1.0 / c.x_scale;
  double n0[3], Fn[3], A[9], B[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) n0[i] = ((k == 0) ? w(X3 + i, 0) : w(x_arr + i, k)) * xs;
  rk4_interval3(m, EaR, c.n_rk4, m.Ts, n0, w(u_arr, k), c.Fconv, Fn, A, B);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    w(b_arr + i, k) = B[i] * ixs;
    w(g_arr + i, k) = Fn[i] * ixs - w(x_arr + i, k + 1);
  }
#pragma unroll
  for (int i = 0; i < 9; ++i) w(a_arr + i, k) = A[i];
}

// The objective at the states x_arr and the temperature part of q into
// q_arr (the intervals already shot); returns f.
__device__ __noinline__ double evaluate3_obj(const DevModel& m, const DevCtrl& c, int N,
                                             const Ws& w, int x_arr, int q_arr) {
  const double sz = c.x_scale * m.iV;
  double f = 0.0;
  w(q_arr, 0) = 0.0;
  for (int k = 1; k <= N; ++k) {
    const double dz = w(x_arr + 2, k) * sz - w(ZB3, k);
    f += c.Qz * dz * dz * m.Ts;
    w(q_arr, k) = 2.0 * c.Qz * dz * m.Ts * sz;
  }
  return f;
}

// Shooting of all intervals at (u_arr, x_arr) with sensitivities into
// (a_arr, b_arr, g_arr) and the temperature part of q into q_arr; returns f.
__device__ __forceinline__ double evaluate3(const DevModel& m, const DevCtrl& c, double EaR,
                                            int N, const Ws& w, int u_arr, int x_arr, int a_arr,
                                            int b_arr, int g_arr, int q_arr) {
  for (int k = 0; k < N; ++k) shoot3_interval(m, c, EaR, w, k, u_arr, x_arr, a_arr, b_arr, g_arr);
  return evaluate3_obj(m, c, N, w, x_arr, q_arr);
}

// damped BFGS of an n x n symmetric block held in registers (n <= 4)
__device__ __forceinline__ void bfgs_blockn(int n, double* W, const double* s, const double* y) {
  const double eps_m = 2.220446049250313e-16;
  double Ws[4], rr[4];
  double sWs = 0.0, sy = 0.0, sr = 0.0;
  for (int i = 0; i < n; ++i) {
    double t = 0.0;
    for (int j = 0; j < n; ++j) t += W[i * 4 + j] * s[j];
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
  const double isWs = 1.0 / sWs, isr = 1.0 / sr;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      W[i * 4 + j] = W[i * 4 + j] - Ws[i] * Ws[j] * isWs + rr[i] * rr[j] * isr;
}

__device__ __forceinline__ bool chol_pd(int n, const double* W) {
  double a[16];
  for (int i = 0; i < 16; ++i) a[i] = W[i];
  for (int j = 0; j < n; ++j) {
    double d = a[j * 4 + j];
    for (int k = 0; k < j; ++k) d -= a[j * 4 + k] * a[j * 4 + k];
    if (!(d > 0.0)) return false;
    d = sqrt(d);
    a[j * 4 + j] = d;
    const double id = 1.0 / d;
    for (int i = j + 1; i < n; ++i) {
      double s = a[i * 4 + j];
      for (int k = 0; k < j; ++k) s -= a[i * 4 + k] * a[j * 4 + k];
      a[i * 4 + j] = s * id;
    }
  }
  return true;
}

// W blocks in the scratch as 4x4 (stage k = 1..N-1: x then u), W_0 = [u],
// W_N = [x]; load / store them through these helpers.
__device__ __forceinline__ void load_block(const Ws& w, int k, int N, double* W) {
  for (int i = 0; i < 16; ++i) W[i] = 0.0;
  if (k == 0) {
    W[0] = w(WUU3, 0);
    return;
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) W[i * 4 + j] = w(WXX3 + s3(i, j), k);
  if (k < N) {
    for (int i = 0; i < 3; ++i) W[i * 4 + 3] = W[3 * 4 + i] = w(WXU3 + i, k);
    W[15] = w(WUU3, k);
  }
}
__device__ __forceinline__ void store_block(const Ws& w, int k, int N, const double* W) {
  if (k == 0) {
    w(WUU3, 0) = W[0];
    return;
  }
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) w(WXX3 + s3(i, j), k) = W[i * 4 + j];
  if (k < N) {
    for (int i = 0; i < 3; ++i) w(WXU3 + i, k) = W[i * 4 + 3];
    w(WUU3, k) = W[15];
  }
}
__device__ __forceinline__ void identity_blocks(const Ws& w, int N) {
  for (int k = 0; k <= N; ++k) {
    for (int i = 0; i < 6; ++i) w(WXX3 + i, k) = (i == 0 || i == 3 || i == 5) ? 1.0 : 0.0;
    for (int i = 0; i < 3; ++i) w(WXU3 + i, k) = 0.0;
    w(WUU3, k) = 1.0;
  }
}

// Gradient of the Lagrangian at the evaluation in (EA3, EB3, EQ3):
//   gu_k = -lam_k^T B_k - pil_k + piu_k, gx_k = q_k - A_k^T lam_k + lam_{k-1}.
__device__ __forceinline__ double lagr_gu(const Ws& w, int k) {
  double s = -w(PIL3, k) + w(PIU3, k);
  for (int i = 0; i < 3; ++i) s -= w(LAM3 + i, k) * w(EB3 + i, k);
  return s;
}
__device__ __forceinline__ double lagr_gx(const Ws& w, int k, int N, int i) {
  double s = (i == 2 ? w(EQ3, k) : 0.0) + w(LAM3 + i, k - 1);
  if (k < N)
    for (int a = 0; a < 3; ++a) s -= w(EA3 + a * 3 + i, k) * w(LAM3 + a, k);
  return s;
}

// Damped block BFGS on every block (s = alpha (du, dx), y = grad L at the
// new point minus grad L at the old point, both with the new multipliers);
// false when some block lost positive definiteness.
__device__ __noinline__ bool bfgs3_pass(const Ws& w, int N, double alpha) {
  bool pd = true;
  for (int k = 0; k <= N; ++k) {
    double W[16], s[4], y[4];
    load_block(w, k, N, W);
    int n;
    if (k == 0) {
      n = 1;
      s[0] = alpha * w(DU3, 0);
      y[0] = lagr_gu(w, 0) - w(GLU3, 0);
    } else {
      for (int i = 0; i < 3; ++i) {
        s[i] = alpha * w(DX3 + i, k);
        y[i] = lagr_gx(w, k, N, i) - w(GLX3 + i, k);
      }
      n = 3;
      if (k < N) {
        s[3] = alpha * w(DU3, k);
        y[3] = lagr_gu(w, k) - w(GLU3, k);
        n = 4;
      }
    }
    bfgs_blockn(n, W, s, y);
    store_block(w, k, N, W);
    pd = pd && chol_pd(n, W);
  }
  return pd;
}

// The SQP of Sec. IV for one three-state OCP, as resumable phases (as for the
// one-state OCP in mc_sqp.cuh):
//   sqp3_begin         W = I; the first evaluation at the warm start follows
//   sqp3_check         block BFGS, the scaled KKT test, the QP, the merit
//                      slope, and the first trial point
//   (shooting of the trial point)
//   sqp3_trial_result  Armijo test; accept and step, or halve the step
// sqp3_solve chains them for one OCP.
struct Sqp3State {
  int N, max_it, l, hv;
  double f, ft, alpha, T0, DT0;
  SqpInfo info;
};

__device__ __forceinline__ void sqp3_begin(const Ws& w, int N, int max_it, Sqp3State& st) {
  identity_blocks(w, N);
  st.N = N;
  st.max_it = max_it;
  st.l = 0;
  st.hv = 0;
  st.f = st.ft = st.alpha = st.T0 = st.DT0 = 0.0;
  st.info = SqpInfo{};
}

// Trial point xi + alpha dxi (u clipped into its bounds against rounding).
__device__ __forceinline__ void sqp3_trial_point(const DevCtrl& c, const Ws& w,
                                                 const Sqp3State& st) {
  for (int k = 0; k < st.N; ++k) {
    w(UT3, k) = fmin(fmax(w(U3, k) + st.alpha * w(DU3, k), c.vmin), c.vmax);
    for (int i = 0; i < 3; ++i)
      w(XT3 + i, k + 1) = w(X3 + i, k + 1) + st.alpha * w(DX3 + i, k + 1);
  }
}

// Top of an SQP iteration at xi^[l] (evaluated, f in st.f).  Returns true when
// the OCP is finished (st.info.status set); else prepares the first trial.
__device__ __noinline__ bool sqp3_check(const DevCtrl& c, const Ws& w, Sqp3State& st) {
  const int N = st.N;
  const double s_max = 100.0;
  if (st.l > 0 && !bfgs3_pass(w, N, st.alpha)) {
    identity_blocks(w, N);
    st.info.n_hess_reset++;
  }
  // scaled convergence test
  double mult1 = 0.0, kg = 0.0, ke = 0.0;
  for (int k = 0; k < N; ++k) {
    mult1 += fabs(w(PIL3, k)) + fabs(w(PIU3, k));
    for (int i = 0; i < 3; ++i) mult1 += fabs(w(LAM3 + i, k));
    kg = fmax(kg, fabs(lagr_gu(w, k)));
    for (int i = 0; i < 3; ++i) {
      kg = fmax(kg, fabs(lagr_gx(w, k + 1, N, i)));
      ke = fmax(ke, fabs(w(EG3 + i, k)));
    }
  }
  const double s_d = fmax(s_max, mult1 / (5.0 * N)) / s_max;
  kg /= s_d;
  st.info.kkt_grad = kg;
  st.info.kkt_eq = ke;
  st.info.f = st.f;
  if (kg <= c.sqp_tol && ke <= c.sqp_tol) {
    st.info.status = 0;
    return true;
  }
  if (st.l >= st.max_it) {
    st.info.status = 1;
    return true;
  }
  // QP at xi^[l]
  for (int k = 0; k < N; ++k) {
    const double u = w(U3, k);
    w(LB3, k) = c.vmin - u;
    w(UB3, k) = c.vmax - u;
  }
  const QpResult qr = qp3_active_set(w, N, 10 * N + 20);
  st.info.qp_iters += qr.iters;
  if (qr.status != 0) st.info.qp_fail++;
  st.info.iters++;
  double pen = 0.0, dfd = 0.0;
  for (int k = 0; k < N; ++k)
    for (int i = 0; i < 3; ++i) {
      const double am = fabs(w(MU3 + i, k));
      const double sg = (st.l == 0) ? am : fmax(am, 0.5 * (w(SIG3 + i, k) + am));
      w(SIG3 + i, k) = sg;
      pen += sg * fabs(w(EG3 + i, k));
    }
  for (int k = 1; k <= N; ++k) dfd += w(EQ3, k) * w(DX3 + 2, k);
  st.T0 = st.f + pen;
  st.DT0 = dfd - pen;
  st.alpha = 1.0;
  st.hv = 0;
  sqp3_trial_point(c, w, st);
  return false;
}

// Armijo test of the evaluated trial point (st.ft; its shooting in TA3, TB3,
// TG3, TQ3).  Returns 0 when the step was accepted (continue with
// sqp3_check), 1 when the line search ran out of halvings (status 2; the OCP
// is finished at the current iterate), 2 when the step was halved (evaluate
// the new trial point).
__device__ __noinline__ int sqp3_trial_result(const DevCtrl& c, const Ws& w, Sqp3State& st) {
  const int N = st.N;
  const double c1 = 1e-4;
  st.info.ls_trials++;
  double pt = 0.0;
  for (int k = 0; k < N; ++k)
    for (int i = 0; i < 3; ++i) pt += w(SIG3 + i, k) * fabs(w(TG3 + i, k));
  if (!(st.ft + pt <= st.T0 + c1 * st.alpha * st.DT0)) {
    st.alpha *= 0.5;
    st.hv++;
    if (st.hv > c.ls_max) {
      st.info.status = 2;
      return 1;
    }
    sqp3_trial_point(c, w, st);
    return 2;
  }
  const double alpha = st.alpha;
  // multipliers, old-point gradient at the new multipliers, accept the point
  for (int k = 0; k < N; ++k) {
    for (int i = 0; i < 3; ++i)
      w(LAM3 + i, k) = w(LAM3 + i, k) + alpha * (w(MU3 + i, k) - w(LAM3 + i, k));
    w(PIL3, k) = w(PIL3, k) + alpha * (w(NUL3, k) - w(PIL3, k));
    w(PIU3, k) = w(PIU3, k) + alpha * (w(NUU3, k) - w(PIU3, k));
  }
  for (int k = 0; k < N; ++k) {
    w(GLU3, k) = lagr_gu(w, k);
    for (int i = 0; i < 3; ++i) w(GLX3 + i, k + 1) = lagr_gx(w, k + 1, N, i);
  }
  const double ialpha = 1.0 / alpha;  // alpha is a power of two: exact
  for (int k = 0; k < N; ++k) {
    const double un = w(UT3, k);
    w(DU3, k) = (un - w(U3, k)) * ialpha;
    w(U3, k) = un;
    for (int i = 0; i < 3; ++i) {
      w(DX3 + i, k + 1) = (w(XT3 + i, k + 1) - w(X3 + i, k + 1)) * ialpha;
      w(X3 + i, k + 1) = w(XT3 + i, k + 1);
      w(EB3 + i, k) = w(TB3 + i, k);
      w(EG3 + i, k) = w(TG3 + i, k);
    }
    for (int i = 0; i < 9; ++i) w(EA3 + i, k) = w(TA3 + i, k);
    w(EQ3, k + 1) = w(TQ3, k + 1);
  }
  st.f = st.ft;
  st.l++;
  return 0;
}

// One three-state OCP from the warm start in (U3, X3, LAM3, PIL3, PIU3) with
// x_0 in X3(., 0) and the set-points in ZB3.
__device__ __noinline__ SqpInfo sqp3_solve(const DevModel& m, const DevCtrl& c, double EaR,
                                           const Ws& w, int N, int max_it) {
  Sqp3State st;
  sqp3_begin(w, N, max_it, st);
  st.f = evaluate3(m, c, EaR, N, w, U3, X3, EA3, EB3, EG3, EQ3);
  while (!sqp3_check(c, w, st)) {
    int r;
    do {
      st.ft = evaluate3(m, c, EaR, N, w, UT3, XT3, TA3, TB3, TG3, TQ3);
      r = sqp3_trial_result(c, w, st);
    } while (r == 2);
    if (r == 1) break;
  }
  return st.info;
}

// ---------------------------------------------------------------------------
// Closed loop with the three-state NMPC (plant, measurement, Phi as in
// traj_nmpc; FP64 only), split into the steps both schedules share.

struct Nmpc3Traj {
  uint32_t j;
  int i;                   // current sample
  TrajParams tp;
  double n[3], xh[3], P[6], F_prev, phi;
  TrajOut out;
};

__device__ __forceinline__ void nmpc3_begin(const DevModel& m, const DevCtrl& c, uint32_t j,
                                            const Ws& w, Nmpc3Traj& T) {
  T.j = j;
  T.i = 0;
  T.tp = traj_params(m, c, j);
  const int N = T.tp.N;
  T.n[0] = m.cA_in * m.V;
  T.n[1] = m.cB_in * m.V;
  T.n[2] = m.T_in * m.V;
  for (int q = 0; q < 3; ++q) T.xh[q] = T.n[q];
  T.P[0] = c.P0; T.P[1] = 0.0; T.P[2] = 0.0; T.P[3] = c.P0; T.P[4] = 0.0; T.P[5] = c.P0;
  T.F_prev = 0.0;
  T.phi = 0.0;
  T.out = TrajOut{};
  double v0 = Fss(m, T.tp.EaR_c, zbar_at(m, 0)) / c.Fconv;
  v0 = fmin(fmax(v0, c.vmin), c.vmax);
  for (int k = 0; k < N; ++k) {
    w(U3, k) = v0;
    w(PIL3, k) = 0.0;
    w(PIU3, k) = 0.0;
    for (int i = 0; i < 3; ++i) w(LAM3 + i, k) = 0.0;
  }
  for (int k = 0; k <= N; ++k)
    for (int i = 0; i < 3; ++i) w(X3 + i, k) = T.xh[i] / c.x_scale;
}

// Sample i: Phi term, and unless the trajectory ends there the measurement,
// the CD-EKF and the start of the OCP (its first evaluation is the caller's).
// Returns false when the trajectory is finished (T.out is final).
__device__ __noinline__ bool nmpc3_sample(const DevModel& m, const DevCtrl& c, const Ws& w,
                                          Nmpc3Traj& T, Sqp3State& st) {
  const int N = T.tp.N, K = m.n_steps, i = T.i;
  const double cT = T.n[2] / m.V;
  bool bad = !isfinite(cT);
  for (int q = 0; q < 3; ++q) bad = bad || !isfinite(T.xh[q]);
  for (int q = 0; q < 6; ++q) bad = bad || !isfinite(T.P[q]);
  if (bad) {
    T.out.cnt[6] = 1;
    T.out.phi = nan("");
    return false;
  }
  const double ez = cT - zbar_at(m, i);
  T.phi += ez * ez;
  if (i == K) {
    T.out.phi = T.phi / (double)(K + 1);
    return false;
  }
  const double y = cT + m.meas_sd * meas_noise<double>(m, T.j, (uint32_t)i);
  if (i > 0) ekf3_predict(m, T.tp.EaR_c, c.n_rk4, T.F_prev, T.xh, T.P);
  ekf3_filter(m, y, T.xh, T.P);
  for (int k = 1; k <= N; ++k) w(ZB3, k) = zbar_at(m, i + k);
  for (int q = 0; q < 3; ++q) w(X3 + q, 0) = T.xh[q] / c.x_scale;
  sqp3_begin(w, N, T.tp.max_it, st);
  return true;
}

// After the OCP of sample i: count it, apply u_0, shift the warm start,
// simulate the plant to t_{i+1}.
__device__ __noinline__ void nmpc3_apply(const DevModel& m, const DevCtrl& c, const Ws& w,
                                         Nmpc3Traj& T, const SqpInfo& si) {
  const int N = T.tp.N;
  T.out.cnt[0] += (si.status == 1);
  T.out.cnt[1] += si.iters;
  T.out.cnt[2] += si.ls_trials;
  T.out.cnt[3] += si.n_hess_reset;
  T.out.cnt[4] += (si.status == 2);
  T.out.cnt[5] += si.qp_iters;
  T.out.cnt[7] += si.qp_fail;
  const double F = w(U3, 0) * c.Fconv;
  for (int k = 0; k < N - 1; ++k) {
    w(U3, k) = w(U3, k + 1);
    w(PIL3, k) = w(PIL3, k + 1);
    w(PIU3, k) = w(PIU3, k + 1);
    for (int q = 0; q < 3; ++q) {
      w(X3 + q, k + 1) = w(X3 + q, k + 2);
      w(LAM3 + q, k) = w(LAM3 + q, k + 1);
    }
  }
  plant_interval<double>(m, T.tp, T.j, T.i, F, T.n);
  T.F_prev = F;
  T.i++;
}

// Static schedule: one trajectory per thread, the OCPs run to completion.
__device__ TrajOut traj_nmpc3(const DevModel& m, const DevCtrl& c, uint32_t j, const Ws& w) {
  Nmpc3Traj T;
  Sqp3State st;
  nmpc3_begin(m, c, j, w, T);
  while (nmpc3_sample(m, c, w, T, st)) {
    st.f = evaluate3(m, c, T.tp.EaR_c, st.N, w, U3, X3, EA3, EB3, EG3, EQ3);
    while (!sqp3_check(c, w, st)) {
      int r;
      do {
        st.ft = evaluate3(m, c, T.tp.EaR_c, st.N, w, UT3, XT3, TA3, TB3, TG3, TQ3);
        r = sqp3_trial_result(c, w, st);
      } while (r == 2);
      if (r == 1) break;
    }
    nmpc3_apply(m, c, w, T, st.info);
  }
  return T.out;
}

// Persistent schedule, as nmpc_persistent for the one-state NMPC: every lane
// runs its cheap phases until it needs shooting (a trial point, or the first
// evaluation of a new OCP), then the warp shoots all pending intervals as one
// pool, interval-major, lane t taking jobs t, t + 32, ...; each job is one
// call of shoot3_interval, so the results are those of the static schedule
// bit for bit.  Every lane of the warp must call this; the block is one warp.
enum Lane3Phase : int { k3New = 0, k3Sample = 1, k3Check = 2, k3Trial = 3, k3Start = 4, k3Done = 5 };

struct Pool3Tab {
  unsigned mask[MC_MAX_HORIZON];  // lanes with a job at position i
  int pref[MC_MAX_HORIZON];       // jobs before position i
  double EaR[32];
  int trial[32];
};

__device__ __forceinline__ void pool3_shoot(const DevModel& m, const DevCtrl& c, const Ws& w,
                                            int n_jobs, bool trial, double EaR, Pool3Tab& tab) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int max_jobs = (int)__reduce_max_sync(full, (unsigned)n_jobs);
  __syncwarp();  // the previous round's readers of tab are done
  tab.EaR[lane] = EaR;
  tab.trial[lane] = trial ? 1 : 0;
  int total = 0;
  for (int i = 0; i < max_jobs; ++i) {
    const unsigned mi = __ballot_sync(full, n_jobs > i);
    if (lane == 0) {
      tab.mask[i] = mi;
      tab.pref[i] = total;
    }
    total += __popc(mi);
  }
  __syncwarp();  // tab and the owners' points are visible to every lane
  for (int q = lane; q < total; q += 32) {
    int lo = 0, hi = max_jobs;  // pref[lo] <= q < pref[hi], pref[max_jobs] = total
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (tab.pref[mid] <= q) lo = mid;
      else hi = mid;
    }
    unsigned mo = tab.mask[lo];
    for (int r = q - tab.pref[lo]; r > 0; --r) mo &= mo - 1u;
    const int o = __ffs(mo) - 1;
    const bool tr = tab.trial[o] != 0;
    const Ws wo{w.p + (o - lane), w.ld, w.N1};
    shoot3_interval(m, c, tab.EaR[o], wo, lo, tr ? UT3 : U3, tr ? XT3 : X3, tr ? TA3 : EA3,
                    tr ? TB3 : EB3, tr ? TG3 : EG3);
  }
  __syncwarp();  // the shot intervals are visible to their owners
}

__device__ void nmpc3_persistent(const DevModel& m, const DevCtrl& c, const Ws& w, int64_t j0,
                                 int64_t n, const uint32_t* __restrict__ order,
                                 unsigned long long* next, double* __restrict__ phi_out,
                                 int32_t* __restrict__ cnt_out) {
  __shared__ Pool3Tab tab;  // one per block: the kernel runs one warp per block
  Nmpc3Traj T;
  Sqp3State st;
  int phase = k3New;
  for (;;) {
    while (phase != k3Trial && phase != k3Start && phase != k3Done) {
      if (phase == k3New) {
        const unsigned long long q = atomicAdd(next, 1ull);
        if (q >= (unsigned long long)n) {
          phase = k3Done;
          break;
        }
        const uint32_t j = order ? order[q] : (uint32_t)(j0 + (int64_t)q);
        nmpc3_begin(m, c, j, w, T);
        phase = k3Sample;
      }
      if (phase == k3Sample) {
        if (nmpc3_sample(m, c, w, T, st)) {
          phase = k3Start;
        } else {
          phi_out[T.j] = T.out.phi;
#pragma unroll
          for (int q = 0; q < kNCounters; ++q)
            cnt_out[(int64_t)T.j * kNCounters + q] = T.out.cnt[q];
          phase = k3New;
        }
        continue;
      }
      if (phase == k3Check) {
        if (sqp3_check(c, w, st)) {
          nmpc3_apply(m, c, w, T, st.info);
          phase = k3Sample;
        } else {
          phase = k3Trial;
        }
      }
    }
    if (!__ballot_sync(0xffffffffu, phase != k3Done)) break;
    const int n_jobs = (phase == k3Trial || phase == k3Start) ? st.N : 0;
    pool3_shoot(m, c, w, n_jobs, phase == k3Trial, T.tp.EaR_c, tab);
    if (phase == k3Start) {
      st.f = evaluate3_obj(m, c, st.N, w, X3, EQ3);
      phase = k3Check;
    } else if (phase == k3Trial) {
      st.ft = evaluate3_obj(m, c, st.N, w, XT3, TQ3);
      const int r = sqp3_trial_result(c, w, st);
      if (r == 0) {
        phase = k3Check;
      } else if (r == 1) {
        nmpc3_apply(m, c, w, T, st.info);
        phase = k3Sample;
      }
    }
  }
}

}  // namespace mc
