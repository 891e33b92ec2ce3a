// mc_grad_nmpc.cuh -- gradient of Phi_j with respect to the NMPC weights
// (Q_z, R_u, Q_n) of the extended objective, through the closed loop.
//
// Model of the derivative: every OCP is represented by its solution map
// u_0 = U(x-hat_{i|i}, theta) at the KKT point the SQP returns, differentiated
// implicitly (the tangent of a KKT point solves the equality-constrained QP
// whose Hessian is that of the Lagrangian and whose linear term is the
// derivative of the Lagrangian gradient with respect to the parameter, with
// the active bounds held); the plant (Euler-Maruyama), the measurement and
// the CD-EKF (prediction and Joseph filter) are differentiated exactly, in
// forward mode, three directions at once.  The warm start of the next OCP does
// not enter (the KKT point does not depend on it).  FP64, one thread per
// trajectory, in either of two ways that give the same bits:
//   static      traj_nmpc_grad carries the tangents along the static
//               schedule's closed loop;
//   persistent  the persistent schedule's closed loop records, per sample, the
//               state the tangents start from and the OCP's KKT point
//               (Recorder), and traj_nmpc_tangent then propagates the tangents
//               through the recorded samples, every lane of a warp on the
//               same sample (the tangent work has no data-dependent length).
#pragma once

#include "mc_closedloop.cuh"
#include "mc_nmpc3.cuh"

namespace mc {

// One-state model with second derivatives: f, f_x, f_F, f_xx, f_xF.
//   f = F (T_in - c_T) + beta r(c_T) V,  c_T = x / V,  r = k c_A c_B,
//   k = k0 exp(-E/c_T), c_A = c_A,in + (T_in - c_T)/beta, c_B = c_B,in + 2 (T_in - c_T)/beta;
//   f_x = (-F + beta V r') / V, f_xx = beta r'' / V, f_F = T_in - c_T, f_xF = -1/V,
//   r' = k' c_A c_B + k (c_A' c_B + c_A c_B'),
//   r'' = k'' c_A c_B + 2 k' (c_A' c_B + c_A c_B') + 2 k c_A' c_B',
//   k' = k E / c_T^2, k'' = k E (E - 2 c_T) / c_T^4.
// Evaluated with one reciprocal and k0 in the exponent, as model1 does: with
// g = E / c_T and i = 1 / c_T, k' = k g i and k'' = k g i^2 (g - 2);
// c_A' c_B + c_A c_B' = -(c_B + 2 c_A) / beta = -(rw0 + rw1 d) for
// d = T_in - c_T; 2 c_A' c_B' = rw1.
__device__ __forceinline__ void model1_d2(const DevModel& m, double EaR, double x, double F,
                                          double& f, double& fx, double& fF, double& fxx,
                                          double& fxF) {
  const double cT = x * m.iV;
  const double d = fma(-x, m.iV, m.T_in);
  const double iT = rcp_newton(cT);
  const double g = EaR * iT;
  const double k = expr(fma(-EaR, iT, m.lnk0));
  const double cA = fma(d, m.ib, m.cA_in), cB = fma(d, m.ib2, m.cB_in);
  const double p = cA * cB;
  const double r = k * p;
  const double ibw = fma(m.rw1, d, m.rw0);
  const double k1 = k * (g * iT);
  const double k2 = k1 * (iT * (g - 2.0));
  const double r1 = fma(k1, p, -(k * ibw));
  const double r2 = fma(k2, p, fma(-2.0 * k1, ibw, k * m.rw1));
  f = fma(m.bV, r, F * d);
  fx = fma(m.beta, r1, -(F * m.iV));
  fF = d;
  fxx = m.beta * r2 * m.iV;
  fxF = -m.iV;
}

// One shooting interval (n_rk4 RK4 steps) with first- and second-order
// forward sensitivities of the end state with respect to x0 and v, obtained
// by differentiating every RK4 stage twice.
// The results come back by value (references would put the caller's variables
// in local memory).
struct D2 {
  double xF, a, b, aa, ab, bb;
};

__device__ __noinline__ D2 rk4_interval_d2(const DevModel& m, double EaR, int n_rk4, double Ts,
                                           double x0, double v, double Fconv) {
  const double h = Ts / (double)n_rk4;
  const double F = v * Fconv;
  double x = x0;
  double a = 1.0, b = 0.0, aa = 0.0, ab = 0.0, bb = 0.0;
  for (int s = 0; s < n_rk4; ++s) {
    double Kx = 0, Ka = 0, Kb = 0, Kaa = 0, Kab = 0, Kbb = 0;        // previous stage
    double Sx = 0, Sa = 0, Sb = 0, Saa = 0, Sab = 0, Sbb = 0;        // weighted sums
#pragma unroll
    for (int st = 0; st < 4; ++st) {
      const double c = (st == 0) ? 0.0 : ((st == 3) ? h : 0.5 * h);
      const double X = x + c * Kx, Xa = a + c * Ka, Xb = b + c * Kb;
      const double Xaa = aa + c * Kaa, Xab = ab + c * Kab, Xbb = bb + c * Kbb;
      double f, fx, fF, fxx, fxF;
      model1_d2(m, EaR, X, F, f, fx, fF, fxx, fxF);
      Kx = f;
      Ka = fx * Xa;
      Kb = fx * Xb + fF * Fconv;
      Kaa = fxx * Xa * Xa + fx * Xaa;
      Kab = fxx * Xa * Xb + fxF * Fconv * Xa + fx * Xab;
      Kbb = fxx * Xb * Xb + 2.0 * fxF * Fconv * Xb + fx * Xbb;
      const double wgt = (st == 0 || st == 3) ? 1.0 : 2.0;
      Sx += wgt * Kx;
      Sa += wgt * Ka;
      Sb += wgt * Kb;
      Saa += wgt * Kaa;
      Sab += wgt * Kab;
      Sbb += wgt * Kbb;
    }
    const double h6 = h / 6.0;
    x += h6 * Sx;
    a += h6 * Sa;
    b += h6 * Sb;
    aa += h6 * Saa;
    ab += h6 * Sab;
    bb += h6 * Sbb;
  }
  return D2{x, a, b, aa, ab, bb};
}

// Columns of the second-order sensitivities of interval k at the KKT point
// (a = dx/dx0, b = dx/dv and their second derivatives, x in K L).  They reuse
// the interior-point QP's slack and dual columns, which are dead from the end
// of an OCP to the next QP (the interior-point method starts each QP afresh).
enum : int { D2A = TL, D2B = TU, D2AA = ZL, D2AB = ZU, D2BB = DUA };

// The second-order shooting of interval k at (x_k, u_k).
__device__ __forceinline__ void ocp_d2(const DevModel& m, const DevCtrl& c, double EaR,
                                       const Ws& w, int k) {
  const D2 d2 = rk4_interval_d2(m, EaR, c.n_rk4, m.Ts, w(X, k) * c.x_scale, w(U, k), c.Fconv);
  w(D2A, k) = d2.a;
  w(D2B, k) = d2.b;
  w(D2AA, k) = d2.aa;
  w(D2AB, k) = d2.ab;
  w(D2BB, k) = d2.bb;
}

// du_0 / d(x_0, Q_z, R_u, Q_n) at the KKT point in (U, X, LAM, PIL, PIU) with
// x_0 in X(., 0), set-points in ZB and steady-state inputs in VB (needed for
// the R_u direction whatever R_u is), the second-order sensitivities of every
// interval in the D2 columns.  Backward Riccati sweep of the tangent QP with
// the exact Lagrangian Hessian and four right-hand sides; only u_0 is needed,
// so there is no forward sweep.  A bound is active when u_k lies on it and
// its multiplier exceeds 1e-10.  Returns false (and zeros) when a pivot of a
// free input is not positive (the reduced Hessian is not positive definite).
__device__ bool ocp_sens_sweep(const DevModel& m, const DevCtrl& c, int N, const Ws& w,
                               double out[4]) {
  const double xs = c.x_scale, Ts = m.Ts, sz = xs / m.V;
  double P = (2.0 * Ts * c.Qz + 2.0 * c.Qn) * sz * sz;
  double p[4];
  {
    const double dzN = w(X, N) * sz - w(ZB, N);
    p[0] = 0.0;
    p[1] = 2.0 * Ts * dzN * sz;
    p[2] = 0.0;
    p[3] = 2.0 * dzN * sz;
  }
  for (int k = N - 1; k >= 0; --k) {
    const double xk = w(X, k), uk = w(U, k), lam = w(LAM, k);
    const double A = w(D2A, k), B = w(D2B, k) / xs, Fxx = w(D2AA, k) * xs, Fxu = w(D2AB, k),
                 Fuu = w(D2BB, k) / xs;
    const double Huu = 2.0 * Ts * c.Ru - lam * Fuu;
    const double Hxu = -lam * Fxu;
    const double Hxx = 2.0 * Ts * c.Qz * sz * sz - lam * Fxx;
    // linear terms of the four directions at stage k, and the offset of the
    // first dynamics row (dx_1 = A_0 dx_0 + B_0 du_0)
    double cu[4] = {0.0, 0.0, 0.0, 0.0}, cx[4] = {0.0, 0.0, 0.0, 0.0}, bo[4] = {0, 0, 0, 0};
    cu[2] = 2.0 * Ts * (uk - w(VB, k + 1));
    if (k == 0) {
      cu[0] = Hxu;          // x_0 cross term, dx_0 = 1 in direction 0
      bo[0] = A;
    } else {
      const double dz = xk * sz - w(ZB, k);
      cx[1] = 2.0 * Ts * dz * sz;
    }
    const bool act = (uk - c.vmin <= 1e-12 && w(PIL, k) > 1e-10) ||
                     (c.vmax - uk <= 1e-12 && w(PIU, k) > 1e-10);
    double Pn, pn[4];
    if (act) {
      // du_k = 0
      Pn = ((k > 0) ? Hxx : 0.0) + ((k > 0) ? A * A * P : 0.0);
#pragma unroll
      for (int d = 0; d < 4; ++d) {
        pn[d] = cx[d] + ((k > 0) ? A * (P * bo[d] + p[d]) : 0.0);
        if (k == 0) out[d] = 0.0;
      }
    } else {
      const double Rb = Huu + B * B * P;
      if (!(Rb > 0.0)) {
#pragma unroll
        for (int d = 0; d < 4; ++d) out[d] = 0.0;
        return false;
      }
      const double iR = 1.0 / Rb;
      const double Sb = (k > 0) ? Hxu + A * P * B : 0.0;
      Pn = (k > 0) ? Hxx + A * A * P - Sb * Sb * iR : 0.0;
#pragma unroll
      for (int d = 0; d < 4; ++d) {
        const double Pbp = P * bo[d] + p[d];
        const double sb = cu[d] + B * Pbp;
        if (k == 0) out[d] = -sb * iR;
        pn[d] = (k > 0) ? cx[d] + A * Pbp - Sb * sb * iR : 0.0;
      }
    }
    P = Pn;
#pragma unroll
    for (int d = 0; d < 4; ++d) p[d] = pn[d];
  }
  return true;
}

// ocp_sens_sweep after the second-order shooting of every interval.
__device__ bool ocp_sens(const DevModel& m, const DevCtrl& c, double EaR, int N, const Ws& w,
                         double out[4]) {
  for (int k = 0; k < N; ++k) ocp_d2(m, c, EaR, w, k);
  return ocp_sens_sweep(m, c, N, w, out);
}

// Tangent of the CD-EKF prediction (RK4 on x' = f, P' = 2 f_x P + (F s_T)^2)
// in three directions, from (x, P) with tangents (dx, dP) and input tangent dF.
__device__ void ekf_predict_tan(const DevModel& m, double EaR, int n_rk4, double F, double x,
                                double P, const double dF[3], double dx[3], double dP[3]) {
  const double h = m.Ts / (double)n_rk4, hh = 0.5 * h, h6 = h / 6.0;
  const double sT = m.sigma[2];
  const double q = F * sT * F * sT;
  double dq[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) dq[d] = 2.0 * F * sT * sT * dF[d];
  for (int s = 0; s < n_rk4; ++s) {
    double fs = 0, ps = 0, kx = 0, kp = 0;
    double dfs[3] = {0, 0, 0}, dps[3] = {0, 0, 0}, dkx[3] = {0, 0, 0}, dkp[3] = {0, 0, 0};
#pragma unroll
    for (int st = 0; st < 4; ++st) {
      const double cst = (st == 0) ? 0.0 : ((st == 3) ? h : hh);
      const double X = x + cst * kx, PP = P + cst * kp;
      double f, fx, fF, fxx, fxF;
      model1_d2(m, EaR, X, F, f, fx, fF, fxx, fxF);
      const double pk = 2.0 * fx * PP + q;
      const double wgt = (st == 0 || st == 3) ? 1.0 : 2.0;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const double dX = dx[d] + cst * dkx[d], dPP = dP[d] + cst * dkp[d];
        const double dfv = fx * dX + fF * dF[d];
        const double dfx = fxx * dX + fxF * dF[d];
        const double dpk = 2.0 * dfx * PP + 2.0 * fx * dPP + dq[d];
        dkx[d] = dfv;
        dkp[d] = dpk;
        dfs[d] += wgt * dfv;
        dps[d] += wgt * dpk;
      }
      kx = f;
      kp = pk;
      fs += wgt * f;
      ps += wgt * pk;
    }
    x += h6 * fs;
    P += h6 * ps;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      dx[d] += h6 * dfs[d];
      dP[d] += h6 * dps[d];
    }
  }
}

// Tangent of the Joseph-form filter with y = x/V + v: x, P before the update.
__device__ __forceinline__ void ekf_filter_tan(const DevModel& m, double y, double x, double P,
                                               const double dy[3], double dx[3], double dP[3]) {
  const double R = m.meas_sd * m.meas_sd, C = 1.0 / m.V;
  const double e = y - x / m.V;
  const double Re = R + C * P * C;
  const double K = P * C / Re;
  const double ImKC = 1.0 - K * C;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double de = dy[d] - dx[d] / m.V;
    const double dRe = C * C * dP[d];
    const double dK = (dP[d] * C * Re - P * C * dRe) / (Re * Re);
    const double dImKC = -dK * C;
    const double dPn = 2.0 * ImKC * dImKC * P + ImKC * ImKC * dP[d] + 2.0 * K * dK * R;
    dx[d] = dx[d] + dK * e + K * de;
    dP[d] = dPn;
  }
}

// Tangent of one sample of the plant (N_s Euler-Maruyama substeps from n with
// flow F) in three directions: dn (3 directions x 3 states), dF per direction.
__device__ void plant_interval_tan(const DevModel& m, const TrajParams& tp, uint32_t j, int i,
                                   double F, const double dF[3], const double n_in[3],
                                   double dn[3][3]) {
  const double h = m.hEM, sqh = m.sqhEM;
  double n[3] = {n_in[0], n_in[1], n_in[2]};
  for (int s = 0; s < m.n_em; ++s) {
    const int64_t ks = (int64_t)i * m.n_em + s;
    const double Tin = inlet_T_at(m, tp, ks);
    double xi[3];
    process_noise<double>(m, j, (uint32_t)ks, xi);
    double f[3], J[9], fF[3];
    drift3(m, tp.EaR, Tin, n, F, f, J, fF);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      double nd[3];
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        double s2 = fF[p] * dF[d];
#pragma unroll
        for (int q = 0; q < 3; ++q) s2 += J[p * 3 + q] * dn[d][q];
        nd[p] = dn[d][p] + h * s2 + dF[d] * m.sigma[p] * sqh * xi[p];
      }
#pragma unroll
      for (int p = 0; p < 3; ++p) dn[d][p] = nd[p];
    }
    em_step<double>(m, tp.EaR, Tin, n, F, h, sqh, xi);
  }
}

// Tangents of one trajectory, kept between the steps below in rows of a
// structure-of-arrays buffer (row r at p[r ld], one column per lane):
// dn (direction d, state q at 3 d + q), d x-hat, d P, d F of the applied
// input, the running sum of d(z - zbar)^2, and what the tangents of the
// current sample start from: the plant temperature, the CD-EKF state and the
// previous input, and the CD-EKF prediction.
enum TgRow : int {
  TG_DN = 0, TG_DXH = 9, TG_DPH = 12, TG_DFP = 15, TG_DPHI = 18,
  TG_CT = 21, TG_XH0 = 22, TG_PH0 = 23, TG_FP = 24, TG_XP = 25, TG_PP = 26, kTgRows = 27
};

struct Tg {
  double* p;
  int64_t ld;
  __device__ __forceinline__ double& operator()(int r) const { return p[r * ld]; }
};

__device__ __forceinline__ void grad_begin(const Tg& g) {
#pragma unroll
  for (int r = 0; r < kTgRows; ++r) g(r) = 0.0;
}

// Before nmpc_sample of sample i: the starting values (the plant's n_T, the
// CD-EKF's x-hat and P, the previous input's flow, the CD-EKF prediction),
// and this sample's term of dPhi.
__device__ __forceinline__ void grad_sample_start(const DevModel& m, const Tg& g, int i,
                                                  double nT, double xhat, double P,
                                                  double F_prev, double xp, double Pp) {
  const double cT = nT / m.V;
  g(TG_CT) = cT;
  g(TG_XH0) = xhat;
  g(TG_PH0) = P;
  g(TG_FP) = F_prev;
  g(TG_XP) = xp;
  g(TG_PP) = Pp;
  if (isfinite(cT)) {
    const double zi = zbar_at(m, i);
#pragma unroll
    for (int d = 0; d < 3; ++d) g(TG_DPHI + d) += 2.0 * (cT - zi) * g(TG_DN + 3 * d + 2) / m.V;
  }
}

// The prediction the last OCP's interval-0 shooting carried (read before the
// next OCP's evaluation overwrites it); at sample 0 the initial estimate.
__device__ __forceinline__ double2 ekf_prior(const Ws& w, const NmpcTraj& T) {
  return (T.i > 0) ? make_double2(w(EPR, 0), w(EPR, 1)) : make_double2(T.xhat, T.P);
}

// After nmpc_sample started the OCP of sample i: the steady-state inputs the
// R_u direction needs, and the tangents of the measurement and the CD-EKF.
__device__ __noinline__ void grad_sample_end(const DevModel& m, const DevCtrl& c, const Ws& w,
                                             double EaR_c, int N, uint32_t j, int i, Tg g) {
  if (c.Ru == 0.0)  // the R_u direction needs the steady-state inputs
    for (int k = 1; k <= N; ++k) w(VB, k) = Fss(m, EaR_c, w(ZB, k)) / c.Fconv;
  double dy[3], dxh[3], dPh[3], dFp[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    dy[d] = g(TG_DN + 3 * d + 2) / m.V;
    dxh[d] = g(TG_DXH + d);
    dPh[d] = g(TG_DPH + d);
    dFp[d] = g(TG_DFP + d);
  }
  if (i > 0) ekf_predict_tan(m, EaR_c, c.n_rk4, g(TG_FP), g(TG_XH0), g(TG_PH0), dFp, dxh, dPh);
  const double y = g(TG_CT) + m.meas_sd * meas_noise<double>(m, j, (uint32_t)i);
  ekf_filter_tan(m, y, g(TG_XP), g(TG_PP), dy, dxh, dPh);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    g(TG_DXH + d) = dxh[d];
    g(TG_DPH + d) = dPh[d];
  }
}

// After the OCP of sample i, with the second-order sensitivities of its
// intervals in the D2 columns and before nmpc_apply: the input tangent and
// the plant's tangents over the sample from n.  Returns false when the
// tangent QP's reduced Hessian was not positive definite (the input tangent
// is then 0).
__device__ __noinline__ bool grad_ocp_end(const DevModel& m, const DevCtrl& c, const Ws& w,
                                          TrajParams tp, uint32_t j, int i, double n0,
                                          double n1, double n2, Tg g) {
  double S[4];
  const bool ok = ocp_sens_sweep(m, c, tp.N, w, S);
  double dF[3], dn[3][3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    dF[d] = (S[0] * g(TG_DXH + d) / c.x_scale + S[1 + d]) * c.Fconv;
#pragma unroll
    for (int q = 0; q < 3; ++q) dn[d][q] = g(TG_DN + 3 * d + q);
  }
  const double F = w(U, 0) * c.Fconv;
  const double n[3] = {n0, n1, n2};
  plant_interval_tan(m, tp, j, i, F, dF, n, dn);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    g(TG_DFP + d) = dF[d];
#pragma unroll
    for (int q = 0; q < 3; ++q) g(TG_DN + 3 * d + q) = dn[d][q];
  }
  return ok;
}

// dPhi_j in the directions (Q_z, R_u, Q_n) once the trajectory has ended.
__device__ __forceinline__ void grad_finish(const DevModel& m, double phi, const Tg& g,
                                            double* __restrict__ dphi_j) {
  const double wK = 1.0 / (double)(m.n_steps + 1);
#pragma unroll
  for (int d = 0; d < 3; ++d) dphi_j[d] = isfinite(phi) ? g(TG_DPHI + d) * wK : nan("");
}

// The closed loop of the NMPC (static schedule, FP64) with the tangents of
// Phi_j in the directions (Q_z, R_u, Q_n) in g.  cnt[7] also counts the OCPs
// whose sensitivity could not be formed (their input tangent is taken as 0).
__device__ TrajOut traj_nmpc_grad(const DevModel& m, const DevCtrl& c, uint32_t j, const Ws& w,
                                  const Tg& g) {
  NmpcTraj T;
  SqpState s;
  nmpc_begin(m, c, j, w, T);
  grad_begin(g);
  for (;;) {
    const double2 pr = ekf_prior(w, T);
    grad_sample_start(m, g, T.i, T.n[2], T.xhat, T.P, T.F_prev, pr.x, pr.y);
    if (!nmpc_sample<double>(m, c, w, T, s)) break;
    grad_sample_end(m, c, w, T.tp.EaR_c, T.tp.N, T.j, T.i, g);
    // the OCP
    while (!sqp_check<double>(c, w, s)) {
      int r;
      do {
        sqp_eval_trial<double>(m, c, T.tp.EaR_c, w, s);
        r = sqp_trial_result<double>(c, w, s);
      } while (r == 2);
      if (r == 1) break;
    }
    for (int k = 0; k < T.tp.N; ++k) ocp_d2(m, c, T.tp.EaR_c, w, k);
    if (!grad_ocp_end(m, c, w, T.tp, T.j, T.i, T.n[0], T.n[1], T.n[2], g)) s.info.qp_fail++;
    nmpc_apply<double>(m, c, w, T, s.info);
  }
  return T.out;
}

// The persistent schedule's recorder (nmpc_persistent with G = Recorder).
// Sample i of trajectory j (j0 <= j < j0 + cn) is a record of RW = 5 (N+1) + 8
// words; word a of it is at rec[(i RW + a) cn + j - j0], so that the first
// 5 (N+1) words are the columns U, X, LAM, PIL, PIU of a scratch view
// (Ws{., cn, N+1}) and the lanes of a warp touch consecutive doubles.  Words
// 5 (N+1) + 0..7: the plant's n (3), the CD-EKF's x-hat and P, the previous
// input's flow, and the CD-EKF prediction (x, P), all as the sample starts.
// kj[j - j0] is the sample at which the trajectory ended (n_steps unless it
// became non-finite); records 0 .. kj exist, the last without an OCP.
struct Recorder {
  static constexpr bool kRecord = true;
  double* rec;
  int64_t cn, j0;
  int RW;
  int32_t* kj;

  __device__ __forceinline__ Ws view(uint32_t j, int i, int N1) const {
    return Ws{rec + (int64_t)i * RW * cn + ((int64_t)j - j0), cn, N1};
  }
  __device__ __forceinline__ void sample(const Ws& w, const NmpcTraj& T) const {
    const Ws r = view(T.j, T.i, w.N1);
    const double2 pr = ekf_prior(w, T);
    r(5, 0) = T.n[0];
    r(5, 1) = T.n[1];
    r(5, 2) = T.n[2];
    r(5, 3) = T.xhat;
    r(5, 4) = T.P;
    r(5, 5) = T.F_prev;
    r(5, 6) = pr.x;
    r(5, 7) = pr.y;
  }
  // the KKT point, before nmpc_apply shifts it
  __device__ __forceinline__ void ocp(const Ws& w, const NmpcTraj& T) const {
    const Ws r = view(T.j, T.i, w.N1);
    const int N = T.tp.N;
    for (int k = 0; k <= N; ++k) r(X, k) = w(X, k);
    for (int k = 0; k < N; ++k) {
      r(U, k) = w(U, k);
      r(LAM, k) = w(LAM, k);
      r(PIL, k) = w(PIL, k);
      r(PIU, k) = w(PIU, k);
    }
  }
  __device__ __forceinline__ void finish(const NmpcTraj& T) const {
    kj[(int64_t)T.j - j0] = T.i;
  }
};

// Threads per block of the tangent pass: one warp, to spread the trajectories
// over the SMs as evenly as the warp granularity allows.
constexpr int kTangentThreads = 32;

// The tangents of Phi_j in (Q_z, R_u, Q_n) through the recorded samples of
// trajectory j: the steps of traj_nmpc_grad, with the closed loop's values
// read from the record instead of computed.  Adds the OCPs without a
// sensitivity to *qp_fail_j (counter 7).
__device__ void traj_nmpc_tangent(const DevModel& m, const DevCtrl& c, uint32_t j, const Ws& w,
                                  const Tg& g, const Recorder& rc, double phi,
                                  int32_t* qp_fail_j, double* __restrict__ dphi_j) {
  const TrajParams tp = traj_params(m, c, j);
  const int N = tp.N, Kj = rc.kj[(int64_t)j - rc.j0];
  grad_begin(g);
  int fails = 0;
  for (int i = 0;; ++i) {
    const Ws r = rc.view(j, i, w.N1);
    grad_sample_start(m, g, i, r(5, 2), r(5, 3), r(5, 4), r(5, 5), r(5, 6), r(5, 7));
    if (i == Kj) break;
    // set-points and steady-state inputs as nmpc_sample and grad_sample_end set them
    for (int k = 1; k <= N; ++k) w(ZB, k) = zbar_at(m, i + k);
    if (c.Ru != 0.0)
      for (int k = 1; k <= N; ++k) w(VB, k) = Fss(m, tp.EaR_c, w(ZB, k)) / c.Fconv;
    grad_sample_end(m, c, w, tp.EaR_c, N, j, i, g);
    for (int k = 0; k <= N; ++k) w(X, k) = r(X, k);
    for (int k = 0; k < N; ++k) {
      w(U, k) = r(U, k);
      w(LAM, k) = r(LAM, k);
      w(PIL, k) = r(PIL, k);
      w(PIU, k) = r(PIU, k);
    }
    for (int k = 0; k < N; ++k) ocp_d2(m, c, tp.EaR_c, w, k);
    if (!grad_ocp_end(m, c, w, tp, j, i, r(5, 0), r(5, 1), r(5, 2), g)) ++fails;
  }
  grad_finish(m, phi, g, dphi_j);
  *qp_fail_j += fails;
}

}  // namespace mc
