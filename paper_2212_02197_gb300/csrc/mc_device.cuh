// mc_device.cuh -- device building blocks of the closed-loop Monte Carlo path:
// counter-based noise, the CSTR model, Euler-Maruyama, RK4 shooting with
// forward sensitivities, the CD-EKF and the PI law.
//
// Everything is per thread: one thread owns one trajectory (SIMT across
// trajectories), so every FP64 instruction a warp issues does useful work for
// 32 trajectories at once.  Functions are templated on the arithmetic type R
// where the mixed-precision path runs them in FP32.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

// the QP/SQP building blocks are plain arithmetic and also compile for the host
#define MC_HD __host__ __device__ __forceinline__

namespace mc {

constexpr int kMaxSp = 16;
constexpr int kMaxN = 64;
constexpr int kNCounters = 8;

// Plant/model/closed-loop parameters as passed by value to every kernel.
struct DevModel {
  double V, k0, EaR, beta, cA_in, cB_in, T_in;
  double sigma[3];
  double meas_sd;
  double Ts, t0;
  int n_steps, n_em, n_sp;
  int Ea_plant_only;   // 1: the controller's model keeps the nominal E_a/R
  double sp_time[kMaxSp], sp_value[kMaxSp];
  double Ea_logsd, dTin;
  double iV, ib;       // 1/V and 1/beta
  double rw0, rw1, bV, ib2;  // one-state rate law: ib (cB_in + 2 cA_in), 4 ib^2,
                            // beta V, 2 ib
  uint32_t key0, key1;
  double lnk0;          // log k0: the rate constant as one exp, k0 e^{-g} = e^{log k0 - g}
  int sp_step[kMaxSp];  // first sample i with t0 + i Ts >= sp_time[s] (set-point segments)
  double hEM, sqhEM;    // Euler-Maruyama step Ts / N_s and its square root
};

struct DevCtrl {
  int kind, precision, N, n_rk4;
  int sqp_max_it, ls_max, qp_solver, ip_max_it;
  int N_min, it_min;   // > 0: per-trajectory N in [N_min, N], limit in [it_min, sqp_max_it]
  int nx_model;        // NMPC model: 1 = one-state, 3 = three-state
  int spec_lanes;      // speculative backtracking while at most this many lanes are busy
  double Ru, Qn;       // input-deviation and terminal weights of the extended objective
  double r_scale;      // 2 R_u T_s: r_k = r_scale (v_k - vbar_{k+1})
  double u_min, u_max, kP, kI, kaw, Qz, P0, sqp_tol, ip_tol, u_scale, x_scale;
  double Fconv;        // OCP input unit -> L/s
  double vmin, vmax;   // input bounds in OCP units
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64-bit products whose high halves are xored with the other counter
// words and the round key; the key advances by two Weyl constants per round.

MC_HD uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
  return __umulhi(a, b);
#else
  return (uint32_t)(((uint64_t)a * (uint64_t)b) >> 32);
#endif
}

// (host and device: the host uses it to order trajectories by their horizon)
MC_HD uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi0 = mulhi32(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = mulhi32(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// Open-interval uniform from 52 bits (26 of each word): (m + 1/2) 2^-52.
__device__ __forceinline__ double u52(uint32_t hi, uint32_t lo) {
  const double m = __uint2double_rn(hi >> 6) * 67108864.0 + __uint2double_rn(lo >> 6);
  return (m + 0.5) * (1.0 / 4503599627370496.0);
}

// Open-interval uniform from the top 24 bits of one word, for the FP32 path.
__device__ __forceinline__ float u24(uint32_t w) {
  return (__uint2float_rn(w >> 8) + 0.5f) * (1.0f / 16777216.0f);
}

// Box-Muller pair.
template <class R> struct Normal2;
template <> struct Normal2<double> {
  static __device__ __forceinline__ double2 from(uint4 w) {
    const double u1 = u52(w.x, w.y), u2 = u52(w.z, w.w);
    const double rad = sqrt(-2.0 * log(u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    return make_double2(rad * c, rad * s);
  }
};
template <> struct Normal2<float> {
  static __device__ __forceinline__ double2 from(uint4 w) {
    const float u1 = u24(w.x), u2 = u24(w.z);
    const float rad = sqrtf(-2.0f * logf(u1));
    float s, c;
    sincospif(2.0f * u2, &s, &c);
    return make_double2((double)(rad * c), (double)(rad * s));
  }
};

// Counter layout: (k, j, tag, 0); tags 0/1 process noise of global substep k,
// 2 measurement noise of sample k, 3 per-trajectory parameters.
template <class R>
__device__ __forceinline__ void process_noise(const DevModel& m, uint32_t j, uint32_t k,
                                              R xi[3]) {
  const double2 a = Normal2<R>::from(philox4x32_10(make_uint4(k, j, 0u, 0u), m.key0, m.key1));
  const double2 b = Normal2<R>::from(philox4x32_10(make_uint4(k, j, 1u, 0u), m.key0, m.key1));
  xi[0] = (R)a.x;
  xi[1] = (R)a.y;
  xi[2] = (R)b.x;
}

template <class R>
__device__ __forceinline__ R meas_noise(const DevModel& m, uint32_t j, uint32_t i) {
  return (R)Normal2<R>::from(philox4x32_10(make_uint4(i, j, 2u, 0u), m.key0, m.key1)).x;
}

struct TrajParams {
  double EaR;      // the plant's E_a/R
  double EaR_c;    // the controller's (EKF, OCP model, steady-state input)
  double t_d, dTin;
  int64_t ks_d;    // first Euler-Maruyama substep whose start t0 + ks h is >= t_d
  int N, max_it;   // horizon and SQP iteration limit of this trajectory's OCPs
};

// Start time t0 + ks h of substep ks, rounded as two separate operations
// (product, then sum) so that the inlet step switches at the same substep
// wherever the time is formed that way.
__device__ __forceinline__ double substep_time(const DevModel& m, int64_t ks) {
  return __dadd_rn(m.t0, __dmul_rn((double)ks, m.hEM));
}

// Per-trajectory horizon and SQP iteration limit: uniform integers from the
// words of counter (2, j, 3, 0) when the controller gives ranges.
MC_HD void traj_horizon(const DevCtrl& c, uint32_t key0, uint32_t key1, uint32_t j, int& N,
                        int& max_it) {
  N = c.N;
  max_it = c.sqp_max_it;
  if (c.N_min <= 0 && c.it_min <= 0) return;
  const uint4 w = philox4x32_10(make_uint4(2u, j, 3u, 0u), key0, key1);
  if (c.N_min > 0) N = c.N_min + (int)(w.x % (uint32_t)(c.N - c.N_min + 1));
  if (c.it_min > 0) max_it = c.it_min + (int)(w.y % (uint32_t)(c.sqp_max_it - c.it_min + 1));
}

// Time and sign of the T_in step (uniform on [t0, tf)), the lognormal E_a/R,
// and the OCP horizon and iteration limit.
__device__ __forceinline__ TrajParams traj_params(const DevModel& m, const DevCtrl& c,
                                                  uint32_t j) {
  TrajParams p;
  traj_horizon(c, m.key0, m.key1, j, p.N, p.max_it);
  const uint4 w = philox4x32_10(make_uint4(0u, j, 3u, 0u), m.key0, m.key1);
  const double tf = m.t0 + (double)m.n_steps * m.Ts;
  p.t_d = m.t0 + u52(w.x, w.y) * (tf - m.t0);
  p.dTin = (w.z & 1u) ? m.dTin : -m.dTin;
  const double2 z = Normal2<double>::from(philox4x32_10(make_uint4(1u, j, 3u, 0u), m.key0, m.key1));
  p.EaR = (m.Ea_logsd != 0.0) ? m.EaR * exp(m.Ea_logsd * z.x) : m.EaR;
  p.EaR_c = m.Ea_plant_only ? m.EaR : p.EaR;
  // the substep at which the inlet step begins, found once per trajectory so
  // that each substep compares integers
  p.ks_d = INT64_MAX;
  const double est = (p.t_d - m.t0) / m.hEM;
  if (isfinite(est) && est < 9.0e15) {
    int64_t ks = est > 0.0 ? (int64_t)ceil(est) : 0;
    for (int it = 0; it < 8 && ks > 0 && substep_time(m, ks - 1) >= p.t_d; ++it) --ks;
    for (int it = 0; it < 8 && substep_time(m, ks) < p.t_d; ++it) ++ks;
    p.ks_d = ks;
  }
  return p;
}

// Inlet temperature of substep ks: T_in, stepped by dTin from the substep
// whose start reaches t_d on.
__device__ __forceinline__ double inlet_T_at(const DevModel& m, const TrajParams& tp,
                                             int64_t ks) {
  return (m.dTin != 0.0 && ks >= tp.ks_d) ? m.T_in + tp.dTin : m.T_in;
}

// ---------------------------------------------------------------------------
// CSTR, Eq. (CSTR): dn/dt = C_in F - c F + S^T r(c) V, S = [-1, -2, beta],
// r = k0 exp(-(E_a/R)/c_T) c_A c_B.

// exp in FP64 by Tang's table-driven method (P. T. P. Tang, ACM TOMS 15(2),
// 1989), with 2048 table entries: x = (2048 m + j) ln2/2048 + r with
// |r| <= ln2/4096, so e^x = 2^m 2^(j/2048) e^r.  2^(j/2048) comes from a table
// of the correctly rounded doubles (16 KB, written by gen_exp2_table.py),
// e^r - 1 from its Taylor series to degree 3 (the next term, r^4/24, is below
// 4e-17 of the result), and 2^m is added to the exponent field.  ln2/2048 is
// split into a head of 21 significant bits (n ln2/2048 is exact for
// |n| < 2^32) and a tail.  The range test runs on the integer pipe (the high
// word of x): |x| >= 700, infinities and NaN go to the library exp; below it
// the result is normal.  Eight FP64 operations.
__device__ const double kExp2j2048[2048] = {
#include "mc_exp2_table.inc"
};

__device__ __forceinline__ double exp_table(double x) {
  if ((__double2hiint(x) & 0x7fffffff) >= 0x4085e000) return exp(x);   // |x| >= 700
  const double inv_l = 0x1.71547652b82fep+11;   // 2048 / ln 2
  const double shifter = 0x1.8p+52;             // adding it rounds to an integer
  const double l_hi = 0x1.62e4300000000p-12;    // ln2/2048, head
  const double l_lo = -0x1.05c610ca86c39p-40;   // ln2/2048, tail
  const double t = fma(x, inv_l, shifter);
  const double n = t - shifter;
  const int k = __double2loint(t);              // n as an integer
  double r = fma(n, -l_hi, x);
  r = fma(n, -l_lo, r);
  const double p = fma(1.0 / 6.0, r, 0.5);
  const double q = fma(p, r * r, r);            // e^r - 1
  const double T = __ldg(&kExp2j2048[k & 2047]);
  const double y = fma(T, q, T);
  return __hiloint2double(__double2hiint(y) + ((k >> 11) << 20), __double2loint(y));
}

__device__ __forceinline__ double expr(double x) { return exp_table(x); }

// 1/x by Newton-Raphson refinement of the hardware's approximate FP64
// reciprocal: y <- y + y (1 - x y) twice, each step doubling the correct bits
// of the approximation, to within about 1 ulp of 1/x.  Zeros, infinities and
// NaN (and denormals, which the approximation flushes) keep the approximate
// value, which for them is already 1/x; the test is on the integer pipe.
__device__ __forceinline__ double rcp_newton(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const int ex = __double2hiint(x) & 0x7ff00000;
  if (ex == 0 || ex == 0x7ff00000) return y;
  double e = fma(-x, y, 1.0);
  y = fma(y, e, y);
  e = fma(-x, y, 1.0);
  return fma(y, e, y);
}
__device__ __forceinline__ float rcp_newton(float x) { return 1.0f / x; }
__device__ __forceinline__ float expr(float x) { return expf(x); }

template <class R>
__device__ __forceinline__ void plant_drift(const DevModel& m, R EaR, R T_in, const R n[3],
                                            R F, R f[3]) {
  const R iV = (R)m.iV;
  const R cA = n[0] * iV, cB = n[1] * iV, cT = n[2] * iV;
  const R k = (R)m.k0 * expr(-EaR / cT);
  const R rV = k * cA * cB * (R)m.V;
  f[0] = (R)m.cA_in * F - cA * F - rV;
  f[1] = (R)m.cB_in * F - cB * F - (R)2 * rV;
  f[2] = T_in * F - cT * F + (R)m.beta * rV;
}

// One Euler-Maruyama substep: n += f h + F sigma-bar sqrt(h) xi.
template <class R>
__device__ __forceinline__ void em_step(const DevModel& m, R EaR, R T_in, R n[3], R F, R h,
                                        R sqh, const R xi[3]) {
  R f[3];
  plant_drift<R>(m, EaR, T_in, n, F, f);
#pragma unroll
  for (int i = 0; i < 3; ++i) n[i] = n[i] + f[i] * h + F * (R)m.sigma[i] * sqh * xi[i];
}

// One-state model (Sec. VI) in x = n_T; c_A, c_B from the reaction invariants.
// Returns f and df/dx, df/dF.  With c_T = x / V, d = T_in - c_T, the invariants
// give c_A = c_A,in + d / beta and c_B = c_B,in + 2 d / beta, and
//   r = k(c_T) c_A c_B,  k = k_0 exp(-g),  g = (E_a/R) / c_T,
//   f = F d + beta V r,
//   dr/dc_T = r g / c_T - k (c_B + 2 c_A) / beta,
//   df/dx = -F / V + beta dr/dc_T,
// where (c_B + 2 c_A) / beta = rw0 + rw1 d is affine in d.  Every rounding is
// written out (fma where a product meets a sum), so that the compiler has no
// contraction to choose and every function that inlines the model (the
// schedules' shooting functions) rounds alike.  Written this way the
// evaluation takes 15 FP64 operations besides the exp and the reciprocal (and
// one, F / V, that stays the same over an interval); the reciprocal is
// rcp_newton's and k0 enters the exponent as log k0.
template <class R>
__device__ __forceinline__ void model1(const DevModel& m, R EaR, R x, R F, R& f, R& fx,
                                       R& fF) {
  const R iV = (R)m.iV, ib = (R)m.ib;
  const R cT = x * iV;
  const R d = fma(-x, iV, (R)m.T_in);
  const R iT = rcp_newton(cT);
  const R g = EaR * iT;
  const R k = expr(fma(-EaR, iT, (R)m.lnk0));
  const R cA = fma(d, ib, (R)m.cA_in);
  const R cB = fma(d, (R)m.ib2, (R)m.cB_in);
  const R r = k * (cA * cB);
  f = fma((R)m.bV, r, F * d);
  const R ibw = fma((R)m.rw1, d, (R)m.rw0);
  const R dr = fma(r, g * iT, -(k * ibw));
  fx = fma((R)m.beta, dr, -(F * iV));
  fF = d;
}

// Sums whose operands may be products, rounded as written: the compiler never
// merges these into a multiply-add.
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }

// The RK4 weighted sum k1 + 2 k2 + 2 k3 + k4, every rounding written out.
template <class R>
__device__ __forceinline__ R rk4_sum(R k1, R k2, R k3, R k4) {
  return add_rn(fma((R)2, k3, fma((R)2, k2, k1)), k4);
}

// One shooting interval: n_rk4 classical RK4 steps over Ts from x0 (K L) with
// flow F = v Fconv, and the forward sensitivities a = dx/dx0, B = dx/dv.
// The RK4 stages propagate b = dx/dF, whose forcing is df/dF itself; B is
// Fconv b, formed once at the end.
// With cov, the same stages also carry the CD-EKF covariance of Eq.
// (predictionEquations), dP/dt = 2 (df/dx) P + (F sigma_T)^2, from P0 into
// P1: xF and P1 are then the CD-EKF prediction, RK4 on (x, P) over one sample
// from (x0, P0) under this input.  As in model1, every rounding is written
// out.
template <class R, bool kSens>
__device__ __forceinline__ void rk4_interval(const DevModel& m, R EaR, int n_rk4, R Ts, R x0,
                                             R v, R Fconv, R& xF, R& A, R& B,
                                             bool cov = false, R P0 = 0, R* P1 = nullptr) {
  const R h = Ts / (R)n_rk4;
  const R hh = (R)0.5 * h, h6 = h / (R)6;
  const R F = v * Fconv;
  const R sq = F * (R)m.sigma[2];
  const R q = sq * sq;
  R x = x0, a = 1, b = 0, Ps = P0;
  for (int s = 0; s < n_rk4; ++s) {
    R f1, fx1, fF1, f2, fx2, fF2, f3, fx3, fF3, f4, fx4, fF4;
    model1<R>(m, EaR, x, F, f1, fx1, fF1);
    const R x2 = fma(hh, f1, x);
    model1<R>(m, EaR, x2, F, f2, fx2, fF2);
    const R x3 = fma(hh, f2, x);
    model1<R>(m, EaR, x3, F, f3, fx3, fF3);
    const R x4 = fma(h, f3, x);
    model1<R>(m, EaR, x4, F, f4, fx4, fF4);
    if (kSens) {
      const R a1 = fx1 * a, b1 = fma(fx1, b, fF1);
      const R a2 = fx2 * fma(hh, a1, a), b2 = fma(fx2, fma(hh, b1, b), fF2);
      const R a3 = fx3 * fma(hh, a2, a), b3 = fma(fx3, fma(hh, b2, b), fF3);
      const R a4 = fx4 * fma(h, a3, a), b4 = fma(fx4, fma(h, b3, b), fF4);
      a = fma(h6, rk4_sum(a1, a2, a3, a4), a);
      b = fma(h6, rk4_sum(b1, b2, b3, b4), b);
    }
    if (cov) {
      const R p1 = fma((R)2 * fx1, Ps, q);
      const R p2 = fma((R)2 * fx2, fma(hh, p1, Ps), q);
      const R p3 = fma((R)2 * fx3, fma(hh, p2, Ps), q);
      const R p4 = fma((R)2 * fx4, fma(h, p3, Ps), q);
      Ps = fma(h6, rk4_sum(p1, p2, p3, p4), Ps);
    }
    x = fma(h6, rk4_sum(f1, f2, f3, f4), x);
  }
  xF = x;
  A = a;
  B = kSens ? b * Fconv : b;
  if (cov) *P1 = Ps;
}

// CD-EKF filtering with the Joseph-form covariance, Eq. (Josph); always FP64.
__device__ __forceinline__ void ekf_filter(const DevModel& m, double y, double& x, double& P) {
  const double R = m.meas_sd * m.meas_sd;
  const double C = 1.0 / m.V;
  const double e = y - x / m.V;
  const double Re = R + C * P * C;
  const double K = P * C / Re;
  const double ImKC = 1.0 - K * C;
  P = ImKC * P * ImKC + K * R * K;
  x = x + K * e;
}

// Piecewise-constant set-point z-bar(t).
__device__ __forceinline__ double zbar(const DevModel& m, double t) {
  double z = m.sp_value[0];
  for (int s = 1; s < m.n_sp; ++s)
    if (t >= m.sp_time[s]) z = m.sp_value[s];
  return z;
}

// The same set-point at sample time t_i = t0 + i T_s, from the segments' first
// sample indices (integer compares only).
__device__ __forceinline__ double zbar_at(const DevModel& m, int i) {
  double z = m.sp_value[0];
  for (int s = 1; s < m.n_sp; ++s)
    if (i >= m.sp_step[s]) z = m.sp_value[s];
  return z;
}

// Steady-state flow (L/s) of the one-state model at temperature Tbar.
__device__ __forceinline__ double Fss(const DevModel& m, double EaR, double Tbar) {
  const double cA = m.cA_in + (m.T_in - Tbar) / m.beta;
  const double cB = m.cB_in + 2.0 * (m.T_in - Tbar) / m.beta;
  const double r = m.k0 * exp(-EaR / Tbar) * cA * cB;
  return m.beta * r * m.V / (Tbar - m.T_in);
}

// PI law with anti-windup, Eq. (PI); flows in L/s.  The error e and the
// unclipped input u-hat are returned too when asked for (the adjoint).
template <class R>
__device__ __forceinline__ R pi_step(const DevCtrl& c, R Ts, R ybar, R y, R ubar, R& Ihat,
                                     R* e_out = nullptr, R* uhat_out = nullptr) {
  const R umin = (R)(c.u_min / 60000.0), umax = (R)(c.u_max / 60000.0);
  const R e = ybar - y;
  const R P = (R)c.kP * e;
  const R I = Ihat + Ts * (R)c.kI * e;
  const R uhat = ubar + P + I;
  const R u = fmax(umin, fmin(umax, uhat));
  Ihat = I + Ts * (R)c.kaw * (uhat - u);
  if (e_out) *e_out = e;
  if (uhat_out) *uhat_out = uhat;
  return u;
}

}  // namespace mc
