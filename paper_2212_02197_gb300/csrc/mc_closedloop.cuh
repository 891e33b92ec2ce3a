// mc_closedloop.cuh -- one stochastic closed-loop simulation per thread
// (Sec. VII): plant SDE by Euler-Maruyama, noisy measurement, controller
// (NMPC = CD-EKF + SQP, or PI), and the performance index Phi, Eq. (Phi).
#pragma once

#include "mc_sqp.cuh"

namespace mc {

struct TrajOut {
  double phi;
  int32_t cnt[kNCounters];  // n_ocp_failed, sqp_iters, ls_trials, n_hess_reset,
                            // n_ls_fail, qp_iters, nonfinite, qp_fail
};

// Plant between two samples: N_s Euler-Maruyama substeps with zero-order hold
// on the flow F (L/s) and the inlet temperature (which steps at t_d).
template <class R>
__device__ __forceinline__ void plant_interval(const DevModel& m, const TrajParams& tp,
                                               uint32_t j, int i, double F, double n[3]) {
  const double h = m.Ts / (double)m.n_em;
  const R hR = (R)h, sqh = (R)sqrt(h);
  R nr[3] = {(R)n[0], (R)n[1], (R)n[2]};
  const R EaR = (R)tp.EaR, FR = (R)F;
  for (int s = 0; s < m.n_em; ++s) {
    const int64_t ks = (int64_t)i * m.n_em + s;
    const double tau = m.t0 + (double)ks * h;
    const double Tin = (m.dTin != 0.0 && tau >= tp.t_d) ? m.T_in + tp.dTin : m.T_in;
    R xi[3];
    process_noise<R>(m, j, (uint32_t)ks, xi);
    em_step<R>(m, EaR, (R)Tin, nr, FR, hR, sqh, xi);
  }
  n[0] = (double)nr[0];
  n[1] = (double)nr[1];
  n[2] = (double)nr[2];
}

template <class R>
__device__ TrajOut traj_pi(const DevModel& m, const DevCtrl& c, uint32_t j) {
  TrajOut out{};
  const TrajParams tp = traj_params(m, j);
  double n[3] = {m.cA_in * m.V, m.cB_in * m.V, m.T_in * m.V};
  const int K = m.n_steps;
  double phi = 0.0;
  R Ihat = 0;
  for (int i = 0; i <= K; ++i) {
    const double t_i = m.t0 + (double)i * m.Ts;
    const double cT = n[2] / m.V;
    if (!isfinite(cT)) {
      out.cnt[6] = 1;
      phi = nan("");
      break;
    }
    const double zi = zbar(m, t_i);
    const double ez = cT - zi;
    phi += ez * ez;
    if (i == K) break;
    const double y = cT + m.meas_sd * (double)meas_noise<R>(m, j, (uint32_t)i);
    const double ubar = Fss(m, tp.EaR, zi);
    const double F = (double)pi_step<R>(c, (R)m.Ts, (R)zi, (R)y, (R)ubar, Ihat);
    plant_interval<R>(m, tp, j, i, F, n);
  }
  out.phi = phi / (double)(K + 1);
  return out;
}

// R = double: the FP64 path.  R = float: the mixed-precision path -- plant
// SDE, noise transform, EKF prediction and the OCP shooting in FP32; the
// Joseph-form filter update, the QP (Riccati pivots), merit, BFGS and the SQP
// convergence test in FP64.
template <class R>
__device__ TrajOut traj_nmpc(const DevModel& m, const DevCtrl& c, uint32_t j, const Ws& w) {
  TrajOut out{};
  const TrajParams tp = traj_params(m, j);
  const double EaR = tp.EaR;
  double n[3] = {m.cA_in * m.V, m.cB_in * m.V, m.T_in * m.V};
  const int K = m.n_steps, N = c.N;
  const double ixs = 1.0 / c.x_scale;
  double phi = 0.0;
  double xhat = m.T_in * m.V, P = c.P0;
  double F_prev = 0.0;
  {
    // first OCP guess: steady-state input of the first set-point, clipped
    double v0 = Fss(m, EaR, zbar(m, m.t0)) / c.Fconv;
    v0 = fmin(fmax(v0, c.vmin), c.vmax);
    for (int k = 0; k < N; ++k) {
      w(U, k) = v0;
      w(X, k + 1) = xhat * ixs;
      w(LAM, k) = 0.0;
      w(PIL, k) = 0.0;
      w(PIU, k) = 0.0;
    }
  }
  for (int i = 0; i <= K; ++i) {
    const double t_i = m.t0 + (double)i * m.Ts;
    const double cT = n[2] / m.V;
    if (!isfinite(cT) || !isfinite(xhat) || !isfinite(P)) {
      out.cnt[6] = 1;
      phi = nan("");
      break;
    }
    const double ez = cT - zbar(m, t_i);
    phi += ez * ez;
    if (i == K) break;

    const double y = cT + m.meas_sd * (double)meas_noise<R>(m, j, (uint32_t)i);
    if (i > 0) {
      R xr = (R)xhat, Pr = (R)P;
      ekf_predict<R>(m, (R)EaR, c.n_rk4, (R)F_prev, xr, Pr);
      xhat = (double)xr;
      P = (double)Pr;
    }
    ekf_filter(m, y, xhat, P);
    for (int k = 1; k <= N; ++k) w(ZB, k) = zbar(m, m.t0 + (double)(i + k) * m.Ts);
    const SqpInfo si = sqp_solve<R>(m, c, EaR, xhat * ixs, w, i > 0);
    out.cnt[0] += (si.status == 1);
    out.cnt[1] += si.iters;
    out.cnt[2] += si.ls_trials;
    out.cnt[3] += si.n_hess_reset;
    out.cnt[4] += (si.status == 2);
    out.cnt[5] += si.qp_iters;
    out.cnt[7] += si.qp_fail;
    const double F = w(U, 0) * c.Fconv;
    // receding horizon: shift one interval, duplicating the last one; the
    // final evaluation shifts along (its intervals 1..N-2 stay valid)
    for (int k = 0; k < N - 1; ++k) {
      w(U, k) = w(U, k + 1);
      w(X, k + 1) = w(X, k + 2);
      w(LAM, k) = w(LAM, k + 1);
      w(PIL, k) = w(PIL, k + 1);
      w(PIU, k) = w(PIU, k + 1);
      w(EA, k) = w(EA, k + 1);
      w(EB, k) = w(EB, k + 1);
      w(EG, k) = w(EG, k + 1);
    }
    plant_interval<R>(m, tp, j, i, F, n);
    F_prev = F;
  }
  out.phi = phi / (double)(K + 1);
  return out;
}

}  // namespace mc
