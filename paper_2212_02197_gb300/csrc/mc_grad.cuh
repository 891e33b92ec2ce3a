// mc_grad.cuh -- gradient of the performance index of the PI study (Eq. (Phi),
// Sec. VII) with respect to the controller gains (k_P, k_I, k_aw) of Eq. (PI),
// by a hand-written discrete adjoint (reverse mode) of the closed loop.
//
// One thread per trajectory, FP64.
//   forward sweep   the closed loop as k_pi runs it, storing the plant state n
//                   and the integral state I-hat every C steps (checkpoints);
//   backward sweep  segment by segment from the last: the segment's sample
//                   states are recomputed from its checkpoint, then each
//                   sample is reversed -- its Euler-Maruyama substeps (states
//                   and noise recomputed from the sample state), then the PI
//                   law, then the Phi term of the sample.
// Per trajectory the sweeps cost about four forward simulations and hold
// C sample states plus N_s substep states in local memory.
//
// The input clip u = max(u_min, min(u_max, u-hat)) passes u-hat through only
// strictly inside the bounds; at a bound the derivative is taken as zero.
#pragma once

#include "mc_closedloop.cuh"

namespace mc {

constexpr int kGradMaxSeg = 32;  // checkpoint interval limit (samples)
constexpr int kGradMaxEm = 32;   // Euler-Maruyama substeps per sample limit

// Adjoint of one substep n+ = n + f(n, F) h + F sigma-bar sqrt(h) xi of the
// three-state CSTR, Eq. (CSTR), at the state n before it.  On entry nb is the
// adjoint of n+, on exit that of n; Fb accumulates the adjoint of F.
// df_p/dn_q = -(F/V) delta_pq + S_p d(rV)/dn_q with S = (-1, -2, beta) and
// rV = k0 exp(-(E_a/R)/c_T) c_A c_B V.
__device__ __forceinline__ void em_step_adjoint(const DevModel& m, double EaR, double T_in,
                                                const double n[3], double F, double h,
                                                double sqh, const double xi[3], double nb[3],
                                                double& Fb) {
  const double iV = m.iV;
  const double cA = n[0] * iV, cB = n[1] * iV, cT = n[2] * iV;
  const double k = m.k0 * expr(-EaR / cT);
  const double rV = k * cA * cB * m.V;
  Fb += nb[0] * (h * (m.cA_in - cA) + m.sigma[0] * sqh * xi[0]) +
        nb[1] * (h * (m.cB_in - cB) + m.sigma[1] * sqh * xi[1]) +
        nb[2] * (h * (T_in - cT) + m.sigma[2] * sqh * xi[2]);
  const double g = -nb[0] - 2.0 * nb[1] + m.beta * nb[2];
  const double d0 = k * cB * m.V * iV;
  const double d1 = k * cA * m.V * iV;
  const double d2 = rV * EaR / (cT * cT) * iV;
  const double a = h * F * iV;
  nb[0] = nb[0] - a * nb[0] + h * g * d0;
  nb[1] = nb[1] - a * nb[1] + h * g * d1;
  nb[2] = nb[2] - a * nb[2] + h * g * d2;
}

// Inlet temperature during substep ks (steps at t_d by dTin).
__device__ __forceinline__ double inlet_T(const DevModel& m, const TrajParams& tp, int64_t ks,
                                          double) {
  return inlet_T_at(m, tp, ks);
}

// Trajectory j: Phi_j and dPhi_j / d(k_P, k_I, k_aw).  The checkpoints live in
// ck[(q * n_ck + s) * ck_ld + j], q = n_A, n_B, n_T, I-hat, s = step / C.
__global__ void __launch_bounds__(128) k_pi_grad(DevModel m, DevCtrl c, int64_t j0, int64_t j1,
                                                 int C, int n_ck, double* __restrict__ ck,
                                                 int64_t ck_ld, double* __restrict__ phi_out,
                                                 int32_t* __restrict__ cnt_out,
                                                 double* __restrict__ dphi) {
  const int64_t jj = j0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (jj >= j1) return;
  const uint32_t j = (uint32_t)jj;
  const TrajParams tp = traj_params(m, c, j);
  const int K = m.n_steps;
  auto CK = [&](int q, int s) -> double& { return ck[((int64_t)q * n_ck + s) * ck_ld + jj]; };

  // ---- forward sweep with checkpoints
  double n[3] = {m.cA_in * m.V, m.cB_in * m.V, m.T_in * m.V};
  double Ihat = 0.0, phi = 0.0, ezK = 0.0;
  bool finite = true;
  for (int i = 0; i <= K; ++i) {
    const double cT = n[2] / m.V;
    if (!isfinite(cT)) {
      finite = false;
      break;
    }
    const double zi = zbar_at(m, i);
    const double ez = cT - zi;
    phi += ez * ez;
    if (i == K) {
      ezK = ez;
      break;
    }
    if (i % C == 0) {
      CK(0, i / C) = n[0];
      CK(1, i / C) = n[1];
      CK(2, i / C) = n[2];
      CK(3, i / C) = Ihat;
    }
    const double y = cT + m.meas_sd * meas_noise<double>(m, j, (uint32_t)i);
    const double ubar = Fss(m, tp.EaR_c, zi);
    const double F = pi_step<double>(c, m.Ts, zi, y, ubar, Ihat);
    plant_interval<double>(m, tp, j, i, F, n);
  }
#pragma unroll
  for (int q = 0; q < kNCounters; ++q) cnt_out[jj * kNCounters + q] = 0;
  if (!finite) {
    phi_out[jj] = nan("");
    cnt_out[jj * kNCounters + 6] = 1;
    dphi[jj * 3 + 0] = dphi[jj * 3 + 1] = dphi[jj * 3 + 2] = nan("");
    return;
  }
  const double wK = 1.0 / (double)(K + 1);
  phi_out[jj] = phi / (double)(K + 1);

  // ---- backward sweep
  const double h = m.hEM, sqh = m.sqhEM;
  const double umin = c.u_min / 60000.0, umax = c.u_max / 60000.0;
  const double Ts = m.Ts;
  double nb[3] = {0.0, 0.0, 2.0 * ezK * wK / m.V};
  double Ib = 0.0, gP = 0.0, gI = 0.0, gaw = 0.0;
  double sn[kGradMaxSeg][4];
  double sub[kGradMaxEm][6];
  for (int sg = (K - 1) / C; K > 0 && sg >= 0; --sg) {
    const int i0 = sg * C, i1 = (i0 + C < K) ? i0 + C : K;
    double nn[3] = {CK(0, sg), CK(1, sg), CK(2, sg)};
    double Ih = CK(3, sg);
    for (int i = i0; i < i1; ++i) {
      sn[i - i0][0] = nn[0];
      sn[i - i0][1] = nn[1];
      sn[i - i0][2] = nn[2];
      sn[i - i0][3] = Ih;
      const double cT = nn[2] / m.V;
      const double zi = zbar_at(m, i);
      const double y = cT + m.meas_sd * meas_noise<double>(m, j, (uint32_t)i);
      const double F = pi_step<double>(c, m.Ts, zi, y, Fss(m, tp.EaR_c, zi), Ih);
      plant_interval<double>(m, tp, j, i, F, nn);
    }
    for (int i = i1 - 1; i >= i0; --i) {
      double ns[3] = {sn[i - i0][0], sn[i - i0][1], sn[i - i0][2]};
      double Ih2 = sn[i - i0][3];
      const double cT = ns[2] / m.V;
      const double zi = zbar_at(m, i);
      const double y = cT + m.meas_sd * meas_noise<double>(m, j, (uint32_t)i);
      double e, uhat;
      const double F = pi_step<double>(c, m.Ts, zi, y, Fss(m, tp.EaR_c, zi), Ih2, &e, &uhat);
      // substep states and noise of this sample
      for (int s = 0; s < m.n_em; ++s) {
        const int64_t ks = (int64_t)i * m.n_em + s;
        double xi[3];
        process_noise<double>(m, j, (uint32_t)ks, xi);
        sub[s][0] = ns[0];
        sub[s][1] = ns[1];
        sub[s][2] = ns[2];
        sub[s][3] = xi[0];
        sub[s][4] = xi[1];
        sub[s][5] = xi[2];
        em_step<double>(m, tp.EaR, inlet_T(m, tp, ks, h), ns, F, h, sqh, xi);
      }
      double Fb = 0.0;
      for (int s = m.n_em - 1; s >= 0; --s) {
        const int64_t ks = (int64_t)i * m.n_em + s;
        em_step_adjoint(m, tp.EaR, inlet_T(m, tp, ks, h), &sub[s][0], F, h, sqh, &sub[s][3],
                        nb, Fb);
      }
      // Eq. (PI) backwards: I-hat+ = I + Ts k_aw (u-hat - u), u = clip(u-hat),
      // u-hat = u-bar + k_P e + I, I = I-hat + Ts k_I e, e = z-bar - y
      double ub = Fb;
      double Ilb = Ib;
      double uhb = Ts * c.kaw * Ib;
      ub -= Ts * c.kaw * Ib;
      gaw += Ts * (uhat - F) * Ib;
      if (uhat > umin && uhat < umax) uhb += ub;
      Ilb += uhb;
      gP += e * uhb;
      double eb = c.kP * uhb;
      gI += Ts * e * Ilb;
      eb += Ts * c.kI * Ilb;
      Ib = Ilb;
      // y = c_T + v; the Phi term of sample i
      const double cTb = -eb + 2.0 * (cT - zi) * wK;
      nb[2] += cTb / m.V;
    }
  }
  dphi[jj * 3 + 0] = gP;
  dphi[jj * 3 + 1] = gI;
  dphi[jj * 3 + 2] = gaw;
}

// Mean of dPhi_j over the trajectories of j0 .. j1-1 with a finite Phi_j, in
// a fixed order (one block: strided partial sums, then a tree); out = (mean
// of the three derivatives, number of finite trajectories).
constexpr int kGradThreads = 256;
__global__ void __launch_bounds__(kGradThreads) k_grad_mean(const double* __restrict__ phi,
                                                            const double* __restrict__ dphi,
                                                            int64_t j0, int64_t j1,
                                                            double* __restrict__ out) {
  __shared__ double sh[4][kGradThreads];
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, n = 0.0;
  for (int64_t jj = j0 + threadIdx.x; jj < j1; jj += kGradThreads) {
    if (isfinite(phi[jj])) {
      a0 += dphi[jj * 3 + 0];
      a1 += dphi[jj * 3 + 1];
      a2 += dphi[jj * 3 + 2];
      n += 1.0;
    }
  }
  const int t = threadIdx.x;
  sh[0][t] = a0;
  sh[1][t] = a1;
  sh[2][t] = a2;
  sh[3][t] = n;
  __syncthreads();
  for (int w = kGradThreads / 2; w > 0; w >>= 1) {
    if (t < w)
      for (int q = 0; q < 4; ++q) sh[q][t] += sh[q][t + w];
    __syncthreads();
  }
  if (t == 0) {
    const double cnt = sh[3][0];
    for (int q = 0; q < 3; ++q) out[q] = cnt > 0 ? sh[q][0] / cnt : 0.0;
    out[3] = cnt;
  }
}

}  // namespace mc
