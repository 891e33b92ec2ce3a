// mc_capi.cu -- kernels and the C ABI declared in include/mc.h.
//
// Kernels:
//   k_nmpc       one thread per NMPC trajectory (grid-stride over trajectories),
//                per-thread arrays in a structure-of-arrays scratch buffer
//   k_pi         one thread per PI trajectory, registers only
//   k_stats_*    reduction of Phi and of the per-trajectory counters: block
//                partials (count/mean/M2 merged by Chan's formula, min, max,
//                counter sums) then one block merging them and binning Phi
//   k_philox, k_noise, k_qp_batch, k_ocp_batch   building blocks on their own
#include <chrono>
#include <cmath>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include <cuda.h>  // driver types for SM partitions; entry points are resolved at run time

#include "../../include/mc.h"
#include "mc_closedloop.cuh"
#include "mc_grad.cuh"
#include "mc_qp_par.cuh"
#include "mc_nmpc3.cuh"
#include "mc_grad_nmpc.cuh"
#include "mc_peaks.cuh"

namespace mc {

// --------------------------------------------------------------- kernels

template <class R>
__global__ void __launch_bounds__(32) k_nmpc(DevModel m, DevCtrl c, int64_t j0, int64_t j1,
                                              double* __restrict__ phi,
                                              int32_t* __restrict__ cnt, double* ws,
                                              int64_t ld) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ld) return;
  const Ws w{ws + t, ld, c.N + 1};
  for (int64_t j = j0 + t; j < j1; j += ld) {
    const TrajOut o = traj_nmpc<R>(m, c, (uint32_t)j, w);
    phi[j] = o.phi;
#pragma unroll
    for (int q = 0; q < kNCounters; ++q) cnt[j * kNCounters + q] = o.cnt[q];
  }
}

// The NMPC closed loop with the tangents of Phi_j in the weights (Q_z, R_u,
// Q_n) (FP64, static schedule); dphi is n_sims x 3, tg kTgRows rows of ld
// columns (the tangents in flight).
__global__ void __launch_bounds__(32) k_nmpc_grad(DevModel m, DevCtrl c, int64_t j0, int64_t j1,
                                                  double* __restrict__ phi,
                                                  int32_t* __restrict__ cnt,
                                                  double* __restrict__ dphi, double* ws,
                                                  int64_t ld, double* tg) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ld) return;
  const Ws w{ws + t, ld, c.N + 1};
  const Tg g{tg + t, ld};
  for (int64_t j = j0 + t; j < j1; j += ld) {
    const TrajOut o = traj_nmpc_grad(m, c, (uint32_t)j, w, g);
    phi[j] = o.phi;
#pragma unroll
    for (int q = 0; q < kNCounters; ++q) cnt[j * kNCounters + q] = o.cnt[q];
    grad_finish(m, o.phi, g, dphi + j * 3);
  }
}

// The NMPC closed loop on the persistent schedule (FP64, launched as
// k_nmpc_persist) that records, per sample, what the tangents of Phi_j need
// (Recorder: trajectories rc.j0 .. rc.j0 + n - 1).
__global__ void __launch_bounds__(32) k_nmpc_persist_rec(DevModel m, DevCtrl c, int64_t n,
                                                         const uint32_t* order,
                                                         unsigned long long* next,
                                                         double* __restrict__ phi,
                                                         int32_t* __restrict__ cnt, double* ws,
                                                         int64_t ld, double* nz,
                                                         unsigned long long* wtrace,
                                                         Recorder rc) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const Ws w{ws + t, ld, c.N + 1};
  nmpc_persistent<double, Recorder>(m, c, w, nz + t, rc.j0, n, order, next, phi, cnt, wtrace,
                                    rc);
}

// The tangents of Phi_j through the recorded samples of trajectories
// rc.j0 .. rc.j0 + n - 1, one thread per trajectory, ld threads (ld columns
// of scratch and of tg, the tangents in flight); dphi is n_sims x 3.
__global__ void __launch_bounds__(kTangentThreads) k_nmpc_tangent(DevModel m, DevCtrl c,
                                                                  int64_t n,
                                                                  const double* __restrict__ phi,
                                                                  int32_t* __restrict__ cnt,
                                                                  double* __restrict__ dphi,
                                                                  double* ws, int64_t ld,
                                                                  double* tg, Recorder rc) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ld) return;
  const Ws w{ws + t, ld, c.N + 1};
  const Tg g{tg + t, ld};
  for (int64_t q = t; q < n; q += ld) {
    const int64_t j = rc.j0 + q;
    traj_nmpc_tangent(m, c, (uint32_t)j, w, g, rc, phi[j], cnt + j * kNCounters + 7,
                      dphi + j * 3);
  }
}

// The three-state NMPC closed loop (FP64, static schedule).
__global__ void __launch_bounds__(32) k_nmpc3(DevModel m, DevCtrl c, int64_t j0, int64_t j1,
                                              double* __restrict__ phi,
                                              int32_t* __restrict__ cnt, double* ws,
                                              int64_t ld) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ld) return;
  const Ws w{ws + t, ld, c.N + 1};
  for (int64_t j = j0 + t; j < j1; j += ld) {
    const TrajOut o = traj_nmpc3(m, c, (uint32_t)j, w);
    phi[j] = o.phi;
#pragma unroll
    for (int q = 0; q < kNCounters; ++q) cnt[j * kNCounters + q] = o.cnt[q];
  }
}

// The three-state NMPC closed loop on the persistent schedule (one warp per
// block, every lane in the warp votes of nmpc3_persistent).
__global__ void __launch_bounds__(32) k_nmpc3_persist(DevModel m, DevCtrl c, int64_t j0,
                                                      int64_t n, const uint32_t* order,
                                                      unsigned long long* next,
                                                      double* __restrict__ phi,
                                                      int32_t* __restrict__ cnt, double* ws,
                                                      int64_t ld) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const Ws w{ws + t, ld, c.N + 1};
  nmpc3_persistent(m, c, w, j0, n, order, next, phi, cnt);
}

template <class R>
__global__ void __launch_bounds__(32) k_nmpc_persist(DevModel m, DevCtrl c, int64_t j0,
                                                     int64_t n, const uint32_t* order,
                                                     unsigned long long* next,
                                                     double* __restrict__ phi,
                                                     int32_t* __restrict__ cnt, double* ws,
                                                     int64_t ld, double* nz,
                                                     unsigned long long* wtrace) {
  // launched with whole warps and at most ld threads; every lane takes part in
  // the warp votes of nmpc_persistent.  nz: 3 n_em rows of ld columns, the
  // pooled plant noise; wtrace: the per-warp record (may be null).
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const Ws w{ws + t, ld, c.N + 1};
  nmpc_persistent<R>(m, c, w, nz + t, j0, n, order, next, phi, cnt, wtrace);
}

template <class R>
__global__ void __launch_bounds__(128) k_pi(DevModel m, DevCtrl c, int64_t j0, int64_t j1,
                                            double* __restrict__ phi,
                                            int32_t* __restrict__ cnt) {
  const int64_t j = j0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= j1) return;
  const TrajOut o = traj_pi<R>(m, c, (uint32_t)j);
  phi[j] = o.phi;
#pragma unroll
  for (int q = 0; q < kNCounters; ++q) cnt[j * kNCounters + q] = o.cnt[q];
}

struct Partial {
  double n, mean, m2, mn, mx;
  long long sums[kNCounters];
  long long n_nonfinite;
};

// Chan et al. merge of (count, mean, M2).
__device__ __forceinline__ void chan_merge(double& n, double& mean, double& m2, double nb,
                                           double meanb, double m2b) {
  if (nb == 0.0) return;
  if (n == 0.0) {
    n = nb;
    mean = meanb;
    m2 = m2b;
    return;
  }
  const double nt = n + nb;
  const double d = meanb - mean;
  mean = mean + d * (nb / nt);
  m2 = m2 + m2b + d * d * (n * nb / nt);
  n = nt;
}

constexpr int kStatThreads = 256;

__device__ void block_reduce_partial(Partial& p) {
  __shared__ double sh[kStatThreads / 32][5];
  __shared__ long long shc[kStatThreads / 32][kNCounters + 1];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int off = 16; off > 0; off >>= 1) {
    const double nb = __shfl_down_sync(0xffffffffu, p.n, off);
    const double mb = __shfl_down_sync(0xffffffffu, p.mean, off);
    const double qb = __shfl_down_sync(0xffffffffu, p.m2, off);
    const double mnb = __shfl_down_sync(0xffffffffu, p.mn, off);
    const double mxb = __shfl_down_sync(0xffffffffu, p.mx, off);
    chan_merge(p.n, p.mean, p.m2, nb, mb, qb);
    p.mn = fmin(p.mn, mnb);
    p.mx = fmax(p.mx, mxb);
    for (int q = 0; q < kNCounters; ++q) p.sums[q] += __shfl_down_sync(0xffffffffu, p.sums[q], off);
    p.n_nonfinite += __shfl_down_sync(0xffffffffu, p.n_nonfinite, off);
  }
  if (lane == 0) {
    sh[wid][0] = p.n; sh[wid][1] = p.mean; sh[wid][2] = p.m2; sh[wid][3] = p.mn; sh[wid][4] = p.mx;
    for (int q = 0; q < kNCounters; ++q) shc[wid][q] = p.sums[q];
    shc[wid][kNCounters] = p.n_nonfinite;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int v = 1; v < kStatThreads / 32; ++v) {
      chan_merge(p.n, p.mean, p.m2, sh[v][0], sh[v][1], sh[v][2]);
      p.mn = fmin(p.mn, sh[v][3]);
      p.mx = fmax(p.mx, sh[v][4]);
      for (int q = 0; q < kNCounters; ++q) p.sums[q] += shc[v][q];
      p.n_nonfinite += shc[v][kNCounters];
    }
  }
}

__device__ __forceinline__ Partial empty_partial() {
  Partial p;
  p.n = 0.0; p.mean = 0.0; p.m2 = 0.0; p.mn = INFINITY; p.mx = -INFINITY;
  for (int q = 0; q < kNCounters; ++q) p.sums[q] = 0;
  p.n_nonfinite = 0;
  return p;
}

// Block partials over trajectories j0 .. j1-1 (grid-stride).
__global__ void __launch_bounds__(kStatThreads) k_stats_partial(const double* __restrict__ phi,
                                                                 const int32_t* __restrict__ cnt,
                                                                 int64_t j0, int64_t j1,
                                                                 Partial* __restrict__ part) {
  Partial p = empty_partial();
  for (int64_t j = j0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < j1;
       j += (int64_t)gridDim.x * blockDim.x) {
    const double v = phi[j];
    if (isfinite(v)) {
      chan_merge(p.n, p.mean, p.m2, 1.0, v, 0.0);
      p.mn = fmin(p.mn, v);
      p.mx = fmax(p.mx, v);
    } else {
      p.n_nonfinite++;
    }
    for (int q = 0; q < kNCounters; ++q) p.sums[q] += cnt[j * kNCounters + q];
  }
  block_reduce_partial(p);
  if (threadIdx.x == 0) part[blockIdx.x] = p;
}

struct DevStats {
  double n, mean, m2, mn, mx, lo, hi;
  long long sums[kNCounters];
  long long n_nonfinite;
  long long hist[MC_MAX_BINS];
};

// One block: merge the partials, fix the histogram range, bin Phi.
__global__ void __launch_bounds__(kStatThreads) k_stats_final(const Partial* __restrict__ part,
                                                               int nparts,
                                                               const double* __restrict__ phi,
                                                               int64_t j0, int64_t j1, int n_bins,
                                                               double lo, double hi,
                                                               DevStats* __restrict__ out) {
  __shared__ unsigned long long hist[MC_MAX_BINS];
  __shared__ double range[2];
  Partial p = empty_partial();
  for (int b = threadIdx.x; b < nparts; b += blockDim.x) {
    const Partial& q = part[b];
    chan_merge(p.n, p.mean, p.m2, q.n, q.mean, q.m2);
    p.mn = fmin(p.mn, q.mn);
    p.mx = fmax(p.mx, q.mx);
    for (int k = 0; k < kNCounters; ++k) p.sums[k] += q.sums[k];
    p.n_nonfinite += q.n_nonfinite;
  }
  for (int b = threadIdx.x; b < MC_MAX_BINS; b += blockDim.x) hist[b] = 0ull;
  block_reduce_partial(p);
  if (threadIdx.x == 0) {
    double l = lo, h = hi;
    if (!(l < h)) {
      l = p.mn;
      h = p.mx;
      if (!(l < h)) h = l + 1.0;
    }
    range[0] = l;
    range[1] = h;
    out->n = p.n; out->mean = p.mean; out->m2 = p.m2; out->mn = p.mn; out->mx = p.mx;
    out->lo = l; out->hi = h;
    for (int k = 0; k < kNCounters; ++k) out->sums[k] = p.sums[k];
    out->n_nonfinite = p.n_nonfinite;
  }
  __syncthreads();
  const double l = range[0], scale = (double)n_bins / (range[1] - range[0]);
  for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
    const double v = phi[j];
    if (!isfinite(v)) continue;
    int b = (int)floor((v - l) * scale);
    b = b < 0 ? 0 : (b >= n_bins ? n_bins - 1 : b);
    atomicAdd(&hist[b], 1ull);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < MC_MAX_BINS; b += blockDim.x)
    out->hist[b] = (b < n_bins) ? (long long)hist[b] : 0;
}

__global__ void k_philox(const uint4* __restrict__ ctr, uint32_t k0, uint32_t k1, int64_t n,
                         uint4* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = philox4x32_10(ctr[i], k0, k1);
}

template <bool kRcp>
__global__ void k_elementary(const double* __restrict__ x, int64_t n, double* __restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = kRcp ? rcp_newton(x[i]) : expr(x[i]);
}

__global__ void k_noise(DevModel m, uint32_t j, int64_t k0, int64_t nk, int precision,
                        double* __restrict__ out, double* __restrict__ meas) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nk) return;
  const uint32_t k = (uint32_t)(k0 + i);
  if (precision == 0) {
    double xi[3];
    process_noise<double>(m, j, k, xi);
    out[3 * i] = xi[0]; out[3 * i + 1] = xi[1]; out[3 * i + 2] = xi[2];
    meas[i] = meas_noise<double>(m, j, k);
  } else {
    float xi[3];
    process_noise<float>(m, j, k, xi);
    out[3 * i] = xi[0]; out[3 * i + 1] = xi[1]; out[3 * i + 2] = xi[2];
    meas[i] = meas_noise<float>(m, j, k);
  }
}

struct QpBatch {
  const double *A, *B, *b, *Wxx, *Wxu, *Wuu, *q, *r, *lb, *ub;
  double *du, *dx, *mu, *nul, *nuu;
  int32_t *iters, *status;
};

__global__ void k_qp_batch(int N, int64_t n, int solver, int max_it, double tol, QpBatch d,
                           double* ws, int64_t ld) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const Ws w{ws + t, ld, N + 1};
  const int64_t o1 = t * N, o2 = t * (N + 1);
  for (int k = 0; k < N; ++k) {
    w(EA, k) = d.A[o1 + k];
    w(EB, k) = d.B[o1 + k];
    w(EG, k) = d.b[o1 + k];
    w(QR, k) = d.r[o1 + k];
    w(LB, k) = d.lb[o1 + k];
    w(UB, k) = d.ub[o1 + k];
  }
  for (int k = 0; k <= N; ++k) {
    w(WXX, k) = d.Wxx[o2 + k];
    w(WXU, k) = d.Wxu[o2 + k];
    w(WUU, k) = d.Wuu[o2 + k];
    w(EQ, k) = d.q[o2 + k];
  }
  const QpResult r = (solver == MC_QP_IPM) ? qp_ipm(w, N, true, max_it, tol)
                                            : qp_active_set(w, N, true, max_it);
  for (int k = 0; k < N; ++k) {
    d.du[o1 + k] = w(DU, k);
    d.mu[o1 + k] = w(MU, k);
    d.nul[o1 + k] = w(NUL, k);
    d.nuu[o1 + k] = w(NUU, k);
  }
  d.dx[o2] = 0.0;
  for (int k = 1; k <= N; ++k) d.dx[o2 + k] = w(DX, k);
  d.iters[t] = r.iters;
  d.status[t] = r.status;
}

// One warp per QP: the parallel-in-horizon solver (lanes over the stages).
constexpr int kQpWarpsPerBlock = 4;
__global__ void __launch_bounds__(32 * kQpWarpsPerBlock)
    k_qp_batch_warp(int N, int64_t n, int max_it, QpBatch d, double* ws, int64_t ld) {
  const int64_t t = (int64_t)blockIdx.x * kQpWarpsPerBlock + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (t >= n) return;  // whole warps leave together
  const Ws w{ws + t, ld, N + 1};
  const int64_t o1 = t * N, o2 = t * (N + 1);
  for (int k = lane; k < N; k += 32) {
    w(EA, k) = d.A[o1 + k];
    w(EB, k) = d.B[o1 + k];
    w(EG, k) = d.b[o1 + k];
    w(QR, k) = d.r[o1 + k];
    w(LB, k) = d.lb[o1 + k];
    w(UB, k) = d.ub[o1 + k];
  }
  for (int k = lane; k <= N; k += 32) {
    w(WXX, k) = d.Wxx[o2 + k];
    w(WXU, k) = d.Wxu[o2 + k];
    w(WUU, k) = d.Wuu[o2 + k];
    w(EQ, k) = d.q[o2 + k];
  }
  __syncwarp();
  const QpResult r = qp_active_set_warp(w, N, true, max_it, lane);
  __syncwarp();
  for (int k = lane; k < N; k += 32) {
    d.du[o1 + k] = w(DU, k);
    d.mu[o1 + k] = w(MU, k);
    d.nul[o1 + k] = w(NUL, k);
    d.nuu[o1 + k] = w(NUU, k);
    d.dx[o2 + k + 1] = w(DX, k + 1);
  }
  if (lane == 0) {
    d.dx[o2] = 0.0;
    d.iters[t] = r.iters;
    d.status[t] = r.status;
  }
}

struct OcpBatch {
  const double *x0, *EaR, *zbar;
  double *u, *x, *lam, *pil, *piu, *kkt;
  int32_t* info;
};

__global__ void k_ocp_batch(DevModel m, DevCtrl c, int64_t n, OcpBatch d, double* ws,
                            int64_t ld) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int N = c.N;
  const Ws w{ws + t, ld, N + 1};
  const int64_t o1 = t * N, o2 = t * (N + 1);
  for (int k = 0; k < N; ++k) {
    w(U, k) = d.u[o1 + k];
    w(LAM, k) = d.lam[o1 + k];
    w(PIL, k) = d.pil[o1 + k];
    w(PIU, k) = d.piu[o1 + k];
  }
  for (int k = 0; k <= N; ++k) {
    w(X, k) = d.x[o2 + k];
    w(ZB, k) = d.zbar[o2 + k];
    if (c.Ru != 0.0 && k >= 1) w(VB, k) = Fss(m, d.EaR[t], w(ZB, k)) / c.Fconv;
  }
  const SqpInfo si = (c.precision == MC_MIXED) ? sqp_solve<float>(m, c, d.EaR[t], d.x0[t], w)
                                               : sqp_solve<double>(m, c, d.EaR[t], d.x0[t], w);
  for (int k = 0; k < N; ++k) {
    d.u[o1 + k] = w(U, k);
    d.lam[o1 + k] = w(LAM, k);
    d.pil[o1 + k] = w(PIL, k);
    d.piu[o1 + k] = w(PIU, k);
  }
  for (int k = 0; k <= N; ++k) d.x[o2 + k] = w(X, k);
  d.info[4 * t + 0] = si.iters;
  d.info[4 * t + 1] = si.status;
  d.info[4 * t + 2] = si.ls_trials;
  d.info[4 * t + 3] = si.qp_iters;
  d.kkt[3 * t + 0] = si.kkt_grad;
  d.kkt[3 * t + 1] = si.kkt_eq;
  d.kkt[3 * t + 2] = si.f;
}

// du_0/d(x_0, Q_z, R_u, Q_n) at given OCP solutions (one thread per OCP).
__global__ void k_ocp_sens_batch(DevModel m, DevCtrl c, int64_t n, OcpBatch d, double* sens,
                                 double* ws, int64_t ld) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int N = c.N;
  const Ws w{ws + t, ld, N + 1};
  const int64_t o1 = t * N, o2 = t * (N + 1);
  for (int k = 0; k < N; ++k) {
    w(U, k) = d.u[o1 + k];
    w(LAM, k) = d.lam[o1 + k];
    w(PIL, k) = d.pil[o1 + k];
    w(PIU, k) = d.piu[o1 + k];
  }
  for (int k = 0; k <= N; ++k) {
    w(X, k) = d.x[o2 + k];
    w(ZB, k) = d.zbar[o2 + k];
    if (k >= 1) w(VB, k) = Fss(m, d.EaR[t], w(ZB, k)) / c.Fconv;
  }
  w(X, 0) = d.x0[t];
  double out[4];
  const bool ok = ocp_sens(m, c, d.EaR[t], N, w, out);
  for (int q = 0; q < 4; ++q) sens[t * 4 + q] = out[q];
  d.info[t] = ok ? 0 : 1;
}

}  // namespace mc

// =========================================================================
// host side
// =========================================================================

using namespace mc;

namespace {

thread_local std::string g_create_error;

// One warp per block: the FP64 pipe's time on an SM is proportional to the
// number of warps it holds, so warp-sized blocks spread the trajectories over
// the 152 SMs as evenly as the warp granularity allows.
constexpr int kNmpcThreads = 32;
constexpr int kMaxStatBlocks = 1024;
// Device memory the persistent NMPC gradient's sample records may take: 6.5 GB
// hold the 30,000-trajectory, 240-step, N = 20 study in one chunk.
constexpr size_t kRecordBudget = (size_t)8 << 30;

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace

struct mc_handle {
  DevModel m;
  DevCtrl c;
  int64_t n_sims = 0;
  int n_bins = 64;
  double bin_lo = 0.0, bin_hi = 0.0;
  double* phi = nullptr;       // n_sims
  int32_t* cnt = nullptr;      // n_sims x kNCounters
  double* ws = nullptr;        // NMPC scratch: kNArr * (N+1) x ws_ld
  double* nz = nullptr;        // inside ws: 3 n_em x ws_ld plant normals (one-state)
  int64_t ws_ld = 0;
  int schedule = MC_SCHED_STATIC;
  uint32_t* order = nullptr;   // trajectories, longest horizon first (uneven batches)
  unsigned long long* next = nullptr;  // queue position of the persistent schedule
  int64_t persist_threads = 0;
  bool use_graph = false;
  struct Graph {
    int64_t j0, j1;
    cudaGraphExec_t exec;
  };
  std::vector<Graph> graphs;   // captured runs, by trajectory range
  Partial* part = nullptr;     // kMaxStatBlocks
  DevStats* dstats = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  bool ran = false;
  int64_t last_j0 = 0, last_j1 = 0;
  // gradients of the PI study (allocated by the first mc_pi_grad)
  double* dphi = nullptr;      // n_sims x 3
  double* ck = nullptr;        // checkpoints, 4 x n_ck x n_sims
  int64_t ck_words = 0;
  double* gmean = nullptr;     // mean gradient and the finite count
  double* tg = nullptr;        // NMPC tangents in flight, kTgRows x ws_ld
  double* rec = nullptr;       // the persistent NMPC gradient's sample records
  size_t rec_bytes = 0;
  size_t rec_budget = kRecordBudget;  // bytes the records may take
  int32_t* kj = nullptr;       // the sample each recorded trajectory ended at
  // per-warp record of the last one-state persistent launch (ws_ld / 32 warps)
  unsigned long long* wtrace = nullptr;
  int64_t wtrace_warps = 0;
  bool grad_ran = false;
  // SM partition (green context): launches go to pstream, forked from and
  // joined back into the caller's stream
  CUgreenCtx gctx = nullptr;
  CUstream pstream = nullptr;
  int part_sms = 0;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  std::string err;
};

static mc_status fail(mc_handle* h, mc_status s, const std::string& msg) {
  if (h)
    h->err = msg;
  else
    g_create_error = msg;
  return s;
}

static mc_status cuda_fail(mc_handle* h, cudaError_t e, const char* what) {
  return fail(h, MC_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define MC_CUDA(h, call)                                   \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail((h), e_, #call); \
  } while (0)

static mc_status fill_dev(const mc_model_t* mm, const mc_controller_t* cc, uint64_t seed,
                          DevModel* m, DevCtrl* c, std::string* why) {
  auto bad = [&](const char* s) {
    *why = s;
    return MC_EINVAL;
  };
  if (!mm || !cc) return bad("null model or controller");
  if (!(mm->V > 0) || !(mm->beta > 0) || !(mm->k0 >= 0) || !(mm->EaR > 0))
    return bad("CSTR parameters must be positive (V, beta, EaR > 0, k0 >= 0)");
  if (!(mm->Ts > 0) || mm->n_em < 1 || mm->n_steps < 0)
    return bad("need Ts > 0, n_em >= 1, n_steps >= 0");
  if (mm->n_setpoints < 1 || mm->n_setpoints > MC_MAX_SETPOINTS || !mm->sp_time || !mm->sp_value)
    return bad("need 1..16 set-point segments with time and value arrays");
  if (!(mm->meas_sd >= 0) || !(mm->sigma[0] >= 0) || !(mm->sigma[1] >= 0) || !(mm->sigma[2] >= 0))
    return bad("noise intensities must be non-negative");
  if ((int64_t)mm->n_steps * mm->n_em >= (int64_t)1 << 32)
    return bad("n_steps * n_em must stay below 2^32 (Philox counter word)");
  if (cc->kind != MC_CTRL_NMPC && cc->kind != MC_CTRL_PI) return bad("unknown controller kind");
  if (cc->precision != MC_FP64 && cc->precision != MC_MIXED) return bad("unknown precision");
  if (!(cc->u_min <= cc->u_max)) return bad("need u_min <= u_max");
  if (cc->kind == MC_CTRL_NMPC) {
    if (cc->N < 1 || cc->N > MC_MAX_HORIZON) return bad("NMPC horizon N must be in 1..64");
    if (cc->n_rk4 < 1) return bad("n_rk4 must be >= 1");
    if (cc->sqp_max_it < 0 || cc->ls_max < 0) return bad("iteration limits must be >= 0");
    if (!(cc->sqp_tol > 0)) return bad("sqp_tol must be > 0");
    if (!(mm->meas_sd > 0)) return bad("the CD-EKF needs a measurement noise sd > 0");
    if (!(cc->u_scale > 0) || !(cc->x_scale > 0)) return bad("u_scale and x_scale must be > 0");
    if (cc->qp_solver == MC_QP_ACTIVE_SET_WARP)
      return bad("the warp-per-QP solver is a building block (mc_qp_solve_batch); the closed "
                 "loop runs one trajectory per lane");
    if (cc->qp_solver != MC_QP_ACTIVE_SET && cc->qp_solver != MC_QP_IPM)
      return bad("unknown QP solver");
    if (cc->qp_solver == MC_QP_IPM && (cc->ip_max_it < 1 || !(cc->ip_tol > 0)))
      return bad("the interior-point solver needs ip_max_it >= 1 and ip_tol > 0");
    if (cc->N_min < 0 || cc->N_min > cc->N) return bad("need 0 <= N_min <= N");
    if (cc->sqp_max_it_min < 0 || cc->sqp_max_it_min > cc->sqp_max_it)
      return bad("need 0 <= sqp_max_it_min <= sqp_max_it");
    if (cc->schedule != MC_SCHED_STATIC && cc->schedule != MC_SCHED_PERSISTENT)
      return bad("unknown schedule");
    if (cc->threads_per_sm < 0 || cc->threads_per_sm > 2048)
      return bad("threads_per_sm must be 0..2048");
    if (cc->ls_spec_lanes > 32) return bad("ls_spec_lanes must be <= 32");
    if (cc->nx_model != 0 && cc->nx_model != 1 && cc->nx_model != 3)
      return bad("nx_model must be 0, 1 or 3");
    if (!(cc->Ru >= 0.0) || !(cc->Qn >= 0.0) || !std::isfinite(cc->Ru) || !std::isfinite(cc->Qn))
      return bad("the objective weights Ru and Qn must be finite and >= 0");
    if (cc->nx_model == 3 && (cc->Ru != 0.0 || cc->Qn != 0.0))
      return bad("the three-state NMPC has the paper's objective only (Ru = Qn = 0)");
    if (cc->nx_model == 3 && (cc->precision != MC_FP64 || cc->qp_solver != MC_QP_ACTIVE_SET))
      return bad("the three-state NMPC runs in FP64 with the active-set QP");
  }
  memset(m, 0, sizeof(*m));
  m->V = mm->V; m->k0 = mm->k0; m->EaR = mm->EaR; m->beta = mm->beta;
  m->cA_in = mm->cA_in; m->cB_in = mm->cB_in; m->T_in = mm->T_in;
  for (int i = 0; i < 3; ++i) m->sigma[i] = mm->sigma[i];
  m->meas_sd = mm->meas_sd; m->Ts = mm->Ts; m->t0 = mm->t0;
  m->n_steps = mm->n_steps; m->n_em = mm->n_em; m->n_sp = mm->n_setpoints;
  for (int s = 0; s < mm->n_setpoints; ++s) {
    m->sp_time[s] = mm->sp_time[s];
    m->sp_value[s] = mm->sp_value[s];
    if (s > 0 && !(mm->sp_time[s] > mm->sp_time[s - 1]))
      return bad("set-point times must increase");
  }
  if (mm->Ea_plant_only != 0 && mm->Ea_plant_only != 1) return bad("Ea_plant_only must be 0 or 1");
  m->Ea_logsd = mm->Ea_logsd; m->dTin = mm->dT_in_step;
  m->Ea_plant_only = mm->Ea_plant_only;
  m->iV = 1.0 / mm->V; m->ib = 1.0 / mm->beta;
  m->rw0 = m->ib * (mm->cB_in + 2.0 * mm->cA_in);
  m->rw1 = 4.0 * m->ib * m->ib;
  m->bV = mm->beta * mm->V;
  m->ib2 = 2.0 * m->ib;
  m->key0 = (uint32_t)seed; m->key1 = (uint32_t)(seed >> 32);
  m->lnk0 = std::log(mm->k0);   // -inf for k0 = 0: the rate vanishes
  m->hEM = mm->Ts / (double)mm->n_em;
  m->sqhEM = std::sqrt(m->hEM);
  // first sample index of each set-point segment: the smallest i >= 0 with
  // t0 + i Ts >= sp_time[s], the time formed as product then sum
  m->sp_step[0] = 0;
  for (int s = 1; s < mm->n_setpoints; ++s) {
    const double est = (mm->sp_time[s] - mm->t0) / mm->Ts;
    if (!(est < 2.0e9)) {
      m->sp_step[s] = INT32_MAX;
      continue;
    }
    int64_t i = est > 2.0 ? (int64_t)std::floor(est) - 2 : 0;
    for (;;) {
      volatile double prod = (double)i * mm->Ts;
      const double t = mm->t0 + prod;
      if (t >= mm->sp_time[s] || i >= INT32_MAX) break;
      ++i;
    }
    m->sp_step[s] = (int)i;
  }
  memset(c, 0, sizeof(*c));
  c->kind = cc->kind; c->precision = cc->precision; c->N = cc->N; c->n_rk4 = cc->n_rk4;
  c->sqp_max_it = cc->sqp_max_it; c->ls_max = cc->ls_max; c->qp_solver = cc->qp_solver;
  c->spec_lanes = cc->ls_spec_lanes == 0 ? 32 : (cc->ls_spec_lanes < 0 ? 0 : cc->ls_spec_lanes);
  c->ip_max_it = cc->ip_max_it;
  c->u_min = cc->u_min; c->u_max = cc->u_max; c->kP = cc->kP; c->kI = cc->kI; c->kaw = cc->kaw;
  c->Qz = cc->Qz; c->P0 = cc->P0; c->sqp_tol = cc->sqp_tol; c->ip_tol = cc->ip_tol;
  c->u_scale = cc->u_scale; c->x_scale = cc->x_scale;
  c->N_min = cc->N_min; c->it_min = cc->sqp_max_it_min;
  c->nx_model = (cc->kind == MC_CTRL_NMPC && cc->nx_model == 3) ? 3 : 1;
  c->Ru = (cc->kind == MC_CTRL_NMPC) ? cc->Ru : 0.0;
  c->Qn = (cc->kind == MC_CTRL_NMPC) ? cc->Qn : 0.0;
  c->r_scale = 2.0 * c->Ru * mm->Ts;
  if (cc->kind == MC_CTRL_NMPC) {
    c->Fconv = cc->u_scale / 60000.0;
    c->vmin = cc->u_min / cc->u_scale;
    c->vmax = cc->u_max / cc->u_scale;
  }
  return MC_OK;
}

template <class T>
static bool to_dev(T** d, const T* h, size_t n) {
  if (cudaMalloc((void**)d, sizeof(T) * (n ? n : 1)) != cudaSuccess) return false;
  if (n && h && cudaMemcpy(*d, h, sizeof(T) * n, cudaMemcpyHostToDevice) != cudaSuccess)
    return false;
  return true;
}

static int64_t nmpc_threads_for(int64_t n, int nx_model) {
  // every trajectory gets its own thread while they fit on the GPU at once
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int per_sm = 0;
  const cudaError_t oe =
      (nx_model == 3)
          ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_nmpc3, kNmpcThreads, 0)
          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_nmpc<double>, kNmpcThreads,
                                                          0);
  if (oe != cudaSuccess || per_sm < 1) per_sm = 4;
  const int64_t cap = (int64_t)sms * per_sm * kNmpcThreads;
  // equal numbers of trajectories per thread when they exceed the resident threads
  const int64_t passes = (n + cap - 1) / cap;
  int64_t t = passes > 0 ? (n + passes - 1) / passes : 0;
  t = (t + kNmpcThreads - 1) / kNmpcThreads * kNmpcThreads;
  return t < kNmpcThreads ? kNmpcThreads : t;
}

extern "C" {

const char* mc_status_str(mc_status s) {
  switch (s) {
    case MC_OK: return "ok";
    case MC_EINVAL: return "invalid argument";
    case MC_ENOMEM: return "out of device memory";
    case MC_ECUDA: return "CUDA error";
    case MC_ETIMEOUT: return "timed out waiting for the GPU";
    case MC_ENOTRUN: return "no run yet";
    case MC_WARN_NONFINITE: return "some trajectories became non-finite";
  }
  return "unknown status";
}

const char* mc_last_error(const mc_handle* h) {
  return h ? h->err.c_str() : g_create_error.c_str();
}

static void drop_graphs(mc_handle* h);
static void drop_partition(mc_handle* h);

void mc_destroy(mc_handle* h) {
  if (!h) return;
  drop_graphs(h);
  cudaFree(h->phi);
  cudaFree(h->cnt);
  cudaFree(h->ws);
  cudaFree(h->part);
  cudaFree(h->dstats);
  cudaFree(h->order);
  cudaFree(h->next);
  cudaFree(h->dphi);
  cudaFree(h->ck);
  cudaFree(h->gmean);
  cudaFree(h->tg);
  cudaFree(h->rec);
  cudaFree(h->kj);
  cudaFree(h->wtrace);
  drop_partition(h);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  delete h;
}

mc_status mc_create(const mc_model_t* model, const mc_controller_t* ctrl, int64_t n_sims,
                    uint64_t seed, mc_handle** out) {
  if (!out) return fail(nullptr, MC_EINVAL, "out is null");
  *out = nullptr;
  if (n_sims < 0 || n_sims > ((int64_t)1 << 32))
    return fail(nullptr, MC_EINVAL, "n_sims must be in 0..2^32");
  auto* h = new mc_handle();
  std::string why;
  if (fill_dev(model, ctrl, seed, &h->m, &h->c, &why) != MC_OK) {
    delete h;
    return fail(nullptr, MC_EINVAL, why);
  }
  h->n_sims = n_sims;
  h->schedule = ctrl->schedule;
  auto alloc = [&](void** p, size_t bytes) -> bool {
    if (bytes == 0) bytes = 8;
    return cudaMalloc(p, bytes) == cudaSuccess;
  };
  bool ok = alloc((void**)&h->phi, sizeof(double) * n_sims) &&
            alloc((void**)&h->cnt, sizeof(int32_t) * kNCounters * n_sims) &&
            alloc((void**)&h->part, sizeof(Partial) * kMaxStatBlocks) &&
            alloc((void**)&h->dstats, sizeof(DevStats));
  if (ok && h->c.kind == MC_CTRL_NMPC && n_sims > 0) {
    h->ws_ld = nmpc_threads_for(n_sims, h->c.nx_model);
    // the one-state path adds the persistent schedule's plant noise rows
    const size_t main_words =
        (size_t)(h->c.nx_model == 3 ? (int)kNArr3 : (int)kNArr) * (h->c.N + 1) * (size_t)h->ws_ld;
    const size_t words =
        main_words + (h->c.nx_model == 3 ? 0 : (size_t)3 * h->m.n_em * (size_t)h->ws_ld);
    ok = alloc((void**)&h->ws, words * sizeof(double)) &&
         alloc((void**)&h->next, sizeof(unsigned long long)) &&
         alloc((void**)&h->wtrace, sizeof(unsigned long long) * kWarpTraceWords *
                                       (size_t)((h->ws_ld + kNmpcThreads - 1) / kNmpcThreads));
    if (ok) h->nz = h->ws + main_words;
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess)
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t pt = h->ws_ld;
    if (ctrl->threads_per_sm > 0) {
      const int64_t want = ((int64_t)ctrl->threads_per_sm * sms + 31) / 32 * 32;
      pt = want < pt ? want : pt;
    }
    h->persist_threads = pt;
    if (ok && (h->c.N_min > 0 || h->c.it_min > 0)) {
      // queue order: longest horizon (then highest iteration limit) first, so
      // the warps take trajectories of equal horizon and the long ones start
      // early; a counting sort on the host, once per handle
      std::vector<uint32_t> ord((size_t)n_sims);
      std::vector<int64_t> bucket((size_t)(MC_MAX_HORIZON + 1) * 128 + 1, 0);
      std::vector<int> key((size_t)n_sims);
      for (int64_t j = 0; j < n_sims; ++j) {
        int Nj, itj;
        traj_horizon(h->c, h->m.key0, h->m.key1, (uint32_t)j, Nj, itj);
        const int itk = itj < 127 ? itj : 127;
        key[(size_t)j] = (MC_MAX_HORIZON - Nj) * 128 + (127 - itk);
        bucket[(size_t)key[(size_t)j] + 1]++;
      }
      for (size_t b = 1; b < bucket.size(); ++b) bucket[b] += bucket[b - 1];
      for (int64_t j = 0; j < n_sims; ++j)
        ord[(size_t)bucket[(size_t)key[(size_t)j]]++] = (uint32_t)j;
      ok = alloc((void**)&h->order, sizeof(uint32_t) * n_sims) &&
           cudaMemcpy(h->order, ord.data(), sizeof(uint32_t) * n_sims,
                      cudaMemcpyHostToDevice) == cudaSuccess;
    }
  }
  if (!ok) {
    cudaGetLastError();
    mc_destroy(h);
    return fail(nullptr, MC_ENOMEM, "cudaMalloc failed for the trajectory buffers");
  }
  if (cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess) {
    mc_destroy(h);
    return fail(nullptr, MC_ECUDA, "cudaEventCreate failed");
  }
  *out = h;
  return MC_OK;
}

mc_status mc_set_histogram(mc_handle* h, int32_t n_bins, double lo, double hi) {
  if (!h) return MC_EINVAL;
  if (n_bins < 1 || n_bins > MC_MAX_BINS) return fail(h, MC_EINVAL, "n_bins must be 1..256");
  h->n_bins = n_bins;
  h->bin_lo = lo;
  h->bin_hi = hi;
  drop_graphs(h);  // the bins are baked into captured runs
  return MC_OK;
}

static mc_status launch_stats(mc_handle* h, int64_t j0, int64_t j1, cudaStream_t st) {
  const int64_t n = j1 - j0;
  int nb = (int)((n + kStatThreads - 1) / kStatThreads);
  nb = nb < 1 ? 1 : (nb > kMaxStatBlocks ? kMaxStatBlocks : nb);
  k_stats_partial<<<nb, kStatThreads, 0, st>>>(h->phi, h->cnt, j0, j1, h->part);
  k_stats_final<<<1, kStatThreads, 0, st>>>(h->part, nb, h->phi, j0, j1, h->n_bins, h->bin_lo,
                                            h->bin_hi, h->dstats);
  MC_CUDA(h, cudaGetLastError());
  return MC_OK;
}

}  // extern "C"

// The launches of one run of trajectories j0 .. j1-1 (closed loops and
// reductions), enqueued on st; the NMPC model may be a shortened copy (probe
// runs of the autotuner).
static mc_status enqueue_run(mc_handle* h, const DevModel& m, int64_t j0, int64_t j1,
                             int64_t persist_threads, cudaStream_t st) {
  if (j1 > j0) {
    if (h->c.kind == MC_CTRL_NMPC && h->schedule == MC_SCHED_PERSISTENT) {
      const int64_t n = j1 - j0;
      int64_t threads = n < persist_threads ? n : persist_threads;
      threads = (threads + kNmpcThreads - 1) / kNmpcThreads * kNmpcThreads;
      if (threads > h->ws_ld) threads = h->ws_ld;
      const uint32_t* order = (j0 == 0 && j1 == h->n_sims) ? h->order : nullptr;
      MC_CUDA(h, cudaMemsetAsync(h->next, 0, sizeof(unsigned long long), st));
      const unsigned blocks = (unsigned)(threads / kNmpcThreads);
      if (h->c.nx_model == 3)
        k_nmpc3_persist<<<blocks, kNmpcThreads, 0, st>>>(m, h->c, j0, n, order, h->next, h->phi,
                                                         h->cnt, h->ws, h->ws_ld);
      else if (h->c.precision == MC_FP64)
        k_nmpc_persist<double><<<blocks, kNmpcThreads, 0, st>>>(
            m, h->c, j0, n, order, h->next, h->phi, h->cnt, h->ws, h->ws_ld, h->nz, h->wtrace);
      else
        k_nmpc_persist<float><<<blocks, kNmpcThreads, 0, st>>>(
            m, h->c, j0, n, order, h->next, h->phi, h->cnt, h->ws, h->ws_ld, h->nz, h->wtrace);
      if (h->c.nx_model != 3) h->wtrace_warps = blocks;
    } else if (h->c.kind == MC_CTRL_NMPC) {
      const int64_t n = j1 - j0;
      int64_t threads = n < h->ws_ld ? n : h->ws_ld;
      const int64_t blocks = (threads + kNmpcThreads - 1) / kNmpcThreads;
      // the scratch stride is the allocation's, the thread count the range's
      if (h->c.nx_model == 3)
        k_nmpc3<<<(unsigned)blocks, kNmpcThreads, 0, st>>>(m, h->c, j0, j1, h->phi, h->cnt,
                                                           h->ws, h->ws_ld);
      else if (h->c.precision == MC_FP64)
        k_nmpc<double><<<(unsigned)blocks, kNmpcThreads, 0, st>>>(m, h->c, j0, j1, h->phi,
                                                                  h->cnt, h->ws, h->ws_ld);
      else
        k_nmpc<float><<<(unsigned)blocks, kNmpcThreads, 0, st>>>(m, h->c, j0, j1, h->phi,
                                                                 h->cnt, h->ws, h->ws_ld);
    } else {
      const int64_t blocks = (j1 - j0 + 127) / 128;
      if (h->c.precision == MC_FP64)
        k_pi<double><<<(unsigned)blocks, 128, 0, st>>>(m, h->c, j0, j1, h->phi, h->cnt);
      else
        k_pi<float><<<(unsigned)blocks, 128, 0, st>>>(m, h->c, j0, j1, h->phi, h->cnt);
    }
    MC_CUDA(h, cudaGetLastError());
  }
  return launch_stats(h, j0, j1, st);
}

static void drop_graphs(mc_handle* h) {
  for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
  h->graphs.clear();
}

// ---------------------------------------------------------------- SM partitions
// Green contexts (driver API) restrict a stream's kernels to a subset of the
// SMs.  The driver entry points are looked up through the runtime, so the
// library does not link against libcuda.

namespace {
struct GreenApi {
  CUresult (*dev_get)(CUdevice*, int) = nullptr;
  CUresult (*dev_resource)(CUdevice, CUdevResource*, CUdevResourceType) = nullptr;
  CUresult (*split)(CUdevResource*, unsigned int*, const CUdevResource*, CUdevResource*,
                    unsigned int, unsigned int) = nullptr;
  CUresult (*gen_desc)(CUdevResourceDesc*, CUdevResource*, unsigned int) = nullptr;
  CUresult (*create)(CUgreenCtx*, CUdevResourceDesc, CUdevice, unsigned int) = nullptr;
  CUresult (*destroy)(CUgreenCtx) = nullptr;
  CUresult (*stream_create)(CUstream*, CUgreenCtx, unsigned int, int) = nullptr;
  CUresult (*stream_destroy)(CUstream) = nullptr;
  bool ok = false;
};

const GreenApi& green_api() {
  static const GreenApi api = [] {
    GreenApi a;
    auto get = [](const char* name, void** fn) {
      cudaDriverEntryPointQueryResult q;
      return cudaGetDriverEntryPointByVersion(name, fn, 13000, cudaEnableDefault, &q) ==
                 cudaSuccess &&
             q == cudaDriverEntryPointSuccess && *fn != nullptr;
    };
    a.ok = get("cuDeviceGet", (void**)&a.dev_get) &&
           get("cuDeviceGetDevResource", (void**)&a.dev_resource) &&
           get("cuDevSmResourceSplitByCount", (void**)&a.split) &&
           get("cuDevResourceGenerateDesc", (void**)&a.gen_desc) &&
           get("cuGreenCtxCreate", (void**)&a.create) &&
           get("cuGreenCtxDestroy", (void**)&a.destroy) &&
           get("cuGreenCtxStreamCreate", (void**)&a.stream_create) &&
           get("cuStreamDestroy", (void**)&a.stream_destroy);
    cudaGetLastError();
    return a;
  }();
  return api;
}
}  // namespace

static void drop_partition(mc_handle* h) {
  const GreenApi& g = green_api();
  if (h->pstream && g.stream_destroy) g.stream_destroy(h->pstream);
  if (h->gctx && g.destroy) g.destroy(h->gctx);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  h->pstream = nullptr;
  h->gctx = nullptr;
  h->ev_fork = h->ev_join = nullptr;
  h->part_sms = 0;
}

// The stream the handle's kernels go to: the caller's, or the partition's
// stream made to wait for the caller's work so far.
static cudaStream_t fork_stream(mc_handle* h, cudaStream_t st) {
  if (!h->pstream) return st;
  cudaEventRecord(h->ev_fork, st);
  cudaStreamWaitEvent((cudaStream_t)h->pstream, h->ev_fork, 0);
  return (cudaStream_t)h->pstream;
}

// The caller's stream waits for what was launched on ls.
static void join_stream(mc_handle* h, cudaStream_t st, cudaStream_t ls) {
  if (ls == st) return;
  cudaEventRecord(h->ev_join, ls);
  cudaStreamWaitEvent(st, h->ev_join, 0);
}

extern "C" {

mc_status mc_set_sm_partition(mc_handle* h, int32_t n_sms, int32_t* n_sms_out) {
  if (!h) return MC_EINVAL;
  if (n_sms < 0) return fail(h, MC_EINVAL, "n_sms must be >= 0");
  MC_CUDA(h, cudaDeviceSynchronize());
  drop_partition(h);
  drop_graphs(h);
  int dev = 0, sms = 0;
  MC_CUDA(h, cudaGetDevice(&dev));
  MC_CUDA(h, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (n_sms == 0 || n_sms >= sms) {
    if (n_sms_out) *n_sms_out = sms;
    return MC_OK;
  }
  const GreenApi& g = green_api();
  if (!g.ok) return fail(h, MC_ECUDA, "the driver offers no green contexts (SM partitions)");
  auto drv = [&](CUresult r, const char* what) -> mc_status {
    if (r == CUDA_SUCCESS) return MC_OK;
    drop_partition(h);
    return fail(h, MC_ECUDA, std::string(what) + " failed (CUresult " + std::to_string((int)r) +
                                 ")");
  };
  CUdevice cdev;
  mc_status s = drv(g.dev_get(&cdev, dev), "cuDeviceGet");
  if (s != MC_OK) return s;
  CUdevResource all, part, rest;
  memset(&all, 0, sizeof(all));
  memset(&part, 0, sizeof(part));
  memset(&rest, 0, sizeof(rest));
  if ((s = drv(g.dev_resource(cdev, &all, CU_DEV_RESOURCE_TYPE_SM), "cuDeviceGetDevResource")) !=
      MC_OK)
    return s;
  unsigned int groups = 1;
  if ((s = drv(g.split(&part, &groups, &all, &rest, 0, (unsigned)n_sms),
               "cuDevSmResourceSplitByCount")) != MC_OK)
    return s;
  if (groups < 1) return fail(h, MC_EINVAL, "no SM partition of that size");
  CUdevResourceDesc desc;
  if ((s = drv(g.gen_desc(&desc, &part, 1), "cuDevResourceGenerateDesc")) != MC_OK) return s;
  if ((s = drv(g.create(&h->gctx, desc, cdev, CU_GREEN_CTX_DEFAULT_STREAM), "cuGreenCtxCreate")) !=
      MC_OK)
    return s;
  if ((s = drv(g.stream_create(&h->pstream, h->gctx, CU_STREAM_NON_BLOCKING, 0),
               "cuGreenCtxStreamCreate")) != MC_OK)
    return s;
  if (cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    drop_partition(h);
    return fail(h, MC_ECUDA, "cudaEventCreate failed");
  }
  h->part_sms = (int)part.sm.smCount;
  if (n_sms_out) *n_sms_out = h->part_sms;
  return MC_OK;
}

mc_status mc_run_range(mc_handle* h, int64_t j0, int64_t j1, void* cuda_stream) {
  if (!h) return MC_EINVAL;
  if (j0 < 0 || j1 < j0 || j1 > h->n_sims) return fail(h, MC_EINVAL, "bad trajectory range");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  MC_CUDA(h, cudaEventRecord(h->ev0, st));
  if (h->use_graph && st != nullptr && !h->pstream) {
    // replay the captured launches of this range, capturing them on first use
    cudaGraphExec_t exec = nullptr;
    for (const auto& g : h->graphs)
      if (g.j0 == j0 && g.j1 == j1) exec = g.exec;
    if (!exec) {
      MC_CUDA(h, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      const mc_status s = enqueue_run(h, h->m, j0, j1, h->persist_threads, st);
      cudaGraph_t graph = nullptr;
      const cudaError_t e = cudaStreamEndCapture(st, &graph);
      if (s != MC_OK) {
        if (graph) cudaGraphDestroy(graph);
        return s;
      }
      if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
      const cudaError_t e2 = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e2 != cudaSuccess) return cuda_fail(h, e2, "cudaGraphInstantiate");
      h->graphs.push_back({j0, j1, exec});
    }
    MC_CUDA(h, cudaGraphLaunch(exec, st));
  } else {
    const cudaStream_t ls = fork_stream(h, st);
    const mc_status s = enqueue_run(h, h->m, j0, j1, h->persist_threads, ls);
    join_stream(h, st, ls);
    if (s != MC_OK) return s;
  }
  MC_CUDA(h, cudaEventRecord(h->ev1, st));
  h->ran = true;
  h->last_j0 = j0;
  h->last_j1 = j1;
  return MC_OK;
}

mc_status mc_set_graph(mc_handle* h, int on) {
  if (!h) return MC_EINVAL;
  h->use_graph = on != 0;
  if (!h->use_graph) drop_graphs(h);
  return MC_OK;
}

mc_status mc_autotune(mc_handle* h, int32_t probe_steps, void* cuda_stream,
                      int32_t* threads_per_sm) {
  if (!h) return MC_EINVAL;
  if (h->c.kind != MC_CTRL_NMPC || h->schedule != MC_SCHED_PERSISTENT)
    return fail(h, MC_EINVAL, "mc_autotune tunes the persistent NMPC schedule only");
  if (probe_steps < 1) return fail(h, MC_EINVAL, "probe_steps must be >= 1");
  if (h->n_sims == 0) return MC_OK;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 152;
  MC_CUDA(h, cudaGetDevice(&dev));
  MC_CUDA(h, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (h->part_sms > 0) sms = h->part_sms;
  DevModel probe = h->m;
  probe.n_steps = probe_steps < h->m.n_steps ? probe_steps : h->m.n_steps;
  static const int cand[] = {32, 64, 96, 128, 160, 192, 256, 384, 512};
  float best_ms = 0.f;
  int best = 0;
  int64_t best_threads = h->persist_threads;
  cudaEvent_t a, b;
  MC_CUDA(h, cudaEventCreate(&a));
  MC_CUDA(h, cudaEventCreate(&b));
  for (int ci = 0; ci <= (int)(sizeof(cand) / sizeof(cand[0])); ++ci) {
    // the candidates, then one thread per trajectory up to the capacity
    const bool last = ci == (int)(sizeof(cand) / sizeof(cand[0]));
    const int tps = last ? (int)((h->ws_ld + sms - 1) / sms) : cand[ci];
    const int64_t threads = (int64_t)tps * sms;
    if (!last && threads >= h->ws_ld) continue;
    const int64_t pt = threads < h->ws_ld ? threads : h->ws_ld;
    MC_CUDA(h, cudaEventRecord(a, st));
    const cudaStream_t ls = fork_stream(h, st);
    mc_status s = enqueue_run(h, probe, 0, h->n_sims, pt, ls);
    join_stream(h, st, ls);
    if (s != MC_OK) return s;
    MC_CUDA(h, cudaEventRecord(b, st));
    MC_CUDA(h, cudaEventSynchronize(b));
    float ms = 0.f;
    MC_CUDA(h, cudaEventElapsedTime(&ms, a, b));
    if (best == 0 || ms < best_ms) {
      best_ms = ms;
      best = tps;
      best_threads = pt;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  h->persist_threads = best_threads;
  drop_graphs(h);
  if (threads_per_sm) *threads_per_sm = best;
  return MC_OK;
}

mc_status mc_run(mc_handle* h, void* cuda_stream) {
  if (!h) return MC_EINVAL;
  return mc_run_range(h, 0, h->n_sims, cuda_stream);
}

mc_status mc_sync(mc_handle* h, int64_t timeout_ms) {
  if (!h) return MC_EINVAL;
  if (!h->ran) return fail(h, MC_ENOTRUN, "mc_run has not been called");
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t e = cudaEventQuery(h->ev1);
    if (e == cudaSuccess) return MC_OK;
    if (e != cudaErrorNotReady) return cuda_fail(h, e, "waiting for the run");
    if (timeout_ms > 0) {
      const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(
                          std::chrono::steady_clock::now() - t0).count();
      if (ms > timeout_ms) return fail(h, MC_ETIMEOUT, "the run did not finish in time");
    }
    std::this_thread::sleep_for(std::chrono::microseconds(200));
  }
}

mc_status mc_stats(mc_handle* h, mc_stats_t* out, int64_t timeout_ms) {
  if (!h || !out) return MC_EINVAL;
  mc_status s = mc_sync(h, timeout_ms);
  if (s != MC_OK) return s;
  DevStats d;
  MC_CUDA(h, cudaMemcpy(&d, h->dstats, sizeof(d), cudaMemcpyDeviceToHost));
  memset(out, 0, sizeof(*out));
  const int64_t n = h->last_j1 - h->last_j0;
  out->n_traj = n;
  out->n_ocp = (h->c.kind == MC_CTRL_NMPC) ? n * (int64_t)h->m.n_steps : 0;
  out->n_ocp_failed = d.sums[0];
  out->sqp_iters = d.sums[1];
  out->ls_trials = d.sums[2];
  out->n_hess_reset = d.sums[3];
  out->n_ls_fail = d.sums[4];
  out->qp_iters = d.sums[5];
  out->n_nonfinite = d.n_nonfinite;
  out->qp_fail = d.sums[7];
  out->phi_mean = d.mean;
  out->phi_var = (d.n > 1) ? d.m2 / (d.n - 1.0) : 0.0;
  out->phi_min = d.mn;
  out->phi_max = d.mx;
  out->n_bins = h->n_bins;
  out->bin_lo = d.lo;
  out->bin_hi = d.hi;
  for (int b = 0; b < MC_MAX_BINS; ++b) out->hist[b] = d.hist[b];
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, h->ev0, h->ev1) == cudaSuccess) out->gpu_ms = ms;
  return d.n_nonfinite > 0 ? MC_WARN_NONFINITE : MC_OK;
}

mc_status mc_copy_phi(mc_handle* h, int64_t j0, int64_t n, double* dst, int dst_is_device) {
  if (!h || (!dst && n > 0)) return MC_EINVAL;
  if (j0 < 0 || n < 0 || j0 + n > h->n_sims) return fail(h, MC_EINVAL, "bad range");
  if (n == 0) return MC_OK;
  mc_status s = mc_sync(h, 0);
  if (s != MC_OK) return s;
  MC_CUDA(h, cudaMemcpy(dst, h->phi + j0, sizeof(double) * n,
                        dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost));
  return MC_OK;
}

mc_status mc_copy_counters(mc_handle* h, int64_t j0, int64_t n, int32_t* dst,
                           int dst_is_device) {
  if (!h || (!dst && n > 0)) return MC_EINVAL;
  if (j0 < 0 || n < 0 || j0 + n > h->n_sims) return fail(h, MC_EINVAL, "bad range");
  if (n == 0) return MC_OK;
  mc_status s = mc_sync(h, 0);
  if (s != MC_OK) return s;
  MC_CUDA(h, cudaMemcpy(dst, h->cnt + j0 * kNCounters, sizeof(int32_t) * kNCounters * n,
                        dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost));
  return MC_OK;
}

mc_status mc_copy_warp_trace(mc_handle* h, uint64_t* out_host, int64_t max_warps,
                             int64_t* n_warps_out) {
  if (!h || !n_warps_out || max_warps < 0 || (max_warps > 0 && !out_host)) return MC_EINVAL;
  *n_warps_out = 0;
  if (h->wtrace_warps == 0)
    return fail(h, MC_ENOTRUN, "no one-state persistent NMPC launch has run on this handle");
  mc_status s = mc_sync(h, 0);
  if (s != MC_OK) return s;
  const int64_t n = h->wtrace_warps < max_warps ? h->wtrace_warps : max_warps;
  if (n > 0)
    MC_CUDA(h, cudaMemcpy(out_host, h->wtrace, sizeof(uint64_t) * kWarpTraceWords * n,
                          cudaMemcpyDeviceToHost));
  *n_warps_out = h->wtrace_warps;
  return MC_OK;
}

// ------------------------------------------------ gradients of the PI study

mc_status mc_set_pi_gains(mc_handle* h, double kP, double kI, double kaw) {
  if (!h) return MC_EINVAL;
  if (h->c.kind != MC_CTRL_PI) return fail(h, MC_EINVAL, "mc_set_pi_gains needs a PI handle");
  if (!std::isfinite(kP) || !std::isfinite(kI) || !std::isfinite(kaw))
    return fail(h, MC_EINVAL, "the gains must be finite");
  h->c.kP = kP;
  h->c.kI = kI;
  h->c.kaw = kaw;
  drop_graphs(h);  // captured launches hold the old gains
  return MC_OK;
}

mc_status mc_pi_grad(mc_handle* h, int64_t j0, int64_t j1, int32_t checkpoint_every,
                     void* cuda_stream) {
  if (!h) return MC_EINVAL;
  if (h->c.kind != MC_CTRL_PI) return fail(h, MC_EINVAL, "mc_pi_grad needs a PI handle");
  if (h->c.precision != MC_FP64) return fail(h, MC_EINVAL, "mc_pi_grad runs in FP64 only");
  if (j0 < 0 || j1 < j0 || j1 > h->n_sims) return fail(h, MC_EINVAL, "bad trajectory range");
  if (checkpoint_every < 1 || checkpoint_every > kGradMaxSeg)
    return fail(h, MC_EINVAL, "checkpoint_every must be 1..32");
  if (h->m.n_em > kGradMaxEm) return fail(h, MC_EINVAL, "the gradient supports n_em <= 32");
  const int K = h->m.n_steps;
  const int n_ck = K > 0 ? (K + checkpoint_every - 1) / checkpoint_every : 1;
  const int64_t words = (int64_t)4 * n_ck * (h->n_sims > 0 ? h->n_sims : 1);
  if (!h->dphi) {
    if (cudaMalloc((void**)&h->dphi, sizeof(double) * 3 * (h->n_sims > 0 ? h->n_sims : 1)) !=
            cudaSuccess ||
        cudaMalloc((void**)&h->gmean, sizeof(double) * 4) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, MC_ENOMEM, "cudaMalloc failed for the gradient buffers");
    }
  }
  if (words > h->ck_words) {
    cudaFree(h->ck);
    h->ck = nullptr;
    h->ck_words = 0;
    if (cudaMalloc((void**)&h->ck, sizeof(double) * words) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, MC_ENOMEM, "cudaMalloc failed for the checkpoints");
    }
    h->ck_words = words;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  MC_CUDA(h, cudaEventRecord(h->ev0, st));
  const cudaStream_t ls = fork_stream(h, st);
  if (j1 > j0) {
    const int64_t blocks = (j1 - j0 + 127) / 128;
    k_pi_grad<<<(unsigned)blocks, 128, 0, ls>>>(h->m, h->c, j0, j1, checkpoint_every, n_ck, h->ck,
                                                h->n_sims, h->phi, h->cnt, h->dphi);
  }
  k_grad_mean<<<1, kGradThreads, 0, ls>>>(h->phi, h->dphi, j0, j1, h->gmean);
  const mc_status s = launch_stats(h, j0, j1, ls);
  join_stream(h, st, ls);
  MC_CUDA(h, cudaGetLastError());
  if (s != MC_OK) return s;
  MC_CUDA(h, cudaEventRecord(h->ev1, st));
  h->ran = true;
  h->grad_ran = true;
  h->last_j0 = j0;
  h->last_j1 = j1;
  return MC_OK;
}

mc_status mc_set_nmpc_weights(mc_handle* h, double Qz, double Ru, double Qn) {
  if (!h) return MC_EINVAL;
  if (h->c.kind != MC_CTRL_NMPC) return fail(h, MC_EINVAL, "mc_set_nmpc_weights needs an NMPC handle");
  if (!(Qz >= 0.0) || !(Ru >= 0.0) || !(Qn >= 0.0) || !std::isfinite(Qz) || !std::isfinite(Ru) ||
      !std::isfinite(Qn))
    return fail(h, MC_EINVAL, "the weights must be finite and >= 0");
  if (h->c.nx_model == 3 && (Ru != 0.0 || Qn != 0.0))
    return fail(h, MC_EINVAL, "the three-state NMPC has the paper's objective only (Ru = Qn = 0)");
  h->c.Qz = Qz;
  h->c.Ru = Ru;
  h->c.Qn = Qn;
  h->c.r_scale = 2.0 * Ru * h->m.Ts;
  drop_graphs(h);  // captured launches hold the old weights
  return MC_OK;
}

mc_status mc_set_grad_record_budget(mc_handle* h, int64_t bytes) {
  if (!h) return MC_EINVAL;
  if (h->c.kind != MC_CTRL_NMPC)
    return fail(h, MC_EINVAL, "mc_set_grad_record_budget needs an NMPC handle");
  const size_t per_traj =
      sizeof(double) * (size_t)(5 * (h->c.N + 1) + 8) * (size_t)(h->m.n_steps + 1);
  if (bytes < 0 || (bytes > 0 && (size_t)bytes < per_traj))
    return fail(h, MC_EINVAL, "the record budget must be 0 or hold one trajectory's records");
  h->rec_budget = bytes == 0 ? kRecordBudget : (size_t)bytes;
  return MC_OK;
}

mc_status mc_nmpc_grad(mc_handle* h, int64_t j0, int64_t j1, void* cuda_stream) {
  if (!h) return MC_EINVAL;
  if (h->c.kind != MC_CTRL_NMPC) return fail(h, MC_EINVAL, "mc_nmpc_grad needs an NMPC handle");
  if (h->c.precision != MC_FP64 || h->c.nx_model == 3)
    return fail(h, MC_EINVAL, "mc_nmpc_grad runs the one-state NMPC in FP64");
  if (j0 < 0 || j1 < j0 || j1 > h->n_sims) return fail(h, MC_EINVAL, "bad trajectory range");
  if (!h->dphi) {
    if (cudaMalloc((void**)&h->dphi, sizeof(double) * 3 * (h->n_sims > 0 ? h->n_sims : 1)) !=
            cudaSuccess ||
        cudaMalloc((void**)&h->gmean, sizeof(double) * 4) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, MC_ENOMEM, "cudaMalloc failed for the gradient buffers");
    }
  }
  if (!h->tg && h->ws_ld > 0) {
    if (cudaMalloc((void**)&h->tg, sizeof(double) * kTgRows * (size_t)h->ws_ld) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, MC_ENOMEM, "cudaMalloc failed for the gradient buffers");
    }
  }
  const int N1 = h->c.N + 1, RW = 5 * N1 + 8;
  const size_t per_traj = sizeof(double) * (size_t)RW * (size_t)(h->m.n_steps + 1);
  int64_t cn = (int64_t)(h->rec_budget / per_traj);
  if (h->schedule == MC_SCHED_PERSISTENT && j1 > j0) {
    // records of chunks of at most cn trajectories, allocated once per handle
    cn = cn < 1 ? 1 : (cn > j1 - j0 ? j1 - j0 : cn);
    if (h->rec_bytes < per_traj * (size_t)cn) {
      cudaFree(h->rec);
      h->rec = nullptr;
      h->rec_bytes = 0;
      if (cudaMalloc((void**)&h->rec, per_traj * (size_t)cn) != cudaSuccess) {
        cudaGetLastError();
        return fail(h, MC_ENOMEM, "cudaMalloc failed for the gradient's sample records");
      }
      h->rec_bytes = per_traj * (size_t)cn;
    }
    if (!h->kj && cudaMalloc((void**)&h->kj, sizeof(int32_t) * (size_t)h->n_sims) !=
                      cudaSuccess) {
      cudaGetLastError();
      return fail(h, MC_ENOMEM, "cudaMalloc failed for the gradient's sample records");
    }
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  MC_CUDA(h, cudaEventRecord(h->ev0, st));
  const cudaStream_t ls = fork_stream(h, st);
  if (j1 > j0 && h->schedule == MC_SCHED_PERSISTENT) {
    // each chunk: the recording closed loop (launched as enqueue_run launches
    // k_nmpc_persist), then the tangent pass over its records
    for (int64_t a = j0; a < j1; a += cn) {
      const int64_t b = (j1 - a < cn) ? j1 : a + cn, nc = b - a;
      const Recorder rc{h->rec, nc, a, RW, h->kj + a};
      int64_t threads = nc < h->persist_threads ? nc : h->persist_threads;
      threads = (threads + kNmpcThreads - 1) / kNmpcThreads * kNmpcThreads;
      if (threads > h->ws_ld) threads = h->ws_ld;
      const uint32_t* order = (a == 0 && b == h->n_sims) ? h->order : nullptr;
      MC_CUDA(h, cudaMemsetAsync(h->next, 0, sizeof(unsigned long long), ls));
      k_nmpc_persist_rec<<<(unsigned)(threads / kNmpcThreads), kNmpcThreads, 0, ls>>>(
          h->m, h->c, nc, order, h->next, h->phi, h->cnt, h->ws, h->ws_ld, h->nz, h->wtrace, rc);
      h->wtrace_warps = threads / kNmpcThreads;
      const int64_t tt = nc < h->ws_ld ? nc : h->ws_ld;
      k_nmpc_tangent<<<(unsigned)((tt + kTangentThreads - 1) / kTangentThreads),
                       kTangentThreads, 0, ls>>>(h->m, h->c, nc, h->phi, h->cnt, h->dphi, h->ws,
                                                 tt, h->tg, rc);
    }
  } else if (j1 > j0) {
    const int64_t n = j1 - j0;
    const int64_t threads = n < h->ws_ld ? n : h->ws_ld;
    const int64_t blocks = (threads + kNmpcThreads - 1) / kNmpcThreads;
    k_nmpc_grad<<<(unsigned)blocks, kNmpcThreads, 0, ls>>>(h->m, h->c, j0, j1, h->phi, h->cnt,
                                                           h->dphi, h->ws, h->ws_ld, h->tg);
  }
  k_grad_mean<<<1, kGradThreads, 0, ls>>>(h->phi, h->dphi, j0, j1, h->gmean);
  const mc_status s = launch_stats(h, j0, j1, ls);
  join_stream(h, st, ls);
  MC_CUDA(h, cudaGetLastError());
  if (s != MC_OK) return s;
  MC_CUDA(h, cudaEventRecord(h->ev1, st));
  h->ran = true;
  h->grad_ran = true;
  h->last_j0 = j0;
  h->last_j1 = j1;
  return MC_OK;
}

mc_status mc_grad_mean(mc_handle* h, double out[3], int64_t timeout_ms) {
  if (!h || !out) return MC_EINVAL;
  if (!h->grad_ran) return fail(h, MC_ENOTRUN, "mc_pi_grad has not been called");
  mc_status s = mc_sync(h, timeout_ms);
  if (s != MC_OK) return s;
  double g[4];
  MC_CUDA(h, cudaMemcpy(g, h->gmean, sizeof(g), cudaMemcpyDeviceToHost));
  out[0] = g[0];
  out[1] = g[1];
  out[2] = g[2];
  return (g[3] < (double)(h->last_j1 - h->last_j0)) ? MC_WARN_NONFINITE : MC_OK;
}

mc_status mc_copy_grad(mc_handle* h, int64_t j0, int64_t n, double* dst, int dst_is_device) {
  if (!h || (!dst && n > 0)) return MC_EINVAL;
  if (!h->grad_ran) return fail(h, MC_ENOTRUN, "mc_pi_grad has not been called");
  if (j0 < 0 || n < 0 || j0 + n > h->n_sims) return fail(h, MC_EINVAL, "bad range");
  if (n == 0) return MC_OK;
  mc_status s = mc_sync(h, 0);
  if (s != MC_OK) return s;
  MC_CUDA(h, cudaMemcpy(dst, h->dphi + 3 * j0, sizeof(double) * 3 * n,
                        dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost));
  return MC_OK;
}

// ----------------------------------------------------------- building blocks

mc_status mc_philox(const uint32_t* ctr_host, const uint32_t key[2], int64_t n,
                    uint32_t* out_host) {
  if (n < 0 || (n > 0 && (!ctr_host || !out_host || !key)))
    return fail(nullptr, MC_EINVAL, "mc_philox: bad arguments");
  if (n == 0) return MC_OK;
  uint4 *dc = nullptr, *dout = nullptr;
  mc_status s = MC_OK;
  if (!to_dev(&dc, (const uint4*)ctr_host, n) || !to_dev<uint4>(&dout, nullptr, n)) {
    s = fail(nullptr, MC_ENOMEM, "mc_philox: allocation");
  } else {
    k_philox<<<(unsigned)((n + 255) / 256), 256>>>(dc, key[0], key[1], n, dout);
    cudaError_t e = cudaMemcpy(out_host, dout, sizeof(uint4) * n, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) s = cuda_fail(nullptr, e, "mc_philox");
  }
  cudaFree(dc);
  cudaFree(dout);
  return s;
}

mc_status mc_noise(uint64_t seed, int64_t j, int64_t k0, int64_t nk, int32_t precision,
                   double* out_host, double* meas_host) {
  if (nk < 0 || j < 0 || k0 < 0 || (nk > 0 && (!out_host || !meas_host)))
    return fail(nullptr, MC_EINVAL, "mc_noise: bad arguments");
  if (nk == 0) return MC_OK;
  DevModel m;
  memset(&m, 0, sizeof(m));
  m.key0 = (uint32_t)seed;
  m.key1 = (uint32_t)(seed >> 32);
  double *d = nullptr, *dm = nullptr;
  mc_status s = MC_OK;
  if (!to_dev<double>(&d, nullptr, 3 * nk) || !to_dev<double>(&dm, nullptr, nk)) {
    s = fail(nullptr, MC_ENOMEM, "mc_noise: allocation");
  } else {
    k_noise<<<(unsigned)((nk + 127) / 128), 128>>>(m, (uint32_t)j, k0, nk, precision, d, dm);
    cudaError_t e = cudaMemcpy(out_host, d, sizeof(double) * 3 * nk, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(meas_host, dm, sizeof(double) * nk, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) s = cuda_fail(nullptr, e, "mc_noise");
  }
  cudaFree(d);
  cudaFree(dm);
  return s;
}

static mc_status elementary_batch(const char* name, bool rcp, const double* x_host, int64_t n,
                                  double* out_host) {
  if (n < 0 || (n > 0 && (!x_host || !out_host)))
    return fail(nullptr, MC_EINVAL, std::string(name) + ": bad arguments");
  if (n == 0) return MC_OK;
  double *dx = nullptr, *dy = nullptr;
  mc_status s = MC_OK;
  if (!to_dev<double>(&dx, x_host, n) || !to_dev<double>(&dy, nullptr, n)) {
    s = fail(nullptr, MC_ENOMEM, std::string(name) + ": allocation");
  } else {
    const unsigned grid = (unsigned)((n + 255) / 256);
    if (rcp) k_elementary<true><<<grid, 256>>>(dx, n, dy);
    else k_elementary<false><<<grid, 256>>>(dx, n, dy);
    const cudaError_t e = cudaMemcpy(out_host, dy, sizeof(double) * n, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) s = cuda_fail(nullptr, e, name);
  }
  cudaFree(dx);
  cudaFree(dy);
  return s;
}

mc_status mc_exp_batch(const double* x_host, int64_t n, double* out_host) {
  return elementary_batch("mc_exp_batch", false, x_host, n, out_host);
}

mc_status mc_rcp_batch(const double* x_host, int64_t n, double* out_host) {
  return elementary_batch("mc_rcp_batch", true, x_host, n, out_host);
}

mc_status mc_pipe_probe(int32_t kind, int64_t iters, double* ms_out, double* steps_out) {
  if (kind < 0 || kind >= kNumProbes || iters < 1 || iters > ((int64_t)1 << 30) || !ms_out ||
      !steps_out)
    return fail(nullptr, MC_EINVAL, "mc_pipe_probe: bad arguments");
  int dev = 0, sms = 152;
  MC_CUDA(nullptr, cudaGetDevice(&dev));
  MC_CUDA(nullptr, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // 16 blocks of 4 warps per SM: enough warps per scheduler to keep any pipe busy
  const unsigned blocks = (unsigned)sms * 16u;
  const int64_t threads = (int64_t)blocks * 128;
  double* out = nullptr;
  if (cudaMalloc((void**)&out, sizeof(double) * threads) != cudaSuccess) {
    cudaGetLastError();
    return fail(nullptr, MC_ENOMEM, "mc_pipe_probe: allocation");
  }
  cudaEvent_t a = nullptr, b = nullptr;
  mc_status s = MC_OK;
  auto launch = [&](int64_t it) {
    switch (kind) {
      case kProbeDfma: k_pipe_probe<kProbeDfma><<<blocks, 128>>>(it, 1.0, out); break;
      case kProbeNone: k_pipe_probe<kProbeNone><<<blocks, 128>>>(it, 1.0, out); break;
      case kProbeExpTab: k_pipe_probe<kProbeExpTab><<<blocks, 128>>>(it, 1.0, out); break;
      case kProbeExpLib: k_pipe_probe<kProbeExpLib><<<blocks, 128>>>(it, 1.0, out); break;
      case kProbeDiv: k_pipe_probe<kProbeDiv><<<blocks, 128>>>(it, 1.0, out); break;
      case kProbeLog: k_pipe_probe<kProbeLog><<<blocks, 128>>>(it, 1.0, out); break;
      case kProbeSqrt: k_pipe_probe<kProbeSqrt><<<blocks, 128>>>(it, 1.0, out); break;
      case kProbeSincos: k_pipe_probe<kProbeSincos><<<blocks, 128>>>(it, 1.0, out); break;
      case kProbeFfma: k_pipe_probe<kProbeFfma><<<blocks, 128>>>(it, 1.0, out); break;
      case kProbeExpf: k_pipe_probe<kProbeExpf><<<blocks, 128>>>(it, 1.0, out); break;
      case kProbeRcp: k_pipe_probe<kProbeRcp><<<blocks, 128>>>(it, 1.0, out); break;
      default: k_pipe_probe<kProbeNoneF><<<blocks, 128>>>(it, 1.0, out); break;
    }
  };
  float ms = 0.f;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    s = fail(nullptr, MC_ECUDA, "mc_pipe_probe: cudaEventCreate failed");
  } else {
    launch(iters < 64 ? iters : 64);   // warm-up (clocks, instruction cache)
    cudaEventRecord(a, 0);
    launch(iters);
    cudaEventRecord(b, 0);
    const cudaError_t e = cudaEventSynchronize(b);
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess)
      s = cuda_fail(nullptr, e != cudaSuccess ? e : cudaErrorUnknown, "mc_pipe_probe");
    else
      cudaEventElapsedTime(&ms, a, b);
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFree(out);
  *ms_out = ms;
  *steps_out = (double)threads * (double)kChains * (double)iters;
  return s;
}

mc_status mc_qp_solve_batch(int32_t N, int64_t n, int32_t solver, int32_t max_it, double tol,
                            const double* A, const double* B, const double* b,
                            const double* Wxx, const double* Wxu, const double* Wuu,
                            const double* q, const double* r, const double* lb,
                            const double* ub, double* du, double* dx, double* mu, double* nul,
                            double* nuu, int32_t* iters, int32_t* status) {
  if (N < 1 || N > MC_MAX_HORIZON || n < 0 || max_it < 1)
    return fail(nullptr, MC_EINVAL, "mc_qp_solve_batch: bad sizes");
  if (solver != MC_QP_ACTIVE_SET && solver != MC_QP_IPM && solver != MC_QP_ACTIVE_SET_WARP)
    return fail(nullptr, MC_EINVAL, "mc_qp_solve_batch: unknown solver");
  if (n == 0) return MC_OK;
  const size_t n1 = (size_t)n * N, n2 = (size_t)n * (N + 1);
  QpBatch d{};
  std::vector<void*> owned;
  bool ok = true;
  auto up = [&](const double** dst, const double* src, size_t cnt) {
    double* p = nullptr;
    ok = ok && to_dev(&p, src, cnt);
    owned.push_back(p);
    *dst = p;
  };
  auto mk = [&](double** dst, size_t cnt) {
    double* p = nullptr;
    ok = ok && to_dev<double>(&p, nullptr, cnt);
    owned.push_back(p);
    *dst = p;
  };
  up(&d.A, A, n1); up(&d.B, B, n1); up(&d.b, b, n1); up(&d.r, r, n1);
  up(&d.lb, lb, n1); up(&d.ub, ub, n1);
  up(&d.Wxx, Wxx, n2); up(&d.Wxu, Wxu, n2); up(&d.Wuu, Wuu, n2); up(&d.q, q, n2);
  mk(&d.du, n1); mk(&d.mu, n1); mk(&d.nul, n1); mk(&d.nuu, n1); mk(&d.dx, n2);
  int32_t *di = nullptr, *ds = nullptr;
  ok = ok && to_dev<int32_t>(&di, nullptr, n) && to_dev<int32_t>(&ds, nullptr, n);
  owned.push_back(di);
  owned.push_back(ds);
  d.iters = di;
  d.status = ds;
  double* ws = nullptr;
  const int64_t ld = n;
  ok = ok && to_dev<double>(&ws, nullptr, (size_t)kNArr * (N + 1) * ld);
  owned.push_back(ws);
  mc_status s = MC_OK;
  if (!ok) {
    s = fail(nullptr, MC_ENOMEM, "mc_qp_solve_batch: allocation");
  } else {
    if (solver == MC_QP_ACTIVE_SET_WARP)
      k_qp_batch_warp<<<(unsigned)((n + kQpWarpsPerBlock - 1) / kQpWarpsPerBlock),
                        32 * kQpWarpsPerBlock>>>(N, n, max_it, d, ws, ld);
    else
      k_qp_batch<<<(unsigned)((n + 127) / 128), 128>>>(N, n, solver, max_it, tol, d, ws, ld);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(du, d.du, sizeof(double) * n1, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(mu, d.mu, sizeof(double) * n1, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(nul, d.nul, sizeof(double) * n1, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(nuu, d.nuu, sizeof(double) * n1, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(dx, d.dx, sizeof(double) * n2, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(iters, di, sizeof(int32_t) * n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(status, ds, sizeof(int32_t) * n, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) s = cuda_fail(nullptr, e, "mc_qp_solve_batch");
  }
  for (void* p : owned) cudaFree(p);
  return s;
}

mc_status mc_ocp_solve_batch(const mc_model_t* model, const mc_controller_t* ctrl, int64_t n,
                             const double* x0, const double* EaR, const double* zbar,
                             double* u, double* x, double* lam, double* pil, double* piu,
                             int32_t* info, double* kkt) {
  DevModel m;
  DevCtrl c;
  std::string why;
  if (fill_dev(model, ctrl, 0, &m, &c, &why) != MC_OK)
    return fail(nullptr, MC_EINVAL, "mc_ocp_solve_batch: " + why);
  if (c.kind != MC_CTRL_NMPC) return fail(nullptr, MC_EINVAL, "mc_ocp_solve_batch: NMPC only");
  if (n < 0) return fail(nullptr, MC_EINVAL, "mc_ocp_solve_batch: n < 0");
  if (n == 0) return MC_OK;
  const int N = c.N;
  const size_t n1 = (size_t)n * N, n2 = (size_t)n * (N + 1);
  OcpBatch d{};
  std::vector<void*> owned;
  bool ok = true;
  auto up = [&](double** dst, const double* src, size_t cnt) {
    double* p = nullptr;
    ok = ok && to_dev(&p, src, cnt);
    owned.push_back(p);
    *dst = p;
  };
  double *dx0, *dEaR, *dzb;
  up(&dx0, x0, n); up(&dEaR, EaR, n); up(&dzb, zbar, n2);
  d.x0 = dx0; d.EaR = dEaR; d.zbar = dzb;
  up(&d.u, u, n1); up(&d.x, x, n2); up(&d.lam, lam, n1); up(&d.pil, pil, n1);
  up(&d.piu, piu, n1); up(&d.kkt, nullptr, 3 * n);
  int32_t* di = nullptr;
  ok = ok && to_dev<int32_t>(&di, nullptr, 4 * n);
  owned.push_back(di);
  d.info = di;
  double* ws = nullptr;
  ok = ok && to_dev<double>(&ws, nullptr, (size_t)kNArr * (N + 1) * n);
  owned.push_back(ws);
  mc_status s = MC_OK;
  if (!ok) {
    s = fail(nullptr, MC_ENOMEM, "mc_ocp_solve_batch: allocation");
  } else {
    k_ocp_batch<<<(unsigned)((n + 127) / 128), 128>>>(m, c, n, d, ws, n);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(u, d.u, sizeof(double) * n1, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(x, d.x, sizeof(double) * n2, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(lam, d.lam, sizeof(double) * n1, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(pil, d.pil, sizeof(double) * n1, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(piu, d.piu, sizeof(double) * n1, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(info, di, sizeof(int32_t) * 4 * n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(kkt, d.kkt, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) s = cuda_fail(nullptr, e, "mc_ocp_solve_batch");
  }
  for (void* p : owned) cudaFree(p);
  return s;
}

mc_status mc_ocp_sens_batch(const mc_model_t* model, const mc_controller_t* ctrl, int64_t n,
                            const double* x0, const double* EaR, const double* zbar,
                            const double* u, const double* x, const double* lam,
                            const double* pil, const double* piu, double* sens,
                            int32_t* status) {
  if (n < 0 || (n > 0 && (!x0 || !EaR || !zbar || !u || !x || !lam || !pil || !piu || !sens ||
                          !status)))
    return fail(nullptr, MC_EINVAL, "mc_ocp_sens_batch: bad arguments");
  DevModel m;
  DevCtrl c;
  std::string why;
  if (fill_dev(model, ctrl, 0, &m, &c, &why) != MC_OK) return fail(nullptr, MC_EINVAL, why);
  if (c.kind != MC_CTRL_NMPC || c.nx_model == 3)
    return fail(nullptr, MC_EINVAL, "mc_ocp_sens_batch: one-state NMPC controller needed");
  if (n == 0) return MC_OK;
  const int N = c.N;
  const size_t n1 = (size_t)n * N, n2 = (size_t)n * (N + 1);
  OcpBatch d{};
  std::vector<void*> owned;
  bool ok = true;
  auto up = [&](const double** dst, const double* src, size_t cnt) {
    double* p = nullptr;
    ok = ok && to_dev(&p, src, cnt);
    owned.push_back(p);
    *dst = p;
  };
  auto upm = [&](double** dst, const double* src, size_t cnt) {
    double* p = nullptr;
    ok = ok && to_dev(&p, src, cnt);
    owned.push_back(p);
    *dst = p;
  };
  up(&d.x0, x0, n); up(&d.EaR, EaR, n); up(&d.zbar, zbar, n2);
  upm(&d.u, u, n1); upm(&d.x, x, n2); upm(&d.lam, lam, n1); upm(&d.pil, pil, n1);
  upm(&d.piu, piu, n1);
  int32_t* dinfo = nullptr;
  double *dsens = nullptr, *ws = nullptr;
  ok = ok && to_dev<int32_t>(&dinfo, nullptr, n) && to_dev<double>(&dsens, nullptr, 4 * n) &&
       to_dev<double>(&ws, nullptr, (size_t)kNArr * (N + 1) * n);
  owned.push_back(dinfo);
  owned.push_back(dsens);
  owned.push_back(ws);
  d.info = dinfo;
  mc_status s = MC_OK;
  if (!ok) {
    s = fail(nullptr, MC_ENOMEM, "mc_ocp_sens_batch: allocation");
  } else {
    k_ocp_sens_batch<<<(unsigned)((n + 127) / 128), 128>>>(m, c, n, d, dsens, ws, n);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(sens, dsens, sizeof(double) * 4 * n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(status, dinfo, sizeof(int32_t) * n, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) s = cuda_fail(nullptr, e, "mc_ocp_sens_batch");
  }
  for (void* p : owned) cudaFree(p);
  return s;
}

// ------------------------------------------------------- no-allocation reduce

}  // extern "C"

// Scratch of mc_reduce_noalloc: block partials for at most
// MC_NOALLOC_MAX_TRAJ / kStatThreads blocks and one result record.  Device
// code could name these directly; host code must go through the device
// address that cudaGetSymbolAddress returns (the host-side name is only a
// stand-in, not a device address).
static __device__ __align__(256) Partial g_noalloc_part[MC_NOALLOC_MAX_TRAJ / kStatThreads];
static __device__ __align__(256) DevStats g_noalloc_stats;

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
Partial* g_noalloc_part_ptr[kMaxDevices] = {};
DevStats* g_noalloc_stats_ptr[kMaxDevices] = {};

// Device addresses of the scratch on the current device; looked up once per
// device, with that device current.
cudaError_t noalloc_scratch(Partial** part, DevStats** st) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_part_ptr[dev]) {
    void* p = nullptr;
    void* q = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_part);
    if (e != cudaSuccess) return e;
    e = cudaGetSymbolAddress(&q, g_noalloc_stats);
    if (e != cudaSuccess) return e;
    g_noalloc_part_ptr[dev] = (Partial*)p;
    g_noalloc_stats_ptr[dev] = (DevStats*)q;
  }
  *part = g_noalloc_part_ptr[dev];
  *st = g_noalloc_stats_ptr[dev];
  return cudaSuccess;
}
}  // namespace

extern "C" {

mc_status mc_reduce_noalloc(const double* phi_dev, const int32_t* counters_dev, int64_t n,
                            int32_t n_bins, double lo, double hi, void* cuda_stream,
                            mc_stats_t* out_host) {
  if (!phi_dev || !counters_dev || !out_host)
    return fail(nullptr, MC_EINVAL, "mc_reduce_noalloc: null pointer");
  if (n < 0 || n > MC_NOALLOC_MAX_TRAJ)
    return fail(nullptr, MC_EINVAL,
                "mc_reduce_noalloc: n must be in 0..262144 (MC_NOALLOC_MAX_TRAJ), the size "
                "of its static scratch");
  if (n_bins < 1 || n_bins > MC_MAX_BINS)
    return fail(nullptr, MC_EINVAL, "mc_reduce_noalloc: n_bins must be 1..256");
  Partial* part = nullptr;
  DevStats* dst = nullptr;
  cudaError_t e = noalloc_scratch(&part, &dst);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "mc_reduce_noalloc: scratch address");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int nb = (int)((n + kStatThreads - 1) / kStatThreads);
  if (nb < 1) nb = 1;
  k_stats_partial<<<nb, kStatThreads, 0, st>>>(phi_dev, counters_dev, 0, n, part);
  k_stats_final<<<1, kStatThreads, 0, st>>>(part, nb, phi_dev, 0, n, n_bins, lo, hi, dst);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "mc_reduce_noalloc: launch");
  DevStats d;
  e = cudaMemcpyAsync(&d, dst, sizeof(d), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "mc_reduce_noalloc: result copy");
  memset(out_host, 0, sizeof(*out_host));
  out_host->n_traj = n;
  out_host->n_ocp_failed = d.sums[0];
  out_host->sqp_iters = d.sums[1];
  out_host->ls_trials = d.sums[2];
  out_host->n_hess_reset = d.sums[3];
  out_host->n_ls_fail = d.sums[4];
  out_host->qp_iters = d.sums[5];
  out_host->n_nonfinite = d.n_nonfinite;
  out_host->qp_fail = d.sums[7];
  out_host->phi_mean = d.mean;
  out_host->phi_var = (d.n > 1) ? d.m2 / (d.n - 1.0) : 0.0;
  out_host->phi_min = d.mn;
  out_host->phi_max = d.mx;
  out_host->n_bins = n_bins;
  out_host->bin_lo = d.lo;
  out_host->bin_hi = d.hi;
  for (int b = 0; b < MC_MAX_BINS; ++b) out_host->hist[b] = d.hist[b];
  return d.n_nonfinite > 0 ? MC_WARN_NONFINITE : MC_OK;
}

}  // extern "C"
