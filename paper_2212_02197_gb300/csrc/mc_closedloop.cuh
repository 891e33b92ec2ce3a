// mc_closedloop.cuh -- one stochastic closed-loop simulation per thread
// (Sec. VII): plant SDE by Euler-Maruyama, noisy measurement, controller
// (NMPC = CD-EKF + SQP, or PI), and the performance index Phi, Eq. (Phi).
//
// Two schedules of the NMPC closed loop:
//   traj_nmpc        one trajectory per thread, SQPs run to completion one after
//                    the other; the lanes of a warp wait for the slowest OCP
//   nmpc_persistent  a per-lane state machine: every lane advances its own
//                    trajectory through the cheap phases until it needs
//                    shooting (a line-search trial point, or the first
//                    evaluation of a new OCP), and the warp then shoots all
//                    pending intervals as one pool spread over its lanes;
//                    finished lanes take the next trajectory from a queue.
//                    Same arithmetic per trajectory, bit for bit.
#pragma once

#include "mc_sqp.cuh"

namespace mc {

struct TrajOut {
  double phi;
  int32_t cnt[kNCounters];  // n_ocp_failed, sqp_iters, ls_trials, n_hess_reset,
                            // n_ls_fail, qp_iters, nonfinite, qp_fail
};

// Plant between two samples: N_s Euler-Maruyama substeps with zero-order hold
// on the flow F (L/s) and the inlet temperature (which steps at t_d).  The
// substeps' normals are drawn here, or read from nzc (substep s, component d
// at nzc[(3 s + d) nz_ld]) where the persistent schedule's pool drew them.
template <class R>
__device__ __forceinline__ void plant_interval(const DevModel& m, const TrajParams& tp,
                                               uint32_t j, int i, double F, double n[3],
                                               const double* nzc = nullptr,
                                               int64_t nz_ld = 0) {
  const R hR = (R)m.hEM, sqh = (R)m.sqhEM;
  R nr[3] = {(R)n[0], (R)n[1], (R)n[2]};
  const R EaR = (R)tp.EaR, FR = (R)F;
  for (int s = 0; s < m.n_em; ++s) {
    const int64_t ks = (int64_t)i * m.n_em + s;
    const double Tin = inlet_T_at(m, tp, ks);
    R xi[3];
    if (nzc) {
#pragma unroll
      for (int d = 0; d < 3; ++d) xi[d] = (R)nzc[(3 * s + d) * nz_ld];
    } else {
      process_noise<R>(m, j, (uint32_t)ks, xi);
    }
    em_step<R>(m, EaR, (R)Tin, nr, FR, hR, sqh, xi);
  }
  n[0] = (double)nr[0];
  n[1] = (double)nr[1];
  n[2] = (double)nr[2];
}

template <class R>
__device__ TrajOut traj_pi(const DevModel& m, const DevCtrl& c, uint32_t j) {
  TrajOut out{};
  const TrajParams tp = traj_params(m, c, j);
  double n[3] = {m.cA_in * m.V, m.cB_in * m.V, m.T_in * m.V};
  const int K = m.n_steps;
  double phi = 0.0;
  R Ihat = 0;
  for (int i = 0; i <= K; ++i) {
    const double cT = n[2] / m.V;
    if (!isfinite(cT)) {
      out.cnt[6] = 1;
      phi = nan("");
      break;
    }
    const double zi = zbar_at(m, i);
    const double ez = cT - zi;
    phi += ez * ez;
    if (i == K) break;
    const double y = cT + m.meas_sd * (double)meas_noise<R>(m, j, (uint32_t)i);
    const double ubar = Fss(m, tp.EaR_c, zi);
    const double F = (double)pi_step<R>(c, (R)m.Ts, (R)zi, (R)y, (R)ubar, Ihat);
    plant_interval<R>(m, tp, j, i, F, n);
  }
  out.phi = phi / (double)(K + 1);
  return out;
}

// ---------------------------------------------------------------------------
// NMPC closed loop, split into the steps both schedules share.

struct NmpcTraj {
  uint32_t j;
  int i;                   // current sample
  TrajParams tp;
  double n[3], xhat, P, F_prev, phi;
  TrajOut out;
};

// Trajectory start (Sec. VII-A): plant filled with feed, EKF at x-hat_{-1|-1},
// first OCP guess u = F_ss(z-bar(t_0)) clipped, states at the estimate.
__device__ __forceinline__ void nmpc_begin(const DevModel& m, const DevCtrl& c, uint32_t j,
                                           const Ws& w, NmpcTraj& T) {
  T.j = j;
  T.i = 0;
  T.tp = traj_params(m, c, j);
  T.n[0] = m.cA_in * m.V;
  T.n[1] = m.cB_in * m.V;
  T.n[2] = m.T_in * m.V;
  T.xhat = m.T_in * m.V;
  T.P = c.P0;
  T.F_prev = 0.0;
  T.phi = 0.0;
  T.out = TrajOut{};
  double v0 = Fss(m, T.tp.EaR_c, zbar_at(m, 0)) / c.Fconv;
  v0 = fmin(fmax(v0, c.vmin), c.vmax);
  const double ixs = 1.0 / c.x_scale;
  for (int k = 0; k < T.tp.N; ++k) {
    w(U, k) = v0;
    w(X, k + 1) = T.xhat * ixs;
    w(LAM, k) = 0.0;
    w(PIL, k) = 0.0;
    w(PIU, k) = 0.0;
  }
}

// Sample i: Phi term, and unless the trajectory ends there the measurement,
// the CD-EKF and the start of the OCP.  Returns false when the trajectory is
// finished (T.out is final).
template <class R>
__device__ __forceinline__ bool nmpc_sample_body(const DevModel& m, const DevCtrl& c,
                                                 const Ws& w, NmpcTraj& T, SqpState& s,
                                                 bool shoot) {
  const int K = m.n_steps, N = T.tp.N;
  const double cT = T.n[2] / m.V;
  if (!isfinite(cT) || !isfinite(T.xhat) || !isfinite(T.P)) {
    T.out.cnt[6] = 1;
    T.out.phi = nan("");
    return false;
  }
  const double ez = cT - zbar_at(m, T.i);
  T.phi += ez * ez;
  if (T.i == K) {
    T.out.phi = T.phi / (double)(K + 1);
    return false;
  }
  const double y = cT + m.meas_sd * (double)meas_noise<R>(m, T.j, (uint32_t)T.i);
  if (T.i > 0) {
    // the CD-EKF prediction from x-hat_{i-1|i-1}, P_{i-1|i-1} under the applied
    // input: the last OCP's interval-0 shooting at its final iterate carried it
    T.xhat = w(EPR, 0);
    T.P = w(EPR, 1);
  }
  ekf_filter(m, y, T.xhat, T.P);
  w(PIN, 0) = T.P;
  for (int k = 1; k <= N; ++k) w(ZB, k) = zbar_at(m, T.i + k);
  if (c.Ru != 0.0)
    for (int k = 1; k <= N; ++k) w(VB, k) = Fss(m, T.tp.EaR_c, w(ZB, k)) / c.Fconv;
  sqp_start<R>(m, c, T.tp.EaR_c, T.xhat * (1.0 / c.x_scale), w, N, T.tp.max_it, T.i > 0, s,
               shoot);
  return true;
}

// The receding-horizon shift of the warm start and of the final evaluation
// by one interval, the last entry duplicated (columns as in the SQP passes).
__device__ __forceinline__ void shift_pass(int N, int64_t ld, double* __restrict__ u_,
                                           double* __restrict__ x1_, double* __restrict__ lam_,
                                           double* __restrict__ pil_, double* __restrict__ piu_,
                                           double* __restrict__ ea_, double* __restrict__ eb_,
                                           double* __restrict__ eg_) {
#pragma unroll 2
  for (int k = 0; k < N - 1; ++k) {
    const int64_t o = k * ld;
    u_[o] = u_[o + ld];
    x1_[o] = x1_[o + ld];
    lam_[o] = lam_[o + ld];
    pil_[o] = pil_[o + ld];
    piu_[o] = piu_[o + ld];
    ea_[o] = ea_[o + ld];
    eb_[o] = eb_[o + ld];
    eg_[o] = eg_[o + ld];
  }
}

// After the OCP of sample i: count it, apply u_0, shift the warm start (and
// the final evaluation) one interval, simulate the plant to t_{i+1}.
template <class R>
__device__ __forceinline__ void nmpc_apply_body(const DevModel& m, const DevCtrl& c,
                                                const Ws& w, NmpcTraj& T, const SqpInfo& si,
                                                const double* nzc, int64_t nz_ld) {
  const int N = T.tp.N;
  T.out.cnt[0] += (si.status == 1);
  T.out.cnt[1] += si.iters;
  T.out.cnt[2] += si.ls_trials;
  T.out.cnt[3] += si.n_hess_reset;
  T.out.cnt[4] += (si.status == 2);
  T.out.cnt[5] += si.qp_iters;
  T.out.cnt[7] += si.qp_fail;
  const double F = w(U, 0) * c.Fconv;
  shift_pass(N, w.ld, ws_col(w, U), ws_col(w, X) + w.ld, ws_col(w, LAM), ws_col(w, PIL),
             ws_col(w, PIU), ws_col(w, EA), ws_col(w, EB), ws_col(w, EG));
  plant_interval<R>(m, T.tp, T.j, T.i, F, T.n, nzc, nz_ld);
  T.F_prev = F;
  T.i++;
}

// Code placement as for sqp_check: separate functions on the mixed path.
template <class R>
__device__ __noinline__ bool nmpc_sample_call(const DevModel& m, const DevCtrl& c, const Ws& w,
                                              NmpcTraj& T, SqpState& s, bool shoot) {
  return nmpc_sample_body<R>(m, c, w, T, s, shoot);
}
template <class R>
__device__ __noinline__ void nmpc_apply_call(const DevModel& m, const DevCtrl& c, const Ws& w,
                                             NmpcTraj& T, const SqpInfo& si,
                                             const double* nzc, int64_t nz_ld) {
  nmpc_apply_body<R>(m, c, w, T, si, nzc, nz_ld);
}
// shoot = false: the OCP's first evaluation is left to the caller (the
// persistent schedule's pool, then sqp_start_eval).
template <class R>
__device__ __forceinline__ bool nmpc_sample(const DevModel& m, const DevCtrl& c, const Ws& w,
                                            NmpcTraj& T, SqpState& s, bool shoot = true) {
  if constexpr (sizeof(R) == 4) return nmpc_sample_call<R>(m, c, w, T, s, shoot);
  else return nmpc_sample_body<R>(m, c, w, T, s, shoot);
}
// nzc: the plant interval's normals, drawn beforehand (see plant_interval).
template <class R>
__device__ __forceinline__ void nmpc_apply(const DevModel& m, const DevCtrl& c, const Ws& w,
                                           NmpcTraj& T, const SqpInfo& si,
                                           const double* nzc = nullptr, int64_t nz_ld = 0) {
  if constexpr (sizeof(R) == 4) nmpc_apply_call<R>(m, c, w, T, si, nzc, nz_ld);
  else nmpc_apply_body<R>(m, c, w, T, si, nzc, nz_ld);
}

// R = double: the FP64 path.  R = float: the mixed-precision path -- plant
// SDE, noise transform, EKF prediction and the OCP shooting in FP32; the
// Joseph-form filter update, the QP (Riccati pivots), merit, BFGS and the SQP
// convergence test in FP64.
template <class R>
__device__ TrajOut traj_nmpc(const DevModel& m, const DevCtrl& c, uint32_t j, const Ws& w) {
  NmpcTraj T;
  SqpState s;
  nmpc_begin(m, c, j, w, T);
  while (nmpc_sample<R>(m, c, w, T, s)) {
    while (!sqp_check<R>(c, w, s)) {
      int r;
      do {
        sqp_eval_trial<R>(m, c, T.tp.EaR_c, w, s);
        r = sqp_trial_result<R>(c, w, s);
      } while (r == 2);
      if (r == 1) break;
    }
    nmpc_apply<R>(m, c, w, T, s.info);
  }
  return T.out;
}

// ---------------------------------------------------------------------------
// Persistent schedule: the shooting pool.
//
// Every shooting interval the warp needs in a round -- the N_o intervals of
// each pending trial point, and the intervals 0 and N-1 (all N on the first
// sample) of each OCP that just started -- is one job.  The jobs are numbered
// interval-major (job position i of every lane that has one, lanes in order,
// then position i + 1) and lane t takes jobs t, t + 32, ...; so a round with
// every lane pending shoots like the joint loop (lane t integrates its own
// interval i, coalesced), and a round with few pending lanes spreads their
// intervals over the whole warp.  Each job is one call of the shoot_interval
// body, whichever lane runs it: the results are those of evaluate, bit for bit.

enum PoolMode : int { kPoolTrial = 0, kPoolStartEnds = 1, kPoolStartAll = 2 };

// A trial job's position is q N + k: interval k of line-search candidate q.
struct PoolTab {
  unsigned mask[MC_MAX_HORIZON * kLsCand];  // lanes with a job at position i
  int pref[MC_MAX_HORIZON * kLsCand];       // jobs before position i
  double EaR[32];
  int N[32], mode[32];
  uint32_t j[32];                 // trajectory and sample of each lane's OCP
  int i[32];
};

template <class R>
__device__ __forceinline__ void pool_shoot(const DevModel& m, const DevCtrl& c, const Ws& w,
                                           int n_jobs, int mode, int N, double EaR,
                                           PoolTab& tab) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int max_jobs = (int)__reduce_max_sync(full, (unsigned)n_jobs);
  __syncwarp();  // the previous round's readers of tab are done
  tab.EaR[lane] = EaR;
  tab.N[lane] = N;
  tab.mode[lane] = mode;
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
  const double xs = c.x_scale, ixs = 1.0 / c.x_scale;
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
    const int md = tab.mode[o];
    const bool trial = (md == kPoolTrial);
    const int cq = trial ? lo / tab.N[o] : 0;  // line-search candidate of a trial job
    const int k = (md == kPoolStartEnds && lo == 1) ? tab.N[o] - 1 : lo - cq * tab.N[o];
    const int ua = trial ? lsc_col(UT, cq) : U, xa = trial ? lsc_col(XT, cq) : X;
    const int aa = trial ? lsc_col(TA, cq) : EA, ba = trial ? lsc_col(TB, cq) : EB;
    const int ga = trial ? lsc_col(TG, cq) : EG;
    const Ws wo{w.p + (o - lane), w.ld, w.N1};
    const double xk = (k == 0) ? wo(X, 0) : wo(xa, k);
    const Shot r = shoot_interval<R>(m, c, tab.EaR[o], xk, wo(ua, k), wo(xa, k + 1), xs, ixs,
                                     k == 0, wo(PIN, 0));
    wo(aa, k) = r.A;
    wo(ba, k) = r.B;
    wo(ga, k) = r.g;
    if (k == 0) {
      const int pa = trial ? lsc_col(TPR, cq) : EPR;
      wo(pa, 0) = r.xpr;
      wo(pa, 1) = r.Ppr;
    }
  }
  __syncwarp();  // the shot intervals are visible to their owners
}

// One Box-Muller pair of process noise (counter (ks, j, tag, 0)); not inlined,
// so that the elementary functions do not add to the schedule's registers.
template <class R>
__device__ __noinline__ double2 pool_normal_pair(const DevModel& m, uint32_t ks, uint32_t j,
                                                 uint32_t tag) {
  return Normal2<R>::from(philox4x32_10(make_uint4(ks, j, tag, 0u), m.key0, m.key1));
}

// The normals of the plant interval that follows each OCP started this round
// (2 N_s Box-Muller pairs per lane: tags 0 and 1 of each substep, Philox
// counters as in process_noise), drawn by the whole warp, substep-major, into
// the owners' columns of nz (substep s, component d at nz[(3 s + d) ld]).
template <class R>
__device__ __forceinline__ void pool_noise(const DevModel& m, double* nzl, int64_t ld,
                                           bool starting, uint32_t j, int i, PoolTab& tab) {
  const unsigned sm = __ballot_sync(0xffffffffu, starting);
  if (!sm) return;
  const int lane = threadIdx.x & 31;
  tab.j[lane] = j;
  tab.i[lane] = i;
  __syncwarp();
  const int P = __popc(sm);
  const int total = P * 2 * m.n_em;
  for (int q = lane; q < total; q += 32) {
    const int e = q / P;
    unsigned mo = sm;
    for (int r = q - e * P; r > 0; --r) mo &= mo - 1u;
    const int o = __ffs(mo) - 1;
    const int sub = e >> 1;
    const uint32_t tag = (uint32_t)(e & 1);
    const uint32_t ks = (uint32_t)((int64_t)tab.i[o] * m.n_em + sub);
    const double2 z = pool_normal_pair<R>(m, ks, tab.j[o], tag);
    double* no = nzl + (o - lane);
    if (tag == 0) {
      no[(3 * sub) * ld] = (double)(R)z.x;
      no[(3 * sub + 1) * ld] = (double)(R)z.y;
    } else {
      no[(3 * sub + 2) * ld] = (double)(R)z.x;
    }
  }
  __syncwarp();
}

// Every lane of the warp must call this (it uses warp votes); trajectories
// come from the queue `next` (positions 0 .. n-1, mapped through `order` when
// given, else to j0 + position) and are written to phi_out / cnt_out.
//
// A round: each lane runs its cheap phases until it needs shooting -- a trial
// point (kTrial), or the first evaluation of the OCP it just started (kStart)
// -- then the warp shoots all of it in the pool, and each lane finishes its
// evaluation.  A lane whose line search backtracks has the next halvings shot
// together (sqp_trial_points_spec) and tests them in order.  A started OCP takes its first QP in the next round's check,
// together with the other lanes' checks, rather than on its own.
//
// With G::kRecord (G = the NMPC-weight gradient's Recorder, FP64) the loop
// also hands the recorder, per sample, the state the sample starts from and
// the OCP's KKT point; the tangents are propagated afterwards, by all lanes in
// step.  G = NoRecord runs the closed loop alone.
//
// wtrace (may be null) receives the warp's record, kWarpTraceWords words per
// warp (warp = block): the pool rounds it ran, its lane-rounds (the sum over
// those rounds of its lanes still holding a trajectory), the GPU's global
// timer (ns) when it started and finished, and the SM it ran on.
enum LanePhase : int { kNewTraj = 0, kSample = 1, kCheck = 2, kTrial = 3, kStart = 4, kDone = 5 };

struct NoRecord {
  static constexpr bool kRecord = false;
};

constexpr int kWarpTraceWords = 5;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <class R, class G = NoRecord>
__device__ void nmpc_persistent(const DevModel& m, const DevCtrl& c, const Ws& w, double* nzl,
                                int64_t j0, int64_t n, const uint32_t* __restrict__ order,
                                unsigned long long* next, double* __restrict__ phi_out,
                                int32_t* __restrict__ cnt_out,
                                unsigned long long* __restrict__ wtrace, G g = G{}) {
  __shared__ PoolTab tab;  // one per block: the kernel runs one warp per block
  NmpcTraj T;
  SqpState s;
  int phase = kNewTraj;
  const unsigned long long t_start = global_ns();
  unsigned long long rounds = 0, lane_rounds = 0;
  for (;;) {
    // cheap, divergent phases until this lane needs shooting
    while (phase != kTrial && phase != kStart && phase != kDone) {
      if (phase == kNewTraj) {
        const unsigned long long q = atomicAdd(next, 1ull);
        if (q >= (unsigned long long)n) {
          phase = kDone;
          break;
        }
        const uint32_t j = order ? order[q] : (uint32_t)(j0 + (int64_t)q);
        nmpc_begin(m, c, j, w, T);
        phase = kSample;
      }
      if (phase == kSample) {
        if constexpr (G::kRecord) g.sample(w, T);
        if (nmpc_sample<R>(m, c, w, T, s, false)) {
          phase = kStart;
        } else {
          phi_out[T.j] = T.out.phi;
#pragma unroll
          for (int q = 0; q < kNCounters; ++q)
            cnt_out[(int64_t)T.j * kNCounters + q] = T.out.cnt[q];
          if constexpr (G::kRecord) g.finish(T);
          phase = kNewTraj;
        }
        continue;
      }
      if (phase == kCheck) {
        if (sqp_check<R>(c, w, s)) {
          if constexpr (G::kRecord) g.ocp(w, T);
          nmpc_apply<R>(m, c, w, T, s.info, nzl, w.ld);
          phase = kSample;
        } else {
          phase = kTrial;
        }
      }
    }
    const unsigned busy = __ballot_sync(0xffffffffu, phase != kDone);
    if (!busy) break;
    const int nbusy = __popc(busy);
    ++rounds;
    lane_rounds += (unsigned)nbusy;
    pool_noise<R>(m, nzl, w.ld, phase == kStart, T.j, T.i, tab);
    int n_jobs = 0, mode = kPoolTrial;
    if (phase == kTrial) {
      n_jobs = s.N * s.nc;
    } else if (phase == kStart) {
      const bool ends = (T.i > 0);
      mode = ends ? kPoolStartEnds : kPoolStartAll;
      n_jobs = ends ? (s.N > 1 ? 2 : 1) : s.N;
    }
    pool_shoot<R>(m, c, w, n_jobs, mode, s.N, T.tp.EaR_c, tab);
    if (phase == kStart) {
      sqp_start_eval<R>(m, c, T.tp.EaR_c, w, s);
      phase = kCheck;
    } else if (phase == kTrial) {
      // the shot candidates in order, as the sequential line search tries them
      int r = 2;
      for (int q = 0; q < s.nc && r == 2; ++q) {
        sqp_eval_trial_shot<R>(m, c, T.tp.EaR_c, w, s, q);
        r = sqp_trial_result<R>(c, w, s, q, false);
      }
      if (r == 0) {
        phase = kCheck;
      } else if (r == 1) {
        if constexpr (G::kRecord) g.ocp(w, T);
        nmpc_apply<R>(m, c, w, T, s.info, nzl, w.ld);
        phase = kSample;
      } else {
        sqp_trial_points_spec(c, w, s, nbusy);  // backtracking: the next halvings together
      }
    }
  }
  if (wtrace && (threadIdx.x & 31) == 0) {
    unsigned smid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    unsigned long long* o = wtrace + (int64_t)blockIdx.x * kWarpTraceWords;
    o[0] = rounds;
    o[1] = lane_rounds;
    o[2] = t_start;
    o[3] = global_ns();
    o[4] = smid;
  }
}

}  // namespace mc
