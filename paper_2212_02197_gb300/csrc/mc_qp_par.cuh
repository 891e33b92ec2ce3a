// mc_qp_par.cuh -- the structured QP of Eq. (QP-subproblem) (one state, one
// input per stage, input bounds) solved by one warp, the lanes over the
// stages: a parallel-in-horizon Riccati recursion inside the primal
// active-set method of qp_active_set (same working-set rule, same outputs).
//
// The three recursions of a Riccati solve are compositions of maps, so each
// is an associative scan over the stages (depth log2 32 = 5 shuffles):
//   P_k = M_k(P_{k+1})   with M_k a linear-fractional map: for a free input
//        P_k = W_xx + A^2 P - (W_xu + A B P)^2 / (W_uu + B^2 P)
//            = (alpha P + beta) / (gamma P + delta),
//        alpha = W_xx B^2 + A^2 W_uu - 2 A B W_xu, beta = W_xx W_uu - W_xu^2,
//        gamma = B^2, delta = W_uu (the P^2 terms cancel); for an input held
//        at a bound P_k = A^2 P + W_xx.  Such maps compose as 2x2 matrix
//        products, normalised by their largest entry (the map is unchanged).
//   p_k = a_k p_{k+1} + c_k       (affine once the P_{k+1} are known)
//   dx_{k+1} = e_k dx_k + f_k     (affine once the gains are known; dx_0 = 0)
// Lane l owns the ceil(N/32) consecutive stages starting at l * ceil(N/32);
// an exclusive scan gives the value at its chunk boundary, the serial
// formulas then run through the chunk.  The ratio test and the multiplier
// test are warp arg-min reductions that keep the serial order's tie-break
// (the first stage attaining the minimum), so the working sets evolve as in
// qp_active_set and the solution agrees with it to rounding.
#pragma once

#include "mc_qp.cuh"

namespace mc {

constexpr int kQpParMaxChunk = (kMaxN + 31) / 32;  // stages per lane

struct Mob {  // p -> (a p + b) / (c p + d)
  double a, b, c, d;
};
struct Aff {  // x -> a x + c
  double a, c;
};

// x o y (apply y first)
__device__ __forceinline__ Mob mob_compose(const Mob& x, const Mob& y) {
  Mob r{x.a * y.a + x.b * y.c, x.a * y.b + x.b * y.d, x.c * y.a + x.d * y.c,
        x.c * y.b + x.d * y.d};
  const double s = fmax(fmax(fabs(r.a), fabs(r.b)), fmax(fabs(r.c), fabs(r.d)));
  if (s > 0.0 && isfinite(s)) {
    const double is = 1.0 / s;
    r.a *= is;
    r.b *= is;
    r.c *= is;
    r.d *= is;
  }
  return r;
}
__device__ __forceinline__ Aff aff_compose(const Aff& x, const Aff& y) {
  return Aff{x.a * y.a, x.a * y.c + x.c};
}

__device__ __forceinline__ Mob shfl_down(const Mob& m, int d) {
  return Mob{__shfl_down_sync(0xffffffffu, m.a, d), __shfl_down_sync(0xffffffffu, m.b, d),
             __shfl_down_sync(0xffffffffu, m.c, d), __shfl_down_sync(0xffffffffu, m.d, d)};
}
__device__ __forceinline__ Aff shfl_down(const Aff& m, int d) {
  return Aff{__shfl_down_sync(0xffffffffu, m.a, d), __shfl_down_sync(0xffffffffu, m.c, d)};
}
__device__ __forceinline__ Aff shfl_up(const Aff& m, int d) {
  return Aff{__shfl_up_sync(0xffffffffu, m.a, d), __shfl_up_sync(0xffffffffu, m.c, d)};
}

// Exclusive suffix scan: lane l gets x_{l+1} o x_{l+2} o ... o x_31
// (the identity on the last lane).
__device__ __forceinline__ Mob suffix_exclusive(Mob x, int lane) {
  for (int d = 1; d < 32; d <<= 1) {
    const Mob o = shfl_down(x, d);
    if (lane + d < 32) x = mob_compose(x, o);
  }
  Mob e = shfl_down(x, 1);
  if (lane == 31) e = Mob{1.0, 0.0, 0.0, 1.0};
  return e;
}
__device__ __forceinline__ Aff suffix_exclusive(Aff x, int lane) {
  for (int d = 1; d < 32; d <<= 1) {
    const Aff o = shfl_down(x, d);
    if (lane + d < 32) x = aff_compose(x, o);
  }
  Aff e = shfl_down(x, 1);
  if (lane == 31) e = Aff{1.0, 0.0};
  return e;
}
// Exclusive prefix scan: lane l gets x_{l-1} o ... o x_0 (identity on lane 0).
__device__ __forceinline__ Aff prefix_exclusive(Aff x, int lane) {
  for (int d = 1; d < 32; d <<= 1) {
    const Aff o = shfl_up(x, d);
    if (lane >= d) x = aff_compose(x, o);
  }
  Aff e = shfl_up(x, 1);
  if (lane == 0) e = Aff{1.0, 0.0};
  return e;
}

// First (lowest k) stage attaining the minimum of v over the warp; k < 0 for
// lanes without a candidate (v = +inf).
__device__ __forceinline__ void warp_argmin(double& v, int& k) {
  for (int d = 16; d > 0; d >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, v, d);
    const int ok = __shfl_xor_sync(0xffffffffu, k, d);
    if (ov < v || (ov == v && ok >= 0 && (k < 0 || ok < k))) {
      v = ov;
      k = ok;
    }
  }
}

// Every lane of the warp calls this for the QP in column w (reads EA, EB,
// EG, WXX, WXU, WUU, EQ, QR if has_r, LB, UB; writes DU, DX, MU, NUL, NUU).
__device__ QpResult qp_active_set_warp(const Ws& w, int N, bool has_r, int max_it, int lane) {
  const int C = (N + 31) / 32;
  const int k0 = lane * C;
  int nk = N - k0;
  nk = nk < 0 ? 0 : (nk > C ? C : nk);
  double A[kQpParMaxChunk], B[kQpParMaxChunk], b[kQpParMaxChunk], Wxx[kQpParMaxChunk],
      Wxu[kQpParMaxChunk], Wuu[kQpParMaxChunk], q[kQpParMaxChunk], r[kQpParMaxChunk],
      lb[kQpParMaxChunk], ub[kQpParMaxChunk], du[kQpParMaxChunk], z[kQpParMaxChunk],
      Pn[kQpParMaxChunk], pn[kQpParMaxChunk], K[kQpParMaxChunk], kf[kQpParMaxChunk],
      dxn[kQpParMaxChunk], mu[kQpParMaxChunk], dxk[kQpParMaxChunk];
  bool lo[kQpParMaxChunk], up[kQpParMaxChunk];
#pragma unroll
  for (int i = 0; i < kQpParMaxChunk; ++i) dxk[i] = dxn[i] = mu[i] = z[i] = 0.0;
  double gscale = 1.0;
#pragma unroll
  for (int i = 0; i < kQpParMaxChunk; ++i) {
    const int k = k0 + i;
    lo[i] = up[i] = false;
    A[i] = B[i] = b[i] = Wxx[i] = Wxu[i] = Wuu[i] = q[i] = r[i] = lb[i] = ub[i] = du[i] = 0.0;
    if (i < nk) {
      A[i] = (k > 0) ? w(EA, k) : 0.0;
      B[i] = w(EB, k);
      b[i] = w(EG, k);
      Wxx[i] = w(WXX, k);
      Wxu[i] = w(WXU, k);
      Wuu[i] = w(WUU, k);
      q[i] = w(EQ, k);
      r[i] = has_r ? w(QR, k) : 0.0;
      lb[i] = w(LB, k);
      ub[i] = w(UB, k);
      if (lb[i] >= 0.0) {
        lo[i] = true;
        du[i] = lb[i];
      } else if (ub[i] <= 0.0) {
        up[i] = true;
        du[i] = ub[i];
      }
      gscale = fmax(gscale, fabs(w(EQ, k + 1)));
      if (has_r) gscale = fmax(gscale, fabs(r[i]));
    }
  }
  for (int d = 16; d > 0; d >>= 1) gscale = fmax(gscale, __shfl_xor_sync(0xffffffffu, gscale, d));
  const double mult_tol = 1e-13 * gscale;
  const double PN = w(WXX, N), qN = w(EQ, N);

  QpResult res{0, 1};
  for (int it = 0; it < max_it; ++it) {
    res.iters = it + 1;
    // ---- P_{k+1} for every stage: scan of the stage maps
    Mob chunk{1.0, 0.0, 0.0, 1.0};
    #pragma unroll
    for (int i = kQpParMaxChunk - 1; i >= 0; --i) if (i < nk) {
      Mob Mk;
      if (lo[i] || up[i]) {
        Mk = Mob{A[i] * A[i], Wxx[i], 0.0, 1.0};
      } else {
        Mk = Mob{Wxx[i] * B[i] * B[i] + A[i] * A[i] * Wuu[i] - 2.0 * A[i] * B[i] * Wxu[i],
                 Wxx[i] * Wuu[i] - Wxu[i] * Wxu[i], B[i] * B[i], Wuu[i]};
      }
      chunk = mob_compose(Mk, chunk);  // M_{k0} o ... o M_{k0+nk-1}
    }
    const Mob after = suffix_exclusive(chunk, lane);
    double P = (after.a * PN + after.b) / (after.c * PN + after.d);  // P at k0 + nk
    if (k0 + nk >= N) P = PN;
    bool pd = true;
    #pragma unroll
    for (int i = kQpParMaxChunk - 1; i >= 0; --i) if (i < nk) {
      Pn[i] = P;
      if (lo[i] || up[i]) {
        P = Wxx[i] + A[i] * A[i] * P;
      } else {
        const double Rb = Wuu[i] + B[i] * B[i] * P;
        pd = pd && (Rb > 0.0);
        const double Sb = Wxu[i] + A[i] * P * B[i];
        P = Wxx[i] + A[i] * A[i] * P - Sb * Sb / Rb;
      }
    }
    if (!__all_sync(0xffffffffu, pd)) {
      res.status = 2;
      return res;
    }
    // ---- p_{k+1}: scan of the affine maps p_k = a_k p_{k+1} + c_k
    Aff pchunk{1.0, 0.0};
    Aff pa[kQpParMaxChunk];
#pragma unroll
    for (int i = 0; i < kQpParMaxChunk; ++i) {
      pa[i] = Aff{1.0, 0.0};
      if (i >= nk) continue;
      const double Pk = Pn[i];
      if (lo[i] || up[i]) {
        const double c = du[i];
        pa[i] = Aff{A[i], q[i] + Wxu[i] * c + A[i] * Pk * (B[i] * c + b[i])};
      } else {
        const double Rb = Wuu[i] + B[i] * B[i] * Pk;
        const double iR = 1.0 / Rb;
        const double Sb = Wxu[i] + A[i] * Pk * B[i];
        pa[i] = Aff{A[i] - Sb * B[i] * iR,
                    q[i] + A[i] * Pk * b[i] - Sb * (r[i] + B[i] * Pk * b[i]) * iR};
      }
    }
    #pragma unroll
    for (int i = kQpParMaxChunk - 1; i >= 0; --i) if (i < nk) pchunk = aff_compose(pa[i], pchunk);
    const Aff pafter = suffix_exclusive(pchunk, lane);
    double pv = pafter.a * qN + pafter.c;
    if (k0 + nk >= N) pv = qN;
    #pragma unroll
    for (int i = kQpParMaxChunk - 1; i >= 0; --i) if (i < nk) {
      pn[i] = pv;
      const double Pk = Pn[i];
      const double Pbp = Pk * b[i] + pv;
      if (lo[i] || up[i]) {
        K[i] = 0.0;
        kf[i] = du[i];
      } else {
        const double Rb = Wuu[i] + B[i] * B[i] * Pk;
        const double iR = 1.0 / Rb;
        const double Sb = (k0 + i > 0) ? Wxu[i] + A[i] * Pk * B[i] : 0.0;
        K[i] = -Sb * iR;
        kf[i] = -(r[i] + B[i] * Pbp) * iR;
      }
      pv = pa[i].a * pv + pa[i].c;
    }
    // ---- forward rollout: dx_{k+1} = (A + B K) dx_k + (B kf + b), dx_0 = 0
    Aff fchunk{1.0, 0.0};
    #pragma unroll
    for (int i = 0; i < kQpParMaxChunk; ++i) if (i < nk)
      fchunk = aff_compose(Aff{A[i] + B[i] * K[i], B[i] * kf[i] + b[i]}, fchunk);
    const Aff before = prefix_exclusive(fchunk, lane);
    double dx = before.c;  // from dx_0 = 0
    #pragma unroll
    for (int i = 0; i < kQpParMaxChunk; ++i) if (i < nk) {
      dxk[i] = dx;
      z[i] = K[i] * dx + kf[i];
      const double d1 = A[i] * dx + B[i] * z[i] + b[i];
      dxn[i] = d1;
      mu[i] = -(Pn[i] * d1 + pn[i]);
      dx = d1;
    }
    // ---- ratio test over the free inputs (first blocking stage)
    double tmin = 1.0;
    int kb = -1;
    bool blo = false;
    #pragma unroll
    for (int i = 0; i < kQpParMaxChunk; ++i) if (i < nk) {
      if (lo[i] || up[i]) continue;
      const double pk = z[i] - du[i];
      if (pk < 0.0 && z[i] < lb[i]) {
        const double t = (lb[i] - du[i]) / pk;
        if (t < tmin) { tmin = t; kb = k0 + i; blo = true; }
      } else if (pk > 0.0 && z[i] > ub[i]) {
        const double t = (ub[i] - du[i]) / pk;
        if (t < tmin) { tmin = t; kb = k0 + i; blo = false; }
      }
    }
    double tv = (kb >= 0) ? tmin : INFINITY;
    int tk = kb;
    warp_argmin(tv, tk);
    const bool tlo = __shfl_sync(0xffffffffu, blo, tk >= 0 ? (tk / C) : 0);
    if (tk >= 0) {
      const double alpha = tv < 0.0 ? 0.0 : tv;
      #pragma unroll
      for (int i = 0; i < kQpParMaxChunk; ++i) if (i < nk) {
        if (lo[i] || up[i]) continue;
        du[i] = du[i] + alpha * (z[i] - du[i]);
        if (k0 + i == tk) {
          if (tlo) { lo[i] = true; du[i] = lb[i]; }
          else { up[i] = true; du[i] = ub[i]; }
        }
      }
      continue;
    }
    // ---- subspace minimiser reached; multipliers of the working set
    double wv = INFINITY;
    int wk = -1;
    #pragma unroll
    for (int i = 0; i < kQpParMaxChunk; ++i) if (i < nk) {
      const bool f = lo[i] || up[i];
      if (!f) {
        du[i] = z[i];
        continue;
      }
      const double cross = (k0 + i > 0) ? Wxu[i] * dxk[i] : 0.0;
      const double v = Wuu[i] * du[i] + cross + r[i] - mu[i] * B[i];
      const double lam = lo[i] ? v : -v;
      if (lam < -mult_tol && lam < wv) { wv = lam; wk = k0 + i; }
    }
    warp_argmin(wv, wk);
    if (wk < 0) {
      res.status = 0;
      break;
    }
    #pragma unroll
    for (int i = 0; i < kQpParMaxChunk; ++i) if (i < nk)
      if (k0 + i == wk) lo[i] = up[i] = false;
  }
  // the solution (or, at the iteration limit, the last working-set point) and
  // the bound multipliers from stationarity in du
  #pragma unroll
  for (int i = 0; i < kQpParMaxChunk; ++i) if (i < nk) {
    const int k = k0 + i;
    double nl = 0.0, nu = 0.0;
    if (lo[i] || up[i]) {
      const double cross = (k > 0) ? Wxu[i] * dxk[i] : 0.0;
      const double v = Wuu[i] * du[i] + cross + r[i] - mu[i] * B[i];
      if (lo[i]) nl = v; else nu = -v;
    }
    w(DU, k) = du[i];
    w(DX, k + 1) = dxn[i];
    w(MU, k) = mu[i];
    w(NUL, k) = nl;
    w(NUU, k) = nu;
  }
  if (lane == 0) w(DX, 0) = 0.0;
  return res;
}

}  // namespace mc
