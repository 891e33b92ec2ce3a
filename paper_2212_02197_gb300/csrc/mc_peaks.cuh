// mc_peaks.cuh -- throughput probes of the arithmetic the closed loop runs on,
// for the roofline of the simulation kernels: FP64 fused multiply-adds (the
// pipe the FP64 path is bound by), FP32 fused multiply-adds, and the FP64
// elementary operations of the rate law, the CD-EKF and the noise transform
// (exp -- the kernel's own table-driven one and the library's -- division,
// the rate law's Newton-refined reciprocal, log, sqrt, sincospi) and FP32
// expf.
//
// Every thread runs kChains independent chains for `iters` iterations.  Each
// chain step is x = fma(x, a, b) (keeps x in a fixed range) followed by
// y += op(x); the DFMA probe runs only the fma, and the "none" probe the fma
// and the add, so the cost of op in DFMA equivalents is
//   (t_op - t_none) / t_dfma_step,
// with t_dfma_step the time of one DFMA from the DFMA probe.  Results are
// written out so that nothing is optimised away.
#pragma once

#include "mc_device.cuh"

namespace mc {

enum PipeProbe : int {
  kProbeDfma = 0,   // x = fma(x, a, b)            (1 DFMA per step)
  kProbeNone = 1,   // x = fma(x, a, b); y += x    (1 DFMA + 1 DADD)
  kProbeExpTab = 2, // ... y += exp_table(x), x in [-31, -20] (the rate law's range)
  kProbeExpLib = 3, // ... y += exp(x)
  kProbeDiv = 4,    // ... y += 1 / x, x near 300
  kProbeLog = 5,    // ... y += log(x), x in (0, 1)
  kProbeSqrt = 6,   // ... y += sqrt(x)
  kProbeSincos = 7, // ... y += s + c, sincospi(x)
  kProbeFfma = 8,   // FP32: x = fmaf(x, a, b)     (1 FFMA per step)
  kProbeExpf = 9,   // FP32: x = fmaf(x, a, b); y += expf(x)
  kProbeNoneF = 10, // FP32: x = fmaf(x, a, b); y += x
  kProbeRcp = 11,   // ... y += rcp_newton(x), x near 300
  kNumProbes = 12
};

constexpr int kChains = 8;

template <int kKind>
__global__ void __launch_bounds__(128) k_pipe_probe(int64_t iters, double seed,
                                                    double* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const double jitter = 1e-9 * (double)(t & 1023);
  if constexpr (kKind == kProbeFfma || kKind == kProbeExpf || kKind == kProbeNoneF) {
    float x[kChains], y[kChains];
    const float a = (float)(1.0 - 1e-7 * seed), b = (float)(-2.5e-6 * seed);
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
      x[i] = (float)(-25.0 - 0.5 * i - jitter);
      y[i] = 0.0f;
    }
    for (int64_t s = 0; s < iters; ++s) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) {
        x[i] = fmaf(x[i], a, b);
        if constexpr (kKind == kProbeExpf) y[i] += expf(x[i]);
        if constexpr (kKind == kProbeNoneF) y[i] += x[i];
      }
    }
    float acc = 0.0f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) acc += x[i] + y[i];
    out[t] = (double)acc;
  } else {
    double x[kChains], y[kChains];
    // x stays in the range the probed operation sees in the closed loop
    double x0 = -25.0, a = 1.0 - 1e-9 * seed, b = -2.5e-8 * seed;
    if (kKind == kProbeDiv || kKind == kProbeRcp) { x0 = 300.0; b = 3e-7 * seed; }
    if (kKind == kProbeLog || kKind == kProbeSqrt || kKind == kProbeSincos) {
      x0 = 0.5; b = 5e-10 * seed;
    }
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
      x[i] = x0 - 0.01 * i - jitter;
      y[i] = 0.0;
    }
    for (int64_t s = 0; s < iters; ++s) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) {
        x[i] = fma(x[i], a, b);
        if constexpr (kKind == kProbeNone) y[i] += x[i];
        if constexpr (kKind == kProbeExpTab) y[i] += exp_table(x[i]);
        if constexpr (kKind == kProbeExpLib) y[i] += exp(x[i]);
        if constexpr (kKind == kProbeDiv) y[i] += 1.0 / x[i];
        if constexpr (kKind == kProbeRcp) y[i] += rcp_newton(x[i]);
        if constexpr (kKind == kProbeLog) y[i] += log(x[i]);
        if constexpr (kKind == kProbeSqrt) y[i] += sqrt(x[i]);
        if constexpr (kKind == kProbeSincos) {
          double sn, cs;
          sincospi(x[i], &sn, &cs);
          y[i] += sn + cs;
        }
      }
    }
    double acc = 0.0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) acc += x[i] + y[i];
    out[t] = acc;
  }
}

}  // namespace mc
