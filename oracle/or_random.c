/*
 * or_random.c -- counter-based random numbers for the oracle.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The paper runs every Monte Carlo simulation with "different process noise"
 * (Sec. VII-B, VII-C) but does not name its generator.  Both this oracle and
 * the CUDA path implement, each on its own, Philox4x32-10 from its published
 * definition (J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel
 * random numbers: as easy as 1, 2, 3", SC'11), so a trajectory sees the same
 * noise on both sides.
 *
 * Counter layout: ctr = (k, j, tag, 0), key = (seed_lo, seed_hi), where j is
 * the trajectory index and k the global Euler-Maruyama substep (tags 0, 1),
 * the sample index (tag 2) or a parameter slot (tag 3).
 */
#include <math.h>
#include "oracle.h"

/* One Philox round: two 32x32->64 products, the high halves mixed with the
 * other two counter words and the round key. */
static void philox_round(uint32_t c[4], const uint32_t k[2]) {
  const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
  const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
  const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
  const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
  const uint32_t n0 = hi1 ^ c[1] ^ k[0];
  const uint32_t n2 = hi0 ^ c[3] ^ k[1];
  c[0] = n0;
  c[1] = lo1;
  c[2] = n2;
  c[3] = lo0;
}

/* Philox4x32 with 10 rounds; the key is advanced by the Weyl constants
 * (golden ratio and sqrt(3)-1 in 32-bit fixed point) between rounds. */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  uint32_t k[2] = {key[0], key[1]};
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k[0] += 0x9E3779B9u;
      k[1] += 0xBB67AE85u;
    }
    philox_round(c, k);
  }
  for (int i = 0; i < 4; ++i) out[i] = c[i];
}

/* Uniform on the open interval (0, 1) from 52 random bits: the top 26 bits
 * of `hi` and of `lo` form an integer m in [0, 2^52); the value is
 * (m + 1/2) 2^-52, exact in double precision and never 0 or 1. */
double or_uniform52(uint32_t hi, uint32_t lo) {
  const double m = (double)(hi >> 6) * 67108864.0 + (double)(lo >> 6);
  return (m + 0.5) * (1.0 / 4503599627370496.0);
}

/* Box-Muller transform: two independent standard normals from two uniforms. */
void or_normal_pair(const uint32_t w[4], double z[2]) {
  const double u1 = or_uniform52(w[0], w[1]);
  const double u2 = or_uniform52(w[2], w[3]);
  const double rad = sqrt(-2.0 * log(u1));
  const double ang = 2.0 * M_PI * u2;
  z[0] = rad * cos(ang);
  z[1] = rad * sin(ang);
}

static void draw(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t tag, uint32_t w[4]) {
  const uint32_t ctr[4] = {c0, c1, tag, 0u};
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  or_philox4x32_10(ctr, key, w);
}

/* Three standard normals driving d omega on one Euler-Maruyama substep. */
void or_process_noise(uint64_t seed, int64_t j, int64_t substep, double xi[3]) {
  uint32_t w[4];
  double z[2];
  draw(seed, (uint32_t)substep, (uint32_t)j, 0u, w);
  or_normal_pair(w, z);
  xi[0] = z[0];
  xi[1] = z[1];
  draw(seed, (uint32_t)substep, (uint32_t)j, 1u, w);
  or_normal_pair(w, z);
  xi[2] = z[0];
}

/* Standard normal of the measurement noise v(t_i). */
double or_meas_noise(uint64_t seed, int64_t j, int64_t step) {
  uint32_t w[4];
  double z[2];
  draw(seed, (uint32_t)step, (uint32_t)j, 2u, w);
  or_normal_pair(w, z);
  return z[0];
}

/* Per-trajectory parameters: the time and sign of the inlet-temperature step
 * and the lognormal perturbation of the activation energy. */
void or_traj_params(const or_model* m, uint64_t seed, int64_t j, double* EaR_j,
                    double* t_d, double* dTin) {
  uint32_t w[4];
  double z[2];
  draw(seed, 0u, (uint32_t)j, 3u, w);
  const double tf = m->t0 + (double)m->n_steps * m->Ts;
  *t_d = m->t0 + or_uniform52(w[0], w[1]) * (tf - m->t0);
  *dTin = (w[2] & 1u) ? m->dTin_step : -m->dTin_step;
  draw(seed, 1u, (uint32_t)j, 3u, w);
  or_normal_pair(w, z);
  *EaR_j = (m->Ea_logsd != 0.0) ? m->EaR * exp(m->Ea_logsd * z[0]) : m->EaR;
}

/* Uneven batches: the OCP horizon and SQP iteration limit of trajectory j,
 * uniform integers from the first two words of counter (2, j, 3, 0). */
void or_traj_horizon(const or_ctrl* c, uint64_t seed, int64_t j, int* N, int* max_it) {
  uint32_t w[4];
  *N = c->N;
  *max_it = c->sqp_max_it;
  if (c->N_min <= 0 && c->it_min <= 0) return;
  draw(seed, 2u, (uint32_t)j, 3u, w);
  if (c->N_min > 0) *N = c->N_min + (int)(w[0] % (uint32_t)(c->N - c->N_min + 1));
  if (c->it_min > 0)
    *max_it = c->it_min + (int)(w[1] % (uint32_t)(c->sqp_max_it - c->it_min + 1));
}
