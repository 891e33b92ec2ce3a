/*
 * or_count.hpp -- an operation-counting double for the oracle.
 *
 * TEST AND MEASUREMENT INFRASTRUCTURE ONLY (see oracle.h).  opcount.py
 * compiles the oracle's own C sources as C++ with this header forced in
 * first: after it, the word `double` names or_real, a value type that
 * behaves like a double and counts each floating-point operation it
 * performs -- additions and subtractions, multiplications, divisions,
 * square roots, exponentials, logarithms, sines and cosines, comparisons,
 * minima and maxima -- into the category of the oracle function being run
 * (markers that opcount.py inserts at the top of the functions of the
 * shooting, the plant and its noise, the CD-EKF, the QP subproblem, the
 * NLP evaluation and the SQP).
 * The oracle's arithmetic is unchanged: every operation is the same double
 * operation in the same order; only the counters are added.
 */
#ifndef OR_COUNT_HPP
#define OR_COUNT_HPP

#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>
#include <cmath>

enum { ORC_ADD, ORC_MUL, ORC_DIV, ORC_SQRT, ORC_EXP, ORC_LOG, ORC_SIN, ORC_COS, ORC_CMP,
       ORC_MINMAX, ORC_NKIND };
/* categories: 0 everything else, then the marked functions */
enum { ORC_OTHER, ORC_RK4_INTERVAL, ORC_EM_STEP, ORC_PROCESS_NOISE, ORC_MEAS_NOISE,
       ORC_EKF_PREDICT, ORC_EKF_FILTER, ORC_QP_SOLVE, ORC_EVALUATE, ORC_SQP, ORC_NCAT };

extern "C" {
extern uint64_t orc_ops[ORC_NCAT][ORC_NKIND];
extern uint64_t orc_calls[ORC_NCAT];
}
extern int orc_cat;

struct OrcCat {
  int saved;
  explicit OrcCat(int c) : saved(orc_cat) {
    orc_cat = c;
    orc_calls[c]++;
  }
  ~OrcCat() { orc_cat = saved; }
};

static inline void orc_tick(int kind) { orc_ops[orc_cat][kind]++; }

struct or_real {
  double v;
  or_real() = default;
  constexpr or_real(double x) : v(x) {}
  constexpr or_real(float x) : v(x) {}
  constexpr or_real(int x) : v(x) {}
  constexpr or_real(unsigned x) : v(x) {}
  constexpr or_real(long x) : v((double)x) {}
  constexpr or_real(unsigned long x) : v((double)x) {}
  constexpr or_real(long long x) : v((double)x) {}
  constexpr or_real(unsigned long long x) : v((double)x) {}
  explicit operator int() const { return (int)v; }
  explicit operator long() const { return (long)v; }
  explicit operator long long() const { return (long long)v; }
  explicit operator unsigned() const { return (unsigned)v; }
  or_real& operator+=(or_real o) { orc_tick(ORC_ADD); v += o.v; return *this; }
  or_real& operator-=(or_real o) { orc_tick(ORC_ADD); v -= o.v; return *this; }
  or_real& operator*=(or_real o) { orc_tick(ORC_MUL); v *= o.v; return *this; }
  or_real& operator/=(or_real o) { orc_tick(ORC_DIV); v /= o.v; return *this; }
};

static inline or_real operator+(or_real a, or_real b) { orc_tick(ORC_ADD); return a.v + b.v; }
static inline or_real operator-(or_real a, or_real b) { orc_tick(ORC_ADD); return a.v - b.v; }
static inline or_real operator*(or_real a, or_real b) { orc_tick(ORC_MUL); return a.v * b.v; }
static inline or_real operator/(or_real a, or_real b) { orc_tick(ORC_DIV); return a.v / b.v; }
static inline or_real operator-(or_real a) { return -a.v; }
static inline or_real operator+(or_real a) { return a; }
static inline bool operator<(or_real a, or_real b) { orc_tick(ORC_CMP); return a.v < b.v; }
static inline bool operator>(or_real a, or_real b) { orc_tick(ORC_CMP); return a.v > b.v; }
static inline bool operator<=(or_real a, or_real b) { orc_tick(ORC_CMP); return a.v <= b.v; }
static inline bool operator>=(or_real a, or_real b) { orc_tick(ORC_CMP); return a.v >= b.v; }
static inline bool operator==(or_real a, or_real b) { orc_tick(ORC_CMP); return a.v == b.v; }
static inline bool operator!=(or_real a, or_real b) { orc_tick(ORC_CMP); return a.v != b.v; }
static inline bool operator!(or_real a) { return !a.v; }

static inline or_real exp(or_real a) { orc_tick(ORC_EXP); return ::exp(a.v); }
static inline or_real log(or_real a) { orc_tick(ORC_LOG); return ::log(a.v); }
static inline or_real sqrt(or_real a) { orc_tick(ORC_SQRT); return ::sqrt(a.v); }
static inline or_real sin(or_real a) { orc_tick(ORC_SIN); return ::sin(a.v); }
static inline or_real cos(or_real a) { orc_tick(ORC_COS); return ::cos(a.v); }
static inline or_real fabs(or_real a) { return ::fabs(a.v); }
static inline or_real fmax(or_real a, or_real b) { orc_tick(ORC_MINMAX); return ::fmax(a.v, b.v); }
static inline or_real fmin(or_real a, or_real b) { orc_tick(ORC_MINMAX); return ::fmin(a.v, b.v); }
static inline bool isfinite(or_real a) { return std::isfinite(a.v); }
static inline bool isnan(or_real a) { return std::isnan(a.v); }

static_assert(sizeof(or_real) == sizeof(double), "or_real must have the layout of double");

#define double or_real

#endif
