// Host-side parameter tables: prime chain, roots, NTT twiddles, encoder
// twiddles and the chi (rounded Gaussian) thresholds.
//
// Compiled with -ffp-contract=off: the double-double arithmetic below relies
// on every product and sum being rounded separately, identically on x86-64
// and aarch64 hosts.
#include "zn_host.h"

#include <cmath>
#include <cstring>

namespace zn {

typedef unsigned __int128 u128;

static inline u64 mulmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }

u64 powmod(u64 b, u64 e, u64 q) {
  u64 r = 1 % q;
  b %= q;
  while (e) {
    if (e & 1) r = mulmod(r, b, q);
    b = mulmod(b, b, q);
    e >>= 1;
  }
  return r;
}

// Deterministic Miller-Rabin: the first 12 prime bases decide every n < 3.3e24.
bool is_prime(u64 n) {
  static const u64 bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  if (n < 2) return false;
  for (u64 p : bases)
    if (n % p == 0) return n == p;
  u64 d = n - 1;
  int s = 0;
  while ((d & 1) == 0) { d >>= 1; ++s; }
  for (u64 a : bases) {
    u64 x = powmod(a, d, n);
    if (x == 1 || x == n - 1) continue;
    bool composite = true;
    for (int r = 1; r < s; ++r) {
      x = mulmod(x, x, n);
      if (x == n - 1) { composite = false; break; }
    }
    if (composite) return false;
  }
  return true;
}

// For each bit size b: the largest prime q < 2^b with q = 1 (mod 2N) that is
// not already in the chain.
int gen_primes(uint32_t log_n, const uint32_t* bits, uint32_t count, u64* out) {
  const u64 two_n = 2ull << log_n;
  for (uint32_t i = 0; i < count; ++i) {
    u64 top = (bits[i] >= 64) ? ~0ull : ((1ull << bits[i]) - 2);
    u64 q = (top / two_n) * two_n + 1;
    bool found = false;
    for (; q > two_n; q -= two_n) {
      bool used = false;
      for (uint32_t k = 0; k < i; ++k) used |= (out[k] == q);
      if (!used && is_prime(q)) { found = true; break; }
    }
    if (!found) return -1;
    out[i] = q;
  }
  return 0;
}

// The smallest primitive 2N-th root of unity mod q.
u64 find_psi(u64 q, uint32_t log_n) {
  const u64 n = 1ull << log_n, two_n = 2 * n;
  u64 psi0 = 0;
  for (u64 g = 2;; ++g) {
    psi0 = powmod(g, (q - 1) / two_n, q);
    if (powmod(psi0, n, q) == q - 1) break;
  }
  u64 best = psi0, step = mulmod(psi0, psi0, q), x = psi0;
  for (u64 k = 1; k < n; ++k) {
    x = mulmod(x, step, q);
    if (x < best) best = x;
  }
  return best;
}

static inline uint32_t brv(uint32_t x, uint32_t bits) {
  uint32_t r = 0;
  for (uint32_t i = 0; i < bits; ++i) { r = (r << 1) | (x & 1); x >>= 1; }
  return r;
}

u64 shoup(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }

// tw[k] = psi^brv(k), itw[k] = psi^-brv(k) (k < N), with Shoup companions.
void ntt_tables(u64 q, u64 psi, uint32_t log_n, u64* tw, u64* tws, u64* itw, u64* itws) {
  const uint32_t n = 1u << log_n;
  const u64 psi_inv = powmod(psi, 2ull * n - 1, q);
  u64 p = 1, pi = 1;
  // powers in natural order, then scattered to bit-reversed positions
  for (uint32_t k = 0; k < n; ++k) {
    uint32_t r = brv(k, log_n);
    tw[r] = p;
    itw[r] = pi;
    p = mulmod(p, psi, q);
    pi = mulmod(pi, psi_inv, q);
  }
  for (uint32_t k = 0; k < n; ++k) {
    tws[k] = shoup(tw[k], q);
    itws[k] = shoup(itw[k], q);
  }
}

// ------------------------------------------------------------ double-double
struct dd { double hi, lo; };

static inline dd two_sum(double a, double b) {
  double s = a + b, bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
static inline dd quick_two_sum(double a, double b) {
  double s = a + b;
  return {s, b - (s - a)};
}
static inline dd two_prod(double a, double b) {
  double p = a * b;
  return {p, std::fma(a, b, -p)};
}
static inline dd dd_add(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi), t = two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = quick_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return quick_two_sum(s.hi, s.lo);
}
static inline dd dd_neg(dd a) { return {-a.hi, -a.lo}; }
static inline dd dd_mul(dd a, dd b) {
  dd p = two_prod(a.hi, b.hi);
  p.lo += a.hi * b.lo + a.lo * b.hi;
  return quick_two_sum(p.hi, p.lo);
}
static inline dd dd_mul_d(dd a, double b) {
  dd p = two_prod(a.hi, b);
  p.lo += a.lo * b;
  return quick_two_sum(p.hi, p.lo);
}
static inline dd dd_div(dd a, dd b) {
  double q1 = a.hi / b.hi;
  dd r = dd_add(a, dd_neg(dd_mul_d(b, q1)));
  double q2 = r.hi / b.hi;
  r = dd_add(r, dd_neg(dd_mul_d(b, q2)));
  double q3 = r.hi / b.hi;
  return dd_add(quick_two_sum(q1, q2), dd{q3, 0.0});
}
static inline dd dd_div_d(dd a, double b) { return dd_div(a, dd{b, 0.0}); }
static inline double dd_abs_hi(dd a) { return std::fabs(a.hi); }

// pi to double-double precision (hi = nearest double, lo = pi - hi rounded)
static const dd kPi = {3.141592653589793116e+00, 1.224646799147353207e-16};

// sin and cos of x in [0, pi/4] by Taylor series in double-double
static void dd_sincos(dd x, dd* s_out, dd* c_out) {
  dd x2 = dd_mul(x, x);
  dd term_s = x, sum_s = x;
  dd term_c = {1.0, 0.0}, sum_c = {1.0, 0.0};
  for (int n = 1; n < 40; ++n) {
    term_c = dd_div_d(dd_mul(term_c, x2), (double)((2 * n - 1) * (2 * n)));
    term_s = dd_div_d(dd_mul(term_s, x2), (double)((2 * n) * (2 * n + 1)));
    if (n & 1) {
      sum_c = dd_add(sum_c, dd_neg(term_c));
      sum_s = dd_add(sum_s, dd_neg(term_s));
    } else {
      sum_c = dd_add(sum_c, term_c);
      sum_s = dd_add(sum_s, term_s);
    }
    if (dd_abs_hi(term_c) < 1e-40 && dd_abs_hi(term_s) < 1e-40) break;
  }
  *s_out = sum_s;
  *c_out = sum_c;
}

// T[k] = cos(pi k/N) - i sin(pi k/N), k < N.  Angles are reduced to [0, pi/4]
// by exact symmetries in the integer k; each part is the double nearest the
// double-double value (correct rounding except within ~2^-100 of a tie).
int encoder_twiddles(uint32_t log_n, double* re, double* im) {
  const uint32_t n = 1u << log_n, quarter = n / 4;
  // (cos, sin) of pi k / N for k in [0, N/4]
  double* cs = new double[2 * (quarter + 1)];
  for (uint32_t k = 0; k <= quarter; ++k) {
    if (k == 0) { cs[0] = 1.0; cs[1] = 0.0; continue; }
    dd th = dd_mul_d(kPi, (double)k);
    th = {th.hi / n, th.lo / n};            // exact: n is a power of two
    dd s, c;
    dd_sincos(th, &s, &c);
    cs[2 * k] = c.hi;
    cs[2 * k + 1] = s.hi;
  }
  for (uint32_t k = 0; k < n; ++k) {
    double c, s;
    if (k <= quarter) {
      c = cs[2 * k]; s = cs[2 * k + 1];
    } else if (k <= n / 2) {                 // pi/2 - x
      uint32_t j = n / 2 - k; c = cs[2 * j + 1]; s = cs[2 * j];
    } else if (k <= 3 * quarter) {           // pi/2 + x
      uint32_t j = k - n / 2; c = -cs[2 * j + 1]; s = cs[2 * j];
    } else {                                 // pi - x
      uint32_t j = n - k; c = -cs[2 * j]; s = cs[2 * j + 1];
    }
    re[k] = c;
    im[k] = -s;
  }
  delete[] cs;
  return 0;
}

// floor(2^62 x + 1/2) for a double-double x in [0, 1]: hi * 2^62 and
// lo * 2^62 are exact; the integer part of the first is exact, and the
// fractional remainder plus the second decides the rounding (correct except
// within ~2^-40 of a tie).
static int64_t q62_of(dd x) {
  const double a = std::ldexp(x.hi, 62), b = std::ldexp(x.lo, 62);
  const double ai = std::floor(a);
  const double f = (a - ai) + b;
  return (int64_t)ai + (int64_t)std::floor(f + 0.5);
}

// C[k] = floor(2^62 cos(pi k/N) + 1/2), S[k] = floor(2^62 sin(pi k/N) + 1/2),
// k < N, with the same exact angle reductions as encoder_twiddles.
int encoder_twiddles_q62(uint32_t log_n, int64_t* c_out, int64_t* s_out) {
  const uint32_t n = 1u << log_n, quarter = n / 4;
  int64_t* cs = new int64_t[2 * (quarter + 1)];
  for (uint32_t k = 0; k <= quarter; ++k) {
    if (k == 0) { cs[0] = (int64_t)1 << 62; cs[1] = 0; continue; }
    dd th = dd_mul_d(kPi, (double)k);
    th = {th.hi / n, th.lo / n};
    dd s, c;
    dd_sincos(th, &s, &c);
    cs[2 * k] = q62_of(c);
    cs[2 * k + 1] = q62_of(s);
  }
  for (uint32_t k = 0; k < n; ++k) {
    int64_t c, s;
    if (k <= quarter) {
      c = cs[2 * k]; s = cs[2 * k + 1];
    } else if (k <= n / 2) {
      uint32_t j = n / 2 - k; c = cs[2 * j + 1]; s = cs[2 * j];
    } else if (k <= 3 * quarter) {
      uint32_t j = k - n / 2; c = -cs[2 * j + 1]; s = cs[2 * j];
    } else {
      uint32_t j = n - k; c = -cs[2 * j]; s = cs[2 * j + 1];
    }
    c_out[k] = c;
    s_out[k] = s;
  }
  delete[] cs;
  return 0;
}

// sum_n (-1)^n x^(2n+1) / (n! (2n+1)) = erf(x) sqrt(pi)/2, double-double
static dd erf_core(dd x) {
  dd x2 = dd_mul(x, x);
  dd term = x, sum = {0.0, 0.0};
  for (int n = 0; n < 400; ++n) {
    dd c = dd_div_d(term, (double)(2 * n + 1));
    sum = (n & 1) ? dd_add(sum, dd_neg(c)) : dd_add(sum, c);
    term = dd_div_d(dd_mul(term, x2), (double)(n + 1));
    if (n > 5 && dd_abs_hi(term) < 1e-40) break;
  }
  return sum;
}

static dd dd_sqrt2() {
  double s = std::sqrt(2.0);
  dd r = dd_add(dd{2.0, 0.0}, dd_neg(two_prod(s, s)));
  return quick_two_sum(s, r.hi / (2.0 * s));
}

// floor of a non-negative double-double below 2^64
static u64 dd_floor_u64(dd v) {
  double f = std::floor(v.hi);
  double frac = (v.hi - f) + v.lo;           // v.hi - f is exact
  double adj = std::floor(frac);
  return (u64)f + (u64)(int64_t)adj;
}

// chi thresholds: T_j = floor(2^64 F(j - 20)), j = 1..38, F the CDF of the
// normal (sigma = 16/5) rounded to integers and truncated to [-19, 19]:
// F(v) = (E(a_v) + E(A)) / (2 E(A)), a_v = (v + 1/2)/(sigma sqrt 2),
// A = 19.5/(sigma sqrt 2), E the erf series above (its constant cancels).
int cdt_thresholds(u64 out[38]) {
  const dd r2 = dd_sqrt2();
  // 1 / (2 sigma sqrt 2) = 5 / (32 sqrt 2)
  const dd k = dd_div(dd{5.0, 0.0}, dd_mul_d(r2, 32.0));
  const dd big = erf_core(dd_mul_d(k, 39.0));
  const dd den = dd_mul_d(big, 2.0);
  for (int v = -19; v < 19; ++v) {
    dd a = dd_mul_d(k, (double)(2 * v + 1));
    dd f = dd_div(dd_add(erf_core(a), big), den);
    dd scaled = {f.hi * 18446744073709551616.0, f.lo * 18446744073709551616.0};
    out[v + 19] = dd_floor_u64(scaled);
  }
  return 0;
}

}  // namespace zn
