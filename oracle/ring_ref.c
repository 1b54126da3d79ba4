/*
 * Definitional ring arithmetic for the oracle.  TEST INFRASTRUCTURE ONLY: only
 * tests, the smoke check and the CPU-baseline leg of the benchmark load this
 * library; the GPU library never does.
 *
 * Everything here is the plain definition, evaluated term by term:
 *
 *   NTT (the RNS "DFT" of Section "Theoretical Analysis", negacyclic form):
 *       ahat[i] = sum_j a_j * psi^((2 brv(i) + 1) j)  mod q
 *     i.e. evaluation of a(X) at the odd powers of psi, listed in bit-reversed
 *     order of the exponent; psi is a primitive 2N-th root of unity mod q.
 *   inverse:
 *       a_j = N^-1 sum_i ahat[i] * psi^(-(2 brv(i) + 1) j)  mod q
 *   negacyclic (schoolbook) product in Z_q[X]/(X^N + 1):
 *       c_k = sum_{i+j=k} a_i b_j - sum_{i+j=k+N} a_i b_j  mod q
 *
 * Exponents are reduced modulo 2N (psi has order 2N) and looked up in a table
 * of psi^t, t < 2N.  Products use exact 128-bit integers.
 */
#include <stdint.h>
#include <stdlib.h>

typedef unsigned __int128 u128;
typedef __int128 i128;

static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t q) {
  return (uint64_t)(((u128)a * b) % q);
}

static uint64_t powmod(uint64_t b, uint64_t e, uint64_t q) {
  uint64_t r = 1 % q;
  b %= q;
  while (e) {
    if (e & 1) r = mulmod(r, b, q);
    b = mulmod(b, b, q);
    e >>= 1;
  }
  return r;
}

static uint32_t brv(uint32_t x, int bits) {
  uint32_t r = 0;
  for (int i = 0; i < bits; i++) { r = (r << 1) | (x & 1); x >>= 1; }
  return r;
}

static int log2u(uint32_t n) { int l = 0; while ((1u << l) < n) l++; return l; }

/* table[t] = base^t mod q for t < 2n */
static uint64_t* power_table(uint64_t base, uint32_t n, uint64_t q) {
  uint64_t* t = (uint64_t*)malloc(sizeof(uint64_t) * 2 * (size_t)n);
  t[0] = 1 % q;
  for (uint32_t i = 1; i < 2 * n; i++) t[i] = mulmod(t[i - 1], base, q);
  return t;
}

/* ahat[idx[t]] for each requested output index (out[t]). */
int oracle_ntt_eval(const uint64_t* a, uint32_t n, uint64_t q, uint64_t psi,
                    const uint32_t* idx, uint32_t n_idx, uint64_t* out) {
  int logn = log2u(n);
  uint64_t* pw = power_table(psi, n, q);
  if (!pw) return 1;
  uint64_t mask = 2ull * n - 1;          /* reduction mod 2N (a power of two) */
#pragma omp parallel for schedule(dynamic, 8)
  for (long t = 0; t < (long)n_idx; t++) {
    uint64_t e = 2ull * brv(idx[t], logn) + 1;
    uint64_t acc = 0;
    for (uint32_t j = 0; j < n; j++) {
      acc += mulmod(a[j], pw[(e * j) & mask], q);
      if (acc >= q) acc -= q;
    }
    out[t] = acc;
  }
  free(pw);
  return 0;
}

/* Full forward transform: every output index. */
int oracle_ntt(const uint64_t* a, uint32_t n, uint64_t q, uint64_t psi, uint64_t* out) {
  uint32_t* idx = (uint32_t*)malloc(sizeof(uint32_t) * n);
  if (!idx) return 1;
  for (uint32_t i = 0; i < n; i++) idx[i] = i;
  int r = oracle_ntt_eval(a, n, q, psi, idx, n, out);
  free(idx);
  return r;
}

/* Inverse transform (all coefficients). */
int oracle_intt(const uint64_t* ahat, uint32_t n, uint64_t q, uint64_t psi, uint64_t* out) {
  int logn = log2u(n);
  uint64_t psi_inv = powmod(psi, 2ull * n - 1, q);        /* psi^-1 = psi^(2N-1) */
  uint64_t n_inv = powmod(n % q, q - 2, q);               /* q prime */
  uint64_t* pw = power_table(psi_inv, n, q);
  if (!pw) return 1;
  uint64_t mask = 2ull * n - 1;          /* reduction mod 2N (a power of two) */
#pragma omp parallel for schedule(dynamic, 8)
  for (long j = 0; j < (long)n; j++) {
    uint64_t acc = 0;
    for (uint32_t i = 0; i < n; i++) {
      uint64_t e = ((2ull * brv(i, logn) + 1) * (uint64_t)j) & mask;
      acc += mulmod(ahat[i], pw[e], q);
      if (acc >= q) acc -= q;
    }
    out[j] = mulmod(acc, n_inv, q);
  }
  free(pw);
  return 0;
}

/* c = a * b in Z_q[X]/(X^N+1), a residues in [0, q), b small signed integers
 * (|b_j| < 2^40); the sums are exact in 128-bit integers, reduced at the end. */
int oracle_negacyclic_mul_small(const uint64_t* a, const int64_t* b, uint32_t n,
                                uint64_t q, uint64_t* c) {
#pragma omp parallel for schedule(static)
  for (long k = 0; k < (long)n; k++) {
    i128 acc = 0;
    for (uint32_t i = 0; i < n; i++) {
      long j = k - (long)i;
      if (j >= 0) acc += (i128)a[i] * b[j];
      else acc -= (i128)a[i] * b[j + n];
    }
    i128 r = acc % (i128)q;
    if (r < 0) r += q;
    c[k] = (uint64_t)r;
  }
  return 0;
}

/* c = a * b in Z_q[X]/(X^N+1), both operands residues in [0, q). */
int oracle_negacyclic_mul(const uint64_t* a, const uint64_t* b, uint32_t n,
                          uint64_t q, uint64_t* c) {
#pragma omp parallel for schedule(static)
  for (long k = 0; k < (long)n; k++) {
    uint64_t pos = 0, neg = 0;
    for (uint32_t i = 0; i < n; i++) {
      long j = k - (long)i;
      if (j >= 0) { pos += mulmod(a[i], b[j], q); if (pos >= q) pos -= q; }
      else        { neg += mulmod(a[i], b[j + n], q); if (neg >= q) neg -= q; }
    }
    c[k] = pos >= neg ? pos - neg : pos + (q - neg);
  }
  return 0;
}

/* Threads the OpenMP runtime would use (1 without OpenMP). */
int oracle_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}
