"""Samplers for R_2, chi and R_q (Section "Polynomials and Distributions").
TEST INFRASTRUCTURE ONLY (see oracle/__init__).

Readings (the paper only names the distributions):

* chi: the continuous normal N(0, sigma^2), sigma = 3.2, rounded to the nearest
  integer and truncated to [-19, 19] (6 sigma = 19.2), renormalised.  Sampled
  by inversion of its CDF ("CDT"): with 38 thresholds
  T_j = floor(2^64 * F(j - 20)), j = 1..38, and a 64-bit uniform U the sample
  is -19 + #{j : U >= T_j}.
* R_2: t = floor(3 * w / 2^32) for a 32-bit uniform word w; the coefficient
  is t - 1 (bias at most 2^-32).
* R_q (per RNS prime q_i): a 128-bit uniform W gives floor(W * q_i / 2^128).

Counter layout for Philox4x32-10: key = (lo32(seed), hi32(seed)); counter =
(block, domain << 24 | poly << 16 | prime, lo32(ct_index), hi32(ct_index)).
Domains: 0 vanilla Enc (u, e0, e1), 1 Zinc randomiser (e1', e2'),
2 Gen (s, a, e), 3 Zinc cache Enc(0) (u, e0, e1).  Coefficient placement
(one Philox block feeds coefficients N/4 or N/2 apart):
* ternary: block b in [0, N/4), word w -> coefficient b + w N/4;
* chi:     block b in [0, N/2), words (0,1) -> b, words (2,3) -> b + N/2,
           U = word_hi * 2^32 + word_lo;
* R_q:     block b in [0, N) -> coefficient b, W = w3:w2:w1:w0.
"""
from decimal import Decimal, getcontext, localcontext
import functools

import numpy as np

from .philox import philox4x32_10

SIGMA_NUM, SIGMA_DEN = 16, 5        # sigma = 3.2 exactly
BOUND = 19                          # truncation |e| <= 19

DOM_ENC, DOM_ZINC, DOM_KEYGEN, DOM_CACHE = 0, 1, 2, 3


def _erf_core(x: Decimal) -> Decimal:
    """sum_n (-1)^n x^(2n+1) / (n! (2n+1)) = erf(x) * sqrt(pi) / 2 (Taylor series)."""
    x2 = x * x
    term = x                       # x^(2n+1)/n!
    total = Decimal(0)
    n = 0
    eps = Decimal(10) ** -(getcontext().prec + 5)
    while True:
        contrib = term / (2 * n + 1)
        total += contrib if n % 2 == 0 else -contrib
        n += 1
        term = term * x2 / n
        if abs(term) < eps and n > 5:
            return total


@functools.lru_cache(maxsize=None)
def cdt_thresholds():
    """The 38 CDT thresholds T_j = floor(2^64 F(j - 20)), j = 1..38, as Python ints."""
    with localcontext() as ctx:
        ctx.prec = 80
        root2 = Decimal(2).sqrt()
        sigma = Decimal(SIGMA_NUM) / Decimal(SIGMA_DEN)

        def arg(v2):               # v2 = 2v+1 -> (v + 1/2) / (sigma sqrt 2)
            return Decimal(v2) / (2 * sigma * root2)

        big = _erf_core(arg(2 * BOUND + 1))
        out = []
        for v in range(-BOUND, BOUND):            # F(-19) .. F(18)
            f = (_erf_core(arg(2 * v + 1)) + big) / (2 * big)
            out.append(int((f * (Decimal(2) ** 64)).to_integral_value(rounding="ROUND_FLOOR")))
    return tuple(out)


def _counter_word1(domain, poly, prime):
    return (domain << 24) | (poly << 16) | prime


def sample_ternary(n, seed, domain, poly, ct_index, prime=0):
    """Coefficients in {-1, 0, 1} (int64 array of length n)."""
    q4 = n // 4
    b = np.arange(q4, dtype=np.uint64)
    w = philox4x32_10(b, _counter_word1(domain, poly, prime), ct_index & 0xFFFFFFFF,
                      ct_index >> 32, seed & 0xFFFFFFFF, seed >> 32)
    out = np.empty(n, dtype=np.int64)
    for j in range(4):
        t = (w[j] * np.uint64(3)) >> np.uint64(32)
        out[j * q4:(j + 1) * q4] = t.astype(np.int64) - 1
    return out


def cdt_lookup(u64):
    """-19 + #{j : U >= T_j} for an array of 64-bit uniforms."""
    u = np.asarray(u64, dtype=np.uint64)
    cnt = np.zeros(u.shape, dtype=np.int64)
    for t in cdt_thresholds():
        cnt += (u >= np.uint64(t))
    return cnt - BOUND


def sample_gaussian(n, seed, domain, poly, ct_index, prime=0):
    """Rounded Gaussian chi (sigma 3.2, |e| <= 19), int64 array of length n."""
    h = n // 2
    b = np.arange(h, dtype=np.uint64)
    w = philox4x32_10(b, _counter_word1(domain, poly, prime), ct_index & 0xFFFFFFFF,
                      ct_index >> 32, seed & 0xFFFFFFFF, seed >> 32)
    u_lo = (w[1] << np.uint64(32)) | w[0]
    u_hi = (w[3] << np.uint64(32)) | w[2]
    return np.concatenate([cdt_lookup(u_lo), cdt_lookup(u_hi)])


def sample_uniform_mod(n, q, seed, domain, poly, prime, ct_index=0):
    """Uniform residues mod q (R_q restricted to one RNS prime), as Python ints in a list."""
    b = np.arange(n, dtype=np.uint64)
    w = philox4x32_10(b, _counter_word1(domain, poly, prime), ct_index & 0xFFFFFFFF,
                      ct_index >> 32, seed & 0xFFFFFFFF, seed >> 32)
    out = []
    for i in range(n):
        W = (int(w[3][i]) << 96) | (int(w[2][i]) << 64) | (int(w[1][i]) << 32) | int(w[0][i])
        out.append((W * q) >> 128)
    return out
