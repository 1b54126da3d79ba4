"""Zinc with its error polynomials generated in the NTT domain -- the
further optimisation the paper's Conclusion names: generating the randomised
error polynomials directly in the Fourier space, so that Zinc's encryption
needs no transform and becomes O(N).  TEST INFRASTRUCTURE ONLY (see
oracle/__init__).

The paper gives no construction; this module implements the following
reading (a change of the error distribution, with no security claim):

* a basis of K cached error polynomials per ciphertext component,
  E_{c,j} <- chi (c in {0, 1}, j < K), sampled once with the basis seed
  (domain 4, poly 16 c + j, ct_index 0) and kept in NTT form;
* per ciphertext, for each (c, j), a uniform rotation r_{c,j} in [0, 2N)
  (domain 5, poly c, Philox block j, word 0, low log2(2N) bits);
* e'_c = sum_j X^{r_{c,j}} E_{c,j} in Z[X]/(X^N + 1)  (X^N = -1, so
  r >= N also flips the sign) -- every coefficient is a sum of K values of
  chi, variance K sigma^2;
* Enc_z over a pre-encoded plaintext (the paper's Construction assumes m is
  already encoded): c = zero + m; c' = (c0 + e'_0, c1 + e'_1).

In the NTT domain X^r is the pointwise factor psi^{(2 brv(i) + 1) r} at
output i, so e'_c is K pointwise products and additions per coefficient.
This module computes everything in the coefficient domain (rotations by
index shifting) and is compared in NTT form through ckks.ct_ntt.
"""
import numpy as np

from . import sampler
from .ckks import ZincCt, _add_small
from .philox import philox4x32_10

DOM_NBASIS = 4      # the cached basis E_{c,j}
DOM_NROT = 5        # the per-ciphertext rotations r_{c,j}
MAX_K = 16


def basis(n, K, seed):
    """E[c][j] (int64 [N]) for c in {0, 1}, j < K."""
    if not 1 <= K <= MAX_K:
        raise ValueError("K must be in [1, 16]")
    return [[sampler.sample_gaussian(n, seed, DOM_NBASIS, 16 * c + j, 0) for j in range(K)] for c in range(2)]


def rotations(n, K, seed, ct_index):
    """r[c][j] uniform in [0, 2N): word 0 of Philox block j, tag (domain 5, poly c)."""
    out = []
    for c in range(2):
        w = philox4x32_10(np.arange(K, dtype=np.uint64), (DOM_NROT << 24) | (c << 16), ct_index & 0xFFFFFFFF,
                          ct_index >> 32, seed & 0xFFFFFFFF, seed >> 32)
        out.append([int(x) & (2 * n - 1) for x in w[0]])
    return out


def rotate(e, r):
    """X^r e(X) in Z[X]/(X^N + 1), 0 <= r < 2N (coefficient index shift with sign)."""
    n = len(e)
    out = np.zeros(n, dtype=np.int64)
    for k in range(n):
        d = k + r
        sign = 1
        while d >= n:
            d -= n
            sign = -sign
        out[d] += sign * int(e[k])
    return out


def error(E_c, r_c):
    """e'_c = sum_j X^{r_j} E_{c,j}."""
    acc = np.zeros(len(E_c[0]), dtype=np.int64)
    for e, r in zip(E_c, r_c):
        acc += rotate(e, r)
    return acc


def zinc_encrypt_coeff(P, zero, E, m, seed, ct_index) -> ZincCt:
    """Enc_z with NTT-domain errors: (zero_0 + m + e'_0, zero_1 + e'_1), m the
    encoded message (int64 coefficients), E the basis of `basis`."""
    n = P.n
    K = len(E[0])
    r = rotations(n, K, seed, ct_index)
    e0, e1 = error(E[0], r[0]), error(E[1], r[1])
    m = np.asarray(m, dtype=np.int64)
    c0 = [_add_small(zero.c0[i], m + e0, q) for i, q in enumerate(P.primes)]
    c1 = [_add_small(zero.c1[i], e1, q) for i, q in enumerate(P.primes)]
    return ZincCt(c0=c0, c1=c1, m=m, e1p=e0, e2p=e1)
