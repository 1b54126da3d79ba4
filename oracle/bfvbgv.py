"""BFV and BGV public-key encryption with their Zinc forms (Section "Scheme
Flexibility", Eqs. 12 and 13), written from the paper.
TEST INFRASTRUCTURE ONLY (see oracle/__init__).

Plaintext space R_t = Z_t[X]/(X^N + 1), t << q; a plaintext is given by its
N coefficients, taken mod t (coefficient encoding; the paper leaves the
plaintext encoding to the schemes' own papers).  Q = q_0 ... q_{L-1} is the
whole chain; the second ciphertext component uses pk_2 (read as in Eq. 8).

* BFV (Eq. 12): Delta = floor(Q/t);
    c0 = pk0 u + e0 + Delta m,  c1 = pk1 u + e1   under Gen's key (Eq. 7).
  Zinc: the cached zero is CKKS's (a vanilla encryption of 0, sampling
  domain 3), and Enc_z(m) = (z0 + Delta m + e1', z1 + e2') ("we may use the
  Zinc without modification").
  Dec: m = round(t [c0 + c1 s]_Q / Q) mod t.
* BGV (Eq. 13): the errors carry the factor t, also in the key:
    pk0 = -a s + t e, pk1 = a;   c0 = pk0 u + t e0 + m,  c1 = pk1 u + t e1.
  Zinc: the cached zero is a BGV encryption of 0 (domain 3), and
  Enc_z(m) = (z0 + m + t e1', z1 + t e2').
  Dec: m = ([c0 + c1 s]_Q centred) mod t.

Randomness: the CKKS samplers with the same tags (Gen domain 2; vanilla
domain 0: u poly 0, e0 poly 1, e1 poly 2; Zinc domain 1: e1' poly 0, e2'
poly 1; cache domain 3).  Everything is computed in the coefficient domain
with schoolbook products; ciphertexts are compared in NTT form through
ckks.ct_ntt / ckks.ct_ntt_sampled.
"""
import numpy as np

from . import ring, sampler
from .ckks import CoeffCt, Keys, ZincCt, _add, _add_small
from .sampler import DOM_CACHE, DOM_ENC, DOM_KEYGEN, DOM_ZINC


def modulus(P):
    Q = 1
    for q in P.primes:
        Q *= q
    return Q


def delta_bfv(P, t):
    """Delta = floor(Q / t) (Eq. 12)."""
    return modulus(P) // t


def plaintext(m, t):
    """Coefficients taken mod t, as Python ints in [0, t)."""
    return [int(x) % t for x in m]


def _add_big(res, vals, q):
    """Residues + arbitrary Python integers, mod q."""
    return np.array([(int(r) + int(v)) % q for r, v in zip(res, vals)], dtype=np.uint64)


def _scaled(v, f):
    return [int(x) * f for x in v]


# --------------------------------------------------------------------- BFV
def bfv_encrypt_coeff(P, K: Keys, m, t, seed, ct_index, domain=DOM_ENC) -> CoeffCt:
    """Eq. 12: c0 = pk0 u + e0 + Delta m, c1 = pk1 u + e1 (mod each q_i)."""
    n = P.n
    mt = plaintext(m, t)
    dm = _scaled(mt, delta_bfv(P, t))
    u = sampler.sample_ternary(n, seed, domain, 0, ct_index)
    e0 = sampler.sample_gaussian(n, seed, domain, 1, ct_index)
    e1 = sampler.sample_gaussian(n, seed, domain, 2, ct_index)
    c0, c1 = [], []
    for i, q in enumerate(P.primes):
        a0 = _add_small(ring.negacyclic_mul_small(K.pk0[i], u, q), e0, q)
        c0.append(_add_big(a0, dm, q))
        c1.append(_add_small(ring.negacyclic_mul_small(K.pk1[i], u, q), e1, q))
    return CoeffCt(c0=c0, c1=c1, m=np.array(mt, dtype=object), u=u, e0=e0, e1=e1)


def bfv_zinc_encrypt_coeff(P, zero: CoeffCt, m, t, seed, ct_index) -> ZincCt:
    """Algorithm 1 on BFV: c = zero + Delta m; e1', e2' <- chi; (c0 + e1', c1 + e2')."""
    n = P.n
    mt = plaintext(m, t)
    dm = _scaled(mt, delta_bfv(P, t))
    e1p = sampler.sample_gaussian(n, seed, DOM_ZINC, 0, ct_index)
    e2p = sampler.sample_gaussian(n, seed, DOM_ZINC, 1, ct_index)
    c0, c1 = [], []
    for i, q in enumerate(P.primes):
        c = _add_big(zero.c0[i], dm, q)
        c0.append(_add_small(c, e1p, q))
        c1.append(_add_small(zero.c1[i], e2p, q))
    return ZincCt(c0=c0, c1=c1, m=np.array(mt, dtype=object), e1p=e1p, e2p=e2p)


def _crt(P, residues):
    """Per coefficient, the integer in [0, Q) with the given residues."""
    Q = modulus(P)
    coef = []
    for q in P.primes:
        Mi = Q // q
        coef.append(Mi * pow(Mi, -1, q))
    out = []
    for k in range(P.n):
        out.append(sum(int(r[k]) * c for r, c in zip(residues, coef)) % Q)
    return out, Q


def dec_poly(P, K: Keys, c0, c1):
    """[c0 + c1 s]_Q per coefficient, centred in [-Q/2, Q/2) (Eq. 10 over Q)."""
    res = [_add(c0[i], ring.negacyclic_mul_small(c1[i], K.s, q), q) for i, q in enumerate(P.primes)]
    xs, Q = _crt(P, res)
    return [x - Q if 2 * x >= Q else x for x in xs], Q


def bfv_decrypt(P, K: Keys, c0, c1, t):
    """m = round(t x / Q) mod t, x = [c0 + c1 s]_Q; round half up, exact rationals."""
    xs, Q = dec_poly(P, K, c0, c1)
    return [((2 * t * x + Q) // (2 * Q)) % t for x in xs]


# --------------------------------------------------------------------- BGV
def bgv_keygen(P, t, seed) -> Keys:
    """Gen with the error scaled by t: pk0 = -a s + t e, pk1 = a (same samples as Gen)."""
    n = P.n
    s = sampler.sample_ternary(n, seed, DOM_KEYGEN, 0, 0)
    e = sampler.sample_gaussian(n, seed, DOM_KEYGEN, 2, 0)
    te = [int(x) * t for x in e]
    a, pk0, pk1 = [], [], []
    for i, q in enumerate(P.primes):
        ai = np.array(sampler.sample_uniform_mod(n, q, seed, DOM_KEYGEN, 1, i), dtype=np.uint64)
        a_s = ring.negacyclic_mul_small(ai, s, q)
        neg = ((q - a_s.astype(object)) % q).astype(np.uint64)
        pk0.append(_add_big(neg, te, q))
        pk1.append(ai)
        a.append(ai)
    return Keys(s=s, e=e, a=a, pk0=pk0, pk1=pk1)


def bgv_encrypt_coeff(P, K: Keys, m, t, seed, ct_index, domain=DOM_ENC) -> CoeffCt:
    """Eq. 13: c0 = pk0 u + t e0 + m, c1 = pk1 u + t e1 (mod each q_i)."""
    n = P.n
    mt = plaintext(m, t)
    u = sampler.sample_ternary(n, seed, domain, 0, ct_index)
    e0 = sampler.sample_gaussian(n, seed, domain, 1, ct_index)
    e1 = sampler.sample_gaussian(n, seed, domain, 2, ct_index)
    m0 = [int(e) * t + v for e, v in zip(e0, mt)]
    te1 = _scaled(e1, t)
    c0, c1 = [], []
    for i, q in enumerate(P.primes):
        c0.append(_add_big(ring.negacyclic_mul_small(K.pk0[i], u, q), m0, q))
        c1.append(_add_big(ring.negacyclic_mul_small(K.pk1[i], u, q), te1, q))
    return CoeffCt(c0=c0, c1=c1, m=np.array(mt, dtype=object), u=u, e0=e0, e1=e1)


def bgv_zinc_precompute_coeff(P, K: Keys, t, seed) -> CoeffCt:
    """The cached zero of BGV Zinc: a BGV encryption of 0, cache domain, ct_index 0."""
    return bgv_encrypt_coeff(P, K, np.zeros(P.n, dtype=np.int64), t, seed, 0, domain=DOM_CACHE)


def bgv_zinc_encrypt_coeff(P, zero: CoeffCt, m, t, seed, ct_index) -> ZincCt:
    """Algorithm 1 on BGV with the scaled errors: (z0 + m + t e1', z1 + t e2')."""
    n = P.n
    mt = plaintext(m, t)
    e1p = sampler.sample_gaussian(n, seed, DOM_ZINC, 0, ct_index)
    e2p = sampler.sample_gaussian(n, seed, DOM_ZINC, 1, ct_index)
    m0 = [int(e) * t + v for e, v in zip(e1p, mt)]
    te2 = _scaled(e2p, t)
    c0 = [_add_big(zero.c0[i], m0, q) for i, q in enumerate(P.primes)]
    c1 = [_add_big(zero.c1[i], te2, q) for i, q in enumerate(P.primes)]
    return ZincCt(c0=c0, c1=c1, m=np.array(mt, dtype=object), e1p=e1p, e2p=e2p)


def bgv_decrypt(P, K: Keys, c0, c1, t):
    """m = ([c0 + c1 s]_Q centred) mod t."""
    xs, _ = dec_poly(P, K, c0, c1)
    return [x % t for x in xs]


# ------------------------------------------------------- batching (slots)
# Plaintext slots for BFV / BGV (a reading; the paper defers encoding to the
# schemes' papers): for a prime t = 1 mod 2N with psi_t its minimal primitive
# 2N-th root, R_t is isomorphic to Z_t^N by evaluation at the odd powers of
# psi_t.  Slot s < N/2 is the value at psi_t^(5^s mod 2N), slot N/2 + s the
# value at psi_t^(-5^s mod 2N) (the slot order of the CKKS encoder, both
# conjugate halves).

def slot_exponents(log_n):
    """a_s with slot s <-> evaluation at psi_t^(a_s)."""
    n = 1 << log_n
    out, g = [], 1
    for _ in range(n // 2):
        out.append(g)
        g = g * 5 % (2 * n)
    return out + [(2 * n - a) % (2 * n) for a in out]


def batch_encode(slots, t, log_n):
    """The m in R_t with m(psi_t^(a_s)) = slots[s] mod t (coefficients in [0, t))."""
    from . import numtheory
    n = 1 << log_n
    psi = numtheory.find_psi(t, log_n)
    # the definitional NTT evaluates at psi^(2 brv(i) + 1): place slot s at
    # the output index i with 2 brv(i) + 1 = a_s
    y = np.zeros(n, dtype=np.uint64)
    for s, a in enumerate(slot_exponents(log_n)):
        y[numtheory.brv((a - 1) // 2, log_n)] = int(slots[s]) % t
    return [int(v) for v in ring.intt(y, t, psi)]


def batch_decode(m, t, log_n):
    """slots[s] = m(psi_t^(a_s)) mod t."""
    from . import numtheory
    psi = numtheory.find_psi(t, log_n)
    y = ring.ntt(np.array([int(v) % t for v in m], dtype=np.uint64), t, psi)
    return [int(y[numtheory.brv((a - 1) // 2, log_n)]) for a in slot_exponents(log_n)]
