"""RNS-CKKS public-key encryption, vanilla and Zinc, written from the paper.
TEST INFRASTRUCTURE ONLY (see oracle/__init__).

Notation: the paper's ciphertext (c_1, c_2) and public key (pk_1, pk_2) are
called (c0, c1) and (pk0, pk1) here; c0 carries the message.

* Gen (Eq. 7): sk = s <- R_2, a <- R_q, e <- chi; pk0 = -a s + e, pk1 = a.
* Enc (Eq. 8, with the second component read as pk_2 u + e_2, the form the
  proof of Theorem 1 uses): u <- R_2, e0, e1 <- chi;
  c0 = pk0 u + e0 + m, c1 = pk1 u + e1 (mod each q_i).
* Zinc precompute (Section "Precomputation"): one cached Enc(0).
* Enc_z (Algorithm 1, Eq. 9): c = zero + m; e1', e2' <- chi;
  c' = (c0 + e1', c1 + e2').
* Dec (Eq. 10): c0 + c1 s (mod q).
* Modulus-switched vanilla Enc (the paper's SEAL implementation, Sections
  "System Implementation" and "Theoretical Analysis"): the last prime of the
  chain is the special prime p; Enc computes (pk0 u + e0, pk1 u + e1) at the
  key level (every prime), then divides and rounds by p -- for each data
  prime q_i, c'_i = (c_i + h - r) p^-1 mod q_i with h = floor(p/2) and
  r = (c_p + h) mod p, i.e. c' = floor((c + h) / p) mod Q -- and adds m at
  the data level (every prime but p).

Everything is computed in the coefficient domain with schoolbook negacyclic
products; the stored ciphertexts, keys and cache are the NTT images of those
coefficient vectors (SEAL's convention for CKKS), taken by the definitional
transform (all outputs for small N, selected outputs for large N).
"""
from dataclasses import dataclass, field

import numpy as np

from . import encoder, numtheory, ring, sampler
from .sampler import DOM_CACHE, DOM_ENC, DOM_KEYGEN, DOM_ZINC


@dataclass
class Params:
    log_n: int
    bits: tuple
    log2_delta: int
    primes: list = field(default=None)
    psis: list = field(default=None)

    def __post_init__(self):
        self.bits = tuple(self.bits)
        if self.primes is None:
            self.primes = numtheory.gen_primes(self.log_n, self.bits)
        if self.psis is None:
            self.psis = [numtheory.find_psi(q, self.log_n) for q in self.primes]

    @property
    def n(self):
        return 1 << self.log_n

    @property
    def n_primes(self):
        return len(self.primes)


def _res(v, q):
    return ring.to_residues(v, q)


def _add_small(a, v, q):
    """a (residues) + v (small signed ints) mod q."""
    return ((a.astype(object) + np.asarray(v, dtype=np.int64).astype(object)) % q).astype(np.uint64)


def _add(a, b, q):
    return ((a.astype(object) + b.astype(object)) % q).astype(np.uint64)


@dataclass
class Keys:
    s: np.ndarray            # int64 [N], ternary secret
    e: np.ndarray            # int64 [N]
    a: list                  # per prime, residues [N]
    pk0: list                # per prime, coefficient-domain residues
    pk1: list


def keygen(P: Params, seed: int) -> Keys:
    """Gen, Eq. 7, in the coefficient domain."""
    n = P.n
    s = sampler.sample_ternary(n, seed, DOM_KEYGEN, 0, 0)
    e = sampler.sample_gaussian(n, seed, DOM_KEYGEN, 2, 0)
    a, pk0, pk1 = [], [], []
    for i, q in enumerate(P.primes):
        ai = np.array(sampler.sample_uniform_mod(n, q, seed, DOM_KEYGEN, 1, i), dtype=np.uint64)
        a_s = ring.negacyclic_mul_small(ai, s, q)                 # a * s
        neg = ((q - a_s.astype(object)) % q).astype(np.uint64)    # -a * s
        pk0.append(_add_small(neg, e, q))                         # -a s + e
        pk1.append(ai)                                            # a
        a.append(ai)
    return Keys(s=s, e=e, a=a, pk0=pk0, pk1=pk1)


@dataclass
class CoeffCt:
    """A ciphertext in the coefficient domain, plus the randomness used."""
    c0: list
    c1: list
    m: np.ndarray
    u: np.ndarray = None
    e0: np.ndarray = None
    e1: np.ndarray = None


def _enc_with(P, K, m, u, e0, e1):
    c0, c1 = [], []
    for i, q in enumerate(P.primes):
        c0.append(_add_small(ring.negacyclic_mul_small(K.pk0[i], u, q), e0 + m, q))
        c1.append(_add_small(ring.negacyclic_mul_small(K.pk1[i], u, q), e1, q))
    return CoeffCt(c0=c0, c1=c1, m=m, u=u, e0=e0, e1=e1)


def encrypt_coeff(P: Params, K: Keys, z, seed: int, ct_index: int, domain=DOM_ENC) -> CoeffCt:
    """Vanilla Enc, Eq. 8 (second component with pk1), coefficient domain."""
    n = P.n
    m = encoder.encode(z, P.log_n, P.log2_delta) if z is not None else np.zeros(n, dtype=np.int64)
    u = sampler.sample_ternary(n, seed, domain, 0, ct_index)
    e0 = sampler.sample_gaussian(n, seed, domain, 1, ct_index)
    e1 = sampler.sample_gaussian(n, seed, domain, 2, ct_index)
    return _enc_with(P, K, m, u, e0, e1)


def zinc_precompute_coeff(P: Params, K: Keys, seed: int) -> CoeffCt:
    """The cached Enc(0) (Section "Precomputation"): vanilla Enc of the zero
    plaintext with the cache domain tag and ct_index 0."""
    return encrypt_coeff(P, K, None, seed, 0, domain=DOM_CACHE)


@dataclass
class ZincCt:
    c0: list
    c1: list
    m: np.ndarray
    e1p: np.ndarray
    e2p: np.ndarray


def zinc_encrypt_coeff(P: Params, zero: CoeffCt, z, seed: int, ct_index: int) -> ZincCt:
    """Enc_z, Algorithm 1: c = zero + m; e1', e2' <- chi; c' = (c0 + e1', c1 + e2')."""
    n = P.n
    m = encoder.encode(z, P.log_n, P.log2_delta)
    e1p = sampler.sample_gaussian(n, seed, DOM_ZINC, 0, ct_index)
    e2p = sampler.sample_gaussian(n, seed, DOM_ZINC, 1, ct_index)
    c0, c1 = [], []
    for i, q in enumerate(P.primes):
        c = _add_small(zero.c0[i], m, q)              # step 1: zero + m
        c0.append(_add_small(c, e1p, q))              # step 3: c_1 + e_1'
        c1.append(_add_small(zero.c1[i], e2p, q))     #         c_2 + e_2'
    return ZincCt(c0=c0, c1=c1, m=m, e1p=e1p, e2p=e2p)


def to_ntt(P: Params, polys):
    """NTT images (definition) of a per-prime list of coefficient vectors."""
    return [ring.ntt(p, q, psi) for p, q, psi in zip(polys, P.primes, P.psis)]


def ct_ntt(P: Params, ct):
    """Ciphertext as the library lays it out: uint64 [2][L][N], NTT form."""
    return np.stack([np.stack(to_ntt(P, ct.c0)), np.stack(to_ntt(P, ct.c1))])


def ct_ntt_sampled(P: Params, ct, positions):
    """Selected NTT-form residues; positions is a list of (poly, prime, index)."""
    out = []
    for poly, i, k in positions:
        src = ct.c0[i] if poly == 0 else ct.c1[i]
        out.append(int(ring.ntt_eval(src, P.primes[i], P.psis[i], [k])[0]))
    return np.array(out, dtype=np.uint64)


def pk_ntt(P: Params, K: Keys):
    """Public key as the library lays it out: uint64 [2][L][N], NTT form."""
    return np.stack([np.stack(to_ntt(P, K.pk0)), np.stack(to_ntt(P, K.pk1))])


def data_params(P: Params) -> Params:
    """The data level of a key-level chain: every prime but the last (the special prime)."""
    return Params(P.log_n, P.bits[:-1], P.log2_delta, primes=list(P.primes[:-1]), psis=list(P.psis[:-1]))


def mod_switch_coeff(P: Params, polys):
    """Divide and round by the special prime p = P.primes[-1]: per data prime
    q_i, (c_i + h - r) p^-1 mod q_i with h = floor(p/2), r = (c_p + h) mod p
    (coefficient domain, a per-prime list of residue vectors in, data-level list out)."""
    p = P.primes[-1]
    h = p // 2
    r = (polys[-1].astype(object) + h) % p
    out = []
    for i, q in enumerate(P.primes[:-1]):
        pinv = pow(p, -1, q)
        out.append((((polys[i].astype(object) + h - r) % q) * pinv % q).astype(np.uint64))
    return out


def encrypt_ms_coeff(P: Params, K: Keys, z, seed: int, ct_index: int, domain=DOM_ENC) -> CoeffCt:
    """Modulus-switched vanilla Enc: (pk0 u + e0, pk1 u + e1) at the key level,
    divided and rounded by the special prime, then + m at the data level.  The
    randomness (u, e0, e1) is that of encrypt_coeff with the same arguments."""
    n = P.n
    m = encoder.encode(z, P.log_n, P.log2_delta) if z is not None else np.zeros(n, dtype=np.int64)
    u = sampler.sample_ternary(n, seed, domain, 0, ct_index)
    e0 = sampler.sample_gaussian(n, seed, domain, 1, ct_index)
    e1 = sampler.sample_gaussian(n, seed, domain, 2, ct_index)
    zero = np.zeros(n, dtype=np.int64)
    key_level = _enc_with(P, K, zero, u, e0, e1)          # pk u + e at every prime
    c0 = mod_switch_coeff(P, key_level.c0)
    c1 = mod_switch_coeff(P, key_level.c1)
    Pd = data_params(P)
    c0 = [_add_small(c, m, q) for c, q in zip(c0, Pd.primes)]
    return CoeffCt(c0=c0, c1=c1, m=m, u=u, e0=e0, e1=e1)


def zinc_precompute_ms_coeff(P: Params, K: Keys, seed: int) -> CoeffCt:
    """The cached Enc(0) at the data level, made by modulus-switched Enc (cache domain, ct_index 0)."""
    return encrypt_ms_coeff(P, K, None, seed, 0, domain=DOM_CACHE)


def decrypt_coeff(P: Params, K: Keys, c0, c1):
    """Dec, Eq. 10: c0 + c1 s mod each q_i (coefficient domain)."""
    return [_add(c0[i], ring.negacyclic_mul_small(c1[i], K.s, q), q)
            for i, q in enumerate(P.primes)]


def crt_centered(P: Params, residues, n_use=2):
    """Centered integer coefficients from the first n_use primes (CRT)."""
    qs = P.primes[:n_use]
    Q = 1
    for q in qs:
        Q *= q
    out = []
    for k in range(P.n):
        x = 0
        for q, r in zip(qs, residues[:n_use]):
            Mi = Q // q
            x += int(r[k]) * Mi * pow(Mi, -1, q)
        x %= Q
        if x > Q // 2:
            x -= Q
        out.append(x)
    return out


def decrypt_decode(P: Params, K: Keys, c0, c1, n_slots):
    d = decrypt_coeff(P, K, c0, c1)
    m = crt_centered(P, d, min(2, P.n_primes))
    return encoder.decode(m, P.log_n, P.log2_delta, n_slots)
