"""Pins for the oracle's BFV and BGV encryptions and their Zinc forms
(Section "Scheme Flexibility", Eqs. 12 and 13): exact noise identities in the
style of Theorem 1 with the noise computed by numpy.convolve, decryption by
exact rational arithmetic, the defining inequalities of Delta = floor(Q/t),
the key identity with the scaled error, the CRT against known integers, and
additive homomorphism.  A dropped Delta, a missing factor t, a wrong
component or a transposed key fails one of them.
"""
import numpy as np
import pytest

from oracle import bfvbgv as B
from oracle import ckks, ring

T_VALUES = [2, 257, 65537, (1 << 20) + 7]


def _conv(a, b, n):
    """Exact negacyclic product of small integer vectors (numpy.convolve)."""
    full = np.convolve(np.asarray(a, dtype=np.int64), np.asarray(b, dtype=np.int64))
    full = np.concatenate([full, np.zeros(2 * n - full.size, dtype=np.int64)])
    return full[:n] - full[n:]


@pytest.fixture(scope="module")
def params():
    P = ckks.Params(6, (40, 40, 41), 20)
    K = ckks.keygen(P, 11)
    return P, K


def _msg(n, t, seed):
    # arbitrary integers, including negatives and values >= t (taken mod t)
    rng = np.random.default_rng(seed)
    return rng.integers(-3 * t, 3 * t, n)


def test_delta_definition(params):
    P, _ = params
    Q = B.modulus(P)
    assert Q == P.primes[0] * P.primes[1] * P.primes[2]
    for t in T_VALUES:
        d = B.delta_bfv(P, t)
        assert d * t <= Q < (d + 1) * t


def test_crt_reproduces_known_integers(params):
    P, _ = params
    Q = B.modulus(P)
    rng = np.random.default_rng(1)
    xs = [int(v) for v in rng.integers(0, 2 ** 62, P.n)]
    xs = [(x * 1000003 + 17) % Q for x in xs]
    xs[:3] = [0, 1, Q - 1]
    res = [np.array([x % q for x in xs], dtype=np.uint64) for q in P.primes]
    got, Q2 = B._crt(P, res)
    assert Q2 == Q and got == xs


@pytest.mark.parametrize("t", T_VALUES)
def test_bfv_noise_identity_and_decrypt(params, t):
    # [c0 + c1 s]_Q = Delta m + e u + e0 + e1 s (mod Q), and Dec recovers m mod t
    P, K = params
    Q = B.modulus(P)
    m = _msg(P.n, t, t)
    ct = B.bfv_encrypt_coeff(P, K, m, t, seed=3, ct_index=5)
    v = _conv(K.e, ct.u, P.n) + ct.e0 + _conv(ct.e1, K.s, P.n)
    x, _ = B.dec_poly(P, K, ct.c0, ct.c1)
    d = B.delta_bfv(P, t)
    mt = [int(a) % t for a in m]
    assert all((x[k] - d * mt[k] - int(v[k])) % Q == 0 for k in range(P.n))
    assert B.bfv_decrypt(P, K, ct.c0, ct.c1, t) == mt


@pytest.mark.parametrize("t", T_VALUES)
def test_bfv_zinc_identity_and_decrypt(params, t):
    # Zinc over CKKS's cached zero: noise = zero's noise + e1' + e2' s exactly
    P, K = params
    Q = B.modulus(P)
    zero = ckks.zinc_precompute_coeff(P, K, seed=2)
    m = _msg(P.n, t, t + 1)
    ct = B.bfv_zinc_encrypt_coeff(P, zero, m, t, seed=4, ct_index=9)
    vz = _conv(K.e, zero.u, P.n) + zero.e0 + _conv(zero.e1, K.s, P.n)
    v = vz + ct.e1p + _conv(ct.e2p, K.s, P.n)
    x, _ = B.dec_poly(P, K, ct.c0, ct.c1)
    d = B.delta_bfv(P, t)
    mt = [int(a) % t for a in m]
    assert all((x[k] - d * mt[k] - int(v[k])) % Q == 0 for k in range(P.n))
    assert B.bfv_decrypt(P, K, ct.c0, ct.c1, t) == mt
    # the second component is the cache's plus e2' only
    for i, q in enumerate(P.primes):
        assert np.array_equal(ct.c1[i], ckks._add_small(zero.c1[i], ct.e2p, q))


@pytest.mark.parametrize("t", T_VALUES)
def test_bgv_keygen_identity(params, t):
    # pk0 + pk1 s = t e (mod q), with Gen's own samples
    P, K0 = params
    K = B.bgv_keygen(P, t, 11)
    assert np.array_equal(K.s, K0.s) and np.array_equal(K.e, K0.e)
    for i, q in enumerate(P.primes):
        assert np.array_equal(K.pk1[i], K0.pk1[i])
        lhs = (K.pk0[i].astype(object) + ring.negacyclic_mul_small(K.pk1[i], K.s, q).astype(object)) % q
        assert [int(a) for a in lhs] == [(t * int(e)) % q for e in K.e]


@pytest.mark.parametrize("t", T_VALUES)
def test_bgv_noise_identity_and_decrypt(params, t):
    # [c0 + c1 s]_Q (centred) = m + t (e u + e0 + e1 s) exactly, Dec = m mod t
    P, _ = params
    K = B.bgv_keygen(P, t, 11)
    m = _msg(P.n, t, 2 * t)
    ct = B.bgv_encrypt_coeff(P, K, m, t, seed=3, ct_index=5)
    v = _conv(K.e, ct.u, P.n) + ct.e0 + _conv(ct.e1, K.s, P.n)
    x, _ = B.dec_poly(P, K, ct.c0, ct.c1)
    mt = [int(a) % t for a in m]
    assert x == [mt[k] + t * int(v[k]) for k in range(P.n)]
    assert B.bgv_decrypt(P, K, ct.c0, ct.c1, t) == mt


@pytest.mark.parametrize("t", T_VALUES)
def test_bgv_zinc_identity_and_decrypt(params, t):
    P, _ = params
    K = B.bgv_keygen(P, t, 11)
    zero = B.bgv_zinc_precompute_coeff(P, K, t, seed=2)
    m = _msg(P.n, t, 3 * t)
    ct = B.bgv_zinc_encrypt_coeff(P, zero, m, t, seed=4, ct_index=9)
    vz = _conv(K.e, zero.u, P.n) + zero.e0 + _conv(zero.e1, K.s, P.n)
    v = vz + ct.e1p + _conv(ct.e2p, K.s, P.n)
    x, _ = B.dec_poly(P, K, ct.c0, ct.c1)
    mt = [int(a) % t for a in m]
    assert x == [mt[k] + t * int(v[k]) for k in range(P.n)]
    assert B.bgv_decrypt(P, K, ct.c0, ct.c1, t) == mt
    # the cached zero decrypts to 0 and uses the cache domain, ct_index 0
    assert B.bgv_decrypt(P, K, zero.c0, zero.c1, t) == [0] * P.n
    z2 = B.bgv_encrypt_coeff(P, K, np.zeros(P.n, dtype=np.int64), t, 2, 0, domain=3)
    assert all(np.array_equal(a, b) for a, b in zip(z2.c0, zero.c0))


def test_additive_homomorphism(params):
    P, K = params
    t = 65537
    ma, mb = _msg(P.n, t, 1), _msg(P.n, t, 2)
    ca = B.bfv_encrypt_coeff(P, K, ma, t, 1, 1)
    cb = B.bfv_zinc_encrypt_coeff(P, ckks.zinc_precompute_coeff(P, K, 2), mb, t, 1, 2)
    s0 = [ckks._add(a, b, q) for a, b, q in zip(ca.c0, cb.c0, P.primes)]
    s1 = [ckks._add(a, b, q) for a, b, q in zip(ca.c1, cb.c1, P.primes)]
    assert B.bfv_decrypt(P, K, s0, s1, t) == [(int(a) + int(b)) % t for a, b in zip(ma, mb)]
    Kg = B.bgv_keygen(P, t, 11)
    ga = B.bgv_encrypt_coeff(P, Kg, ma, t, 1, 1)
    gb = B.bgv_zinc_encrypt_coeff(P, B.bgv_zinc_precompute_coeff(P, Kg, t, 2), mb, t, 1, 2)
    s0 = [ckks._add(a, b, q) for a, b, q in zip(ga.c0, gb.c0, P.primes)]
    s1 = [ckks._add(a, b, q) for a, b, q in zip(ga.c1, gb.c1, P.primes)]
    assert B.bgv_decrypt(P, Kg, s0, s1, t) == [(int(a) + int(b)) % t for a, b in zip(ma, mb)]


def test_bfv_and_bgv_share_the_vanilla_randomness(params):
    # same (u, e0, e1) as the CKKS vanilla encryption with the same seed and index
    P, K = params
    a = B.bfv_encrypt_coeff(P, K, np.zeros(P.n, dtype=np.int64), 257, seed=6, ct_index=8)
    b = ckks.encrypt_coeff(P, K, None, seed=6, ct_index=8)
    assert np.array_equal(a.u, b.u) and np.array_equal(a.e0, b.e0) and np.array_equal(a.e1, b.e1)
    # BFV of the zero plaintext is CKKS's encryption of zero
    assert all(np.array_equal(x, y) for x, y in zip(a.c0, b.c0))
