"""Pins for the oracle's NTT-domain Zinc randomiser (oracle/nttrand.py): the
rotation against the schoolbook product by the monomial X^r (C library) and
its closed forms, the NTT-domain form of a rotation (the pointwise factor
psi^{(2 brv(i) + 1) r}) against the definitional NTT, the uniformity of the
rotations, the size and variance of the error, and the exact decryption
identity of the resulting Zinc ciphertexts.
"""
import numpy as np
import pytest

from oracle import ckks, encoder, nttrand, numtheory, ring


def _small_conv(a, b, n):
    """Exact negacyclic product of small integer vectors via numpy.convolve (library)."""
    full = np.convolve(np.asarray(a, dtype=np.int64), np.asarray(b, dtype=np.int64))
    full = np.concatenate([full, np.zeros(2 * n - full.size, dtype=np.int64)])
    return full[:n] - full[n:]


def _monomial(n, r, q):
    """X^r mod (X^N + 1) as residues (schoolbook input)."""
    m = np.zeros(n, dtype=np.int64)
    m[r % n] = 1 if r < n else -1
    return m


@pytest.mark.parametrize("n", [16, 64])
def test_rotate_is_the_monomial_product(n):
    q = numtheory.gen_primes(int(np.log2(n)), (40,))[0]
    rng = np.random.default_rng(n)
    e = rng.integers(-19, 20, n)
    for r in [0, 1, n - 1, n, n + 3, 2 * n - 1] + list(rng.integers(0, 2 * n, 6)):
        got = np.mod(nttrand.rotate(e, int(r)), q).astype(np.uint64)
        ref = ring.negacyclic_mul_small(np.mod(e, q).astype(np.uint64), _monomial(n, int(r), q), q)
        assert np.array_equal(got, ref), r


def test_rotate_closed_forms():
    n = 32
    e = np.arange(1, n + 1, dtype=np.int64)
    assert np.array_equal(nttrand.rotate(e, 0), e)
    assert np.array_equal(nttrand.rotate(e, n), -e)
    one = np.zeros(n, dtype=np.int64)
    one[0] = 1
    x = nttrand.rotate(one, 1)
    assert x[1] == 1 and x.sum() == 1
    top = np.zeros(n, dtype=np.int64)
    top[n - 1] = 1
    assert np.array_equal(nttrand.rotate(top, 1), -one)          # X^(N-1) X = -1
    for a, b in [(3, 5), (n - 1, n + 2), (2 * n - 1, 1)]:
        assert np.array_equal(nttrand.rotate(nttrand.rotate(e, a), b), nttrand.rotate(e, (a + b) % (2 * n)))


@pytest.mark.parametrize("log_n,bits", [(4, (30,)), (6, (50,)), (10, (60,))])
def test_rotation_in_ntt_form_is_a_pointwise_factor(log_n, bits):
    # NTT(X^r e)[i] = psi^((2 brv(i) + 1) r) NTT(e)[i]: the form the GPU evaluates
    n = 1 << log_n
    q = numtheory.gen_primes(log_n, bits)[0]
    psi = numtheory.find_psi(q, log_n)
    rng = np.random.default_rng(log_n)
    e = rng.integers(-19, 20, n)
    eh = ring.ntt(np.mod(e, q).astype(np.uint64), q, psi)
    for r in [0, 1, n, 2 * n - 1, int(rng.integers(0, 2 * n))]:
        rot = ring.ntt(np.mod(nttrand.rotate(e, r), q).astype(np.uint64), q, psi)
        for i in range(n):
            a = 2 * numtheory.brv(i, log_n) + 1
            assert int(rot[i]) == int(eh[i]) * pow(psi, (a * r) % (2 * n), q) % q, (r, i)


def test_rotations_uniform_and_independent():
    n, K = 1024, 4
    rs = np.array([nttrand.rotations(n, K, 9, ct) for ct in range(600)])   # [600][2][K]
    assert rs.min() >= 0 and rs.max() < 2 * n
    # chi-square over 16 bins of the 4800 draws
    hist = np.bincount((rs.reshape(-1) * 16) // (2 * n), minlength=16)
    exp = rs.size / 16
    assert ((hist - exp) ** 2 / exp).sum() < 45
    assert not np.array_equal(rs[:, 0], rs[:, 1])
    assert nttrand.rotations(n, K, 9, 5) == nttrand.rotations(n, K, 9, 5)


def test_error_size_and_variance():
    n, K = 4096, 4
    E = nttrand.basis(n, K, 3)
    errs = np.concatenate([nttrand.error(E[0], nttrand.rotations(n, K, 3, ct)[0]) for ct in range(8)])
    assert np.max(np.abs(errs)) <= 19 * K
    var = errs.var()
    assert abs(var - K * (3.2 ** 2 + 1 / 12)) < 0.15 * K * 10.3


@pytest.mark.parametrize("K", [1, 4])
def test_zinc_ntt_decryption_identity(K):
    # Dec(c') = Dec(zero) + m + e'_0 + e'_1 s, exactly
    P = ckks.Params(6, (40, 40, 41), 20)
    Kk = ckks.keygen(P, 11)
    zero = ckks.zinc_precompute_coeff(P, Kk, 2)
    E = nttrand.basis(P.n, K, 7)
    z = np.random.default_rng(4).uniform(-1, 1, 20)
    m = encoder.encode(z, P.log_n, P.log2_delta)
    ct = nttrand.zinc_encrypt_coeff(P, zero, E, m, seed=5, ct_index=3)
    dz = ckks.crt_centered(P, ckks.decrypt_coeff(P, Kk, zero.c0, zero.c1), P.n_primes)
    dc = ckks.crt_centered(P, ckks.decrypt_coeff(P, Kk, ct.c0, ct.c1), P.n_primes)
    e = ct.e1p + _small_conv(ct.e2p, Kk.s, P.n)
    assert [dc[k] - dz[k] for k in range(P.n)] == [int(m[k]) + int(e[k]) for k in range(P.n)]
    r = nttrand.rotations(P.n, K, 5, 3)
    assert np.array_equal(ct.e1p, nttrand.error(E[0], r[0])) and np.array_equal(ct.e2p, nttrand.error(E[1], r[1]))
