"""GPU parity of Zinc with NTT-domain errors: zinc_nbasis_create /
ckks_encode_ntt / zinc_encrypt_ntt (called through the C ABI) against the
oracle's nttrand module on the same seeded inputs.

Pre-encoded plaintexts and ciphertext residues must be bit-exact.  Decoded
slots must lie within sqrt(K) times the tolerance of the other Zinc tests
(each error coefficient is a sum of K chi values).
"""
import functools

import numpy as np
import pytest

from oracle import ckks as O
from oracle import encoder as OE
from oracle import nttrand as ON
from oracle import ring as OR
from paper_2408_07304_gb300 import api, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIGMA = 3.2


def tol(log_n, ld, K):
    n = 1 << log_n
    return (10 * n * SIGMA * np.sqrt(K) + n) / 2.0 ** ld


@functools.lru_cache(maxsize=None)
def gpu_model(log_n, bits, ld, K, kseed=1, cseed=2, bseed=3):
    from paper_2408_07304_gb300 import build
    build.build()
    ctx = api.Context(log_n, bits, ld, device=0)
    sk, pk = api.ckks_keygen(ctx, kseed)
    zc = api.zinc_precompute(ctx, pk, cseed)
    nb = api.zinc_nbasis_create(ctx, K, bseed)
    return ctx, sk, pk, zc, nb


@functools.lru_cache(maxsize=None)
def oracle_model(log_n, bits, ld, K, kseed=1, cseed=2, bseed=3):
    P = O.Params(log_n, bits, ld)
    Kk = O.keygen(P, kseed)
    zero = O.zinc_precompute_coeff(P, Kk, cseed)
    return P, Kk, zero, ON.basis(P.n, K, bseed)


def dev(a, dtype):
    return torch.tensor(np.asarray(a), dtype=dtype, device="cuda:0")


SMALL = [(10, (40, 40, 41), 30, 500, 1), (10, (50, 60), 30, 512, 4), (12, (36, 36, 36), 30, 2048, 16),
         (13, (60, 40), 40, 100, 2)]


@pytest.mark.parametrize("log_n,bits,ld,n_slots,K", SMALL)
def test_zinc_ntt_bit_exact_full(log_n, bits, ld, n_slots, K):
    ctx, sk, pk, zc, nb = gpu_model(log_n, bits, ld, K)
    P, Kk, zero, E = oracle_model(log_n, bits, ld, K)
    z = workloads.slots(workloads.small(log_n, bits, ld, 3, n_slots, seed=9))
    m_hat = api.ckks_encode_ntt(ctx, dev(z, torch.float64))
    api.zn_sync_status(ctx)
    got_m = api.as_u64(m_hat)
    idx = np.array([0, 7, 2 ** 40 + 3], dtype=np.int64)
    ct = api.zinc_encrypt_ntt(ctx, zc, nb, m_hat, 5, dev(idx, torch.int64))
    g = api.as_u64(ct)
    for b in range(3):
        m = OE.encode(z[b], log_n, ld)
        for i, (q, psi) in enumerate(zip(P.primes, P.psis)):
            assert np.array_equal(got_m[b, i], OR.ntt(np.mod(m, q).astype(np.uint64), q, psi)), ("encode", b, i)
        ref = O.ct_ntt(P, ON.zinc_encrypt_coeff(P, zero, E, m, 5, int(idx[b])))
        assert np.array_equal(g[b], ref), ("zinc ntt", b)
    back = api.ckks_decrypt_decode(ctx, sk, ct, n_slots).cpu().numpy()
    assert np.max(np.abs(back - z)) < tol(log_n, ld, K)


def test_batch_equals_solo_and_invalid_arguments():
    log_n, bits, ld, K = 12, (36, 36, 36), 30, 4
    ctx, sk, pk, zc, nb = gpu_model(log_n, bits, ld, K)
    z = dev(np.random.default_rng(1).uniform(-1, 1, (4, 300)), torch.float64)
    m_hat = api.ckks_encode_ntt(ctx, z)
    idx = dev([5, 1, 2 ** 33, 2], torch.int64)
    full = api.zinc_encrypt_ntt(ctx, zc, nb, m_hat, 11, idx)
    for b in (3, 0):
        one = api.zinc_encrypt_ntt(ctx, zc, nb, m_hat[b:b + 1].contiguous(), 11, idx[b:b + 1])
        assert torch.equal(one[0], full[b])
    for K_bad in (0, 17):
        with pytest.raises(api.ZincError):
            api.zinc_nbasis_create(ctx, K_bad, 1)
    other = api.Context(log_n, (36, 36, 37), ld, device=0)
    with pytest.raises(api.ZincError):                       # basis of another context
        api.zinc_encrypt_ntt(other, api.zinc_precompute(other, api.ckks_keygen(other, 1)[1], 2), nb,
                             torch.zeros((1, 3, 1 << log_n), dtype=torch.int64, device="cuda:0"), 0,
                             idx[:1])
    small = api.Context(9, (40,), 20, device=0)
    with pytest.raises(api.ZincError):                       # rings below 2^10
        api.zinc_nbasis_create(small, 2, 1)


@pytest.mark.parametrize("name,K", [("throughput", 4), ("large", 2)])
def test_full_size_sampled(name, K):
    """The benchmark's configuration: the whole batch in one call."""
    w = workloads.WORKLOADS[name]
    ctx, sk, pk, zc, nb = gpu_model(w.log_n, w.bits, w.log2_delta, K, workloads.KEYGEN_SEED, workloads.CACHE_SEED,
                                    workloads.NBASIS_SEED)
    P, Kk, zero, E = oracle_model(w.log_n, w.bits, w.log2_delta, K, workloads.KEYGEN_SEED, workloads.CACHE_SEED,
                                  workloads.NBASIS_SEED)
    z = workloads.slots(w)
    m_hat = api.ckks_encode_ntt(ctx, dev(z, torch.float64))
    idx = np.arange(w.batch, dtype=np.int64)
    ct = api.zinc_encrypt_ntt(ctx, zc, nb, m_hat, w.seed, dev(idx, torch.int64))
    api.zn_sync_status(ctx)
    got = api.as_u64(ct)
    rng = np.random.default_rng(5)
    for b in (0, w.batch - 1):
        m = OE.encode(z[b], w.log_n, w.log2_delta)
        oct_ = ON.zinc_encrypt_coeff(P, zero, E, m, w.seed, b)
        pos = [(p, i, int(k)) for p in (0, 1) for i in (0, w.L // 2, w.L - 1)
               for k in np.concatenate([[0, w.n - 1], rng.integers(0, w.n, 4)])]
        ref = O.ct_ntt_sampled(P, oct_, pos)
        assert np.array_equal(np.array([got[b, p, i, k] for p, i, k in pos], dtype=np.uint64), ref), b
    lim = tol(w.log_n, w.log2_delta, K) * max(abs(w.lo), abs(w.hi))
    for b0 in range(0, w.batch, 256):
        back = api.ckks_decrypt_decode(ctx, sk, ct[b0:b0 + 256].contiguous(), w.n_slots).cpu().numpy()
        assert np.max(np.abs(back - z[b0:b0 + 256])) < lim
