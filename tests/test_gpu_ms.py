"""GPU parity of the modulus-switched (SEAL-ordered) vanilla encryption and of
Zinc over its cache: ckks_encrypt_ms / zinc_precompute_ms (called through the
C ABI) against the oracle's encrypt_ms_coeff / zinc_precompute_ms_coeff on the
same seeded inputs.

Ciphertext residues must be bit-exact.  Decoded slots must lie within the
tolerance of the plain encryption's tests, (10 N sigma + N) / Delta: the
modulus-switched noise is smaller (|v/p| + the rounding term, at most
(N + 1)/2 + 1 per coefficient) and Zinc adds e1' + e2' s on top of it.
Small rings are compared in full; the full-size workloads (whole batch in one
call, as the benchmark times it) on sampled outputs.
"""
import functools

import numpy as np
import pytest

from oracle import ckks as O
from paper_2408_07304_gb300 import api, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIGMA = 3.2


def tol(log_n, ld):
    n = 1 << log_n
    return (10 * n * SIGMA + n) / 2.0 ** ld


@functools.lru_cache(maxsize=None)
def gpu_ctx(log_n, bits, ld):
    from paper_2408_07304_gb300 import build
    build.build()
    return api.Context(log_n, bits, ld, device=0)


@functools.lru_cache(maxsize=None)
def gpu_model(log_n, bits, ld, kseed, cseed):
    """Key-level context and key, data-level context, secret key and cache there."""
    ctx = gpu_ctx(log_n, bits, ld)
    dctx = gpu_ctx(log_n, bits[:-1], ld)
    sk, pk = api.ckks_keygen(ctx, kseed)
    sk_d = api.zn_sk_import(dctx, api.zn_sk_export(sk))
    zc = api.zinc_precompute_ms(ctx, pk, cseed, dctx)
    return ctx, dctx, pk, sk_d, zc


@functools.lru_cache(maxsize=None)
def oracle_model(log_n, bits, ld, kseed, cseed):
    P = O.Params(log_n, bits, ld)
    K = O.keygen(P, kseed)
    Pd = O.data_params(P)
    zero = O.zinc_precompute_ms_coeff(P, K, cseed)
    return P, K, Pd, zero


def dev(a, dtype):
    return torch.tensor(np.asarray(a), dtype=dtype, device="cuda:0")


# N = 2^15 runs the four-CTA cluster kernels (a relaxed and a Harvey data prime)
SMALL = [(4, (30, 40), 20, 8), (6, (40, 41, 50), 25, 20), (10, (40, 40, 41), 30, 500),
         (12, (36, 36, 36), 30, 2048), (13, (60, 40, 60), 40, 100), (14, (50, 60, 60), 50, 8192),
         (15, (55, 60, 60), 55, 16384)]


@pytest.mark.parametrize("log_n,bits,ld,n_slots", SMALL)
def test_ms_bit_exact_full(log_n, bits, ld, n_slots):
    ctx, dctx, pk, sk_d, zc = gpu_model(log_n, bits, ld, 1, 2)
    P, K, Pd, zero = oracle_model(log_n, bits, ld, 1, 2)
    assert dctx.primes == Pd.primes == ctx.primes[:-1]
    assert np.array_equal(api.zn_zcache_export(zc), O.ct_ntt(Pd, zero))
    B, seed = 3, 6
    z = workloads.slots(workloads.small(log_n, bits, ld, B, n_slots, seed=9))
    idx = np.array([0, 7, 2 ** 40 + 3], dtype=np.int64)
    ct_m = api.ckks_encrypt_ms(ctx, pk, dev(z, torch.float64), seed, dev(idx, torch.int64))
    ct_z = api.zinc_encrypt(dctx, zc, dev(z, torch.float64), seed, dev(idx, torch.int64))
    api.zn_sync_status(ctx)
    api.zn_sync_status(dctx)
    assert tuple(ct_m.shape) == (B, 2, len(bits) - 1, 1 << log_n)
    gm, gz = api.as_u64(ct_m), api.as_u64(ct_z)
    for b in range(B):
        ref_m = O.ct_ntt(Pd, O.encrypt_ms_coeff(P, K, z[b], seed, int(idx[b])))
        ref_z = O.ct_ntt(Pd, O.zinc_encrypt_coeff(Pd, zero, z[b], seed, int(idx[b])))
        assert np.array_equal(gm[b], ref_m), ("modulus-switched", b)
        assert np.array_equal(gz[b], ref_z), ("zinc", b)
    for ct in (ct_m, ct_z):
        back = api.ckks_decrypt_decode(dctx, sk_d, ct, n_slots).cpu().numpy()
        assert np.max(np.abs(back - z)) < tol(log_n, ld)


def test_ms_zero_message_and_batch_equals_solo():
    log_n, bits, ld = 10, (40, 40, 41), 30
    ctx, dctx, pk, sk_d, _ = gpu_model(log_n, bits, ld, 1, 2)
    P, K, Pd, _ = oracle_model(log_n, bits, ld, 1, 2)
    idx = np.array([5, 1, 2 ** 33, 9], dtype=np.int64)
    c0 = api.ckks_encrypt_ms(ctx, pk, dev(np.zeros((4, 0)), torch.float64), 4, dev(idx, torch.int64))
    ref = O.ct_ntt(Pd, O.encrypt_ms_coeff(P, K, None, 4, 2 ** 33))
    assert np.array_equal(api.as_u64(c0)[2], ref)
    back = api.ckks_decrypt_decode(dctx, sk_d, c0, 16).cpu().numpy()
    assert np.max(np.abs(back)) < tol(log_n, ld)
    z = workloads.slots(workloads.small(log_n, bits, ld, 4, 300, seed=3))
    full = api.as_u64(api.ckks_encrypt_ms(ctx, pk, dev(z, torch.float64), 11, dev(idx, torch.int64)))
    for b in (3, 0):
        one = api.ckks_encrypt_ms(ctx, pk, dev(z[b:b + 1], torch.float64), 11, dev(idx[b:b + 1], torch.int64))
        assert np.array_equal(api.as_u64(one)[0], full[b])


def test_ms_invalid_arguments():
    ctx1 = gpu_ctx(10, (40,), 30)
    _, pk1 = api.ckks_keygen(ctx1, 1)
    z = dev(np.zeros((1, 4)), torch.float64)
    i0 = dev(np.array([0]), torch.int64)
    with pytest.raises(api.ZincError) as e:                      # no special prime
        api.ckks_encrypt_ms(ctx1, pk1, z, 0, i0, out=torch.empty((1, 2, 0, 1024), dtype=torch.int64,
                                                                  device="cuda:0"))
    assert e.value.status == api.ZN_EINVAL
    ctx, dctx, pk, _, _ = gpu_model(10, (40, 40, 41), 30, 1, 2)
    wrong = gpu_ctx(10, (40, 41), 30)                             # second prime differs
    for bad in (wrong, gpu_ctx(10, (40, 40), 31), ctx):
        with pytest.raises(api.ZincError) as e:
            api.zinc_precompute_ms(ctx, pk, 2, bad)
        assert e.value.status == api.ZN_EINVAL
    with pytest.raises(api.ZincError):                            # key of another context
        api.ckks_encrypt_ms(dctx, pk, z, 0, i0)
    empty = torch.empty((0, 2, 2, 1024), dtype=torch.int64, device="cuda:0")
    api.ckks_encrypt_ms(ctx, pk, dev(np.zeros((0, 4)), torch.float64), 0,
                        torch.empty((0,), dtype=torch.int64, device="cuda:0"), out=empty)


def test_ms_imported_key_equals_generated():
    log_n, bits, ld = 12, (36, 36, 36), 30
    ctx, _, pk, _, _ = gpu_model(log_n, bits, ld, 1, 2)
    pk2 = api.zn_pk_import(ctx, api.zn_pk_export(pk))
    z = dev(np.random.default_rng(1).uniform(-1, 1, (2, 100)), torch.float64)
    idx = dev(np.array([1, 2]), torch.int64)
    assert torch.equal(api.ckks_encrypt_ms(ctx, pk, z, 3, idx), api.ckks_encrypt_ms(ctx, pk2, z, 3, idx))


def _check_sampled(w, ct, zinc, z, idx, rows):
    P, K, Pd, zero = oracle_model(w.log_n, w.bits, w.log2_delta, workloads.KEYGEN_SEED, workloads.CACHE_SEED)
    Ld = w.L - 1
    rng = np.random.default_rng(321)
    got = api.as_u64(ct)
    for b in rows:
        if zinc:
            oct_ = O.zinc_encrypt_coeff(Pd, zero, z[b], w.seed, int(idx[b]))
        else:
            oct_ = O.encrypt_ms_coeff(P, K, z[b], w.seed, int(idx[b]))
        pos = [(p, i, int(k)) for p in (0, 1) for i in (0, Ld // 2, Ld - 1)
               for k in np.concatenate([[0, w.n - 1], rng.integers(0, w.n, 4)])]
        ref = O.ct_ntt_sampled(Pd, oct_, pos)
        assert np.array_equal(np.array([got[b, p, i, k] for p, i, k in pos], dtype=np.uint64), ref), (b, zinc)


@pytest.mark.parametrize("name", ["throughput", "large"])
def test_ms_full_size_sampled(name):
    """Whole batch in one call, as the benchmark's special-prime leg times it."""
    w = workloads.WORKLOADS[name]
    ctx, dctx, pk, sk_d, zc = gpu_model(w.log_n, w.bits, w.log2_delta, workloads.KEYGEN_SEED,
                                        workloads.CACHE_SEED)
    z = workloads.slots(w)
    idx = np.arange(w.batch, dtype=np.int64)
    zd = dev(z, torch.float64)
    ct_m = api.ckks_encrypt_ms(ctx, pk, zd, w.seed, dev(idx, torch.int64))
    ct_z = api.zinc_encrypt(dctx, zc, zd, w.seed, dev(idx, torch.int64))
    api.zn_sync_status(ctx)
    api.zn_sync_status(dctx)
    rows = [0, w.batch - 1, w.batch // 2 + 1]
    _check_sampled(w, ct_m, False, z, idx, rows)
    _check_sampled(w, ct_z, True, z, idx, rows)
    lim = tol(w.log_n, w.log2_delta) * max(abs(w.lo), abs(w.hi))
    for ct in (ct_m, ct_z):
        for b0 in range(0, w.batch, 256):
            back = api.ckks_decrypt_decode(dctx, sk_d, ct[b0:b0 + 256].contiguous(), w.n_slots).cpu().numpy()
            assert np.max(np.abs(back - z[b0:b0 + 256])) < lim


def test_ms_encode_overflow_latched_on_the_key_level_context():
    # an encoded coefficient of 2^62 or more is an overflow: latched, context usable
    bad = gpu_ctx(10, (50, 50, 51), 60)
    _, bpk = api.ckks_keygen(bad, 1)
    api.ckks_encrypt_ms(bad, bpk, dev(np.full((1, 8), 1e6), torch.float64), 0, dev(np.array([0]), torch.int64))
    with pytest.raises(api.ZincError) as e:
        api.zn_sync_status(bad)
    assert e.value.status == api.ZN_EOVERFLOW
    api.zn_sync_status(bad)
    api.ckks_encrypt_ms(bad, bpk, dev(np.zeros((1, 8)), torch.float64), 0, dev(np.array([0]), torch.int64))
    api.zn_sync_status(bad)
