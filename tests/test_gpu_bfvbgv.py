"""GPU parity of the BFV (Eq. 12) and BGV (Eq. 13) encryptions and their Zinc
forms: bfv_encrypt / bfv_zinc_encrypt / bgv_keygen / bgv_zinc_precompute /
bgv_encrypt / bgv_zinc_encrypt (called through the C ABI) against the
oracle's bfvbgv module on the same seeded inputs.

Keys, caches and ciphertext residues must be bit-exact; decryption
(bfv_decrypt / bgv_decrypt, GPU) must return every plaintext coefficient
exactly, and agree with the oracle's exact rational decryption.  Small rings
are compared in full; the full-size workloads on sampled residues with every
ciphertext decrypted.
"""
import functools

import numpy as np
import pytest

from oracle import bfvbgv as OB
from oracle import ckks as O
from paper_2408_07304_gb300 import api, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=None)
def gpu_ctx(log_n, bits, ld=20):
    from paper_2408_07304_gb300 import build
    build.build()
    return api.Context(log_n, bits, ld, device=0)


@functools.lru_cache(maxsize=None)
def gpu_bfv(log_n, bits, kseed=1, cseed=2):
    ctx = gpu_ctx(log_n, bits)
    sk, pk = api.ckks_keygen(ctx, kseed)
    zc = api.zinc_precompute(ctx, pk, cseed)
    return ctx, sk, pk, zc


@functools.lru_cache(maxsize=None)
def gpu_bgv(log_n, bits, t, kseed=1, cseed=2):
    ctx = gpu_ctx(log_n, bits)
    sk, pk = api.bgv_keygen(ctx, t, kseed)
    zc = api.bgv_zinc_precompute(ctx, pk, cseed)
    return ctx, sk, pk, zc


@functools.lru_cache(maxsize=None)
def oracle_bfv(log_n, bits, kseed=1, cseed=2):
    P = O.Params(log_n, bits, 20)
    K = O.keygen(P, kseed)
    return P, K, O.zinc_precompute_coeff(P, K, cseed)


@functools.lru_cache(maxsize=None)
def oracle_bgv(log_n, bits, t, kseed=1, cseed=2):
    P = O.Params(log_n, bits, 20)
    K = OB.bgv_keygen(P, t, kseed)
    return P, K, OB.bgv_zinc_precompute_coeff(P, K, t, cseed)


def dev(a):
    return torch.tensor(np.asarray(a), dtype=torch.int64, device="cuda:0")


def plaintexts(n, t, batch, seed):
    # arbitrary int64 coefficients (negative, >= t): the library takes them mod t
    rng = np.random.default_rng(seed)
    return rng.integers(-4 * t, 4 * t, (batch, n), dtype=np.int64)


# N = 2^15 runs the four-CTA cluster kernels (a relaxed and a Harvey prime)
SMALL = [(10, (40, 40, 41), 65537), (10, (50, 60), 2), (12, (36, 36, 36), 257), (13, (60, 40, 60), (1 << 20) + 7),
         (14, (50, 60), 65537), (15, (55, 60), 65537)]


@pytest.mark.parametrize("log_n,bits,t", SMALL)
def test_bfv_bit_exact_full(log_n, bits, t):
    ctx, sk, pk, zc = gpu_bfv(log_n, bits)
    P, K, zero = oracle_bfv(log_n, bits)
    m = plaintexts(1 << log_n, t, 3, t)
    idx = np.array([0, 7, 2 ** 40 + 3], dtype=np.int64)
    cv = api.bfv_encrypt(ctx, pk, t, dev(m), 5, dev(idx))
    cz = api.bfv_zinc_encrypt(ctx, zc, t, dev(m), 5, dev(idx))
    gv, gz = api.as_u64(cv), api.as_u64(cz)
    for b in range(3):
        rv = OB.bfv_encrypt_coeff(P, K, m[b], t, 5, int(idx[b]))
        rz = OB.bfv_zinc_encrypt_coeff(P, zero, m[b], t, 5, int(idx[b]))
        assert np.array_equal(gv[b], O.ct_ntt(P, rv)), ("bfv", b)
        assert np.array_equal(gz[b], O.ct_ntt(P, rz)), ("bfv zinc", b)
    want = np.mod(m, t)
    for ct in (cv, cz):
        assert np.array_equal(api.bfv_decrypt(ctx, sk, t, ct).cpu().numpy(), want)
    # the GPU decryption agrees with the oracle's exact one on a ciphertext
    assert OB.bfv_decrypt(P, K, rz.c0, rz.c1, t) == want[2].tolist()


@pytest.mark.parametrize("log_n,bits,t", SMALL)
def test_bgv_bit_exact_full(log_n, bits, t):
    ctx, sk, pk, zc = gpu_bgv(log_n, bits, t)
    P, K, zero = oracle_bgv(log_n, bits, t)
    assert np.array_equal(api.zn_pk_export(pk), O.pk_ntt(P, K))
    assert np.array_equal(api.zn_zcache_export(zc), O.ct_ntt(P, zero))
    m = plaintexts(1 << log_n, t, 3, t + 1)
    idx = np.array([3, 0, 2 ** 35], dtype=np.int64)
    cv = api.bgv_encrypt(ctx, pk, dev(m), 6, dev(idx))
    cz = api.bgv_zinc_encrypt(ctx, zc, dev(m), 6, dev(idx))
    gv, gz = api.as_u64(cv), api.as_u64(cz)
    for b in range(3):
        rv = OB.bgv_encrypt_coeff(P, K, m[b], t, 6, int(idx[b]))
        rz = OB.bgv_zinc_encrypt_coeff(P, zero, m[b], t, 6, int(idx[b]))
        assert np.array_equal(gv[b], O.ct_ntt(P, rv)), ("bgv", b)
        assert np.array_equal(gz[b], O.ct_ntt(P, rz)), ("bgv zinc", b)
    want = np.mod(m, t)
    for ct in (cv, cz):
        assert np.array_equal(api.bgv_decrypt(ctx, sk, t, ct).cpu().numpy(), want)
    assert OB.bgv_decrypt(P, K, rv.c0, rv.c1, t) == want[2].tolist()


def test_homomorphic_add_and_batch_equals_solo():
    log_n, bits, t = 12, (36, 36, 36), 65537
    ctx, sk, pk, zc = gpu_bfv(log_n, bits)
    _, gsk, gpk, gzc = gpu_bgv(log_n, bits, t)
    ma, mb = plaintexts(1 << log_n, t, 2, 1)
    idx = dev([4, 9])
    want = np.mod(ma + mb, t)
    a = api.bfv_encrypt(ctx, pk, t, dev(ma[None]), 1, idx[:1])
    b = api.bfv_zinc_encrypt(ctx, zc, t, dev(mb[None]), 1, idx[1:])
    assert np.array_equal(api.bfv_decrypt(ctx, sk, t, api.ckks_add(ctx, a, b)).cpu().numpy()[0], want)
    a = api.bgv_encrypt(ctx, gpk, dev(ma[None]), 1, idx[:1])
    b = api.bgv_zinc_encrypt(ctx, gzc, dev(mb[None]), 1, idx[1:])
    assert np.array_equal(api.bgv_decrypt(ctx, gsk, t, api.ckks_add(ctx, a, b)).cpu().numpy()[0], want)
    m = plaintexts(1 << log_n, t, 4, 3)
    idx = dev([5, 1, 2 ** 33, 2])
    for fn, key in ((lambda *a: api.bfv_encrypt(ctx, pk, t, *a), None),
                    (lambda *a: api.bfv_zinc_encrypt(ctx, zc, t, *a), None),
                    (lambda *a: api.bgv_encrypt(ctx, gpk, *a), None),
                    (lambda *a: api.bgv_zinc_encrypt(ctx, gzc, *a), None)):
        full = fn(dev(m), 7, idx)
        for b in (3, 0):
            assert torch.equal(fn(dev(m[b:b + 1]), 7, idx[b:b + 1])[0], full[b])


def test_invalid_arguments():
    log_n, bits = 10, (40, 40, 41)
    ctx, sk, pk, zc = gpu_bfv(log_n, bits)
    _, gsk, gpk, gzc = gpu_bgv(log_n, bits, 257)
    m = dev(np.zeros((1, 1 << log_n), dtype=np.int64))
    i0 = dev([0])
    for t in (0, 1, ctx.primes[0], (1 << 58) + 1):
        with pytest.raises(api.ZincError) as e:
            api.bfv_encrypt(ctx, pk, t, m, 0, i0)
        assert e.value.status == api.ZN_EINVAL
        with pytest.raises(api.ZincError):
            api.bgv_keygen(ctx, t, 1)
    with pytest.raises(api.ZincError):                 # a BGV key is not Gen's
        api.bfv_encrypt(ctx, gpk, 257, m, 0, i0)
    with pytest.raises(api.ZincError):
        api.ckks_encrypt(ctx, gpk, torch.zeros((1, 4), dtype=torch.float64, device="cuda:0"), 0, i0)
    with pytest.raises(api.ZincError):                 # and Gen's key is not BGV's
        api.bgv_encrypt(ctx, pk, m, 0, i0)
    with pytest.raises(api.ZincError):
        api.bgv_zinc_encrypt(ctx, zc, m, 0, i0)
    with pytest.raises(api.ZincError):
        api.bfv_zinc_encrypt(ctx, gzc, 257, m, 0, i0)
    small = gpu_ctx(9, (40, 41))                       # below 2^10
    _, spk = api.ckks_keygen(small, 1)
    with pytest.raises(api.ZincError):
        api.bfv_encrypt(small, spk, 257, dev(np.zeros((1, 512), dtype=np.int64)), 0, i0)


def _sampled(w, t, got, rows, ref_fn, P):
    rng = np.random.default_rng(77)
    for b in rows:
        oct_ = ref_fn(b)
        pos = [(p, i, int(k)) for p in (0, 1) for i in (0, w.L // 2, w.L - 1)
               for k in np.concatenate([[0, w.n - 1], rng.integers(0, w.n, 3)])]
        ref = O.ct_ntt_sampled(P, oct_, pos)
        assert np.array_equal(np.array([got[b, p, i, k] for p, i, k in pos], dtype=np.uint64), ref), b


@pytest.mark.parametrize("name,t", [("throughput", 65537), ("large", (1 << 40) + 15)])
def test_full_size_sampled_and_decrypted(name, t):
    """Whole batch in one call (the benchmark's BFV/BGV leg); every ciphertext decrypts exactly."""
    w = workloads.WORKLOADS[name]
    B = min(w.batch, 1024)
    m = workloads.int_plaintexts(w, t, batch=B)
    idx = np.arange(B, dtype=np.int64)
    ctx, sk, pk, zc = gpu_bfv(w.log_n, w.bits, workloads.KEYGEN_SEED, workloads.CACHE_SEED)
    _, gsk, gpk, gzc = gpu_bgv(w.log_n, w.bits, t, workloads.KEYGEN_SEED, workloads.CACHE_SEED)
    P, K, zero = oracle_bfv(w.log_n, w.bits, workloads.KEYGEN_SEED, workloads.CACHE_SEED)
    _, KG, zeroG = oracle_bgv(w.log_n, w.bits, t, workloads.KEYGEN_SEED, workloads.CACHE_SEED)
    rows = [0, B - 1]
    want = np.mod(m, t)
    md, idd = dev(m), dev(idx)
    cases = [
        (api.bfv_encrypt(ctx, pk, t, md, w.seed, idd), api.bfv_decrypt,
         lambda b: OB.bfv_encrypt_coeff(P, K, m[b], t, w.seed, b), sk),
        (api.bfv_zinc_encrypt(ctx, zc, t, md, w.seed, idd), api.bfv_decrypt,
         lambda b: OB.bfv_zinc_encrypt_coeff(P, zero, m[b], t, w.seed, b), sk),
        (api.bgv_encrypt(ctx, gpk, md, w.seed, idd), api.bgv_decrypt,
         lambda b: OB.bgv_encrypt_coeff(P, KG, m[b], t, w.seed, b), gsk),
        (api.bgv_zinc_encrypt(ctx, gzc, md, w.seed, idd), api.bgv_decrypt,
         lambda b: OB.bgv_zinc_encrypt_coeff(P, zeroG, m[b], t, w.seed, b), gsk),
    ]
    for ct, dec, ref_fn, key in cases:
        _sampled(w, t, api.as_u64(ct), rows, ref_fn, P)
        assert np.array_equal(dec(ctx, key, t, ct).cpu().numpy(), want)
        del ct
