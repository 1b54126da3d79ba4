"""GPU parity: the sm_103a library (called through its C ABI) against the CPU
oracle on the same seeded inputs.

Integer results (samples, NTT outputs, encoder coefficients, keys and
ciphertext residues) must be bit-exact.  Decoded slots must lie within the
noise tolerance derived from the arithmetic:
    tol(N, Delta) = (10 * N * sigma + N) / Delta,
ten standard deviations of the worst (Zinc) slot error N*sigma*sqrt(2/3*1.5)/Delta
plus the deterministic rounding term N/2/Delta, twice over.
Small rings are compared in full.  The full-size workloads run in the launch
configuration the benchmark times (the whole batch in one call); whole
ciphertexts of them (the first and last of the call, both sides of a chunk
boundary) are compared in full, others on sampled outputs the oracle computes
one by one.
"""
import functools

import numpy as np
import pytest

from oracle import ckks as O
from oracle import encoder as OE
from oracle import ring as OR
from oracle import sampler as OS
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
def gpu_keys(log_n, bits, ld, seed):
    ctx = gpu_ctx(log_n, bits, ld)
    sk, pk = api.ckks_keygen(ctx, seed)
    return sk, pk


@functools.lru_cache(maxsize=None)
def gpu_cache(log_n, bits, ld, kseed, cseed):
    ctx = gpu_ctx(log_n, bits, ld)
    _, pk = gpu_keys(log_n, bits, ld, kseed)
    return api.zinc_precompute(ctx, pk, cseed)


@functools.lru_cache(maxsize=None)
def oracle_model(log_n, bits, ld, kseed, cseed):
    P = O.Params(log_n, bits, ld)
    K = O.keygen(P, kseed)
    zero = O.zinc_precompute_coeff(P, K, cseed)
    return P, K, zero


def dev(a, dtype):
    return torch.tensor(np.asarray(a), dtype=dtype, device="cuda:0")


# ------------------------------------------------------------------ samplers
@pytest.mark.parametrize("log_n,bits", [(4, (30,)), (10, (40, 40)), (14, (60, 50, 50))])
def test_sampler_bit_exact(log_n, bits):
    ctx = gpu_ctx(log_n, bits, 20)
    n = 1 << log_n
    for seed, dom, poly, ct0 in ((0, 0, 0, 0), (12345, 1, 1, 2 ** 33 + 5), (2 ** 63 + 7, 3, 2, 77)):
        t = api.as_u64(api.zn_sample(ctx, api.KIND_TERNARY, seed, dom, poly, 0, ct0, 3)).view(np.int64)
        g = api.as_u64(api.zn_sample(ctx, api.KIND_GAUSSIAN, seed, dom, poly, 0, ct0, 3)).view(np.int64)
        for c in range(3):
            assert np.array_equal(t[c], OS.sample_ternary(n, seed, dom, poly, ct0 + c))
            assert np.array_equal(g[c], OS.sample_gaussian(n, seed, dom, poly, ct0 + c))
        for i, q in enumerate(ctx.primes):
            u = api.as_u64(api.zn_sample(ctx, api.KIND_UNIFORM, seed, 2, 1, i, 0, 1))[0]
            assert u.tolist() == OS.sample_uniform_mod(n, q, seed, 2, 1, i)


# ---------------------------------------------------------------------- NTT
@pytest.mark.parametrize("log_n,bits", [(4, (30, 61)), (6, (50,)), (10, (36, 60)), (12, (36, 36, 36)),
                                        (13, (60, 40))])
def test_ntt_forward_bit_exact(log_n, bits):
    ctx = gpu_ctx(log_n, bits, 20)
    n, L = 1 << log_n, len(bits)
    rng = np.random.default_rng(log_n)
    x = np.stack([np.stack([rng.integers(0, q, n, dtype=np.uint64) for q in ctx.primes]) for _ in range(2)])
    d = dev(x.view(np.int64), torch.int64)
    api.zn_ntt_forward(ctx, d)
    got = api.as_u64(d)
    for b in range(2):
        for i, (q, psi) in enumerate(zip(ctx.primes, ctx.psis)):
            assert np.array_equal(got[b, i], OR.ntt(x[b, i], q, psi)), (b, i)
    api.zn_ntt_inverse(ctx, d)
    assert np.array_equal(api.as_u64(d), x)


@pytest.mark.parametrize("log_n,bits", [(14, (60, 50)), (15, (55, 60))])
def test_ntt_large_sampled(log_n, bits):
    ctx = gpu_ctx(log_n, bits, 20)
    n = 1 << log_n
    rng = np.random.default_rng(log_n)
    x = np.stack([rng.integers(0, q, n, dtype=np.uint64) for q in ctx.primes])[None]
    d = dev(x.view(np.int64), torch.int64)
    api.zn_ntt_forward(ctx, d)
    got = api.as_u64(d)
    idx = np.concatenate([[0, 1, n // 2 - 1, n // 2, n - 1], rng.integers(0, n, 59)]).astype(np.uint32)
    for i, (q, psi) in enumerate(zip(ctx.primes, ctx.psis)):
        assert np.array_equal(got[0, i, idx], OR.ntt_eval(x[0, i], q, psi, idx))
    api.zn_ntt_inverse(ctx, d)
    assert np.array_equal(api.as_u64(d), x)


def test_chi_table_search_boundaries():
    # the lookup of the encryption path (a bucket index over the top 8 bits of
    # U, then the thresholds inside the bucket) equals -19 + #{j : U >= T_j}
    # at every threshold, one below and one above it, at every bucket edge,
    # the extremes and random U
    from oracle import sampler as OS
    ctx = gpu_ctx(10, (50,), 30)
    T = [int(t) for t in OS.cdt_thresholds()]
    us = {0, 1, 2 ** 64 - 1, 2 ** 63}
    for t in T:
        us.update({t - 1, t, t + 1})
    for x in range(1, 256):
        us.update({(x << 56) - 1, x << 56, (x << 56) + 1})
    us = sorted(v for v in us if 0 <= v < 2 ** 64)
    rnd = np.random.default_rng(12).integers(0, 2 ** 63, 5000, dtype=np.uint64) * np.uint64(2) + np.uint64(1)
    u = np.concatenate([np.array(us, dtype=np.uint64), rnd])
    got = api.zn_chi_eval(ctx, torch.tensor(u.view(np.int64), device="cuda:0")).cpu().numpy()
    assert np.array_equal(got, OS.cdt_lookup(u).astype(np.int32))


# ------------------------------------------------------------------ encoder
@pytest.mark.parametrize("log_n,ld,n_slots,lo,hi", [(4, 20, 8, -1, 1), (4, 20, 3, -1, 1), (10, 30, 512, -1, 1),
                                                    (10, 40, 37, -5, 5), (12, 30, 2048, -1, 1),
                                                    (13, 40, 4096, -8, 8), (14, 50, 8192, -1, 1),
                                                    (14, 50, 1000, -1, 1), (15, 55, 16384, -100, 100),
                                                    (12, 30, 0, -1, 1)])
def test_encode_bit_exact(log_n, ld, n_slots, lo, hi):
    ctx = gpu_ctx(log_n, (50,), ld)
    rng = np.random.default_rng(n_slots + log_n)
    z = rng.uniform(lo, hi, (3, n_slots))
    out = api.ckks_encode(ctx, dev(z, torch.float64))
    api.zn_sync_status(ctx)
    got = out.cpu().numpy()
    for b in range(3):
        assert np.array_equal(got[b], OE.encode(z[b], log_n, ld)), b


@pytest.mark.parametrize("z", [np.array([[5e-324, -1e-310, 3e-300, 0.0]]), np.array([[1e9, -1.0, 1e-300, 2.5]]),
                               np.array([[0.0, 0.0, -0.0]]), np.array([[1.0]]), np.array([[-2.0 ** -30] * 7]),
                               np.array([[0.5, -0.5, 0.5, 1.5, -2.5, 3.5, 1e-17, 7.0]])])
def test_encode_edge_inputs_bit_exact(z):
    # subnormal, mixed-magnitude, all-zero, single-slot and tie-prone vectors
    log_n, ld = 10, 30
    ctx = gpu_ctx(log_n, (50,), ld)
    out = api.ckks_encode(ctx, dev(z, torch.float64))
    api.zn_sync_status(ctx)
    assert np.array_equal(out.cpu().numpy()[0], OE.encode(z[0], log_n, ld))


def test_encode_non_finite_latched():
    ctx = gpu_ctx(10, (50,), 30)
    for bad in (np.nan, np.inf, -np.inf):
        api.ckks_encode(ctx, dev(np.array([[1.0, bad, 0.5]]), torch.float64))
        with pytest.raises(api.ZincError) as e:
            api.zn_sync_status(ctx)
        assert e.value.status == api.ZN_EOVERFLOW
    api.zn_sync_status(ctx)


def test_encode_overflow_latched():
    ctx = gpu_ctx(10, (50,), 60)
    z = np.full((1, 8), 1e6)
    api.ckks_encode(ctx, dev(z, torch.float64))
    with pytest.raises(api.ZincError) as e:
        api.zn_sync_status(ctx)
    assert e.value.status == api.ZN_EOVERFLOW
    api.zn_sync_status(ctx)            # cleared; the context stays usable
    api.ckks_encode(ctx, dev(np.zeros((1, 8)), torch.float64))
    api.zn_sync_status(ctx)


# -------------------------------------------------------------------- keygen
@pytest.mark.parametrize("log_n,bits", [(4, (30,)), (10, (40, 41)), (12, (36, 36, 36))])
def test_keygen_bit_exact(log_n, bits):
    sk, pk = gpu_keys(log_n, bits, 20, 1)
    P, K, _ = oracle_model(log_n, bits, 20, 1, 2)
    assert np.array_equal(api.zn_pk_export(pk), O.pk_ntt(P, K))
    assert np.array_equal(api.zn_sk_export(sk).astype(np.int64), K.s)


@pytest.mark.parametrize("name", ["throughput", "large"])
def test_keygen_sampled_full_size(name):
    w = workloads.WORKLOADS[name]
    _, pk = gpu_keys(w.log_n, w.bits, w.log2_delta, workloads.KEYGEN_SEED)
    P, K, _ = oracle_model(w.log_n, w.bits, w.log2_delta, workloads.KEYGEN_SEED, workloads.CACHE_SEED)
    got = api.zn_pk_export(pk)
    rng = np.random.default_rng(0)
    for i in (0, 1, w.L - 1):
        idx = rng.integers(0, w.n, 16).astype(np.uint32)
        assert np.array_equal(got[0, i, idx], OR.ntt_eval(K.pk0[i], P.primes[i], P.psis[i], idx))
        assert np.array_equal(got[1, i, idx], OR.ntt_eval(K.pk1[i], P.primes[i], P.psis[i], idx))


# ---------------------------------------------------------------- encryption
SMALL = [(4, (30,), 20, 8), (6, (40, 41), 25, 20), (10, (40, 40, 41), 30, 500), (12, (36, 36, 36), 30, 2048),
         (14, (50, 60), 40, 8192)]


@pytest.mark.parametrize("log_n,bits,ld,n_slots", SMALL)
def test_encrypt_bit_exact_full(log_n, bits, ld, n_slots):
    ctx = gpu_ctx(log_n, bits, ld)
    sk, pk = gpu_keys(log_n, bits, ld, 1)
    zc = gpu_cache(log_n, bits, ld, 1, 2)
    P, K, zero = oracle_model(log_n, bits, ld, 1, 2)
    assert np.array_equal(api.zn_zcache_export(zc), O.ct_ntt(P, zero))
    B, seed = 3, 0
    z = workloads.slots(workloads.small(log_n, bits, ld, B, n_slots, seed=9))
    idx = np.array([0, 7, 2 ** 40 + 3], dtype=np.int64)
    ct_v = api.ckks_encrypt(ctx, pk, dev(z, torch.float64), seed, dev(idx, torch.int64))
    ct_z = api.zinc_encrypt(ctx, zc, dev(z, torch.float64), seed, dev(idx, torch.int64))
    api.zn_sync_status(ctx)
    gv, gz = api.as_u64(ct_v), api.as_u64(ct_z)
    for b in range(B):
        ref_v = O.ct_ntt(P, O.encrypt_coeff(P, K, z[b], seed, int(idx[b])))
        ref_z = O.ct_ntt(P, O.zinc_encrypt_coeff(P, zero, z[b], seed, int(idx[b])))
        assert np.array_equal(gv[b], ref_v), ("vanilla", b)
        assert np.array_equal(gz[b], ref_z), ("zinc", b)
    # Dec (Eq. 10) in the coefficient domain, bit-exact against the oracle
    dv = api.as_u64(api.ckks_decrypt(ctx, sk, ct_v))
    ov = O.encrypt_coeff(P, K, z[1], seed, int(idx[1]))
    ref = O.decrypt_coeff(P, K, ov.c0, ov.c1)
    assert all(np.array_equal(dv[1, i], ref[i]) for i in range(P.n_primes))
    # decoded slots within the noise tolerance
    for ct in (ct_v, ct_z):
        back = api.ckks_decrypt_decode(ctx, sk, ct, n_slots).cpu().numpy()
        assert np.max(np.abs(back - z)) < tol(log_n, ld)


def _check_sampled(w, ct, zinc, z, idx, rows, seed):
    P, K, zero = oracle_model(w.log_n, w.bits, w.log2_delta, workloads.KEYGEN_SEED, workloads.CACHE_SEED)
    rng = np.random.default_rng(123)
    got = api.as_u64(ct)
    for b in rows:
        if zinc:
            oct_ = O.zinc_encrypt_coeff(P, zero, z[b], seed, int(idx[b]))
        else:
            oct_ = O.encrypt_coeff(P, K, z[b], seed, int(idx[b]))
        pos = [(p, i, int(k)) for p in (0, 1) for i in (0, w.L // 2, w.L - 1)
               for k in np.concatenate([[0, w.n - 1], rng.integers(0, w.n, 4)])]
        ref = O.ct_ntt_sampled(P, oct_, pos)
        assert np.array_equal(np.array([got[b, p, i, k] for p, i, k in pos], dtype=np.uint64), ref), (b, zinc)


def _check_whole(w, ct, zinc, z, idx, rows, seed):
    """Every residue of the given rows (all 2 L N of them) against the oracle's
    definitional transform of its coefficient-domain ciphertext."""
    P, K, zero = oracle_model(w.log_n, w.bits, w.log2_delta, workloads.KEYGEN_SEED, workloads.CACHE_SEED)
    got = api.as_u64(ct)
    for b in rows:
        if zinc:
            ref = O.ct_ntt(P, O.zinc_encrypt_coeff(P, zero, z[b], seed, int(idx[b])))
        else:
            ref = O.ct_ntt(P, O.encrypt_coeff(P, K, z[b], seed, int(idx[b])))
        assert np.array_equal(got[b], ref), (b, zinc)


# rows compared in full: the first and last ciphertext of the call and two
# in between (every workload's call is one launch pair: up to 512 MiB of
# prepared words; launch boundaries are checked in test_gpu_ragged.py)
WHOLE_ROWS = {"batched": {False: (0, 255, 256, 1023), True: (0, 255, 256, 1023)},
              "throughput": {False: (0, 2047, 2048, 4095), True: (0, 2047, 2048, 4095)},
              "large": {False: (511,), True: (0,)}}


@pytest.mark.parametrize("name", ["batched", "throughput", "large"])
def test_encrypt_full_size(name):
    """The benchmark's launch configuration: the whole batch in one call; whole
    ciphertexts and sampled residues of others against the oracle."""
    w = workloads.WORKLOADS[name]
    ctx = gpu_ctx(w.log_n, w.bits, w.log2_delta)
    sk, pk = gpu_keys(w.log_n, w.bits, w.log2_delta, workloads.KEYGEN_SEED)
    zc = gpu_cache(w.log_n, w.bits, w.log2_delta, workloads.KEYGEN_SEED, workloads.CACHE_SEED)
    z = workloads.slots(w)
    idx = np.arange(w.batch, dtype=np.int64)
    zd = dev(z, torch.float64)
    ct_v = api.ckks_encrypt(ctx, pk, zd, w.seed, dev(idx, torch.int64))
    ct_z = api.zinc_encrypt(ctx, zc, zd, w.seed, dev(idx, torch.int64))
    api.zn_sync_status(ctx)
    _check_whole(w, ct_v, False, z, idx, WHOLE_ROWS[name][False], w.seed)
    _check_whole(w, ct_z, True, z, idx, WHOLE_ROWS[name][True], w.seed)
    rows = [w.batch // 2 + 1, w.batch // 3, w.batch - 2]
    _check_sampled(w, ct_v, False, z, idx, rows, w.seed)
    _check_sampled(w, ct_z, True, z, idx, rows, w.seed)
    # every ciphertext decrypts within tolerance (a property that holds at any size)
    lim = tol(w.log_n, w.log2_delta) * max(abs(w.lo), abs(w.hi))
    for ct in (ct_v, ct_z):
        for b0 in range(0, w.batch, 256):
            back = api.ckks_decrypt_decode(ctx, sk, ct[b0:b0 + 256].contiguous(), w.n_slots).cpu().numpy()
            assert np.max(np.abs(back - z[b0:b0 + 256])) < lim
    if w.log_n == 14:
        assert lim < 2.0 ** -20     # the paper-scale accuracy claim holds here


def test_batch_equals_solo():
    w = workloads.small(10, (40, 41), 30, 5, 300, seed=4)
    ctx = gpu_ctx(10, (40, 41), 30)
    _, pk = gpu_keys(10, (40, 41), 30, 1)
    zc = gpu_cache(10, (40, 41), 30, 1, 2)
    z = workloads.slots(w)
    idx = np.array([9, 1, 5, 2 ** 35, 4], dtype=np.int64)
    for fn, key in ((api.ckks_encrypt, pk), (api.zinc_encrypt, zc)):
        full = api.as_u64(fn(ctx, key, dev(z, torch.float64), 11, dev(idx, torch.int64)))
        for b in (4, 0, 3):
            one = api.as_u64(fn(ctx, key, dev(z[b:b + 1], torch.float64), 11, dev(idx[b:b + 1], torch.int64)))
            assert np.array_equal(one[0], full[b])


def test_homomorphic_add_and_zero_message():
    log_n, bits, ld = 12, (36, 36, 36), 30
    ctx = gpu_ctx(log_n, bits, ld)
    sk, pk = gpu_keys(log_n, bits, ld, 1)
    zc = gpu_cache(log_n, bits, ld, 1, 2)
    rng = np.random.default_rng(5)
    za, zb = rng.uniform(-1, 1, (2, 1, 2048))
    idx = dev(np.array([3]), torch.int64)
    ca = api.ckks_encrypt(ctx, pk, dev(za, torch.float64), 1, idx)
    cb = api.zinc_encrypt(ctx, zc, dev(zb, torch.float64), 1, idx)
    s = api.ckks_add(ctx, ca, cb)
    back = api.ckks_decrypt_decode(ctx, sk, s, 2048).cpu().numpy()
    assert np.max(np.abs(back - (za + zb))) < 2 * tol(log_n, ld)
    # n_slots = 0 encrypts the zero plaintext
    c0 = api.ckks_encrypt(ctx, pk, dev(np.zeros((1, 0)), torch.float64), 1, idx)
    back = api.ckks_decrypt_decode(ctx, sk, c0, 16).cpu().numpy()
    assert np.max(np.abs(back)) < tol(log_n, ld)


def test_export_import_roundtrip():
    log_n, bits, ld = 10, (40, 41), 30
    ctx = gpu_ctx(log_n, bits, ld)
    sk, pk = gpu_keys(log_n, bits, ld, 1)
    zc = gpu_cache(log_n, bits, ld, 1, 2)
    pk2 = api.zn_pk_import(ctx, api.zn_pk_export(pk))
    sk2 = api.zn_sk_import(ctx, api.zn_sk_export(sk))
    zc2 = api.zn_zcache_import(ctx, api.zn_zcache_export(zc))
    z = dev(np.random.default_rng(1).uniform(-1, 1, (2, 100)), torch.float64)
    idx = dev(np.array([1, 2]), torch.int64)
    assert torch.equal(api.ckks_encrypt(ctx, pk, z, 3, idx), api.ckks_encrypt(ctx, pk2, z, 3, idx))
    assert torch.equal(api.zinc_encrypt(ctx, zc, z, 3, idx), api.zinc_encrypt(ctx, zc2, z, 3, idx))
    ct = api.ckks_encrypt(ctx, pk, z, 3, idx)
    assert torch.equal(api.ckks_decrypt(ctx, sk, ct), api.ckks_decrypt(ctx, sk2, ct))
    bad = api.zn_pk_export(pk)
    bad[0, 0, 0] = ctx.primes[0]           # not a residue
    with pytest.raises(api.ZincError):
        api.zn_pk_import(ctx, bad)


def test_invalid_arguments():
    ctx = gpu_ctx(10, (40, 41), 30)
    _, pk = gpu_keys(10, (40, 41), 30, 1)
    z = dev(np.zeros((1, 600)), torch.float64)          # more slots than N/2
    with pytest.raises(api.ZincError) as e:
        api.ckks_encrypt(ctx, pk, z, 0, dev(np.array([0]), torch.int64))
    assert e.value.status == api.ZN_EINVAL
    other = gpu_ctx(10, (40, 42), 30)
    with pytest.raises(api.ZincError):                    # key from another context
        api.ckks_encrypt(other, pk, dev(np.zeros((1, 4)), torch.float64), 0, dev(np.array([0]), torch.int64))
    # empty batch is a no-op
    out = torch.empty((0, 2, 2, 1024), dtype=torch.int64, device="cuda:0")
    api.ckks_encrypt(ctx, pk, dev(np.zeros((0, 4)), torch.float64), 0,
                     torch.empty((0,), dtype=torch.int64, device="cuda:0"), out=out)


@pytest.mark.parametrize("log_n,bits,ld", [(10, (40, 60), 30), (11, (50,), 40), (12, (36, 36, 36), 30),
                                           (13, (60, 40), 40), (14, (60, 50, 60), 50), (15, (55, 60), 55)])
def test_launch_variants_bit_identical(log_n, bits, ld):
    """Every launch shape the autotuner may choose gives the same ciphertexts."""
    ctx = gpu_ctx(log_n, bits, ld)
    # a new context starts at the radix-8 kernels where they apply (at 2^15
    # the four-CTA cluster kernel)
    default = api.zn_get_variant(ctx)
    assert default == (6 if 10 <= log_n <= 15 else 0)
    _, pk = gpu_keys(log_n, bits, ld, 1)
    zc = gpu_cache(log_n, bits, ld, 1, 2)
    w = workloads.small(log_n, bits, ld, 3, (1 << log_n) // 2 - 5, seed=8)
    z = dev(workloads.slots(w), torch.float64)
    idx = dev(np.array([4, 0, 2 ** 34]), torch.int64)
    outs = []
    for v in range(api.VARIANTS):
        api.zn_set_variant(ctx, v)
        assert api.zn_get_variant(ctx) == v
        outs.append((api.ckks_encrypt(ctx, pk, z, 5, idx), api.zinc_encrypt(ctx, zc, z, 5, idx)))
    for o in outs[1:]:
        assert torch.equal(o[0], outs[0][0]) and torch.equal(o[1], outs[0][1])
    chosen, ms = api.zn_autotune(ctx, pk, zc, 8)
    assert chosen in range(api.VARIANTS) and all(m > 0 for m in ms)
    assert api.zn_get_variant(ctx) == chosen
    api.zn_set_variant(ctx, default)


@pytest.mark.parametrize("zinc", [False, True])
def test_multipoly_variant_misaligned_output(zinc):
    """The multi-polynomial kernel needs 16-byte aligned output rows; an output
    that starts 8 bytes off takes the per-polynomial kernel, same ciphertexts."""
    log_n, bits, ld = 13, (60, 40), 40
    ctx = gpu_ctx(log_n, bits, ld)
    _, pk = gpu_keys(log_n, bits, ld, 1)
    zc = gpu_cache(log_n, bits, ld, 1, 2)
    key = zc if zinc else pk
    fn = api.zinc_encrypt if zinc else api.ckks_encrypt
    w = workloads.small(log_n, bits, ld, 2, 100, seed=9)
    z = dev(workloads.slots(w), torch.float64)
    idx = dev(np.array([1, 7]), torch.int64)
    shape = (2, 2, len(bits), 1 << log_n)
    default = api.zn_get_variant(ctx)
    api.zn_set_variant(ctx, 0)
    ref = fn(ctx, key, z, 3, idx)
    api.zn_set_variant(ctx, 2)                          # kind 1, prime-major
    aligned = fn(ctx, key, z, 3, idx)
    flat = torch.empty(int(np.prod(shape)) + 1, dtype=torch.int64, device="cuda:0")
    off = flat[1:].view(shape)
    assert off.data_ptr() % 16 == 8
    fn(ctx, key, z, 3, idx, out=off)
    api.zn_set_variant(ctx, default)
    assert torch.equal(aligned, ref) and torch.equal(off, ref)
