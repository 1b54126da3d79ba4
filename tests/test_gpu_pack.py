"""Packed ciphertext serialization (zn_ct_pack / zn_ct_unpack /
zn_encrypt_host_packed, through the C ABI).  The packed words are checked
against the format's definition built here with Python integers (each limb's
residues concatenated as one little-endian bit stream of bit-length-of-q_i
fields), on rings whose limbs end mid-word and on the throughput workload's
chain; unpacking restores the ciphertexts exactly; the host-buffer entry
point's packed output equals packing its plain output; a field not below its
prime is latched and reported by zn_sync_status.
"""
import numpy as np
import pytest

from paper_2408_07304_gb300 import api, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ctx(log_n, bits, ld):
    from paper_2408_07304_gb300 import build
    build.build()
    ctx = api.Context(log_n, bits, ld, device=0)
    sk, pk = api.ckks_keygen(ctx, 1)
    return ctx, pk


def _limb_words(residues, nbits):
    """The format's definition: one integer holding every residue at its bit
    offset, cut into 64-bit words (little-endian)."""
    acc = 0
    for j, r in enumerate(residues):
        acc |= int(r) << (j * nbits)
    n_words = -(-len(residues) * nbits // 64)
    return [(acc >> (64 * w)) & (2 ** 64 - 1) for w in range(n_words)]


def _reference(ctx, ct_u64, b):
    out = []
    for c in range(2):
        for i, q in enumerate(ctx.primes):
            out += _limb_words(ct_u64[b, c, i], int(q).bit_length())
    return np.array(out, dtype=np.uint64)


def _encrypt(ctx, pk, B, seed=5):
    z = torch.tensor(np.random.default_rng(seed).uniform(-1, 1, (B, min(64, ctx.n // 2))), device="cuda:0")
    return api.ckks_encrypt(ctx, pk, z, seed, torch.arange(B, dtype=torch.int64, device="cuda:0")), z


# N >= 1024 with 16-byte aligned buffers runs the bulk-copy tile kernels, smaller rings the per-word ones
@pytest.mark.parametrize("log_n,bits,ld", [(4, (30, 40), 20), (6, (31, 45, 60), 25), (10, (40, 40, 41), 30),
                                           (12, (36, 59, 20, 61), 30)])
def test_pack_matches_definition_and_round_trips(log_n, bits, ld):
    ctx, pk = _ctx(log_n, bits, ld)
    ct, _ = _encrypt(ctx, pk, 3)
    W = api.zn_ct_packed_words(ctx)
    assert W == 2 * sum(-(-ctx.n * int(q).bit_length() // 64) for q in ctx.primes)
    packed = api.zn_ct_pack(ctx, ct)
    got, ref_ct = api.as_u64(packed), api.as_u64(ct)
    for b in range(3):
        assert np.array_equal(got[b], _reference(ctx, ref_ct, b)), b
    assert torch.equal(api.zn_ct_unpack(ctx, packed), ct)
    api.zn_sync_status(ctx)


def test_throughput_chain_packed_size_and_sampled_limbs():
    w = workloads.WORKLOADS["throughput"]
    ctx, pk = _ctx(w.log_n, w.bits, w.log2_delta)
    assert api.zn_ct_packed_words(ctx) * 64 == 2 * ctx.n * sum(int(q).bit_length() for q in ctx.primes)
    assert sum(int(q).bit_length() for q in ctx.primes) == 420           # 420 / 512 of the plain words
    ct, _ = _encrypt(ctx, pk, 4)
    packed = api.zn_ct_pack(ctx, ct)
    got, ref_ct = api.as_u64(packed), api.as_u64(ct)
    off = 0
    for c in range(2):
        for i, q in enumerate(ctx.primes):
            nb = int(q).bit_length()
            words = _limb_words(ref_ct[3, c, i], nb)
            assert np.array_equal(got[3, off:off + len(words)], np.array(words, dtype=np.uint64)), (c, i)
            off += len(words)
    assert torch.equal(api.zn_ct_unpack(ctx, packed), ct)


def test_encrypt_host_packed_equals_packed_device_ciphertexts():
    ctx, pk = _ctx(12, (36, 36, 37), 30)
    zc = api.zinc_precompute(ctx, pk, 2)
    B = 600
    rng = np.random.default_rng(7)
    hz = torch.tensor(rng.uniform(-1, 1, (B, 100))).pin_memory()
    hidx = torch.tensor(rng.integers(0, 2 ** 40, B), dtype=torch.int64).pin_memory()
    # chunk 256: 256 + 256 + 88 (a ragged last chunk); 0: the default, a
    # quarter of the batch here (four chunks of 150); 7: many chunks, ragged
    for key, chunk in ((pk, 256), (zc, 256), (pk, 0), (zc, 7)):
        out = torch.empty((B, api.zn_ct_packed_words(ctx)), dtype=torch.int64, pin_memory=True)
        api.zn_encrypt_host_packed(ctx, key, hz, 9, hidx, out, chunk=chunk)
        fn = api.zinc_encrypt if key is zc else api.ckks_encrypt
        dev_ct = fn(ctx, key, hz.cuda(), 9, hidx.cuda())
        assert torch.equal(out, api.zn_ct_pack(ctx, dev_ct).cpu()), chunk
        assert torch.equal(api.zn_ct_unpack(ctx, out.cuda()), dev_ct)
        plain = torch.empty((B, 2, ctx.L, ctx.n), dtype=torch.int64, pin_memory=True)
        api.zn_encrypt_host(ctx, key, hz, 9, hidx, plain, chunk=chunk)
        assert torch.equal(plain, dev_ct.cpu()), chunk


def test_unpack_latches_out_of_range_field():
    ctx, pk = _ctx(10, (40, 40, 41), 30)
    ct, _ = _encrypt(ctx, pk, 2)
    packed = api.zn_ct_pack(ctx, ct)
    api.zn_sync_status(ctx)
    bad = packed.clone()
    q0 = int(ctx.primes[0])
    first = int(api.as_u64(bad[1:2])[0, 0]) & ~((1 << 40) - 1) | q0      # residue 0 of limb 0 := q_0
    bad[1, 0] = np.array([first], dtype=np.uint64).view(np.int64)[0]
    api.zn_ct_unpack(ctx, bad)
    with pytest.raises(api.ZincError) as e:
        api.zn_sync_status(ctx)
    assert e.value.status == api.ZN_EINVAL
    assert torch.equal(api.zn_ct_unpack(ctx, packed), ct)              # the context stays usable
    api.zn_sync_status(ctx)


def test_tile_and_word_kernels_agree():
    # 16-byte aligned buffers take the bulk-copy tile kernels, buffers 8 bytes
    # off the per-word ones: the same words and residues either way, on the
    # benchmark chain (50- and 60-bit fields, words spanning residues)
    w = workloads.WORKLOADS["throughput"]
    ctx, pk = _ctx(w.log_n, w.bits, w.log2_delta)
    ct, _ = _encrypt(ctx, pk, 5)
    W = api.zn_ct_packed_words(ctx)
    flat_c = torch.empty(ct.numel() + 1, dtype=torch.int64, device="cuda:0")
    flat_p = torch.empty(5 * W + 1, dtype=torch.int64, device="cuda:0")
    off_c = flat_c[1:].view(tuple(ct.shape))
    off_p = flat_p[1:].view(5, W)
    assert off_c.data_ptr() % 16 == 8 and off_p.data_ptr() % 16 == 8
    off_c.copy_(ct)
    aligned = api.zn_ct_pack(ctx, ct)
    api.zn_ct_pack(ctx, off_c, out=off_p)
    assert torch.equal(aligned, off_p)
    back = torch.empty_like(ct)
    api.zn_ct_unpack(ctx, aligned, out=back)
    api.zn_ct_unpack(ctx, off_p, out=off_c)
    api.zn_sync_status(ctx)
    assert torch.equal(back, ct) and torch.equal(off_c, ct)
