"""Per-vector slot counts at the boundary (ckks_encode_ragged,
ckks_encrypt_ragged, zinc_encrypt_ragged): vector b takes the first
n_slots[b] entries of its row, missing slots are zero.  Results are checked
against the oracle (the encoder on the row's own slots; Eq. 8 and Algorithm
1 for whole ciphertexts) and against the scalar-count entry points on the
zero-padded rows, which give the same integers because padding is exact."""
import functools

import numpy as np
import pytest

from oracle import ckks as O
from oracle import encoder as OE
from paper_2408_07304_gb300 import api

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=None)
def ring(log_n, bits, ld):
    from paper_2408_07304_gb300 import build
    build.build()
    ctx = api.Context(log_n, bits, ld, device=0)
    sk, pk = api.ckks_keygen(ctx, 1)
    return ctx, sk, pk, api.zinc_precompute(ctx, pk, 2)


@functools.lru_cache(maxsize=None)
def oracle(log_n, bits, ld):
    P = O.Params(log_n, bits, ld)
    K = O.keygen(P, 1)
    return P, K, O.zinc_precompute_coeff(P, K, 2)


def rows(log_n, counts, stride, seed):
    rng = np.random.default_rng(seed)
    z = rng.uniform(-1, 1, (len(counts), stride))
    for b, k in enumerate(counts):
        z[b, k:] = 0.0 if b % 2 else 7.5e3     # entries past the count are never read
    return z


@pytest.mark.parametrize("log_n,ld", [(10, 30), (14, 50), (15, 55)])
def test_encode_ragged_matches_oracle(log_n, ld):
    ctx, _, _, _ = ring(log_n, (50,), ld)
    half = (1 << log_n) // 2
    counts = [0, 1, half, 37, half - 1, 5]
    z = rows(log_n, counts, half, log_n)
    out = api.ckks_encode_ragged(ctx, torch.tensor(z, device="cuda:0"),
                                 torch.tensor(counts, dtype=torch.int32, device="cuda:0"))
    api.zn_sync_status(ctx)
    got = out.cpu().numpy()
    for b, k in enumerate(counts):
        assert np.array_equal(got[b], OE.encode(z[b, :k], log_n, ld)), (b, k)


@pytest.mark.parametrize("log_n,bits,ld", [(10, (40, 40, 41), 30), (13, (60, 40, 60), 40)])
def test_encrypt_ragged_matches_oracle_and_padded(log_n, bits, ld):
    ctx, sk, pk, zc = ring(log_n, bits, ld)
    P, K, zero = oracle(log_n, bits, ld)
    half = (1 << log_n) // 2
    counts = [3, 0, half, 100, 1]
    stride = half
    z = rows(log_n, counts, stride, 5)
    zd = torch.tensor(z, device="cuda:0")
    nd = torch.tensor(counts, dtype=torch.int32, device="cuda:0")
    idx = torch.tensor([4, 0, 2 ** 36, 9, 11], dtype=torch.int64, device="cuda:0")
    cv = api.ckks_encrypt_ragged(ctx, pk, zd, nd, 6, idx)
    cz = api.zinc_encrypt_ragged(ctx, zc, zd, nd, 6, idx)
    api.zn_sync_status(ctx)
    gv, gz = api.as_u64(cv), api.as_u64(cz)
    padded = z.copy()
    for b, k in enumerate(counts):
        padded[b, k:] = 0.0
        ref_v = O.ct_ntt(P, O.encrypt_coeff(P, K, z[b, :k], 6, int(idx[b])))
        ref_z = O.ct_ntt(P, O.zinc_encrypt_coeff(P, zero, z[b, :k], 6, int(idx[b])))
        assert np.array_equal(gv[b], ref_v), ("vanilla", b)
        assert np.array_equal(gz[b], ref_z), ("zinc", b)
    pd = torch.tensor(padded, device="cuda:0")
    assert torch.equal(cv, api.ckks_encrypt(ctx, pk, pd, 6, idx))
    assert torch.equal(cz, api.zinc_encrypt(ctx, zc, pd, 6, idx))


def test_encrypt_ragged_two_launches():
    # N = 2^15 holds at most 2048 ciphertexts per launch (512 MiB of prepared
    # words), so 2050 run as two equal launches of 1025: rows on both sides of
    # the boundary are checked
    ctx, sk, pk, zc = ring(15, (55, 60), 55)
    B, half = 2050, 1 << 14
    rng = np.random.default_rng(3)
    counts = rng.integers(0, half + 1, B).astype(np.int32)
    stride = int(counts.max())
    z = rng.uniform(-1, 1, (B, stride))
    zd = torch.tensor(z, device="cuda:0")
    nd = torch.tensor(counts, device="cuda:0")
    idx = torch.arange(B, dtype=torch.int64, device="cuda:0")
    cz = api.zinc_encrypt_ragged(ctx, zc, zd, nd, 8, idx)
    api.zn_sync_status(ctx)
    for b in (0, 1024, 1025, B - 1):
        k = int(counts[b])
        one = api.zinc_encrypt(ctx, zc, torch.tensor(z[b:b + 1, :k], device="cuda:0"), 8, idx[b:b + 1])
        assert torch.equal(cz[b:b + 1], one), b
    back = api.ckks_decrypt_decode(ctx, sk, cz[:8].contiguous(), stride).cpu().numpy()
    for b in range(8):
        k = int(counts[b])
        want = np.concatenate([z[b, :k], np.zeros(stride - k)])
        assert np.max(np.abs(back[b] - want)) < (10 * (1 << 15) * 3.2 + (1 << 15)) / 2.0 ** 55


def test_ragged_count_above_stride_latched():
    ctx, _, pk, zc = ring(10, (40, 40, 41), 30)
    z = torch.zeros((2, 8), dtype=torch.float64, device="cuda:0")
    nd = torch.tensor([3, 9], dtype=torch.int32, device="cuda:0")       # 9 > stride 8
    idx = torch.tensor([0, 1], dtype=torch.int64, device="cuda:0")
    api.ckks_encrypt_ragged(ctx, pk, z, nd, 1, idx)
    with pytest.raises(api.ZincError) as e:
        api.zn_sync_status(ctx)
    assert e.value.status == api.ZN_EINVAL
    api.zn_sync_status(ctx)                          # cleared; the context stays usable
    with pytest.raises(api.ZincError):               # a stride above N/2 is refused on the host
        api.zinc_encrypt_ragged(ctx, zc, torch.zeros((1, 513), dtype=torch.float64, device="cuda:0"),
                                torch.tensor([1], dtype=torch.int32, device="cuda:0"), 1, idx[:1])
