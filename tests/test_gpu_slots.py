"""GPU parity of the BFV / BGV slot batching (zn_slots_encode / zn_slots_decode,
through the C ABI) against the oracle's batch_encode / batch_decode, and the
slot round trip through encryption: slots -> plaintext -> BFV / BGV (vanilla
and Zinc) -> decryption -> slots, exactly, with slot-wise addition under the
homomorphic sum.
"""
import functools

import numpy as np
import pytest

from oracle import bfvbgv as OB
from paper_2408_07304_gb300 import api

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=None)
def model(log_n, bits, t):
    from paper_2408_07304_gb300 import build
    build.build()
    ctx = api.Context(log_n, bits, 20, device=0)
    se = api.zn_slot_encoder_create(ctx, t)
    return ctx, se


def dev(a):
    return torch.tensor(np.asarray(a), dtype=torch.int64, device="cuda:0")


@pytest.mark.parametrize("log_n,bits,t", [(10, (40, 41), 12289), (12, (50, 51), 65537), (14, (60, 50), 65537)])
def test_slots_bit_exact(log_n, bits, t):
    ctx, se = model(log_n, bits, t)
    n = 1 << log_n
    rng = np.random.default_rng(log_n)
    x = rng.integers(-3 * t, 3 * t, (2, n))
    m = api.zn_slots_encode(se, dev(x)).cpu().numpy()
    assert m[0].tolist() == OB.batch_encode(x[0], t, log_n)
    y = rng.integers(0, t, (2, n))
    d = api.zn_slots_decode(se, dev(y)).cpu().numpy()
    assert d[1].tolist() == OB.batch_decode(y[1], t, log_n)
    assert np.array_equal(api.zn_slots_decode(se, dev(m)).cpu().numpy(), np.mod(x, t))


@pytest.mark.parametrize("log_n,bits", [(13, (60, 40, 60)), (15, (55, 55, 60))])
def test_slot_round_trip_through_encryption(log_n, bits):
    t = 65537
    ctx, se = model(log_n, bits, t)
    n = 1 << log_n
    sk, pk = api.ckks_keygen(ctx, 1)
    zc = api.zinc_precompute(ctx, pk, 2)
    gsk, gpk = api.bgv_keygen(ctx, t, 1)
    gzc = api.bgv_zinc_precompute(ctx, gpk, 2)
    rng = np.random.default_rng(3)
    xa, xb = rng.integers(0, t, (2, 2, n))
    ma, mb = api.zn_slots_encode(se, dev(xa)), api.zn_slots_encode(se, dev(xb))
    idx = dev([0, 1])
    for enc_a, enc_b, dec, key in (
            (lambda m: api.bfv_encrypt(ctx, pk, t, m, 4, idx), lambda m: api.bfv_zinc_encrypt(ctx, zc, t, m, 5, idx),
             api.bfv_decrypt, sk),
            (lambda m: api.bgv_encrypt(ctx, gpk, m, 4, idx), lambda m: api.bgv_zinc_encrypt(ctx, gzc, m, 5, idx),
             api.bgv_decrypt, gsk)):
        ca, cb = enc_a(ma), enc_b(mb)
        assert np.array_equal(api.zn_slots_decode(se, dec(ctx, key, t, ca)).cpu().numpy(), xa)
        assert np.array_equal(api.zn_slots_decode(se, dec(ctx, key, t, cb)).cpu().numpy(), xb)
        s = api.ckks_add(ctx, ca, cb)
        assert np.array_equal(api.zn_slots_decode(se, dec(ctx, key, t, s)).cpu().numpy(), np.mod(xa + xb, t))


def test_slot_encoder_rejects_invalid_t():
    ctx, _ = model(10, (40, 41), 12289)
    for bad in (12288, 12289 * 3, 65539, 7683):   # even, composite, prime but not 1 mod 2N, composite
        with pytest.raises(api.ZincError) as e:
            api.zn_slot_encoder_create(ctx, bad)
        assert e.value.status == api.ZN_EINVAL
