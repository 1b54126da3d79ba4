"""The stream-ordered encryption calls can be captured into a CUDA graph: their
scratch comes from the context's stream-ordered pool and nothing in them
synchronises the host.  Each call is run once eagerly (kernel attributes set,
pool warmed), then captured on a side stream and replayed twice; the replays
must reproduce the eager ciphertexts bit for bit and see new inputs written
into the captured buffers.
"""
import numpy as np
import pytest

from paper_2408_07304_gb300 import api

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ctx():
    from paper_2408_07304_gb300 import build
    build.build()
    ctx = api.Context(12, (36, 36, 37), 30, device=0)
    sk, pk = api.ckks_keygen(ctx, 1)
    return ctx, sk, pk


def test_capture_replay_equals_eager():
    ctx, sk, pk = _ctx()
    zc = api.zinc_precompute(ctx, pk, 2)
    nb = api.zinc_nbasis_create(ctx, 2, 3)
    B, n = 4, ctx.n
    rng = np.random.default_rng(0)
    slots = torch.tensor(rng.uniform(-1, 1, (B, 700)), device="cuda:0")
    idx = torch.arange(B, dtype=torch.int64, device="cuda:0")
    m_int = torch.tensor(rng.integers(0, 65537, (B, n)), device="cuda:0")
    outs = {
        "vanilla": torch.empty((B, 2, ctx.L, n), dtype=torch.int64, device="cuda:0"),
        "zinc": torch.empty((B, 2, ctx.L, n), dtype=torch.int64, device="cuda:0"),
        "ms": torch.empty((B, 2, ctx.L - 1, n), dtype=torch.int64, device="cuda:0"),
        "bfv": torch.empty((B, 2, ctx.L, n), dtype=torch.int64, device="cuda:0"),
        "ntt": torch.empty((B, 2, ctx.L, n), dtype=torch.int64, device="cuda:0"),
    }
    m_hat = torch.empty((B, ctx.L, n), dtype=torch.int64, device="cuda:0")

    def step(stream=None):
        api.ckks_encrypt(ctx, pk, slots, 5, idx, out=outs["vanilla"], stream=stream)
        api.zinc_encrypt(ctx, zc, slots, 5, idx, out=outs["zinc"], stream=stream)
        api.ckks_encrypt_ms(ctx, pk, slots, 5, idx, out=outs["ms"], stream=stream)
        api.bfv_encrypt(ctx, pk, 65537, m_int, 5, idx, out=outs["bfv"], stream=stream)
        api.ckks_encode_ntt(ctx, slots, out=m_hat, stream=stream)
        api.zinc_encrypt_ntt(ctx, zc, nb, m_hat, 5, idx, out=outs["ntt"], stream=stream)

    step()
    torch.cuda.synchronize()
    eager = {k: v.clone() for k, v in outs.items()}
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        step(stream=s)
    for v in outs.values():
        v.zero_()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    api.zn_sync_status(ctx)
    for k in outs:
        assert torch.equal(outs[k], eager[k]), k
    # new inputs in the captured buffers: the replay encrypts them
    slots.copy_(torch.tensor(rng.uniform(-1, 1, (B, 700)), device="cuda:0"))
    m_int.copy_(torch.tensor(rng.integers(0, 65537, (B, n)), device="cuda:0"))
    g.replay()
    torch.cuda.synchronize()
    replayed = {k: v.clone() for k, v in outs.items()}
    step()
    torch.cuda.synchronize()
    for k in outs:
        assert torch.equal(replayed[k], outs[k]), k
        assert not torch.equal(replayed[k], eager[k]), k
    back = api.ckks_decrypt_decode(ctx, sk, outs["zinc"], 700).cpu().numpy()
    assert np.max(np.abs(back - slots.cpu().numpy())) < 1e-3
    assert torch.equal(api.bfv_decrypt(ctx, sk, 65537, outs["bfv"]), m_int)
