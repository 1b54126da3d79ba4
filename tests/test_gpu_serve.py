"""Serving loop: requests of mixed ring degree and mode, arriving over time,
are continuously batched onto several streams.  Each request's ciphertext is
bit-identical to the same request encrypted alone, decrypts to its slots
within the noise tolerance, and every request completes exactly once -- also
under an HBM budget small enough to serialise the batches."""
import numpy as np
import pytest

from paper_2408_07304_gb300 import api, serve

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def server():
    from paper_2408_07304_gb300 import build
    build.build()
    return serve.Server(device=0, n_streams=3, max_batch=32, hbm_budget=4 << 30, keep_results=True)


def tol(ctx):
    return (10 * ctx.n * 3.2 + ctx.n) / 2.0 ** ctx.log2_delta


def test_mixed_results_equal_alone(server):
    reqs = serve.poisson_requests(240, rate=20000.0, seed=9)
    done, info = server.run(reqs)
    assert sorted(d.rid for d in done) == list(range(len(reqs)))
    assert info["peak_inflight_batches"] >= 2          # batches overlapped on the device
    by = {d.rid: d for d in done}
    rng = np.random.default_rng(0)
    for rid in rng.choice(len(reqs), 24, replace=False):
        r = reqs[rid]
        alone = server.encrypt_one(r)
        assert torch.equal(by[rid].ct, alone), (rid, r.ring, r.zinc)
    for rid in rng.choice(len(reqs), 6, replace=False):
        r = reqs[rid]
        ctx, sk = server.rings[r.ring][0], server.rings[r.ring][1]
        back = api.ckks_decrypt_decode(ctx, sk, by[rid].ct[None].contiguous(), r.slots.shape[0])
        assert float((back.cpu()[0] - torch.tensor(r.slots)).abs().max()) < tol(ctx)
    s = serve.summarize(done, info, len(reqs))
    assert s["p99_ms"] >= s["p50_ms"] > 0


def test_tight_budget_serialises(server):
    old = server.budget
    server.budget = server.batch_bytes("n32768", 1, 16384) + 1     # room for one big request
    try:
        reqs = serve.poisson_requests(40, rate=None, seed=4)
        done, info = server.run(reqs)
        assert sorted(d.rid for d in done) == list(range(40))
        assert info["peak_reserved_bytes"] <= server.budget
    finally:
        server.budget = old
