"""Error paths under host-side fault injection (no GPU fault): per-call
scratch allocations made to fail with zn_inject_alloc_failures.  A refused
call returns ZN_ENOMEM before launching anything and leaves its context
usable -- the next call gives the same ciphertexts as an undisturbed one --
and the serving loop puts a refused batch back at the head of its queue,
retries it, and completes every request bit-identically; when the retries
run out with nothing in flight, only that batch's requests fail.  The
device-side bounded wait (the packed-serialization tiles' mbarrier wait) is
made to run out on a barrier that nothing arrives on: it latches
ZN_ETIMEOUT in the context's status word and the context stays usable.
"""
import numpy as np
import pytest

from paper_2408_07304_gb300 import api, serve

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _clear():
    yield
    api.zn_inject_alloc_failures(0)


def _ctx():
    from paper_2408_07304_gb300 import build
    build.build()
    ctx = api.Context(12, (36, 36, 37), 30, device=0)
    sk, pk = api.ckks_keygen(ctx, 1)
    return ctx, sk, pk


def test_refused_call_leaves_context_usable():
    ctx, sk, pk = _ctx()
    zc = api.zinc_precompute(ctx, pk, 2)
    z = torch.tensor(np.random.default_rng(0).uniform(-1, 1, (3, 100)), device="cuda:0")
    idx = torch.arange(3, dtype=torch.int64, device="cuda:0")
    calls = [lambda: api.ckks_encrypt(ctx, pk, z, 5, idx), lambda: api.zinc_encrypt(ctx, zc, z, 5, idx),
             lambda: api.ckks_encrypt_ms(ctx, pk, z, 5, idx)]
    for call in calls:
        ref = call()
        torch.cuda.synchronize()
        api.zn_inject_alloc_failures(1)
        with pytest.raises(api.ZincError) as e:
            call()
        assert e.value.status == api.ZN_ENOMEM
        assert torch.equal(call(), ref)
    api.zn_sync_status(ctx)
    # the host-buffer entry point refuses as a whole and then runs normally
    hz, hidx = z.cpu().pin_memory(), idx.cpu().pin_memory()
    out = torch.empty((3, 2, ctx.L, ctx.n), dtype=torch.int64, pin_memory=True)
    api.zn_inject_alloc_failures(1)
    with pytest.raises(api.ZincError) as e:
        api.zn_encrypt_host(ctx, pk, hz, 5, hidx, out)
    assert e.value.status == api.ZN_ENOMEM
    api.zn_encrypt_host(ctx, pk, hz, 5, hidx, out)
    assert torch.equal(out, calls[0]().cpu())


@pytest.fixture(scope="module")
def server():
    from paper_2408_07304_gb300 import build
    build.build()
    return serve.Server(device=0, n_streams=3, max_batch=16, hbm_budget=4 << 30, keep_results=True)


def test_server_retries_refused_batches(server):
    reqs = serve.poisson_requests(96, rate=20000.0, seed=21)
    api.zn_inject_alloc_failures(5)
    done, info = server.run(reqs)
    assert info["alloc_retries"] == 5 and not info["failed"]
    assert sorted(d.rid for d in done) == list(range(len(reqs)))
    by = {d.rid: d for d in done}
    for rid in np.random.default_rng(1).choice(len(reqs), 12, replace=False):
        assert torch.equal(by[rid].ct, server.encrypt_one(reqs[rid])), rid
    s = serve.summarize(done, info, len(reqs))
    assert s["alloc_retries"] == 5 and s["failed"] == 0


def test_server_fails_batch_when_retries_run_out(server):
    old = server.max_alloc_retries
    server.max_alloc_retries = 2
    try:
        reqs = serve.poisson_requests(1, rate=None, seed=3)
        api.zn_inject_alloc_failures(3)        # the first try and both retries
        done, info = server.run(reqs)
        assert not done and info["failed"] == [(0, api.ZN_ENOMEM)] and info["alloc_retries"] == 2
        done, info = server.run(reqs)          # nothing left to inject: served normally
        assert [d.rid for d in done] == [0] and not info["failed"]
        assert torch.equal(done[0].ct, server.encrypt_one(reqs[0]))
    finally:
        server.max_alloc_retries = old


def test_handles_released_after_their_context_leave_no_error():
    # Python's cycle collector may release a context before its keys; each
    # handle keeps its device, and no release leaves a CUDA error behind
    ctx, sk, pk = _ctx()
    zc = api.zinc_precompute(ctx, pk, 2)
    nb = api.zinc_nbasis_create(ctx, 2, 3)
    se = api.zn_slot_encoder_create(ctx, 65537)
    ctx.close()
    for h in (zc, nb, se, pk, sk):
        h.close()
    x = torch.arange(1 << 20, dtype=torch.float64, device="cuda:0")
    assert float(x.sum()) == (1 << 20) * ((1 << 20) - 1) / 2
    torch.cuda.synchronize()


def test_bounded_wait_times_out_and_context_stays_usable():
    ctx, sk, pk = _ctx()
    z = torch.tensor(np.random.default_rng(1).uniform(-1, 1, (2, 64)), device="cuda:0")
    idx = torch.arange(2, dtype=torch.int64, device="cuda:0")
    ref = api.ckks_encrypt(ctx, pk, z, 7, idx)
    packed = api.zn_ct_pack(ctx, ref)
    api.zn_sync_status(ctx)
    for tries in (1, 1024):
        api.zn_probe_wait_timeout(ctx, tries)
        with pytest.raises(api.ZincError) as e:
            api.zn_sync_status(ctx)
        assert e.value.status == api.ZN_ETIMEOUT
        api.zn_sync_status(ctx)              # read and cleared
    # the context, its stream and the tiles' own waits work as before
    assert torch.equal(api.ckks_encrypt(ctx, pk, z, 7, idx), ref)
    assert torch.equal(api.zn_ct_unpack(ctx, api.zn_ct_pack(ctx, ref)), ref)
    assert torch.equal(api.zn_ct_pack(ctx, ref), packed)
    api.zn_sync_status(ctx)
    for bad in (0, (1 << 20) + 1):
        with pytest.raises(api.ZincError) as e:
            api.zn_probe_wait_timeout(ctx, bad)
        assert e.value.status == api.ZN_EINVAL
