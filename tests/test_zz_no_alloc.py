"""The allocation-free Zinc entry point (zinc_encrypt_noalloc).

Some callers cannot allocate device memory inside a call -- a real-time loop
that must keep a fixed memory footprint, a host application that owns every
allocation, or a process whose device memory is already reserved -- so this
entry point keeps its intermediates in a fixed array inside the library and
takes only caller-provided inputs and outputs.  Its ciphertexts must be
identical to zinc_encrypt's (the tolerance the other ciphertext tests use is
bit equality), on consecutive calls that reuse the shared array, and a batch
too large for the array must be refused with ZN_ELIMIT before any launch.
"""
import numpy as np
import pytest

from paper_2408_07304_gb300 import api, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _setup(log_n, bits, ld):
    from paper_2408_07304_gb300 import build
    build.build()
    ctx = api.Context(log_n, bits, ld, device=0)
    _, pk = api.ckks_keygen(ctx, 1)
    zc = api.zinc_precompute(ctx, pk, 2)
    return ctx, zc


@pytest.mark.parametrize("log_n,bits,ld,batch", [(14, (60, 50, 50, 60), 50, 16), (15, (55, 60), 55, 3),
                                                 (12, (36, 36, 36), 30, 40)])
def test_noalloc_equals_zinc_encrypt_on_consecutive_calls(log_n, bits, ld, batch):
    ctx, zc = _setup(log_n, bits, ld)
    out = torch.empty((batch, 2, ctx.L, ctx.n), dtype=torch.int64, device="cuda:0")
    for call in range(2):
        w = workloads.small(log_n, bits, ld, batch, ctx.n // 2 - 3 * call, seed=40 + call)
        z = torch.tensor(workloads.slots(w), dtype=torch.float64, device="cuda:0")
        idx = torch.tensor(np.arange(batch) + 1000 * call, dtype=torch.int64, device="cuda:0")
        api.zinc_encrypt_noalloc(ctx, zc, z, 9, idx, out)
        ref = api.zinc_encrypt(ctx, zc, z, 9, idx)
        api.zn_sync_status(ctx)
        assert torch.equal(out, ref), call


def test_noalloc_refuses_batches_beyond_its_array():
    ctx, zc = _setup(14, (60, 50, 50, 60), 50)
    per_ct = 10 * ctx.n
    batch = api.NOALLOC_SCRATCH_BYTES // per_ct + 1
    z = torch.zeros((batch, 4), dtype=torch.float64, device="cuda:0")
    idx = torch.zeros((batch,), dtype=torch.int64, device="cuda:0")
    out = torch.full((batch, 2, ctx.L, ctx.n), 7, dtype=torch.int64, device="cuda:0")
    with pytest.raises(api.ZincError) as e:
        api.zinc_encrypt_noalloc(ctx, zc, z, 9, idx, out)
    assert e.value.status == api.ZN_ELIMIT
    assert bool((out == 7).all())                 # nothing was launched


def test_noalloc_takes_nothing_from_the_pool():
    """The defining property: the call draws no scratch from the context's
    memory pool.  With one pool allocation set to fail, the allocation-free
    call still succeeds and the next pooled call is the one refused."""
    ctx, zc = _setup(12, (36, 36, 36), 30)
    batch = 4
    w = workloads.small(12, (36, 36, 36), 30, batch, 100, seed=3)
    z = torch.tensor(workloads.slots(w), dtype=torch.float64, device="cuda:0")
    idx = torch.arange(batch, dtype=torch.int64, device="cuda:0")
    out = torch.empty((batch, 2, ctx.L, ctx.n), dtype=torch.int64, device="cuda:0")
    api.zn_inject_alloc_failures(1)
    try:
        api.zinc_encrypt_noalloc(ctx, zc, z, 9, idx, out)
        with pytest.raises(api.ZincError) as e:
            api.zinc_encrypt(ctx, zc, z, 9, idx)
        assert e.value.status == api.ZN_ENOMEM
    finally:
        api.zn_inject_alloc_failures(0)
    assert torch.equal(out, api.zinc_encrypt(ctx, zc, z, 9, idx))
