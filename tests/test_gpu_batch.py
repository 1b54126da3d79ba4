"""Mixed-ring batches (persistent launches, CUDA-graph replay): each job's
first and last ciphertext equal, residue for residue, the oracle's (Eq. 8 and
Algorithm 1 in the coefficient domain, then the definitional transform), and
every job's ciphertexts equal, bit for bit, those of the single-ring entry
points.  Ragged job sizes exercise partially filled packets (idle sub-groups)
and the persistent cluster kernels of 2^14 and 2^15 rings in both modes."""
import functools

import numpy as np
import pytest

from oracle import ckks as O
from paper_2408_07304_gb300 import api, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=None)
def ring(log_n, bits, ld):
    from paper_2408_07304_gb300 import build
    build.build()
    ctx = api.Context(log_n, bits, ld, device=0)
    sk, pk = api.ckks_keygen(ctx, 1)
    zc = api.zinc_precompute(ctx, pk, 2)
    return ctx, sk, pk, zc


JOBS = [  # (log_n, bits, log2_delta, zinc, count, n_slots)
    (12, (36, 36, 36), 30, False, 5, 2048),
    (12, (36, 36, 36), 30, True, 3, 100),
    (13, (60, 40, 40, 60), 40, True, 7, 4096),
    (14, (60, 50, 50, 60), 50, False, 2, 8192),
    (14, (60, 50, 50, 60), 50, True, 3, 5000),
    (15, (55, 55, 60), 55, False, 1, 16384),
    (15, (55, 55, 60), 55, True, 2, 3000),
    (10, (40, 41), 30, True, 17, 512),
    (11, (45, 45), 35, False, 9, 0),
]


def _make(seed_shift=0):
    jobs, refs = [], []
    for k, (log_n, bits, ld, zinc, count, ns) in enumerate(JOBS):
        ctx, sk, pk, zc = ring(log_n, bits, ld)
        w = workloads.small(log_n, bits, ld, count, ns, seed=100 + k + seed_shift)
        z = torch.tensor(workloads.slots(w), dtype=torch.float64, device="cuda:0")
        idx = torch.tensor(np.arange(count) * 3 + k * 1000, dtype=torch.int64, device="cuda:0")
        out = torch.full((count, 2, ctx.L, ctx.n), -1, dtype=torch.int64, device="cuda:0")
        jobs.append({"ctx": ctx, "zinc": zinc, "key": zc if zinc else pk, "slots": z, "seed": 7 + k,
                     "ct_index": idx, "out": out})
    return jobs


def _reference(j):
    fn = api.zinc_encrypt if j["zinc"] else api.ckks_encrypt
    return fn(j["ctx"], j["key"], j["slots"], j["seed"], j["ct_index"])


@pytest.mark.parametrize("graph", [False, True])
def test_batch_matches_single_ring(graph):
    jobs = _make()
    b = api.zn_batch_create(jobs)
    expect_packets = 0
    for log_n, bits, _, _, count, _ in JOBS:
        # 2^(13 - log_n) limbs per 256-thread block below 2^14; one limb per
        # two-CTA cluster at 2^14 and per four-CTA cluster at 2^15
        per = 1 << (13 - log_n) if log_n <= 13 else 1
        expect_packets += len(bits) * (-(-count // per) if log_n <= 13 else count)
    assert b.prep_units == sum(j[4] for j in JOBS) and b.packets == expect_packets
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        api.zn_batch_run(b, s, graph=graph)
        api.zn_batch_run(b, s, graph=graph)          # a replay gives the same result
    s.synchronize()
    for j in jobs:
        api.zn_sync_status(j["ctx"])
        assert torch.equal(j["out"], _reference(j)), (j["ctx"].log_n, j["zinc"])


@functools.lru_cache(maxsize=None)
def oracle_ring(log_n, bits, ld):
    P = O.Params(log_n, bits, ld)
    K = O.keygen(P, 1)
    return P, K, O.zinc_precompute_coeff(P, K, 2)


def test_batch_matches_oracle():
    """The persistent kernels' own results (one graph launch) against the
    oracle: the first and the last ciphertext of every job, all residues."""
    jobs = _make()
    b = api.zn_batch_create(jobs)
    s = torch.cuda.Stream()
    api.zn_batch_run(b, s, graph=True)
    s.synchronize()
    for k, (j, (log_n, bits, ld, zinc, count, ns)) in enumerate(zip(jobs, JOBS)):
        api.zn_sync_status(j["ctx"])
        P, K, zero = oracle_ring(log_n, bits, ld)
        assert P.primes == j["ctx"].primes
        z = j["slots"].cpu().numpy()
        idx = j["ct_index"].cpu().numpy()
        got = api.as_u64(j["out"])
        for r in sorted({0, count - 1}):
            if zinc:
                ref = O.ct_ntt(P, O.zinc_encrypt_coeff(P, zero, z[r], j["seed"], int(idx[r])))
            else:
                ref = O.ct_ntt(P, O.encrypt_coeff(P, K, z[r], j["seed"], int(idx[r])))
            assert np.array_equal(got[r], ref), (log_n, zinc, r)


def test_batch_graph_sees_new_inputs():
    jobs = _make()
    b = api.zn_batch_create(jobs)
    s = torch.cuda.Stream()
    api.zn_batch_run(b, s, graph=True)
    s.synchronize()
    fresh = _make(seed_shift=50)
    for j, f in zip(jobs, fresh):          # same buffers, new contents
        j["slots"].copy_(f["slots"])
        j["ct_index"].add_(1)
    api.zn_batch_run(b, s, graph=True)
    s.synchronize()
    for j in jobs:
        assert torch.equal(j["out"], _reference(j))


def test_batch_rejects_bad_jobs():
    ctx, _, pk, zc = ring(12, (36, 36, 36), 30)
    z = torch.zeros((1, 8), dtype=torch.float64, device="cuda:0")
    idx = torch.zeros((1,), dtype=torch.int64, device="cuda:0")
    out = torch.empty((1, 2, ctx.L, ctx.n), dtype=torch.int64, device="cuda:0")
    with pytest.raises(api.ZincError):       # a vanilla job carrying a cache instead of a key
        api.zn_batch_create([{"ctx": ctx, "zinc": False, "key": zc, "slots": z, "seed": 0,
                              "ct_index": idx, "out": out}])
    tiny = api.Context(9, (40,), 20)          # below the batch kernel's smallest ring
    tpk = api.ckks_keygen(tiny, 1)[1]
    with pytest.raises(api.ZincError):
        api.zn_batch_create([{"ctx": tiny, "zinc": False, "key": tpk, "slots": z, "seed": 0, "ct_index": idx,
                              "out": torch.empty((1, 2, 1, 512), dtype=torch.int64, device="cuda:0")}])


@pytest.mark.parametrize("pinned,log_n,bits", [(True, 13, (60, 40, 40, 60)), (False, 13, (60, 40, 40, 60)),
                                               (True, 14, (60, 50, 60))])
def test_host_pipeline_matches_device_api(pinned, log_n, bits):
    """zn_encrypt_host (host buffers, chunked copy/compute overlap on three
    streams) gives the device entry points' ciphertexts, with a ragged last
    chunk; at 2^14 the chunks' cluster kernels run concurrently."""
    ctx, _, pk, zc = ring(log_n, bits, 40)
    B, ns = 37, 1500
    w = workloads.small(log_n, bits, 40, B, ns, seed=77)
    z = torch.tensor(workloads.slots(w), dtype=torch.float64)
    idx = torch.arange(B, dtype=torch.int64) * 5 + 3
    if pinned:
        z, idx = z.pin_memory(), idx.pin_memory()
    for key, fn in ((pk, api.ckks_encrypt), (zc, api.zinc_encrypt)):
        out = torch.empty((B, 2, ctx.L, ctx.n), dtype=torch.int64, pin_memory=pinned)
        api.zn_encrypt_host(ctx, key, z, 4, idx, out, chunk=8)
        ref = fn(ctx, key, z.cuda(), 4, idx.cuda()).cpu()
        assert torch.equal(out, ref)
