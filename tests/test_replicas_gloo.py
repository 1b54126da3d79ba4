"""The multi-GPU path is replicas: each rank encrypts its own ct_index range,
no collective touches the data, and the timings are reduced by a maximum.
Two gloo ranks on the CPU check, with the oracle on a tiny ring, that the
union of the ranks' ciphertexts equals one process encrypting the whole
range (the randomness is keyed by ct_index, not by rank or batch position),
and that the timing reduction is the element-wise maximum.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

WORLD, B = 2, 3
LOG_N, BITS, LD, SEED = 4, (30, 31), 20, 9


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _encrypt_range(lo, hi):
    from oracle import ckks as O
    from paper_2408_07304_gb300 import workloads
    P = O.Params(LOG_N, BITS, LD)
    K = O.keygen(P, 1)
    zero = O.zinc_precompute_coeff(P, K, 2)
    w = workloads.small(LOG_N, BITS, LD, WORLD * B, 5, seed=4)
    z = workloads.slots(w, batch=hi - lo, first=lo)
    out = []
    for b, ct_index in enumerate(range(lo, hi)):
        out.append(O.ct_ntt(P, O.encrypt_coeff(P, K, z[b], SEED, ct_index)))
        out.append(O.ct_ntt(P, O.zinc_encrypt_coeff(P, zero, z[b], SEED, ct_index)))
    return np.stack(out)


def _worker(rank, port, results):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        lo, hi = bench.replica_range(rank, B)
        cts = _encrypt_range(lo, hi)
        timings = bench.max_over_ranks([1.0 + rank, 10.0 - 3 * rank], WORLD, "cpu", dist)
        gathered = [None] * WORLD
        dist.all_gather_object(gathered, (rank, lo, hi, cts))
        if rank == 0:
            results.put((timings, gathered))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_replicas_equal_one_process_and_timing_is_max():
    ctx = mp.get_context("spawn")
    results = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, port, results)) for r in range(WORLD)]
    for p in procs:
        p.start()
    timings, gathered = results.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert timings == [2.0, 10.0]
    gathered.sort(key=lambda g: g[0])
    ranges = [(lo, hi) for _, lo, hi, _ in gathered]
    assert ranges == [(0, B), (B, 2 * B)]                       # disjoint, covering [0, WORLD B)
    union = np.concatenate([g[3] for g in gathered])
    assert np.array_equal(union, _encrypt_range(0, WORLD * B))
