"""Continuous-batching encryption server on one GPU.

Requests (a ring, a mode -- vanilla CKKS or Zinc -- and a slot vector of any
length up to N/2) arrive over time.  The server keeps every ring's public key
and Zinc cache resident on the device and runs an event loop:

* arrived requests join a queue per (ring, mode);
* whenever a CUDA stream is free and the HBM budget allows, the queue whose
  head has waited longest is cut into a batch (up to ``max_batch``
  requests), its slots staged in rows of the batch's longest vector with
  each request's own slot count (the per-vector count entry points: a
  request's missing slots are zero, so its ciphertext is the same as alone)
  and copied on that stream, and the encryption launched on the same stream;
* batches on different streams overlap on the device; a batch's HBM
  reservation (slots, ciphertexts, scratch) is released when its completion
  event fires, which admits the next requests;
* a launch refused for lack of device memory (``ZN_ENOMEM``: the budget is
  an estimate, the pool is shared) puts its batch back at the head of its
  queue, in arrival order, to be retried after the next completion -- or,
  with nothing in flight, after a short pause, at most ``max_alloc_retries``
  times in a row; any other error, or running out of retries, fails only
  that batch's requests, which are reported and not retried.

Each request's ciphertext depends only on (key, seed, request id, slots):
the request id is the Philox ct_index, so a result is bit-identical whether
the request ran alone or in any mix.  Latency is measured on the device
timeline, from the request's arrival to its ciphertext being complete in
HBM; the host copy of results is not part of it.
"""
import argparse
import collections
import dataclasses
import json
import time

import numpy as np

from . import api, workloads

RINGS = {"n8192": "batched", "n16384": "throughput", "n32768": "large"}


@dataclasses.dataclass
class Request:
    rid: int
    ring: str
    zinc: bool
    slots: np.ndarray
    arrival: float          # seconds after the start of the run


@dataclasses.dataclass
class Done:
    rid: int
    ring: str
    zinc: bool
    arrival: float
    finish: float           # seconds, device timeline
    ct: object = None       # device tensor [2, L, N] when results are kept


def poisson_requests(n, rate, seed=5, weights=(0.5, 0.3, 0.2), zinc_frac=0.8):
    """Synthetic request stream: exponential inter-arrival gaps at `rate`
    requests/s (all at t = 0 if rate is None), ring drawn from 2^13 / 2^14 /
    2^15 with `weights`, 1..N/2 slots U[-1, 1], Zinc with probability
    `zinc_frac`."""
    rng = np.random.Generator(np.random.PCG64(seed))
    names = list(RINGS)
    t = 0.0
    out = []
    for rid in range(n):
        if rate:
            t += rng.exponential(1.0 / rate)
        ring = names[rng.choice(len(names), p=weights)]
        half = workloads.WORKLOADS[RINGS[ring]].n // 2
        ns = int(rng.integers(1, half + 1))
        out.append(Request(rid, ring, bool(rng.random() < zinc_frac), rng.uniform(-1.0, 1.0, ns), t))
    return out


class Server:
    def __init__(self, device=0, n_streams=4, max_batch=256, hbm_budget=16 << 30, seed=11, keep_results=False,
                 max_alloc_retries=100):
        import torch
        self.torch = torch
        self.max_alloc_retries = max_alloc_retries
        self.dev = torch.device("cuda", device)
        torch.cuda.set_device(self.dev)
        self.max_batch = max_batch
        self.budget = hbm_budget
        self.seed = seed
        self.keep = keep_results
        self.rings = {}
        for name, wname in RINGS.items():
            w = workloads.WORKLOADS[wname]
            ctx = api.Context(w.log_n, w.bits, w.log2_delta, device=device)
            sk, pk = api.ckks_keygen(ctx, workloads.KEYGEN_SEED)
            zc = api.zinc_precompute(ctx, pk, workloads.CACHE_SEED)
            self.rings[name] = (ctx, sk, pk, zc)
        self.streams = [torch.cuda.Stream(self.dev) for _ in range(n_streams)]

    def ct_bytes(self, ring):
        ctx = self.rings[ring][0]
        return 2 * ctx.L * ctx.n * 8

    def batch_bytes(self, ring, count, n_slots):
        ctx = self.rings[ring][0]
        # ciphertexts + staged slots + ct indices + prep scratch (int64 + 2 int8 per coefficient)
        return count * (self.ct_bytes(ring) + n_slots * 8 + 8 + 10 * ctx.n)

    def encrypt_one(self, req):
        """The same request alone (reference for the mixed run)."""
        torch = self.torch
        ctx, _, pk, zc = self.rings[req.ring]
        z = torch.tensor(req.slots[None, :], dtype=torch.float64, device=self.dev)
        idx = torch.tensor([req.rid], dtype=torch.int64, device=self.dev)
        fn = api.zinc_encrypt if req.zinc else api.ckks_encrypt
        return fn(ctx, zc if req.zinc else pk, z, self.seed, idx)[0]

    def run(self, requests):
        torch = self.torch
        reqs = sorted(requests, key=lambda r: r.arrival)
        pending = collections.deque(reqs)
        queues = collections.OrderedDict()
        free = list(range(len(self.streams)))
        inflight = []
        reserved = 0
        done = []
        failed = []             # (rid, status) of requests whose batch failed
        alloc_retries = 0
        enomem_streak = 0       # consecutive refusals with nothing in flight
        peak_inflight = 0
        peak_reserved = 0
        t_ref = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(self.dev)
        t_ref.record(torch.cuda.current_stream(self.dev))
        torch.cuda.synchronize(self.dev)
        t0 = time.perf_counter()
        while pending or inflight or any(queues.values()):
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now:
                r = pending.popleft()
                queues.setdefault((r.ring, r.zinc), collections.deque()).append(r)
            # retire finished batches (frees streams and HBM reservation)
            still = []
            for f in inflight:
                ev, si, batch, nbytes, out = f
                if ev.query():
                    finish = t_ref.elapsed_time(ev) / 1e3
                    for k, r in enumerate(batch):
                        done.append(Done(r.rid, r.ring, r.zinc, r.arrival, finish, out[k] if self.keep else None))
                    reserved -= nbytes
                    free.append(si)
                else:
                    still.append(f)
            inflight = still
            # launch while a stream and budget are available
            launched = False
            refused = False
            while free and not refused:
                heads = [(q[0].arrival, key) for key, q in queues.items() if q]
                if not heads:
                    break
                _, key = min(heads)
                q = queues[key]
                ring, zinc = key
                batch = []
                ns = 0
                while q and len(batch) < self.max_batch:
                    r = q[0]
                    cand = max(ns, r.slots.shape[0])
                    if self.batch_bytes(ring, len(batch) + 1, cand) > self.budget - reserved:
                        break
                    batch.append(q.popleft())
                    ns = cand
                if not batch:
                    break           # over budget: wait for a completion
                si = free.pop()
                nbytes = self.batch_bytes(ring, len(batch), ns)
                try:
                    out = self._launch(self.streams[si], ring, zinc, batch, ns)
                except api.ZincError as e:
                    free.append(si)
                    if e.status == api.ZN_ENOMEM and (inflight or enomem_streak < self.max_alloc_retries):
                        q.extendleft(reversed(batch))       # retried first, arrival order kept
                        alloc_retries += 1
                        enomem_streak += 0 if inflight else 1
                        refused = True                      # wait for a completion (or a pause)
                    else:
                        failed.extend((r.rid, e.status) for r in batch)
                    continue
                enomem_streak = 0
                reserved += nbytes
                peak_reserved = max(peak_reserved, reserved)
                ev = torch.cuda.Event(enable_timing=True)
                ev.record(self.streams[si])
                inflight.append((ev, si, batch, nbytes, out))
                peak_inflight = max(peak_inflight, len(inflight))
                launched = True
            if refused and not inflight:
                time.sleep(1e-3)    # a pool short with nothing in flight: pause before the retry
            elif not launched:
                if pending and not inflight and not any(queues.values()):
                    time.sleep(max(0.0, min(pending[0].arrival - (time.perf_counter() - t0), 1e-3)))
                else:
                    time.sleep(20e-6)
        torch.cuda.synchronize(self.dev)
        wall = time.perf_counter() - t0
        return done, {"wall_s": wall, "peak_inflight_batches": peak_inflight, "peak_reserved_bytes": peak_reserved,
                      "failed": failed, "alloc_retries": alloc_retries}

    def _launch(self, stream, ring, zinc, batch, ns):
        torch = self.torch
        ctx, _, pk, zc = self.rings[ring]
        B = len(batch)
        # rows of the longest vector, entries past a request's count left as
        # they are (never read)
        host = torch.empty((B, ns), dtype=torch.float64, pin_memory=True)
        hv = host.numpy()
        for k, r in enumerate(batch):
            hv[k, : r.slots.shape[0]] = r.slots
        hidx = torch.tensor([r.rid for r in batch], dtype=torch.int64).pin_memory()
        hcnt = torch.tensor([r.slots.shape[0] for r in batch], dtype=torch.int32).pin_memory()
        with torch.cuda.stream(stream):
            z = host.to(self.dev, non_blocking=True)
            idx = hidx.to(self.dev, non_blocking=True)
            cnt = hcnt.to(self.dev, non_blocking=True)
            out = torch.empty((B, 2, ctx.L, ctx.n), dtype=torch.int64, device=self.dev)
            fn = api.zinc_encrypt_ragged if zinc else api.ckks_encrypt_ragged
            fn(ctx, zc if zinc else pk, z, cnt, self.seed, idx, out=out, stream=stream)
            # keep the staging buffers alive until the stream has consumed them
            z.record_stream(stream)
            idx.record_stream(stream)
            cnt.record_stream(stream)
        out._staging = (host, hidx, hcnt)
        return out


def summarize(done, info, n_requests):
    lat = np.array([d.finish - d.arrival for d in done]) * 1e3
    by_ring = collections.Counter(d.ring for d in done)
    return {"requests": n_requests, "completed": len(done), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "enc_per_s": len(done) / info["wall_s"], "wall_s": info["wall_s"],
            "zinc_fraction": float(np.mean([d.zinc for d in done])), "per_ring": dict(by_ring),
            "peak_inflight_batches": info["peak_inflight_batches"],
            "peak_reserved_gib": info["peak_reserved_bytes"] / 2 ** 30,
            "failed": len(info.get("failed", ())), "alloc_retries": info.get("alloc_retries", 0)}


def serve_benchmark(n_requests=20000, load=0.7, device=0, seed=5, **kw):
    """Measure the mixed capacity (all requests at t = 0), then run a Poisson
    stream at `load` x that capacity; returns both summaries."""
    srv = Server(device=device, **kw)
    cap_reqs = poisson_requests(min(n_requests, 5000), None, seed=seed + 1)
    srv.run(cap_reqs[:256])                                 # warm-up
    done, info = srv.run(cap_reqs)
    capacity = summarize(done, info, len(cap_reqs))
    rate = load * capacity["enc_per_s"]
    reqs = poisson_requests(n_requests, rate, seed=seed)
    done, info = srv.run(reqs)
    stream = summarize(done, info, n_requests)
    stream["rate_per_s"] = rate
    stream["load"] = load
    return {"capacity_enc_per_s": capacity["enc_per_s"], "stream": stream}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--requests", type=int, default=20000)
    ap.add_argument("--load", type=float, default=0.7)
    ap.add_argument("--streams", type=int, default=4)
    ap.add_argument("--max-batch", type=int, default=256)
    ap.add_argument("--budget-gib", type=float, default=16.0)
    a = ap.parse_args()
    r = serve_benchmark(a.requests, a.load, n_streams=a.streams, max_batch=a.max_batch,
                        hbm_budget=int(a.budget_gib * 2 ** 30))
    print(json.dumps(r))


if __name__ == "__main__":
    main()
