#!/usr/bin/env python
"""Benchmark: RNS-CKKS public-key encryptions per second on GB300, vanilla
(Eq. 8) and Zinc (Algorithm 1), at N = 2^14 (60 + 6 x 50 + 60-bit chain,
Delta = 2^50, 4096 vectors of 8192 slots U[-1, 1]) by default.

One step = encrypt the whole batch once with vanilla CKKS and once with Zinc
(encoding, sampling, NTTs and the key multiply-add / cache add all inside),
inputs resident in HBM.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...   (the CPU oracle on a bounded sample)

Multi-GPU: one process per GPU (torchrun); every rank runs an independent
replica on its own ct_index range (no collective on the data path).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2408_07304_gb300 import workloads  # noqa: E402

METRIC = "encryptions/s, vanilla CKKS vs Zinc, at N=2^14, 1 GB300; HBM roofline %; p99 ms"
UNIT = "encryptions/s"


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per ciphertext
# of the encrypt kernels, from separate ncu captures (not measured by this
# run): a 512-ciphertext launch of the throughput workload (N = 2^14) and a
# 64-ciphertext launch of the paper-shaped one (N = 2^15), keyed by the kernel
# each was taken on and scaled to the launch size timed here (a 256-ciphertext
# capture at N = 2^14 gave 2.7 % less per ciphertext: part of a smaller
# launch's output is still in L2 when it ends).  Valid only while that kernel
# is unchanged and selected.
NCU_TRAFFIC_PER_CT = {
    ("throughput", "k_encrypt_pair<vanilla,2-CTA cluster,radix-8,3 blocks/SM>"): (99.60192e6 + 1098.81e6) / 512,
    ("paper", "k_encrypt_quarter<vanilla,4-CTA cluster,radix-8,3 blocks/SM>"): (51.4816e6 + 481.318912e6) / 64,
}
# Busy fraction of the SM's integer multiply-add pipe (ncu
# sm__pipe_fmaheavy_cycles_active, which is also the kernel's
# sm__throughput: the busiest unit of the SM) in the same captures.
NCU_INT_PIPE = {
    ("throughput", "k_encrypt_pair<vanilla,2-CTA cluster,radix-8,3 blocks/SM>"): 0.7209,
    ("paper", "k_encrypt_quarter<vanilla,4-CTA cluster,radix-8,3 blocks/SM>"): 0.7392,
}
VARIANT_KERNEL = {6: "k_encrypt_pair<{mode},2-CTA cluster,radix-8,3 blocks/SM>",
                  7: "k_encrypt_pair<{mode},2-CTA cluster,radix-8,3 blocks/SM,ciphertext-major>"}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        try:
            with open(self.path) as f:
                for ln in f:
                    p = [x.strip() for x in ln.split(",")]
                    if len(p) >= 9:
                        rows.append(p)
            os.unlink(self.path)
        except Exception:
            return None
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------- CPU oracle
def oracle_setup(w):
    """Keys and Zinc cache of the CPU oracle for workload `w` (untimed)."""
    from oracle import ckks as O
    P = O.Params(w.log_n, w.bits, w.log2_delta)
    K = O.keygen(P, workloads.KEYGEN_SEED)
    zero = O.zinc_precompute_coeff(P, K, workloads.CACHE_SEED)
    return P, K, zero, workloads.slots(w, batch=1)[0]


def oracle_sample(w, setup, reps=1):
    """Time the CPU oracle on a bounded sample of workload `w`: one vanilla and
    one Zinc ciphertext of the workload, every prime (encode, sampling,
    schoolbook products, definitional NTT of both components).  Returns
    (seconds per sample, threads used, description)."""
    from oracle import ckks as O
    from oracle import ring
    P, K, zero, z = setup
    t0 = time.perf_counter()
    for r in range(reps):
        O.ct_ntt(P, O.encrypt_coeff(P, K, z, w.seed, r))
        O.ct_ntt(P, O.zinc_encrypt_coeff(P, zero, z, w.seed, r))
    dt = (time.perf_counter() - t0) / reps
    desc = f"one vanilla + one Zinc ciphertext of the {w.name} workload (N={w.n}, {w.L} primes), all residues"
    return dt, ring.threads(), desc


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    setup = oracle_setup(w)
    for _ in range(args.warmup):
        oracle_sample(w, setup)
    times = []
    for _ in range(args.steps):
        dt, cores, desc = oracle_sample(w, setup)
        times.append(dt)
    per_step = sum(times) / len(times)
    value = 2.0 / per_step
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": {"workload": f"{w.name}: {w.describe()}", "parallelism": "cpu oracle"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ replicas
def replica_range(rank, batch):
    """ct_index range [rank * batch, (rank + 1) * batch) of one replica.
    Encryptions are independent and their randomness is keyed by ct_index,
    so the ranks share no data and no collective runs on the data path."""
    return rank * batch, (rank + 1) * batch


def max_over_ranks(values, world, device, dist=None):
    """Element-wise maximum of per-rank timings (all_reduce MAX when world > 1)."""
    import torch
    t = torch.tensor(values, dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


# ------------------------------------------------------------------ GPU arm
def butterflies_per_ct(w, zinc):
    """Algorithmic butterflies per ciphertext: (N/2) log2 N per NTT, 3 NTTs per
    prime (vanilla: m + e0, u, e1) or 2 (Zinc: m + e1', e2')."""
    return w.L * (2 if zinc else 3) * (w.n // 2) * w.log_n


def key_products_per_ct(w, zinc):
    """Pointwise key products per ciphertext: pk0 u and pk1 u per prime (vanilla)."""
    return 0 if zinc else 2 * w.L * w.n


def decode_error(api, ctx, sk, ct, slots, chunk=256):
    """Measured decrypt-decode error of a batch of ciphertexts against the
    slot vectors they encrypt: max and RMS over every slot (absolute), and the
    max relative to max |z|."""
    import torch
    B, ns = slots.shape
    mx, ss = 0.0, 0.0
    for b0 in range(0, B, chunk):
        back = api.ckks_decrypt_decode(ctx, sk, ct[b0:b0 + chunk].contiguous(), ns)
        d = (back - slots[b0:b0 + chunk]).abs()
        mx = max(mx, float(d.max()))
        ss += float((d * d).sum())
    zmax = float(slots.abs().max())
    return {"max": mx, "rms": (ss / (B * ns)) ** 0.5, "max_rel": mx / zmax if zmax else None,
            "ciphertexts": B, "slots_per_ct": ns}


def run_ours(args, w):
    import torch
    import torch.distributed as dist

    from paper_2408_07304_gb300 import api

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    ctx = api.Context(w.log_n, w.bits, w.log2_delta, device=local)
    sk, pk = api.ckks_keygen(ctx, workloads.KEYGEN_SEED)
    zc = api.zinc_precompute(ctx, pk, workloads.CACHE_SEED)
    B = w.batch
    lo, hi = replica_range(rank, B)
    z = workloads.slots(w, batch=B, first=lo)
    slots = torch.tensor(z, dtype=torch.float64, device=dev)
    idx = torch.arange(lo, hi, dtype=torch.int64, device=dev)
    out_v = torch.empty((B, 2, w.L, w.n), dtype=torch.int64, device=dev)
    out_z = torch.empty_like(out_v)
    stream = torch.cuda.current_stream(dev)
    if args.variant is None:
        tune = api.zn_autotune(ctx, pk, zc, min(B, 512))
    else:
        api.zn_set_variant(ctx, args.variant)
        tune = (args.variant, None)

    def step():
        api.ckks_encrypt(ctx, pk, slots, w.seed, idx, out=out_v, stream=stream)
        api.zinc_encrypt(ctx, zc, slots, w.seed, idx, out=out_z, stream=stream)

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        step()
    api.zn_sync_status(ctx, stream)
    torch.cuda.synchronize(dev)
    barrier()

    # ---- device-timed steps (inputs resident in HBM)
    api.zn_timing_enable(ctx, True)
    clocks = ClockSampler(local)
    clocks.start()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps + 1)]
    torch.cuda.synchronize(dev)
    barrier()
    evs[0].record(stream)
    for k in range(args.steps):
        api.ckks_encrypt(ctx, pk, slots, w.seed, idx, out=out_v, stream=stream)
        evs[2 * k + 1].record(stream)
        api.zinc_encrypt(ctx, zc, slots, w.seed, idx, out=out_z, stream=stream)
        evs[2 * k + 2].record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    clk = clocks.stop()
    total_ms = evs[0].elapsed_time(evs[-1])
    van_ms = sum(evs[2 * k].elapsed_time(evs[2 * k + 1]) for k in range(args.steps))
    zin_ms = sum(evs[2 * k + 1].elapsed_time(evs[2 * k + 2]) for k in range(args.steps))
    enc_ms, enc_n = api.zn_timing_read(ctx, api.TIME_ENCODE)
    kv_ms, kv_n = api.zn_timing_read(ctx, api.TIME_ENCRYPT)
    kz_ms, kz_n = api.zn_timing_read(ctx, api.TIME_ZINC)
    api.zn_timing_enable(ctx, False)
    api.zn_sync_status(ctx, stream)
    launches = enc_n + kv_n + kz_n

    total_ms, van_ms, zin_ms = max_over_ranks([total_ms, van_ms, zin_ms], world, dev, dist)
    cts = 2 * B * world * args.steps
    value = cts / (total_ms / 1e3)
    van_rate = B * world * args.steps / (van_ms / 1e3)
    zin_rate = B * world * args.steps / (zin_ms / 1e3)

    # ---- measured decryption accuracy of every ciphertext of the last step,
    # per mode (Theorem 1: Zinc adds e1' + e2' s to the cached zero's noise)
    sig = 3.2
    accuracy = {"vanilla": decode_error(api, ctx, sk, out_v, slots),
                "zinc": decode_error(api, ctx, sk, out_z, slots),
                "bound": (10 * w.n * sig + w.n) / 2.0 ** w.log2_delta * max(abs(w.lo), abs(w.hi)),
                "bound_formula": "(10 N sigma + N) / Delta x max|z|"}
    accuracy["zinc_over_vanilla_rms"] = accuracy["zinc"]["rms"] / accuracy["vanilla"]["rms"]

    # ---- roofline of the dominant kernel (the vanilla encrypt kernel): its
    # algorithmic HBM bytes (ciphertexts written + slots read, per ciphertext)
    # over its event-timed launch duration against the measured copy peak.
    # The kernel is bound by 64-bit modular arithmetic on the integer pipes,
    # so it is also reported against (a) the probe-measured ceiling of the
    # same butterfly running from registers and (b) a peak derived from unit
    # counts and clocks -- SMs x 64 32-bit IMAD/clk x 2.07 GHz at 10 IMAD per
    # Harvey/Shoup butterfly (an assumption: a 64 x 64 high product = 4, two
    # 64-bit low products = 3 each).
    hbm_peak, peak_src = peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    derived_peak = sms * 64 * 2.07e9 / 10 / 1e9          # Gbutterfly/s
    # practical ceiling: the probe rates of the two butterfly forms, weighted by
    # the share of the workload's butterflies on primes below 2^59 (relaxed)
    probe_h = api.zn_probe_butterfly(local) / 1e9
    probe_r = api.zn_probe_butterfly_relaxed(local) / 1e9
    f_rel = sum(1 for q in ctx.primes if q < (1 << 59)) / w.L
    probe = 1.0 / (f_rel / probe_r + (1.0 - f_rel) / probe_h)
    ct_bytes = 2 * w.L * w.n * 8
    per_ct_bytes = ct_bytes + w.n_slots * 8
    chunk_cts = B * args.steps / max(kv_n, 1)
    kv_avg = kv_ms / max(kv_n, 1)
    kz_avg = kz_ms / max(kz_n, 1)
    bfly_v = chunk_cts * butterflies_per_ct(w, False)
    bfly_z = chunk_cts * butterflies_per_ct(w, True)
    kprod_v = chunk_cts * key_products_per_ct(w, False)
    alg_bytes = chunk_cts * per_ct_bytes
    hbm_achieved = alg_bytes / (kv_avg / 1e3) / 1e9
    hbm_achieved_z = alg_bytes / (kz_avg / 1e3) / 1e9
    achieved = bfly_v / (kv_avg / 1e3) / 1e9
    if w.log_n == 14:
        kname = VARIANT_KERNEL.get(tune[0], "k_encrypt<{mode}> variant %d" % tune[0])
    elif w.log_n == 15 and tune[0] in (6, 7):
        kname = "k_encrypt_quarter<{mode},4-CTA cluster,radix-8,3 blocks/SM>"
    else:
        kname = f"k_encrypt<{w.log_n},{{mode}}> variant {tune[0]}"
    per_ct_traffic = NCU_TRAFFIC_PER_CT.get((w.name, kname.format(mode="vanilla")))
    traffic = per_ct_traffic * chunk_cts if per_ct_traffic else None
    int_pipe = NCU_INT_PIPE.get((w.name, kname.format(mode="vanilla")))
    roofline = {"bound": "hbm", "achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": hbm_achieved / hbm_peak, "traffic": traffic,
                "traffic_source": "ncu capture of this kernel (512 ciphertexts at N=2^14, 64 at the paper's "
                                  "parameters), taken separately (not by this run), scaled per ciphertext to this "
                                  "launch size; null when the selected kernel has none",
                "traffic_over_algorithmic": (traffic / alg_bytes) if traffic else None,
                "algorithmic_bytes_per_launch": alg_bytes, "ciphertexts_per_launch": chunk_cts,
                "algorithmic_bytes_per_ct": per_ct_bytes,
                "kernel": kname.format(mode="vanilla") + f" (variant {tune[0]})",
                "peak_source": f"{peak_src} HBM copy rate (hbm_gbs)",
                "zinc_kernel": {"achieved": hbm_achieved_z, "frac": hbm_achieved_z / hbm_peak,
                                "ms_per_launch": kz_avg},
                "alu": {"note": "the kernel's binding unit: 64-bit modular products on the integer pipes",
                        "unit": "Gbutterfly/s", "butterflies_per_ct": butterflies_per_ct(w, False),
                        "key_products_per_ct": key_products_per_ct(w, False),
                        "achieved": achieved, "achieved_with_key_products": (bfly_v + kprod_v) / (kv_avg / 1e3) / 1e9,
                        "probe_peak": probe, "probe_frac": achieved / probe,
                        "probe_frac_with_key_products": (bfly_v + kprod_v) / (kv_avg / 1e3) / 1e9 / probe,
                        "probe_source": "measured: the same butterfly from registers on every SM "
                                        "(zn_probe_butterfly / _relaxed, weighted by the chain's prime mix)",
                        "probe_harvey": probe_h, "probe_relaxed": probe_r, "relaxed_prime_share": f_rel,
                        "derived_peak": derived_peak, "derived_frac": achieved / derived_peak,
                        "derived_source": "assumption: SMs x 64 IMAD/clk x 2.07 GHz / 10 IMAD per butterfly",
                        "zinc_kernel_achieved": bfly_z / (kz_avg / 1e3) / 1e9,
                        "zinc_kernel_probe_frac": bfly_z / (kz_avg / 1e3) / 1e9 / probe,
                        "int_pipe": {"pipe": "fmaheavy (32-bit integer multiply-add)", "busy_frac": int_pipe,
                                     "source": "ncu sm__pipe_fmaheavy_cycles_active of the same capture as "
                                               "traffic (not this run)"}}}

    # ---- the same step through the mixed-ring persistent path (one CUDA-graph
    # launch per step: a vanilla job and a Zinc job over the batch)
    persistent = None
    if not args.no_persistent:
        b = api.zn_batch_create([
            {"ctx": ctx, "zinc": False, "key": pk, "slots": slots, "seed": w.seed, "ct_index": idx, "out": out_v},
            {"ctx": ctx, "zinc": True, "key": zc, "slots": slots, "seed": w.seed, "ct_index": idx, "out": out_z}],
            device=local)
        gs = torch.cuda.Stream(dev)
        for _ in range(args.warmup):
            api.zn_batch_run(b, gs, graph=True)
        torch.cuda.synchronize(dev)
        barrier()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(gs)
        for _ in range(args.steps):
            api.zn_batch_run(b, gs, graph=True)
        g1.record(gs)
        torch.cuda.synchronize(dev)
        gms = g0.elapsed_time(g1)
        persistent = {"enc_per_s": 2 * B * args.steps / (gms / 1e3), "ms_per_step": gms / args.steps,
                      "prep_units": b.prep_units, "packets": b.packets, "graph_launches_per_step": 1}
        b.close()

    # ---- end to end through the host-buffer entry point: every step copies
    # the slot vectors and ct indices in (once per mode) and every ciphertext
    # out, pipelined in chunks over three streams
    e2e = None
    if not args.no_e2e:
        e2e_steps = max(1, min(2 * args.steps, 21))
        host_slots = torch.tensor(z, dtype=torch.float64).pin_memory()
        host_idx = idx.cpu().pin_memory()
        host_v = torch.empty(out_v.shape, dtype=torch.int64, pin_memory=True)
        host_z = torch.empty(out_z.shape, dtype=torch.int64, pin_memory=True)
        api.zn_encrypt_host(ctx, pk, host_slots, w.seed, host_idx, host_v)      # warm-up, both modes
        api.zn_encrypt_host(ctx, zc, host_slots, w.seed, host_idx, host_z)      # (first touch of each buffer)
        torch.cuda.synchronize(dev)
        # the device-to-host link of this machine, copied the way the entry point
        # copies (chunks of 256 ciphertexts over three streams, into the same
        # pinned buffer): the end-to-end rate cannot exceed it
        cstreams = [torch.cuda.Stream(dev) for _ in range(3)]

        def copy_pass(dsts):
            """Seconds to copy the device ciphertexts into `dsts` (one buffer
            per mode) with the entry point's copy pattern, copies only."""
            torch.cuda.synchronize(dev)
            l0 = time.perf_counter()
            k = 0
            for src, dst in dsts:
                for c0 in range(0, B, 256):
                    with torch.cuda.stream(cstreams[k % 3]):
                        dst[c0:c0 + 256].copy_(src[c0:c0 + 256], non_blocking=True)
                    k += 1
            torch.cuda.synchronize(dev)
            return time.perf_counter() - l0

        def link_probe(reps=3):
            # the best of a few: other tenants' traffic only slows a copy down
            return max(host_v.numel() * 8 / copy_pass([(out_v, host_v)]) / 1e9 for _ in range(reps))

        # the same step with the ciphertexts packed on the device (residues at
        # their primes' bit lengths, zn_encrypt_host_packed): fewer bytes on
        # the link, every value kept
        pw = api.zn_ct_packed_words(ctx)
        # the packed outputs reuse the front of the plain buffers (no second
        # set of page-locked gigabytes)
        host_pv = host_v.view(-1)[: B * pw].view(B, pw)
        host_pz = host_z.view(-1)[: B * pw].view(B, pw)
        api.zn_encrypt_host_packed(ctx, pk, host_slots, w.seed, host_idx, host_pv)
        api.zn_encrypt_host_packed(ctx, zc, host_slots, w.seed, host_idx, host_pz)
        torch.cuda.synchronize(dev)
        link_before = link_probe()
        barrier()
        # each step timed on its own, the plain and the packed format in
        # alternation: the host link of these boxes is shared with other
        # tenants and fluctuates, so each value is the median step of its
        # format over the same stretch of time
        # a third, copy-only step moves the plain step's device-to-host bytes
        # with the same copy pattern and no kernels: the link's own rate over
        # the same stretch of time
        step_s, p_step_s, c_step_s = [], [], []
        for _ in range(e2e_steps):
            t_start = time.perf_counter()
            api.zn_encrypt_host(ctx, pk, host_slots, w.seed, host_idx, host_v)
            api.zn_encrypt_host(ctx, zc, host_slots, w.seed, host_idx, host_z)
            step_s.append(time.perf_counter() - t_start)
            t_start = time.perf_counter()
            api.zn_encrypt_host_packed(ctx, pk, host_slots, w.seed, host_idx, host_pv)
            api.zn_encrypt_host_packed(ctx, zc, host_slots, w.seed, host_idx, host_pz)
            p_step_s.append(time.perf_counter() - t_start)
            c_step_s.append(copy_pass([(out_v, host_v), (out_z, host_z)]))
        step_s = max_over_ranks(step_s, world, dev, dist)
        p_step_s = max_over_ranks(p_step_s, world, dev, dist)
        c_step_s = max_over_ranks(c_step_s, world, dev, dist)
        copy_gbs = 2 * host_v.numel() * 8 * e2e_steps / sum(c_step_s) / 1e9
        link_after = link_probe()
        link_gbs = max(link_before, link_after)
        e2e_s = sum(step_s) / len(step_s)
        link_bound = link_gbs * 1e9 / (2 * w.L * w.n * 8)
        e2e = {"value": 2 * B * world * e2e_steps / sum(step_s), "unit": UNIT,
               "statistic": f"all ciphertexts of {e2e_steps} timed steps / their total time",
               "step_s": step_s, "median_enc_s": 2 * B * world / statistics.median(step_s),
               "d2h_link_gbs": link_gbs, "d2h_link_gbs_before_after": [link_before, link_after],
               "copy_only": {"step_s": c_step_s, "gbs": copy_gbs,
                             "median_gbs": 2 * host_v.numel() * 8 / statistics.median(c_step_s) / 1e9,
                             "what": "the plain step's device-to-host bytes, same copy pattern, no kernels, "
                                     "interleaved with the timed steps"},
               "of_copy_only_rate": (2 * B * e2e_steps / sum(step_s)) * (2 * w.L * w.n * 8) / (copy_gbs * 1e9),
               "link_bound_enc_s": link_bound * world,
               "of_link_bound": 2 * B / e2e_s / link_bound,
               "d2h_gbs_fastest_step": 2 * host_v.numel() * 8 / min(step_s) / 1e9,
               "h2d_bytes_per_step": int(2 * (host_slots.numel() * 8 + host_idx.numel() * 8)),
               "d2h_bytes_per_step": int(2 * host_v.numel() * 8),
               "steps": e2e_steps, "api": "zn_encrypt_host (pinned host buffers, automatic chunks (256 ciphertexts here) over 3 streams)",
               "packed": {"value": 2 * B * world * e2e_steps / sum(p_step_s), "unit": UNIT,
                          "statistic": f"all ciphertexts of {e2e_steps} timed steps / their total time, "
                                       "alternating with the plain ones",
                          "median_enc_s": 2 * B * world / statistics.median(p_step_s),
                          "step_s": p_step_s,
                          "d2h_bytes_per_step": int(2 * host_pv.numel() * 8),
                          "packed_over_plain_bytes": pw / (2 * w.L * w.n),
                          "api": "zn_encrypt_host_packed (ciphertexts bit-packed on the device, "
                                 "each residue in its prime's bit length; unpacked exactly by zn_ct_unpack)"}}
        del host_v, host_z, host_pv, host_pz

    # ---- SEAL's ordering, which the paper measured: the chain's last prime is
    # the special prime; modulus-switched vanilla encryption (key-level
    # encryption divided and rounded by p, message added at the data level)
    # against Zinc at the data level over a cache made the same way
    seal = None
    if not args.no_special and w.L >= 2:
        dctx = api.data_level(ctx)
        zc_d = api.zinc_precompute_ms(ctx, pk, workloads.CACHE_SEED, dctx)
        out_m = torch.empty((B, 2, w.L - 1, w.n), dtype=torch.int64, device=dev)
        out_mz = torch.empty_like(out_m)
        for _ in range(args.warmup):
            api.ckks_encrypt_ms(ctx, pk, slots, w.seed, idx, out=out_m, stream=stream)
            api.zinc_encrypt(dctx, zc_d, slots, w.seed, idx, out=out_mz, stream=stream)
        torch.cuda.synchronize(dev)
        barrier()
        api.zn_timing_enable(ctx, True)
        sev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps + 1)]
        sev[0].record(stream)
        for k in range(args.steps):
            api.ckks_encrypt_ms(ctx, pk, slots, w.seed, idx, out=out_m, stream=stream)
            sev[2 * k + 1].record(stream)
            api.zinc_encrypt(dctx, zc_d, slots, w.seed, idx, out=out_mz, stream=stream)
            sev[2 * k + 2].record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        ms_ms = sum(sev[2 * k].elapsed_time(sev[2 * k + 1]) for k in range(args.steps))
        mz_ms = sum(sev[2 * k + 1].elapsed_time(sev[2 * k + 2]) for k in range(args.steps))
        kp_ms, kp_n = api.zn_timing_read(ctx, api.TIME_ENCODE)
        ks_ms, ks_n = api.zn_timing_read(ctx, api.TIME_MS_SPECIAL)
        kd_ms, kd_n = api.zn_timing_read(ctx, api.TIME_MS_DATA)
        api.zn_timing_enable(ctx, False)
        api.zn_sync_status(ctx, stream)
        api.zn_sync_status(dctx, stream)
        ms_ms, mz_ms = max_over_ranks([ms_ms, mz_ms], world, dev, dist)
        ms_rate = B * world * args.steps / (ms_ms / 1e3)
        mz_rate = B * world * args.steps / (mz_ms / 1e3)
        sk_d = api.zn_sk_import(dctx, api.zn_sk_export(sk))
        seal_acc = {"vanilla_ms": decode_error(api, dctx, sk_d, out_m, slots),
                    "zinc_data_level": decode_error(api, dctx, sk_d, out_mz, slots)}
        seal_acc["zinc_over_vanilla_rms"] = seal_acc["zinc_data_level"]["rms"] / seal_acc["vanilla_ms"]["rms"]
        seal = {"vanilla_ms_enc_s": ms_rate, "zinc_data_level_enc_s": mz_rate, "zinc_speedup": mz_rate / ms_rate,
                "decode_err": seal_acc,
                "data_primes": w.L - 1, "special_prime_bits": w.bits[-1],
                "kernel_ms_per_launch": {"prep": kp_ms / max(kp_n, 1), "special": ks_ms / max(ks_n, 1),
                                         "data": kd_ms / max(kd_n, 1)},
                "launches_per_step": (kp_n + ks_n + kd_n) / args.steps,
                "paper_speedup_context": "Table 2 totals, CKKS over Zinc: 2.34x, 2.51x, 2.44x (SEAL, one EPYC 7302P thread, N=32768)"}
        del out_m, out_mz, zc_d, sk_d, dctx

    # ---- BFV (Eq. 12) and BGV (Eq. 13), vanilla and Zinc, on the same ring
    # and chain: coefficient plaintexts uniform in [0, t), t = 65537
    intl = None
    if not args.no_int and 10 <= w.log_n <= 15:
        t_pt = 65537
        m_int = torch.tensor(workloads.int_plaintexts(w, t_pt, batch=B, first=lo), device=dev)
        out_i = torch.empty((B, 2, w.L, w.n), dtype=torch.int64, device=dev)
        gsk, gpk = api.bgv_keygen(ctx, t_pt, workloads.KEYGEN_SEED)
        gzc = api.bgv_zinc_precompute(ctx, gpk, workloads.CACHE_SEED)
        legs = {"bfv": lambda: api.bfv_encrypt(ctx, pk, t_pt, m_int, w.seed, idx, out=out_i, stream=stream),
                "bfv_zinc": lambda: api.bfv_zinc_encrypt(ctx, zc, t_pt, m_int, w.seed, idx, out=out_i, stream=stream),
                "bgv": lambda: api.bgv_encrypt(ctx, gpk, m_int, w.seed, idx, out=out_i, stream=stream),
                "bgv_zinc": lambda: api.bgv_zinc_encrypt(ctx, gzc, m_int, w.seed, idx, out=out_i, stream=stream)}
        rates = {}
        for name, fn in legs.items():
            for _ in range(args.warmup):
                fn()
            torch.cuda.synchronize(dev)
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            t_ms = max_over_ranks([e0.elapsed_time(e1)], world, dev, dist)[0]
            rates[name + "_enc_s"] = B * world * args.steps / (t_ms / 1e3)
        api.zn_sync_status(ctx, stream)
        # every plaintext of the last (BGV Zinc) batch decrypts exactly
        ok = bool(torch.equal(api.bgv_decrypt(ctx, gsk, t_pt, out_i), m_int))
        intl = dict(rates, t=t_pt, plaintext="coefficients uniform in [0, t)",
                    bfv_zinc_speedup=rates["bfv_zinc_enc_s"] / rates["bfv_enc_s"],
                    bgv_zinc_speedup=rates["bgv_zinc_enc_s"] / rates["bgv_enc_s"], decrypt_exact=ok)
        del out_i, m_int, gzc, gpk, gsk

    # ---- Zinc with NTT-domain errors (the Conclusion's O(N) remark): plaintexts
    # pre-encoded in NTT form (untimed, as the paper's Construction assumes an
    # encoded m), K cached basis errors per component rotated per ciphertext
    nttz = None
    if not args.no_nttz and 10 <= w.log_n <= 15:
        m_hat = api.ckks_encode_ntt(ctx, slots)
        out_n = torch.empty((B, 2, w.L, w.n), dtype=torch.int64, device=dev)
        nttz = {"plaintext": "pre-encoded in NTT form (ckks_encode_ntt, untimed)"}
        for K in (1, 2, 4):
            nb = api.zinc_nbasis_create(ctx, K, workloads.NBASIS_SEED)
            for _ in range(args.warmup):
                api.zinc_encrypt_ntt(ctx, zc, nb, m_hat, w.seed, idx, out=out_n, stream=stream)
            torch.cuda.synchronize(dev)
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                api.zinc_encrypt_ntt(ctx, zc, nb, m_hat, w.seed, idx, out=out_n, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            t_ms = max_over_ranks([e0.elapsed_time(e1)], world, dev, dist)[0]
            rate = B * world * args.steps / (t_ms / 1e3)
            # algorithmic HBM bytes per ciphertext: the plaintext read and the ciphertext written
            per = 3 * w.L * w.n * 8
            gbs = B * args.steps * per / (t_ms / 1e3) / 1e9
            nttz[f"K{K}"] = {"enc_s": rate, "hbm_gbs": gbs, "hbm_frac": gbs / hbm_peak,
                             "ms_per_launch": t_ms / args.steps, "bytes_per_ct": per}
            nb.close()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        api.ckks_encode_ntt(ctx, slots, out=m_hat, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        nttz["encode_ntt_enc_s"] = B / (e0.elapsed_time(e1) / 1e3)
        del m_hat, out_n

    # ---- serving: Poisson stream of mixed-ring requests, continuous batching
    serving = None
    if rank == 0 and world == 1 and not args.no_serve:
        from paper_2408_07304_gb300 import serve
        del out_v, out_z
        torch.cuda.empty_cache()
        serving = serve.serve_benchmark(args.serve_requests, 0.7, device=local)

    # ---- CPU baseline: the oracle on a bounded sample (rank 0, one GPU only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        dt, cores, desc = oracle_sample(w, oracle_setup(w))
        cpu = {"value": 2.0 / dt, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": f"{w.name}: {w.describe()}", "global_batch": 2 * B * world,
                       "parallelism": f"replicas x{world}",
                       "l2": "working set above L2: slots 256 MiB read and 16 GiB of ciphertexts written per step"
                             if w.name == "throughput" else "see workload"},
            "vanilla_enc_s": van_rate, "zinc_enc_s": zin_rate, "zinc_speedup": zin_rate / van_rate,
            "decode_err": accuracy,
            "hbm_frac_whole_step": value * per_ct_bytes / (hbm_peak * 1e9),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
            "serving": serving, "persistent_graph": persistent, "special_prime": seal, "bfv_bgv": intl,
            "zinc_ntt_domain": nttz,
            "kernel_ms_per_launch": {"prep": enc_ms / max(enc_n, 1), "encrypt_vanilla": kv_avg,
                                     "encrypt_zinc": kz_avg},
            "autotune": {"variant": tune[0], "ms_per_variant": tune[1]},
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="throughput", choices=sorted(workloads.WORKLOADS))
    ap.add_argument("--batch", type=int, default=None, help="override the workload's batch (profiling runs)")
    ap.add_argument("--variant", type=int, default=None, help="fixed encryption launch shape instead of autotuning")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving (p50/p99) run")
    ap.add_argument("--no-persistent", action="store_true", help="skip the persistent-graph path")
    ap.add_argument("--no-special", action="store_true", help="skip the special-prime (SEAL-ordered) leg")
    ap.add_argument("--no-int", action="store_true", help="skip the BFV / BGV leg")
    ap.add_argument("--no-nttz", action="store_true", help="skip the NTT-domain Zinc leg")
    ap.add_argument("--serve-requests", type=int, default=20000)
    args = ap.parse_args()
    w = workloads.WORKLOADS[args.workload]
    if args.batch:
        import dataclasses
        w = dataclasses.replace(w, batch=args.batch)
    if args.impl == "reference":
        run_reference(args, w)
    else:
        run_ours(args, w)


if __name__ == "__main__":
    main()
