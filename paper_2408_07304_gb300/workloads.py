"""Seeded synthetic workloads (slot vectors and parameter sets).

Holds none of the method's arithmetic: only parameter sets and numpy PCG64
draws with the shapes and value ranges of the workloads.  Tests feed the same
draws to the GPU library and to the CPU oracle.  The paper's own datasets
(Covid-19, Bitcoin, hg38; Section "Experimental Setup") are not used; these
synthetic vectors stand in for them.

Parameter sets:
  single   N = 4096, 3 x 36-bit primes, Delta = 2^30, 2048 slots U[-1, 1], 1 vector
  batched  N = 8192, {60, 40, 40, 60}, Delta = 2^40, 1024 vectors x 4096 slots,
           N(0, 1) clipped to [-8, 8]
  throughput  N = 16384, 60 + 6 x 50 + 60, Delta = 2^50, 4096 vectors x 8192 slots U[-1, 1]
  large    N = 32768, 60 + 12 x 55 + 60, Delta = 2^55, 512 vectors x 16384 slots U[-100, 100]
  paper    N = 32768, 15 x 55 + 56 bits (881 bits, the paper's SEAL modulus size), Delta = 2^55
"""
from dataclasses import dataclass

import numpy as np

KEYGEN_SEED = 1     # Gen
CACHE_SEED = 2      # the cached Enc(0)
NBASIS_SEED = 3     # the cached error basis of the NTT-domain Zinc randomiser


@dataclass(frozen=True)
class Workload:
    name: str
    log_n: int
    bits: tuple
    log2_delta: int
    batch: int
    n_slots: int
    dist: str           # "uniform" or "normal_clip"
    lo: float
    hi: float
    seed: int

    @property
    def n(self):
        return 1 << self.log_n

    @property
    def L(self):
        return len(self.bits)

    def describe(self):
        chain = "+".join(str(b) for b in self.bits)
        return (f"N={self.n} primes={chain} log2Delta={self.log2_delta} batch={self.batch} "
                f"slots={self.n_slots} {self.dist}[{self.lo},{self.hi}] seed={self.seed}")


WORKLOADS = {
    "single": Workload("single", 12, (36, 36, 36), 30, 1, 2048, "uniform", -1.0, 1.0, 0),
    "batched": Workload("batched", 13, (60, 40, 40, 60), 40, 1024, 4096, "normal_clip", -8.0, 8.0, 2),
    "throughput": Workload("throughput", 14, (60,) + (50,) * 6 + (60,), 50, 4096, 8192, "uniform", -1.0, 1.0, 3),
    "large": Workload("large", 15, (60,) + (55,) * 12 + (60,), 55, 512, 16384, "uniform", -100.0, 100.0, 4),
    "paper": Workload("paper", 15, (55,) * 15 + (56,), 55, 64, 16384, "uniform", -1.0, 1.0, 5),
}


def slots(w: Workload, batch: int = None, first: int = 0, n_slots: int = None, seed: int = None):
    """Slot vectors [batch, n_slots] (float64).  Vector b is drawn from its own
    stream (seed, first + b), so any sub-range reproduces the same vectors."""
    batch = w.batch if batch is None else batch
    n_slots = w.n_slots if n_slots is None else n_slots
    seed = w.seed if seed is None else seed
    out = np.empty((batch, n_slots))
    for b in range(batch):
        rng = np.random.Generator(np.random.PCG64([seed, first + b]))
        if w.dist == "uniform":
            out[b] = rng.uniform(w.lo, w.hi, n_slots)
        else:
            out[b] = np.clip(rng.standard_normal(n_slots), w.lo, w.hi)
    return out


def int_plaintexts(w: Workload, t: int, batch: int = None, first: int = 0, seed: int = None):
    """Coefficient plaintexts for BFV / BGV: int64 [batch, N] uniform in [0, t),
    vector b drawn from its own stream (seed, first + b, t)."""
    batch = w.batch if batch is None else batch
    seed = w.seed if seed is None else seed
    out = np.empty((batch, w.n), dtype=np.int64)
    for b in range(batch):
        rng = np.random.Generator(np.random.PCG64([seed, first + b, t]))
        out[b] = rng.integers(0, t, w.n, dtype=np.int64)
    return out


def small(log_n, bits, log2_delta, batch, n_slots, seed=0, lo=-1.0, hi=1.0):
    """An ad-hoc uniform workload (tests)."""
    return Workload(f"n{1 << log_n}", log_n, tuple(bits), log2_delta, batch, n_slots, "uniform", lo, hi, seed)
