"""Pins for the CPU oracle: each check ties an oracle function to something
other than itself -- a closed form, brute force, an algebraic invariant, an
independent library routine, or published known-answer values -- so that a
dropped term, a wrong sign or index, or a transposed operand fails here.
"""
import math
import os

from fractions import Fraction

import numpy as np
import pytest

from oracle import ckks, encoder, numtheory, philox, ring, sampler
from paper_2408_07304_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------- primes
def test_is_prime_matches_trial_division():
    # brute force on small n
    def trial(n):
        if n < 2:
            return False
        f = 2
        while f * f <= n:
            if n % f == 0:
                return False
            f += 1
        return True
    assert all(numtheory.is_prime(n) == trial(n) for n in range(3000))
    # Carmichael and strong pseudoprimes to small bases must be rejected
    for n in (561, 1105, 1729, 2047, 3215031751, 3825123056546413051):
        assert not numtheory.is_prime(n)


@pytest.mark.parametrize("log_n,bits", [(12, (36, 36, 36)), (13, (60, 40, 40, 60)),
                                        (14, (60, 50, 50, 50, 50, 50, 50, 60))])
def test_prime_chain_rule(log_n, bits):
    sympy = pytest.importorskip("sympy")
    two_n = 2 << log_n
    qs = numtheory.gen_primes(log_n, bits)
    assert len(set(qs)) == len(qs)
    for i, (q, b) in enumerate(zip(qs, bits)):
        assert sympy.isprime(q) and q % two_n == 1 and q < 2 ** b
        # maximality: every candidate above q (below 2^b, 1 mod 2N) is composite or already used
        c = q + two_n
        while c < 2 ** b:
            assert (not sympy.isprime(c)) or c in qs[:i]
            c += two_n


def test_psi_is_minimal_primitive_root_small():
    # enumeration on small NTT-friendly primes: nothing below psi is a primitive 2N-th root
    for q, log_n in ((7681, 8), (12289, 10), (40961, 12), (65537, 4)):
        n = 1 << log_n
        psi = numtheory.find_psi(q, log_n)
        assert pow(psi, n, q) == q - 1 and pow(psi, 2 * n, q) == 1
        assert all(pow(x, n, q) != q - 1 for x in range(2, psi))


@pytest.mark.parametrize("log_n,bits", [(12, (36, 36, 36)), (14, (60, 50, 60))])
def test_psi_of_chain(log_n, bits):
    n = 1 << log_n
    for q in numtheory.gen_primes(log_n, bits):
        psi = numtheory.find_psi(q, log_n)
        assert pow(psi, n, q) == q - 1            # order exactly 2N
        # psi is the minimum of the set of all primitive 2N-th roots {psi^k : k odd}
        x, step = psi, psi * psi % q
        for _ in range(n - 1):
            x = x * step % q
            assert x > psi


# --------------------------------------------------------------------- philox
def test_philox_known_answers():
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = philox.philox4x32_10(*v[:6])
        assert [int(o) for o in out] == v[6:]


def test_philox_matches_triton_interpreter():
    # an independent library implementation of Philox4x32 (triton.language.randint4x,
    # counter = (offset, 0, 0, 0), key = seed) run by triton's CPU interpreter
    os.environ["TRITON_INTERPRET"] = "1"
    triton = pytest.importorskip("triton")
    import torch
    tl = pytest.importorskip("triton.language")

    @triton.jit
    def k(out_ptr, seed, N: tl.constexpr):
        offs = tl.arange(0, N)
        a, b, c, d = tl.randint4x(seed, offs, 10)
        tl.store(out_ptr + offs * 4 + 0, a)
        tl.store(out_ptr + offs * 4 + 1, b)
        tl.store(out_ptr + offs * 4 + 2, c)
        tl.store(out_ptr + offs * 4 + 3, d)

    for seed in (0, 12345, 0x7FFFFFFF):
        out = torch.zeros(64 * 4, dtype=torch.int32)
        try:
            k[(1,)](out, seed, N=64)
        except Exception as exc:  # pragma: no cover - interpreter not usable here
            pytest.skip(f"triton interpreter unavailable: {exc}")
        got = np.array(out.tolist(), dtype=np.int64).reshape(64, 4) & 0xFFFFFFFF
        ref = philox.philox4x32_10(np.arange(64), 0, 0, 0, seed & 0xFFFFFFFF, seed >> 32)
        assert np.array_equal(got, np.stack([r.astype(np.int64) for r in ref], axis=1))


# -------------------------------------------------------------------- sampler
def test_cdt_thresholds_match_mpmath():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 60
    s = mpmath.mpf(16) / 5

    def cdf(x):
        return mpmath.ncdf(x, 0, s)

    lo, hi = cdf(mpmath.mpf(-19.5)), cdf(mpmath.mpf(19.5))
    ref = [int(mpmath.floor((cdf(v + mpmath.mpf(0.5)) - lo) / (hi - lo) * mpmath.mpf(2) ** 64))
           for v in range(-19, 19)]
    assert list(sampler.cdt_thresholds()) == ref


def test_cdt_thresholds_shape():
    t = sampler.cdt_thresholds()
    assert len(t) == 38 and all(a < b for a, b in zip(t, t[1:]))
    assert 0 < t[0] and t[-1] < 2 ** 64
    # symmetry of the rounded normal: P(X <= -v-1) = P(X >= v+1) = 1 - F(v)
    for v in range(0, 19):
        a = t[(-v - 1) + 19]
        b = 2 ** 64 - t[v + 19]
        assert abs(a - b) <= 1


def test_cdt_lookup_edges():
    t = sampler.cdt_thresholds()
    u = np.array([0, t[0] - 1, t[0], t[18] - 1, t[18], t[37] - 1, t[37], 2 ** 64 - 1], dtype=np.uint64)
    assert sampler.cdt_lookup(u).tolist() == [-19, -19, -18, -1, 0, 18, 19, 19]


def test_gaussian_distribution():
    n = 1 << 17
    e = np.concatenate([sampler.sample_gaussian(n, 99, 0, 1, c) for c in range(4)])
    assert e.min() >= -19 and e.max() <= 19
    # exact probabilities of the rounded normal, then a chi-square goodness of fit
    t = [0] + list(sampler.cdt_thresholds()) + [2 ** 64]
    p = np.array([(t[i + 1] - t[i]) / 2 ** 64 for i in range(39)])
    counts = np.bincount(e + 19, minlength=39)
    expected = p * e.size
    mask = expected > 20
    chi2 = np.sum((counts[mask] - expected[mask]) ** 2 / expected[mask])
    assert chi2 < 80          # ~25 degrees of freedom; p ~ 1e-7 at 80
    var_exact = float(np.sum(p * (np.arange(-19, 20) ** 2)))
    assert abs(var_exact - (3.2 ** 2 + 1 / 12)) < 0.01     # rounding adds 1/12
    assert abs(e.var() - var_exact) < 0.1
    assert abs(e.mean()) < 0.03


def test_ternary_distribution_and_edges():
    u = np.concatenate([sampler.sample_ternary(1 << 16, 7, 0, 0, c) for c in range(4)])
    assert set(np.unique(u).tolist()) == {-1, 0, 1}
    c = np.bincount(u + 1)
    exp = u.size / 3
    assert np.sum((c - exp) ** 2 / exp) < 20
    # the word -> value rule at its boundaries: floor(3 w / 2^32) - 1
    w = np.array([0, (2 ** 32 + 2) // 3 - 1, (2 ** 32 + 2) // 3, 2 * ((2 ** 32 + 2) // 3),
                  2 ** 32 - 1], dtype=np.uint64)
    t = ((w * np.uint64(3)) >> np.uint64(32)).astype(np.int64) - 1
    assert t.tolist() == [-1, -1, 0, 1, 1]


def test_counter_layout_placement():
    # one Philox block feeds coefficients N/4 (ternary) or N/2 (chi) apart
    n = 64
    u = sampler.sample_ternary(n, 5, 0, 0, 3)
    w = philox.philox4x32_10(np.arange(n // 4), 0, 3, 0, 5, 0)
    for j in range(4):
        assert np.array_equal(u[j * 16:(j + 1) * 16],
                              ((w[j] * np.uint64(3)) >> np.uint64(32)).astype(np.int64) - 1)
    e = sampler.sample_gaussian(n, 5, 1, 1, 2 ** 33 + 4)
    w = philox.philox4x32_10(np.arange(n // 2), (1 << 24) | (1 << 16), 4, 2, 5, 0)
    assert np.array_equal(e[:32], sampler.cdt_lookup((w[1] << np.uint64(32)) | w[0]))
    assert np.array_equal(e[32:], sampler.cdt_lookup((w[3] << np.uint64(32)) | w[2]))


def test_uniform_mod_q():
    q = 1152921504606748673
    v = sampler.sample_uniform_mod(4096, q, 3, 2, 1, 0)
    assert all(0 <= x < q for x in v)
    assert abs(np.mean([x / q for x in v]) - 0.5) < 0.03
    assert len(set(v)) == len(v)


# ----------------------------------------------------------------------- ring
def _poly_mul_negacyclic_numpy(a, b, q):
    """Library route: full integer product by numpy.polymul on object arrays, then X^N = -1."""
    n = len(a)
    full = np.polymul(np.array(a[::-1], dtype=object), np.array(b[::-1], dtype=object))[::-1]
    full = list(full) + [0] * (2 * n - 1 - len(full))
    return [int(full[k] - (full[k + n] if k + n < len(full) else 0)) % q for k in range(n)]


@pytest.mark.parametrize("log_n", [2, 4, 6])
def test_schoolbook_vs_library(log_n):
    n = 1 << log_n
    q = numtheory.gen_primes(log_n, (40,))[0]
    rng = np.random.default_rng(log_n)
    a = rng.integers(0, q, n, dtype=np.uint64)
    b = rng.integers(0, q, n, dtype=np.uint64)
    s = rng.integers(-20, 21, n)
    ref = _poly_mul_negacyclic_numpy([int(x) for x in a], [int(x) for x in b], q)
    assert ring.negacyclic_mul(a, b, q).tolist() == ref
    ref = _poly_mul_negacyclic_numpy([int(x) for x in a], [int(x) for x in s], q)
    assert ring.negacyclic_mul_small(a, s, q).tolist() == ref


def test_negacyclic_wrap_closed_form():
    n, q = 64, numtheory.gen_primes(6, (30,))[0]
    xa = np.zeros(n, dtype=np.uint64)
    xa[n - 1] = 1
    xb = np.zeros(n, dtype=np.int64)
    xb[1] = 1
    c = ring.negacyclic_mul_small(xa, xb, q)         # X^(N-1) * X = X^N = -1
    assert c[0] == q - 1 and not c[1:].any()


@pytest.mark.parametrize("log_n,bits", [(4, 30), (6, 50), (10, 60), (12, 36)])
def test_ntt_convolution_theorem(log_n, bits):
    n = 1 << log_n
    q = numtheory.gen_primes(log_n, (bits,))[0]
    psi = numtheory.find_psi(q, log_n)
    rng = np.random.default_rng(bits)
    a = rng.integers(0, q, n, dtype=np.uint64)
    b = rng.integers(0, q, n, dtype=np.uint64)
    ab = ring.negacyclic_mul(a, b, q)
    lhs = [(int(x) * int(y)) % q for x, y in zip(ring.ntt(a, q, psi), ring.ntt(b, q, psi))]
    assert ring.ntt(ab, q, psi).tolist() == lhs
    assert np.array_equal(ring.intt(ring.ntt(a, q, psi), q, psi), a)


def test_ntt_closed_forms_and_ordering():
    log_n = 6
    n = 1 << log_n
    q = numtheory.gen_primes(log_n, (40,))[0]
    psi = numtheory.find_psi(q, log_n)
    one = np.zeros(n, dtype=np.uint64)
    one[0] = 1
    assert ring.ntt(one, q, psi).tolist() == [1] * n          # constants are fixed points
    x = np.zeros(n, dtype=np.uint64)
    x[1] = 1
    r = [int(v) for v in ring.ntt(x, q, psi)]                # the N roots of X^N + 1
    assert len(set(r)) == n and all(pow(v, n, q) == q - 1 for v in r)
    # bit-reversed order: neighbours 2i, 2i+1 evaluate at opposite roots
    assert all((r[2 * i] + r[2 * i + 1]) % q == 0 for i in range(n // 2))
    # and the first half holds the roots of X^(N/2) - sqrt(-1) for one fixed square root
    # of -1, i.e. {r : r^(N/2) = psi^(N/2)}
    assert all(pow(v, n // 2, q) == pow(psi, n // 2, q) for v in r[: n // 2])
    # the first output is the evaluation at psi itself
    assert r[0] == psi
    # ntt_eval agrees with the full transform at arbitrary indices
    a = np.random.default_rng(1).integers(0, q, n, dtype=np.uint64)
    full = ring.ntt(a, q, psi)
    idx = [0, 5, 17, 63]
    assert ring.ntt_eval(a, q, psi, idx).tolist() == full[idx].tolist()


# -------------------------------------------------------------------- encoder
def test_twiddles_correctly_rounded():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 200
    log_n = 8
    n = 1 << log_n
    re, im = encoder.twiddles(log_n)
    for k in range(n):
        x = mpmath.mpf(k) / n
        assert re[k] == float(mpmath.cospi(x)) and im[k] == float(-mpmath.sinpi(x)), k


def test_twiddles_near_libm():
    for log_n in (12, 14):
        re, im = encoder.twiddles(log_n)
        k = np.arange(1 << log_n)
        assert np.max(np.abs(re - np.cos(np.pi * k / (1 << log_n)))) < 6e-16
        assert np.max(np.abs(im + np.sin(np.pi * k / (1 << log_n)))) < 6e-16
        assert re[(1 << log_n) // 2] == 0.0 and im[(1 << log_n) // 2] == -1.0


@pytest.mark.parametrize("log_n", [4, 9])
def test_twiddles_q62_correctly_rounded(log_n):
    # C[k] = floor(2^62 cos(pi k/N) + 1/2), S[k] likewise with sin, against 200-bit mpmath
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 200
    n = 1 << log_n
    C, S = encoder.twiddles_q62(log_n)
    for k in range(n):
        x = mpmath.mpf(k) / n
        assert int(C[k]) == int(mpmath.floor(mpmath.cospi(x) * 2 ** 62 + mpmath.mpf(1) / 2)), k
        assert int(S[k]) == int(mpmath.floor(mpmath.sinpi(x) * 2 ** 62 + mpmath.mpf(1) / 2)), k


def test_twiddles_q62_exact_points():
    # the two twiddles whose products the kernels may skip are exact
    for log_n in (4, 14):
        C, S = encoder.twiddles_q62(log_n)
        n = 1 << log_n
        assert (C[0], S[0]) == (1 << 62, 0) and (C[n // 2], S[n // 2]) == (0, 1 << 62)
        # |W| = 1 up to the quantisation (|C|, |S| off by <= 1/2 each)
        mod2 = C.astype(object) ** 2 + S.astype(object) ** 2
        assert all(abs(v - (1 << 124)) <= (1 << 63) + 1 for v in mod2)


def test_slot_index_is_bijection():
    for log_n in (4, 10, 13):
        t = encoder.slot_index(log_n)
        assert sorted(t.tolist()) == list(range(1 << (log_n - 1)))


@pytest.mark.parametrize("z", [np.array([1.0, -0.5, 0.25]), np.array([5e-324, -1e-310, 3e-300]),
                               np.array([1e300, -1.0, 1e-300]), np.random.default_rng(4).uniform(-8, 8, 4096),
                               np.array([-2.0 ** 40])])
def test_block_scale_invariants(z):
    # step 0: |Y_j - z_j 2^F| <= 1/2 exactly, sum |Y| < 2^59 + n/2, and the
    # scale is the largest that keeps n max|z| 2^F <= 2^59 (n = N/2 slots)
    log_n = 13
    n = 1 << (log_n - 1)
    F, Y = encoder.block_scale(z, log_n)
    frac2 = Fraction(2)
    for v, y in zip(z, Y):
        assert abs(Fraction(float(v)) * frac2 ** F - y) <= Fraction(1, 2)
    assert sum(abs(y) for y in Y) < 2 ** 59 + n / 2
    M = Fraction(float(np.max(np.abs(z))))
    assert n * M * frac2 ** F < 2 ** 59 <= n * M * frac2 ** (F + 1)


def test_encode_zero_padding_invariant():
    # appending zero slots changes nothing (batches pad vectors to a common length)
    log_n, ld = 10, 30
    z = np.random.default_rng(8).uniform(-3, 3, 37)
    m = encoder.encode(z, log_n, ld)
    for pad in (1, 100, 512 - 37):
        assert np.array_equal(encoder.encode(np.concatenate([z, np.zeros(pad)]), log_n, ld), m)


def _canonical(z, log_n, ld, mpmath):
    """(2 Delta / N) Re sum_j z_j zeta^(-5^j k), k < N, at 60 digits."""
    n = 1 << log_n
    g = [pow(5, j, 2 * n) for j in range(len(z))]
    out = []
    for k in range(n):
        acc = mpmath.mpf(0)
        for j, v in enumerate(z):
            acc += mpmath.mpf(float(v)) * mpmath.cospi(mpmath.mpf((g[j] * k) % (2 * n)) / n)
        out.append(acc * 2 * mpmath.mpf(2) ** ld / n)
    return out


@pytest.mark.parametrize("log_n,ld,z", [
    (4, 20, np.array([0.3, -0.7, 0.1, 0.9, -0.2, 0.5, -1.0, 0.25])),
    (4, 40, np.array([1e-12, -3.0, 0.0])),
    (5, 30, np.random.default_rng(6).uniform(-1, 1, 16)),
    (6, 25, np.concatenate([np.random.default_rng(7).uniform(-100, 100, 5), [1e-9, -1e-20]])),
    (6, 60, np.array([2.0 ** -1060, -2.0 ** -1050])),
])
def test_encode_vs_canonical_embedding_brute_force(log_n, ld, z):
    # brute force on tiny rings: the unrounded fixed-point result is within the
    # derived bound of the exact embedding, and m is its rounding (within 1/2 + bound)
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 60
    exact = _canonical(z, log_n, ld, mpmath)
    real = encoder.encode_real(z, log_n, ld)
    m = encoder.encode(z, log_n, ld)
    bound = encoder.encode_error_bound(z, log_n, ld)
    for k in range(1 << log_n):
        err = abs(mpmath.mpf(float(real[k])) - exact[k])
        assert err <= bound * (1 + 1e-12) + abs(float(real[k])) * 2.0 ** -52, (k, err, bound)
        assert abs(mpmath.mpf(int(m[k])) - exact[k]) <= 0.5 + bound * (1 + 1e-12) + 1e-9, k


@pytest.mark.parametrize("c", [0.5, -0.75, 1.0 / 3.0])
def test_encode_constant_closed_form(c):
    # z_j = c for all j encodes to the constant polynomial Delta c (up to rounding)
    log_n, ld = 12, 30
    z = np.full(1 << (log_n - 1), c)
    m = encoder.encode(z, log_n, ld)
    tol = 0.5 + encoder.encode_error_bound(z, log_n, ld)
    assert abs(m[0] - c * 2.0 ** ld) <= tol and np.max(np.abs(m[1:])) <= tol


@pytest.mark.parametrize("j", [0, 1, 7, 1000])
def test_encode_single_slot_closed_form(j):
    # z = e_j encodes to m_k = rnd((2 Delta / N) cos(pi 5^j k / N))
    log_n, ld = 12, 30
    n = 1 << log_n
    z = np.zeros(n // 2)
    z[j] = 1.0
    m = encoder.encode(z, log_n, ld)
    k = np.arange(n)
    e = (pow(5, j, 2 * n) * k) % (2 * n)
    ref = (2.0 * 2.0 ** ld / n) * np.cos(np.pi * e / n)
    assert np.max(np.abs(m - ref)) <= 0.5 + encoder.encode_error_bound(z, log_n, ld) + 1e-6


@pytest.mark.parametrize("log_n,ld,n_slots", [(10, 30, 512), (12, 30, 2048), (12, 40, 700), (4, 20, 8)])
def test_encode_fft_vs_definition(log_n, ld, n_slots):
    # against the FP64 direct sum, within both error bounds
    z = np.random.default_rng(log_n + n_slots).uniform(-1, 1, n_slots)
    real = encoder.encode_real(z, log_n, ld)
    direct = encoder.encode_direct(z, log_n, ld)
    direct_err = encoder.encode_direct_error_bound(z, log_n, ld)
    assert np.max(np.abs(real - direct)) <= encoder.encode_error_bound(z, log_n, ld) + direct_err


@pytest.mark.parametrize("name,rows", [("throughput", (0, 4095)), ("large", (0,)), ("batched", (1023,))])
def test_encode_fixed_vs_definition_full_size(name, rows):
    # The benchmarked rings: the fixed-point procedure's unrounded output and its
    # integers m_k against the defining sum of the canonical embedding, on the
    # workloads' own vectors (full slot count, their value ranges).
    w = workloads.WORKLOADS[name]
    for b in rows:
        z = workloads.slots(w, batch=1, first=b)[0]
        direct = encoder.encode_direct(z, w.log_n, w.log2_delta)
        bound = (encoder.encode_error_bound(z, w.log_n, w.log2_delta)
                 + encoder.encode_direct_error_bound(z, w.log_n, w.log2_delta))
        real = encoder.encode_real(z, w.log_n, w.log2_delta)
        assert np.max(np.abs(real - direct)) <= bound
        m = encoder.encode(z, w.log_n, w.log2_delta)
        assert np.max(np.abs(m - direct)) <= 0.5 + bound
        # Parseval: m evaluated at the N odd 2N-th roots gives Delta z_j at each
        # slot root and at its conjugate, so sum_k m_k^2 = 2 Delta^2 sum_j z_j^2 / N
        # exactly for the defining sum (fixes its scale and that no slot is lost)
        ratio = math.fsum(direct ** 2) / (2.0 ** (2 * w.log2_delta + 1) * math.fsum(z ** 2) / w.n)
        assert abs(ratio - 1.0) < 1e-9


def test_encode_direct_error_bound_holds():
    # The direct sum's own bound against an exact evaluation with Python
    # fractions of the same table cosines, so that the products and the
    # pairwise additions are the roundings measured (the table's own rounding,
    # also in the bound, is pinned against mpmath elsewhere).
    from fractions import Fraction
    log_n, ld = 7, 30
    n = 1 << log_n
    z = np.random.default_rng(77).uniform(-3, 3, n // 2)
    direct = encoder.encode_direct(z, log_n, ld)
    cos_t = encoder._cos_table(log_n)
    g = [pow(5, j, 2 * n) for j in range(n // 2)]
    bound = encoder.encode_direct_error_bound(z, log_n, ld)
    scale = Fraction(2) ** (ld + 1 - log_n)
    for k in range(0, n, 5):
        exact = sum(Fraction(float(z[j])) * Fraction(float(cos_t[g[j] * k % (2 * n)])) for j in range(n // 2))
        assert abs(Fraction(float(direct[k])) - exact * scale) <= Fraction(bound)


def test_encode_linear_and_decode_roundtrip():
    log_n, ld = 11, 40
    rng = np.random.default_rng(3)
    z1, z2 = rng.uniform(-1, 1, 1024), rng.uniform(-1, 1, 1024)
    m1, m2, m12 = (encoder.encode(z, log_n, ld) for z in (z1, z2, z1 + z2))
    assert np.max(np.abs(m12 - m1 - m2)) <= 2
    back = encoder.decode(m1, log_n, ld, 1024)
    # rounding error <= 1/2 per coefficient: |z - z'| <= N/2 / Delta (loose, deterministic)
    assert np.max(np.abs(back - z1)) < (1 << log_n) / 2 / 2.0 ** ld


def test_encode_zero_and_empty():
    assert not encoder.encode(np.zeros(5), 6, 30).any()
    assert not encoder.encode(np.zeros(0), 6, 30).any()


def test_encode_overflow_detected():
    with pytest.raises(OverflowError):
        encoder.encode(np.full(8, 2.0 ** 30), 4, 40)
    with pytest.raises(OverflowError):
        encoder.encode(np.array([1.0, np.nan]), 4, 20)
    with pytest.raises(OverflowError):
        encoder.encode(np.array([np.inf]), 4, 20)


# ----------------------------------------------------------- Gen / Enc / Dec
@pytest.fixture(scope="module")
def small():
    P = ckks.Params(6, (40, 40, 41), 20)
    K = ckks.keygen(P, 11)
    return P, K


def _small_conv(a, b, n):
    """Exact negacyclic product of small integer vectors via numpy.convolve (library)."""
    full = np.convolve(np.asarray(a, dtype=np.int64), np.asarray(b, dtype=np.int64))
    full = np.concatenate([full, np.zeros(2 * n - full.size, dtype=np.int64)])
    return full[:n] - full[n:]


def test_keygen_identity(small):
    P, K = small
    assert set(np.unique(K.s).tolist()) <= {-1, 0, 1}
    for i, q in enumerate(P.primes):
        # Eq. 7: pk0 + pk1 s = e (mod q)
        lhs = (K.pk0[i].astype(object) + ring.negacyclic_mul_small(K.pk1[i], K.s, q).astype(object)) % q
        assert np.array_equal(lhs, np.mod(K.e, q).astype(object))


def test_theorem1_identity_vanilla(small):
    P, K = small
    z = np.random.default_rng(0).uniform(-1, 1, 20)
    ct = ckks.encrypt_coeff(P, K, z, seed=5, ct_index=9)
    # Dec = m + e u + e0 + e1 s exactly (proof of Theorem 1 with e_b = e1, e_a = e0)
    v = _small_conv(K.e, ct.u, P.n) + ct.e0 + _small_conv(ct.e1, K.s, P.n)
    dec = ckks.decrypt_coeff(P, K, ct.c0, ct.c1)
    for i, q in enumerate(P.primes):
        assert np.array_equal(dec[i].astype(object), np.mod((ct.m + v).astype(object), q))


def test_theorem1_identity_zinc(small):
    P, K = small
    zero = ckks.zinc_precompute_coeff(P, K, seed=2)
    z = np.random.default_rng(1).uniform(-1, 1, 32)
    ct = ckks.zinc_encrypt_coeff(P, zero, z, seed=5, ct_index=3)
    # Dec(Enc_z(m)) = m + e u + e_a + e_b s with e_a = e0 + e1', e_b = e1 + e2'
    ea = zero.e0 + ct.e1p
    eb = zero.e1 + ct.e2p
    v = _small_conv(K.e, zero.u, P.n) + ea + _small_conv(eb, K.s, P.n)
    dec = ckks.decrypt_coeff(P, K, ct.c0, ct.c1)
    for i, q in enumerate(P.primes):
        assert np.array_equal(dec[i].astype(object), np.mod((ct.m + v).astype(object), q))


def test_zinc_structure_identity(small):
    P, K = small
    zero = ckks.zinc_precompute_coeff(P, K, seed=2)
    a = ckks.zinc_encrypt_coeff(P, zero, np.ones(4), seed=5, ct_index=1)
    b = ckks.zinc_encrypt_coeff(P, zero, -np.ones(4), seed=5, ct_index=2)
    for i, q in enumerate(P.primes):
        # c1 components differ by exactly e2'_a - e2'_b; c0 by m_a - m_b + e1'_a - e1'_b
        d1 = (a.c1[i].astype(object) - b.c1[i].astype(object)) % q
        assert np.array_equal(d1, np.mod((a.e2p - b.e2p).astype(object), q))
        d0 = (a.c0[i].astype(object) - b.c0[i].astype(object)) % q
        assert np.array_equal(d0, np.mod((a.m - b.m + a.e1p - b.e1p).astype(object), q))


def test_decrypt_decode_and_homomorphism():
    P = ckks.Params(10, (40, 40), 30)
    K = ckks.keygen(P, 1)
    rng = np.random.default_rng(4)
    za, zb = rng.uniform(-1, 1, 512), rng.uniform(-1, 1, 512)
    ca = ckks.encrypt_coeff(P, K, za, 0, 1)
    zero = ckks.zinc_precompute_coeff(P, K, 2)
    cb = ckks.zinc_encrypt_coeff(P, zero, zb, 0, 2)
    # noise bound: |v_k| <= ||e u||_inf + ... <= 19 (N + 1 + N) + 19 N; slot error <= N max|v| / Delta
    bound = (1 << 10) * (19 * (3 * (1 << 10) + 2)) / 2.0 ** 30
    assert np.max(np.abs(ckks.decrypt_decode(P, K, ca.c0, ca.c1, 512) - za)) < bound
    assert np.max(np.abs(ckks.decrypt_decode(P, K, cb.c0, cb.c1, 512) - zb)) < bound
    # Eq. 2 (additive homomorphism): Dec(c_a + c_b) ~ m_a + m_b
    s0 = [(x.astype(object) + y.astype(object)) % q for x, y, q in zip(ca.c0, cb.c0, P.primes)]
    s1 = [(x.astype(object) + y.astype(object)) % q for x, y, q in zip(ca.c1, cb.c1, P.primes)]
    s0 = [np.array(x, dtype=np.uint64) for x in s0]
    s1 = [np.array(x, dtype=np.uint64) for x in s1]
    assert np.max(np.abs(ckks.decrypt_decode(P, K, s0, s1, 512) - (za + zb))) < 2 * bound


# ---------------------------------------- modulus-switched (SEAL-ordered) Enc
def _crt(residues, primes):
    M = 1
    for q in primes:
        M *= q
    x = 0
    for r, q in zip(residues, primes):
        Mi = M // q
        x += int(r) * Mi * pow(Mi, -1, q)
    return x % M, M


def test_mod_switch_is_divide_and_round():
    # per coefficient, c' = floor((C + floor(p/2)) / p) mod Q for the CRT value
    # C in [0, Q p), checked with Python big integers -- including C = k p + h
    # (rounds down) and k p + h + 1 (rounds up), the nearest-integer boundary
    P = ckks.Params(4, (40, 41, 50), 20)
    p, qs = P.primes[-1], P.primes[:-1]
    Q = qs[0] * qs[1]
    h = p // 2
    rng = np.random.default_rng(3)
    Cs = [int(v) for v in rng.integers(0, 2 ** 62, 10)]
    Cs = [(c * 977 + 12345) % (Q * p) for c in Cs]
    Cs += [0, p - 1, 5 * p + h, 5 * p + h + 1, Q * p - 1, (Q - 1) * p + h + 1]
    Cs = Cs[:16]
    polys = [np.array([C % q for C in Cs], dtype=np.uint64) for q in P.primes]
    out = ckks.mod_switch_coeff(P, polys)
    for k, C in enumerate(Cs):
        want = ((C + h) // p) % Q
        got, _ = _crt([out[0][k], out[1][k]], qs)
        assert got == want, (k, C)
    assert int(out[0][10]) == 0 and int(out[0][12]) == 5 and int(out[0][13]) == 6


@pytest.fixture(scope="module")
def small3():
    P = ckks.Params(6, (40, 41, 50), 20)
    K = ckks.keygen(P, 11)
    return P, K


@pytest.mark.parametrize("bits,ld", [((40, 41, 50), 20), ((40, 41, 30), 35)])
def test_modswitch_noise_identity(bits, ld):
    # p (Dec(c') - m) = v + (h - r0) + (h - r1) s exactly, v = e u + e0 + e1 s the
    # key-level noise, r_j = (c_j,p + h) mod p from the special-prime component;
    # the second set has m much larger than p (m enters only after the division)
    P = ckks.Params(6, bits, ld)
    K = ckks.keygen(P, 11)
    Pd = ckks.data_params(P)
    p = P.primes[-1]
    h = p // 2
    z = np.random.default_rng(2).uniform(-1, 1, 16)
    ct = ckks.encrypt_ms_coeff(P, K, z, seed=5, ct_index=9)
    v = _small_conv(K.e, ct.u, P.n) + ct.e0 + _small_conv(ct.e1, K.s, P.n)
    cp0 = ring.negacyclic_mul_small(K.pk0[-1], ct.u, p).astype(object) + ct.e0.astype(object)
    cp1 = ring.negacyclic_mul_small(K.pk1[-1], ct.u, p).astype(object) + ct.e1.astype(object)
    r0 = (cp0 + h) % p
    r1 = (cp1 + h) % p
    d1 = [h - int(x) for x in r1]
    d1s = [0] * P.n                                   # (h - r1) * s, negacyclic, exact
    for i in range(P.n):
        for j in range(P.n):
            if K.s[j]:
                k = i + j
                sgn = 1 if k < P.n else -1
                d1s[k % P.n] += sgn * d1[i] * int(K.s[j])
    rhs = [int(v[k]) + (h - int(r0[k])) + d1s[k] for k in range(P.n)]
    dec = ckks.decrypt_coeff(Pd, K, ct.c0, ct.c1)
    cen = ckks.crt_centered(Pd, dec, Pd.n_primes)
    assert [p * (cen[k] - int(ct.m[k])) for k in range(P.n)] == rhs
    # and therefore |Dec - m| <= (19 (2N + 1)) / p + (1 + N) / 2
    assert max(abs(cen[k] - int(ct.m[k])) for k in range(P.n)) <= (1 + P.n) / 2 + 1


def test_modswitch_randomness_is_vanilla(small3):
    # the same (u, e0, e1) as vanilla Enc with the same seed and index; data level = all primes but the last
    P, K = small3
    a = ckks.encrypt_ms_coeff(P, K, np.ones(3), seed=4, ct_index=7)
    b = ckks.encrypt_coeff(P, K, np.ones(3), seed=4, ct_index=7)
    assert np.array_equal(a.u, b.u) and np.array_equal(a.e0, b.e0) and np.array_equal(a.e1, b.e1)
    Pd = ckks.data_params(P)
    assert Pd.primes == P.primes[:-1] and len(a.c0) == len(a.c1) == Pd.n_primes


def test_zinc_on_modswitched_cache(small3):
    # Enc_z over a modulus-switched cache: Dec = m + e1' + e2' s + (the cache's Dec), exactly
    P, K = small3
    Pd = ckks.data_params(P)
    zero = ckks.zinc_precompute_ms_coeff(P, K, seed=2)
    z = np.random.default_rng(5).uniform(-1, 1, 32)
    ct = ckks.zinc_encrypt_coeff(Pd, zero, z, seed=5, ct_index=3)
    dz = ckks.crt_centered(Pd, ckks.decrypt_coeff(Pd, K, zero.c0, zero.c1), Pd.n_primes)
    dc = ckks.crt_centered(Pd, ckks.decrypt_coeff(Pd, K, ct.c0, ct.c1), Pd.n_primes)
    e = ct.e1p + _small_conv(ct.e2p, K.s, P.n)
    assert [dc[k] - dz[k] for k in range(P.n)] == [int(ct.m[k]) + int(e[k]) for k in range(P.n)]


def test_ntt_form_ciphertext_matches_sampled(small):
    P, K = small
    ct = ckks.encrypt_coeff(P, K, np.ones(3), seed=1, ct_index=0)
    full = ckks.ct_ntt(P, ct)
    pos = [(0, 0, 0), (1, 2, 63), (0, 1, 17)]
    assert ckks.ct_ntt_sampled(P, ct, pos).tolist() == [int(full[p][i][k]) for p, i, k in pos]
