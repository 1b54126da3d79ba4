"""CKKS encoder and decoder (canonical embedding).  TEST INFRASTRUCTURE ONLY.

The paper assumes the message is already encoded (Section "Zinc",
"Construction") and fixes only the scale Delta = 2^55 (Section "System
Implementation").  Definition used (standard CKKS): for real slots z_j,
j < n = N/2 (missing slots are zero), the plaintext polynomial m in
Z[X]/(X^N + 1) has coefficients

    m_k = round( (2 Delta / N) * Re sum_j z_j * zeta^(-5^j k) ),   zeta = exp(i pi / N),

i.e. m(zeta^(5^j)) ~ Delta z_j.  With t_j = (5^j mod 2N - 1)/4 (a bijection of
[0, n)) the sum S_k = sum_j z_j zeta^(-5^j k), k < n, equals
zeta^(-k) * DFT_n(y)_k with y_{t_j} = z_j, and m_k = scale Re S_k,
m_{k+n} = scale Im S_k (because zeta^(-5^j n) = -i).

Two forms:
* ``encode_direct``: the defining sum, evaluated term by term in FP64 (pin only).
* ``encode``: a block-scaled fixed-point procedure on integers whose every
  step is specified, so that an independent implementation reproduces the
  coefficients bit for bit.  All roundings are rnd(x) = floor(x + 1/2) of an
  exact rational x.  y is real, so its length-n DFT is taken through a
  complex DFT of half the length (the standard real-input split):
    0. scale: if no slot is given or all z_j = 0, m = 0.  M = max_j |z_j| (a
       non-finite M is an overflow); e with 2^(e-1) <= M < 2^e;
       F = 59 - log2 n - e = 60 - log2 N - e (the ring's slot count, not the
       number of given slots, so that zero padding leaves m unchanged);
       Y_j = rnd(z_j 2^F), so that sum_j |Y_j| < 2^59 + n/2 and no
       intermediate below exceeds 2^61 in magnitude;
    1. y[t_j] = Y_j (other entries 0); g_s = y[2s] + i y[2s+1], s < h = n/2;
    2. G = DFT_h(g) by radix-2 decimation in time: g in bit-reversed order
       (log2 h bits); for hh = 1, 2, .., h/2, every block of 2hh and k < hh:
       (a, c) = (X[b+k], X[b+k+hh]); t = cmul(c, W[k N / hh]);
       X[b+k] = a + t; X[b+k+hh] = a - t;
    3. split, for k = 0..h with G[h] = G[0]: a = G[k], b = G[h-k];
       sr = a.re + b.re; si = a.im - b.im; dr = a.re - b.re; di = a.im + b.im;
       t = cmul((di, -dr), V) with V = W[4k] for k < h, V = (-2^62, 0) for k = h;
       X2[k] = (sr + t.re, si + t.im)  (twice the split output, no halving);
       X2[n-k] = conj(X2[k]) for 0 < k < h;
    4. twist: S2[k] = cmul(X2[k], W[k]), k < n;
    5. m_k = rnd(2^d S2[k].re), m_{k+n} = rnd(2^d S2[k].im), d = s - F - 1,
       s = log2 Delta + 1 - log2 N; |m_k| >= 2^62 is an overflow.
  Twiddles W[k] = (C[k], -S[k]) with C[k] = rnd(2^62 cos(pi k / N)) and
  S[k] = rnd(2^62 sin(pi k / N)), k < N (computed here in 50-digit decimal);
  cmul((ar, ai), (wr, wi)) = (rnd((ar wr - ai wi) / 2^62), rnd((ar wi + ai wr) / 2^62)),
  each numerator exact (128-bit), rounded once.  Multiplication by
  W[0] = (2^62, 0) and W[N/2] = (0, -2^62) is exact, so implementations may
  skip those products.

The FP64 twiddles ``twiddles`` (correctly rounded cos, -sin) serve the
decoder and the direct sum only.
"""
from decimal import Decimal, localcontext
from fractions import Fraction
import functools
import math

import numpy as np

OVERFLOW_LIMIT = 2.0 ** 62     # |m_k| must stay below this (encode error otherwise)


def _pi(prec):
    """pi by Machin's formula in the current decimal context."""
    def arctan_inv(x):
        x = Decimal(x)
        x2 = x * x
        term = 1 / x
        total = term
        n = 1
        eps = Decimal(10) ** -(prec + 5)
        while abs(term) > eps:
            term = -term / x2
            total += term / (2 * n + 1)
            n += 1
        return total
    return 16 * arctan_inv(5) - 4 * arctan_inv(239)


def _sin_cos(theta, prec):
    s = Decimal(0)
    c = Decimal(0)
    term = Decimal(1)          # theta^n / n!
    eps = Decimal(10) ** -(prec + 5)
    n = 0
    while True:
        r = n % 4
        if r == 0:
            c += term
        elif r == 1:
            s += term
        elif r == 2:
            c -= term
        else:
            s -= term
        n += 1
        term = term * theta / n
        if term < eps and n > 4:
            return s, c


@functools.lru_cache(maxsize=None)
def twiddles(log_n: int):
    """T[k] = exp(-i pi k / N) for k < N; (re, im) float64 arrays, correctly rounded."""
    n = 1 << log_n
    quarter = n // 4
    with localcontext() as ctx:
        ctx.prec = 50
        pi = _pi(50)
        cs = []                  # (cos, sin) of pi k / N for k in [0, N/4]
        for k in range(quarter + 1):
            if k == 0:
                cs.append((1.0, 0.0))
                continue
            s, c = _sin_cos(pi * k / n, 50)
            cs.append((float(c), float(s)))
    re = np.empty(n)
    im = np.empty(n)
    for k in range(n):
        # reduce the angle pi k / N to [0, pi/4] by exact symmetries
        if k <= quarter:
            c, s = cs[k]
        elif k <= n // 2:                     # x = pi/2 - theta in [0, pi/4)
            s, c = cs[n // 2 - k]             # cos = sin x, sin = cos x
        elif k <= 3 * quarter:                # x = theta - pi/2 in (0, pi/4]
            cx, sx = cs[k - n // 2]
            c, s = -sx, cx                    # cos = -sin x, sin = cos x
        else:                                 # x = pi - theta in (0, pi/4)
            cx, sx = cs[n - k]
            c, s = -cx, sx                    # cos = -cos x, sin = sin x
        re[k] = c
        im[k] = -s
    return re, im


def slot_index(log_n: int):
    """t_j = (5^j mod 2N - 1) / 4 for j < N/2 (int64 array)."""
    n = 1 << log_n
    half = n // 2
    out = np.empty(half, dtype=np.int64)
    g = 1
    for j in range(half):
        out[j] = (g - 1) // 4
        g = g * 5 % (2 * n)
    return out


def _brv_perm(bits):
    idx = np.arange(1 << bits)
    r = np.zeros_like(idx)
    for b in range(bits):
        r |= ((idx >> b) & 1) << (bits - 1 - b)
    return r


@functools.lru_cache(maxsize=None)
def twiddles_q62(log_n: int):
    """(C, S) int64 arrays: C[k] = rnd(2^62 cos(pi k / N)), S[k] = rnd(2^62 sin(pi k / N)), k < N."""
    n = 1 << log_n
    quarter = n // 4
    one = 1 << Q
    with localcontext() as ctx:
        ctx.prec = 50
        pi = _pi(50)
        scale = Decimal(2) ** Q
        cs = []                  # (C, S) of pi k / N for k in [0, N/4]
        for k in range(quarter + 1):
            if k == 0:
                cs.append((one, 0))
                continue
            s, c = _sin_cos(pi * k / n, 50)
            cs.append((int((c * scale + Decimal("0.5")).to_integral_value(rounding="ROUND_FLOOR")),
                       int((s * scale + Decimal("0.5")).to_integral_value(rounding="ROUND_FLOOR"))))
    C = np.empty(n, dtype=np.int64)
    S = np.empty(n, dtype=np.int64)
    for k in range(n):
        # the same exact symmetries as the FP64 table
        if k <= quarter:
            c, s_ = cs[k]
        elif k <= n // 2:
            s_, c = cs[n // 2 - k]
        elif k <= 3 * quarter:
            cx, sx = cs[k - n // 2]
            c, s_ = -sx, cx
        else:
            cx, sx = cs[n - k]
            c, s_ = -cx, sx
        C[k] = c
        S[k] = s_
    return C, S


Q = 62
HALF_Q = 1 << (Q - 1)


def _obj(a):
    return np.array([int(v) for v in a], dtype=object)


def _cmul(ar, ai, wr, wi):
    """Fixed-point complex product (Python integers, elementwise): each part's
    numerator is exact and rounded once, floor(x / 2^62 + 1/2)."""
    return (ar * wr - ai * wi + HALF_Q) >> Q, (ar * wi + ai * wr + HALF_Q) >> Q


def block_scale(z, log_n: int):
    """Step 0: (F, Y) with Y_j = rnd(z_j 2^F) as Python integers; F is None
    for an all-zero (or empty) input."""
    z = np.asarray(z, dtype=np.float64)
    ns = z.shape[0]
    if ns == 0:
        return None, []
    M = float(np.max(np.abs(z)))
    if not math.isfinite(M):
        raise OverflowError("non-finite slot value")
    if M == 0.0:
        return None, [0] * ns
    e = math.frexp(M)[1]                       # 2^(e-1) <= M < 2^e
    F = 59 - (log_n - 1) - e
    Y = [math.floor(Fraction(float(v)) * Fraction(2) ** F + Fraction(1, 2)) for v in z]
    return F, Y


def encode_fixed(z, log_n: int):
    """Steps 0-4: (F, S2re, S2im) with S2 = 2 * 2^F * S (Python integers, k < n),
    or (None, zeros, zeros) for a zero input."""
    n_ring = 1 << log_n
    n = n_ring // 2
    h = n // 2
    z = np.asarray(z, dtype=np.float64)
    assert z.ndim == 1 and z.shape[0] <= n
    F, Y = block_scale(z, log_n)
    if F is None:
        zero = np.zeros(n, dtype=object)
        return None, zero, zero.copy()
    y = [0] * n
    t = slot_index(log_n)
    for j, v in enumerate(Y):
        y[int(t[j])] = v
    C, S = twiddles_q62(log_n)
    Wr, Wi = _obj(C), -_obj(S)
    lg = h.bit_length() - 1
    perm = _brv_perm(lg)
    xr = _obj(y[0::2])[perm]                   # step 1
    xi = _obj(y[1::2])[perm]
    hh = 1                                     # step 2
    while hh < h:
        k = np.arange(hh)
        wr, wi = Wr[k * (n_ring // hh)], Wi[k * (n_ring // hh)]
        xr = xr.reshape(-1, 2 * hh)
        xi = xi.reshape(-1, 2 * hh)
        ar, ai = xr[:, :hh], xi[:, :hh]
        tr, ti = _cmul(xr[:, hh:], xi[:, hh:], wr, wi)
        xr = np.concatenate([ar + tr, ar - tr], axis=1).reshape(-1)
        xi = np.concatenate([ai + ti, ai - ti], axis=1).reshape(-1)
        hh *= 2
    k = np.arange(h + 1)                       # step 3
    Gr = np.concatenate([xr, xr[:1]])
    Gi = np.concatenate([xi, xi[:1]])
    ar, ai = Gr[k], Gi[k]
    br, bi = Gr[h - k], Gi[h - k]
    sr, si = ar + br, ai - bi
    dr, di = ar - br, ai + bi
    vr = np.concatenate([Wr[4 * k[:-1]], _obj([-(1 << Q)])])
    vi = np.concatenate([Wi[4 * k[:-1]], _obj([0])])
    tr, ti = _cmul(di, -dr, vr, vi)
    x2r = np.empty(n, dtype=object)
    x2i = np.empty(n, dtype=object)
    x2r[: h + 1] = sr + tr
    x2i[: h + 1] = si + ti
    x2r[h + 1:] = x2r[1:h][::-1]
    x2i[h + 1:] = -x2i[1:h][::-1]
    s2r, s2i = _cmul(x2r, x2i, Wr[:n], Wi[:n])  # step 4
    return F, s2r, s2i


def encode_real(z, log_n: int, log2_delta: int):
    """The unrounded coefficients 2^(s-F-1) S2 of step 5 (float64, length N)."""
    F, s2r, s2i = encode_fixed(z, log_n)
    if F is None:
        return np.zeros(1 << log_n)
    d = log2_delta + 1 - log_n - F - 1
    return np.array([math.ldexp(float(v), d) for v in np.concatenate([s2r, s2i])])


def _rnd_shift(v, d):
    """rnd(2^d v) for a Python integer v."""
    if d >= 0:
        return v << d
    return (v + (1 << (-d - 1))) >> (-d)


def encode(z, log_n: int, log2_delta: int):
    """Integer plaintext coefficients m_k (int64 array of length N)."""
    n_ring = 1 << log_n
    F, s2r, s2i = encode_fixed(z, log_n)
    if F is None:
        return np.zeros(n_ring, dtype=np.int64)
    d = log2_delta + 1 - log_n - F - 1
    m = [_rnd_shift(int(v), d) for v in np.concatenate([s2r, s2i])]
    if any(abs(v) >= OVERFLOW_LIMIT for v in m):
        raise OverflowError("encoded coefficient magnitude >= 2^62")
    return np.array(m, dtype=np.int64)


def _cos_table(log_n: int):
    """cos(pi x / N) for x < 2N, correctly rounded: the table ``twiddles`` gives
    x < N, and cos(pi + t) = -cos(t) gives the rest exactly (a sign flip)."""
    re, _ = twiddles(log_n)
    return np.concatenate([re, -re])


def encode_direct(z, log_n: int, log2_delta: int, chunk: int = 256):
    """The defining sum (2 Delta / N) Re sum_j z_j zeta^(-5^j k), k < N, in FP64
    (pin only; O(N^2)).  Term j of output k is z_j cos(pi x / N) with the
    exponent x = 5^j k mod 2N reduced exactly and the cosine taken from the
    correctly rounded table (one rounding), the product rounded once; the terms
    of each output are added pairwise (zero-padded to a power of two, halves
    added level by level), so the result is within
    ``encode_direct_error_bound`` of the exact sum."""
    n = 1 << log_n
    z = np.asarray(z, dtype=np.float64)
    ns = z.shape[0]
    if ns == 0:
        return np.zeros(n)
    width = 1 << max(0, (ns - 1).bit_length())
    zp = np.zeros(width)
    zp[:ns] = z
    g = np.zeros(width, dtype=np.int64)
    g[:ns] = [pow(5, j, 2 * n) for j in range(ns)]
    cos_t = _cos_table(log_n)
    out = np.empty(n)
    for k0 in range(0, n, chunk):
        k = np.arange(k0, min(k0 + chunk, n), dtype=np.int64)
        t = cos_t[(k[:, None] * g[None, :]) % (2 * n)] * zp[None, :]
        while t.shape[1] > 1:                       # pairwise: one rounding per level
            h = t.shape[1] // 2
            t = t[:, :h] + t[:, h:]
        out[k0:k0 + k.shape[0]] = t[:, 0]
    return out * (2.0 * 2.0 ** log2_delta / n)       # a power of two: exact


def encode_direct_error_bound(z, log_n: int, log2_delta: int):
    """|encode_direct - exact| (coefficient units), by standard floating-point
    error analysis with unit roundoff u = 2^-53 and gamma_k = k u / (1 - k u):
    a term is z_j c (1 + d1)(1 + d2), |d1|, |d2| <= u (table entry, product),
    so it is off by at most gamma_2 |z_j|; pairwise summation over 2^L terms
    adds at most gamma_L times the sum of the terms' moduli; together
    gamma_(L+2) sum_j |z_j|, plus half the smallest subnormal per product
    (gradual underflow), times the exact scale 2 Delta / N."""
    z = np.asarray(z, dtype=np.float64)
    ns = z.shape[0]
    if ns == 0:
        return 0.0
    L = max(0, (ns - 1).bit_length())
    u = 2.0 ** -53
    k = L + 2
    gamma = k * u / (1.0 - k * u)
    return (gamma * math.fsum(abs(float(v)) for v in z) + ns * 2.0 ** -1075) * 2.0 ** (log2_delta + 1 - log_n)


def decode(m, log_n: int, log2_delta: int, n_slots: int):
    """Slots z_j = Delta^-1 m(zeta^(5^j)) (real parts), from exact integer
    coefficients (a sequence of Python ints or an int array); direct sum."""
    n = 1 << log_n
    mf = np.array([float(int(x)) for x in m], dtype=np.float64)
    k = np.arange(n, dtype=np.int64)
    out = np.empty(n_slots)
    g = 1
    for j in range(n_slots):
        e = (g * k) % (2 * n)
        out[j] = np.dot(mf, np.cos(np.pi * e / n))
        g = g * 5 % (2 * n)
    return out / 2.0 ** log2_delta


def encode_error_bound(z, log_n: int, log2_delta: int):
    """A bound on |encode_real - exact| (in coefficient units) for the
    fixed-point procedure, in units of Y (2^-F): a cmul part is off by at most
    1/2 (rounding) + 2^-63 (|a.re| + |a.im|) (twiddle quantisation, <= 0.18
    for operands of modulus <= 2^60), so a cmul adds at most 0.96 in modulus;
    an input part by at most 1/2 (0.71 for g).  Through the L = log2 h DIT
    stages errors pass with unit-modulus weights: a DFT output is off by at
    most 2^L (0.71 + 0.96); the split gives X2 off by at most 4 of those plus
    0.96, the twist adds 0.96: 6.68 h + 1.92 <= 3.4 n + 2.  Coefficients are
    2^(s-F-1) S2 (s = log2 Delta + 1 - log2 N)."""
    n = 1 << (log_n - 1)
    F, _ = block_scale(z, log_n)
    if F is None:
        return 0.0
    return math.ldexp(3.4 * n + 2.0, log2_delta + 1 - log_n - F - 1)
