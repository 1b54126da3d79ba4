"""CKKS encoder and decoder (canonical embedding).  TEST INFRASTRUCTURE ONLY.

The paper assumes the message is already encoded (Section "Zinc",
"Construction") and fixes only the scale Delta = 2^55 (Section "System
Implementation").  Definition used (standard CKKS): for real slots z_j,
j < n = N/2 (missing slots are zero), the plaintext polynomial m in
Z[X]/(X^N + 1) has coefficients

    m_k = rint( (2 Delta / N) * Re sum_j z_j * zeta^(-5^j k) ),   zeta = exp(i pi / N),

i.e. m(zeta^(5^j)) ~ Delta z_j.  With t_j = (5^j mod 2N - 1)/4 (a bijection of
[0, n)) the sum S_k = sum_j z_j zeta^(-5^j k), k < n, equals
zeta^(-k) * DFT_n(y)_k with y_{t_j} = z_j, and m_k = scale Re S_k,
m_{k+n} = scale Im S_k (because zeta^(-5^j n) = -i).

Two forms:
* ``encode_direct``: the defining sum, evaluated term by term (pin only).
* ``encode``: the FP64 procedure whose every IEEE operation is specified, so
  that an independent implementation can reproduce the integers bit for bit:
    1. y[t_j] = z_j; X = y in bit-reversed order (log2 n bits);
    2. radix-2 decimation-in-time: for h = 1, 2, .., n/2, every block of 2h and
       k < h: w = T[k N / h]; (a, c) = (X[b+k], X[b+k+h]);
       tr = c.re*w.re - c.im*w.im; ti = c.re*w.im + c.im*w.re;
       X[b+k] = (a.re + tr, a.im + ti); X[b+k+h] = (a.re - tr, a.im - ti);
    3. twist: S[k] = X[k] * T[k] with the same complex product formula;
    4. m_k = rint(2^s Re S[k]), m_{k+n} = rint(2^s Im S[k]), s = log2 Delta + 1 - log2 N
       (an exact power-of-two scaling), ties to even.
  Each product and sum is a separate correctly rounded FP64 operation (no
  fused multiply-add).  T[k] = cos(pi k / N) - i sin(pi k / N), k < N, each
  part correctly rounded to FP64 (computed here in 50-digit decimal).
"""
from decimal import Decimal, localcontext
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


def encode_real(z, log_n: int, log2_delta: int):
    """Steps 1-3 of the specified FFT procedure and the power-of-two scaling
    (exact); returns the N unrounded coefficients as float64."""
    n = 1 << log_n
    half = n // 2
    z = np.asarray(z, dtype=np.float64)
    assert z.ndim == 1 and z.shape[0] <= half
    y = np.zeros(half)
    y[slot_index(log_n)[: z.shape[0]]] = z
    lg = half.bit_length() - 1
    xr = y[_brv_perm(lg)].copy()
    xi = np.zeros(half)
    tr_, ti_ = twiddles(log_n)
    h = 1
    while h < half:
        k = np.arange(h)
        wr = tr_[k * (n // h)]
        wi = ti_[k * (n // h)]
        xr = xr.reshape(-1, 2 * h)
        xi = xi.reshape(-1, 2 * h)
        ar, ai = xr[:, :h].copy(), xi[:, :h].copy()
        cr, ci = xr[:, h:].copy(), xi[:, h:].copy()
        tr = cr * wr - ci * wi
        ti = cr * wi + ci * wr
        xr = np.concatenate([ar + tr, ar - tr], axis=1).reshape(-1)
        xi = np.concatenate([ai + ti, ai - ti], axis=1).reshape(-1)
        h *= 2
    wr = tr_[:half]
    wi = ti_[:half]
    sr = xr * wr - xi * wi
    si = xr * wi + xi * wr
    scale = 2.0 ** (log2_delta + 1 - log_n)
    return np.concatenate([sr * scale, si * scale])


def encode(z, log_n: int, log2_delta: int):
    """Integer plaintext coefficients m_k (int64 array of length N)."""
    m = np.rint(encode_real(z, log_n, log2_delta))
    if not np.all(np.isfinite(m)) or np.any(np.abs(m) >= OVERFLOW_LIMIT):
        raise OverflowError("encoded coefficient magnitude >= 2^62")
    return m.astype(np.int64)


def encode_direct(z, log_n: int, log2_delta: int):
    """The defining sum (2 Delta / N) Re sum_j z_j zeta^(-5^j k), k < N, in FP64
    term by term with exactly reduced angles (pin only; O(N^2))."""
    n = 1 << log_n
    z = np.asarray(z, dtype=np.float64)
    g = np.array([pow(5, j, 2 * n) for j in range(z.shape[0])], dtype=np.int64)
    k = np.arange(n, dtype=np.int64)
    out = np.zeros(n)
    for j in range(z.shape[0]):
        e = (g[j] * k) % (2 * n)                      # exponent of zeta^(+5^j k), exact
        out += z[j] * np.cos(np.pi * e / n)           # Re zeta^(-x) = cos(pi x / N)
    return out * (2.0 * 2.0 ** log2_delta / n)


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
    """A bound on |encode_real - exact| from FP64 rounding: each of the
    log2(n)+1 levels of products/sums adds at most ~4 ulp of the running
    magnitude, which is bounded by sum |z| (times the scale)."""
    n = 1 << log_n
    lg = (n // 2).bit_length() - 1
    scale = 2.0 ** (log2_delta + 1 - log_n)
    mag = float(np.sum(np.abs(z))) * scale
    return 8.0 * (lg + 2) * mag * 2.0 ** -53 + math.ulp(max(mag, 1.0))
