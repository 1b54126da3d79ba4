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
  that an independent implementation can reproduce the integers bit for bit.
  y is real, so its length-n DFT is taken through a complex DFT of half the
  length (the standard real-input split):
    1. y[t_j] = z_j (other entries 0); g_s = y[2s] + i y[2s+1], s < h = n/2;
    2. G = DFT_h(g) by radix-2 decimation in time: g in bit-reversed order
       (log2 h bits); for hh = 1, 2, .., h/2, every block of 2hh and k < hh:
       w = T[k N / hh]; (a, c) = (X[b+k], X[b+k+hh]);
       tr = c.re*w.re - c.im*w.im; ti = c.re*w.im + c.im*w.re;
       X[b+k] = (a.re + tr, a.im + ti); X[b+k+hh] = (a.re - tr, a.im - ti);
    3. split, for k = 0..h with G[h] = G[0]: a = G[k], b = G[h-k];
       sr = a.re + b.re; si = a.im - b.im; dr = a.re - b.re; di = a.im + b.im;
       E = (0.5*sr, 0.5*si); O = (0.5*di, -(0.5*dr));
       W = T[4k] for k < h, W = (-1, 0) for k = h;
       t = (O.re*W.re - O.im*W.im, O.re*W.im + O.im*W.re);
       X[k] = (E.re + t.re, E.im + t.im); X[n-k] = conj(X[k]) for 0 < k < h;
    4. twist: S[k] = X[k] * T[k] (the same complex product formula), k < n;
    5. m_k = rint(2^s Re S[k]), m_{k+n} = rint(2^s Im S[k]), s = log2 Delta + 1 - log2 N
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


def _dit(xr, xi, log_n, tr_, ti_):
    """Radix-2 DIT butterflies (step 2) on bit-reversed input, in place order."""
    n_ring = 1 << log_n
    size = xr.shape[0]
    hh = 1
    while hh < size:
        k = np.arange(hh)
        wr = tr_[k * (n_ring // hh)]
        wi = ti_[k * (n_ring // hh)]
        xr = xr.reshape(-1, 2 * hh)
        xi = xi.reshape(-1, 2 * hh)
        ar, ai = xr[:, :hh].copy(), xi[:, :hh].copy()
        cr, ci = xr[:, hh:].copy(), xi[:, hh:].copy()
        tr = cr * wr - ci * wi
        ti = cr * wi + ci * wr
        xr = np.concatenate([ar + tr, ar - tr], axis=1).reshape(-1)
        xi = np.concatenate([ai + ti, ai - ti], axis=1).reshape(-1)
        hh *= 2
    return xr, xi


def encode_real(z, log_n: int, log2_delta: int):
    """Steps 1-4 of the specified procedure and the power-of-two scaling
    (exact); returns the N unrounded coefficients as float64."""
    n_ring = 1 << log_n
    n = n_ring // 2
    h = n // 2
    z = np.asarray(z, dtype=np.float64)
    assert z.ndim == 1 and z.shape[0] <= n
    y = np.zeros(n)
    y[slot_index(log_n)[: z.shape[0]]] = z
    lg = h.bit_length() - 1
    perm = _brv_perm(lg)
    tr_, ti_ = twiddles(log_n)
    gr, gi = _dit(y[0::2][perm].copy(), y[1::2][perm].copy(), log_n, tr_, ti_)   # steps 1, 2
    # step 3: split the half-length transform into X[0..n)
    k = np.arange(h + 1)
    Gr = np.concatenate([gr, gr[:1]])
    Gi = np.concatenate([gi, gi[:1]])
    ar, ai = Gr[k], Gi[k]
    br, bi = Gr[h - k], Gi[h - k]
    sr = ar + br
    si = ai - bi
    dr = ar - br
    di = ai + bi
    er = 0.5 * sr
    ei = 0.5 * si
    o_r = 0.5 * di
    o_i = -(0.5 * dr)
    wr = np.where(k < h, tr_[(4 * k) % n_ring], -1.0)
    wi = np.where(k < h, ti_[(4 * k) % n_ring], 0.0)
    t_r = o_r * wr - o_i * wi
    t_i = o_r * wi + o_i * wr
    xk_r = er + t_r
    xk_i = ei + t_i
    xr = np.empty(n)
    xi = np.empty(n)
    xr[: h + 1] = xk_r
    xi[: h + 1] = xk_i
    xr[h + 1:] = xk_r[1:h][::-1]
    xi[h + 1:] = -xk_i[1:h][::-1]
    # step 4: twist
    wr = tr_[:n]
    wi = ti_[:n]
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
