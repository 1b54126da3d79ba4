"""Number theory for the RNS prime chain.  TEST INFRASTRUCTURE ONLY (see oracle/__init__).

The paper takes its coefficient modulus from SEAL (Section "System
Implementation") and does not state how primes or roots are chosen.  The
reading used here:

* prime rule: for each bit size b of the chain, left to right, the largest
  prime q < 2^b with q = 1 (mod 2N) that is not already in the chain;
* root rule: psi = the smallest primitive 2N-th root of unity mod q, i.e. the
  minimum of psi0^k over odd k for any primitive 2N-th root psi0.
"""

_MR_BASES = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)


def is_prime(n: int) -> bool:
    """Deterministic Miller-Rabin; the first 12 prime bases are exact for n < 3.3e24."""
    if n < 2:
        return False
    for p in _MR_BASES:
        if n % p == 0:
            return n == p
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in _MR_BASES:
        x = pow(a, d, n)
        if x == 1 or x == n - 1:
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def gen_primes(log_n: int, bits) -> list:
    """Prime chain: largest unused prime q < 2^b, q = 1 mod 2N, per entry b."""
    two_n = 2 << log_n
    out = []
    for b in bits:
        q = ((2 ** b - 2) // two_n) * two_n + 1   # largest value < 2^b that is 1 mod 2N
        while q > two_n:
            if q not in out and is_prime(q):
                break
            q -= two_n
        else:
            raise ValueError(f"no prime below 2^{b} that is 1 mod {two_n}")
        out.append(q)
    return out


def find_psi(q: int, log_n: int) -> int:
    """Smallest primitive 2N-th root of unity mod q (psi^N = -1 mod q)."""
    n = 1 << log_n
    two_n = 2 * n
    assert (q - 1) % two_n == 0
    g = 2
    while True:
        psi0 = pow(g, (q - 1) // two_n, q)
        if pow(psi0, n, q) == q - 1:
            break
        g += 1
    best = psi0
    step = psi0 * psi0 % q
    x = psi0
    for _ in range(n - 1):          # psi0^k for odd k in [3, 2N)
        x = x * step % q
        if x < best:
            best = x
    return best


def brv(x: int, bits: int) -> int:
    """Bit reversal of x over `bits` bits."""
    r = 0
    for _ in range(bits):
        r = (r << 1) | (x & 1)
        x >>= 1
    return r
