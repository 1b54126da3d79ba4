"""Pins for the oracle's BFV / BGV slot batching (oracle/bfvbgv.py):
evaluation of the encoded polynomial at psi_t^(a_s) by Horner's rule (the
defining property, written out independently of the NTT), closed forms (the
constant vector and the monomial X), the bijection, and the ring isomorphism
(slot-wise products are negacyclic products mod t, schoolbook from the C
library).
"""
import numpy as np
import pytest

from oracle import bfvbgv as B
from oracle import numtheory, ring

CASES = [(4, 97), (4, 65537), (6, 257), (8, 65537), (10, 12289)]


def _t_ok(log_n, t):
    return numtheory.is_prime(t) and t % (2 << log_n) == 1


@pytest.mark.parametrize("log_n,t", CASES)
def test_encode_evaluates_at_the_slot_roots(log_n, t):
    assert _t_ok(log_n, t)
    n = 1 << log_n
    rng = np.random.default_rng(log_n)
    x = rng.integers(0, t, n)
    m = B.batch_encode(x, t, log_n)
    psi = numtheory.find_psi(t, log_n)
    exps = B.slot_exponents(log_n)
    assert sorted(exps) == list(range(1, 2 * n, 2))           # every odd power once
    for s in list(range(4)) + [n // 2, n // 2 + 1, n - 1]:
        r = pow(psi, exps[s], t)
        acc = 0
        for c in reversed(m):                                  # Horner
            acc = (acc * r + c) % t
        assert acc == int(x[s]) % t, s


@pytest.mark.parametrize("log_n,t", CASES)
def test_closed_forms_and_bijection(log_n, t):
    n = 1 << log_n
    assert B.batch_encode([7] * n, t, log_n) == [7] + [0] * (n - 1)
    psi = numtheory.find_psi(t, log_n)
    X = [0, 1] + [0] * (n - 2)
    assert B.batch_decode(X, t, log_n) == [pow(psi, a, t) for a in B.slot_exponents(log_n)]
    rng = np.random.default_rng(1)
    x = [int(v) for v in rng.integers(0, t, n)]
    assert B.batch_decode(B.batch_encode(x, t, log_n), t, log_n) == x
    m = [int(v) for v in rng.integers(0, t, n)]
    assert B.batch_encode(B.batch_decode(m, t, log_n), t, log_n) == m


@pytest.mark.parametrize("log_n,t", [(4, 97), (6, 257), (8, 65537)])
def test_slotwise_product_is_ring_product(log_n, t):
    n = 1 << log_n
    rng = np.random.default_rng(2)
    x, y = rng.integers(0, t, n), rng.integers(0, t, n)
    mx = np.array(B.batch_encode(x, t, log_n), dtype=np.uint64)
    my = np.array(B.batch_encode(y, t, log_n), dtype=np.uint64)
    prod = ring.negacyclic_mul(mx, my, t)
    assert [int(v) for v in prod] == B.batch_encode([(int(a) * int(b)) % t for a, b in zip(x, y)], t, log_n)
