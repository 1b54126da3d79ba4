"""The C ABI library loads without a GPU, exports every entry point that
include/zinc.h declares, and its host-side tables (prime chain, roots,
encoder twiddles, chi thresholds) equal the oracle's, computed independently.
"""
import os
import re

import numpy as np
import pytest

from oracle import encoder, numtheory, sampler
from paper_2408_07304_gb300 import api, workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    from paper_2408_07304_gb300 import build
    build.build()
    return api.lib()


def _declared():
    text = open(os.path.join(ROOT, "include", "zinc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b((?:zn|ckks|zinc)_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported(built):
    names = _declared()
    assert len(names) >= 25
    for n in names:
        assert hasattr(built, n), n
        assert n in api._SIGS, f"binding lacks {n}"


def test_strerror(built):
    assert api.strerror(0) == "ok"
    assert "overflow" in api.strerror(api.ZN_EOVERFLOW)


@pytest.mark.parametrize("name", ["single", "batched", "throughput", "large", "paper"])
def test_prime_chain_and_roots_match_oracle(built, name):
    w = workloads.WORKLOADS[name]
    qs = api.zn_host_primes(w.log_n, w.bits)
    assert qs == numtheory.gen_primes(w.log_n, w.bits)
    for q in qs[:3]:
        assert api.zn_host_psi(q, w.log_n) == numtheory.find_psi(q, w.log_n)


@pytest.mark.parametrize("log_n", [4, 8, 12, 13, 14, 15])
def test_encoder_twiddles_bitwise(built, log_n):
    re_, im_ = api.zn_host_encoder_twiddles(log_n)
    ore, oim = encoder.twiddles(log_n)
    assert np.array_equal(re_.view(np.uint64), ore.view(np.uint64))
    assert np.array_equal(im_.view(np.uint64), oim.view(np.uint64))


@pytest.mark.parametrize("log_n", [4, 8, 12, 13, 14, 15])
def test_encoder_twiddles_q62_equal(built, log_n):
    c, s = api.zn_host_encoder_twiddles_q62(log_n)
    oc, os_ = encoder.twiddles_q62(log_n)
    assert np.array_equal(c, oc) and np.array_equal(s, os_)


def test_cdt_thresholds_equal(built):
    assert api.zn_host_cdt() == list(sampler.cdt_thresholds())


def test_invalid_params_rejected_without_gpu(built):
    # parameter validation happens before any device call
    with pytest.raises(api.ZincError) as e:
        api.Context(3, (40,), 20)
    assert e.value.status == api.ZN_EINVAL
    with pytest.raises(api.ZincError):
        api.Context(12, (70,), 20)
    with pytest.raises(api.ZincError):
        api.Context(12, (40,) * 17, 20)
    with pytest.raises(api.ZincError) as e:
        api.zn_host_primes(12, (20,) * 40)        # runs out of 20-bit primes = 1 mod 8192
    assert e.value.status == api.ZN_ENOPRIME


def test_alloc_fault_injector_arguments(built):
    # host-side only: sets a counter, touches no device state
    api.zn_inject_alloc_failures(3)
    api.zn_inject_alloc_failures(0)
    with pytest.raises(api.ZincError) as e:
        api.zn_inject_alloc_failures(-1)
    assert e.value.status == api.ZN_EINVAL


def test_wait_probe_arguments_without_gpu(built):
    # a null context is refused before any device call
    lib = api.lib()
    assert lib.zn_probe_wait_timeout(None, 1, None) == api.ZN_EINVAL
    assert lib.zn_probe_wait_timeout(None, 0, None) == api.ZN_EINVAL
