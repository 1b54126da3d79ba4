"""GB300-native (sm_103a) RNS-CKKS public-key encryption, vanilla and Zinc
(arXiv 2408.07304), behind the C ABI of include/zinc.h.

The compute path is libzinc.so (built by ``build.build()``); ``api`` is its
ctypes binding with the same entry-point names.
"""
from . import workloads  # noqa: F401
from .api import (  # noqa: F401
    Context, PublicKey, SecretKey, ZincCache, ZincError, as_u64, ckks_add, ckks_decrypt, ckks_decrypt_decode,
    ckks_encode, ckks_encode_ragged, ckks_encrypt, ckks_encrypt_ms, ckks_encrypt_ragged, ckks_keygen, data_level,
    lib, zinc_encrypt, zinc_encrypt_ragged, zinc_precompute,
    zinc_precompute_ms, zn_ctx_create, zn_host_cdt,
    zn_host_encoder_twiddles, zn_host_primes, zn_host_psi, zn_ntt_forward, zn_ntt_inverse, zn_pk_export,
    zn_pk_import, zn_sample, zn_sk_export, zn_sk_import, zn_sync_status, zn_zcache_export, zn_zcache_import,
)
