"""ctypes binding of include/zinc.h, with the same entry-point names.

Argument marshalling only: every step of encoding, sampling, transforming and
encrypting runs in the sm_103a kernels of libzinc.so.  Device buffers are
torch CUDA tensors (uint64 residues are carried in int64 tensors, bit for
bit); torch supplies memory and streams, nothing else.  There is no CPU
fallback: if libzinc.so has not been built, the first call raises.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libzinc.so")
MAX_PRIMES = 16

ZN_OK, ZN_EINVAL, ZN_ENOMEM, ZN_EOVERFLOW, ZN_ECUDA, ZN_ETIMEOUT, ZN_ENOPRIME, ZN_ELIMIT = 0, -1, -2, -3, -4, -5, -6, -7
NOALLOC_SCRATCH_BYTES = 16 << 20

# sampler kinds for zn_sample
KIND_TERNARY, KIND_GAUSSIAN, KIND_UNIFORM = 0, 1, 2
# sampling domains (counter word 1, bits 24..31)
DOM_ENC, DOM_ZINC, DOM_KEYGEN, DOM_CACHE = 0, 1, 2, 3


class ZincError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__(f"{what}: {strerror(status)} ({status})")


class _Params(ctypes.Structure):
    _fields_ = [("log_n", ctypes.c_uint32), ("n_primes", ctypes.c_uint32),
                ("prime_bits", ctypes.c_uint32 * MAX_PRIMES), ("log2_delta", ctypes.c_uint32)]


_lib = None
_vp = ctypes.c_void_p
_u32 = ctypes.c_uint32
_u64 = ctypes.c_uint64
_i32 = ctypes.c_int
_pp = ctypes.POINTER(ctypes.c_void_p)

_SIGS = {
    "zn_ctx_create": (_i32, [ctypes.POINTER(_Params), _i32, _pp]),
    "zn_ctx_destroy": (None, [_vp]),
    "zn_ctx_primes": (_i32, [_vp, _vp, _vp]),
    "zn_sync_status": (_i32, [_vp, _vp]),
    "zn_strerror": (ctypes.c_char_p, [_i32]),
    "ckks_keygen": (_i32, [_vp, _u64, _pp, _pp]),
    "zn_sk_destroy": (None, [_vp]),
    "zn_pk_destroy": (None, [_vp]),
    "zn_pk_export": (_i32, [_vp, _vp]),
    "zn_pk_import": (_i32, [_vp, _vp, _pp]),
    "zn_sk_export": (_i32, [_vp, _vp]),
    "zn_sk_import": (_i32, [_vp, _vp, _pp]),
    "ckks_encode": (_i32, [_vp, _vp, _u32, _u32, _vp, _vp]),
    "ckks_encode_ragged": (_i32, [_vp, _vp, _vp, _u32, _u32, _vp, _vp]),
    "ckks_encrypt_ragged": (_i32, [_vp, _vp, _vp, _vp, _u32, _u32, _u64, _vp, _vp, _vp]),
    "zinc_encrypt_ragged": (_i32, [_vp, _vp, _vp, _vp, _u32, _u32, _u64, _vp, _vp, _vp]),
    "ckks_encrypt": (_i32, [_vp, _vp, _vp, _u32, _u32, _u64, _vp, _vp, _vp]),
    "zinc_precompute": (_i32, [_vp, _vp, _u64, _pp]),
    "zn_zcache_destroy": (None, [_vp]),
    "zn_zcache_export": (_i32, [_vp, _vp]),
    "zn_zcache_import": (_i32, [_vp, _vp, _pp]),
    "zinc_encrypt": (_i32, [_vp, _vp, _vp, _u32, _u32, _u64, _vp, _vp, _vp]),
    "zinc_encrypt_noalloc": (_i32, [_vp, _vp, _vp, _u32, _u32, _u64, _vp, _vp, _vp]),
    "ckks_encrypt_ms": (_i32, [_vp, _vp, _vp, _u32, _u32, _u64, _vp, _vp, _vp]),
    "zinc_precompute_ms": (_i32, [_vp, _vp, _u64, _vp, _pp]),
    "zn_slot_encoder_create": (_i32, [_vp, _u64, _pp]),
    "zn_slot_encoder_destroy": (None, [_vp]),
    "zn_slots_encode": (_i32, [_vp, _vp, _u32, _vp, _vp]),
    "zn_slots_decode": (_i32, [_vp, _vp, _u32, _vp, _vp]),
    "zinc_nbasis_create": (_i32, [_vp, _u32, _u64, _pp]),
    "zn_nbasis_destroy": (None, [_vp]),
    "ckks_encode_ntt": (_i32, [_vp, _vp, _u32, _u32, _vp, _vp]),
    "zinc_encrypt_ntt": (_i32, [_vp, _vp, _vp, _vp, _u32, _u64, _vp, _vp, _vp]),
    "bfv_encrypt": (_i32, [_vp, _vp, _u64, _vp, _u32, _u64, _vp, _vp, _vp]),
    "bfv_zinc_encrypt": (_i32, [_vp, _vp, _u64, _vp, _u32, _u64, _vp, _vp, _vp]),
    "bfv_decrypt": (_i32, [_vp, _vp, _u64, _vp, _u32, _vp, _vp]),
    "bgv_keygen": (_i32, [_vp, _u64, _u64, _pp, _pp]),
    "bgv_zinc_precompute": (_i32, [_vp, _vp, _u64, _pp]),
    "bgv_encrypt": (_i32, [_vp, _vp, _vp, _u32, _u64, _vp, _vp, _vp]),
    "bgv_zinc_encrypt": (_i32, [_vp, _vp, _vp, _u32, _u64, _vp, _vp, _vp]),
    "bgv_decrypt": (_i32, [_vp, _vp, _u64, _vp, _u32, _vp, _vp]),
    "ckks_decrypt": (_i32, [_vp, _vp, _vp, _u32, _vp, _vp]),
    "ckks_decrypt_decode": (_i32, [_vp, _vp, _vp, _u32, _u32, _vp, _vp]),
    "ckks_add": (_i32, [_vp, _vp, _vp, _u32, _vp, _vp]),
    "zn_ntt_forward": (_i32, [_vp, _vp, _u32, _vp]),
    "zn_ntt_inverse": (_i32, [_vp, _vp, _u32, _vp]),
    "zn_sample": (_i32, [_vp, _i32, _u64, _u32, _u32, _u32, _u64, _u32, _vp, _vp]),
    "zn_chi_eval": (_i32, [_vp, _vp, _u32, _vp, _vp]),
    "zn_encrypt_host": (_i32, [_vp, _vp, _vp, _vp, _u32, _u32, _u64, _vp, _vp, _u32]),
    "zn_encrypt_host_packed": (_i32, [_vp, _vp, _vp, _vp, _u32, _u32, _u64, _vp, _vp, _u32]),
    "zn_ct_packed_words": (ctypes.c_size_t, [_vp]),
    "zn_ct_pack": (_i32, [_vp, _vp, ctypes.c_size_t, _vp, _vp]),
    "zn_ct_unpack": (_i32, [_vp, _vp, ctypes.c_size_t, _vp, _vp]),
    "zn_batch_create": (_i32, [_vp, _u32, _i32, _pp]),
    "zn_batch_destroy": (None, [_vp]),
    "zn_batch_run": (_i32, [_vp, _vp, _i32]),
    "zn_batch_info": (_i32, [_vp, _vp, _vp]),
    "zn_set_variant": (_i32, [_vp, _i32]),
    "zn_get_variant": (_i32, [_vp]),
    "zn_autotune": (_i32, [_vp, _vp, _vp, _u32, _vp, _vp]),
    "zn_probe_butterfly": (_i32, [_i32, _vp]),
    "zn_probe_butterfly_relaxed": (_i32, [_i32, _vp]),
    "zn_inject_alloc_failures": (_i32, [_i32]),
    "zn_probe_wait_timeout": (_i32, [_vp, _u32, _vp]),
    "zn_timing_enable": (_i32, [_vp, _i32]),
    "zn_timing_read": (_i32, [_vp, _i32, _vp, _vp]),
    "zn_host_primes": (_i32, [_u32, _vp, _u32, _vp]),
    "zn_host_psi": (_u64, [_u64, _u32]),
    "zn_host_encoder_twiddles": (_i32, [_u32, _vp, _vp]),
    "zn_host_encoder_twiddles_q62": (_i32, [_u32, _vp, _vp]),
    "zn_host_cdt": (_i32, [_vp]),
}


def lib():
    """Load libzinc.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libzinc.so is not built ({LIB_PATH}); run "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def strerror(status):
    return lib().zn_strerror(status).decode()


def _check(status, what):
    if status != ZN_OK:
        raise ZincError(status, what)


def _stream(stream):
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dev(t, dtype, shape, what):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what}: expected a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{what}: expected dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{what}: tensor must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{what}: expected shape {tuple(shape)}, got {tuple(t.shape)}")
    return t.data_ptr()


# ----------------------------------------------------------------- handles

class Context:
    """A parameter set resident on one device (zn_ctx)."""

    def __init__(self, log_n, prime_bits, log2_delta, device=0):
        if len(prime_bits) > MAX_PRIMES or len(prime_bits) == 0:
            raise ZincError(ZN_EINVAL, "zn_ctx_create")
        p = _Params()
        p.log_n = log_n
        p.n_primes = len(prime_bits)
        for i, b in enumerate(prime_bits):
            p.prime_bits[i] = b
        p.log2_delta = log2_delta
        h = ctypes.c_void_p()
        _check(lib().zn_ctx_create(ctypes.byref(p), device, ctypes.byref(h)), "zn_ctx_create")
        self._h = h
        self.log_n = log_n
        self.n = 1 << log_n
        self.prime_bits = tuple(prime_bits)
        self.L = len(prime_bits)
        self.log2_delta = log2_delta
        self.device = device
        qs = (ctypes.c_uint64 * self.L)()
        ps = (ctypes.c_uint64 * self.L)()
        _check(lib().zn_ctx_primes(h, qs, ps), "zn_ctx_primes")
        self.primes = [int(x) for x in qs]
        self.psis = [int(x) for x in ps]

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            lib().zn_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _Handle:
    _destroy = None

    def __init__(self, ctx, h):
        self.ctx = ctx
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            getattr(lib(), self._destroy)(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SecretKey(_Handle):
    _destroy = "zn_sk_destroy"


class PublicKey(_Handle):
    _destroy = "zn_pk_destroy"


class ZincCache(_Handle):
    _destroy = "zn_zcache_destroy"


class NttBasis(_Handle):
    _destroy = "zn_nbasis_destroy"


class SlotEncoder(_Handle):
    _destroy = "zn_slot_encoder_destroy"


# ------------------------------------------------------------ entry points

def zn_ctx_create(log_n, prime_bits, log2_delta, device=0):
    return Context(log_n, prime_bits, log2_delta, device)


def zn_sync_status(ctx, stream=None):
    _check(lib().zn_sync_status(ctx.handle, _stream(stream)), "device status")


def ckks_keygen(ctx, seed):
    sk, pk = ctypes.c_void_p(), ctypes.c_void_p()
    _check(lib().ckks_keygen(ctx.handle, seed, ctypes.byref(sk), ctypes.byref(pk)), "ckks_keygen")
    return SecretKey(ctx, sk), PublicKey(ctx, pk)


def zn_pk_export(pk):
    ctx = pk.ctx
    out = np.empty((2, ctx.L, ctx.n), dtype=np.uint64)
    _check(lib().zn_pk_export(pk.handle, out.ctypes.data), "zn_pk_export")
    return out


def zn_pk_import(ctx, arr):
    arr = np.ascontiguousarray(arr, dtype=np.uint64).reshape(2, ctx.L, ctx.n)
    h = ctypes.c_void_p()
    _check(lib().zn_pk_import(ctx.handle, arr.ctypes.data, ctypes.byref(h)), "zn_pk_import")
    return PublicKey(ctx, h)


def zn_sk_export(sk):
    out = np.empty(sk.ctx.n, dtype=np.int8)
    _check(lib().zn_sk_export(sk.handle, out.ctypes.data), "zn_sk_export")
    return out


def zn_sk_import(ctx, arr):
    arr = np.ascontiguousarray(arr, dtype=np.int8).reshape(ctx.n)
    h = ctypes.c_void_p()
    _check(lib().zn_sk_import(ctx.handle, arr.ctypes.data, ctypes.byref(h)), "zn_sk_import")
    return SecretKey(ctx, h)


def _out(out, shape, dtype, device):
    import torch
    if out is None:
        return torch.empty(shape, dtype=dtype, device=device)
    return out


def ckks_encode(ctx, slots, out=None, stream=None):
    """slots: CUDA float64 [B, n_slots] -> int64 [B, N] plaintext coefficients."""
    import torch
    B, ns = slots.shape
    out = _out(out, (B, ctx.n), torch.int64, slots.device)
    _dev(slots, torch.float64, None, "slots")
    _dev(out, torch.int64, (B, ctx.n), "out")
    _check(lib().ckks_encode(ctx.handle, slots.data_ptr(), ns, B, out.data_ptr(), _stream(stream)), "ckks_encode")
    return out


def ckks_encode_ragged(ctx, slots, n_slots, out=None, stream=None):
    """Per-vector slot counts: slots CUDA float64 [B, stride], n_slots CUDA
    int32 [B] (vector b uses its first n_slots[b] entries) -> int64 [B, N]."""
    import torch
    B, stride = slots.shape
    out = _out(out, (B, ctx.n), torch.int64, slots.device)
    _dev(slots, torch.float64, None, "slots")
    _dev(n_slots, torch.int32, (B,), "n_slots")
    _dev(out, torch.int64, (B, ctx.n), "out")
    _check(lib().ckks_encode_ragged(ctx.handle, slots.data_ptr(), n_slots.data_ptr(), stride, B, out.data_ptr(),
                                    _stream(stream)), "ckks_encode_ragged")
    return out


def _enc_ragged(fn, ctx, key, slots, n_slots, seed, ct_index, out, stream, name):
    import torch
    B, stride = slots.shape
    out = _out(out, (B, 2, ctx.L, ctx.n), torch.int64, slots.device)
    _dev(slots, torch.float64, None, "slots")
    _dev(n_slots, torch.int32, (B,), "n_slots")
    _dev(ct_index, torch.int64, (B,), "ct_index")
    _dev(out, torch.int64, (B, 2, ctx.L, ctx.n), "out")
    _check(fn(ctx.handle, key.handle, slots.data_ptr(), n_slots.data_ptr(), stride, B, seed, ct_index.data_ptr(),
              out.data_ptr(), _stream(stream)), name)
    return out


def ckks_encrypt_ragged(ctx, pk, slots, n_slots, seed, ct_index, out=None, stream=None):
    """Vanilla encryption with a slot count per vector (n_slots CUDA int32 [B])."""
    return _enc_ragged(lib().ckks_encrypt_ragged, ctx, pk, slots, n_slots, seed, ct_index, out, stream,
                       "ckks_encrypt_ragged")


def zinc_encrypt_ragged(ctx, zc, slots, n_slots, seed, ct_index, out=None, stream=None):
    """Zinc encryption with a slot count per vector (n_slots CUDA int32 [B])."""
    return _enc_ragged(lib().zinc_encrypt_ragged, ctx, zc, slots, n_slots, seed, ct_index, out, stream,
                       "zinc_encrypt_ragged")


def _enc(fn, ctx, key, slots, seed, ct_index, out, stream, name):
    import torch
    B, ns = slots.shape
    out = _out(out, (B, 2, ctx.L, ctx.n), torch.int64, slots.device)
    _dev(slots, torch.float64, None, "slots")
    _dev(ct_index, torch.int64, (B,), "ct_index")
    _dev(out, torch.int64, (B, 2, ctx.L, ctx.n), "out")
    _check(fn(ctx.handle, key.handle, slots.data_ptr(), ns, B, seed, ct_index.data_ptr(), out.data_ptr(),
              _stream(stream)), name)
    return out


def ckks_encrypt(ctx, pk, slots, seed, ct_index, out=None, stream=None):
    """Vanilla encryption (Eq. 8): CUDA float64 [B, n_slots] -> int64 [B, 2, L, N] (uint64 residues)."""
    return _enc(lib().ckks_encrypt, ctx, pk, slots, seed, ct_index, out, stream, "ckks_encrypt")


def zinc_precompute(ctx, pk, seed):
    h = ctypes.c_void_p()
    _check(lib().zinc_precompute(ctx.handle, pk.handle, seed, ctypes.byref(h)), "zinc_precompute")
    return ZincCache(ctx, h)


def zn_zcache_export(zc):
    ctx = zc.ctx
    out = np.empty((2, ctx.L, ctx.n), dtype=np.uint64)
    _check(lib().zn_zcache_export(zc.handle, out.ctypes.data), "zn_zcache_export")
    return out


def zn_zcache_import(ctx, arr):
    arr = np.ascontiguousarray(arr, dtype=np.uint64).reshape(2, ctx.L, ctx.n)
    h = ctypes.c_void_p()
    _check(lib().zn_zcache_import(ctx.handle, arr.ctypes.data, ctypes.byref(h)), "zn_zcache_import")
    return ZincCache(ctx, h)


def zinc_encrypt(ctx, zc, slots, seed, ct_index, out=None, stream=None):
    """Zinc encryption (Algorithm 1): same shapes as ckks_encrypt."""
    return _enc(lib().zinc_encrypt, ctx, zc, slots, seed, ct_index, out, stream, "zinc_encrypt")


def zinc_encrypt_noalloc(ctx, zc, slots, seed, ct_index, out, stream=None):
    """Zinc encryption that allocates nothing: the caller supplies `out`
    (int64 [B, 2, L, N]); the library's fixed scratch array holds the
    intermediates (see include/zinc.h for the size limit and the rule that
    overlapping calls race)."""
    import torch
    B, ns = slots.shape
    _dev(slots, torch.float64, None, "slots")
    _dev(ct_index, torch.int64, (B,), "ct_index")
    _dev(out, torch.int64, (B, 2, ctx.L, ctx.n), "out")
    _check(lib().zinc_encrypt_noalloc(ctx.handle, zc.handle, slots.data_ptr(), ns, B, seed, ct_index.data_ptr(),
                                      out.data_ptr(), _stream(stream)), "zinc_encrypt_noalloc")
    return out


def data_level(ctx):
    """The data-level context of a key-level one: the same ring and scale, the
    chain without its last (special) prime."""
    if ctx.L < 2:
        raise ZincError(ZN_EINVAL, "data_level")
    return Context(ctx.log_n, ctx.prime_bits[:-1], ctx.log2_delta, ctx.device)


def ckks_encrypt_ms(ctx, pk, slots, seed, ct_index, out=None, stream=None):
    """Modulus-switched vanilla encryption (SEAL's order) under a key-level pk:
    CUDA float64 [B, n_slots] -> int64 [B, 2, L-1, N] at the data level."""
    import torch
    B, ns = slots.shape
    shape = (B, 2, ctx.L - 1, ctx.n)
    out = _out(out, shape, torch.int64, slots.device)
    _dev(slots, torch.float64, None, "slots")
    _dev(ct_index, torch.int64, (B,), "ct_index")
    _dev(out, torch.int64, shape, "out")
    _check(lib().ckks_encrypt_ms(ctx.handle, pk.handle, slots.data_ptr(), ns, B, seed, ct_index.data_ptr(),
                                 out.data_ptr(), _stream(stream)), "ckks_encrypt_ms")
    return out


def zinc_precompute_ms(ctx, pk, seed, data_ctx):
    """Zinc cache made by modulus-switched Enc(0) under the key-level pk; it
    belongs to data_ctx (see data_level) and serves zinc_encrypt there."""
    h = ctypes.c_void_p()
    _check(lib().zinc_precompute_ms(ctx.handle, pk.handle, seed, data_ctx.handle, ctypes.byref(h)),
           "zinc_precompute_ms")
    return ZincCache(data_ctx, h)


# ------------------------------------------- Zinc with NTT-domain errors

def zinc_nbasis_create(ctx, K, seed):
    """Cached error basis (K chi polynomials per component, NTT form) and rotation tables."""
    h = ctypes.c_void_p()
    _check(lib().zinc_nbasis_create(ctx.handle, K, seed, ctypes.byref(h)), "zinc_nbasis_create")
    nb = NttBasis(ctx, h)
    nb.K = K
    return nb


def ckks_encode_ntt(ctx, slots, out=None, stream=None):
    """slots: CUDA float64 [B, n_slots] -> pre-encoded plaintexts int64 [B, L, N] (uint64 residues, NTT form)."""
    import torch
    B, ns = slots.shape
    out = _out(out, (B, ctx.L, ctx.n), torch.int64, slots.device)
    _dev(slots, torch.float64, None, "slots")
    _dev(out, torch.int64, (B, ctx.L, ctx.n), "out")
    _check(lib().ckks_encode_ntt(ctx.handle, slots.data_ptr(), ns, B, out.data_ptr(), _stream(stream)),
           "ckks_encode_ntt")
    return out


def zinc_encrypt_ntt(ctx, zc, nb, m_hat, seed, ct_index, out=None, stream=None):
    """Zinc with NTT-domain errors: m_hat int64 [B, L, N] (from ckks_encode_ntt) -> int64 [B, 2, L, N]."""
    import torch
    B = m_hat.shape[0]
    out = _out(out, (B, 2, ctx.L, ctx.n), torch.int64, m_hat.device)
    _dev(m_hat, torch.int64, (B, ctx.L, ctx.n), "m_hat")
    _dev(ct_index, torch.int64, (B,), "ct_index")
    _dev(out, torch.int64, (B, 2, ctx.L, ctx.n), "out")
    _check(lib().zinc_encrypt_ntt(ctx.handle, zc.handle, nb.handle, m_hat.data_ptr(), B, seed, ct_index.data_ptr(),
                                  out.data_ptr(), _stream(stream)), "zinc_encrypt_ntt")
    return out


# ------------------------------------------------ BFV (Eq. 12), BGV (Eq. 13)

def _int_enc(fn, ctx, key, t, m, seed, ct_index, out, stream, name):
    """m: CUDA int64 [B, N] plaintext coefficients (taken mod t) -> int64 [B, 2, L, N]."""
    import torch
    B = m.shape[0]
    out = _out(out, (B, 2, ctx.L, ctx.n), torch.int64, m.device)
    _dev(m, torch.int64, (B, ctx.n), "m")
    _dev(ct_index, torch.int64, (B,), "ct_index")
    _dev(out, torch.int64, (B, 2, ctx.L, ctx.n), "out")
    args = [ctx.handle, key.handle] + ([t] if t is not None else []) + [m.data_ptr(), B, seed, ct_index.data_ptr(),
                                                                       out.data_ptr(), _stream(stream)]
    _check(fn(*args), name)
    return out


def zn_slot_encoder_create(ctx, t):
    """Slot batching tables for the plaintext modulus t (prime, t = 1 mod 2N)."""
    h = ctypes.c_void_p()
    _check(lib().zn_slot_encoder_create(ctx.handle, t, ctypes.byref(h)), "zn_slot_encoder_create")
    se = SlotEncoder(ctx, h)
    se.t = t
    return se


def zn_slots_encode(se, slots, out=None, stream=None):
    """CUDA int64 [B, N] slot values (taken mod t) -> plaintext coefficients int64 [B, N] in [0, t)."""
    import torch
    ctx = se.ctx
    B = slots.shape[0]
    out = _out(out, (B, ctx.n), torch.int64, slots.device)
    _dev(slots, torch.int64, (B, ctx.n), "slots")
    _dev(out, torch.int64, (B, ctx.n), "out")
    _check(lib().zn_slots_encode(se.handle, slots.data_ptr(), B, out.data_ptr(), _stream(stream)), "zn_slots_encode")
    return out


def zn_slots_decode(se, m, out=None, stream=None):
    import torch
    ctx = se.ctx
    B = m.shape[0]
    out = _out(out, (B, ctx.n), torch.int64, m.device)
    _dev(m, torch.int64, (B, ctx.n), "m")
    _dev(out, torch.int64, (B, ctx.n), "out")
    _check(lib().zn_slots_decode(se.handle, m.data_ptr(), B, out.data_ptr(), _stream(stream)), "zn_slots_decode")
    return out


def bfv_encrypt(ctx, pk, t, m, seed, ct_index, out=None, stream=None):
    """BFV encryption (Eq. 12) under Gen's key."""
    return _int_enc(lib().bfv_encrypt, ctx, pk, t, m, seed, ct_index, out, stream, "bfv_encrypt")


def bfv_zinc_encrypt(ctx, zc, t, m, seed, ct_index, out=None, stream=None):
    """BFV Zinc encryption over the CKKS cache of zinc_precompute."""
    return _int_enc(lib().bfv_zinc_encrypt, ctx, zc, t, m, seed, ct_index, out, stream, "bfv_zinc_encrypt")


def bgv_keygen(ctx, t, seed):
    sk, pk = ctypes.c_void_p(), ctypes.c_void_p()
    _check(lib().bgv_keygen(ctx.handle, t, seed, ctypes.byref(sk), ctypes.byref(pk)), "bgv_keygen")
    return SecretKey(ctx, sk), PublicKey(ctx, pk)


def bgv_zinc_precompute(ctx, pk, seed):
    h = ctypes.c_void_p()
    _check(lib().bgv_zinc_precompute(ctx.handle, pk.handle, seed, ctypes.byref(h)), "bgv_zinc_precompute")
    return ZincCache(ctx, h)


def bgv_encrypt(ctx, pk, m, seed, ct_index, out=None, stream=None):
    """BGV encryption (Eq. 13) under a bgv_keygen key (t recorded in the key)."""
    return _int_enc(lib().bgv_encrypt, ctx, pk, None, m, seed, ct_index, out, stream, "bgv_encrypt")


def bgv_zinc_encrypt(ctx, zc, m, seed, ct_index, out=None, stream=None):
    """BGV Zinc encryption over a bgv_zinc_precompute cache."""
    return _int_enc(lib().bgv_zinc_encrypt, ctx, zc, None, m, seed, ct_index, out, stream, "bgv_zinc_encrypt")


def _int_dec(fn, ctx, sk, t, ct, stream, name):
    import torch
    B = ct.shape[0]
    _dev(ct, torch.int64, (B, 2, ctx.L, ctx.n), "ct")
    out = torch.empty((B, ctx.n), dtype=torch.int64, device=ct.device)
    _check(fn(ctx.handle, sk.handle, t, ct.data_ptr(), B, out.data_ptr(), _stream(stream)), name)
    return out


def bfv_decrypt(ctx, sk, t, ct, stream=None):
    """int64 [B, 2, L, N] -> plaintext coefficients int64 [B, N] in [0, t)."""
    return _int_dec(lib().bfv_decrypt, ctx, sk, t, ct, stream, "bfv_decrypt")


def bgv_decrypt(ctx, sk, t, ct, stream=None):
    return _int_dec(lib().bgv_decrypt, ctx, sk, t, ct, stream, "bgv_decrypt")


def _host_call(name, ctx, key, slots, seed, ct_index, out, out_shape, chunk):
    import torch
    B, ns = slots.shape
    for t, dt, shape, nm in ((slots, torch.float64, None, "slots"), (ct_index, torch.int64, (B,), "ct_index"),
                             (out, torch.int64, out_shape(B), "out")):
        if not isinstance(t, torch.Tensor) or t.is_cuda or t.dtype != dt or not t.is_contiguous():
            raise TypeError(f"{nm}: expected a contiguous CPU tensor of {dt}")
        if shape is not None and tuple(t.shape) != tuple(shape):
            raise ValueError(f"{nm}: expected shape {shape}")
    zinc = isinstance(key, ZincCache)
    _check(getattr(lib(), name)(ctx.handle, None if zinc else key.handle, key.handle if zinc else None,
                                slots.data_ptr(), ns, B, seed, ct_index.data_ptr(), out.data_ptr(), chunk), name)
    return out


def zn_encrypt_host(ctx, key, slots, seed, ct_index, out, chunk=0):
    """Host-to-host encryption (pipelined copies + kernels).  key: PublicKey
    (vanilla) or ZincCache (Zinc); slots: CPU float64 [B, n_slots]; ct_index:
    CPU int64 [B]; out: CPU int64 [B, 2, L, N] (pinned tensors give
    asynchronous copies).  Synchronous."""
    return _host_call("zn_encrypt_host", ctx, key, slots, seed, ct_index, out,
                      lambda B: (B, 2, ctx.L, ctx.n), chunk)


def zn_ct_packed_words(ctx):
    """uint64 words of one packed ciphertext of this context."""
    return int(lib().zn_ct_packed_words(ctx.handle))


def zn_encrypt_host_packed(ctx, key, slots, seed, ct_index, out, chunk=0):
    """zn_encrypt_host with the ciphertexts packed (zn_ct_pack) on the device
    before the copy: out CPU int64 [B, zn_ct_packed_words(ctx)]."""
    return _host_call("zn_encrypt_host_packed", ctx, key, slots, seed, ct_index, out,
                      lambda B: (B, zn_ct_packed_words(ctx)), chunk)


def zn_ct_pack(ctx, ct, out=None, stream=None):
    """Device int64 [B, 2, L, N] -> packed device int64 [B, zn_ct_packed_words(ctx)]."""
    import torch
    B, W = ct.shape[0], zn_ct_packed_words(ctx)
    out = _out(out, (B, W), torch.int64, ct.device)
    _dev(ct, torch.int64, (B, 2, ctx.L, ctx.n), "ct")
    _dev(out, torch.int64, (B, W), "out")
    _check(lib().zn_ct_pack(ctx.handle, ct.data_ptr(), B, out.data_ptr(), _stream(stream)), "zn_ct_pack")
    return out


def zn_ct_unpack(ctx, packed, out=None, stream=None):
    """Packed device int64 [B, zn_ct_packed_words(ctx)] -> device int64 [B, 2, L, N]."""
    import torch
    B, W = packed.shape[0], zn_ct_packed_words(ctx)
    out = _out(out, (B, 2, ctx.L, ctx.n), torch.int64, packed.device)
    _dev(packed, torch.int64, (B, W), "packed")
    _dev(out, torch.int64, (B, 2, ctx.L, ctx.n), "out")
    _check(lib().zn_ct_unpack(ctx.handle, packed.data_ptr(), B, out.data_ptr(), _stream(stream)), "zn_ct_unpack")
    return out


def ckks_decrypt(ctx, sk, ct, out=None, stream=None):
    """Dec (Eq. 10): int64 [B, 2, L, N] -> coefficient residues int64 [B, L, N]."""
    import torch
    B = ct.shape[0]
    out = _out(out, (B, ctx.L, ctx.n), torch.int64, ct.device)
    _dev(ct, torch.int64, (B, 2, ctx.L, ctx.n), "ct")
    _dev(out, torch.int64, (B, ctx.L, ctx.n), "out")
    _check(lib().ckks_decrypt(ctx.handle, sk.handle, ct.data_ptr(), B, out.data_ptr(), _stream(stream)),
           "ckks_decrypt")
    return out


def ckks_decrypt_decode(ctx, sk, ct, n_slots, out=None, stream=None):
    import torch
    B = ct.shape[0]
    out = _out(out, (B, n_slots), torch.float64, ct.device)
    _dev(ct, torch.int64, (B, 2, ctx.L, ctx.n), "ct")
    _dev(out, torch.float64, (B, n_slots), "out")
    _check(lib().ckks_decrypt_decode(ctx.handle, sk.handle, ct.data_ptr(), B, n_slots, out.data_ptr(),
                                     _stream(stream)), "ckks_decrypt_decode")
    return out


def ckks_add(ctx, a, b, out=None, stream=None):
    import torch
    B = a.shape[0]
    out = _out(out, tuple(a.shape), torch.int64, a.device)
    for t, nm in ((a, "a"), (b, "b"), (out, "out")):
        _dev(t, torch.int64, (B, 2, ctx.L, ctx.n), nm)
    _check(lib().ckks_add(ctx.handle, a.data_ptr(), b.data_ptr(), B, out.data_ptr(), _stream(stream)), "ckks_add")
    return out


def zn_ntt_forward(ctx, data, stream=None):
    import torch
    B = data.shape[0]
    _dev(data, torch.int64, (B, ctx.L, ctx.n), "data")
    _check(lib().zn_ntt_forward(ctx.handle, data.data_ptr(), B, _stream(stream)), "zn_ntt_forward")
    return data


def zn_ntt_inverse(ctx, data, stream=None):
    import torch
    B = data.shape[0]
    _dev(data, torch.int64, (B, ctx.L, ctx.n), "data")
    _check(lib().zn_ntt_inverse(ctx.handle, data.data_ptr(), B, _stream(stream)), "zn_ntt_inverse")
    return data


def zn_sample(ctx, kind, seed, domain, poly, prime, ct_index0, count, out=None, device="cuda", stream=None):
    import torch
    out = _out(out, (count, ctx.n), torch.int64, device)
    _dev(out, torch.int64, (count, ctx.n), "out")
    _check(lib().zn_sample(ctx.handle, kind, seed, domain, poly, prime, ct_index0, count, out.data_ptr(),
                           _stream(stream)), "zn_sample")
    return out


def zn_chi_eval(ctx, u, stream=None):
    """chi's table step on device uniforms u (int64 tensor holding uint64 bits) -> int32 tensor."""
    import torch
    _dev(u, torch.int64, None, "u")
    out = torch.empty(u.shape, dtype=torch.int32, device=u.device)
    _check(lib().zn_chi_eval(ctx.handle, u.data_ptr(), u.numel(), out.data_ptr(), _stream(stream)), "zn_chi_eval")
    return out


class _Job(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("zinc", ctypes.c_int), ("pk", ctypes.c_void_p), ("zc", ctypes.c_void_p),
                ("slots", ctypes.c_void_p), ("n_slots", ctypes.c_uint32), ("count", ctypes.c_uint32),
                ("seed", ctypes.c_uint64), ("ct_index", ctypes.c_void_p), ("ct", ctypes.c_void_p)]


class Batch:
    """A planned mixed-ring batch (zn_batch); keeps its jobs' tensors alive."""

    def __init__(self, h, keep, device):
        self._h = h
        self._keep = keep
        self.device = device
        pu, pk = ctypes.c_uint32(), ctypes.c_uint32()
        _check(lib().zn_batch_info(h, ctypes.byref(pu), ctypes.byref(pk)), "zn_batch_info")
        self.prep_units, self.packets = pu.value, pk.value

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            lib().zn_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def zn_batch_create(jobs, device=0):
    """jobs: list of dicts {ctx, zinc (bool), key (PublicKey or ZincCache), slots (CUDA f64 [B, n_slots]),
    seed, ct_index (CUDA int64 [B]), out (CUDA int64 [B, 2, L, N])}."""
    import torch
    arr = (_Job * len(jobs))()
    keep = []
    for k, j in enumerate(jobs):
        ctx, slots, idx, out = j["ctx"], j["slots"], j["ct_index"], j["out"]
        B = slots.shape[0]
        _dev(slots, torch.float64, None, "slots")
        _dev(idx, torch.int64, (B,), "ct_index")
        _dev(out, torch.int64, (B, 2, ctx.L, ctx.n), "out")
        arr[k].ctx = ctx.handle.value
        arr[k].zinc = 1 if j["zinc"] else 0
        arr[k].pk = None if j["zinc"] else j["key"].handle.value
        arr[k].zc = j["key"].handle.value if j["zinc"] else None
        arr[k].slots = slots.data_ptr()
        arr[k].n_slots = slots.shape[1]
        arr[k].count = B
        arr[k].seed = j["seed"]
        arr[k].ct_index = idx.data_ptr()
        arr[k].ct = out.data_ptr()
        keep.append((ctx, j["key"], slots, idx, out))
    h = ctypes.c_void_p()
    _check(lib().zn_batch_create(arr, len(jobs), device, ctypes.byref(h)), "zn_batch_create")
    return Batch(h, keep, device)


def zn_batch_run(batch, stream=None, graph=True):
    _check(lib().zn_batch_run(batch.handle, _stream(stream), 1 if graph else 0), "zn_batch_run")


VARIANTS = 8


def zn_set_variant(ctx, variant):
    _check(lib().zn_set_variant(ctx.handle, variant), "zn_set_variant")


def zn_get_variant(ctx):
    return int(lib().zn_get_variant(ctx.handle))


def zn_autotune(ctx, pk, zc, batch):
    """Time each encryption launch shape on `batch` ciphertexts; keep the fastest.
    Returns (chosen variant, [milliseconds per variant])."""
    ms = (ctypes.c_float * VARIANTS)()
    chosen = ctypes.c_int()
    _check(lib().zn_autotune(ctx.handle, pk.handle, zc.handle, batch, ms, ctypes.byref(chosen)), "zn_autotune")
    return chosen.value, [float(x) for x in ms]


def _device_name(device):
    import torch
    return torch.cuda.get_device_name(device)


def autotune_cached(ctx, pk, zc, batch=512, path=None):
    """The context's launch shape from a JSON cache keyed by device name, ring
    degree and prime chain: set from the cache on a hit, else tuned by
    zn_autotune on `batch` encryptions and stored.  Returns (variant, hit)."""
    import json
    path = path or os.path.join(os.path.expanduser("~"), ".cache", "zinc_gb300_autotune.json")
    key = f"{_device_name(ctx.device)}|{ctx.log_n}|{','.join(str(q) for q in ctx.primes)}"
    try:
        with open(path) as f:
            cache = json.load(f)
    except (OSError, ValueError):
        cache = {}
    v = cache.get(key)
    if isinstance(v, int) and 0 <= v < VARIANTS:
        zn_set_variant(ctx, v)
        return v, True
    v, ms = zn_autotune(ctx, pk, zc, batch)
    cache[key] = v
    d = os.path.dirname(path)
    if d:
        os.makedirs(d, exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)
    return v, False


def zn_probe_butterfly_relaxed(device=0):
    """Register-only butterflies/s of the relaxed butterfly (primes below 2^59)."""
    r = ctypes.c_double()
    _check(lib().zn_probe_butterfly_relaxed(device, ctypes.byref(r)), "zn_probe_butterfly_relaxed")
    return r.value


def zn_probe_wait_timeout(ctx, tries, stream=None):
    """Run the bounded device wait on a barrier nothing arrives on (at most
    `tries` polls): the next zn_sync_status reports ZN_ETIMEOUT."""
    _check(lib().zn_probe_wait_timeout(ctx.handle, int(tries), _stream(stream)), "zn_probe_wait_timeout")


def zn_inject_alloc_failures(count):
    """Make the next `count` per-call scratch allocations fail with ZN_ENOMEM
    (host-side fault injection for tests; 0 clears)."""
    _check(lib().zn_inject_alloc_failures(int(count)), "zn_inject_alloc_failures")


def zn_probe_butterfly(device=0):
    """Register-only butterflies/s of the NTT butterfly on `device` (ALU ceiling)."""
    r = ctypes.c_double()
    _check(lib().zn_probe_butterfly(device, ctypes.byref(r)), "zn_probe_butterfly")
    return r.value


TIME_ENCODE, TIME_ENCRYPT, TIME_ZINC, TIME_MS_SPECIAL, TIME_MS_DATA, TIME_ZINC_NTT = 0, 1, 2, 3, 4, 5


def zn_timing_enable(ctx, on=True):
    _check(lib().zn_timing_enable(ctx.handle, 1 if on else 0), "zn_timing_enable")


def zn_timing_read(ctx, kind):
    """(summed milliseconds, launch count) of the recorded launches of `kind`; clears them."""
    ms = ctypes.c_double()
    n = ctypes.c_uint64()
    _check(lib().zn_timing_read(ctx.handle, kind, ctypes.byref(ms), ctypes.byref(n)), "zn_timing_read")
    return ms.value, n.value


# --------------------------------------------------- host-side (no GPU)

def zn_host_primes(log_n, bits):
    arr = (ctypes.c_uint32 * len(bits))(*bits)
    out = (ctypes.c_uint64 * len(bits))()
    _check(lib().zn_host_primes(log_n, arr, len(bits), out), "zn_host_primes")
    return [int(x) for x in out]


def zn_host_psi(q, log_n):
    return int(lib().zn_host_psi(q, log_n))


def zn_host_encoder_twiddles(log_n):
    n = 1 << log_n
    re = np.empty(n)
    im = np.empty(n)
    _check(lib().zn_host_encoder_twiddles(log_n, re.ctypes.data, im.ctypes.data), "zn_host_encoder_twiddles")
    return re, im


def zn_host_encoder_twiddles_q62(log_n):
    n = 1 << log_n
    c = np.empty(n, dtype=np.int64)
    s = np.empty(n, dtype=np.int64)
    _check(lib().zn_host_encoder_twiddles_q62(log_n, c.ctypes.data, s.ctypes.data), "zn_host_encoder_twiddles_q62")
    return c, s


def zn_host_cdt():
    out = np.empty(38, dtype=np.uint64)
    _check(lib().zn_host_cdt(out.ctypes.data), "zn_host_cdt")
    return [int(x) for x in out]


def as_u64(t):
    """int64 torch tensor (any device) -> numpy uint64 view of the same bits."""
    return t.detach().cpu().numpy().view(np.uint64)
