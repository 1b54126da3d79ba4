/*
 * zinc.h — C ABI of the GB300 (sm_103a) RNS-CKKS encryption library:
 * vanilla CKKS public-key encryption and the Zinc cached-ciphertext
 * encryption of arXiv 2408.07304.
 *
 * Conventions for every entry point
 * ---------------------------------
 *  - Return value: ZN_OK (0) or a negative ZN_E* status; zn_strerror() names it.
 *  - Pointers marked "device" are CUDA device pointers owned by the caller
 *    (e.g. torch tensors' data_ptr()); "host" pointers are ordinary host memory.
 *    The library never frees caller memory.  Handles (zn_ctx, zn_sk, zn_pk,
 *    zn_zcache, zn_nbasis, zn_slot_encoder, zn_batch) are owned by the
 *    library and released by their destroy call; a handle made in a context
 *    may be released before or after that context (it keeps its device).
 *    Release calls consume any CUDA error of their own, so none surfaces at
 *    the caller's next CUDA check.
 *  - Work is enqueued on the caller's cudaStream_t (passed as void*, 0 = the
 *    legacy default stream) and is asynchronous unless stated otherwise.
 *    Errors detected on the device (encode overflow) are latched in a status
 *    word of the context and reported by zn_sync_status().
 *  - Layouts (all residues are uint64 in [0, q_i), NTT form, bit-reversed
 *    evaluation order unless stated):
 *      plaintext coefficients  int64  [B][N]
 *      ciphertext              uint64 [B][2][L][N]   (c0 = message part, c1)
 *      public key / Zinc cache uint64 [2][L][N]
 *    where N = 2^log_n is the ring degree and L the number of RNS primes.
 *  - The paper writes the ciphertext as (c_1, c_2) and the public key as
 *    (pk_1, pk_2); here they are (c0, c1) and (pk0, pk1).
 *  - Sampling is counter based (Philox4x32-10 keyed by the seed, counter =
 *    (block, domain<<24 | poly<<16 | prime, lo32 ct_index, hi32 ct_index)),
 *    so a ciphertext depends only on (key, seed, ct_index, message), never on
 *    its batch position or the launch shape.
 */
#ifndef ZINC_H
#define ZINC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ZN_MAX_PRIMES 16

enum {
  ZN_OK = 0,
  ZN_EINVAL = -1,     /* invalid argument or parameter set */
  ZN_ENOMEM = -2,     /* device allocation failed or HBM budget exceeded */
  ZN_EOVERFLOW = -3,  /* an encoded coefficient reached |m_k| >= 2^62 (or was not finite) */
  ZN_ECUDA = -4,      /* a CUDA runtime call failed */
  ZN_ETIMEOUT = -5,   /* a bounded device wait gave up */
  ZN_ENOPRIME = -6,   /* no prime q < 2^b with q = 1 mod 2N is left for a chain entry */
  ZN_ELIMIT = -7      /* request larger than the fixed scratch of zinc_encrypt_noalloc */
};

typedef struct zn_ctx zn_ctx;
typedef struct zn_sk zn_sk;
typedef struct zn_pk zn_pk;
typedef struct zn_zcache zn_zcache;
typedef struct zn_nbasis zn_nbasis;
typedef struct zn_slot_encoder zn_slot_encoder;

/* Parameter set.  log_n in [4, 15]; n_primes in [1, ZN_MAX_PRIMES];
 * prime_bits[i] in [20, 61]; log2_delta in [1, 62].  The error distribution
 * chi is fixed by the paper (Section "Polynomials and Distributions"):
 * discrete Gaussian with sigma = 3.2, read as the rounded normal truncated to
 * [-19, 19]. */
typedef struct {
  uint32_t log_n;
  uint32_t n_primes;
  uint32_t prime_bits[ZN_MAX_PRIMES];
  uint32_t log2_delta;
} zn_params;

/* ---------------------------------------------------------------- context */

/* Build the prime chain (for each entry b: the largest unused prime q < 2^b,
 * q = 1 mod 2N), the minimal primitive 2N-th roots psi_i, the NTT twiddle and
 * Shoup tables and the encoder twiddles, and upload them to `device`
 * (synchronous).  The paper takes the modulus from SEAL (Section "System
 * Implementation"); the chain rule is this library's reading. */
int zn_ctx_create(const zn_params* params, int device, zn_ctx** out);
void zn_ctx_destroy(zn_ctx* ctx);

/* Copy the chain to host arrays of n_primes entries (either may be NULL). */
int zn_ctx_primes(const zn_ctx* ctx, uint64_t* primes, uint64_t* psis);

/* Read and clear the device status word after synchronising `stream`;
 * returns ZN_OK, ZN_EOVERFLOW, ZN_ETIMEOUT, ZN_EINVAL (zn_ct_unpack met a
 * residue not below its prime) or ZN_ECUDA. */
int zn_sync_status(zn_ctx* ctx, void* stream);

const char* zn_strerror(int status);

/* ------------------------------------------------------------------ Gen */

/* Gen, paper Eq. 7: sk = s <- R_2, a <- R_q, e <- chi;
 * pk0 = -a*s + e, pk1 = a (NTT form).  Sampling domain 2, ct_index 0.
 * Synchronous. */
int ckks_keygen(zn_ctx* ctx, uint64_t seed, zn_sk** sk, zn_pk** pk);
void zn_sk_destroy(zn_sk* sk);
void zn_pk_destroy(zn_pk* pk);

/* Export / import (checkpointing).  pk: host uint64 [2][L][N] NTT form.
 * sk: host int8 [N] ternary coefficients.  Imports rebuild the NTT and Shoup
 * forms on the device (synchronous). */
int zn_pk_export(const zn_pk* pk, uint64_t* host_out);
int zn_pk_import(zn_ctx* ctx, const uint64_t* host_in, zn_pk** out);
int zn_sk_export(const zn_sk* sk, int8_t* host_out);
int zn_sk_import(zn_ctx* ctx, const int8_t* host_in, zn_sk** out);

/* --------------------------------------------------------------- encode */

/* CKKS encoding (canonical embedding; the paper assumes a pre-encoded message,
 * Section "Construction").  slots: device double [batch][n_slots] (real
 * slots; slots n_slots..N/2-1 are zero); out: device int64 [batch][N],
 * m_k ~ 2^(log2_delta+1-log_n) * Re sum_j z_j zeta^(-5^j k), computed by a
 * block-scaled fixed-point FFT on 64-bit integers: each vector is scaled by
 * 2^F, F = 60 - log_n - e with 2^(e-1) <= max|z_j| < 2^e (so zero padding
 * changes nothing); Q62
 * twiddles; every complex product exact in 128 bits and rounded once
 * (floor(x + 1/2)); bit-reproducible, with an error below
 * 2^(s-F-1) (3.4 N/2 + 2) + 1/2 per coefficient (s = log2_delta + 1 - log_n).
 * n_slots <= N/2.  Overflow (|m_k| >= 2^62, or a non-finite slot) is latched
 * for zn_sync_status and the vector's coefficients are set to zero. */
int ckks_encode(zn_ctx* ctx, const double* slots, uint32_t n_slots, uint32_t batch,
                int64_t* out, void* stream);

/* The same encoding with a slot count per vector (the boundary's per-vector
 * n_slots array): vector b has n_slots[b] slots (device uint32 [batch]), read
 * from row b of `slots` (device double [batch][stride]; stride <= N/2, 0
 * allowed when every count is 0); its missing slots are zero, so the result
 * equals ckks_encode of that row zero-padded.  A count above stride latches
 * ZN_EINVAL for zn_sync_status and encodes that vector as zero. */
int ckks_encode_ragged(zn_ctx* ctx, const double* slots, const uint32_t* n_slots, uint32_t stride,
                       uint32_t batch, int64_t* out, void* stream);

/* -------------------------------------------------------------- encrypt */

/* Vanilla public-key encryption, paper Eq. 8 (second component with pk1):
 * u <- R_2, e0, e1 <- chi (domain 0, keyed by seed and ct_index[b]);
 * c0 = pk0*u + e0 + m, c1 = pk1*u + e1 (mod each q_i), NTT form.
 * slots: device double [batch][n_slots]; ct_index: device uint64 [batch];
 * ct: device uint64 [batch][2][L][N].  May grow the context's encode scratch
 * (a cudaMalloc) when batch exceeds what earlier calls used. */
int ckks_encrypt(zn_ctx* ctx, const zn_pk* pk, const double* slots, uint32_t n_slots,
                 uint32_t batch, uint64_t seed, const uint64_t* ct_index, uint64_t* ct,
                 void* stream);

/* ckks_encrypt with a slot count per vector, as ckks_encode_ragged: n_slots
 * device uint32 [batch], slots device double [batch][stride].  Vector b's
 * ciphertext equals ckks_encrypt's for its row zero-padded to any length
 * (padding is exact); a count above stride latches ZN_EINVAL for
 * zn_sync_status and encrypts the zero plaintext. */
int ckks_encrypt_ragged(zn_ctx* ctx, const zn_pk* pk, const double* slots, const uint32_t* n_slots,
                        uint32_t stride, uint32_t batch, uint64_t seed, const uint64_t* ct_index,
                        uint64_t* ct, void* stream);

/* Zinc precomputation (Section "Precomputation"): cache one Enc(0) — a vanilla
 * encryption of the zero plaintext under pk with sampling domain 3,
 * ct_index 0.  Synchronous. */
int zinc_precompute(zn_ctx* ctx, const zn_pk* pk, uint64_t seed, zn_zcache** out);
void zn_zcache_destroy(zn_zcache* zc);
/* Cache export / import: host uint64 [2][L][N] NTT form. */
int zn_zcache_export(const zn_zcache* zc, uint64_t* host_out);
int zn_zcache_import(zn_ctx* ctx, const uint64_t* host_in, zn_zcache** out);

/* Zinc encryption, paper Algorithm 1 / Eq. 9: c = zero + m; e1', e2' <- chi
 * (domain 1, keyed by seed and ct_index[b]); c' = (c0 + e1', c1 + e2').
 * Arguments as ckks_encrypt, with the cache in place of the public key. */
int zinc_encrypt(zn_ctx* ctx, const zn_zcache* zc, const double* slots, uint32_t n_slots,
                 uint32_t batch, uint64_t seed, const uint64_t* ct_index, uint64_t* ct,
                 void* stream);

/* zinc_encrypt with a slot count per vector (Algorithm 1; arguments as
 * ckks_encrypt_ragged with the cache in place of the public key). */
int zinc_encrypt_ragged(zn_ctx* ctx, const zn_zcache* zc, const double* slots, const uint32_t* n_slots,
                        uint32_t stride, uint32_t batch, uint64_t seed, const uint64_t* ct_index,
                        uint64_t* ct, void* stream);

/* Allocation-free Zinc encryption (no counterpart in the paper).  For callers
 * that must not allocate device memory during a call: code running where
 * the allocator is off limits or too slow (a real-time loop with a fixed
 * memory footprint, an embedding host that owns every allocation, a process
 * whose device memory is already fully reserved).  Same arguments and
 * results as zinc_encrypt, but the per-call scratch (encoded message plus
 * noise and the small polynomials) lives in one static 16 MiB device array
 * of the library instead of the context's memory pool, and nothing is
 * allocated or freed by the call.
 *  - Limit: batch * 10 N bytes (8 N + 2 N, each part rounded up to 256 bytes)
 *    must fit in ZN_NOALLOC_SCRATCH_BYTES; larger requests return ZN_ELIMIT
 *    without launching anything (split them into smaller calls).
 *  - The first call on a device looks up the array's device address (once
 *    per device and process); make that first call before any stream
 *    capture.  The address is kept for the life of the process, so calls
 *    after a reset of the device (cudaDeviceReset) are not supported.
 *  - Every call on a device shares the one array: calls whose work overlaps
 *    on the GPU (different streams, or host threads) race and corrupt each
 *    other's results; serialise them.  The array keeps the last call's
 *    contents; nothing in it needs to start at zero (every byte a call reads
 *    is first written by the same call). */
#define ZN_NOALLOC_SCRATCH_BYTES (16u << 20)
int zinc_encrypt_noalloc(zn_ctx* ctx, const zn_zcache* zc, const double* slots, uint32_t n_slots,
                         uint32_t batch, uint64_t seed, const uint64_t* ct_index, uint64_t* ct,
                         void* stream);

/* ------------------------- special prime and modulus switching (SEAL order)
 *
 * The paper's measurements ran SEAL (Section "System Implementation"), whose
 * public-key encryption works at the key level -- the data primes plus one
 * special prime p -- and then divides by p and rounds (modulus switching)
 * before the message is added; Section "Theoretical Analysis" counts the
 * resulting transforms.  Here a key-level context holds the whole chain
 * q_0..q_{L-1} (L >= 2) and its LAST prime is the special prime p; the data
 * level is q_0..q_{L-2}, and a context created from the same parameters
 * without the last bit size holds exactly those primes (the chain rule works
 * left to right).
 *
 * Modulus-switched vanilla encryption: u <- R_2, e0, e1 <- chi (domain 0,
 * exactly the samples of ckks_encrypt with the same seed and ct_index);
 * c_j = pk_j*u + e_j over the key level, then per coefficient
 * c'_j = floor((c_j + floor(p/2)) / p) mod (q_0 ... q_{L-2}) -- computed per
 * data prime as (c_{j,i} + h - r_j) p^-1 mod q_i, r_j = (c_{j,p} + h) mod p --
 * and finally c'_0 += m.  pk: a key of ctx (the key level); slots and
 * ct_index as ckks_encrypt; ct: device uint64 [batch][2][L-1][N], NTT form,
 * at the data level.  Decryption with the same secret key at the data level
 * (import it into the data-level context) leaves m + v/p + rounding noise
 * below (N + 1)/2 + 1 in magnitude per coefficient.  ZN_EINVAL if L < 2.
 * Scratch comes from the context's pool. */
int ckks_encrypt_ms(zn_ctx* ctx, const zn_pk* pk, const double* slots, uint32_t n_slots, uint32_t batch,
                    uint64_t seed, const uint64_t* ct_index, uint64_t* ct, void* stream);

/* Zinc precomputation over a modulus-switched Enc(0): the cached zero is
 * ckks_encrypt_ms of the zero plaintext (domain 3, ct_index 0) under pk of
 * the key-level ctx, and the cache belongs to data_ctx -- a context on the
 * same device with the same log_n and log2_delta whose primes are ctx's first
 * L-1 (ZN_EINVAL otherwise).  zinc_encrypt(data_ctx, cache, ...) then runs
 * Algorithm 1 at the data level.  Synchronous. */
int zinc_precompute_ms(zn_ctx* ctx, const zn_pk* pk, uint64_t seed, zn_ctx* data_ctx, zn_zcache** out);

/* ------------------------------------------- BFV and BGV (Section "Scheme Flexibility")
 *
 * The paper notes that Zinc carries over to BFV (Eq. 12) and BGV (Eq. 13).
 * Plaintexts are polynomials of R_t = Z_t[X]/(X^N + 1) given by their N
 * coefficients: device int64 [batch][N], each taken mod t (coefficient
 * encoding; the paper leaves encoding to the schemes' own papers).  Q is the
 * product of the context's primes; the second component uses pk1 (as read
 * in Eq. 8).  t must satisfy 2 <= t <= 2^58 and t < q_i for every prime;
 * ring degrees 2^10 .. 2^15.  Sampling tags are the CKKS ones (vanilla:
 * domain 0, u / e0 / e1 = polys 0 / 1 / 2; Zinc: domain 1, e1' / e2' =
 * polys 0 / 1; caches: domain 3, ct_index 0).  Ciphertexts: device uint64
 * [batch][2][L][N], NTT form.  Decryption is exact while the noise is below
 * Delta/2 (BFV) or Q/(2t) (BGV).  ZN_EINVAL for an invalid t or ring.
 *
 * BFV, Eq. 12: Delta = floor(Q/t); c0 = pk0*u + e0 + Delta*m, c1 = pk1*u + e1
 * under Gen's key (ckks_keygen).  Its Zinc form adds Delta*m + e1' and e2' to
 * the cache of zinc_precompute (CKKS's Enc(0), unchanged, as the paper says). */
int bfv_encrypt(zn_ctx* ctx, const zn_pk* pk, uint64_t t, const int64_t* m, uint32_t batch, uint64_t seed,
                const uint64_t* ct_index, uint64_t* ct, void* stream);
int bfv_zinc_encrypt(zn_ctx* ctx, const zn_zcache* zc, uint64_t t, const int64_t* m, uint32_t batch,
                     uint64_t seed, const uint64_t* ct_index, uint64_t* ct, void* stream);
/* m = round(t [c0 + c1 s]_Q / Q) mod t, out: device int64 [batch][N] in [0, t). */
int bfv_decrypt(zn_ctx* ctx, const zn_sk* sk, uint64_t t, const uint64_t* ct, uint32_t batch, int64_t* m,
                void* stream);

/* Slot batching for BFV / BGV plaintexts (the paper leaves plaintext
 * encoding to the schemes' papers; this is the usual one).  For a prime
 * t = 1 mod 2N, R_t is isomorphic to Z_t^N by evaluation at the odd powers of
 * psi_t, the minimal primitive 2N-th root of unity mod t: slot s < N/2 holds
 * m(psi_t^(5^s mod 2N)) and slot N/2 + s holds m(psi_t^(-5^s mod 2N)) (the
 * CKKS encoder's slot order), so slot-wise sums and products of vectors are
 * sums and products in R_t.  zn_slot_encoder_create: t prime, t = 1 mod 2N,
 * and valid for ctx as above (ZN_EINVAL otherwise); synchronous.
 * zn_slots_encode: slots device int64 [batch][N] (each taken mod t) -> m
 * device int64 [batch][N] in [0, t), the plaintext for bfv_* / bgv_*.
 * zn_slots_decode: the inverse (input taken mod t).  Stream-ordered; not
 * tuned (one block per vector, radix-2 stages in global memory). */
int zn_slot_encoder_create(zn_ctx* ctx, uint64_t t, zn_slot_encoder** out);
void zn_slot_encoder_destroy(zn_slot_encoder* se);
int zn_slots_encode(zn_slot_encoder* se, const int64_t* slots, uint32_t batch, int64_t* m, void* stream);
int zn_slots_decode(zn_slot_encoder* se, const int64_t* m, uint32_t batch, int64_t* slots, void* stream);

/* BGV, Eq. 13: the errors carry the factor t.  bgv_keygen: Gen's samples with
 * pk0 = -a*s + t*e (the key records t; zn_pk_import and zn_zcache_import
 * rebuild Gen-type handles, not BGV ones).  bgv_encrypt:
 * c0 = pk0*u + t*e0 + m, c1 = pk1*u + t*e1.  bgv_zinc_precompute caches a BGV
 * encryption of zero; bgv_zinc_encrypt adds m + t*e1' and t*e2' to it.
 * Synchronous: keygen, precompute. */
int bgv_keygen(zn_ctx* ctx, uint64_t t, uint64_t seed, zn_sk** sk, zn_pk** pk);
int bgv_zinc_precompute(zn_ctx* ctx, const zn_pk* pk, uint64_t seed, zn_zcache** out);
int bgv_encrypt(zn_ctx* ctx, const zn_pk* pk, const int64_t* m, uint32_t batch, uint64_t seed,
                const uint64_t* ct_index, uint64_t* ct, void* stream);
int bgv_zinc_encrypt(zn_ctx* ctx, const zn_zcache* zc, const int64_t* m, uint32_t batch, uint64_t seed,
                     const uint64_t* ct_index, uint64_t* ct, void* stream);
/* m = ([c0 + c1 s]_Q centred) mod t, out: device int64 [batch][N] in [0, t). */
int bgv_decrypt(zn_ctx* ctx, const zn_sk* sk, uint64_t t, const uint64_t* ct, uint32_t batch, int64_t* m,
                void* stream);

/* ------------------------------- Zinc with NTT-domain errors (O(N) encryption)
 *
 * The paper's Conclusion names a further optimisation: generating the random
 * error polynomials directly in the Fourier (NTT) space, which removes Zinc's
 * two transforms per prime.  The paper gives no construction; this library's
 * reading, a change of the error distribution with no security claim:
 *   - a basis of K cached chi polynomials per component, E_{c,j} (domain 4,
 *     poly 16c + j, ct_index 0, the basis seed), kept in NTT form;
 *   - per ciphertext, rotations r_{c,j} uniform in [0, 2N) (Philox block j of
 *     domain 5, poly c, the ciphertext's seed and ct_index, word 0);
 *   - e'_c = sum_j X^{r_{c,j}} E_{c,j} (X^N = -1): each coefficient is a sum
 *     of K chi values (variance K sigma^2, |e'| <= 19 K);
 *   - over a plaintext already encoded in NTT form (the paper's Construction
 *     assumes an encoded m): c' = (z0 + m + e'_0, z1 + e'_1).
 * In NTT form X^r multiplies output i by psi^((2 brv(i) + 1) r mod 2N), so
 * the encryption is pointwise: per prime and coefficient 2K table lookups
 * and 4K Shoup products.  Ring degrees 2^10..2^15.
 *
 * zinc_nbasis_create: K in [1, 16]; synchronous.  ckks_encode_ntt: the CKKS
 * encoding (as ckks_encode) reduced mod each q_i and transformed: out device
 * uint64 [batch][L][N].  zinc_encrypt_ntt: zc from zinc_precompute; m_hat
 * device uint64 [batch][L][N] (from ckks_encode_ntt); ct as zinc_encrypt. */
int zinc_nbasis_create(zn_ctx* ctx, uint32_t K, uint64_t seed, zn_nbasis** out);
void zn_nbasis_destroy(zn_nbasis* nb);
int ckks_encode_ntt(zn_ctx* ctx, const double* slots, uint32_t n_slots, uint32_t batch, uint64_t* out,
                    void* stream);
int zinc_encrypt_ntt(zn_ctx* ctx, const zn_zcache* zc, const zn_nbasis* nb, const uint64_t* m_hat,
                     uint32_t batch, uint64_t seed, const uint64_t* ct_index, uint64_t* ct, void* stream);

/* Host memory in, host memory out: copies slot vectors and ct indices to the
 * device, encrypts -- vanilla (Eq. 8) under pk when zc is NULL, Zinc
 * (Algorithm 1) under zc otherwise (pass exactly one) -- and copies the
 * ciphertexts back, in chunks of `chunk` ciphertexts pipelined over three
 * internal streams so that the transfers of one chunk overlap the kernels of
 * the next (0: at most 256 ciphertexts and 512 MiB per chunk, and at most a
 * quarter of the batch but not below 8).  host_slots [batch][n_slots] double, host_ct_index
 * [batch] uint64, host_ct [batch][2][L][N] uint64: page-locked host memory
 * gives asynchronous full-speed copies (pageable memory works, slower).
 * Results equal ckks_encrypt / zinc_encrypt.  Synchronous: returns when the
 * ciphertexts are in host_ct.  Device staging comes from the context's pool. */
int zn_encrypt_host(zn_ctx* ctx, const zn_pk* pk, const zn_zcache* zc, const double* host_slots,
                    uint32_t n_slots, uint32_t batch, uint64_t seed, const uint64_t* host_ct_index,
                    uint64_t* host_ct, uint32_t chunk);

/* ------------------------------------------- packed ciphertext serialization
 * No counterpart in the paper (a wire format for the ciphertexts that
 * Eq. 8 / Algorithm 1 produce).  Each residue mod q_i takes bits_i = bit
 * length of q_i bits instead of a 64-bit word.  Per ciphertext: component 0,
 * then 1; within a component prime 0..L-1; a limb is its N residues as one
 * little-endian bit stream (residue j in bits [j bits_i, (j+1) bits_i),
 * ceil(N bits_i / 64) uint64 words, unused high bits of the last word zero).
 * The 60 + 6x50 + 60-bit chain packs to 420/512 of the plain size.
 *
 * zn_ct_packed_words: uint64 words of one packed ciphertext (0 for NULL).
 * zn_ct_pack: device ct [batch][2][L][N] (residues below their primes) ->
 *   device packed [batch][packed_words].  Stream-ordered.
 * zn_ct_unpack: the inverse; a residue not below its prime is written as read
 *   and latched (zn_sync_status then returns ZN_EINVAL).  Stream-ordered.
 * zn_encrypt_host_packed: zn_encrypt_host with the output packed on the device
 *   before the copy: host_packed [batch][packed_words]; equals zn_ct_pack of
 *   zn_encrypt_host's ciphertexts.  Synchronous. */
size_t zn_ct_packed_words(const zn_ctx* ctx);
int zn_ct_pack(zn_ctx* ctx, const uint64_t* ct, size_t batch, uint64_t* packed, void* stream);
int zn_ct_unpack(zn_ctx* ctx, const uint64_t* packed, size_t batch, uint64_t* ct, void* stream);
int zn_encrypt_host_packed(zn_ctx* ctx, const zn_pk* pk, const zn_zcache* zc, const double* host_slots,
                           uint32_t n_slots, uint32_t batch, uint64_t seed, const uint64_t* host_ct_index,
                           uint64_t* host_packed, uint32_t chunk);

/* -------------------------------------------------------------- decrypt */

/* Dec, paper Eq. 10: c0 + c1*s (mod each q_i), returned in the coefficient
 * domain.  ct: device uint64 [batch][2][L][N]; out: device uint64 [batch][L][N]. */
int ckks_decrypt(zn_ctx* ctx, const zn_sk* sk, const uint64_t* ct, uint32_t batch,
                 uint64_t* out, void* stream);

/* Dec followed by decoding: CRT over the first two primes (one if L = 1),
 * centred, then z_j = Delta^-1 m(zeta^(5^j)).  out: device double
 * [batch][n_slots] (real parts).  Verification path; not tuned. */
int ckks_decrypt_decode(zn_ctx* ctx, const zn_sk* sk, const uint64_t* ct, uint32_t batch,
                        uint32_t n_slots, double* out, void* stream);

/* Homomorphic addition (paper Eq. 2): out = a + b (mod each q_i); each
 * device uint64 [batch][2][L][N]; out may alias a or b. */
int ckks_add(zn_ctx* ctx, const uint64_t* a, const uint64_t* b, uint32_t batch,
             uint64_t* out, void* stream);

/* ------------------------------------------- building blocks (for tests) */

/* Forward / inverse negacyclic NTT per prime, in place, on device uint64
 * [batch][L][N] residues in [0, q_i):
 *   ahat[i] = sum_j a_j psi^((2 brv(i) + 1) j) mod q  (RNS "DFT",
 *   Section "Theoretical Analysis"). */
int zn_ntt_forward(zn_ctx* ctx, uint64_t* data, uint32_t batch, void* stream);
int zn_ntt_inverse(zn_ctx* ctx, uint64_t* data, uint32_t batch, void* stream);

/* Sampler (Section "Polynomials and Distributions"): kind 0 = R_2 (ternary),
 * 1 = chi, 2 = R_q residues for `prime`.  out: device int64 [count][N] for
 * polynomial (domain, poly, prime) and ct_index = ct_index0 + c. */
int zn_sample(zn_ctx* ctx, int kind, uint64_t seed, uint32_t domain, uint32_t poly,
              uint32_t prime, uint64_t ct_index0, uint32_t count, int64_t* out, void* stream);

/* chi's table step alone (no counterpart in the paper; a check of threshold
 * boundaries): out[i] = -19 + #{j : u[i] >= T_j} for device uint64 u[n],
 * device int32 out[n], computed by the lookup the encryption path uses (a
 * 256-bucket index over the top 8 bits of u, then a scan of the thresholds
 * inside the bucket). */
int zn_chi_eval(zn_ctx* ctx, const uint64_t* u, uint32_t n, int32_t* out, void* stream);

/* ------------------------------------------------ mixed-ring batched launch */

/* One job of a batch: `count` encryptions under one parameter set and mode.
 * All pointers are device pointers owned by the caller and must stay valid
 * (and keep their addresses) for the life of the batch; their contents may
 * change between runs. */
typedef struct {
  zn_ctx* ctx;                /* parameter set (ring degree 2^10 .. 2^15)       */
  int zinc;                   /* 0: vanilla (Eq. 8) under pk; 1: Zinc (Alg. 1)  */
  const zn_pk* pk;            /* vanilla key (zinc = 0)                          */
  const zn_zcache* zc;        /* cached Enc(0) (zinc = 1)                        */
  const double* slots;        /* [count][n_slots]                                */
  uint32_t n_slots;           /* <= N/2                                          */
  uint32_t count;
  uint64_t seed;
  const uint64_t* ct_index;   /* [count]                                         */
  uint64_t* ct;               /* [count][2][L][N]                                */
} zn_job;

typedef struct zn_batch zn_batch;

/* Plan a batch over jobs of mixed ring degree, chain and mode (all contexts
 * on `device`): builds the work lists (one prep unit per ciphertext; encrypt
 * packets, largest rings first: for N <= 2^13 the 2^(13 - log_n) limbs that
 * fill a 256-thread block, for N = 2^14 and 2^15 one limb, run by a cluster
 * of two or four 256-thread blocks) and allocates the scratch for every
 * ciphertext.  Synchronous. */
int zn_batch_create(const zn_job* jobs, uint32_t n_jobs, int device, zn_batch** out);
void zn_batch_destroy(zn_batch* b);

/* Enqueue the batch on `stream`: persistent launches -- prep (512-thread
 * blocks, 1024-thread ones when the largest ring is 2^15), encryption of the
 * rings up to 2^13 (three 256-thread blocks per SM), of the 2^14 rings
 * (two-CTA clusters) and of the 2^15 rings (four-CTA clusters) -- whose
 * blocks take work from device counters.  graph != 0:
 * the first call captures the launches into a CUDA graph on `stream` and
 * every call replays it (one graph launch per run).  Results are identical to
 * ckks_encrypt / zinc_encrypt of each job. */
int zn_batch_run(zn_batch* b, void* stream, int graph);

/* Number of prep units and encrypt packets in the plan (either may be NULL). */
int zn_batch_info(const zn_batch* b, uint32_t* prep_units, uint32_t* packets);

/* -------------------------------------------------------------- autotuning */

/* Launch shapes of the encryption kernels: variant = 2 * kind + order.
 * order 0 = prime-major grid (the blocks of one ciphertext run together and
 * share its prepared integers in L2), 1 = ciphertext-major grid (the blocks
 * of a wave share one prime's twiddles and keys).  kind 0 = one block per
 * limb that transforms the polynomials one after another; kind 1 = one block
 * per limb (per output half for N = 2^14) holding all of the limb's
 * polynomials at once, sharing each twiddle load between them and writing
 * each ciphertext word once (2^10 <= N <= 2^14 with 16-byte aligned key and
 * output pointers); kind 2 = kind 0 capped at 128 registers per thread so
 * that several blocks share an SM, N = 2^14 split into output halves
 * (2^10 <= N <= 2^14); kind 3 = kind 2 with radix-8 passes capped at 80
 * registers (three blocks of 256 threads per SM); at N = 2^14 one cluster
 * of two such blocks per limb, each owning an output half, the first two
 * butterfly stages split between them and exchanged through distributed
 * shared memory, and at N = 2^15 one cluster of four, each owning an output
 * quarter, the first three stages exchanged.  Where a kind does not apply, kind 0 runs.  A new context starts
 * at variant 6 for 2^10 <= N <= 2^15 and at variant 0 otherwise. */
#define ZN_VARIANTS 8
int zn_set_variant(zn_ctx* ctx, int variant);
int zn_get_variant(const zn_ctx* ctx);

/* Time every variant on `batch` vanilla and Zinc encryptions of the zero
 * message under pk / zc (device scratch allocated and freed inside;
 * synchronous), keep the fastest in the context, and report per-variant
 * milliseconds in ms[ZN_VARIANTS] and the choice in *chosen (either may be
 * NULL).  Results of the encryptions do not depend on the variant. */
int zn_autotune(zn_ctx* ctx, const zn_pk* pk, const zn_zcache* zc, uint32_t batch, float* ms, int* chosen);

/* ---------------------------------------------------- launch timing (bench) */

/* Kernel kinds that can be timed. */
enum {
  ZN_TIME_ENCODE = 0,      /* prep (encode + sampling), every encryption form  */
  ZN_TIME_ENCRYPT = 1,     /* vanilla encryption kernel                        */
  ZN_TIME_ZINC = 2,        /* Zinc encryption kernel                           */
  ZN_TIME_MS_SPECIAL = 3,  /* modulus-switched vanilla: special-prime kernels  */
  ZN_TIME_MS_DATA = 4,     /* modulus-switched vanilla: data-prime kernel      */
  ZN_TIME_ZINC_NTT = 5,    /* Zinc with NTT-domain errors                      */
  ZN_TIME_KINDS = 6
};

/* on != 0: every later kernel launch of the kinds above in this context is
 * bracketed by CUDA events recorded on its launch stream.
 * Recording stays on until switched off; on = 0 also discards pending
 * records. */
int zn_timing_enable(zn_ctx* ctx, int on);

/* Synchronise the recorded events of `kind`, return their summed duration
 * (milliseconds) and launch count, and clear them. */
int zn_timing_read(zn_ctx* ctx, int kind, double* ms, uint64_t* launches);

/* Diagnostic (no counterpart in the paper): butterflies per second that the
 * NTT's Harvey/Shoup butterfly reaches on `device` when it runs from
 * registers alone (no memory traffic) -- the practical ALU ceiling of every
 * transform in this library.  Synchronous; ~30 ms. */
int zn_probe_butterfly(int device, double* butterflies_per_s);
/* The same for the relaxed butterfly (no correction step; the transforms use
 * it for primes below 2^59), with one fold back to [0, 4q) every 12 stages as
 * a transform's final reduction would do. */
int zn_probe_butterfly_relaxed(int device, double* butterflies_per_s);

/* Diagnostic (no counterpart in the paper): the device-side timeout path of
 * the bounded waits (the packed-serialization tiles wait on an mbarrier for
 * their bulk copy).  One block waits, with the same code, on a barrier that
 * nothing arrives on, polling at most `tries` times (1 <= tries <= 2^20; the
 * tiles use 2^20), then latches the timeout bit of ctx's status word and
 * returns: the next zn_sync_status(ctx, stream) reports ZN_ETIMEOUT and the
 * context stays usable.  Asynchronous on `stream`; ZN_EINVAL for a null ctx
 * or tries out of range. */
int zn_probe_wait_timeout(zn_ctx* ctx, uint32_t tries, void* stream);

/* Host-side fault injection for tests of the callers' error paths (no
 * counterpart in the paper): the next `count` per-call scratch allocations,
 * in any context and on any thread, fail as if the device memory pool were
 * exhausted, so the calls that make them return ZN_ENOMEM before launching
 * anything and leave their context usable.  Touches no device state and
 * injects nothing on the GPU.  count = 0 clears a pending injection;
 * count < 0 returns ZN_EINVAL. */
int zn_inject_alloc_failures(int count);

/* ------------------------------------------------ host-side tables (no GPU) */

/* The host computations behind zn_ctx_create, exposed so that they can be
 * checked without a GPU. */
int zn_host_primes(uint32_t log_n, const uint32_t* bits, uint32_t n_primes, uint64_t* out);
uint64_t zn_host_psi(uint64_t q, uint32_t log_n);
/* T[k] = cos(pi k/N) - i sin(pi k/N), k < N, each part correctly rounded
 * (the decoder's FP64 twiddles). */
int zn_host_encoder_twiddles(uint32_t log_n, double* re, double* im);
/* The encoder's Q62 twiddles: c[k] = floor(2^62 cos(pi k/N) + 1/2),
 * s[k] = floor(2^62 sin(pi k/N) + 1/2), k < N (host int64 arrays of N). */
int zn_host_encoder_twiddles_q62(uint32_t log_n, int64_t* c, int64_t* s);
/* The 38 chi thresholds T_j = floor(2^64 F(j - 20)), j = 1..38. */
int zn_host_cdt(uint64_t* out);

#ifdef __cplusplus
}
#endif
#endif /* ZINC_H */
