// Launchers of the sm_103a kernels (zn_kernels.cu); used by the C ABI layer.
#pragma once
#include "zn_device.cuh"

namespace zn {

// Per-ciphertext inputs prepared once for all primes by the prep kernel.
struct PrepArgs {
  const double* slots;  // [B][n_slots], or [B][stride] with per-vector counts
  uint32_t n_slots;     // 0: zero plaintext
  const u64* ct_index;  // [B] or nullptr (then ct_index0 + b)
  u64 ct_index0;
  u64 seed;
  unsigned domain;      // sampling domain (0 vanilla, 1 Zinc, 3 Zinc cache)
  i64* me;              // [B][N] encoded message plus its noise polynomial
  int8_t* small;        // [B][2][N] small polynomials (vanilla: u, e1; Zinc: e2')
  // Per-vector slot counts (device [B], each <= stride <= N/2; rows of
  // `stride` doubles) in place of n_slots; nullptr: n_slots for every vector.
  // A count above `stride` latches kStatusRange and encodes zero.
  const uint32_t* n_slots_v = nullptr;
  uint32_t stride = 0;
};

struct EncArgs {
  int swap;             // grid order: 0 = (prime, ciphertext), 1 = (ciphertext, prime)
  const u64* key;       // vanilla: pk [2][L][N]; Zinc: cache [2][L][N]
  const u64* keys;      // vanilla: pk Shoup companions [2][L][N]; Zinc: unused
  const i64* me;        // [B][N] from the prep kernel
  const int8_t* small;  // [B][2][N] from the prep kernel
  u64* out;             // [B][2][L][N]
};

cudaError_t launch_encode(const DevParams& P, const double* slots, uint32_t n_slots, uint32_t batch, i64* out,
                          cudaStream_t st);
// Per-vector slot counts nv (device [batch]) over rows of `stride` doubles.
cudaError_t launch_encode_ragged(const DevParams& P, const double* slots, const uint32_t* nv, uint32_t stride,
                                 uint32_t batch, i64* out, cudaStream_t st);
cudaError_t launch_prep(const DevParams& P, const PrepArgs& A, bool zinc, uint32_t batch, cudaStream_t st);
// Mixed-ring batches (persistent kernels): one descriptor per job (a ring,
// a mode, a key or cache, buffers), a work list of encrypt packets and one of
// prep units.
struct JobDesc {
  DevParams P;
  EncArgs E;      // me / small point into this job's scratch
  PrepArgs Pr;    // idem
  int zinc;
  int pad;
};
struct EncPacket {
  uint32_t job;
  uint32_t b0;      // first ciphertext of the packet (within the job)
  uint16_t prime;
  uint8_t count;    // ciphertexts in the packet (units sharing one block)
  uint8_t half;     // N = 2^14: which output half
};
struct PrepUnit {
  uint32_t job;
  uint32_t b;
};
cudaError_t batch_set_attributes();
cudaError_t batch_encrypt_attributes();
cudaError_t launch_batch_prep(const JobDesc* jobs, const PrepUnit* units, int n_units, int* counter, int grid,
                              size_t smem, cudaStream_t st);
cudaError_t batch_prep_blocks_per_sm(size_t smem, int* blocks);
// Rings up to 2^14 (three 256-thread blocks per SM).
cudaError_t launch_batch_encrypt(const JobDesc* jobs, const EncPacket* packets, int n_packets, int* counter, int sms,
                                 cudaStream_t st);
// 2^15 rings: persistent four-CTA clusters, one limb per packet.
cudaError_t batch_quarter_attributes();
cudaError_t batch_quarter_clusters(int* clusters);
cudaError_t launch_batch_encrypt_quarter(const JobDesc* jobs, const EncPacket* packets, int n_packets, int* counter,
                                         int clusters, cudaStream_t st);

// N = 2^14 on two-CTA clusters, one output half per CTA (kind 3 at 2^14).
cudaError_t launch_encrypt_pair(const DevParams& P, const EncArgs& A, bool zinc, uint32_t batch, cudaStream_t st);
// 2^14 rings: persistent two-CTA clusters, one limb per packet.
cudaError_t batch_pair_attributes();
cudaError_t batch_pair_clusters(int* clusters);
cudaError_t launch_batch_encrypt_pair(const JobDesc* jobs, const EncPacket* packets, int n_packets, int* counter,
                                      int clusters, cudaStream_t st);
// variant = 2 * kind + order.  order 0 = prime-major grid, 1 =
// ciphertext-major grid (all blocks of a wave share one prime's twiddles and
// keys); kind 0 = per-polynomial kernel, 1 = multi-polynomial kernel, 2 and
// 3 = register-capped per-polynomial kernels with two or three resident
// blocks per SM (kinds 1-3 where they apply).
// Selected by the autotuner.
cudaError_t launch_encrypt(const DevParams& P, const EncArgs& A, bool zinc, uint32_t batch, int variant,
                           cudaStream_t st);
// Multi-polynomial kernel (2^10 <= N <= 2^14; key, companion and output
// pointers 16-byte aligned; grid order from A.swap).
cudaError_t launch_encrypt_mp(const DevParams& P, const EncArgs& A, bool zinc, uint32_t batch, cudaStream_t st);
// Register-capped per-polynomial kernels (kind 2: 2^10 <= N <= 2^14; kind 3:
// 2^10 <= N <= 2^13).
cudaError_t launch_encrypt_occ(const DevParams& P, const EncArgs& A, bool zinc, uint32_t batch, cudaStream_t st);
cudaError_t launch_encrypt_occ3(const DevParams& P, const EncArgs& A, bool zinc, uint32_t batch, cudaStream_t st);
// N = 2^15: one four-CTA cluster per limb, one output quarter per CTA, the
// first three stages exchanged through distributed shared memory.
cudaError_t launch_encrypt_quarter(const DevParams& P, const EncArgs& A, bool zinc, uint32_t batch,
                                   cudaStream_t st);
cudaError_t launch_keygen(const DevParams& P, u64 seed, u64* sk_ntt, u64* pk, u64* pks, cudaStream_t st);
cudaError_t launch_ntt_fwd(const DevParams& P, u64* data, uint32_t batch, u64* tmp, cudaStream_t st);
cudaError_t launch_ntt_inv(const DevParams& P, u64* data, uint32_t batch, cudaStream_t st);
cudaError_t launch_dec_mul(const DevParams& P, const u64* ct, const u64* sk, uint32_t batch, u64* out,
                           cudaStream_t st);
cudaError_t launch_decode(const DevParams& P, const u64* coeffs, uint32_t batch, uint32_t n_slots, double* out,
                          double* work, cudaStream_t st);
cudaError_t launch_add(const DevParams& P, const u64* a, const u64* b, uint32_t batch, u64* out, cudaStream_t st);
cudaError_t launch_sample(const DevParams& P, int kind, u64 seed, unsigned domain, unsigned poly, unsigned prime,
                          u64 ct_index0, uint32_t count, i64* out, cudaStream_t st);
cudaError_t launch_chi_eval(const DevParams& P, const u64* u, uint32_t n, int* out, cudaStream_t st);
cudaError_t launch_shoup(const DevParams& P, const u64* w, u64* ws, uint32_t polys, cudaStream_t st);
// Butterflies per second of k_probe_butterfly (register-only ceiling),
// corrected (Harvey) or relaxed form.
cudaError_t probe_butterfly(int sms, double* per_s, bool relaxed);
cudaError_t launch_sk_residues(const DevParams& P, const int8_t* s, u64* out, cudaStream_t st);

// ------------------------------------------------ modulus-switched encryption
// The key-level chain q_0..q_{L-1} of P ends in the special prime p = q_{L-1};
// the ciphertext has the L-1 data primes.  Per ciphertext:
//   prep (prep_ms):   M = m + 2^62 [N], small = [u, e0, e1] int8 [3][N]
//   special (p):      D_j = d_j + 2^62, d_j = e_j + h - ((pk_j u + e_j)_p + h) mod p,
//                     h = floor(p/2)
//   data primes q_i:  c'_0 = (pk0 p^-1) u^ + NTT(d_0 p^-1 + m),
//                     c'_1 = (pk1 p^-1) u^ + NTT(d_1 p^-1)
// The 2^62 offsets make M and D_j unsigned, so that a data prime reduces
// them with one Shoup product (D_j p^-1) or one Barrett step (M) and removes
// the offsets with the constants kc0, kc1.
struct MsArgs {
  int swap;             // grid order of the data-prime kernel, as EncArgs
  const u64* keyms;     // [2][L-1][N] pk_j p^-1 mod q_i (NTT form), then Shoup companions [2][L-1][N]
  const u64* keyn;      // [2][N] pk_{j,p} N^-1 mod p (NTT form), then Shoup companions [2][N]
  const u64* m;         // [B][N] encoded message + 2^62
  const int8_t* small;  // [B][3][N] u, e0, e1
  u64* d;               // [B][2][N] d_0 + 2^62, d_1 + 2^62
  u64* tmp;             // [B][2][N] inverse-transform halves (N = 2^15 only)
  u64* out;             // [B][2][L-1][N]
  u64 pinv[kMaxL];      // p^-1 mod q_i
  u64 pinvs[kMaxL];     // Shoup companions
  u64 kc1[kMaxL];       // -2^62 p^-1 mod q_i
  u64 kc0[kMaxL];       // -2^62 (p^-1 + 1) mod q_i
};
constexpr u64 kMsOffset = 1ull << 62;
cudaError_t launch_prep_ms(const DevParams& P, const PrepArgs& A, uint32_t batch, cudaStream_t st);
// keyms / keyn (and companions) of MsArgs from a key-level public key [2][L][N].
cudaError_t launch_ms_keys(const DevParams& P, const MsArgs& A, const u64* pk, u64* keyms, u64* keyn,
                           cudaStream_t st);
cudaError_t launch_ms_special(const DevParams& P, const MsArgs& A, uint32_t batch, cudaStream_t st);
cudaError_t launch_ms_data(const DevParams& P, const MsArgs& A, uint32_t batch, cudaStream_t st);

// ------------------------------------------- BFV (Eq. 12) and BGV (Eq. 13)
// Coefficient plaintexts m in Z_t (int64, taken mod t).  The prep kernel
// draws the randomness once per ciphertext (same tags as the CKKS path) and
// writes me = m mod t (BFV) or m mod t + t e_a (BGV), e_a = e0 (vanilla) or
// e1' (Zinc), with small = [u, e0, e1] (vanilla) or [e1', e2'] (Zinc).
struct IntPrepArgs {
  const i64* m;         // [B][N] plaintext coefficients, or nullptr (zero plaintext)
  u64 t;
  u64 seed;
  unsigned domain;
  const u64* ct_index;  // [B] or nullptr (then ct_index0 + b)
  u64 ct_index0;
  i64* me;              // [B][N]
  int8_t* small;        // [B][3][N] vanilla, [B][2][N] Zinc
};
struct IntArgs {
  int swap;             // grid order, as EncArgs
  const u64* key;       // vanilla: pk [2][L][N]; Zinc: cache [2][L][N]
  const u64* keys;      // vanilla: Shoup companions [2][L][N]
  const i64* me;        // [B][N] from the prep kernel
  const int8_t* small;  // [B][3 or 2][N] from the prep kernel
  u64* out;             // [B][2][L][N]
  u64 f[kMaxL];         // BFV: Delta mod q_i (Delta = floor(Q/t)); BGV: t mod q_i
  u64 fs[kMaxL];        // Shoup companions
};
// Decryption constants for the chain q_0..q_{L-1} (Q their product):
//   y_i = (Q/q_i)^-1 mod q_i;  BFV: t y_i = I_i q_i + r_i, It_i = I_i mod t;
//   BGV: Qi_t = (Q/q_i) mod t, Q_t = Q mod t.
struct IntDec {
  u64 t;
  u64 y[kMaxL];
  u64 It[kMaxL];
  u64 r[kMaxL];
  u64 Qit[kMaxL];
  u64 Qt;
};
cudaError_t launch_prep_int(const DevParams& P, const IntPrepArgs& A, bool bgv, bool zinc, uint32_t batch,
                            cudaStream_t st);
cudaError_t launch_encrypt_int(const DevParams& P, const IntArgs& A, bool bgv, bool zinc, uint32_t batch,
                               cudaStream_t st);
// x: [B][L][N] coefficient residues of c0 + c1 s (Dec, Eq. 10) -> m [B][N] in [0, t).
cudaError_t launch_int_decode(const DevParams& P, const IntDec& D, bool bgv, const u64* x, uint32_t batch, i64* m,
                              cudaStream_t st);
// ------------------------------------- Zinc with NTT-domain errors (O(N))
// e'_c = sum_{j<K} X^{r_{c,j}} E_{c,j}: in NTT form the rotation X^r is the
// pointwise factor psi^(a r mod 2N) at output i, a = 2 brv(i) + 1.  With
// i = t + 256 k (t < 256), a = 2^(n-7) brv_8(t) + 2 brv_(n-8)(k) + 1, so the
// factor splits into flo[t] * fhi[k]; a block builds both tables per
// rotation (with Shoup companions) from psi^(64 h) and psi^l 2^64 (one
// Montgomery product each) and multiplies by Shoup products.
struct NttZincArgs {
  const u64* z;           // cached zero [2][L][N]
  const u64* E;           // basis [2][K][L][N], NTT form
  const u64* thi;         // [L][N/32] psi^(64 h) mod q
  const u64* tlo;         // [L][64]   psi^l 2^64 mod q (Montgomery form)
  const u64* m;           // [B][L][N] pre-encoded plaintexts, NTT form
  const u64* ct_index;    // [B]
  u64 seed;
  u64* out;               // [B][2][L][N]
  int K;
  u64 qneg[kMaxL];        // -q_i^-1 mod 2^64 (Montgomery)
};
cudaError_t launch_zinc_ntt(const DevParams& P, const NttZincArgs& A, uint32_t batch, cudaStream_t st);
// int64 coefficients [B][N] -> residues [B][L][N]
cudaError_t launch_residues_batch(const DevParams& P, const i64* v, uint32_t batch, u64* out, cudaStream_t st);

// Slot batching for BFV / BGV plaintexts (a prime t = 1 mod 2N).
struct BatchEnc {
  int log_n;
  u64 t;
  u64 ninv, ninvs;          // N^-1 mod t and its Shoup companion
  const ulonglong2* twp;    // [N] (psi^brv(k), Shoup companion) mod t
  const u64* itw;           // [N] psi^-brv(k) mod t
  const u64* itws;          // [N] Shoup companions
  const int* pos;           // [N] NTT output index of slot s
};
cudaError_t launch_batch_encode(const BatchEnc& E, const i64* slots, uint32_t batch, i64* m, cudaStream_t st);
cudaError_t launch_batch_decode(const BatchEnc& E, const i64* m, uint32_t batch, u64* work, i64* slots,
                                cudaStream_t st);

// Packed ciphertext serialization (zn_pack.cu): bits[i] = bit length of q_i,
// woff[i] = word offset of prime i's limb within a component, cwords = words
// of one component.
struct PackArgs {
  u64* ct;                  // [B][2][L][N] plain residues
  u64* packed;              // [B][2][cwords]
  unsigned bits[kMaxL];
  u64 woff[kMaxL];
  u64 cwords;
};
cudaError_t launch_ct_pack(const DevParams& P, const PackArgs& A, uint32_t batch, cudaStream_t st);
cudaError_t launch_ct_unpack(const DevParams& P, const PackArgs& A, uint32_t batch, cudaStream_t st);
// One block waits on a barrier nothing arrives on, with the tiles' bounded
// wait limited to `tries` polls: latches kStatusTimeout.
cudaError_t launch_wait_probe(const DevParams& P, unsigned tries, cudaStream_t st);

// pk0 += (t - 1) e-hat (per prime, NTT form) and its Shoup companions: Gen's key becomes BGV's.
cudaError_t launch_bgv_key(const DevParams& P, u64 t, const u64* ehat, u64* pk, u64* pks, cudaStream_t st);
// residues [L][N] of a signed int64 polynomial [N]
cudaError_t launch_residues(const DevParams& P, const i64* v, u64* out, cudaStream_t st);

}  // namespace zn
