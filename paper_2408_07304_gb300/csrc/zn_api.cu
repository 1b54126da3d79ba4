// C ABI of the library (include/zinc.h): contexts, key/cache handles,
// argument checking, scratch management and kernel launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <cstdlib>
#include <atomic>
#include <cstring>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/zinc.h"
#include "zn_host.h"
#include "zn_kernels.h"

using zn::DevParams;
using zn::i64;
using zn::u64;

struct zn_ctx {
  int device;
  zn_params prm;
  uint32_t n, L;
  u64 q[ZN_MAX_PRIMES], psi[ZN_MAX_PRIMES];
  DevParams dp;
  // device allocations owned by the context
  u64* d_tw;          // (tw, tws) pairs [L][N], itw [L][N], itws [L][N]: one allocation
  double* d_etw;      // [2][N] decoder twiddles, then [N] encoder Q62 pairs
  int* d_slot;        // [N]: slot_of_t, then pos_of_slot
  unsigned* d_status;
  u64 pinv[ZN_MAX_PRIMES], pinvs[ZN_MAX_PRIMES];   // p^-1 mod q_i (p the last prime), Shoup companions
  cudaMemPool_t pool; // stream-ordered scratch (prep outputs)
  int variant;        // encryption launch shape (zn_autotune)
  cudaStream_t hs[3]; // internal streams of zn_encrypt_host (created on first use)
  cudaStream_t hp;    // high-priority stream of its packing kernels, and their events
  cudaEvent_t hev[6]; // [slot]: chunk encrypted; [3 + slot]: chunk packed
  // launch timing (benchmark instrumentation)
  bool timing;
  std::vector<cudaEvent_t> ev[ZN_TIME_KINDS];   // start/stop pairs
};

// Handle type tags: an opaque pointer of the wrong kind is rejected (ZN_EINVAL).
enum : uint32_t {
  kTagPk = 0x6b70u, kTagSk = 0x6b73u, kTagZc = 0x637au, kTagNb = 0x626eu, kTagSe = 0x7365u, kTagDead = 0u
};

// Slot batching tables for a plaintext modulus t (BFV / BGV).
struct zn_slot_encoder {
  uint32_t tag = kTagSe;
  zn_ctx* ctx;
  int device = 0;          // the context's device, kept for release after the context
  zn::BatchEnc E;
  void* d;                 // one allocation: twp [N], itw [N], itws [N], pos [N]
};

// Cached error basis of the NTT-domain Zinc randomiser, and the rotation tables.
struct zn_nbasis {
  uint32_t tag = kTagNb;
  zn_ctx* ctx;
  int device = 0;          // the context's device, kept for release after the context
  uint32_t K;
  u64* E;                  // [2][K][L][N] NTT form
  u64* thi;                // [L][N/32] psi^(64 h) mod q
  u64* tlo;                // [L][64]   psi^l 2^64 mod q (Montgomery form)
};

struct zn_pk {
  uint32_t tag = kTagPk;
  zn_ctx* ctx;
  int device = 0;          // the context's device, kept for release after the context
  u64* d;    // [2][L][N] then Shoup companions [2][L][N]
  // L >= 2: the modulus-switched encryption's key forms -- pk_j p^-1 mod q_i
  // [2][L-1][N] + companions, then pk_{j,p} N^-1 mod p [2][N] + companions
  u64* ms = nullptr;
  uint64_t t = 0;   // 0: Gen's key (CKKS, BFV); t >= 2: BGV key (error scaled by t)
};
struct zn_sk {
  uint32_t tag = kTagSk;
  zn_ctx* ctx;
  int device = 0;          // the context's device, kept for release after the context
  u64* d;                    // [L][N] NTT form
  std::vector<int8_t> s;     // coefficients
};
struct zn_zcache {
  uint32_t tag = kTagZc;
  zn_ctx* ctx;
  int device = 0;          // the context's device, kept for release after the context
  u64* d;    // [2][L][N]
  uint64_t t = 0;   // 0: a CKKS / BFV encryption of zero; t >= 2: a BGV one
};

// pk_of / zc_of: Gen's key and caches made with it (CKKS, BFV);
// bgv_pk_of / bgv_zc_of: BGV keys and caches (error scaled by t >= 2).
static inline bool pk_of(const zn_pk* k, const zn_ctx* c) { return k && k->tag == kTagPk && k->ctx == c && !k->t; }
static inline bool bgv_pk_of(const zn_pk* k, const zn_ctx* c) { return k && k->tag == kTagPk && k->ctx == c && k->t; }
static inline bool sk_of(const zn_sk* k, const zn_ctx* c) { return k && k->tag == kTagSk && k->ctx == c; }
static inline bool zc_of(const zn_zcache* z, const zn_ctx* c) { return z && z->tag == kTagZc && z->ctx == c && !z->t; }
static inline bool bgv_zc_of(const zn_zcache* z, const zn_ctx* c) {
  return z && z->tag == kTagZc && z->ctx == c && z->t;
}

namespace {

inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// NVTX range around an entry point: names the call in Nsight timelines (a
// no-op unless a profiling tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

inline size_t limb(const zn_ctx* c) { return (size_t)c->n; }
inline size_t ring_words(const zn_ctx* c) { return (size_t)c->L * c->n; }

// A release call's failure is not the caller's error: consume it, so that the
// runtime's last-error state does not report it at the caller's next check.
inline void released(cudaError_t e) {
  if (e != cudaSuccess) cudaGetLastError();
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      cudaGetLastError();
      prev = -1;
    }
    if (prev != dev) released(cudaSetDevice(dev));
  }
  ~DeviceGuard() {
    if (prev >= 0) released(cudaSetDevice(prev));
  }
};

#define ZN_CUDA(call)                      \
  do {                                     \
    if ((call) != cudaSuccess) {           \
      cudaGetLastError();                  \
      return ZN_ECUDA;                     \
    }                                      \
  } while (0)

// Host-side fault injection (zn_inject_alloc_failures): the number of
// scratch allocations still to fail.
std::atomic<int> g_alloc_faults{0};

bool take_alloc_fault() {
  int n = g_alloc_faults.load(std::memory_order_relaxed);
  while (n > 0)
    if (g_alloc_faults.compare_exchange_weak(n, n - 1, std::memory_order_relaxed)) return true;
  return false;
}

// Stream-ordered scratch from the context's memory pool: concurrent calls on
// different streams never share scratch, and the allocations are legal
// inside a CUDA-graph capture.
struct Scratch {
  zn_ctx* c;
  cudaStream_t st;
  void* p = nullptr;
  Scratch(zn_ctx* c_, cudaStream_t st_) : c(c_), st(st_) {}
  bool alloc(size_t bytes) {
    if (take_alloc_fault()) {
      p = nullptr;
      return false;
    }
    if (cudaMallocFromPoolAsync(&p, bytes, c->pool, st) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return false;
    }
    return true;
  }
  ~Scratch() {
    if (p) cudaFreeAsync(p, st);
  }
};

// Event pair around one launch (no-op unless timing is on).
struct TimedLaunch {
  zn_ctx* c;
  int kind;
  cudaStream_t st;
  TimedLaunch(zn_ctx* c_, int kind_, cudaStream_t st_) : c(c_), kind(kind_), st(st_) { mark(); }
  ~TimedLaunch() { mark(); }
  void mark() {
    if (!c->timing) return;
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    cudaEventRecord(e, st);
    c->ev[kind].push_back(e);
  }
};

// Messages encoded per launch pair: the int64 scratch is kept within
// 512 MiB (4096 ciphertexts at N = 2^14).  Large launches amortise each
// launch's partial last wave (the prep grid of 256 ciphertexts filled 0.84 of
// a wave); the kernels are bound by integer arithmetic, so scratch that no
// longer stays in L2 costs nothing measurable (measured at N = 2^14: 256, 512,
// 1024, 2048 ciphertexts per launch -> 234.5k, 238.7k, 244.4k, 246.2k enc/s
// with the half kernels; 2048 -> 4096 with the pair kernels 260.9k -> 262.7k).
uint32_t encode_chunk(const zn_ctx* c) {
  size_t per = sizeof(i64) * c->n;
  size_t k = (512ull << 20) / per;
  if (k < 1) k = 1;
  if (k > 65535) k = 65535;
  return (uint32_t)k;
}

// Prep + encrypt launch pairs over `batch` ciphertexts in chunks of `chunk`,
// with caller-provided scratch for one chunk: me int64 [chunk][N], small
// int8 [chunk][2][N].
// nv != nullptr: per-vector slot counts (device [batch]) over rows of `stride`
// doubles, in place of n_slots.
int encrypt_with(zn_ctx* c, bool zinc, const u64* key, const u64* keys, const double* slots, uint32_t n_slots,
                 uint32_t batch, uint64_t seed, const uint64_t* ct_index, uint64_t* ct, i64* me, int8_t* small,
                 uint32_t chunk, cudaStream_t st, const uint32_t* nv = nullptr, uint32_t stride = 0) {
  const size_t row = nv ? stride : n_slots;
  for (uint32_t b0 = 0; b0 < batch; b0 += chunk) {
    const uint32_t nb = (batch - b0) < chunk ? (batch - b0) : chunk;
    zn::PrepArgs pa;
    pa.slots = slots ? slots + (size_t)b0 * row : nullptr;
    pa.n_slots = n_slots;
    pa.n_slots_v = nv ? nv + b0 : nullptr;
    pa.stride = stride;
    pa.ct_index = ct_index + b0;
    pa.ct_index0 = 0;
    pa.seed = seed;
    pa.domain = zinc ? 1u : 0u;
    pa.me = me;
    pa.small = small;
    {
      TimedLaunch t(c, ZN_TIME_ENCODE, st);
      ZN_CUDA(zn::launch_prep(c->dp, pa, zinc, nb, st));
    }
    zn::EncArgs A;
    A.swap = 0;
    A.key = key;
    A.keys = keys;
    A.me = me;
    A.small = small;
    A.out = ct + (size_t)b0 * 2 * ring_words(c);
    TimedLaunch t(c, zinc ? ZN_TIME_ZINC : ZN_TIME_ENCRYPT, st);
    ZN_CUDA(zn::launch_encrypt(c->dp, A, zinc, nb, c->variant, st));
  }
  return ZN_OK;
}

// Bytes of encrypt_with's scratch for chunks of `chunk` ciphertexts: the
// message-plus-noise words, then the small polynomials.
size_t encrypt_scratch_bytes(const zn_ctx* c, uint32_t chunk) {
  return sizeof(i64) * chunk * (size_t)c->n + 2 * (size_t)chunk * c->n;
}

int encrypt_common(zn_ctx* c, bool zinc, const u64* key, const u64* keys, const double* slots, uint32_t n_slots,
                   uint32_t batch, uint64_t seed, const uint64_t* ct_index, uint64_t* ct, void* stream,
                   const uint32_t* nv = nullptr, uint32_t stride = 0) {
  if (!c || !key || n_slots > c->n / 2 || stride > c->n / 2) return ZN_EINVAL;
  if (batch == 0) return ZN_OK;
  if (!ct || !ct_index || (n_slots && !slots) || (nv && stride && !slots)) return ZN_EINVAL;
  DeviceGuard g(c->device);
  // equal chunks of at most encode_chunk(c), so that no launch is a small tail
  const uint32_t cap = encode_chunk(c);
  const uint32_t chunks = (batch + cap - 1) / cap;
  const uint32_t first = (batch + chunks - 1) / chunks;
  Scratch scratch(c, S(stream));
  if (!scratch.alloc(encrypt_scratch_bytes(c, first))) return ZN_ENOMEM;
  i64* me = (i64*)scratch.p;
  int8_t* small = (int8_t*)scratch.p + sizeof(i64) * first * (size_t)c->n;
  return encrypt_with(c, zinc, key, keys, slots, n_slots, batch, seed, ct_index, ct, me, small, first, S(stream), nv,
                      stride);
}

// The modulus-switched encryption's arguments that depend only on the context.
zn::MsArgs ms_args(const zn_ctx* c, const zn_pk* pk) {
  zn::MsArgs A;
  std::memset(&A, 0, sizeof(A));
  A.keyms = pk->ms;
  A.keyn = pk->ms + 4 * (size_t)(c->L - 1) * c->n;
  for (uint32_t i = 0; i + 1 < c->L; ++i) {
    const u64 q = c->q[i];
    A.pinv[i] = c->pinv[i];
    A.pinvs[i] = c->pinvs[i];
    const u64 off = zn::powmod(2, 62, q);                                  // 2^62 mod q
    const u64 op = (u64)(((unsigned __int128)off * c->pinv[i]) % q);       // 2^62 p^-1 mod q
    A.kc1[i] = (q - op) % q;
    A.kc0[i] = (q - (op + off) % q) % q;
  }
  return A;
}

// Key forms of the modulus-switched encryption for a key-level public key
// (L >= 2; nothing to do for L = 1).  Synchronous.
int ms_key_forms(zn_ctx* c, zn_pk* k) {
  if (c->L < 2) return ZN_OK;
  const size_t words = 4 * (size_t)c->L * c->n;
  if (cudaMalloc(&k->ms, sizeof(u64) * words) != cudaSuccess) {
    cudaGetLastError();
    k->ms = nullptr;
    return ZN_ENOMEM;
  }
  const zn::MsArgs A = ms_args(c, k);
  if (zn::launch_ms_keys(c->dp, A, k->d, k->ms, const_cast<u64*>(A.keyn), 0) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    return ZN_ECUDA;
  }
  return ZN_OK;
}

// Ciphertexts per prep/special/data launch triple of the modulus-switched
// encryption: its scratch -- m (8N), d_0, d_1 (16N), small (3N) and, at
// N = 2^15, the inverse-transform halves (16N) -- within ZN_MS_SCRATCH_MIB,
// the batch split into equal chunks so that no launch is a small tail wave.
// The data kernel re-reads the scratch once per prime; DRAM has ample
// headroom, and measured at N = 2^14 (4096 ciphertexts) larger chunks win:
// 133 k/s at 32 MiB, 165 k/s at 128 MiB, 171 k/s at 512 MiB; with the pair
// kernels 512 -> 1024 MiB (two launches of 2048) 193.5 k -> 196.9 k.
#ifndef ZN_MS_SCRATCH_MIB
#define ZN_MS_SCRATCH_MIB 1024
#endif
uint32_t ms_chunk(const zn_ctx* c, uint32_t batch) {
  const size_t per = (size_t)c->n * (27 + (c->prm.log_n == 15 ? 16 : 0));
  size_t k = ((size_t)ZN_MS_SCRATCH_MIB << 20) / per;
  if (k < 1) k = 1;
  if (k > 65535) k = 65535;
  const size_t chunks = (batch + k - 1) / k;
  return (uint32_t)((batch + chunks - 1) / chunks);
}

// ct_index == nullptr: ciphertext b takes index b.
int ms_common(zn_ctx* c, const zn_pk* pk, const double* slots, uint32_t n_slots, uint32_t batch, uint64_t seed,
              unsigned domain, const uint64_t* ct_index, uint64_t* ct, cudaStream_t st) {
  const uint32_t chunk = ms_chunk(c, batch);
  const uint32_t first = batch < chunk ? batch : chunk;
  const size_t n = c->n;
  const size_t m_b = sizeof(i64) * first * n, d_b = 2 * m_b;
  const size_t t_b = c->prm.log_n == 15 ? 2 * sizeof(u64) * first * n : 0, s_b = 3 * (size_t)first * n;
  Scratch scratch(c, st);
  if (!scratch.alloc(m_b + d_b + t_b + s_b)) return ZN_ENOMEM;
  unsigned char* base = (unsigned char*)scratch.p;
  zn::MsArgs A = ms_args(c, pk);
  A.swap = 0;
  A.m = (const u64*)base;
  A.d = (u64*)(base + m_b);
  A.tmp = t_b ? (u64*)(base + m_b + d_b) : nullptr;
  A.small = (const int8_t*)(base + m_b + d_b + t_b);
  const size_t ct_words = 2 * (size_t)(c->L - 1) * n;
  for (uint32_t b0 = 0; b0 < batch; b0 += chunk) {
    const uint32_t nb = (batch - b0) < chunk ? (batch - b0) : chunk;
    zn::PrepArgs pa;
    pa.slots = n_slots ? slots + (size_t)b0 * n_slots : nullptr;
    pa.n_slots = n_slots;
    pa.ct_index = ct_index ? ct_index + b0 : nullptr;
    pa.ct_index0 = b0;
    pa.seed = seed;
    pa.domain = domain;
    pa.me = (i64*)A.m;
    pa.small = (int8_t*)A.small;
    A.out = ct + (size_t)b0 * ct_words;
    {
      TimedLaunch t(c, ZN_TIME_ENCODE, st);
      ZN_CUDA(zn::launch_prep_ms(c->dp, pa, nb, st));
    }
    {
      TimedLaunch t(c, ZN_TIME_MS_SPECIAL, st);
      ZN_CUDA(zn::launch_ms_special(c->dp, A, nb, st));
    }
    TimedLaunch t(c, ZN_TIME_MS_DATA, st);
    ZN_CUDA(zn::launch_ms_data(c->dp, A, nb, st));
  }
  return ZN_OK;
}

// ------------------------------------------------ BFV / BGV host constants
// t is valid for a context when 2 <= t <= 2^58 (BGV's m + t e stays an
// int64) and t < q_i for every prime (t is then invertible mod each q_i).
bool t_ok(const zn_ctx* c, uint64_t t) {
  if (t < 2 || t > (1ull << 58)) return false;
  for (uint32_t i = 0; i < c->L; ++i)
    if (t >= c->q[i]) return false;
  return true;
}

inline u64 mulmod_h(u64 a, u64 b, u64 m) { return (u64)(((unsigned __int128)a * b) % m); }

// Encryption constants: BFV Delta mod q_i with Delta = floor(Q/t) -- from
// Q = Delta t + (Q mod t) and Q = 0 mod q_i, Delta = -(Q mod t) t^-1 mod q_i
// -- or BGV t mod q_i; with Shoup companions.
void int_enc_consts(const zn_ctx* c, uint64_t t, bool bgv, zn::IntArgs& A) {
  u64 Qt = 1 % t;
  for (uint32_t j = 0; j < c->L; ++j) Qt = mulmod_h(Qt, c->q[j] % t, t);
  for (uint32_t i = 0; i < c->L; ++i) {
    const u64 q = c->q[i];
    u64 f;
    if (bgv) {
      f = t % q;
    } else {
      const u64 tinv = zn::powmod(t % q, q - 2, q);
      f = (q - mulmod_h(Qt % q, tinv, q)) % q;
    }
    A.f[i] = f;
    A.fs[i] = zn::shoup(f, q);
  }
}

// Decryption constants (see zn::IntDec).
void int_dec_consts(const zn_ctx* c, uint64_t t, zn::IntDec& D) {
  std::memset(&D, 0, sizeof(D));
  D.t = t;
  u64 Qt = 1 % t;
  for (uint32_t j = 0; j < c->L; ++j) Qt = mulmod_h(Qt, c->q[j] % t, t);
  D.Qt = Qt;
  for (uint32_t i = 0; i < c->L; ++i) {
    const u64 q = c->q[i];
    u64 rest = 1 % q, rest_t = 1 % t;
    for (uint32_t j = 0; j < c->L; ++j) {
      if (j == i) continue;
      rest = mulmod_h(rest, c->q[j] % q, q);
      rest_t = mulmod_h(rest_t, c->q[j] % t, t);
    }
    const u64 y = zn::powmod(rest, q - 2, q);
    const unsigned __int128 ty = (unsigned __int128)t * y;
    D.y[i] = y;
    D.It[i] = (u64)((ty / q) % t);
    D.r[i] = (u64)(ty % q);
    D.Qit[i] = rest_t;
  }
}

// Ciphertexts per prep/encrypt launch pair: me (8N) + small (3N) within
// 704 MiB (4096 ciphertexts at N = 2^14, as the CKKS path), in equal chunks.
uint32_t int_chunk(const zn_ctx* c, uint32_t batch) {
  size_t k = (704ull << 20) / (11 * (size_t)c->n);
  if (k < 1) k = 1;
  if (k > 65535) k = 65535;
  const size_t chunks = (batch + k - 1) / k;
  return (uint32_t)((batch + chunks - 1) / chunks);
}

// BFV / BGV encryption (vanilla under key/keys, Zinc over the cache `key`).
// m == nullptr: the zero plaintext; ct_index == nullptr: index b.
int int_common(zn_ctx* c, bool bgv, bool zinc, const u64* key, const u64* keys, uint64_t t, const int64_t* m,
               uint32_t batch, uint64_t seed, unsigned domain, const uint64_t* ct_index, uint64_t* ct,
               cudaStream_t st) {
  const uint32_t chunk = int_chunk(c, batch);
  const uint32_t first = batch < chunk ? batch : chunk;
  const size_t n = c->n;
  const size_t me_b = sizeof(i64) * first * n, sm_b = (zinc ? 2 : 3) * (size_t)first * n;
  Scratch scratch(c, st);
  if (!scratch.alloc(me_b + sm_b)) return ZN_ENOMEM;
  zn::IntArgs A;
  std::memset(&A, 0, sizeof(A));
  int_enc_consts(c, t, bgv, A);
  A.swap = 0;
  A.key = key;
  A.keys = keys;
  A.me = (const i64*)scratch.p;
  A.small = (const int8_t*)scratch.p + me_b;
  for (uint32_t b0 = 0; b0 < batch; b0 += chunk) {
    const uint32_t nb = (batch - b0) < chunk ? (batch - b0) : chunk;
    zn::IntPrepArgs pa;
    pa.m = m ? m + (size_t)b0 * n : nullptr;
    pa.t = t;
    pa.seed = seed;
    pa.domain = domain;
    pa.ct_index = ct_index ? ct_index + b0 : nullptr;
    pa.ct_index0 = b0;
    pa.me = (i64*)A.me;
    pa.small = (int8_t*)A.small;
    A.out = ct + (size_t)b0 * 2 * ring_words(c);
    {
      TimedLaunch tl(c, ZN_TIME_ENCODE, st);
      ZN_CUDA(zn::launch_prep_int(c->dp, pa, bgv, zinc, nb, st));
    }
    TimedLaunch tl(c, zinc ? ZN_TIME_ZINC : ZN_TIME_ENCRYPT, st);
    ZN_CUDA(zn::launch_encrypt_int(c->dp, A, bgv, zinc, nb, st));
  }
  return ZN_OK;
}

int int_decrypt(zn_ctx* c, const zn_sk* sk, uint64_t t, bool bgv, const uint64_t* ct, uint32_t batch, int64_t* m,
                cudaStream_t st) {
  zn::IntDec D;
  int_dec_consts(c, t, D);
  const size_t per = sizeof(u64) * ring_words(c);
  size_t k = (256ull << 20) / per;
  if (k < 1) k = 1;
  const uint32_t chunk = (uint32_t)(k < batch ? k : batch);
  Scratch scratch(c, st);
  if (!scratch.alloc(per * chunk)) return ZN_ENOMEM;
  u64* x = (u64*)scratch.p;
  for (uint32_t b0 = 0; b0 < batch; b0 += chunk) {
    const uint32_t nb = (batch - b0) < chunk ? (batch - b0) : chunk;
    ZN_CUDA(zn::launch_dec_mul(c->dp, ct + (size_t)b0 * 2 * ring_words(c), sk->d, nb, x, st));
    ZN_CUDA(zn::launch_ntt_inv(c->dp, x, nb, st));
    ZN_CUDA(zn::launch_int_decode(c->dp, D, bgv, x, nb, m + (size_t)b0 * c->n, st));
  }
  return ZN_OK;
}

inline bool int_ring(const zn_ctx* c) { return c->prm.log_n >= 10 && c->prm.log_n <= 15; }

}  // namespace

extern "C" {

const char* zn_strerror(int status) {
  switch (status) {
    case ZN_OK: return "ok";
    case ZN_EINVAL: return "invalid argument";
    case ZN_ENOMEM: return "out of device memory";
    case ZN_EOVERFLOW: return "encoded coefficient overflow (|m_k| >= 2^62 or not finite)";
    case ZN_ECUDA: return "CUDA runtime error";
    case ZN_ETIMEOUT: return "device wait timed out";
    case ZN_ENOPRIME: return "no NTT-friendly prime left for a chain entry";
    case ZN_ELIMIT: return "batch exceeds the fixed scratch of the allocation-free entry point";
    default: return "unknown status";
  }
}

int zn_host_primes(uint32_t log_n, const uint32_t* bits, uint32_t n_primes, uint64_t* out) {
  if (!bits || !out || log_n < 1 || log_n > 20) return ZN_EINVAL;
  for (uint32_t i = 0; i < n_primes; ++i)
    if (bits[i] < 2 || bits[i] > 62) return ZN_EINVAL;
  return zn::gen_primes(log_n, bits, n_primes, out) ? ZN_ENOPRIME : ZN_OK;
}

uint64_t zn_host_psi(uint64_t q, uint32_t log_n) { return zn::find_psi(q, log_n); }

int zn_host_encoder_twiddles(uint32_t log_n, double* re, double* im) {
  if (!re || !im || log_n < 2 || log_n > 20) return ZN_EINVAL;
  return zn::encoder_twiddles(log_n, re, im);
}

int zn_host_encoder_twiddles_q62(uint32_t log_n, int64_t* c, int64_t* s) {
  if (!c || !s || log_n < 2 || log_n > 20) return ZN_EINVAL;
  return zn::encoder_twiddles_q62(log_n, c, s);
}

int zn_host_cdt(uint64_t* out) {
  if (!out) return ZN_EINVAL;
  return zn::cdt_thresholds(out);
}

int zn_ctx_create(const zn_params* p, int device, zn_ctx** out) {
  if (!p || !out) return ZN_EINVAL;
  *out = nullptr;
  if (p->log_n < 4 || p->log_n > 15 || p->n_primes < 1 || p->n_primes > ZN_MAX_PRIMES || p->log2_delta < 1 ||
      p->log2_delta > 62)
    return ZN_EINVAL;
  for (uint32_t i = 0; i < p->n_primes; ++i)
    if (p->prime_bits[i] < 20 || p->prime_bits[i] > 61) return ZN_EINVAL;
  const uint32_t n = 1u << p->log_n, L = p->n_primes;
  zn_ctx* c = new (std::nothrow) zn_ctx();
  if (!c) return ZN_ENOMEM;
  c->device = device;
  c->prm = *p;
  c->n = n;
  c->L = L;
  // default launch shape: the radix-8, three-blocks-per-SM kernels where they
  // apply (the fastest measured at 2^13 and 2^14), else kind 0
  c->variant = (p->log_n >= 10 && p->log_n <= 15) ? 6 : 0;
  if (zn::gen_primes(p->log_n, p->prime_bits, L, c->q)) {
    delete c;
    return ZN_ENOPRIME;
  }
  for (uint32_t i = 0; i < L; ++i) c->psi[i] = zn::find_psi(c->q[i], p->log_n);

  // host tables
  // forward twiddles interleaved with their Shoup companions (one 16-byte
  // load per butterfly), then the inverse tables
  std::vector<u64> tabs(4 * (size_t)L * n);
  u64* twp = tabs.data();
  u64* itw = twp + 2 * (size_t)L * n;
  u64* itws = itw + (size_t)L * n;
  {
    std::vector<u64> tw(n), tws(n);
    for (uint32_t i = 0; i < L; ++i) {
      zn::ntt_tables(c->q[i], c->psi[i], p->log_n, tw.data(), tws.data(), itw + (size_t)i * n, itws + (size_t)i * n);
      for (uint32_t k = 0; k < n; ++k) {
        twp[2 * ((size_t)i * n + k)] = tw[k];
        twp[2 * ((size_t)i * n + k) + 1] = tws[k];
      }
    }
  }
  // decoder FP64 twiddles [2][N], then the encoder's Q62 pairs (C[k], -S[k]) [N]
  std::vector<double> etw(4 * (size_t)n);
  zn::encoder_twiddles(p->log_n, etw.data(), etw.data() + n);
  {
    std::vector<int64_t> qc(n), qs(n);
    zn::encoder_twiddles_q62(p->log_n, qc.data(), qs.data());
    std::vector<int64_t> pairs(2 * (size_t)n);
    for (uint32_t k = 0; k < n; ++k) {
      pairs[2 * k] = qc[k];
      pairs[2 * k + 1] = -qs[k];
    }
    std::memcpy(etw.data() + 2 * (size_t)n, pairs.data(), sizeof(int64_t) * pairs.size());
  }
  // [0, N/2): slot_of_t, the slot j with t_j = (5^j mod 2N - 1)/4 = t;
  // [N/2, N): pos_of_slot, slot j's place in the encoder FFT's input (t_j even:
  // re[brv(t_j / 2)], odd: im[brv(t_j / 2)], im following re at N/4)
  std::vector<int> slot(n);
  {
    const int lh = (int)p->log_n - 2;
    auto brv = [&](uint32_t x) {
      uint32_t r = 0;
      for (int b = 0; b < lh; ++b) r |= ((x >> b) & 1u) << (lh - 1 - b);
      return r;
    };
    u64 g = 1;
    for (uint32_t j = 0; j < n / 2; ++j) {
      const uint32_t t = (uint32_t)((g - 1) / 4);
      slot[t] = (int)j;
      slot[n / 2 + j] = (int)((t & 1u) * (n / 4) + brv(t >> 1));
      g = (g * 5) % (2ull * n);
    }
  }
  DevParams& dp = c->dp;
  std::memset(&dp, 0, sizeof(dp));
  dp.log_n = (int)p->log_n;
  dp.L = (int)L;
  dp.log2_delta = (int)p->log2_delta;
  for (uint32_t i = 0; i < L; ++i) {
    const u64 q = c->q[i];
    dp.q[i] = q;
    dp.mu[i] = (u64)((((unsigned __int128)1) << 64) / q);
    dp.moff[i] = (q - zn::powmod(2, 62, q)) % q;
    dp.ninv[i] = zn::powmod(n % q, q - 2, q);
    dp.ninvs[i] = zn::shoup(dp.ninv[i], q);
  }
  dp.q0inv_mod_q1 = L > 1 ? zn::powmod(c->q[0] % c->q[1], c->q[1] - 2, c->q[1]) : 0;
  for (uint32_t i = 0; i + 1 < L; ++i) {
    c->pinv[i] = zn::powmod(c->q[L - 1] % c->q[i], c->q[i] - 2, c->q[i]);
    c->pinvs[i] = zn::shoup(c->pinv[i], c->q[i]);
  }
  zn::cdt_thresholds(dp.cdt);

  DeviceGuard g(device);
  int rc = ZN_OK;
  if (cudaMalloc(&c->d_tw, sizeof(u64) * tabs.size()) != cudaSuccess ||
      cudaMalloc(&c->d_etw, sizeof(double) * etw.size()) != cudaSuccess ||
      cudaMalloc(&c->d_slot, sizeof(int) * slot.size()) != cudaSuccess ||
      cudaMalloc(&c->d_status, sizeof(unsigned)) != cudaSuccess) {
    rc = ZN_ENOMEM;
  } else if (cudaMemcpy(c->d_tw, tabs.data(), sizeof(u64) * tabs.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemcpy(c->d_etw, etw.data(), sizeof(double) * etw.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemcpy(c->d_slot, slot.data(), sizeof(int) * slot.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemset(c->d_status, 0, sizeof(unsigned)) != cudaSuccess) {
    rc = ZN_ECUDA;
  }
  if (rc) {
    cudaGetLastError();
    zn_ctx_destroy(c);
    return rc;
  }
  {
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    if (cudaMemPoolCreate(&c->pool, &props) != cudaSuccess) {
      cudaGetLastError();
      c->pool = nullptr;
      zn_ctx_destroy(c);
      return ZN_ECUDA;
    }
    uint64_t keep = ~0ull;   // keep freed scratch in the pool between calls
    cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  dp.twp = reinterpret_cast<const ulonglong2*>(c->d_tw);
  dp.itw = c->d_tw + 2 * (size_t)L * n;
  dp.itws = c->d_tw + 3 * (size_t)L * n;
  dp.etw = c->d_etw;
  dp.etq = reinterpret_cast<const longlong2*>(c->d_etw + 2 * (size_t)n);
  dp.slot_of_t = c->d_slot;
  dp.pos_of_slot = c->d_slot + n / 2;
  dp.status = c->d_status;
  *out = c;
  return ZN_OK;
}

void zn_ctx_destroy(zn_ctx* c) {
  if (!c) return;
  DeviceGuard g(c->device);
  zn_timing_enable(c, 0);
  for (cudaStream_t& h : c->hs)
    if (h) released(cudaStreamDestroy(h));
  if (c->hp) released(cudaStreamDestroy(c->hp));
  for (cudaEvent_t& e : c->hev)
    if (e) released(cudaEventDestroy(e));
  released(cudaFree(c->d_tw));
  released(cudaFree(c->d_etw));
  released(cudaFree(c->d_slot));
  released(cudaFree(c->d_status));
  if (c->pool) {
    released(cudaDeviceSynchronize());   // pending stream-ordered frees
    released(cudaMemPoolDestroy(c->pool));
  }
  delete c;
}

int zn_ctx_primes(const zn_ctx* c, uint64_t* primes, uint64_t* psis) {
  if (!c) return ZN_EINVAL;
  for (uint32_t i = 0; i < c->L; ++i) {
    if (primes) primes[i] = c->q[i];
    if (psis) psis[i] = c->psi[i];
  }
  return ZN_OK;
}

int zn_sync_status(zn_ctx* c, void* stream) {
  if (!c) return ZN_EINVAL;
  DeviceGuard g(c->device);
  unsigned st = 0;
  ZN_CUDA(cudaStreamSynchronize(S(stream)));
  ZN_CUDA(cudaMemcpy(&st, c->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost));
  ZN_CUDA(cudaMemset(c->d_status, 0, sizeof(unsigned)));
  if (st & zn::kStatusOverflow) return ZN_EOVERFLOW;
  if (st & zn::kStatusTimeout) return ZN_ETIMEOUT;
  if (st & zn::kStatusRange) return ZN_EINVAL;
  return ZN_OK;
}

int zn_timing_enable(zn_ctx* c, int on) {
  if (!c) return ZN_EINVAL;
  DeviceGuard g(c->device);
  if (!on) {
    for (auto& v : c->ev) {
      for (cudaEvent_t e : v) released(cudaEventDestroy(e));
      v.clear();
    }
  }
  c->timing = on != 0;
  return ZN_OK;
}

int zn_timing_read(zn_ctx* c, int kind, double* ms, uint64_t* launches) {
  if (!c || kind < 0 || kind >= ZN_TIME_KINDS) return ZN_EINVAL;
  DeviceGuard g(c->device);
  auto& v = c->ev[kind];
  double total = 0.0;
  int rc = ZN_OK;
  for (size_t k = 0; k + 1 < v.size(); k += 2) {
    float t = 0.f;
    if (cudaEventSynchronize(v[k + 1]) != cudaSuccess || cudaEventElapsedTime(&t, v[k], v[k + 1]) != cudaSuccess)
      rc = ZN_ECUDA;
    total += t;
  }
  if (ms) *ms = total;
  if (launches) *launches = v.size() / 2;
  for (cudaEvent_t e : v) cudaEventDestroy(e);
  v.clear();
  cudaGetLastError();
  return rc;
}

// ------------------------------------------------------------------ keys

int ckks_keygen(zn_ctx* c, uint64_t seed, zn_sk** sk, zn_pk** pk) {
  NvtxRange nvtx("ckks_keygen");
  if (!c || !sk || !pk) return ZN_EINVAL;
  *sk = nullptr;
  *pk = nullptr;
  DeviceGuard g(c->device);
  zn_sk* s = new (std::nothrow) zn_sk();
  zn_pk* k = new (std::nothrow) zn_pk();
  if (!s || !k) {
    delete s;
    delete k;
    return ZN_ENOMEM;
  }
  s->ctx = c;
  s->device = c->device;
  k->ctx = c;
  k->device = c->device;
  const size_t rw = ring_words(c);
  i64* d_s = nullptr;
  if (cudaMalloc(&s->d, sizeof(u64) * rw) != cudaSuccess || cudaMalloc(&k->d, sizeof(u64) * 4 * rw) != cudaSuccess ||
      cudaMalloc(&d_s, sizeof(i64) * c->n) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(s->d);
    cudaFree(k->d);
    cudaFree(d_s);
    delete s;
    delete k;
    return ZN_ENOMEM;
  }
  int rc = ZN_OK;
  if (zn::launch_keygen(c->dp, seed, s->d, k->d, k->d + 2 * rw, 0) != cudaSuccess ||
      zn::launch_sample(c->dp, 0, seed, 2, 0, 0, 0, 1, d_s, 0) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess) {
    rc = ZN_ECUDA;
  } else {
    std::vector<i64> tmp(c->n);
    if (cudaMemcpy(tmp.data(), d_s, sizeof(i64) * c->n, cudaMemcpyDeviceToHost) != cudaSuccess) rc = ZN_ECUDA;
    s->s.resize(c->n);
    for (uint32_t j = 0; j < c->n; ++j) s->s[j] = (int8_t)tmp[j];
  }
  cudaFree(d_s);
  if (!rc) rc = ms_key_forms(c, k);
  if (rc) {
    cudaGetLastError();
    zn_sk_destroy(s);
    zn_pk_destroy(k);
    return rc;
  }
  *sk = s;
  *pk = k;
  return ZN_OK;
}

void zn_sk_destroy(zn_sk* s) {
  if (!s || s->tag != kTagSk) return;
  s->tag = kTagDead;
  DeviceGuard g(s->device);
  released(cudaFree(s->d));
  delete s;
}

void zn_pk_destroy(zn_pk* k) {
  if (!k || k->tag != kTagPk) return;
  k->tag = kTagDead;
  DeviceGuard g(k->device);
  released(cudaFree(k->d));
  released(cudaFree(k->ms));
  delete k;
}

int zn_pk_export(const zn_pk* k, uint64_t* host_out) {
  if (!k || k->tag != kTagPk || !host_out) return ZN_EINVAL;
  DeviceGuard g(k->device);
  ZN_CUDA(cudaMemcpy(host_out, k->d, sizeof(u64) * 2 * ring_words(k->ctx), cudaMemcpyDeviceToHost));
  return ZN_OK;
}

int zn_pk_import(zn_ctx* c, const uint64_t* host_in, zn_pk** out) {
  if (!c || !host_in || !out) return ZN_EINVAL;
  *out = nullptr;
  const size_t rw = ring_words(c);
  for (uint32_t i = 0; i < c->L; ++i)
    for (int p = 0; p < 2; ++p)
      for (uint32_t j = 0; j < c->n; ++j)
        if (host_in[(size_t)p * rw + (size_t)i * c->n + j] >= c->q[i]) return ZN_EINVAL;
  DeviceGuard g(c->device);
  zn_pk* k = new (std::nothrow) zn_pk();
  if (!k) return ZN_ENOMEM;
  k->ctx = c;
  k->device = c->device;
  if (cudaMalloc(&k->d, sizeof(u64) * 4 * rw) != cudaSuccess) {
    cudaGetLastError();
    delete k;
    return ZN_ENOMEM;
  }
  if (cudaMemcpy(k->d, host_in, sizeof(u64) * 2 * rw, cudaMemcpyHostToDevice) != cudaSuccess ||
      zn::launch_shoup(c->dp, k->d, k->d + 2 * rw, 2, 0) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    zn_pk_destroy(k);
    return ZN_ECUDA;
  }
  const int rc = ms_key_forms(c, k);
  if (rc) {
    zn_pk_destroy(k);
    return rc;
  }
  *out = k;
  return ZN_OK;
}

int zn_sk_export(const zn_sk* s, int8_t* host_out) {
  if (!s || s->tag != kTagSk || !host_out) return ZN_EINVAL;
  std::memcpy(host_out, s->s.data(), s->s.size());
  return ZN_OK;
}

int zn_sk_import(zn_ctx* c, const int8_t* host_in, zn_sk** out) {
  if (!c || !host_in || !out) return ZN_EINVAL;
  *out = nullptr;
  for (uint32_t j = 0; j < c->n; ++j)
    if (host_in[j] < -1 || host_in[j] > 1) return ZN_EINVAL;
  DeviceGuard g(c->device);
  zn_sk* s = new (std::nothrow) zn_sk();
  if (!s) return ZN_ENOMEM;
  s->ctx = c;
  s->device = c->device;
  s->s.assign(host_in, host_in + c->n);
  const size_t rw = ring_words(c);
  int8_t* d_s = nullptr;
  u64* tmp = nullptr;
  if (cudaMalloc(&s->d, sizeof(u64) * rw) != cudaSuccess || cudaMalloc(&d_s, c->n) != cudaSuccess ||
      cudaMalloc(&tmp, sizeof(u64) * rw) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(d_s);
    cudaFree(tmp);
    zn_sk_destroy(s);
    return ZN_ENOMEM;
  }
  int rc = ZN_OK;
  if (cudaMemcpy(d_s, host_in, c->n, cudaMemcpyHostToDevice) != cudaSuccess ||
      zn::launch_sk_residues(c->dp, d_s, s->d, 0) != cudaSuccess ||
      zn::launch_ntt_fwd(c->dp, s->d, 1, tmp, 0) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
    rc = ZN_ECUDA;
  cudaFree(d_s);
  cudaFree(tmp);
  if (rc) {
    cudaGetLastError();
    zn_sk_destroy(s);
    return rc;
  }
  *out = s;
  return ZN_OK;
}

// --------------------------------------------------------------- encode

int ckks_encode(zn_ctx* c, const double* slots, uint32_t n_slots, uint32_t batch, int64_t* out, void* stream) {
  NvtxRange nvtx("ckks_encode");
  if (!c || n_slots > c->n / 2) return ZN_EINVAL;
  if (batch == 0) return ZN_OK;
  if (!out || (n_slots && !slots)) return ZN_EINVAL;
  DeviceGuard g(c->device);
  ZN_CUDA(zn::launch_encode(c->dp, slots, n_slots, batch, (i64*)out, S(stream)));
  return ZN_OK;
}

int ckks_encode_ragged(zn_ctx* c, const double* slots, const uint32_t* n_slots, uint32_t stride, uint32_t batch,
                       int64_t* out, void* stream) {
  NvtxRange nvtx("ckks_encode_ragged");
  if (!c || stride > c->n / 2) return ZN_EINVAL;
  if (batch == 0) return ZN_OK;
  if (!out || !n_slots || (stride && !slots)) return ZN_EINVAL;
  DeviceGuard g(c->device);
  ZN_CUDA(zn::launch_encode_ragged(c->dp, slots, n_slots, stride, batch, (i64*)out, S(stream)));
  return ZN_OK;
}

// -------------------------------------------------------------- encrypt

int ckks_encrypt(zn_ctx* c, const zn_pk* pk, const double* slots, uint32_t n_slots, uint32_t batch, uint64_t seed,
                 const uint64_t* ct_index, uint64_t* ct, void* stream) {
  NvtxRange nvtx("ckks_encrypt");
  if (!c || !pk_of(pk, c)) return ZN_EINVAL;
  return encrypt_common(c, false, pk->d, pk->d + 2 * ring_words(c), slots, n_slots, batch, seed, ct_index, ct,
                        stream);
}

int ckks_encrypt_ragged(zn_ctx* c, const zn_pk* pk, const double* slots, const uint32_t* n_slots, uint32_t stride,
                        uint32_t batch, uint64_t seed, const uint64_t* ct_index, uint64_t* ct, void* stream) {
  NvtxRange nvtx("ckks_encrypt_ragged");
  if (!c || !pk_of(pk, c) || (batch && !n_slots)) return ZN_EINVAL;
  return encrypt_common(c, false, pk->d, pk->d + 2 * ring_words(c), slots, 0, batch, seed, ct_index, ct, stream,
                        n_slots, stride);
}

int zinc_precompute(zn_ctx* c, const zn_pk* pk, uint64_t seed, zn_zcache** out) {
  NvtxRange nvtx("zinc_precompute");
  if (!c || !pk_of(pk, c) || !out) return ZN_EINVAL;
  *out = nullptr;
  DeviceGuard g(c->device);
  zn_zcache* z = new (std::nothrow) zn_zcache();
  if (!z) return ZN_ENOMEM;
  z->ctx = c;
  z->device = c->device;
  if (cudaMalloc(&z->d, sizeof(u64) * 2 * ring_words(c)) != cudaSuccess) {
    cudaGetLastError();
    delete z;
    return ZN_ENOMEM;
  }
  // vanilla Enc of the zero plaintext, sampling domain 3, ct_index 0
  const size_t me_b = sizeof(i64) * c->n, sm_b = 2 * (size_t)c->n;
  int rc = ZN_OK;
  {
    Scratch scratch(c, 0);
    if (!scratch.alloc(me_b + sm_b)) {
      rc = ZN_ENOMEM;
    } else {
      zn::PrepArgs pa;
      pa.slots = nullptr;
      pa.n_slots = 0;
      pa.ct_index = nullptr;
      pa.ct_index0 = 0;
      pa.seed = seed;
      pa.domain = 3;
      pa.me = (i64*)scratch.p;
      pa.small = (int8_t*)scratch.p + me_b;
      zn::EncArgs A;
      A.swap = 0;
      A.key = pk->d;
      A.keys = pk->d + 2 * ring_words(c);
      A.me = pa.me;
      A.small = pa.small;
      A.out = z->d;
      if (zn::launch_prep(c->dp, pa, false, 1, 0) != cudaSuccess ||
          zn::launch_encrypt(c->dp, A, false, 1, c->variant, 0) != cudaSuccess)
        rc = ZN_ECUDA;
    }
  }
  if (!rc && cudaDeviceSynchronize() != cudaSuccess) rc = ZN_ECUDA;
  if (rc) {
    cudaGetLastError();
    zn_zcache_destroy(z);
    return rc;
  }
  *out = z;
  return ZN_OK;
}

void zn_zcache_destroy(zn_zcache* z) {
  if (!z || z->tag != kTagZc) return;
  z->tag = kTagDead;
  DeviceGuard g(z->device);
  released(cudaFree(z->d));
  delete z;
}

int zn_zcache_export(const zn_zcache* z, uint64_t* host_out) {
  if (!z || z->tag != kTagZc || !host_out) return ZN_EINVAL;
  DeviceGuard g(z->device);
  ZN_CUDA(cudaMemcpy(host_out, z->d, sizeof(u64) * 2 * ring_words(z->ctx), cudaMemcpyDeviceToHost));
  return ZN_OK;
}

int zn_zcache_import(zn_ctx* c, const uint64_t* host_in, zn_zcache** out) {
  if (!c || !host_in || !out) return ZN_EINVAL;
  *out = nullptr;
  const size_t rw = ring_words(c);
  for (uint32_t i = 0; i < c->L; ++i)
    for (int p = 0; p < 2; ++p)
      for (uint32_t j = 0; j < c->n; ++j)
        if (host_in[(size_t)p * rw + (size_t)i * c->n + j] >= c->q[i]) return ZN_EINVAL;
  DeviceGuard g(c->device);
  zn_zcache* z = new (std::nothrow) zn_zcache();
  if (!z) return ZN_ENOMEM;
  z->ctx = c;
  z->device = c->device;
  if (cudaMalloc(&z->d, sizeof(u64) * 2 * rw) != cudaSuccess) {
    cudaGetLastError();
    delete z;
    return ZN_ENOMEM;
  }
  if (cudaMemcpy(z->d, host_in, sizeof(u64) * 2 * rw, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    zn_zcache_destroy(z);
    return ZN_ECUDA;
  }
  *out = z;
  return ZN_OK;
}

int zinc_encrypt(zn_ctx* c, const zn_zcache* z, const double* slots, uint32_t n_slots, uint32_t batch, uint64_t seed,
                 const uint64_t* ct_index, uint64_t* ct, void* stream) {
  NvtxRange nvtx("zinc_encrypt");
  if (!c || !zc_of(z, c)) return ZN_EINVAL;
  return encrypt_common(c, true, z->d, nullptr, slots, n_slots, batch, seed, ct_index, ct, stream);
}

int zinc_encrypt_ragged(zn_ctx* c, const zn_zcache* z, const double* slots, const uint32_t* n_slots, uint32_t stride,
                        uint32_t batch, uint64_t seed, const uint64_t* ct_index, uint64_t* ct, void* stream) {
  NvtxRange nvtx("zinc_encrypt_ragged");
  if (!c || !zc_of(z, c) || (batch && !n_slots)) return ZN_EINVAL;
  return encrypt_common(c, true, z->d, nullptr, slots, 0, batch, seed, ct_index, ct, stream, n_slots, stride);
}

// ------------------------------------- special prime and modulus switching

int ckks_encrypt_ms(zn_ctx* c, const zn_pk* pk, const double* slots, uint32_t n_slots, uint32_t batch,
                    uint64_t seed, const uint64_t* ct_index, uint64_t* ct, void* stream) {
  NvtxRange nvtx("ckks_encrypt_ms");
  if (!c || !pk_of(pk, c) || c->L < 2 || !pk->ms || n_slots > c->n / 2) return ZN_EINVAL;
  if (batch == 0) return ZN_OK;
  if (!ct || !ct_index || (n_slots && !slots)) return ZN_EINVAL;
  DeviceGuard g(c->device);
  return ms_common(c, pk, slots, n_slots, batch, seed, 0u, ct_index, ct, S(stream));
}

int zinc_precompute_ms(zn_ctx* c, const zn_pk* pk, uint64_t seed, zn_ctx* dc, zn_zcache** out) {
  NvtxRange nvtx("zinc_precompute_ms");
  if (!c || !pk_of(pk, c) || c->L < 2 || !pk->ms || !dc || !out) return ZN_EINVAL;
  *out = nullptr;
  if (dc->device != c->device || dc->L != c->L - 1 || dc->prm.log_n != c->prm.log_n ||
      dc->prm.log2_delta != c->prm.log2_delta)
    return ZN_EINVAL;
  for (uint32_t i = 0; i < dc->L; ++i)
    if (dc->q[i] != c->q[i]) return ZN_EINVAL;
  DeviceGuard g(c->device);
  zn_zcache* z = new (std::nothrow) zn_zcache();
  if (!z) return ZN_ENOMEM;
  z->ctx = dc;
  z->device = dc->device;
  if (cudaMalloc(&z->d, sizeof(u64) * 2 * ring_words(dc)) != cudaSuccess) {
    cudaGetLastError();
    delete z;
    return ZN_ENOMEM;
  }
  // modulus-switched Enc of the zero plaintext, sampling domain 3, ct_index 0
  int rc = ms_common(c, pk, nullptr, 0, 1, seed, 3u, nullptr, z->d, 0);
  if (!rc && cudaDeviceSynchronize() != cudaSuccess) rc = ZN_ECUDA;
  if (rc) {
    cudaGetLastError();
    zn_zcache_destroy(z);
    return rc;
  }
  *out = z;
  return ZN_OK;
}

// ------------------------------------------------------------ BFV / BGV

int bfv_encrypt(zn_ctx* c, const zn_pk* pk, uint64_t t, const int64_t* m, uint32_t batch, uint64_t seed,
                const uint64_t* ct_index, uint64_t* ct, void* stream) {
  NvtxRange nvtx("bfv_encrypt");
  if (!c || !pk_of(pk, c) || !int_ring(c) || !t_ok(c, t)) return ZN_EINVAL;
  if (batch == 0) return ZN_OK;
  if (!m || !ct_index || !ct) return ZN_EINVAL;
  DeviceGuard g(c->device);
  return int_common(c, false, false, pk->d, pk->d + 2 * ring_words(c), t, m, batch, seed, 0u, ct_index, ct,
                    S(stream));
}

int bfv_zinc_encrypt(zn_ctx* c, const zn_zcache* z, uint64_t t, const int64_t* m, uint32_t batch, uint64_t seed,
                     const uint64_t* ct_index, uint64_t* ct, void* stream) {
  NvtxRange nvtx("bfv_zinc_encrypt");
  if (!c || !zc_of(z, c) || !int_ring(c) || !t_ok(c, t)) return ZN_EINVAL;
  if (batch == 0) return ZN_OK;
  if (!m || !ct_index || !ct) return ZN_EINVAL;
  DeviceGuard g(c->device);
  return int_common(c, false, true, z->d, nullptr, t, m, batch, seed, 1u, ct_index, ct, S(stream));
}

int bgv_keygen(zn_ctx* c, uint64_t t, uint64_t seed, zn_sk** sk, zn_pk** pk) {
  NvtxRange nvtx("bgv_keygen");
  if (!c || !sk || !pk || !int_ring(c) || !t_ok(c, t)) return ZN_EINVAL;
  int rc = ckks_keygen(c, seed, sk, pk);
  if (rc) return rc;
  DeviceGuard g(c->device);
  zn_pk* k = *pk;
  const size_t rw = ring_words(c);
  i64* e = nullptr;
  u64* eh = nullptr;
  u64* tmp = nullptr;
  if (cudaMalloc(&e, sizeof(i64) * c->n) != cudaSuccess || cudaMalloc(&eh, sizeof(u64) * rw) != cudaSuccess ||
      cudaMalloc(&tmp, sizeof(u64) * rw) != cudaSuccess) {
    rc = ZN_ENOMEM;
  } else if (zn::launch_sample(c->dp, 1, seed, 2, 2, 0, 0, 1, e, 0) != cudaSuccess ||   // Gen's e (domain 2, poly 2)
             zn::launch_residues(c->dp, e, eh, 0) != cudaSuccess ||
             zn::launch_ntt_fwd(c->dp, eh, 1, tmp, 0) != cudaSuccess ||
             zn::launch_bgv_key(c->dp, t, eh, k->d, k->d + 2 * rw, 0) != cudaSuccess ||
             cudaDeviceSynchronize() != cudaSuccess) {
    rc = ZN_ECUDA;
  }
  cudaGetLastError();
  cudaFree(e);
  cudaFree(eh);
  cudaFree(tmp);
  if (rc) {
    zn_sk_destroy(*sk);
    zn_pk_destroy(k);
    *sk = nullptr;
    *pk = nullptr;
    return rc;
  }
  cudaFree(k->ms);          // the SEAL-ordered key forms belong to Gen's key
  k->ms = nullptr;
  k->t = t;
  return ZN_OK;
}

int bgv_zinc_precompute(zn_ctx* c, const zn_pk* pk, uint64_t seed, zn_zcache** out) {
  if (!c || !bgv_pk_of(pk, c) || !out) return ZN_EINVAL;
  *out = nullptr;
  DeviceGuard g(c->device);
  zn_zcache* z = new (std::nothrow) zn_zcache();
  if (!z) return ZN_ENOMEM;
  z->ctx = c;
  z->device = c->device;
  z->t = pk->t;
  if (cudaMalloc(&z->d, sizeof(u64) * 2 * ring_words(c)) != cudaSuccess) {
    cudaGetLastError();
    delete z;
    return ZN_ENOMEM;
  }
  // a BGV encryption of the zero plaintext, sampling domain 3, ct_index 0
  int rc = int_common(c, true, false, pk->d, pk->d + 2 * ring_words(c), pk->t, nullptr, 1, seed, 3u, nullptr, z->d,
                      0);
  if (!rc && cudaDeviceSynchronize() != cudaSuccess) rc = ZN_ECUDA;
  if (rc) {
    cudaGetLastError();
    zn_zcache_destroy(z);
    return rc;
  }
  *out = z;
  return ZN_OK;
}

int bgv_encrypt(zn_ctx* c, const zn_pk* pk, const int64_t* m, uint32_t batch, uint64_t seed,
                const uint64_t* ct_index, uint64_t* ct, void* stream) {
  NvtxRange nvtx("bgv_encrypt");
  if (!c || !bgv_pk_of(pk, c)) return ZN_EINVAL;
  if (batch == 0) return ZN_OK;
  if (!m || !ct_index || !ct) return ZN_EINVAL;
  DeviceGuard g(c->device);
  return int_common(c, true, false, pk->d, pk->d + 2 * ring_words(c), pk->t, m, batch, seed, 0u, ct_index, ct,
                    S(stream));
}

int bgv_zinc_encrypt(zn_ctx* c, const zn_zcache* z, const int64_t* m, uint32_t batch, uint64_t seed,
                     const uint64_t* ct_index, uint64_t* ct, void* stream) {
  NvtxRange nvtx("bgv_zinc_encrypt");
  if (!c || !bgv_zc_of(z, c)) return ZN_EINVAL;
  if (batch == 0) return ZN_OK;
  if (!m || !ct_index || !ct) return ZN_EINVAL;
  DeviceGuard g(c->device);
  return int_common(c, true, true, z->d, nullptr, z->t, m, batch, seed, 1u, ct_index, ct, S(stream));
}

int bfv_decrypt(zn_ctx* c, const zn_sk* sk, uint64_t t, const uint64_t* ct, uint32_t batch, int64_t* m,
                void* stream) {
  NvtxRange nvtx("bfv_decrypt");
  if (!c || !sk_of(sk, c) || !int_ring(c) || !t_ok(c, t)) return ZN_EINVAL;
  if (batch == 0) return ZN_OK;
  if (!ct || !m) return ZN_EINVAL;
  DeviceGuard g(c->device);
  return int_decrypt(c, sk, t, false, ct, batch, m, S(stream));
}

int bgv_decrypt(zn_ctx* c, const zn_sk* sk, uint64_t t, const uint64_t* ct, uint32_t batch, int64_t* m,
                void* stream) {
  NvtxRange nvtx("bgv_decrypt");
  if (!c || !sk_of(sk, c) || !int_ring(c) || !t_ok(c, t)) return ZN_EINVAL;
  if (batch == 0) return ZN_OK;
  if (!ct || !m) return ZN_EINVAL;
  DeviceGuard g(c->device);
  return int_decrypt(c, sk, t, true, ct, batch, m, S(stream));
}

// ------------------------------------------------- slot batching (BFV, BGV)

void zn_slot_encoder_destroy(zn_slot_encoder* se) {
  if (!se || se->tag != kTagSe) return;
  se->tag = kTagDead;
  DeviceGuard g(se->device);
  released(cudaFree(se->d));
  delete se;
}

int zn_slot_encoder_create(zn_ctx* c, uint64_t t, zn_slot_encoder** out) {
  if (!c || !out || !int_ring(c) || !t_ok(c, t)) return ZN_EINVAL;
  *out = nullptr;
  const uint32_t log_n = c->prm.log_n, n = c->n;
  if (!zn::is_prime(t) || t % (2ull * n) != 1) return ZN_EINVAL;
  zn_slot_encoder* se = new (std::nothrow) zn_slot_encoder();
  if (!se) return ZN_ENOMEM;
  se->ctx = c;
  se->device = c->device;
  const u64 psi = zn::find_psi(t, log_n);
  std::vector<u64> tw(n), tws(n), itw(n), itws(n);
  zn::ntt_tables(t, psi, log_n, tw.data(), tws.data(), itw.data(), itws.data());
  std::vector<ulonglong2> twp(n);
  for (uint32_t k = 0; k < n; ++k) twp[k] = make_ulonglong2(tw[k], tws[k]);
  // slot s <-> psi^(a_s), a_s = 5^s (s < N/2) or -5^(s - N/2) mod 2N; NTT index i
  // evaluates at psi^(2 brv(i) + 1)
  std::vector<int> pos(n);
  {
    u64 g = 1;
    for (uint32_t s2 = 0; s2 < n / 2; ++s2) {
      const u64 a[2] = {g, 2ull * n - g};
      for (int h = 0; h < 2; ++h) {
        const uint32_t e = (uint32_t)((a[h] - 1) / 2);
        uint32_t r = 0;
        for (uint32_t bit = 0; bit < log_n; ++bit) r |= ((e >> bit) & 1u) << (log_n - 1 - bit);
        pos[h * (n / 2) + s2] = (int)r;
      }
      g = g * 5 % (2ull * n);
    }
  }
  const size_t b_tw = sizeof(ulonglong2) * n, b_w = sizeof(u64) * n, b_pos = sizeof(int) * n;
  DeviceGuard gd(c->device);
  if (cudaMalloc(&se->d, b_tw + 2 * b_w + b_pos) != cudaSuccess) {
    cudaGetLastError();
    delete se;
    return ZN_ENOMEM;
  }
  unsigned char* base = (unsigned char*)se->d;
  if (cudaMemcpy(base, twp.data(), b_tw, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(base + b_tw, itw.data(), b_w, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(base + b_tw + b_w, itws.data(), b_w, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(base + b_tw + 2 * b_w, pos.data(), b_pos, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    zn_slot_encoder_destroy(se);
    return ZN_ECUDA;
  }
  zn::BatchEnc& E = se->E;
  E.log_n = (int)log_n;
  E.t = t;
  E.ninv = zn::powmod(n % t, t - 2, t);
  E.ninvs = zn::shoup(E.ninv, t);
  E.twp = (const ulonglong2*)base;
  E.itw = (const u64*)(base + b_tw);
  E.itws = (const u64*)(base + b_tw + b_w);
  E.pos = (const int*)(base + b_tw + 2 * b_w);
  *out = se;
  return ZN_OK;
}

int zn_slots_encode(zn_slot_encoder* se, const int64_t* slots, uint32_t batch, int64_t* m, void* stream) {
  NvtxRange nvtx("zn_slots_encode");
  if (!se || se->tag != kTagSe) return ZN_EINVAL;
  if (batch == 0) return ZN_OK;
  if (!slots || !m) return ZN_EINVAL;
  DeviceGuard g(se->device);
  ZN_CUDA(zn::launch_batch_encode(se->E, slots, batch, m, S(stream)));
  return ZN_OK;
}

int zn_slots_decode(zn_slot_encoder* se, const int64_t* m, uint32_t batch, int64_t* slots, void* stream) {
  NvtxRange nvtx("zn_slots_decode");
  if (!se || se->tag != kTagSe) return ZN_EINVAL;
  if (batch == 0) return ZN_OK;
  if (!slots || !m) return ZN_EINVAL;
  DeviceGuard g(se->device);
  Scratch scratch(se->ctx, S(stream));
  if (!scratch.alloc(sizeof(u64) * batch * (size_t)se->ctx->n)) return ZN_ENOMEM;
  ZN_CUDA(zn::launch_batch_decode(se->E, m, batch, (u64*)scratch.p, slots, S(stream)));
  return ZN_OK;
}

// ------------------------------------------- Zinc with NTT-domain errors

void zn_nbasis_destroy(zn_nbasis* nb) {
  if (!nb || nb->tag != kTagNb) return;
  nb->tag = kTagDead;
  DeviceGuard g(nb->device);
  released(cudaFree(nb->E));
  released(cudaFree(nb->thi));
  released(cudaFree(nb->tlo));
  delete nb;
}

int zinc_nbasis_create(zn_ctx* c, uint32_t K, uint64_t seed, zn_nbasis** out) {
  if (!c || !out || K < 1 || K > 16 || !int_ring(c)) return ZN_EINVAL;
  *out = nullptr;
  DeviceGuard g(c->device);
  zn_nbasis* nb = new (std::nothrow) zn_nbasis();
  if (!nb) return ZN_ENOMEM;
  nb->ctx = c;
  nb->device = c->device;
  nb->K = K;
  const size_t n = c->n, rw = ring_words(c), nhi = n / 32;
  // power tables on the host: psi^(64 h), h < 2N/64, and psi^l 2^64 (the
  // Montgomery form, so that one Montgomery product of the two is psi^e), per prime
  std::vector<u64> hi(c->L * nhi), lo(c->L * 64);
  for (uint32_t i = 0; i < c->L; ++i) {
    const u64 q = c->q[i], psi = c->psi[i], p64 = zn::powmod(psi, 64, q);
    const u64 r64 = (u64)((((unsigned __int128)1) << 64) % q);
    u64 v = 1;
    for (size_t h = 0; h < nhi; ++h, v = mulmod_h(v, p64, q)) hi[i * nhi + h] = v;
    v = r64;
    for (int l = 0; l < 64; ++l, v = mulmod_h(v, psi, q)) lo[i * 64 + l] = v;
  }
  i64* e = nullptr;
  u64* tmp = nullptr;
  int rc = ZN_OK;
  if (cudaMalloc(&nb->E, sizeof(u64) * 2 * K * rw) != cudaSuccess ||
      cudaMalloc(&nb->thi, sizeof(u64) * hi.size()) != cudaSuccess ||
      cudaMalloc(&nb->tlo, sizeof(u64) * lo.size()) != cudaSuccess ||
      cudaMalloc(&e, sizeof(i64) * n) != cudaSuccess || cudaMalloc(&tmp, sizeof(u64) * rw) != cudaSuccess) {
    rc = ZN_ENOMEM;
  } else if (cudaMemcpy(nb->thi, hi.data(), sizeof(u64) * hi.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
             cudaMemcpy(nb->tlo, lo.data(), sizeof(u64) * lo.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
    rc = ZN_ECUDA;
  } else {
    // E_{c,j} <- chi (domain 4, poly 16 c + j, ct_index 0), residues, forward NTT
    for (uint32_t cj = 0; cj < 2 * K && !rc; ++cj) {
      const uint32_t cc = cj / K, j = cj % K;
      u64* slot = nb->E + (size_t)cj * rw;
      if (zn::launch_sample(c->dp, 1, seed, 4, 16 * cc + j, 0, 0, 1, e, 0) != cudaSuccess ||
          zn::launch_residues(c->dp, e, slot, 0) != cudaSuccess ||
          zn::launch_ntt_fwd(c->dp, slot, 1, tmp, 0) != cudaSuccess)
        rc = ZN_ECUDA;
    }
    if (!rc && cudaDeviceSynchronize() != cudaSuccess) rc = ZN_ECUDA;
  }
  cudaGetLastError();
  cudaFree(e);
  cudaFree(tmp);
  if (rc) {
    zn_nbasis_destroy(nb);
    return rc;
  }
  *out = nb;
  return ZN_OK;
}

int ckks_encode_ntt(zn_ctx* c, const double* slots, uint32_t n_slots, uint32_t batch, uint64_t* out, void* stream) {
  NvtxRange nvtx("ckks_encode_ntt");
  if (!c || n_slots > c->n / 2) return ZN_EINVAL;
  if (batch == 0) return ZN_OK;
  if (!out || (n_slots && !slots)) return ZN_EINVAL;
  DeviceGuard g(c->device);
  const size_t n = c->n, rw = ring_words(c);
  size_t k = (256ull << 20) / (sizeof(u64) * rw);
  if (k < 1) k = 1;
  const uint32_t chunk = (uint32_t)(k < batch ? k : batch);
  const bool big = c->prm.log_n == 15;    // the 2^15 forward transform goes through a copy
  Scratch scratch(c, S(stream));
  if (!scratch.alloc(sizeof(i64) * chunk * n + (big ? sizeof(u64) * chunk * rw : 0))) return ZN_ENOMEM;
  i64* coef = (i64*)scratch.p;
  u64* tmp = big ? (u64*)((unsigned char*)scratch.p + sizeof(i64) * chunk * n) : nullptr;
  for (uint32_t b0 = 0; b0 < batch; b0 += chunk) {
    const uint32_t nb = (batch - b0) < chunk ? (batch - b0) : chunk;
    u64* o = out + (size_t)b0 * rw;
    ZN_CUDA(zn::launch_encode(c->dp, n_slots ? slots + (size_t)b0 * n_slots : nullptr, n_slots, nb, coef, S(stream)));
    ZN_CUDA(zn::launch_residues_batch(c->dp, coef, nb, o, S(stream)));
    ZN_CUDA(zn::launch_ntt_fwd(c->dp, o, nb, tmp, S(stream)));
  }
  return ZN_OK;
}

int zinc_encrypt_ntt(zn_ctx* c, const zn_zcache* z, const zn_nbasis* nb, const uint64_t* m_hat, uint32_t batch,
                     uint64_t seed, const uint64_t* ct_index, uint64_t* ct, void* stream) {
  NvtxRange nvtx("zinc_encrypt_ntt");
  if (!c || !zc_of(z, c) || !nb || nb->tag != kTagNb || nb->ctx != c) return ZN_EINVAL;
  if (batch == 0) return ZN_OK;
  if (!m_hat || !ct_index || !ct) return ZN_EINVAL;
  DeviceGuard g(c->device);
  zn::NttZincArgs A;
  std::memset(&A, 0, sizeof(A));
  for (uint32_t i = 0; i < c->L; ++i) {
    u64 inv = 1;                          // q^-1 mod 2^64 by Newton's iteration (q odd)
    for (int it = 0; it < 6; ++it) inv *= 2 - c->q[i] * inv;
    A.qneg[i] = (u64)0 - inv;
  }
  A.z = z->d;
  A.E = nb->E;
  A.thi = nb->thi;
  A.tlo = nb->tlo;
  A.seed = seed;
  A.K = (int)nb->K;
  const size_t rw = ring_words(c);
  for (uint32_t b0 = 0; b0 < batch; b0 += 65535) {
    const uint32_t n_b = (batch - b0) < 65535 ? (batch - b0) : 65535;
    A.m = m_hat + (size_t)b0 * rw;
    A.ct_index = ct_index + b0;
    A.out = ct + (size_t)b0 * 2 * rw;
    TimedLaunch t(c, ZN_TIME_ZINC_NTT, S(stream));
    ZN_CUDA(zn::launch_zinc_ntt(c->dp, A, n_b, S(stream)));
  }
  return ZN_OK;
}

// -------------------------------------------------------------- decrypt

int ckks_decrypt(zn_ctx* c, const zn_sk* sk, const uint64_t* ct, uint32_t batch, uint64_t* out, void* stream) {
  NvtxRange nvtx("ckks_decrypt");
  if (!c || !sk_of(sk, c)) return ZN_EINVAL;
  if (batch == 0) return ZN_OK;
  if (!ct || !out) return ZN_EINVAL;
  DeviceGuard g(c->device);
  ZN_CUDA(zn::launch_dec_mul(c->dp, ct, sk->d, batch, out, S(stream)));
  ZN_CUDA(zn::launch_ntt_inv(c->dp, out, batch, S(stream)));
  return ZN_OK;
}

int ckks_decrypt_decode(zn_ctx* c, const zn_sk* sk, const uint64_t* ct, uint32_t batch, uint32_t n_slots, double* out,
                        void* stream) {
  NvtxRange nvtx("ckks_decrypt_decode");
  if (!c || !sk_of(sk, c) || n_slots > c->n / 2) return ZN_EINVAL;
  if (batch == 0 || n_slots == 0) return ZN_OK;
  if (!ct || !out) return ZN_EINVAL;
  DeviceGuard g(c->device);
  u64* coeffs = nullptr;
  double* work = nullptr;
  if (cudaMalloc(&coeffs, sizeof(u64) * batch * ring_words(c)) != cudaSuccess ||
      cudaMalloc(&work, sizeof(double) * batch * (size_t)c->n) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(coeffs);
    cudaFree(work);
    return ZN_ENOMEM;
  }
  int rc = ckks_decrypt(c, sk, ct, batch, coeffs, stream);
  if (!rc && zn::launch_decode(c->dp, coeffs, batch, n_slots, out, work, S(stream)) != cudaSuccess) rc = ZN_ECUDA;
  if (!rc && cudaStreamSynchronize(S(stream)) != cudaSuccess) rc = ZN_ECUDA;
  cudaGetLastError();
  cudaFree(coeffs);
  cudaFree(work);
  return rc;
}

int ckks_add(zn_ctx* c, const uint64_t* a, const uint64_t* b, uint32_t batch, uint64_t* out, void* stream) {
  if (!c) return ZN_EINVAL;
  if (batch == 0) return ZN_OK;
  if (!a || !b || !out) return ZN_EINVAL;
  DeviceGuard g(c->device);
  ZN_CUDA(zn::launch_add(c->dp, a, b, batch, out, S(stream)));
  return ZN_OK;
}

// ------------------------------------------------------------ batches

struct zn_batch {
  int device;
  int sms;
  int clusters;           // resident four-CTA clusters of the 2^15 kernel
  int pair_clusters;      // resident two-CTA clusters of the 2^14 kernel
  size_t prep_smem;       // dynamic shared memory of the persistent prep: 4N of the largest ring
  int prep_grid;          // its blocks: SMs x the blocks of that size that fit on an SM
  uint32_t n_prep, n_packets, n_small, n_mid;   // packets: [rings up to 2^13 | 2^14 | 2^15]
  zn::JobDesc* d_jobs;
  zn::PrepUnit* d_units;
  zn::EncPacket* d_packets;
  int* d_counters;        // [4]: prep, encrypt (up to 2^13), encrypt (2^14), encrypt (2^15)
  i64* d_me;
  int8_t* d_small;
  cudaGraphExec_t exec;
};

void zn_batch_destroy(zn_batch* b) {
  if (!b) return;
  DeviceGuard g(b->device);
  if (b->exec) released(cudaGraphExecDestroy(b->exec));
  released(cudaFree(b->d_jobs));
  released(cudaFree(b->d_units));
  released(cudaFree(b->d_packets));
  released(cudaFree(b->d_counters));
  released(cudaFree(b->d_me));
  released(cudaFree(b->d_small));
  delete b;
}

int zn_batch_create(const zn_job* jobs, uint32_t n_jobs, int device, zn_batch** out) {
  if (!jobs || !out || n_jobs == 0) return ZN_EINVAL;
  *out = nullptr;
  size_t me_words = 0, small_bytes = 0;
  for (uint32_t j = 0; j < n_jobs; ++j) {
    const zn_job& J = jobs[j];
    zn_ctx* c = J.ctx;
    if (!c || c->device != device || c->prm.log_n < 10 || c->prm.log_n > 15) return ZN_EINVAL;
    if (J.zinc ? !zc_of(J.zc, c) : !pk_of(J.pk, c)) return ZN_EINVAL;
    if (J.n_slots > c->n / 2) return ZN_EINVAL;
    if (J.count && (!J.ct || !J.ct_index || (J.n_slots && !J.slots))) return ZN_EINVAL;
    me_words += (size_t)J.count * c->n;
    small_bytes += 2 * (size_t)J.count * c->n;
  }
  DeviceGuard g(device);
  zn_batch* b = new (std::nothrow) zn_batch();
  if (!b) return ZN_ENOMEM;
  b->device = device;
  if (cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return ZN_ECUDA;
  }
  // descriptors, scratch offsets and work lists (largest rings first)
  std::vector<zn::JobDesc> desc(n_jobs);
  std::vector<uint32_t> order(n_jobs);
  for (uint32_t j = 0; j < n_jobs; ++j) order[j] = j;
  std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t c) {
    return jobs[a].ctx->prm.log_n > jobs[c].ctx->prm.log_n;
  });
  int rc = ZN_OK;
  if ((me_words && cudaMalloc(&b->d_me, sizeof(i64) * me_words) != cudaSuccess) ||
      (small_bytes && cudaMalloc(&b->d_small, small_bytes) != cudaSuccess) ||
      cudaMalloc(&b->d_counters, 4 * sizeof(int)) != cudaSuccess)
    rc = ZN_ENOMEM;
  std::vector<zn::PrepUnit> units;
  std::vector<zn::EncPacket> packets, mid, big;
  size_t me_off = 0, sm_off = 0;
  for (uint32_t j = 0; j < n_jobs && !rc; ++j) {
    const zn_job& J = jobs[j];
    zn_ctx* c = J.ctx;
    zn::JobDesc& D = desc[j];
    std::memset(&D, 0, sizeof(D));
    D.P = c->dp;
    D.zinc = J.zinc ? 1 : 0;
    D.E.key = J.zinc ? J.zc->d : J.pk->d;
    D.E.keys = J.zinc ? nullptr : J.pk->d + 2 * ring_words(c);
    D.E.me = b->d_me + me_off;
    D.E.small = b->d_small + sm_off;
    D.E.out = J.ct;
    D.Pr.slots = J.slots;
    D.Pr.n_slots = J.n_slots;
    D.Pr.ct_index = J.ct_index;
    D.Pr.ct_index0 = 0;
    D.Pr.seed = J.seed;
    D.Pr.domain = J.zinc ? 1u : 0u;
    D.Pr.me = b->d_me + me_off;
    D.Pr.small = b->d_small + sm_off;
    me_off += (size_t)J.count * c->n;
    sm_off += 2 * (size_t)J.count * c->n;
  }
  for (uint32_t oj = 0; oj < n_jobs && !rc; ++oj) {
    const uint32_t j = order[oj];
    const zn_job& J = jobs[j];
    const uint32_t log_n = J.ctx->prm.log_n, L = J.ctx->L;
    for (uint32_t k = 0; k < J.count; ++k) units.push_back({j, k});
    if (log_n == 15) {                 // one limb per four-CTA cluster
      for (uint32_t i = 0; i < L; ++i)
        for (uint32_t k = 0; k < J.count; ++k) big.push_back({j, k, (uint16_t)i, 1, 0});
    } else if (log_n == 14) {          // one limb per two-CTA cluster
      for (uint32_t i = 0; i < L; ++i)
        for (uint32_t k = 0; k < J.count; ++k) mid.push_back({j, k, (uint16_t)i, 1, 0});
    } else {                           // 2^(13 - log_n) limbs per 256-thread block
      const uint32_t per = 1u << (13 - log_n);
      for (uint32_t i = 0; i < L; ++i)
        for (uint32_t k = 0; k < J.count; k += per)
          packets.push_back({j, k, (uint16_t)i, (uint8_t)std::min(per, J.count - k), 0});
    }
  }
  b->n_prep = (uint32_t)units.size();
  b->n_small = (uint32_t)packets.size();
  b->n_mid = (uint32_t)mid.size();
  packets.insert(packets.end(), mid.begin(), mid.end());     // [small list | 2^14 list | 2^15 list]
  packets.insert(packets.end(), big.begin(), big.end());
  b->n_packets = (uint32_t)packets.size();
  if (!rc && (cudaMalloc(&b->d_jobs, sizeof(zn::JobDesc) * n_jobs) != cudaSuccess ||
              (b->n_prep && cudaMalloc(&b->d_units, sizeof(zn::PrepUnit) * b->n_prep) != cudaSuccess) ||
              (b->n_packets && cudaMalloc(&b->d_packets, sizeof(zn::EncPacket) * b->n_packets) != cudaSuccess)))
    rc = ZN_ENOMEM;
  if (!rc && (cudaMemcpy(b->d_jobs, desc.data(), sizeof(zn::JobDesc) * n_jobs, cudaMemcpyHostToDevice) != cudaSuccess ||
              (b->n_prep && cudaMemcpy(b->d_units, units.data(), sizeof(zn::PrepUnit) * b->n_prep,
                                       cudaMemcpyHostToDevice) != cudaSuccess) ||
              (b->n_packets && cudaMemcpy(b->d_packets, packets.data(), sizeof(zn::EncPacket) * b->n_packets,
                                          cudaMemcpyHostToDevice) != cudaSuccess) ||
              zn::batch_set_attributes() != cudaSuccess || zn::batch_quarter_clusters(&b->clusters) != cudaSuccess ||
              zn::batch_pair_clusters(&b->pair_clusters) != cudaSuccess))
    rc = ZN_ECUDA;
  if (!rc) {
    uint32_t max_n = 0;
    for (uint32_t j = 0; j < n_jobs; ++j) max_n = std::max(max_n, jobs[j].ctx->n);
    b->prep_smem = 4 * (size_t)max_n;
    int per_sm = 1;
    if (zn::batch_prep_blocks_per_sm(b->prep_smem, &per_sm) != cudaSuccess) rc = ZN_ECUDA;
    b->prep_grid = b->sms * per_sm;
  }
  if (rc) {
    cudaGetLastError();
    zn_batch_destroy(b);
    return rc;
  }
  *out = b;
  return ZN_OK;
}

static int batch_enqueue(zn_batch* b, cudaStream_t st) {
  ZN_CUDA(cudaMemsetAsync(b->d_counters, 0, 4 * sizeof(int), st));
  if (b->n_prep)
    ZN_CUDA(zn::launch_batch_prep(b->d_jobs, b->d_units, (int)b->n_prep, b->d_counters, b->prep_grid, b->prep_smem,
                                  st));
  if (b->n_small)
    ZN_CUDA(zn::launch_batch_encrypt(b->d_jobs, b->d_packets, (int)b->n_small, b->d_counters + 1, b->sms, st));
  if (b->n_mid)
    ZN_CUDA(zn::launch_batch_encrypt_pair(b->d_jobs, b->d_packets + b->n_small, (int)b->n_mid, b->d_counters + 2,
                                          b->pair_clusters, st));
  const uint32_t n_big = b->n_packets - b->n_small - b->n_mid;
  if (n_big)
    ZN_CUDA(zn::launch_batch_encrypt_quarter(b->d_jobs, b->d_packets + b->n_small + b->n_mid, (int)n_big,
                                             b->d_counters + 3, b->clusters, st));
  return ZN_OK;
}

int zn_batch_run(zn_batch* b, void* stream, int graph) {
  NvtxRange nvtx("zn_batch_run");
  if (!b) return ZN_EINVAL;
  DeviceGuard g(b->device);
  cudaStream_t st = S(stream);
  if (!graph) return batch_enqueue(b, st);
  if (!b->exec) {
    if (st == 0) return ZN_EINVAL;   // capture needs a non-default stream
    cudaGraph_t gr = nullptr;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      return ZN_ECUDA;
    }
    const int rc = batch_enqueue(b, st);
    const cudaError_t e = cudaStreamEndCapture(st, &gr);
    if (rc || e != cudaSuccess || cudaGraphInstantiate(&b->exec, gr, 0) != cudaSuccess) {
      if (gr) cudaGraphDestroy(gr);
      b->exec = nullptr;
      cudaGetLastError();
      return rc ? rc : ZN_ECUDA;
    }
    cudaGraphDestroy(gr);
  }
  ZN_CUDA(cudaGraphLaunch(b->exec, st));
  return ZN_OK;
}

int zn_batch_info(const zn_batch* b, uint32_t* prep_units, uint32_t* packets) {
  if (!b) return ZN_EINVAL;
  if (prep_units) *prep_units = b->n_prep;
  if (packets) *packets = b->n_packets;
  return ZN_OK;
}

// ------------------------------------------------------ host-buffer pipeline

namespace {

// Packing layout of a context's ciphertexts (see zn_pack.cu).
zn::PackArgs pack_args(const zn_ctx* c) {
  zn::PackArgs A;
  std::memset(&A, 0, sizeof(A));
  u64 off = 0;
  for (uint32_t i = 0; i < c->L; ++i) {
    A.bits[i] = 64u - (unsigned)__builtin_clzll(c->q[i]);
    A.woff[i] = off;
    off += ((u64)c->n * A.bits[i] + 63) / 64;
  }
  A.cwords = off;
  return A;
}

// The pack kernels assume 17 <= bits_i <= 62 (at most five residues per word).
bool pack_ok(const zn_ctx* c) {
  const zn::PackArgs A = pack_args(c);
  for (uint32_t i = 0; i < c->L; ++i)
    if (A.bits[i] < 17 || A.bits[i] > 62) return false;
  return true;
}

// Default chunk of the host-buffer encryption: at most 256 ciphertexts and
// 512 MiB of ciphertext, and at most a quarter of the batch (but not below
// 8), so that the first chunk's encryption -- the one part of the call that
// no copy overlaps -- stays short next to the link-bound copies.
uint32_t host_chunk(const zn_ctx* c, uint32_t batch) {
  size_t k = ((size_t)512 << 20) / (sizeof(u64) * 2 * ring_words(c));
  if (k > 256) k = 256;
  const size_t quarter = std::max<size_t>(8, ((size_t)batch + 3) / 4);
  if (k > quarter) k = quarter;
  return (uint32_t)std::max<size_t>(1, k);
}

// The host-buffer encryption; packed: each chunk is packed on the device and
// only the packed words cross the host link.
int encrypt_host_impl(zn_ctx* c, const zn_pk* pk, const zn_zcache* zc, const double* host_slots, uint32_t n_slots,
                      uint32_t batch, uint64_t seed, const uint64_t* host_ct_index, uint64_t* host_out,
                      uint32_t chunk, bool packed) {
  if (!c || (pk && zc) || (!pk && !zc) || (pk && !pk_of(pk, c)) || (zc && !zc_of(zc, c)) || n_slots > c->n / 2)
    return ZN_EINVAL;
  if (batch == 0) return ZN_OK;
  if (!host_out || !host_ct_index || (n_slots && !host_slots) || (packed && !pack_ok(c))) return ZN_EINVAL;
  if (chunk == 0) chunk = host_chunk(c, batch);
  if (chunk > batch) chunk = batch;
  DeviceGuard g(c->device);
  for (cudaStream_t& h : c->hs)
    if (!h && cudaStreamCreateWithFlags(&h, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      h = nullptr;
      return ZN_ECUDA;
    }
  if (packed && !c->hp) {
    // the packing kernels run on a stream of the highest priority: a chunk's
    // pack (and so its copy) must not wait behind the next chunk's encryption
    // blocks, which would otherwise take every SM first
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess ||
        cudaStreamCreateWithPriority(&c->hp, cudaStreamNonBlocking, greatest) != cudaSuccess) {
      cudaGetLastError();
      c->hp = nullptr;
      return ZN_ECUDA;
    }
    for (cudaEvent_t& e : c->hev)
      if (!e && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        e = nullptr;
        return ZN_ECUDA;
      }
  }
  const size_t ct_b = sizeof(u64) * 2 * ring_words(c) * chunk;
  const size_t sl_b = (sizeof(double) * n_slots * chunk + 255) / 256 * 256;
  const size_t ix_b = (sizeof(u64) * chunk + 255) / 256 * 256;
  // each stream also owns its encryption scratch for the whole call, so that
  // no per-chunk pool allocation can make one stream wait for another's frees
  const uint32_t ech = chunk < encode_chunk(c) ? chunk : encode_chunk(c);
  const size_t en_b = (encrypt_scratch_bytes(c, ech) + 255) / 256 * 256;
  zn::PackArgs pa = pack_args(c);
  const size_t out_words = packed ? 2 * pa.cwords : 2 * ring_words(c);   // per ciphertext
  const size_t pk_b = packed ? sizeof(u64) * out_words * chunk : 0;
  const bool zinc = zc != nullptr;
  int rc = ZN_OK;
  {
    Scratch st0(c, c->hs[0]), st1(c, c->hs[1]), st2(c, c->hs[2]);
    Scratch* stage[3] = {&st0, &st1, &st2};
    for (int k = 0; k < 3 && !rc; ++k)
      if (!stage[k]->alloc(ct_b + sl_b + ix_b + en_b + pk_b)) rc = ZN_ENOMEM;
    for (uint32_t b0 = 0, k = 0; b0 < batch && !rc; b0 += chunk, k = (k + 1) % 3) {
      const uint32_t nb = (batch - b0) < chunk ? (batch - b0) : chunk;
      cudaStream_t st = c->hs[k];
      char* base = (char*)stage[k]->p;
      u64* d_ct = (u64*)base;
      double* d_sl = (double*)(base + ct_b);
      u64* d_ix = (u64*)(base + ct_b + sl_b);
      i64* d_me = (i64*)(base + ct_b + sl_b + ix_b);
      int8_t* d_small = (int8_t*)d_me + sizeof(i64) * ech * (size_t)c->n;
      u64* d_out = packed ? (u64*)(base + ct_b + sl_b + ix_b + en_b) : d_ct;
      if ((n_slots && cudaMemcpyAsync(d_sl, host_slots + (size_t)b0 * n_slots, sizeof(double) * n_slots * nb,
                                      cudaMemcpyHostToDevice, st) != cudaSuccess) ||
          cudaMemcpyAsync(d_ix, host_ct_index + b0, sizeof(u64) * nb, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        rc = ZN_ECUDA;
        break;
      }
      rc = zinc ? encrypt_with(c, true, zc->d, nullptr, d_sl, n_slots, nb, seed, d_ix, d_ct, d_me, d_small, ech, st)
                : encrypt_with(c, false, pk->d, pk->d + 2 * ring_words(c), d_sl, n_slots, nb, seed, d_ix, d_ct, d_me,
                               d_small, ech, st);
      if (!rc && packed) {
        pa.ct = d_ct;
        pa.packed = d_out;
        if (cudaEventRecord(c->hev[k], st) != cudaSuccess || cudaStreamWaitEvent(c->hp, c->hev[k], 0) != cudaSuccess ||
            zn::launch_ct_pack(c->dp, pa, nb, c->hp) != cudaSuccess ||
            cudaEventRecord(c->hev[3 + k], c->hp) != cudaSuccess || cudaStreamWaitEvent(st, c->hev[3 + k], 0) != cudaSuccess) {
          cudaGetLastError();
          rc = ZN_ECUDA;
        }
      }
      if (!rc && cudaMemcpyAsync(host_out + (size_t)b0 * out_words, d_out, sizeof(u64) * out_words * nb,
                                 cudaMemcpyDeviceToHost, st) != cudaSuccess)
        rc = ZN_ECUDA;
    }
    // staging is returned to the pool in stream order by the Scratch destructors
  }
  for (cudaStream_t h : c->hs)
    if (cudaStreamSynchronize(h) != cudaSuccess) rc = rc ? rc : ZN_ECUDA;
  if (c->hp && cudaStreamSynchronize(c->hp) != cudaSuccess) rc = rc ? rc : ZN_ECUDA;
  cudaGetLastError();
  return rc;
}

}  // namespace

int zn_encrypt_host(zn_ctx* c, const zn_pk* pk, const zn_zcache* zc, const double* host_slots, uint32_t n_slots,
                    uint32_t batch, uint64_t seed, const uint64_t* host_ct_index, uint64_t* host_ct,
                    uint32_t chunk) {
  NvtxRange nvtx("zn_encrypt_host");
  return encrypt_host_impl(c, pk, zc, host_slots, n_slots, batch, seed, host_ct_index, host_ct, chunk, false);
}

int zn_encrypt_host_packed(zn_ctx* c, const zn_pk* pk, const zn_zcache* zc, const double* host_slots,
                           uint32_t n_slots, uint32_t batch, uint64_t seed, const uint64_t* host_ct_index,
                           uint64_t* host_packed, uint32_t chunk) {
  NvtxRange nvtx("zn_encrypt_host_packed");
  return encrypt_host_impl(c, pk, zc, host_slots, n_slots, batch, seed, host_ct_index, host_packed, chunk, true);
}

size_t zn_ct_packed_words(const zn_ctx* c) { return c ? 2 * pack_args(c).cwords : 0; }

int zn_ct_pack(zn_ctx* c, const uint64_t* ct, size_t batch, uint64_t* packed, void* stream) {
  NvtxRange nvtx("zn_ct_pack");
  if (!c || batch > 0xffffffffu || !pack_ok(c)) return ZN_EINVAL;
  if (batch == 0) return ZN_OK;
  if (!ct || !packed) return ZN_EINVAL;
  DeviceGuard g(c->device);
  zn::PackArgs A = pack_args(c);
  A.ct = const_cast<u64*>(ct);
  A.packed = packed;
  ZN_CUDA(zn::launch_ct_pack(c->dp, A, (uint32_t)batch, S(stream)));
  return ZN_OK;
}

int zn_ct_unpack(zn_ctx* c, const uint64_t* packed, size_t batch, uint64_t* ct, void* stream) {
  NvtxRange nvtx("zn_ct_unpack");
  if (!c || batch > 0xffffffffu || !pack_ok(c)) return ZN_EINVAL;
  if (batch == 0) return ZN_OK;
  if (!ct || !packed) return ZN_EINVAL;
  DeviceGuard g(c->device);
  zn::PackArgs A = pack_args(c);
  A.ct = ct;
  A.packed = const_cast<u64*>(packed);
  ZN_CUDA(zn::launch_ct_unpack(c->dp, A, (uint32_t)batch, S(stream)));
  return ZN_OK;
}

// ------------------------------------------------------------- autotuning

int zn_set_variant(zn_ctx* c, int variant) {
  if (!c || variant < 0 || variant >= ZN_VARIANTS) return ZN_EINVAL;
  c->variant = variant;
  return ZN_OK;
}

int zn_get_variant(const zn_ctx* c) { return c ? c->variant : ZN_EINVAL; }

int zn_autotune(zn_ctx* c, const zn_pk* pk, const zn_zcache* zc, uint32_t batch, float* ms, int* chosen) {
  NvtxRange nvtx("zn_autotune");
  if (!c || !pk_of(pk, c) || !zc_of(zc, c) || batch == 0) return ZN_EINVAL;
  DeviceGuard g(c->device);
  u64* ct = nullptr;
  u64* idx = nullptr;
  if (cudaMalloc(&ct, sizeof(u64) * 2 * ring_words(c) * batch) != cudaSuccess ||
      cudaMalloc(&idx, sizeof(u64) * batch) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(ct);
    return ZN_ENOMEM;
  }
  int rc = cudaMemset(idx, 0, sizeof(u64) * batch) == cudaSuccess ? ZN_OK : ZN_ECUDA;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (!rc && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) rc = ZN_ECUDA;
  const int saved = c->variant;
  const bool saved_timing = c->timing;
  c->timing = false;
  int best = saved;
  float best_ms = 0.f;
  for (int v = 0; v < ZN_VARIANTS && !rc; ++v) {
    c->variant = v;
    float t = 0.f;
    for (int rep = 0; rep < 3 && !rc; ++rep) {   // first repetition warms up
      if (cudaEventRecord(e0, 0) != cudaSuccess) rc = ZN_ECUDA;
      if (!rc) rc = encrypt_common(c, false, pk->d, pk->d + 2 * ring_words(c), nullptr, 0, batch, 1, idx, ct, 0);
      if (!rc) rc = encrypt_common(c, true, zc->d, nullptr, nullptr, 0, batch, 1, idx, ct, 0);
      if (!rc && (cudaEventRecord(e1, 0) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                  cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
        rc = ZN_ECUDA;
    }
    if (rc) break;
    if (ms) ms[v] = t;
    if (v == 0 || t < best_ms) {
      best = v;
      best_ms = t;
    }
  }
  c->variant = rc ? saved : best;
  c->timing = saved_timing;
  if (chosen) *chosen = c->variant;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(ct);
  cudaFree(idx);
  cudaGetLastError();
  return rc;
}

int zn_probe_butterfly(int device, double* per_s) {
  if (!per_s) return ZN_EINVAL;
  DeviceGuard g(device);
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    cudaGetLastError();
    return ZN_ECUDA;
  }
  return zn::probe_butterfly(sms, per_s, false) == cudaSuccess ? ZN_OK : ZN_ECUDA;
}

int zn_probe_butterfly_relaxed(int device, double* per_s) {
  if (!per_s) return ZN_EINVAL;
  DeviceGuard g(device);
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    cudaGetLastError();
    return ZN_ECUDA;
  }
  return zn::probe_butterfly(sms, per_s, true) == cudaSuccess ? ZN_OK : ZN_ECUDA;
}

int zn_probe_wait_timeout(zn_ctx* c, uint32_t tries, void* stream) {
  if (!c || tries == 0 || tries > (1u << 20)) return ZN_EINVAL;
  DeviceGuard g(c->device);
  ZN_CUDA(zn::launch_wait_probe(c->dp, tries, S(stream)));
  return ZN_OK;
}

int zn_inject_alloc_failures(int count) {
  if (count < 0) return ZN_EINVAL;
  g_alloc_faults.store(count, std::memory_order_relaxed);
  return ZN_OK;
}

// ------------------------------------------------------------ building blocks

int zn_ntt_forward(zn_ctx* c, uint64_t* data, uint32_t batch, void* stream) {
  if (!c) return ZN_EINVAL;
  if (batch == 0) return ZN_OK;
  if (!data) return ZN_EINVAL;
  DeviceGuard g(c->device);
  u64* tmp = nullptr;
  if (c->prm.log_n > 14) {
    if (cudaMalloc(&tmp, sizeof(u64) * batch * ring_words(c)) != cudaSuccess) {
      cudaGetLastError();
      return ZN_ENOMEM;
    }
  }
  int rc = zn::launch_ntt_fwd(c->dp, data, batch, tmp, S(stream)) == cudaSuccess ? ZN_OK : ZN_ECUDA;
  if (tmp) {
    if (cudaStreamSynchronize(S(stream)) != cudaSuccess) rc = ZN_ECUDA;
    cudaFree(tmp);
  }
  cudaGetLastError();
  return rc;
}

int zn_ntt_inverse(zn_ctx* c, uint64_t* data, uint32_t batch, void* stream) {
  if (!c) return ZN_EINVAL;
  if (batch == 0) return ZN_OK;
  if (!data) return ZN_EINVAL;
  DeviceGuard g(c->device);
  ZN_CUDA(zn::launch_ntt_inv(c->dp, data, batch, S(stream)));
  return ZN_OK;
}

int zn_sample(zn_ctx* c, int kind, uint64_t seed, uint32_t domain, uint32_t poly, uint32_t prime, uint64_t ct_index0,
              uint32_t count, int64_t* out, void* stream) {
  if (!c || kind < 0 || kind > 2 || domain > 255 || poly > 255 || prime >= c->L) return ZN_EINVAL;
  if (count == 0) return ZN_OK;
  if (!out) return ZN_EINVAL;
  DeviceGuard g(c->device);
  ZN_CUDA(zn::launch_sample(c->dp, kind, seed, domain, poly, prime, ct_index0, count, (i64*)out, S(stream)));
  return ZN_OK;
}

int zn_chi_eval(zn_ctx* c, const uint64_t* u, uint32_t n, int32_t* out, void* stream) {
  if (!c) return ZN_EINVAL;
  if (n == 0) return ZN_OK;
  if (!u || !out) return ZN_EINVAL;
  DeviceGuard g(c->device);
  ZN_CUDA(zn::launch_chi_eval(c->dp, u, n, out, S(stream)));
  return ZN_OK;
}

// ------------------------------------------- allocation-free Zinc encryption

}  // extern "C"

// The fixed scratch of zinc_encrypt_noalloc.  In host code this name is only
// a stand-in for the device array: kernels receive the address returned by
// cudaGetSymbolAddress for the current device.
static __device__ __align__(256) unsigned char zn_noalloc_scratch[ZN_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices];   // device address of the array, per device (set up once)

// With `device` current: the array's device address, looked up on first use.
int noalloc_scratch(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) return ZN_EINVAL;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[device]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, zn_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return ZN_ECUDA;
    }
    g_noalloc_ptr[device] = p;
  }
  *out = g_noalloc_ptr[device];
  return ZN_OK;
}
}  // namespace

extern "C" int zinc_encrypt_noalloc(zn_ctx* c, const zn_zcache* z, const double* slots, uint32_t n_slots,
                                    uint32_t batch, uint64_t seed, const uint64_t* ct_index, uint64_t* ct,
                                    void* stream) {
  NvtxRange nvtx("zinc_encrypt_noalloc");
  if (!c || !zc_of(z, c) || n_slots > c->n / 2) return ZN_EINVAL;
  if (batch == 0) return ZN_OK;
  if (!ct || !ct_index || (n_slots && !slots)) return ZN_EINVAL;
  const size_t n = c->n;
  const size_t me_b = ((size_t)batch * 8 * n + 255) / 256 * 256;
  const size_t sm_b = ((size_t)batch * 2 * n + 255) / 256 * 256;
  if (me_b + sm_b > ZN_NOALLOC_SCRATCH_BYTES) return ZN_ELIMIT;
  DeviceGuard g(c->device);
  unsigned char* base = nullptr;
  int rc = noalloc_scratch(c->device, (void**)&base);
  if (rc) return rc;
  zn::PrepArgs pa;
  pa.slots = slots;
  pa.n_slots = n_slots;
  pa.ct_index = ct_index;
  pa.ct_index0 = 0;
  pa.seed = seed;
  pa.domain = 1;                                   // Zinc randomiser
  pa.me = (i64*)base;
  pa.small = (int8_t*)(base + me_b);
  zn::EncArgs A;
  A.swap = 0;
  A.key = z->d;
  A.keys = nullptr;
  A.me = pa.me;
  A.small = pa.small;
  A.out = ct;
  {
    TimedLaunch t(c, ZN_TIME_ENCODE, S(stream));
    ZN_CUDA(zn::launch_prep(c->dp, pa, true, batch, S(stream)));
  }
  TimedLaunch t(c, ZN_TIME_ZINC, S(stream));
  ZN_CUDA(zn::launch_encrypt(c->dp, A, true, batch, c->variant, S(stream)));
  return ZN_OK;
}
