// Modulus-switched vanilla encryption: SEAL's ordering of CKKS public-key
// encryption, which the paper's measurements ran (Section "System
// Implementation"; the cost analysis of Section "Theoretical Analysis").
// The key-level chain q_0..q_{L-1} ends in the special prime p = q_{L-1}:
//   c_j = pk_j u + e_j            over the whole chain (Eq. 8 without m),
//   c'_j = floor((c_j + h) / p)   h = floor(p/2), at the data level,
//   c'_0 += m.
// Per data prime q_i the division is (c_{j,i} + h - r_j) p^-1 with
// r_j = (c_{j,p} + h) mod p.  Writing d_j = e_j + h - r_j (an exact integer,
// |d_j| <= p/2 + 19), everything but d_j is linear, so in NTT form
//   c'_0 = (pk0 p^-1) u^ + NTT(d_0 p^-1 + m),   c'_1 = (pk1 p^-1) u^ + NTT(d_1 p^-1)
// and a data prime runs three forward transforms, like the plain vanilla
// encryption; the special prime runs, per component, the forward transform of
// u, the key product and an inverse transform back to coefficients (r_j).
//
// Kernels: k_ms_special (one block per component and ciphertext; N = 2^15 as
// two half blocks plus k_ms_special_top), then the data primes in the launch
// shapes of the plain encryption's default kernels: k_encrypt_ms (radix 8,
// N <= 2^13), k_encrypt_ms_pair (two-CTA clusters, 2^14), k_encrypt_ms_quarter
// (four-CTA clusters, 2^15).
#include "zn_encrypt_fn.cuh"
#include "zn_pair.cuh"
#include "zn_quarter.cuh"

namespace zn {

// ------------------------------------------------------- inverse transform

// Gentleman-Sande butterfly, lazy: inputs and outputs in [0, 2q).
__device__ __forceinline__ void gs_bfly(u64& x, u64& y, u64 w, u64 ws, u64 q) {
  u64 s = x + y;
  if (s >= 2 * q) s -= 2 * q;
  y = mul_shoup(x - y + 2 * q, w, ws, q);
  x = s;
}

// One inverse pass over index bits [LO, LO+K), stages from distance 2^LO up:
// input in bit-reversed order (as the forward transform leaves it), output in
// natural order.  The twiddle of stage bit b for index idx is
// psi^-brv(tmul 2^(LOGN-1-b) + (idx >> (b+1))) -- the forward transform's
// index with the inverse table.  The last pass (LO + K = LOGN) hands every
// output to store(idx, x), x in [0, q).  The pass decomposition (bit sets)
// is the forward chain's, so the swizzle keeps it free of bank conflicts.
template <int LOGN, int LOGPER, int LO, int K, class Store, int KM>
__device__ __forceinline__ void intt_pass(u64* sm, int t, const u64* __restrict__ itw, const u64* __restrict__ itws,
                                          int tmul, u64 q, Store& store) {
  using S = NttShape<LOGN, LOGPER>;
  constexpr int G = S::PER >> K;
#pragma unroll 1
  for (int j = 0; j < G; ++j) {
    const int g = t + j * S::T;
    const int ghi = g >> LO;
    const int base = (g & ((1 << LO) - 1)) | (ghi << (LO + K));
    const int sb = swz<LOGN, KM>(base);
    u64 v[1 << K];
#pragma unroll
    for (int r = 0; r < (1 << K); ++r) v[r] = sm[sb ^ swz<LOGN, KM>(r << LO)];
#pragma unroll
    for (int s = 0; s < K; ++s) {
      const int tb = (tmul << (LOGN - 1 - LO - s)) + (ghi << (K - s - 1));
#pragma unroll
      for (int r = 0; r < (1 << K); ++r) {
        if (r & (1 << s)) continue;
        const int ti = tb + (r >> (s + 1));
        gs_bfly(v[r], v[r + (1 << s)], __ldg(itw + ti), __ldg(itws + ti), q);
      }
    }
    if constexpr (LO + K == LOGN) {
#pragma unroll
      for (int r = 0; r < (1 << K); ++r) store(base | (r << LO), v[r] >= q ? v[r] - q : v[r]);
    } else {
#pragma unroll
      for (int r = 0; r < (1 << K); ++r) sm[sb ^ swz<LOGN, KM>(r << LO)] = v[r];
    }
  }
}

// Inverse passes over bits [0, HI) from the bottom up, in the forward chain's
// bit sets; no final N^-1 scaling (the callers fold it into a product).
// Begins each pass with a barrier.
template <int LOGN, int LOGPER, int HI, class Store, int KM = NttShape<LOGN>::KMAX>
__device__ __forceinline__ void intt_chain(u64* sm, int t, const u64* itw, const u64* itws, int tmul, u64 q,
                                           Store& store) {
  constexpr int K = HI < KM ? HI : KM;
  constexpr int LO = HI - K;
  if constexpr (LO > 0) intt_chain<LOGN, LOGPER, LO, Store, KM>(sm, t, itw, itws, tmul, q, store);
  __syncthreads();
  intt_pass<LOGN, LOGPER, LO, K, Store, KM>(sm, t, itw, itws, tmul, q, store);
}

// ------------------------------------------------------ the special prime
// D_j[k] = d_j[k] + 2^62, d_j[k] = e_j[k] + h - r, r = (c + e_j[k] + h) mod p
// for c = (pk_j u)_p[k] in [0, p); |d_j| <= p/2 + 19 < 2^61.
__device__ __forceinline__ u64 ms_digit(u64 c, int e, u64 p) {
  const u64 h = p >> 1;
  u64 x = c + small_res(e, p);
  if (x >= p) x -= p;
  u64 r = x + h;
  if (r >= p) r -= p;
  return kMsOffset + (u64)((i64)e + (i64)h - (i64)r);
}

// Component j of ciphertext b, N = 2^LOGN <= 2^14: u -> NTT -> times
// pk_{j,p} N^-1 (in place, in shared memory) -> inverse transform -> d_j.
template <int LOGN>
__global__ void __launch_bounds__(NttShape<LOGN, 5>::T) k_ms_special(DevParams P, MsArgs A) {
  extern __shared__ u64 sm[];
  using S = NttShape<LOGN, 5>;
  constexpr int N = S::N;
  const int j = blockIdx.x;
  const size_t b = blockIdx.y;
  const int ip = P.L - 1;
  const u64 p = P.q[ip];
  const int t = threadIdx.x;
  const int8_t* sp = A.small + b * 3 * N;
  const u64* kn = A.keyn + (size_t)j * N;
  const u64* kns = kn + 2 * (size_t)N;
  gen_i8<LOGN>(sm, t, S::T, sp, p);
  auto st_u = [&](int idx, u64 uh) { sm[swz<LOGN>(idx)] = mul_shoup(uh, __ldg(kn + idx), __ldg(kns + idx), p); };
  ntt_chain<LOGN, 5, LOGN, false, decltype(st_u)>(sm, t, P.twp + (size_t)ip * N, 1, p, st_u);
  const int8_t* e = sp + (size_t)(1 + j) * N;
  u64* d = A.d + (b * 2 + j) * N;
  auto st_c = [&](int idx, u64 c) { d[idx] = ms_digit(c, __ldg(e + idx), p); };
  intt_chain<LOGN, 5, LOGN, decltype(st_c)>(sm, t, P.itw + (size_t)ip * N, P.itws + (size_t)ip * N, 1, p, st_c);
}

// N = 2^15: block (j, h) runs the forward transform's output half h (the
// generator applies the first stage), the key product, and the inverse
// stages below the top one on that half (they never cross halves), writing
// the half to tmp; k_ms_special_top applies the top inverse stage.
template <int LOGH>
__global__ void __launch_bounds__(NttShape<LOGH, 5>::T) k_ms_special_half(DevParams P, MsArgs A) {
  extern __shared__ u64 sm[];
  using S = NttShape<LOGH, 5>;
  constexpr int HALF = S::N, N = 2 * HALF;
  const int j = blockIdx.x >> 1, h = blockIdx.x & 1;
  const size_t b = blockIdx.y;
  const int ip = P.L - 1;
  const u64 p = P.q[ip];
  const int t = threadIdx.x;
  const ulonglong2* tw = P.twp + (size_t)ip * N;
  const ulonglong2 w1 = __ldg(tw + 1);
  const int8_t* sp = A.small + b * 3 * N;
  const u64* kn = A.keyn + (size_t)j * N + (size_t)h * HALF;
  const u64* kns = kn + 2 * (size_t)N;
  gen_i8_half<LOGH, 4, true>(sm, t, S::T, h, sp, p, w1.x, w1.y);
  auto st_u = [&](int idx, u64 uh) { sm[swz<LOGH>(idx)] = mul_shoup(uh, __ldg(kn + idx), __ldg(kns + idx), p); };
  ntt_chain<LOGH, 5, LOGH, false, decltype(st_u)>(sm, t, tw, 2 + h, p, st_u);
  u64* o = A.tmp + (b * 2 + j) * N + (size_t)h * HALF;
  auto st_c = [&](int idx, u64 c) { o[idx] = c; };
  intt_chain<LOGH, 5, LOGH, decltype(st_c)>(sm, t, P.itw + (size_t)ip * N, P.itws + (size_t)ip * N, 2 + h, p, st_c);
}

// Top inverse stage (distance N/2, twiddle psi^-brv(1)) on the two halves,
// then d_j for both outputs of each pair.
__global__ void k_ms_special_top(DevParams P, MsArgs A, uint32_t batch) {
  const int N = 1 << P.log_n, HALF = N >> 1;
  const int ip = P.L - 1;
  const u64 p = P.q[ip];
  const u64 w = __ldg(P.itw + (size_t)ip * N + 1), ws = __ldg(P.itws + (size_t)ip * N + 1);
  const size_t total = (size_t)batch * 2 * HALF;
  for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < total; x += (size_t)gridDim.x * blockDim.x) {
    const size_t bj = x / HALF;
    const int k = (int)(x % HALF);
    const u64* src = A.tmp + bj * N;
    u64 a = src[k], c = src[k + HALF];
    gs_bfly(a, c, w, ws, p);
    a = a >= p ? a - p : a;
    c = c >= p ? c - p : c;
    const size_t b = bj >> 1;
    const int j = (int)(bj & 1);
    const int8_t* e = A.small + b * 3 * N + (size_t)(1 + j) * N;
    u64* d = A.d + bj * N;
    d[k] = ms_digit(a, __ldg(e + k), p);
    d[k + HALF] = ms_digit(c, __ldg(e + k + HALF), p);
  }
}

// The data prime's transform inputs, in [0, 2q):
//   first component   d_0 p^-1 + m = D_0 p^-1 + M + kc0   (mod q)
//   second component  d_1 p^-1     = D_1 p^-1 + kc1       (mod q)
// with D_j p^-1 one Shoup product (any 64-bit input, result in [0, 2q)) and
// M one Barrett step (floor(2^64/q) = mu; result in [0, 2q)).
struct MsVal {
  const u64* d;
  const u64* m;   // nullptr: second component
  u64 q, mu, pv, pvs, kc;
  __device__ __forceinline__ u64 operator()(int k) const {
    u64 x = mul_shoup(__ldg(d + k), pv, pvs, q) + kc;         // [0, 3q)
    if (m) {
      const u64 a = __ldg(m + k);
      x += a - __umul64hi(a, mu) * q;                         // [0, 5q)
      if (x >= 4 * q) x -= 4 * q;
    }
    if (x >= 2 * q) x -= (m ? 2 : 1) * q;
    return x;
  }
};

// ------------------------------------------------------------ data primes
// Data prime i of ciphertext b: the vanilla-shaped generic unit with the
// p^-1-scaled keys and the MsVal inputs.
template <int LOGN, int LOGPER, bool RELAX, int KM>
__device__ __forceinline__ void ms_unit_q(const DevParams& P, const MsArgs& A, int i, size_t b, u64* sm, int t) {
  constexpr int N = 1 << LOGN;
  const int Ld = P.L - 1;
  const u64 q = P.q[i];
  FnLimb o;
  o.c0 = A.out + (b * 2 * Ld + i) * N;
  o.c1 = o.c0 + (size_t)Ld * N;
  o.k0 = A.keyms + (size_t)i * N;
  o.k1 = o.k0 + (size_t)Ld * N;
  o.k0s = o.k0 + 2 * (size_t)Ld * N;
  o.k1s = o.k1 + 2 * (size_t)Ld * N;
  o.u = A.small + b * 3 * N;
  const MsVal v0{A.d + b * 2 * N, A.m + b * N, q, P.mu[i], A.pinv[i], A.pinvs[i], A.kc0[i]};
  const MsVal v1{A.d + b * 2 * N + N, nullptr, q, P.mu[i], A.pinv[i], A.pinvs[i], A.kc1[i]};
  fn_unit_q<LOGN, LOGPER, RELAX, KM, false, true>(P.twp + (size_t)i * N, q, o, v0, v1, sm, t);
}

// grid (L-1, B), or (B, L-1) when A.swap
template <int LOGN, int LOGPER, int MINB, int KM>
__global__ void __launch_bounds__(NttShape<LOGN, LOGPER>::T, MINB) k_encrypt_ms(DevParams P, MsArgs A) {
  extern __shared__ u64 sm[];
  const int i = A.swap ? blockIdx.y : blockIdx.x;
  const size_t b = A.swap ? blockIdx.x : blockIdx.y;
  if constexpr (LOGN >= 10) {
    if (P.q[i] < kRelaxLimit) {
      ms_unit_q<LOGN, LOGPER, true, KM>(P, A, i, b, sm, threadIdx.x);
      return;
    }
  }
  ms_unit_q<LOGN, LOGPER, false, KM>(P, A, i, b, sm, threadIdx.x);
}

// N = 2^15: output quarter j of data prime i on a four-CTA cluster
// (zn_quarter.cuh), the vanilla-shaped unit with the MsVal inputs.
template <bool RELAX>
__device__ __forceinline__ void ms_quarter_unit_q(const DevParams& P, const MsArgs& A, int i, unsigned j, size_t b,
                                                  u64* sm, int t) {
  using namespace quarter;
  const int Ld = P.L - 1;
  const u64 q = P.q[i];
  const size_t off = (size_t)j * kQ;
  FnLimb o;
  o.c0 = A.out + (b * 2 * Ld + i) * kN + off;
  o.c1 = o.c0 + (size_t)Ld * kN;
  o.k0 = A.keyms + (size_t)i * kN + off;
  o.k1 = o.k0 + (size_t)Ld * kN;
  o.k0s = o.k0 + 2 * (size_t)Ld * kN;
  o.k1s = o.k1 + 2 * (size_t)Ld * kN;
  o.u = A.small + b * 3 * kN;
  const MsVal v0{A.d + b * 2 * kN, A.m + b * kN, q, P.mu[i], A.pinv[i], A.pinvs[i], A.kc0[i]};
  const MsVal v1{A.d + b * 2 * kN + kN, nullptr, q, P.mu[i], A.pinv[i], A.pinvs[i], A.kc1[i]};
  const ulonglong2* tw = P.twp + (size_t)i * kN;
  auto gu = [&] { gen_i8<RELAX, true>(sm, t, j, o.u, tw, q); };
  auto g0 = [&] { gen_val<RELAX>(sm, t, j, v0, tw, q); };
  auto g1 = [&] { gen_val<RELAX>(sm, t, j, v1, tw, q); };
  unit<false, RELAX>(sm, t, j, tw, q, o, gu, g0, g1);
}

// grid (4(L-1), B), or (4B, L-1) when A.swap; cluster rank j owns quarter j
__global__ void __launch_bounds__(quarter::kT, 3) k_encrypt_ms_quarter(DevParams P, MsArgs A) {
  extern __shared__ u64 sm[];
  const unsigned j = quarter::cluster_rank();
  const int i = A.swap ? (int)blockIdx.y : (int)(blockIdx.x >> 2);
  const size_t b = A.swap ? (size_t)(blockIdx.x >> 2) : blockIdx.y;
  if (P.q[i] < kRelaxLimit) ms_quarter_unit_q<true>(P, A, i, j, b, sm, threadIdx.x);
  else ms_quarter_unit_q<false>(P, A, i, j, b, sm, threadIdx.x);
}

// N = 2^14: output half h of data prime i on a two-CTA cluster
// (zn_pair.cuh), the vanilla-shaped unit with the MsVal inputs and streaming
// stores for the finished words.
template <bool RELAX>
__device__ __forceinline__ void ms_pair_unit_q(const DevParams& P, const MsArgs& A, int i, unsigned h, size_t b,
                                               u64* sm, int t) {
  using namespace pair;
  const int Ld = P.L - 1;
  const u64 q = P.q[i];
  const size_t off = (size_t)h * kH;
  FnLimb o;
  o.c0 = A.out + (b * 2 * Ld + i) * kN + off;
  o.c1 = o.c0 + (size_t)Ld * kN;
  o.k0 = A.keyms + (size_t)i * kN + off;
  o.k1 = o.k0 + (size_t)Ld * kN;
  o.k0s = o.k0 + 2 * (size_t)Ld * kN;
  o.k1s = o.k1 + 2 * (size_t)Ld * kN;
  o.u = A.small + b * 3 * kN;
  const MsVal v0{A.d + b * 2 * kN, A.m + b * kN, q, P.mu[i], A.pinv[i], A.pinvs[i], A.kc0[i]};
  const MsVal v1{A.d + b * 2 * kN + kN, nullptr, q, P.mu[i], A.pinv[i], A.pinvs[i], A.kc1[i]};
  const ulonglong2* tw = P.twp + (size_t)i * kN;
  auto gu = [&] { gen_i8<RELAX, true>(sm, t, h, o.u, tw, q); };
  auto g0 = [&] { gen_val<RELAX>(sm, t, h, v0, tw, q); };
  auto g1 = [&] { gen_val<RELAX>(sm, t, h, v1, tw, q); };
  unit<false, RELAX, true>(sm, t, h, tw, q, o, gu, g0, g1);
}

// grid (2(L-1), B), or (2B, L-1) when A.swap; cluster rank h owns half h
__global__ void __launch_bounds__(pair::kT, 3) k_encrypt_ms_pair(DevParams P, MsArgs A) {
  extern __shared__ u64 sm[];
  const unsigned h = cluster::cluster_rank();
  const int i = A.swap ? (int)blockIdx.y : (int)(blockIdx.x >> 1);
  const size_t b = A.swap ? (size_t)(blockIdx.x >> 1) : blockIdx.y;
  if (P.q[i] < kRelaxLimit) ms_pair_unit_q<true>(P, A, i, h, b, sm, threadIdx.x);
  else ms_pair_unit_q<false>(P, A, i, h, b, sm, threadIdx.x);
}

// ---------------------------------------------------------------- keys
// keyms[j][i][k] = pk_j[i][k] p^-1 mod q_i (i < L-1), keyn[j][k] = pk_j[L-1][k] N^-1 mod p,
// each followed by its Shoup companions.
__global__ void k_ms_keys(DevParams P, MsArgs A, const u64* __restrict__ pk, u64* keyms, u64* keyn) {
  const int N = 1 << P.log_n, L = P.L, Ld = L - 1;
  const size_t nms = (size_t)2 * Ld * N, total = nms + 2 * (size_t)N;
  for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < total; x += (size_t)gridDim.x * blockDim.x) {
    if (x < nms) {
      const int j = (int)(x / ((size_t)Ld * N));
      const size_t rem = x % ((size_t)Ld * N);
      const int i = (int)(rem / N);
      const u64 q = P.q[i];
      const u64 v = mulmod_slow(pk[(size_t)j * L * N + rem], A.pinv[i], q);
      keyms[x] = v;
      keyms[nms + x] = shoup_of(v, q);
    } else {
      const size_t y = x - nms;
      const int j = (int)(y / N), k = (int)(y % N);
      const u64 p = P.q[L - 1];
      const u64 v = mulmod_slow(pk[((size_t)j * L + L - 1) * N + k], P.ninv[L - 1], p);
      keyn[y] = v;
      keyn[2 * (size_t)N + y] = shoup_of(v, p);
    }
  }
}

// ------------------------------------------------------------- launchers

template <class K>
static cudaError_t set_smem(K kern, size_t bytes) {
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t launch_ms_keys(const DevParams& P, const MsArgs& A, const u64* pk, u64* keyms, u64* keyn,
                           cudaStream_t st) {
  const size_t total = ((size_t)2 * (P.L - 1) + 2) << P.log_n;
  size_t g = (total + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  k_ms_keys<<<(unsigned)g, 256, 0, st>>>(P, A, pk, keyms, keyn);
  return cudaGetLastError();
}

template <int LOGN>
static cudaError_t special_full(const DevParams& P, const MsArgs& A, uint32_t batch, cudaStream_t st) {
  using S = NttShape<LOGN, 5>;
  const size_t smem = sizeof(u64) * S::N;
  cudaError_t e = set_smem(k_ms_special<LOGN>, smem);
  if (e != cudaSuccess) return e;
  k_ms_special<LOGN><<<dim3(2, batch), S::T, smem, st>>>(P, A);
  return cudaGetLastError();
}

static cudaError_t special_halves(const DevParams& P, const MsArgs& A, uint32_t batch, cudaStream_t st) {
  using S = NttShape<14, 5>;
  const size_t smem = sizeof(u64) * S::N;
  cudaError_t e = set_smem(k_ms_special_half<14>, smem);
  if (e != cudaSuccess) return e;
  k_ms_special_half<14><<<dim3(4, batch), S::T, smem, st>>>(P, A);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const size_t total = (size_t)batch * 2 * (S::N);
  size_t g = (total + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  k_ms_special_top<<<(unsigned)g, 256, 0, st>>>(P, A, batch);
  return cudaGetLastError();
}

cudaError_t launch_ms_special(const DevParams& P, const MsArgs& A, uint32_t batch, cudaStream_t st) {
  if (batch == 0) return cudaSuccess;
  if (P.L < 2) return cudaErrorInvalidValue;
  switch (P.log_n) {
    case 4: return special_full<4>(P, A, batch, st);
    case 5: return special_full<5>(P, A, batch, st);
    case 6: return special_full<6>(P, A, batch, st);
    case 7: return special_full<7>(P, A, batch, st);
    case 8: return special_full<8>(P, A, batch, st);
    case 9: return special_full<9>(P, A, batch, st);
    case 10: return special_full<10>(P, A, batch, st);
    case 11: return special_full<11>(P, A, batch, st);
    case 12: return special_full<12>(P, A, batch, st);
    case 13: return special_full<13>(P, A, batch, st);
    case 14: return special_full<14>(P, A, batch, st);
    case 15: return special_halves(P, A, batch, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int LOGN, int LOGPER, int MINB, int KM>
static cudaError_t data_full(const DevParams& P, const MsArgs& A, uint32_t batch, cudaStream_t st) {
  using S = NttShape<LOGN, LOGPER>;
  const size_t smem = sizeof(u64) * S::N;
  auto kern = k_encrypt_ms<LOGN, LOGPER, MINB, KM>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  const dim3 grid = A.swap ? dim3(batch, P.L - 1) : dim3(P.L - 1, batch);
  kern<<<grid, S::T, smem, st>>>(P, A);
  return cudaGetLastError();
}

static cudaError_t data_pair(const DevParams& P, const MsArgs& A, uint32_t batch, cudaStream_t st) {
  if ((!A.swap && batch > 65535u) || (A.swap && 2ull * batch > 0x7fffffffull)) return cudaErrorInvalidValue;
  const dim3 grid = A.swap ? dim3(2 * batch, P.L - 1) : dim3(2 * (P.L - 1), batch);
  return pair::launch(k_encrypt_ms_pair, grid, st, P, A);
}

static cudaError_t data_quarter(const DevParams& P, const MsArgs& A, uint32_t batch, cudaStream_t st) {
  if ((!A.swap && batch > 65535u) || (A.swap && 4ull * batch > 0x7fffffffull)) return cudaErrorInvalidValue;
  const dim3 grid = A.swap ? dim3(4 * batch, P.L - 1) : dim3(4 * (P.L - 1), batch);
  return quarter::launch(k_encrypt_ms_quarter, grid, st, P, A);
}

// The plain encryption's default shapes: radix-8, three 256-thread blocks
// per SM for 2^10..2^13, one block per limb below, two-CTA clusters (one
// output half each) at 2^14, four-CTA clusters (one quarter each) at 2^15.
cudaError_t launch_ms_data(const DevParams& P, const MsArgs& A, uint32_t batch, cudaStream_t st) {
  if (batch == 0) return cudaSuccess;
  if (P.L < 2) return cudaErrorInvalidValue;
  switch (P.log_n) {
    case 4: return data_full<4, 5, 1, 4>(P, A, batch, st);
    case 5: return data_full<5, 5, 1, 4>(P, A, batch, st);
    case 6: return data_full<6, 5, 1, 4>(P, A, batch, st);
    case 7: return data_full<7, 5, 1, 4>(P, A, batch, st);
    case 8: return data_full<8, 5, 1, 4>(P, A, batch, st);
    case 9: return data_full<9, 5, 1, 4>(P, A, batch, st);
    case 10: return data_full<10, 5, 24, 3>(P, A, batch, st);
    case 11: return data_full<11, 5, 12, 3>(P, A, batch, st);
    case 12: return data_full<12, 5, 6, 3>(P, A, batch, st);
    case 13: return data_full<13, 5, 3, 3>(P, A, batch, st);
    case 14: return data_pair(P, A, batch, st);
    case 15: return data_quarter(P, A, batch, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace zn
