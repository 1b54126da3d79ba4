// Gen (Eq. 7), plain forward NTT and the sampler entry point.
#include "zn_kernels.h"

namespace zn {

struct KeyArgs {
  u64 seed;
  u64* sk_ntt;   // [L][N]
  u64* pk;       // [2][L][N]
  u64* pks;      // [2][L][N] Shoup companions
};

// One prime per block: s-hat, a-hat = pk1, pk0 = -a s + e (NTT domain),
// Shoup companions of both key polynomials.  Sampling domain 2, ct_index 0.
template <int LOGN>
__global__ void __launch_bounds__(NttShape<LOGN>::T) k_keygen(DevParams P, KeyArgs A) {
  using S = NttShape<LOGN>;
  extern __shared__ u64 sm[];
  const int i = blockIdx.x, L = P.L;
  const u64 q = P.q[i];
  const ulonglong2* tw = P.twp + (size_t)i * S::N;
  u64* sh = A.sk_ntt + (size_t)i * S::N;
  u64* p0 = A.pk + (size_t)i * S::N;
  u64* p1 = p0 + (size_t)L * S::N;
  u64* p0s = A.pks + (size_t)i * S::N;
  u64* p1s = p0s + (size_t)L * S::N;
  gen_ternary<LOGN>(sm, A.seed, rand_tag(2, 0, 0), 0, q);
  auto st_s = [&](int idx, u64 x) { sh[idx] = x; };
  ntt_forward<LOGN>(sm, tw, 1, q, st_s);
  __syncthreads();
  gen_uniform<LOGN>(sm, A.seed, rand_tag(2, 1, (unsigned)i), 0, q);
  auto st_a = [&](int idx, u64 x) {
    const u64 a = x;
    p1[idx] = a;
    p1s[idx] = shoup_of(a, q);
  };
  ntt_forward<LOGN>(sm, tw, 1, q, st_a);
  __syncthreads();
  gen_gauss<LOGN>(sm, A.seed, rand_tag(2, 2, 0), 0, P.cdt, nullptr, q, P.mu[i]);
  auto st_e = [&](int idx, u64 x) {
    const u64 e = x;
    const u64 as = mulmod_slow(p1[idx], sh[idx], q);
    const u64 pk0 = e >= as ? e - as : e + q - as;
    p0[idx] = pk0;
    p0s[idx] = shoup_of(pk0, q);
  };
  ntt_forward<LOGN>(sm, tw, 1, q, st_e);
}

template <int LOGH>
__global__ void __launch_bounds__(NttShape<LOGH>::T) k_keygen_half(DevParams P, KeyArgs A) {
  constexpr int N = 2 << LOGH, HALF = 1 << LOGH;
  extern __shared__ u64 sm[];
  const int i = blockIdx.x >> 1, h = blockIdx.x & 1, L = P.L;
  const u64 q = P.q[i];
  const ulonglong2* tw = P.twp + (size_t)i * N;
  const ulonglong2 w1p = __ldg(tw + 1);
  const u64 w1 = w1p.x, w1s = w1p.y;
  const size_t off = (size_t)h * HALF;
  u64* sh = A.sk_ntt + (size_t)i * N + off;
  u64* p0 = A.pk + (size_t)i * N + off;
  u64* p1 = p0 + (size_t)L * N;
  u64* p0s = A.pks + (size_t)i * N + off;
  u64* p1s = p0s + (size_t)L * N;
  const int tmul = 2 + h;
  gen_ternary_half<LOGH>(sm, h, A.seed, rand_tag(2, 0, 0), 0, q, w1, w1s);
  auto st_s = [&](int idx, u64 x) { sh[idx] = x; };
  ntt_forward<LOGH>(sm, tw, tmul, q, st_s);
  __syncthreads();
  gen_uniform_half<LOGH>(sm, h, A.seed, rand_tag(2, 1, (unsigned)i), 0, q, w1, w1s);
  auto st_a = [&](int idx, u64 x) {
    const u64 a = x;
    p1[idx] = a;
    p1s[idx] = shoup_of(a, q);
  };
  ntt_forward<LOGH>(sm, tw, tmul, q, st_a);
  __syncthreads();
  gen_gauss_half<LOGH>(sm, h, A.seed, rand_tag(2, 2, 0), 0, P.cdt, nullptr, q, P.mu[i], w1, w1s);
  auto st_e = [&](int idx, u64 x) {
    const u64 e = x;
    const u64 as = mulmod_slow(p1[idx], sh[idx], q);
    const u64 pk0 = e >= as ? e - as : e + q - as;
    p0[idx] = pk0;
    p0s[idx] = shoup_of(pk0, q);
  };
  ntt_forward<LOGH>(sm, tw, tmul, q, st_e);
}

// Out-of-place forward NTT of src [B][L][N] into dst (may alias for N <= 2^14).
template <int LOGN>
__global__ void __launch_bounds__(NttShape<LOGN>::T) k_ntt_fwd(DevParams P, const u64* src, u64* dst) {
  using S = NttShape<LOGN>;
  extern __shared__ u64 sm[];
  const int i = blockIdx.x;
  const u64 q = P.q[i];
  const size_t off = ((size_t)blockIdx.y * P.L + i) * S::N;
  gen_copy<LOGN>(sm, src + off);
  u64* o = dst + off;
  auto st = [&](int idx, u64 x) { o[idx] = x; };
  ntt_forward<LOGN>(sm, P.twp + (size_t)i * S::N, 1, q, st);
}

template <int LOGH>
__global__ void __launch_bounds__(NttShape<LOGH>::T) k_ntt_fwd_half(DevParams P, const u64* src, u64* dst) {
  constexpr int N = 2 << LOGH, HALF = 1 << LOGH;
  extern __shared__ u64 sm[];
  const int i = blockIdx.x >> 1, h = blockIdx.x & 1;
  const u64 q = P.q[i];
  const ulonglong2* tw = P.twp + (size_t)i * N;
  const ulonglong2 w1p = __ldg(tw + 1);
  const size_t off = ((size_t)blockIdx.y * P.L + i) * N;
  gen_copy_half<LOGH>(sm, h, src + off, q, w1p.x, w1p.y);
  u64* o = dst + off + (size_t)h * HALF;
  auto st = [&](int idx, u64 x) { o[idx] = x; };
  ntt_forward<LOGH>(sm, tw, 2 + h, q, st);
}

// Samples of one polynomial kind for `count` ciphertext indices.
__global__ void k_sample(DevParams P, int kind, u64 seed, unsigned domain, unsigned poly, unsigned prime,
                         u64 ct_index0, uint32_t count, i64* out) {
  const int N = 1 << P.log_n;
  const int per = kind == 0 ? N / 4 : kind == 1 ? N / 2 : N;   // Philox blocks per polynomial
  const size_t total = (size_t)count * per;
  const unsigned tag = rand_tag(domain, poly, prime);
  for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < total; x += (size_t)gridDim.x * blockDim.x) {
    const size_t c = x / per;
    const unsigned blk = (unsigned)(x % per);
    i64* o = out + c * N;
    const uint4 w = zn_rand(seed, blk, tag, ct_index0 + c);
    if (kind == 0) {
      o[blk] = ternary_of(w.x);
      o[blk + N / 4] = ternary_of(w.y);
      o[blk + N / 2] = ternary_of(w.z);
      o[blk + 3 * N / 4] = ternary_of(w.w);
    } else if (kind == 1) {
      o[blk] = cdt_of(w.x, w.y, P.cdt);
      o[blk + N / 2] = cdt_of(w.z, w.w, P.cdt);
    } else {
      o[blk] = (i64)uniform_of(w, P.q[prime]);
    }
  }
}

// chi's CDT step on given uniforms, by the bucket-indexed threshold lookup of
// the encryption path (a test hook for threshold boundaries).
__global__ void k_chi_eval(DevParams P, const u64* __restrict__ u, uint32_t n, int* __restrict__ out) {
  __shared__ CdtTab s_cdt;
  stage_cdt_tab(P.cdt, s_cdt);
  __syncthreads();
  for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < n; x += (size_t)gridDim.x * blockDim.x) {
    const u64 v = u[x];
    out[x] = cdt_lookup((unsigned)v, (unsigned)(v >> 32), s_cdt);
  }
}

// ---------------------------------------------------------------- launchers

template <class K>
static cudaError_t smem_attr(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int LOGN>
static cudaError_t keygen_full(const DevParams& P, const KeyArgs& A, cudaStream_t st) {
  using S = NttShape<LOGN>;
  const size_t smem = sizeof(u64) * S::N;
  cudaError_t e = smem_attr(k_keygen<LOGN>, smem);
  if (e != cudaSuccess) return e;
  k_keygen<LOGN><<<P.L, S::T, smem, st>>>(P, A);
  return cudaGetLastError();
}

cudaError_t launch_keygen(const DevParams& P, u64 seed, u64* sk_ntt, u64* pk, u64* pks, cudaStream_t st) {
  KeyArgs A{seed, sk_ntt, pk, pks};
  switch (P.log_n) {
    case 4: return keygen_full<4>(P, A, st);
    case 5: return keygen_full<5>(P, A, st);
    case 6: return keygen_full<6>(P, A, st);
    case 7: return keygen_full<7>(P, A, st);
    case 8: return keygen_full<8>(P, A, st);
    case 9: return keygen_full<9>(P, A, st);
    case 10: return keygen_full<10>(P, A, st);
    case 11: return keygen_full<11>(P, A, st);
    case 12: return keygen_full<12>(P, A, st);
    case 13: return keygen_full<13>(P, A, st);
    case 14: return keygen_full<14>(P, A, st);
    case 15: {
      using S = NttShape<14>;
      const size_t smem = sizeof(u64) * S::N;
      cudaError_t e = smem_attr(k_keygen_half<14>, smem);
      if (e != cudaSuccess) return e;
      k_keygen_half<14><<<2 * P.L, S::T, smem, st>>>(P, A);
      return cudaGetLastError();
    }
    default: return cudaErrorInvalidValue;
  }
}

template <int LOGN>
static cudaError_t ntt_full(const DevParams& P, const u64* src, u64* dst, uint32_t batch, cudaStream_t st) {
  using S = NttShape<LOGN>;
  const size_t smem = sizeof(u64) * S::N;
  cudaError_t e = smem_attr(k_ntt_fwd<LOGN>, smem);
  if (e != cudaSuccess) return e;
  k_ntt_fwd<LOGN><<<dim3(P.L, batch), S::T, smem, st>>>(P, src, dst);
  return cudaGetLastError();
}

// In place for N <= 2^14; for N = 2^15 (two blocks read each input) through tmp.
cudaError_t launch_ntt_fwd(const DevParams& P, u64* data, uint32_t batch, u64* tmp, cudaStream_t st) {
  if (batch == 0) return cudaSuccess;
  switch (P.log_n) {
    case 4: return ntt_full<4>(P, data, data, batch, st);
    case 5: return ntt_full<5>(P, data, data, batch, st);
    case 6: return ntt_full<6>(P, data, data, batch, st);
    case 7: return ntt_full<7>(P, data, data, batch, st);
    case 8: return ntt_full<8>(P, data, data, batch, st);
    case 9: return ntt_full<9>(P, data, data, batch, st);
    case 10: return ntt_full<10>(P, data, data, batch, st);
    case 11: return ntt_full<11>(P, data, data, batch, st);
    case 12: return ntt_full<12>(P, data, data, batch, st);
    case 13: return ntt_full<13>(P, data, data, batch, st);
    case 14: return ntt_full<14>(P, data, data, batch, st);
    case 15: {
      using S = NttShape<14>;
      const size_t smem = sizeof(u64) * S::N;
      cudaError_t e = smem_attr(k_ntt_fwd_half<14>, smem);
      if (e != cudaSuccess) return e;
      k_ntt_fwd_half<14><<<dim3(2 * P.L, batch), S::T, smem, st>>>(P, data, tmp);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
      return cudaMemcpyAsync(data, tmp, sizeof(u64) * ((size_t)batch * P.L << 15), cudaMemcpyDeviceToDevice, st);
    }
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_chi_eval(const DevParams& P, const u64* u, uint32_t n, int* out, cudaStream_t st) {
  size_t g = (n + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  if (g < 1) g = 1;
  k_chi_eval<<<(unsigned)g, 256, 0, st>>>(P, u, n, out);
  return cudaGetLastError();
}

cudaError_t launch_sample(const DevParams& P, int kind, u64 seed, unsigned domain, unsigned poly, unsigned prime,
                          u64 ct_index0, uint32_t count, i64* out, cudaStream_t st) {
  const size_t per = kind == 0 ? (1u << P.log_n) / 4 : kind == 1 ? (1u << P.log_n) / 2 : (1u << P.log_n);
  size_t g = (per * count + 255) / 256;
  if (g > 152 * 64) g = 152 * 64;
  if (g < 1) g = 1;
  k_sample<<<(unsigned)g, 256, 0, st>>>(P, kind, seed, domain, poly, prime, ct_index0, count, out);
  return cudaGetLastError();
}

}  // namespace zn
