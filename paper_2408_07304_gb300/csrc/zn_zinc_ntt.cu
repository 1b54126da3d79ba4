// Zinc with its error polynomials generated in the NTT domain: the
// further optimisation the paper's Conclusion names (random errors made
// directly in the Fourier space, no transform, O(N) encryption).  Reading
// (the paper gives no construction): a cached basis of K chi polynomials per
// component, E_{c,j} (NTT form), and per ciphertext uniform rotations
// r_{c,j} in [0, 2N):
//   e'_c = sum_j X^{r_{c,j}} E_{c,j},   c' = (z0 + m + e'_0, z1 + e'_1)
// over a plaintext m pre-encoded in NTT form (the paper's Construction
// assumes an encoded plaintext).  In NTT form X^r is the pointwise factor
// psi^((2 brv(i) + 1) r mod 2N) at output i, so a ciphertext costs per prime
// and coefficient 4K Shoup products -- no butterflies; the kernel
// streams the plaintext in and the ciphertext out (HBM) and reads the cache
// and the basis from L2.
#include "zn_kernels.h"

namespace zn {

// Montgomery product a b 2^-64 mod q, result in [0, 2q) when a b < q 2^64
// (qneg = -q^-1 mod 2^64).
__device__ __forceinline__ u64 mont_mul(u64 a, u64 b, u64 q, u64 qneg) {
  const u64 lo = a * b, hi = __umul64hi(a, b);
  const u64 m = lo * qneg;
  return hi + __umul64hi(m, q) + (lo != 0 ? 1ull : 0ull);
}

// One block of 256 threads per (prime, ciphertext).  Output i = t + 256 k is
// handled by thread t in trip k.  Per rotation (c, j) the block builds
//   flo[t] = psi^(2^(n-7) brv_8(t) r),   fhi[k] = psi^((2 brv_(n-8)(k) + 1) r)
// (mod q, from psi^(64 h) and psi^l), each with its Shoup companion, so that
// a basis value times its factor is two Shoup products; fhi[k] is read by
// the whole warp at once (broadcast), flo[t] by each thread at its own slot.
// K is a template parameter so that the term loop unrolls and each
// thread's flo entries stay in registers across its trips.
template <int K>
__global__ void __launch_bounds__(256, 4) k_zinc_ntt(DevParams P, NttZincArgs A) {
  extern __shared__ ulonglong2 s_tab[];   // [2][K][N/256] fhi, then [2][K][256] flo
  __shared__ unsigned s_r[32];            // [2][16]
  const int i = blockIdx.x;
  const size_t b = blockIdx.y;
  const int log_n = P.log_n, N = 1 << log_n, L = P.L, NK = N >> 8;
  const unsigned mask2n = 2u * N - 1;
  const u64 q = P.q[i], qn = A.qneg[i];
  const int t = threadIdx.x;
  if (t < 2 * K) {
    const int c = t / K, j = t % K;
    const uint4 w = zn_rand(A.seed, (unsigned)j, rand_tag(5, (unsigned)c, 0), A.ct_index[b]);
    s_r[c * 16 + j] = w.x & mask2n;
  }
  __syncthreads();
  const ulonglong2* fhi = s_tab;
  const ulonglong2* flo = s_tab + 2 * K * NK;
  const u64* thi = A.thi + (size_t)i * (N / 32);
  const u64* tlo = A.tlo + (size_t)i * 64;
  for (int x = t; x < 2 * K * (NK + 256); x += blockDim.x) {
    unsigned e;
    if (x < 2 * K * NK) {
      const int cj = x / NK, k = x % NK;
      const unsigned r = s_r[(cj / K) * 16 + cj % K];
      const unsigned bk = log_n > 8 ? __brev((unsigned)k) >> (40 - log_n) : 0u;
      e = ((2u * bk + 1u) * r) & mask2n;
    } else {
      const int y = x - 2 * K * NK, cj = y >> 8, tt = y & 255;
      const unsigned r = s_r[(cj / K) * 16 + cj % K];
      e = (((__brev((unsigned)tt) >> 24) << (log_n - 7)) * r) & mask2n;   // mod 2N: wraparound is harmless
    }
    u64 v = mont_mul(__ldg(thi + (e >> 6)), __ldg(tlo + (e & 63)), q, qn);   // psi^e, [0, 2q)
    v = v >= q ? v - q : v;
    s_tab[x] = make_ulonglong2(v, shoup_of(v, q));
  }
  __syncthreads();
  const u64* z0 = A.z + (size_t)i * N;
  const u64* z1 = z0 + (size_t)L * N;
  const u64* m = A.m + (b * L + i) * N;
  u64* c0 = A.out + (b * 2 * L + i) * N;
  u64* c1 = c0 + (size_t)L * N;
  const size_t estride = (size_t)L * N;          // between basis polynomials of one prime
  const u64* E0 = A.E + (size_t)i * N + t;       // E_{0,0} at prime i, this thread's column
  const u64* E1 = E0 + (size_t)K * estride;      // E_{1,0}
  constexpr bool REG = K <= 4;                   // flo in registers (no spills up to K = 4)
  constexpr int UNJ = REG ? K : 1;               // term loop unrolled only then
  constexpr int UNK = K == 1 ? 4 : K == 2 ? 2 : 1;
  ulonglong2 lo[REG ? 2 * K : 1];
  if constexpr (REG) {
#pragma unroll
    for (int cj = 0; cj < 2 * K; ++cj) lo[cj] = flo[cj * 256 + t];
  }
#pragma unroll UNK
  for (int k = 0; k < NK; ++k) {
    const int idx = t + (k << 8);
    u64 acc0 = __ldg(z0 + idx) + __ldg(m + idx);  // [0, 2q)
    u64 acc1 = __ldg(z1 + idx);
#pragma unroll UNJ
    for (int j = 0; j < K; ++j) {
      const ulonglong2 h0 = fhi[j * NK + k], l0 = REG ? lo[REG ? j : 0] : flo[j * 256 + t];
      const ulonglong2 h1 = fhi[(K + j) * NK + k], l1 = REG ? lo[REG ? K + j : 0] : flo[(K + j) * 256 + t];
      const u64 x = mul_shoup(mul_shoup(__ldg(E0 + j * estride + (k << 8)), h0.x, h0.y, q), l0.x, l0.y, q);
      const u64 y = mul_shoup(mul_shoup(__ldg(E1 + j * estride + (k << 8)), h1.x, h1.y, q), l1.x, l1.y, q);
      acc0 += x;
      acc1 += y;
      if (acc0 >= 2 * q) acc0 -= 2 * q;
      if (acc1 >= 2 * q) acc1 -= 2 * q;
    }
    c0[idx] = acc0 >= q ? acc0 - q : acc0;
    c1[idx] = acc1 >= q ? acc1 - q : acc1;
  }
}

__global__ void k_residues_batch(DevParams P, const i64* __restrict__ v, uint32_t batch, u64* out) {
  const int N = 1 << P.log_n, L = P.L;
  const size_t total = (size_t)batch * L * N;
  for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < total; x += (size_t)gridDim.x * blockDim.x) {
    const size_t b = x / ((size_t)L * N);
    const int i = (int)((x / N) % L);
    out[x] = reduce_signed(v[b * N + x % N], P.q[i], P.mu[i]);
  }
}

template <int K>
static cudaError_t zinc_ntt_k(const DevParams& P, const NttZincArgs& A, uint32_t batch, cudaStream_t st) {
  const size_t smem = sizeof(ulonglong2) * 2 * K * ((1u << (P.log_n - 8)) + 256);
  cudaError_t e = cudaFuncSetAttribute(k_zinc_ntt<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_zinc_ntt<K><<<dim3(P.L, batch), 256, smem, st>>>(P, A);
  return cudaGetLastError();
}

cudaError_t launch_zinc_ntt(const DevParams& P, const NttZincArgs& A, uint32_t batch, cudaStream_t st) {
  if (batch == 0) return cudaSuccess;
  if (P.log_n < 10 || P.log_n > 15 || A.K < 1 || A.K > 16) return cudaErrorInvalidValue;
  switch (A.K) {
    case 1: return zinc_ntt_k<1>(P, A, batch, st);
    case 2: return zinc_ntt_k<2>(P, A, batch, st);
    case 3: return zinc_ntt_k<3>(P, A, batch, st);
    case 4: return zinc_ntt_k<4>(P, A, batch, st);
    case 5: return zinc_ntt_k<5>(P, A, batch, st);
    case 6: return zinc_ntt_k<6>(P, A, batch, st);
    case 7: return zinc_ntt_k<7>(P, A, batch, st);
    case 8: return zinc_ntt_k<8>(P, A, batch, st);
    case 9: return zinc_ntt_k<9>(P, A, batch, st);
    case 10: return zinc_ntt_k<10>(P, A, batch, st);
    case 11: return zinc_ntt_k<11>(P, A, batch, st);
    case 12: return zinc_ntt_k<12>(P, A, batch, st);
    case 13: return zinc_ntt_k<13>(P, A, batch, st);
    case 14: return zinc_ntt_k<14>(P, A, batch, st);
    case 15: return zinc_ntt_k<15>(P, A, batch, st);
    default: return zinc_ntt_k<16>(P, A, batch, st);
  }
}

cudaError_t launch_residues_batch(const DevParams& P, const i64* v, uint32_t batch, u64* out, cudaStream_t st) {
  if (batch == 0) return cudaSuccess;
  size_t g = (((size_t)batch * P.L << P.log_n) + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  k_residues_batch<<<(unsigned)g, 256, 0, st>>>(P, v, batch, out);
  return cudaGetLastError();
}

}  // namespace zn
