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
// and coefficient 2K table lookups and 4K Shoup products -- no butterflies;
// the kernel streams the plaintext in and the ciphertext out (HBM) and reads
// the cache and the basis from L2.
#include "zn_kernels.h"

namespace zn {

// One block per (prime, ciphertext): the prime's power tables and the
// ciphertext's 2K rotations in shared memory, then a block-strided pass over
// the N outputs (consecutive threads, consecutive coefficients).
__global__ void __launch_bounds__(256) k_zinc_ntt(DevParams P, NttZincArgs A) {
  __shared__ ulonglong2 s_hi[1024];     // N/32 entries, N <= 2^15
  __shared__ ulonglong2 s_lo[64];
  __shared__ unsigned s_r[32];          // [2][K], K <= 16
  const int i = blockIdx.x;
  const size_t b = blockIdx.y;
  const int log_n = P.log_n, N = 1 << log_n, L = P.L, K = A.K;
  const unsigned mask2n = 2u * N - 1;
  const u64 q = P.q[i];
  for (int h = threadIdx.x; h < N / 32; h += blockDim.x) s_hi[h] = __ldg(A.thi + (size_t)i * (N / 32) + h);
  for (int l = threadIdx.x; l < 64; l += blockDim.x) s_lo[l] = __ldg(A.tlo + (size_t)i * 64 + l);
  if (threadIdx.x < 2 * K) {
    const int c = threadIdx.x / K, j = threadIdx.x % K;
    const uint4 w = zn_rand(A.seed, (unsigned)j, rand_tag(5, (unsigned)c, 0), A.ct_index[b]);
    s_r[c * 16 + j] = w.x & mask2n;
  }
  __syncthreads();
  const u64* z0 = A.z + (size_t)i * N;
  const u64* z1 = z0 + (size_t)L * N;
  const u64* m = A.m + (b * L + i) * N;
  u64* c0 = A.out + (b * 2 * L + i) * N;
  u64* c1 = c0 + (size_t)L * N;
  const size_t estride = (size_t)L * N;          // between basis polynomials of one prime
  const u64* E0 = A.E + (size_t)i * N;           // E_{0,0} at prime i
  const u64* E1 = E0 + (size_t)K * estride;      // E_{1,0}
  for (int idx = threadIdx.x; idx < N; idx += blockDim.x) {
    const unsigned a = 2u * (__brev((unsigned)idx) >> (32 - log_n)) + 1u;
    u64 acc0 = __ldg(z0 + idx) + __ldg(m + idx);  // [0, 2q)
    u64 acc1 = __ldg(z1 + idx);
#pragma unroll 4
    for (int j = 0; j < K; ++j) {
      const unsigned e0 = (a * s_r[j]) & mask2n, e1 = (a * s_r[16 + j]) & mask2n;
      const ulonglong2 h0 = s_hi[e0 >> 6], l0 = s_lo[e0 & 63], h1 = s_hi[e1 >> 6], l1 = s_lo[e1 & 63];
      u64 x = mul_shoup(mul_shoup(__ldg(E0 + j * estride + idx), h0.x, h0.y, q), l0.x, l0.y, q);
      u64 y = mul_shoup(mul_shoup(__ldg(E1 + j * estride + idx), h1.x, h1.y, q), l1.x, l1.y, q);
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

cudaError_t launch_zinc_ntt(const DevParams& P, const NttZincArgs& A, uint32_t batch, cudaStream_t st) {
  if (batch == 0) return cudaSuccess;
  if (P.log_n < 10 || P.log_n > 15 || A.K < 1 || A.K > 16) return cudaErrorInvalidValue;
  k_zinc_ntt<<<dim3(P.L, batch), 256, 0, st>>>(P, A);
  return cudaGetLastError();
}

cudaError_t launch_residues_batch(const DevParams& P, const i64* v, uint32_t batch, u64* out, cudaStream_t st) {
  if (batch == 0) return cudaSuccess;
  size_t g = (((size_t)batch * P.L << P.log_n) + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  k_residues_batch<<<(unsigned)g, 256, 0, st>>>(P, v, batch, out);
  return cudaGetLastError();
}

}  // namespace zn
