// Slot batching for BFV / BGV plaintexts: for a prime t = 1 mod 2N, R_t is
// isomorphic to Z_t^N by evaluation at the odd powers of psi_t (the minimal
// primitive 2N-th root mod t).  Slot s < N/2 is the value at
// psi_t^(5^s mod 2N), slot N/2 + s the value at psi_t^(-5^s mod 2N); in the
// NTT's bit-reversed output order that value sits at index pos[s] with
// 2 brv(pos[s]) + 1 = a_s.  Encode: scatter the slots to pos, inverse NTT mod
// t, times N^-1.  Decode: forward NTT mod t, gather from pos.  One block per
// vector; radix-2 stages in place in global memory (not on the encryption
// path).
#include "zn_kernels.h"

namespace zn {

// slots [B][N] (any int64, taken mod t) -> m [B][N] in [0, t)
__global__ void __launch_bounds__(1024) k_batch_encode(BatchEnc E, const i64* __restrict__ slots, i64* __restrict__ m) {
  const int N = 1 << E.log_n;
  const size_t b = blockIdx.x;
  const u64 t = E.t;
  u64* a = reinterpret_cast<u64*>(m + b * N);
  const i64* x = slots + b * N;
  for (int s = threadIdx.x; s < N; s += blockDim.x) {
    const i64 r = x[s] % (i64)t;
    a[__ldg(E.pos + s)] = (u64)(r < 0 ? r + (i64)t : r);
  }
  __syncthreads();
  // Gentleman-Sande, bit-reversed input -> natural order
  for (int lt = 0; lt < E.log_n; ++lt) {
    const int h = 1 << lt, groups = N >> (lt + 1);
    for (int id = threadIdx.x; id < N / 2; id += blockDim.x) {
      const int g = id >> lt, j = id & (h - 1);
      const int j1 = 2 * g * h + j;
      const u64 w = __ldg(E.itw + groups + g), ws = __ldg(E.itws + groups + g);
      const u64 U = a[j1], V = a[j1 + h];
      u64 sum = U + V;
      if (sum >= t) sum -= t;
      const u64 d = U >= V ? U - V : U + t - V;
      u64 r = mul_shoup(d, w, ws, t);
      if (r >= t) r -= t;
      a[j1] = sum;
      a[j1 + h] = r;
    }
    __syncthreads();
  }
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    u64 r = mul_shoup(a[k], E.ninv, E.ninvs, t);
    a[k] = r >= t ? r - t : r;
  }
}

// m [B][N] (any int64, taken mod t) -> slots [B][N] in [0, t); work [B][N] scratch
__global__ void __launch_bounds__(1024) k_batch_decode(BatchEnc E, const i64* __restrict__ m, u64* __restrict__ work,
                                                       i64* __restrict__ slots) {
  const int N = 1 << E.log_n;
  const size_t b = blockIdx.x;
  const u64 t = E.t;
  u64* a = work + b * N;
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    const i64 r = m[b * N + k] % (i64)t;
    a[k] = (u64)(r < 0 ? r + (i64)t : r);
  }
  __syncthreads();
  // Cooley-Tukey, natural input -> bit-reversed output (the library's NTT)
  for (int lm = 0; lm < E.log_n; ++lm) {
    const int groups = 1 << lm, h = N >> (lm + 1);
    for (int id = threadIdx.x; id < N / 2; id += blockDim.x) {
      const int g = id / h, j = id % h;
      const int j1 = 2 * g * h + j;
      const ulonglong2 w = __ldg(E.twp + groups + g);
      const u64 U = a[j1];
      u64 V = mul_shoup(a[j1 + h], w.x, w.y, t);
      if (V >= t) V -= t;
      u64 sum = U + V;
      if (sum >= t) sum -= t;
      a[j1] = sum;
      a[j1 + h] = U >= V ? U - V : U + t - V;
    }
    __syncthreads();
  }
  for (int s = threadIdx.x; s < N; s += blockDim.x) slots[b * N + s] = (i64)a[__ldg(E.pos + s)];
}

cudaError_t launch_batch_encode(const BatchEnc& E, const i64* slots, uint32_t batch, i64* m, cudaStream_t st) {
  if (batch == 0) return cudaSuccess;
  k_batch_encode<<<batch, 1024, 0, st>>>(E, slots, m);
  return cudaGetLastError();
}

cudaError_t launch_batch_decode(const BatchEnc& E, const i64* m, uint32_t batch, u64* work, i64* slots,
                                cudaStream_t st) {
  if (batch == 0) return cudaSuccess;
  k_batch_decode<<<batch, 1024, 0, st>>>(E, m, work, slots);
  return cudaGetLastError();
}

}  // namespace zn
