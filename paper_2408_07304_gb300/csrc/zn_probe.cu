// Diagnostic: the throughput ceiling of this library's modular butterflies.
// Every thread runs the Harvey/Shoup forward butterfly of the NTT (the
// corrected form, or the relaxed form the transforms use for primes below
// 2^59) on 16 register-resident values (radix-16 pattern, no memory traffic)
// and writes one word at the end, so the measured rate is the best any
// transform built from that butterfly can reach on the device.
#include "zn_kernels.h"

namespace zn {

template <bool RELAX>
__global__ void __launch_bounds__(512) k_probe_butterfly(u64* out, u64 q, u64 w, u64 wp, int rounds) {
  u64 v[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = ((u64)threadIdx.x * 16 + r + blockIdx.x) % q;
  for (int it = 0; it < rounds; ++it) {
#pragma unroll
    for (int s = 3; s >= 0; --s) {
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        if (r & (1 << s)) continue;
        if constexpr (RELAX) ct_bfly_relaxed(v[r], v[r + (1 << s)], make_ulonglong2(w, wp), q);
        else ct_bfly(v[r], v[r + (1 << s)], w, wp, q);
      }
    }
    if constexpr (RELAX) {
      // relaxed values grow by at most 2q per stage: after 12 stages from
      // [0, 4q) they are below 28q; fold them back as a transform's final
      // reduction would (about one compare-subtract per butterfly)
      if (it % 3 == 2) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
          if (v[r] >= 16 * q) v[r] -= 16 * q;
          if (v[r] >= 8 * q) v[r] -= 8 * q;
          if (v[r] >= 4 * q) v[r] -= 4 * q;
        }
      }
    }
    w ^= (u64)(it & 1);   // a loop-carried twiddle (stays below q: q is odd and w even)
  }
  u64 acc = 0;
#pragma unroll
  for (int r = 0; r < 16; ++r) acc ^= v[r];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

cudaError_t probe_butterfly(int sms, double* per_s, bool relaxed) {
  const u64 q = 1125899904679937ull;                 // a 50-bit prime = 1 mod 2^16
  const u64 w = 123456789012344ull;                  // even, < q
  const u64 wp = (u64)(((u128)w << 64) / q);
  const int blocks = 2 * sms, threads = 512, rounds = 1000;
  u64* out = nullptr;
  cudaError_t e = cudaMalloc(&out, sizeof(u64) * blocks * threads);
  if (e != cudaSuccess) return e;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  float best = 0.f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(a, 0);
    if (relaxed) k_probe_butterfly<true><<<blocks, threads>>>(out, q, w, wp, rounds);
    else k_probe_butterfly<false><<<blocks, threads>>>(out, q, w, wp, rounds);
    cudaEventRecord(b, 0);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    if (rep == 0 || ms < best) best = ms;
  }
  e = cudaGetLastError();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(out);
  *per_s = (double)blocks * threads * rounds * 32.0 / (best * 1e-3);
  return e;
}

}  // namespace zn
