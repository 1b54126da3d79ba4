// N = 2^15 limbs on a thread-block cluster of four CTAs (shared by the CKKS,
// modulus-switched and BFV / BGV encryption kernels at N = 2^15).
//
// Each CTA owns one output quarter of the limb (2^13 residues, 64 KiB of
// shared memory, 256 threads, at most 80 registers: three CTAs per SM, as
// at N = 2^14).  The forward negacyclic NTT's first three butterfly stages
// (distances N/2, N/4 and N/8; twiddles tw[1], tw[2 + h], tw[4 + j]) mix the
// four quarters: each CTA computes those stages for one quarter of the index
// range and stores every result directly into the shared memory of the CTA
// that owns its quarter (distributed shared memory, st.shared::cluster).
// After a cluster barrier each CTA runs the remaining 12 stages on its
// quarter alone, a 2^13-point transform with tmul = 4 + j, and the epilogue.
// No stage is computed twice, and 24 warps share an SM.
#pragma once
#include <type_traits>

#include "zn_cluster.cuh"
#include "zn_encrypt_fn.cuh"
#include "zn_tmem.cuh"

namespace zn {
namespace quarter {

constexpr int kLog = 13;              // log2 of the quarter
constexpr int kQ = 1 << kLog;         // residues per CTA
constexpr int kN = 4 * kQ;            // N = 2^15
constexpr int kT = 256;               // threads per CTA
constexpr int kKm = 3;                // radix-8 passes (shared-memory layout swz<13, 3>)

using cluster::cluster_rank;
using cluster::cluster_sync;
using cluster::map_rank;
using cluster::st_cluster;

using cluster::below4q;

// Work items of CTA j: index k < N/8, k in [j N/32, (j+1) N/32), with eight
// inputs at k + m N/4 and k + N/8 + m N/4 (m < 4).  x[m] and x[4 + m] hold
// quarter m's values at positions k and k + N/8 after the first two stages;
// this runs the third stage (inside each quarter, twiddle tw[4 + m]) and
// stores the results into the owners' shared memory.
template <bool RELAX>
__device__ __forceinline__ void third_stage_store(u64 (&x)[8], const unsigned (&dst)[4], int k,
                                                  const ulonglong2* tw, u64 q) {
  constexpr int Q2 = kQ / 2;
#pragma unroll
  for (int jj = 0; jj < 4; ++jj) {
    bfly<RELAX>(x[jj], x[4 + jj], __ldg(tw + 4 + jj), q);
    st_cluster(dst[jj] + 8u * (unsigned)swz<kLog, kKm>(k), below4q<RELAX>(x[jj], q));
    st_cluster(dst[jj] + 8u * (unsigned)swz<kLog, kKm>(k + Q2), below4q<RELAX>(x[4 + jj], q));
  }
}

// Coefficients given by v(k) in [0, 2q) (any value functor).
template <bool RELAX, class V>
__device__ __forceinline__ void gen_val(u64* sm, int t, unsigned j, const V& v, const ulonglong2* tw, u64 q) {
  constexpr int Q2 = kQ / 2;
  unsigned dst[4];
#pragma unroll
  for (int jj = 0; jj < 4; ++jj) dst[jj] = map_rank(sm, jj);
  const ulonglong2 w1 = __ldg(tw + 1), w2 = __ldg(tw + 2), w3 = __ldg(tw + 3);
#pragma unroll 1
  for (int r = 0; r < Q2 / 4 / kT; ++r) {
    const int k = (int)j * (Q2 / 4) + r * kT + t;
    u64 x[8];                     // x[m]: input k + m Q, x[4 + m]: input k + Q/2 + m Q
#pragma unroll
    for (int m = 0; m < 8; ++m) x[m] = v(k + (m >> 2) * Q2 + (m & 3) * kQ);
#pragma unroll
    for (int o = 0; o < 2; ++o) {           // first stage, distance N/2
      bfly<RELAX>(x[4 * o + 0], x[4 * o + 2], w1, q);
      bfly<RELAX>(x[4 * o + 1], x[4 * o + 3], w1, q);
    }
#pragma unroll
    for (int o = 0; o < 2; ++o) {           // second stage, distance N/4: halves h = 0 (w2), 1 (w3)
      bfly<RELAX>(x[4 * o + 0], x[4 * o + 1], w2, q);
      bfly<RELAX>(x[4 * o + 2], x[4 * o + 3], w3, q);
    }
    third_stage_store<RELAX>(x, dst, k, tw, q);
  }
}

// Small signed coefficients (int8).  TERN (u, values in {-1, 0, 1}): the first
// two stages from selections -- with w1 = psi^(N/2), w2 = psi^(N/4),
// w3 = psi^(3N/4) and psi^N = -1, w1 w2 = w3 and w1 w3 = -w2, so the quarter
// values after two stages are (u0 + w1 u2) +- (w2 u1 + w3 u3) and
// (u0 - w1 u2) +- (w3 u1 + w2 u3).  Otherwise (chi, |e| <= 19) the first
// stage's products are small ones (outputs below 3q).
template <bool RELAX, bool TERN>
__device__ __forceinline__ void gen_i8(u64* sm, int t, unsigned j, const int8_t* __restrict__ a,
                                       const ulonglong2* tw, u64 q) {
  constexpr int Q2 = kQ / 2;
  unsigned dst[4];
#pragma unroll
  for (int jj = 0; jj < 4; ++jj) dst[jj] = map_rank(sm, jj);
  const ulonglong2 w1 = __ldg(tw + 1), w2 = __ldg(tw + 2), w3 = __ldg(tw + 3);
#pragma unroll 1
  for (int r = 0; r < Q2 / 4 / kT; ++r) {
    const int k = (int)j * (Q2 / 4) + r * kT + t;
    u64 x[8];
#pragma unroll
    for (int o = 0; o < 2; ++o) {
      const int kk = k + o * Q2;
      const int e0 = __ldg(a + kk), e1 = __ldg(a + kk + kQ), e2 = __ldg(a + kk + 2 * kQ), e3 = __ldg(a + kk + 3 * kQ);
      if constexpr (TERN) {
        const u64 s1 = mul_tern(e2, w1.x, q);
        const u64 xp = small_res(e0, q) + s1;                   // u0 + w1 u2, [0, 2q)
        const u64 xm = small_res(e0, q) + q - s1;               // u0 - w1 u2, [0, 2q)
        const u64 p = mul_tern(e1, w2.x, q) + mul_tern(e3, w3.x, q);     // [0, 2q]
        const u64 pp = mul_tern(e1, w3.x, q) + mul_tern(e3, w2.x, q);    // [0, 2q]
        x[4 * o + 0] = xp + p;
        x[4 * o + 1] = xp - p + 2 * q;
        x[4 * o + 2] = xm + pp;
        x[4 * o + 3] = xm - pp + 2 * q;                         // all below 4q
      } else {
        x[4 * o + 0] = small_res(e0, q) + mul_small(e2, w1.x, w1.y, q);
        x[4 * o + 2] = small_res(e0, q) + mul_small(-e2, w1.x, w1.y, q);
        x[4 * o + 1] = small_res(e1, q) + mul_small(e3, w1.x, w1.y, q);
        x[4 * o + 3] = small_res(e1, q) + mul_small(-e3, w1.x, w1.y, q);
      }
    }
    if constexpr (!TERN) {
#pragma unroll
      for (int o = 0; o < 2; ++o) {
        bfly<RELAX>(x[4 * o + 0], x[4 * o + 1], w2, q);
        bfly<RELAX>(x[4 * o + 2], x[4 * o + 3], w3, q);
      }
    }
    third_stage_store<RELAX>(x, dst, k, tw, q);
  }
}

// One quarter unit of cluster rank j: o's outputs and keys point at the
// quarter (offset j N/4); gu, g0, g1 run the generators of u (vanilla shape
// only) and of the two transform inputs.
//   vanilla shape:  c0 = k0 * NTT(u) + NTT(v0),   c1 = k1 * NTT(u) + NTT(v1)
//   Zinc shape:     c0 = z0 + NTT(v0),            c1 = z1 + NTT(v1)
// Local outputs below 28q (relaxed: 4q + 12 * 2q) or 4q (Harvey) go
// unreduced into the epilogue sums (below 30q with a key product).  Vanilla
// parks u-hat unreduced in c1 (one word per coefficient; Shoup's product
// takes any 64-bit input) and each later epilogue forms its own key product;
// the same thread reads and rewrites each index.
//
// Where vanilla parks u-hat between its transform and the two later
// epilogues: in the c1 output words (ParkOut), or in tensor memory
// (ParkTmem, zn_tmem.cuh: the staged epilogue hands thread t the indices
// t + 256 i, i < 32, and i picks the columns).
struct ParkOut {
  u64* c1;
  __device__ __forceinline__ void put(int idx, u64 v) const { c1[idx] = v; }
  __device__ __forceinline__ u64 get(int idx) const { return c1[idx]; }
  __device__ __forceinline__ void done() const {}
};
using ParkTmem = tmem::Park;
static_assert(kT == 256 && kQ == 32 * kT, "ParkTmem: 32 outputs per thread, index t + 256 i");

template <bool ZINC, bool RELAX, class GU, class G0, class G1, class Park>
__device__ __forceinline__ void unit(u64* sm, int t, unsigned j, const ulonglong2* tw, u64 q, const FnLimb& o,
                                     const GU& gu, const G0& g0, const G1& g1, const Park& park) {
  static_assert(4 + 2 * 12 + 2 <= 32, "relaxed sums must stay below 32q");
  static_assert(NttShape<kLog, 5>::T == kT, "256 threads per quarter");
  const int tmul = 4 + (int)j;
  u64* c0 = o.c0;
  u64* c1 = o.c1;
  const u64* k0 = o.k0;
  const u64* k1 = o.k1;
  auto sum = [&](u64 a, u64 x) { return reduce_sum<RELAX>(a + x, q); };
  // every CTA of the cluster is running (and done reading its own buffer)
  // before any CTA writes into it; every write has landed before the transform
  auto transform = [&](const auto& gen, auto& store) {
    cluster_sync();
    gen();
    cluster_sync();
    ntt_chain<kLog, 5, kLog - 1, RELAX, std::remove_reference_t<decltype(store)>, kKm, true, true>(sm, t, tw, tmul,
                                                                                                 q, store);
  };
  // the finished ciphertext words are written once and not read again here:
  // streaming stores (evict first) leave L2 to u-hat, the keys and the inputs
  if constexpr (!ZINC) {
    const u64* k0s = o.k0s;
    const u64* k1s = o.k1s;
    auto st_u = [&](int idx, u64 uh) { park.put(idx, uh); };
    transform(gu, st_u);
    park.done();
    auto st_0 = [&](int idx, u64 x) {
      __stcs(c0 + idx, sum(mul_shoup(park.get(idx), __ldg(k0 + idx), __ldg(k0s + idx), q), x));
    };
    transform(g0, st_0);
    auto st_1 = [&](int idx, u64 x) {
      __stcs(c1 + idx, sum(mul_shoup(park.get(idx), __ldg(k1 + idx), __ldg(k1s + idx), q), x));
    };
    transform(g1, st_1);
  } else {
    auto st_0 = [&](int idx, u64 x) { __stcs(c0 + idx, sum(__ldg(k0 + idx), x)); };
    transform(g0, st_0);
    auto st_1 = [&](int idx, u64 x) { __stcs(c1 + idx, sum(__ldg(k1 + idx), x)); };
    transform(g1, st_1);
  }
}

// u-hat parked in the c1 output words.
template <bool ZINC, bool RELAX, class GU, class G0, class G1>
__device__ __forceinline__ void unit(u64* sm, int t, unsigned j, const ulonglong2* tw, u64 q, const FnLimb& o,
                                     const GU& gu, const G0& g0, const G1& g1) {
  unit<ZINC, RELAX>(sm, t, j, tw, q, o, gu, g0, g1, ParkOut{o.c1});
}

// Launch a quarter kernel: clusters of four consecutive CTAs along x.
template <class... Args>
cudaError_t launch(void (*kern)(Args...), dim3 grid, cudaStream_t st, Args... args) {
  return cluster::launch(4, sizeof(u64) * kQ, kern, grid, kT, st, args...);
}

}  // namespace quarter
}  // namespace zn
