// N = 2^14 limbs on a thread-block cluster of two CTAs (the CKKS encryption
// kernel at N = 2^14).
//
// Each CTA owns one output half of the limb (2^13 residues, 64 KiB of
// shared memory, 256 threads, at most 80 registers: three CTAs per SM).  The
// forward negacyclic NTT's first stage (distance N/2, twiddle tw[1]) mixes
// the halves; the second (distance N/4; tw[2] in half 0, tw[3] in half 1)
// runs inside each half.  Each CTA computes both stages for half of the
// index range k < N/4 (inputs k + m N/4, m < 4) and stores each half's two
// results into that half's CTA (distributed shared memory).  After a cluster
// barrier each CTA runs the remaining 12 stages on its half alone, a
// 2^13-point transform with tmul = 2 + h, and the epilogue.  Without the
// exchange each half ran the first stage for all of its outputs and read
// and reduced all N inputs.
#pragma once
#include <type_traits>

#include "zn_cluster.cuh"
#include "zn_encrypt_fn.cuh"

namespace zn {
namespace pair {

constexpr int kLog = 13;              // log2 of the half
constexpr int kH = 1 << kLog;         // residues per CTA
constexpr int kN = 2 * kH;            // N = 2^14
constexpr int kQ2 = kH / 2;           // N/4
constexpr int kT = 256;               // threads per CTA
constexpr int kKm = 3;                // radix-8 passes (shared-memory layout swz<13, 3>)
constexpr int kItems = kQ2 / 2;       // indices k per CTA

// Outputs of index k after both stages: half 0 takes z0, z1 at local k,
// k + N/4; half 1 takes z2, z3 at the same local indices.
template <bool RELAX>
__device__ __forceinline__ void store_pair(const unsigned (&dst)[2], int k, u64 z0, u64 z1, u64 z2, u64 z3, u64 q) {
  cluster::st_cluster(dst[0] + 8u * (unsigned)swz<kLog, kKm>(k), cluster::below4q<RELAX>(z0, q));
  cluster::st_cluster(dst[0] + 8u * (unsigned)swz<kLog, kKm>(k + kQ2), cluster::below4q<RELAX>(z1, q));
  cluster::st_cluster(dst[1] + 8u * (unsigned)swz<kLog, kKm>(k), cluster::below4q<RELAX>(z2, q));
  cluster::st_cluster(dst[1] + 8u * (unsigned)swz<kLog, kKm>(k + kQ2), cluster::below4q<RELAX>(z3, q));
}

// Coefficients given by v(k) in [0, 2q) (any value functor); CTA j takes
// k in [j N/8, (j + 1) N/8).
template <bool RELAX, class V>
__device__ __forceinline__ void gen_val(u64* sm, int t, unsigned j, const V& v, const ulonglong2* tw, u64 q) {
  const unsigned dst[2] = {cluster::map_rank(sm, 0), cluster::map_rank(sm, 1)};
  const ulonglong2 w1 = __ldg(tw + 1), w2 = __ldg(tw + 2), w3 = __ldg(tw + 3);
#pragma unroll 1
  for (int r = 0; r < kItems / kT; ++r) {
    const int k = (int)j * kItems + r * kT + t;
    u64 x0 = v(k), x1 = v(k + kQ2), x2 = v(k + kH), x3 = v(k + kH + kQ2);
    bfly<RELAX>(x0, x2, w1, q);                // distance N/2
    bfly<RELAX>(x1, x3, w1, q);
    bfly<RELAX>(x0, x1, w2, q);                // distance N/4, half 0
    bfly<RELAX>(x2, x3, w3, q);                // half 1
    store_pair<RELAX>(dst, k, x0, x1, x2, x3, q);
  }
}

// Small signed coefficients (int8).  TERN (u, values in {-1, 0, 1}): both
// stages from selections -- with w1 = psi^(N/2), w2 = psi^(N/4),
// w3 = psi^(3N/4) and psi^N = -1, w1 w2 = w3 and w1 w3 = -w2, so the values
// after two stages are (u0 + w1 u2) +- (w2 u1 + w3 u3) in half 0 and
// (u0 - w1 u2) +- (w3 u1 + w2 u3) in half 1.  Otherwise (chi, |e| <= 19) the
// first stage's products are small ones (outputs below 3q).
template <bool RELAX, bool TERN>
__device__ __forceinline__ void gen_i8(u64* sm, int t, unsigned j, const int8_t* __restrict__ a,
                                       const ulonglong2* tw, u64 q) {
  const unsigned dst[2] = {cluster::map_rank(sm, 0), cluster::map_rank(sm, 1)};
  const ulonglong2 w1 = __ldg(tw + 1), w2 = __ldg(tw + 2), w3 = __ldg(tw + 3);
#pragma unroll 1
  for (int r = 0; r < kItems / kT; ++r) {
    const int k = (int)j * kItems + r * kT + t;
    const int e0 = __ldg(a + k), e1 = __ldg(a + k + kQ2), e2 = __ldg(a + k + kH), e3 = __ldg(a + k + kH + kQ2);
    if constexpr (TERN) {
      const u64 s1 = mul_tern(e2, w1.x, q);
      const u64 xp = small_res(e0, q) + s1;                       // u0 + w1 u2, [0, 2q)
      const u64 xm = small_res(e0, q) + q - s1;                   // u0 - w1 u2, [0, 2q]
      const u64 p = mul_tern(e1, w2.x, q) + mul_tern(e3, w3.x, q);     // [0, 2q]
      const u64 pp = mul_tern(e1, w3.x, q) + mul_tern(e3, w2.x, q);    // [0, 2q]
      store_pair<RELAX>(dst, k, xp + p, xp - p + 2 * q, xm + pp, xm - pp + 2 * q, q);   // all below 4q
    } else {
      u64 x0 = small_res(e0, q) + mul_small(e2, w1.x, w1.y, q);
      u64 x2 = small_res(e0, q) + mul_small(-e2, w1.x, w1.y, q);
      u64 x1 = small_res(e1, q) + mul_small(e3, w1.x, w1.y, q);
      u64 x3 = small_res(e1, q) + mul_small(-e3, w1.x, w1.y, q);
      bfly<RELAX>(x0, x1, w2, q);
      bfly<RELAX>(x2, x3, w3, q);
      store_pair<RELAX>(dst, k, x0, x1, x2, x3, q);
    }
  }
}

// One transform: the generator fills both halves' buffers (after the peer
// has read its buffer for the previous epilogue), then the 12 local stages
// and the epilogue, EU its unroll.
template <bool RELAX, int EU, class Gen, class Store>
__device__ __forceinline__ void transform(u64* sm, int t, const ulonglong2* tw, int tmul, u64 q, const Gen& gen,
                                          Store& store) {
  cluster::cluster_sync();
  gen();
  cluster::cluster_sync();
  ntt_chain<kLog, 5, kLog - 1, RELAX, Store, kKm, true, true, EU>(sm, t, tw, tmul, q, store);
}

// One half unit of cluster rank h: o's outputs and keys point at the half
// (offset h N/2); gu, g0, g1 run the generators of u (vanilla only) and of
// the two transform inputs.
//   vanilla shape:  c0 = k0 * NTT(u) + NTT(v0),   c1 = k1 * NTT(u) + NTT(v1)
//   Zinc shape:     c0 = z0 + NTT(v0),            c1 = z1 + NTT(v1)
// Local outputs below 28q (relaxed: 4q + 12 * 2q) or 4q (Harvey) go
// unreduced into the epilogue sums (below 30q with a key product).  The
// first vanilla epilogue forms both key products while u-hat is in
// registers and parks them, lazily reduced, in c0 and c1; the later ones add
// to them (the same thread reads and rewrites each index).  STREAM writes
// the finished words with streaming stores (put_ct).  The epilogues unroll
// by 4 in both shapes (Zinc: 11.59 -> 11.48 ms per 4096 ciphertexts against
// an unroll of 2, 12.01 with 1).
template <bool ZINC, bool RELAX, bool STREAM = false, class GU, class G0, class G1>
__device__ __forceinline__ void unit(u64* sm, int t, unsigned h, const ulonglong2* tw, u64 q, const FnLimb& o,
                                     const GU& gu, const G0& g0, const G1& g1) {
  static_assert(4 + 2 * 12 + 2 <= 32, "relaxed sums must stay below 32q");
  static_assert(NttShape<kLog, 5>::T == kT, "256 threads per half");
  const int tmul = 2 + (int)h;
  u64* c0 = o.c0;
  u64* c1 = o.c1;
  const u64* k0 = o.k0;
  const u64* k1 = o.k1;
  auto sum = [&](u64 a, u64 x) { return reduce_sum<RELAX>(a + x, q); };
  if constexpr (!ZINC) {
    const u64* k0s = o.k0s;
    const u64* k1s = o.k1s;
    auto st_u = [&](int idx, u64 uh) {
      c0[idx] = mul_shoup(uh, __ldg(k0 + idx), __ldg(k0s + idx), q);
      c1[idx] = mul_shoup(uh, __ldg(k1 + idx), __ldg(k1s + idx), q);
    };
    transform<RELAX, 4>(sm, t, tw, tmul, q, gu, st_u);
    auto st_0 = [&](int idx, u64 x) { put_ct<STREAM>(c0 + idx, sum(c0[idx], x)); };
    transform<RELAX, 4>(sm, t, tw, tmul, q, g0, st_0);
    auto st_1 = [&](int idx, u64 x) { put_ct<STREAM>(c1 + idx, sum(c1[idx], x)); };
    transform<RELAX, 4>(sm, t, tw, tmul, q, g1, st_1);
  } else {
    auto st_0 = [&](int idx, u64 x) { put_ct<STREAM>(c0 + idx, sum(__ldg(k0 + idx), x)); };
    transform<RELAX, 4>(sm, t, tw, tmul, q, g0, st_0);
    auto st_1 = [&](int idx, u64 x) { put_ct<STREAM>(c1 + idx, sum(__ldg(k1 + idx), x)); };
    transform<RELAX, 4>(sm, t, tw, tmul, q, g1, st_1);
  }
}

// Launch a pair kernel: clusters of two consecutive CTAs along x.
template <class... Args>
cudaError_t launch(void (*kern)(Args...), dim3 grid, cudaStream_t st, Args... args) {
  return cluster::launch(2, sizeof(u64) * kH, kern, grid, kT, st, args...);
}

}  // namespace pair
}  // namespace zn
