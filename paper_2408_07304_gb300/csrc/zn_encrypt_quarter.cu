// Hot path at N = 2^15 (the large ring and the paper's own parameters): one
// limb of one ciphertext per four-CTA cluster, one output quarter per CTA
// (zn_quarter.cuh), with the epilogue
//   vanilla (Eq. 8):      c0 = pk0*u + NTT(m + e0),  c1 = pk1*u + NTT(e1)
//   Zinc (Algorithm 1):   c0' = z0 + NTT(m + e1'),   c1' = z1 + NTT(e2')
// on the integers the prep kernel prepared once per ciphertext.
#include "zn_quarter.cuh"

namespace zn {
namespace {

// Park: quarter::ParkTmem, or quarter::ParkOut (its pointer unused: u-hat
// goes to this unit's c1 words).
template <bool ZINC, bool RELAX, class Park>
__device__ __forceinline__ void encrypt_quarter_unit_q(const DevParams& P, const EncArgs& A, int i, unsigned j,
                                                       size_t b, u64* sm, int t, const Park& park) {
  using namespace quarter;
  const int L = P.L;
  const u64 q = P.q[i];
  const ulonglong2* tw = P.twp + (size_t)i * kN;
  const size_t off = (size_t)j * kQ;
  FnLimb o;
  o.c0 = A.out + (b * 2 * L + i) * kN + off;
  o.c1 = o.c0 + (size_t)L * kN;
  o.k0 = A.key + (size_t)i * kN + off;
  o.k1 = o.k0 + (size_t)L * kN;
  o.k0s = ZINC ? nullptr : A.keys + (size_t)i * kN + off;
  o.k1s = ZINC ? nullptr : o.k0s + (size_t)L * kN;
  o.u = nullptr;
  const int8_t* sp = A.small + b * 2 * kN;       // vanilla: u, e1; Zinc: e2'
  const MeVal me{A.me + b * kN, q, P.mu[i], P.moff[i]};
  auto g_me = [&] { gen_val<RELAX>(sm, t, j, me, tw, q); };
  if constexpr (!ZINC) {
    auto g_u = [&] { gen_i8<RELAX, true>(sm, t, j, sp, tw, q); };
    auto g_e1 = [&] { gen_i8<RELAX, false>(sm, t, j, sp + kN, tw, q); };
    if constexpr (std::is_same_v<Park, ParkOut>) unit<false, RELAX>(sm, t, j, tw, q, o, g_u, g_me, g_e1);
    else unit<false, RELAX>(sm, t, j, tw, q, o, g_u, g_me, g_e1, park);
  } else {
    auto g_e2 = [&] { gen_i8<RELAX, false>(sm, t, j, sp, tw, q); };
    unit<true, RELAX>(sm, t, j, tw, q, o, g_me, g_me, g_e2);
  }
}

// grid (4L, B), or (4B, L) when A.swap; the CTA of cluster rank j owns
// output quarter j.  Vanilla parks u-hat in tensor memory.
template <bool ZINC>
__global__ void __launch_bounds__(quarter::kT, 3) k_encrypt_quarter(DevParams P, EncArgs A) {
  extern __shared__ u64 sm[];
  const unsigned j = quarter::cluster_rank();
  const int i = A.swap ? (int)blockIdx.y : (int)(blockIdx.x >> 2);
  const size_t b = A.swap ? (size_t)(blockIdx.x >> 2) : blockIdx.y;
  // the relaxed/Harvey choice is uniform per unit, so all four CTAs of a
  // cluster take the same branch and meet at the same barriers
  const bool relax = P.q[i] < kRelaxLimit;
  if constexpr (ZINC) {
    const quarter::ParkOut park{nullptr};
    if (relax) encrypt_quarter_unit_q<true, true>(P, A, i, j, b, sm, threadIdx.x, park);
    else encrypt_quarter_unit_q<true, false>(P, A, i, j, b, sm, threadIdx.x, park);
  } else {
    __shared__ unsigned s_tmem;
    const tmem::Scope tm(&s_tmem);
    const quarter::ParkTmem park{tmem::thread_base(tm.base)};
    if (relax) encrypt_quarter_unit_q<false, true>(P, A, i, j, b, sm, threadIdx.x, park);
    else encrypt_quarter_unit_q<false, false>(P, A, i, j, b, sm, threadIdx.x, park);
    tm.release();
  }
}

// ---------------------------------------- persistent mixed-ring launch
// Packet: one limb (ciphertext b0, prime `prime`) of a 2^15 job, run by one
// four-CTA cluster.  Inlined: separate register allocation per path
// (__noinline__) measured 3 % slower.
// Vanilla parks u-hat in the c1 output words here: parking it in tensor
// memory, as the single-ring kernel does, measured 38 % slower in this
// kernel (more spills around the four inlined unit variants).
template <bool ZINC, bool RELAX>
__device__ __forceinline__ void batch_quarter(const JobDesc& J, const EncPacket& pk, unsigned j, u64* sm) {
  encrypt_quarter_unit_q<ZINC, RELAX>(J.P, J.E, pk.prime, j, pk.b0, sm, threadIdx.x, quarter::ParkOut{nullptr});
}

__device__ __forceinline__ int ld_cluster_s32(unsigned addr) {
  int v;
  asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}

// Persistent clusters: rank 0 takes the next packet from a global counter
// (zero at launch) into its shared memory; a cluster barrier publishes it,
// every CTA reads it through distributed shared memory, and a second barrier
// keeps rank 0 from overwriting it (or exiting) before all four have read
// it.  No cluster waits for any other.
__global__ void __launch_bounds__(quarter::kT, 3) k_batch_encrypt_quarter(const JobDesc* __restrict__ jobs,
                                                                          const EncPacket* __restrict__ packets,
                                                                          int n_packets, int* counter) {
  extern __shared__ u64 sm[];
  __shared__ int s_next;
  const unsigned j = quarter::cluster_rank();
  const unsigned next0 = quarter::map_rank(&s_next, 0);
  for (;;) {
    if (j == 0 && threadIdx.x == 0) s_next = atomicAdd(counter, 1);
    quarter::cluster_sync();
    const int p = ld_cluster_s32(next0);
    quarter::cluster_sync();
    if (p >= n_packets) break;
    const EncPacket pk = packets[p];
    const JobDesc& J = jobs[pk.job];
    const bool relax = J.P.q[pk.prime] < kRelaxLimit;
    if (J.zinc) {
      if (relax) batch_quarter<true, true>(J, pk, j, sm);
      else batch_quarter<true, false>(J, pk, j, sm);
    } else {
      if (relax) batch_quarter<false, true>(J, pk, j, sm);
      else batch_quarter<false, false>(J, pk, j, sm);
    }
  }
}

cudaLaunchConfig_t batch_quarter_config(int clusters, cudaStream_t st, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(4 * (unsigned)clusters);
  cfg.blockDim = dim3(quarter::kT);
  cfg.dynamicSmemBytes = sizeof(u64) * quarter::kQ;
  cfg.stream = st;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 4;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

}  // namespace

cudaError_t batch_quarter_attributes() {
  return cudaFuncSetAttribute(k_batch_encrypt_quarter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(sizeof(u64) * quarter::kQ));
}

// Clusters of the persistent 2^15 kernel that fit on the device at once (the
// attribute must be set first); at least 1.
cudaError_t batch_quarter_clusters(int* clusters) {
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = batch_quarter_config(1, 0, attr);
  int n = 0;
  cudaError_t e = cudaOccupancyMaxActiveClusters(&n, (void*)k_batch_encrypt_quarter, &cfg);
  *clusters = n > 0 ? n : 1;
  return e;
}

// Capturable: the attribute is set beforehand (batch_quarter_attributes).
cudaError_t launch_batch_encrypt_quarter(const JobDesc* jobs, const EncPacket* packets, int n_packets, int* counter,
                                         int clusters, cudaStream_t st) {
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = batch_quarter_config(clusters, st, attr);
  return cudaLaunchKernelEx(&cfg, k_batch_encrypt_quarter, jobs, packets, n_packets, counter);
}

cudaError_t launch_encrypt_quarter(const DevParams& P, const EncArgs& A, bool zinc, uint32_t batch,
                                   cudaStream_t st) {
  if (batch == 0) return cudaSuccess;
  if (P.log_n != 15 || (!A.swap && batch > 65535u) || (A.swap && 4ull * batch > 0x7fffffffull))
    return cudaErrorInvalidValue;
  const dim3 grid = A.swap ? dim3(4 * batch, P.L) : dim3(4 * P.L, batch);
  return zinc ? quarter::launch(k_encrypt_quarter<true>, grid, st, P, A)
              : quarter::launch(k_encrypt_quarter<false>, grid, st, P, A);
}

}  // namespace zn
