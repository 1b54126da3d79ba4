// Hot path at N = 2^14 (the throughput workload): one limb of one ciphertext
// per two-CTA cluster, one output half per CTA (zn_pair.cuh), with the
// epilogue
//   vanilla (Eq. 8):      c0 = pk0*u + NTT(m + e0),  c1 = pk1*u + NTT(e1)
//   Zinc (Algorithm 1):   c0' = z0 + NTT(m + e1'),   c1' = z1 + NTT(e2')
// on the integers the prep kernel prepared once per ciphertext.
#include "zn_pair.cuh"

namespace zn {
namespace {

template <bool ZINC, bool RELAX>
__device__ __forceinline__ void encrypt_pair_unit_q(const DevParams& P, const EncArgs& A, int i, unsigned h, size_t b,
                                                    u64* sm, int t) {
  using namespace pair;
  const int L = P.L;
  const u64 q = P.q[i];
  const ulonglong2* tw = P.twp + (size_t)i * kN;
  const size_t off = (size_t)h * kH;
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
  auto g_me = [&] { gen_val<RELAX>(sm, t, h, me, tw, q); };
  if constexpr (!ZINC) {
    // streaming stores for the finished words: the parked key products stay
    // in L2 (DRAM traffic 1.42x -> 1.08x of the algorithmic bytes, the
    // launch 0.3 % slower)
    auto g_u = [&] { gen_i8<RELAX, true>(sm, t, h, sp, tw, q); };
    auto g_e1 = [&] { gen_i8<RELAX, false>(sm, t, h, sp + kN, tw, q); };
    unit<false, RELAX, true>(sm, t, h, tw, q, o, g_u, g_me, g_e1);
  } else {
    auto g_e2 = [&] { gen_i8<RELAX, false>(sm, t, h, sp, tw, q); };
    unit<true, RELAX>(sm, t, h, tw, q, o, g_me, g_me, g_e2);
  }
}

// grid (2L, B), or (2B, L) when A.swap; the CTA of cluster rank h owns
// output half h
template <bool ZINC>
__global__ void __launch_bounds__(pair::kT, 3) k_encrypt_pair(DevParams P, EncArgs A) {
  extern __shared__ u64 sm[];
  const unsigned h = cluster::cluster_rank();
  const int i = A.swap ? (int)blockIdx.y : (int)(blockIdx.x >> 1);
  const size_t b = A.swap ? (size_t)(blockIdx.x >> 1) : blockIdx.y;
  // the relaxed/Harvey choice is uniform per unit, so both CTAs of a
  // cluster take the same branch and meet at the same barriers
  if (P.q[i] < kRelaxLimit) encrypt_pair_unit_q<ZINC, true>(P, A, i, h, b, sm, threadIdx.x);
  else encrypt_pair_unit_q<ZINC, false>(P, A, i, h, b, sm, threadIdx.x);
}

// ---------------------------------------- persistent mixed-ring launch
// Packet: one limb (ciphertext b0, prime `prime`) of a 2^14 job, run by one
// two-CTA cluster.  Rank 0 takes the next packet from a global counter (zero
// at launch) into its shared memory; a cluster barrier publishes it, both
// CTAs read it through distributed shared memory, and a second barrier keeps
// rank 0 from overwriting it (or exiting) before the other has read it.  No
// cluster waits for any other.
__device__ __forceinline__ int ld_cluster_s32(unsigned addr) {
  int v;
  asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}

__global__ void __launch_bounds__(pair::kT, 3) k_batch_encrypt_pair(const JobDesc* __restrict__ jobs,
                                                                    const EncPacket* __restrict__ packets,
                                                                    int n_packets, int* counter) {
  extern __shared__ u64 sm[];
  __shared__ int s_next;
  const unsigned h = cluster::cluster_rank();
  const unsigned next0 = cluster::map_rank(&s_next, 0);
  for (;;) {
    if (h == 0 && threadIdx.x == 0) s_next = atomicAdd(counter, 1);
    cluster::cluster_sync();
    const int p = ld_cluster_s32(next0);
    cluster::cluster_sync();
    if (p >= n_packets) break;
    const EncPacket pk = packets[p];
    const JobDesc& J = jobs[pk.job];
    const bool relax = J.P.q[pk.prime] < kRelaxLimit;
    if (J.zinc) {
      if (relax) encrypt_pair_unit_q<true, true>(J.P, J.E, pk.prime, h, pk.b0, sm, threadIdx.x);
      else encrypt_pair_unit_q<true, false>(J.P, J.E, pk.prime, h, pk.b0, sm, threadIdx.x);
    } else {
      if (relax) encrypt_pair_unit_q<false, true>(J.P, J.E, pk.prime, h, pk.b0, sm, threadIdx.x);
      else encrypt_pair_unit_q<false, false>(J.P, J.E, pk.prime, h, pk.b0, sm, threadIdx.x);
    }
  }
}

cudaLaunchConfig_t batch_pair_config(int clusters, cudaStream_t st, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2 * (unsigned)clusters);
  cfg.blockDim = dim3(pair::kT);
  cfg.dynamicSmemBytes = sizeof(u64) * pair::kH;
  cfg.stream = st;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

}  // namespace

cudaError_t batch_pair_attributes() {
  return cudaFuncSetAttribute(k_batch_encrypt_pair, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(sizeof(u64) * pair::kH));
}

// Clusters of the persistent 2^14 kernel that fit on the device at once (the
// attribute must be set first); at least 1.
cudaError_t batch_pair_clusters(int* clusters) {
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = batch_pair_config(1, 0, attr);
  int n = 0;
  cudaError_t e = cudaOccupancyMaxActiveClusters(&n, (void*)k_batch_encrypt_pair, &cfg);
  *clusters = n > 0 ? n : 1;
  return e;
}

// Capturable: the attribute is set beforehand (batch_pair_attributes).
cudaError_t launch_batch_encrypt_pair(const JobDesc* jobs, const EncPacket* packets, int n_packets, int* counter,
                                      int clusters, cudaStream_t st) {
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = batch_pair_config(clusters, st, attr);
  return cudaLaunchKernelEx(&cfg, k_batch_encrypt_pair, jobs, packets, n_packets, counter);
}

cudaError_t launch_encrypt_pair(const DevParams& P, const EncArgs& A, bool zinc, uint32_t batch, cudaStream_t st) {
  if (batch == 0) return cudaSuccess;
  if (P.log_n != 14 || (!A.swap && batch > 65535u) || (A.swap && 2ull * batch > 0x7fffffffull))
    return cudaErrorInvalidValue;
  const dim3 grid = A.swap ? dim3(2 * batch, P.L) : dim3(2 * P.L, batch);
  return zinc ? pair::launch(k_encrypt_pair<true>, grid, st, P, A) : pair::launch(k_encrypt_pair<false>, grid, st, P, A);
}

}  // namespace zn
