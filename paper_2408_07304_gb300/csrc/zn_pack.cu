// Packed ciphertext serialization: each residue of prime q_i stored in
// bits_i = bit length of q_i bits instead of a 64-bit word.  Per ciphertext,
// component c (0, 1), then prime i: the limb's N residues as one
// little-endian bit stream (residue j at bits [j bits_i, (j + 1) bits_i)),
// ceil(N bits_i / 64) words, the last one zero-padded.  For the 60 + 6 x 50
// + 60-bit chain this is 420 / 512 of the plain [2][L][N] words: the bytes a
// ciphertext costs on a host link or a network.  Both directions are
// elementwise and HBM-bound; neither changes a value.
#include "zn_kernels.h"

namespace zn {

// Output word w of limb y = (b, c, i): OR of the residues that overlap bits
// [64 w, 64 w + 64) of the limb's stream -- at most ceil(64 / bits) + 1 <= 5
// of them (the host admits 17 <= bits <= 62), loaded independently.  Bit
// positions stay below N bits <= 2^15 * 62 < 2^32.
__global__ void __launch_bounds__(256) k_ct_pack(DevParams P, PackArgs A, uint32_t b0) {
  const int L = P.L, N = 1 << P.log_n;
  const size_t y = blockIdx.y;
  const size_t b = b0 + y / (2 * L);
  const int c = (int)(y / L) % 2, i = (int)(y % L);
  const unsigned bits = A.bits[i];
  const unsigned w = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned words = ((unsigned)N * bits + 63) / 64;
  if (w >= words) return;
  const u64* src = A.ct + ((b * 2 + c) * L + i) * (size_t)N;
  u64* dst = A.packed + b * 2 * A.cwords + c * A.cwords + A.woff[i];
  const unsigned bit0 = w * 64u;
  const unsigned j0 = bit0 / bits;
  const unsigned sh = bit0 - j0 * bits;                 // residue j0 starts sh bits before the word
  u64 out = __ldg(src + j0) >> sh;
  unsigned s = j0 * bits + bits - bit0;                 // position of residue j0 + 1 in the word
#pragma unroll
  for (unsigned k = 1; k < 5; ++k, s += bits)
    if (s < 64 && j0 + k < (unsigned)N) out |= __ldg(src + j0 + k) << s;
  dst[w] = out;
}

// Residue j of limb y: bits [j bits, (j + 1) bits) of the stream (at most two
// words); a value not below q_i latches kStatusRange and is written as read.
__global__ void __launch_bounds__(256) k_ct_unpack(DevParams P, PackArgs A, uint32_t b0) {
  const int L = P.L, N = 1 << P.log_n;
  const size_t y = blockIdx.y;
  const size_t b = b0 + y / (2 * L);
  const int c = (int)(y / L) % 2, i = (int)(y % L);
  const unsigned j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= (unsigned)N) return;
  const unsigned bits = A.bits[i];
  const u64* src = A.packed + b * 2 * A.cwords + c * A.cwords + A.woff[i];
  const unsigned bit = j * bits, w = bit >> 6, s = bit & 63;
  u64 v = __ldg(src + w) >> s;
  if (s + bits > 64) v |= __ldg(src + w + 1) << (64 - s);
  v &= (1ull << bits) - 1;                              // bits <= 62
  if (v >= P.q[i]) atomicOr(P.status, kStatusRange);
  A.ct[((b * 2 + c) * L + i) * (size_t)N + j] = v;
}

// ------------------------------------------------ bulk-copy (TMA) tiles
// A tile is 1024 residues of one limb: 8 KiB of residues, exactly 16 bits_i
// words of the limb's stream (1024 bits_i is a multiple of 64), so tiles
// never share a word.  A block moves its input tile into shared memory with
// one cp.async.bulk, completed on an mbarrier, and writes its outputs with
// coalesced stores.  Every address is 16-byte aligned when N >= 1024 and the
// two base pointers are (the host checks): limbs start at multiples of
// 8N bytes (plain) or (N/64) bits_i >= 16 words (packed).
constexpr int kTileRes = 1024;

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(u64* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void tile_load(void* dst, const void* src, unsigned bytes, u64* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}

// Waits for phase 0 of the barrier, at most `tries` polls (the default:
// about a second, each try_wait also suspending for a while); false if it
// gave up.
constexpr unsigned kTileWaitTries = 1u << 20;

__device__ __forceinline__ bool tile_wait(u64* bar, unsigned tries = kTileWaitTries) {
  for (unsigned it = 0; it < tries; ++it) {
    unsigned ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(smem_u32(bar)) : "memory");
    if (ok) return true;
  }
  return false;
}

// A wait that gave up latches kStatusTimeout, waits once more (bounded) for
// the copy still in flight, and the block returns without writing.
__device__ __forceinline__ bool tile_arrived(const DevParams& P, u64* bar, unsigned tries = kTileWaitTries) {
  if (tile_wait(bar, tries)) return true;
  if (threadIdx.x == 0) atomicOr(P.status, kStatusTimeout);
  tile_wait(bar, tries);
  return false;
}

// The timeout path on its own: a barrier that nothing arrives on (no copy
// is issued), waited on by the same code as the tiles with a limit of
// `tries` polls; the wait gives up, latches kStatusTimeout and the block
// returns.
__global__ void __launch_bounds__(32) k_wait_probe(DevParams P, unsigned tries) {
  __shared__ __align__(8) u64 s_bar;
  if (threadIdx.x == 0) mbar_init(&s_bar);
  __syncthreads();
  tile_arrived(P, &s_bar, tries);
}

// grid (N / 1024, limbs); tile x of limb y = (b, c, i)
__global__ void __launch_bounds__(256) k_ct_pack_tile(DevParams P, PackArgs A, uint32_t b0) {
  __shared__ __align__(128) u64 s_in[kTileRes];
  __shared__ __align__(8) u64 s_bar;
  const int L = P.L, N = 1 << P.log_n;
  const size_t y = blockIdx.y;
  const size_t b = b0 + y / (2 * L);
  const int c = (int)(y / L) % 2, i = (int)(y % L);
  const unsigned bits = A.bits[i], nw = 16u * bits;
  const u64* src = A.ct + ((b * 2 + c) * L + i) * (size_t)N + (size_t)blockIdx.x * kTileRes;
  u64* dst = A.packed + b * 2 * A.cwords + c * A.cwords + A.woff[i] + (size_t)blockIdx.x * nw;
  if (threadIdx.x == 0) mbar_init(&s_bar);
  __syncthreads();
  if (threadIdx.x == 0) tile_load(s_in, src, sizeof(u64) * kTileRes, &s_bar);
  if (!tile_arrived(P, &s_bar)) return;
  for (unsigned w = threadIdx.x; w < nw; w += blockDim.x) {
    const unsigned bit0 = w * 64u;
    const unsigned j0 = bit0 / bits;
    const unsigned sh = bit0 - j0 * bits;
    u64 out = s_in[j0] >> sh;
    unsigned s = j0 * bits + bits - bit0;
#pragma unroll
    for (unsigned k = 1; k < 5; ++k, s += bits)
      if (s < 64 && j0 + k < (unsigned)kTileRes) out |= s_in[j0 + k] << s;
    dst[w] = out;
  }
}

// grid (N / 1024, limbs): the 16 bits_i words of tile x back to 1024 residues
__global__ void __launch_bounds__(256) k_ct_unpack_tile(DevParams P, PackArgs A, uint32_t b0) {
  __shared__ __align__(128) u64 s_in[16 * 62];
  __shared__ __align__(8) u64 s_bar;
  const int L = P.L, N = 1 << P.log_n;
  const size_t y = blockIdx.y;
  const size_t b = b0 + y / (2 * L);
  const int c = (int)(y / L) % 2, i = (int)(y % L);
  const unsigned bits = A.bits[i];
  const u64* src = A.packed + b * 2 * A.cwords + c * A.cwords + A.woff[i] + (size_t)blockIdx.x * 16u * bits;
  u64* dst = A.ct + ((b * 2 + c) * L + i) * (size_t)N + (size_t)blockIdx.x * kTileRes;
  if (threadIdx.x == 0) mbar_init(&s_bar);
  __syncthreads();
  if (threadIdx.x == 0) tile_load(s_in, src, sizeof(u64) * 16u * bits, &s_bar);
  if (!tile_arrived(P, &s_bar)) return;
  const u64 q = P.q[i], mask = (1ull << bits) - 1;
  for (unsigned j = threadIdx.x; j < (unsigned)kTileRes; j += blockDim.x) {
    const unsigned bit = j * bits, w = bit >> 6, s = bit & 63;
    u64 v = s_in[w] >> s;
    if (s + bits > 64) v |= s_in[w + 1] << (64 - s);
    v &= mask;
    if (v >= q) atomicOr(P.status, kStatusRange);
    dst[j] = v;
  }
}

// Launches in slices of at most 65535 limbs (the grid's y limit).
static cudaError_t launch_pack_dir(const DevParams& P, const PackArgs& A, uint32_t batch, bool pack, cudaStream_t st) {
  const int L = P.L, N = 1 << P.log_n;
  unsigned maxbits = 0;
  for (int i = 0; i < L; ++i) maxbits = A.bits[i] > maxbits ? A.bits[i] : maxbits;
  const bool tiles = N >= kTileRes && (((uintptr_t)A.ct | (uintptr_t)A.packed) & 15) == 0;
  const unsigned per = 65535u / (2u * L);
  for (uint32_t b0 = 0; b0 < batch; b0 += per) {
    const uint32_t nb = batch - b0 < per ? batch - b0 : per;
    if (tiles) {
      const dim3 grid(N / kTileRes, nb * 2 * L);
      if (pack) k_ct_pack_tile<<<grid, 256, 0, st>>>(P, A, b0);
      else k_ct_unpack_tile<<<grid, 256, 0, st>>>(P, A, b0);
    } else if (pack) {
      const unsigned words = (unsigned)(((u64)N * maxbits + 63) / 64);
      k_ct_pack<<<dim3((words + 255) / 256, nb * 2 * L), 256, 0, st>>>(P, A, b0);
    } else {
      k_ct_unpack<<<dim3((N + 255) / 256, nb * 2 * L), 256, 0, st>>>(P, A, b0);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_ct_pack(const DevParams& P, const PackArgs& A, uint32_t batch, cudaStream_t st) {
  return batch ? launch_pack_dir(P, A, batch, true, st) : cudaSuccess;
}

cudaError_t launch_ct_unpack(const DevParams& P, const PackArgs& A, uint32_t batch, cudaStream_t st) {
  return batch ? launch_pack_dir(P, A, batch, false, st) : cudaSuccess;
}

cudaError_t launch_wait_probe(const DevParams& P, unsigned tries, cudaStream_t st) {
  k_wait_probe<<<1, 32, 0, st>>>(P, tries);
  return cudaGetLastError();
}

}  // namespace zn
