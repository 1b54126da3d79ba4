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

// Launches in slices of at most 65535 limbs (the grid's y limit).
static cudaError_t launch_pack_dir(const DevParams& P, const PackArgs& A, uint32_t batch, bool pack, cudaStream_t st) {
  const int L = P.L, N = 1 << P.log_n;
  unsigned maxbits = 0;
  for (int i = 0; i < L; ++i) maxbits = A.bits[i] > maxbits ? A.bits[i] : maxbits;
  const unsigned per = 65535u / (2u * L);
  for (uint32_t b0 = 0; b0 < batch; b0 += per) {
    const uint32_t nb = batch - b0 < per ? batch - b0 : per;
    if (pack) {
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

}  // namespace zn
