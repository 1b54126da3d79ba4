// Encoder (fixed-point FFT with exact 128-bit products), inverse NTT,
// decryption (Eq. 10), decoding (FP64), homomorphic addition and small helpers.
#include "zn_kernels.h"

namespace zn {

// ------------------------------------------------------------------ encode

// Encoder core: one block per slot vector.  (re, im) hold h = N/4 int64
// each, in shared memory.  Fixed-point procedure (bit-reproducible):
//   0. block scale F = 60 - log2 N - e, 2^(e-1) <= max|z| < 2^e;
//      Y_j = floor(z_j 2^F + 1/2);
//   1-2. g_s = y[2s] + i y[2s+1] (y[t_j] = Y_j) in bit-reversed order, radix-2
//      DIT of length h with Q62 twiddles (fft_dit_q62);
//   3. split: X2[k] = (sr, si) + cmul((di, -dr), V), V = W[4k] (k < h) or -1;
//   4. twist S2[k] = cmul(X2[k], W[k]);
//   5. m_k = floor(2^d S2[k].re + 1/2), m_{k+n} likewise with .im, d = s - F - 1.
// out(k, m_k, m_{k+n}) is called once for every k < n.  A non-finite slot or
// |m| >= 2^62 latches the overflow status and gives zero coefficients.
template <class Out>
__device__ __forceinline__ void encode_core(const DevParams& P, const double* __restrict__ z, uint32_t n_slots,
                                            i64* re, i64* im, Out& out) {
  __shared__ u64 s_max[32];
  const int log_n = P.log_n, N = 1 << log_n, n = N >> 1, h = n >> 1, lh = log_n - 2;
  const u64 kAbs = ~(1ull << 63);
  // raw bit patterns in bit-reversed order (missing slots zero), and max |z|
  // (as ordered bits): the slots are read in order (coalesced) and scattered
  // to their FFT input places
  if (n_slots < (uint32_t)n) {
    for (int r = threadIdx.x; r < h; r += blockDim.x) {
      re[r] = 0;
      im[r] = 0;
    }
    __syncthreads();
  }
  u64 mx = 0;
  for (int j = threadIdx.x; j < (int)n_slots; j += blockDim.x) {
    const u64 bits = (u64)__double_as_longlong(__ldg(z + j));
    const int pos = __ldg(P.pos_of_slot + j);
    if (pos < h) re[pos] = (i64)bits;
    else im[pos - h] = (i64)bits;
    mx = max(mx, bits & kAbs);
  }
#pragma unroll
  for (int off = 16; off; off >>= 1) mx = max(mx, (u64)__shfl_xor_sync(0xffffffffu, (unsigned long long)mx, off));
  if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    u64 v = threadIdx.x < (blockDim.x + 31) / 32 ? s_max[threadIdx.x] : 0ull;
#pragma unroll
    for (int off = 16; off; off >>= 1) v = max(v, (u64)__shfl_xor_sync(0xffffffffu, (unsigned long long)v, off));
    if (threadIdx.x == 0) s_max[0] = v;
  }
  __syncthreads();
  const u64 M = s_max[0];
  const int mex = (int)(M >> 52);
  if (M == 0 || mex == 0x7FF) {                 // zero vector, or a non-finite slot
    if (mex == 0x7FF && threadIdx.x == 0) atomicOr(P.status, kStatusOverflow);
    for (int k = threadIdx.x; k < n; k += blockDim.x) out(k, (i64)0, (i64)0);
    return;
  }
  const int e = mex ? mex - 1022 : (64 - __clzll((long long)(M & ((1ull << 52) - 1)))) - 1074;
  const int F = 60 - log_n - e;     // the ring's slot count: zero padding changes nothing
  for (int r = threadIdx.x; r < h; r += blockDim.x) {
    re[r] = to_fixed((u64)re[r], F);
    im[r] = to_fixed((u64)im[r], F);
  }
  __syncthreads();
  fft_dit_q62(re, im, lh, log_n, P.etq);
  const int d = P.log2_delta + 1 - log_n - F - 1;
  auto emit = [&](int k, i64 xr, i64 xi) {
    i64 sr, si, a, b;
    cmul_q62(xr, xi, __ldg(P.etq + k), sr, si);
    const bool ok = from_fixed(sr, d, a) & from_fixed(si, d, b);
    if (!ok) {
      atomicOr(P.status, kStatusOverflow);
      a = 0;
      b = 0;
    }
    out(k, a, b);
  };
  // split: X2[k] from G[k] and G[h-k] (G[h] = G[0]); X2[n-k] = conj(X2[k])
  for (int k = threadIdx.x; k <= h; k += blockDim.x) {
    const int ka = k == h ? 0 : k, kb = k == 0 ? 0 : h - k;
    const i64 ar = re[ka], ai = im[ka], br = re[kb], bi = im[kb];
    const i64 sr = ar + br, si = ai - bi, dr = ar - br, di = ai + bi;
    const longlong2 v = k < h ? __ldg(P.etq + 4 * k) : make_longlong2(-(1ll << 62), 0);
    i64 tr, ti;
    cmul_q62(di, -dr, v, tr, ti);
    const i64 xr = sr + tr, xi = si + ti;
    emit(k, xr, xi);
    if (k > 0 && k < h) emit(n - k, xr, -xi);
  }
}

__device__ __forceinline__ void encode_one(const DevParams& P, const double* __restrict__ z, uint32_t n_slots,
                                           i64* re, i64* im, i64* __restrict__ out) {
  const int n = 1 << (P.log_n - 1);
  auto st = [&](int k, i64 a, i64 b) {
    out[k] = a;
    out[k + n] = b;
  };
  encode_core(P, z, n_slots, re, im, st);
}

// The slot count of vector b: nv[b] (per-vector counts over rows of `stride`
// doubles; a count above stride latches kStatusRange and encodes zero) or the
// call's n_slots.
__device__ __forceinline__ uint32_t slots_of(const DevParams& P, const uint32_t* nv, uint32_t stride,
                                             uint32_t n_slots, size_t b) {
  if (!nv) return n_slots;
  const uint32_t k = __ldg(nv + b);
  if (k <= stride) return k;
  if (threadIdx.x == 0) atomicOr(P.status, kStatusRange);
  return 0;
}

// nv == nullptr: n_slots per vector, rows of n_slots; else rows of `stride`.
__global__ void k_encode_smem(DevParams P, const double* __restrict__ slots, uint32_t n_slots,
                              const uint32_t* __restrict__ nv, uint32_t stride, i64* __restrict__ out) {
  extern __shared__ i64 smi[];
  const int N = 1 << P.log_n, h = N >> 2;
  const size_t b = blockIdx.x;
  const uint32_t ns = slots_of(P, nv, stride, n_slots, b);
  encode_one(P, slots + b * (nv ? stride : n_slots), ns, smi, smi + h, out + b * N);
}

// -------------------------------------------------------------------- prep
// One block per ciphertext: encode the slots and draw all of the
// encryption's randomness once, for every prime (the integers are the same
// for all q_i):
//   vanilla (Eq. 8):    me = m + e0 (poly 1), small = [u (poly 0), e1 (poly 2)]
//   Zinc (Algorithm 1): me = m + e1' (poly 0), small = [e2' (poly 1)]
//   (me stored with the offset 2^62)
//   modulus-switched vanilla (MS): me = m + 2^62, small = [u, e0, e1] (polys
//     0, 1, 2; the noise enters before the division by the special prime, m
//     after it)
// chi block k yields coefficients k and k + N/2 -- the pair that the
// encoder's last loop produces at k.
// cdt: the chi thresholds and their bucket index, staged in shared memory by
// the calling kernel.
template <bool ZINC, bool MS = false>
__device__ __forceinline__ void prep_one(const DevParams& P, const PrepArgs& A, size_t b, i64* re, i64* im,
                                         const CdtTab* cdt) {
  static_assert(!(ZINC && MS), "the modulus-switched form is a vanilla encryption");
  const int N = 1 << P.log_n, n = N >> 1;
  const u64 ct = A.ct_index ? A.ct_index[b] : A.ct_index0 + b;
  i64* me = A.me + b * N;
  int8_t* sp = A.small + b * (MS ? 3 : 2) * (size_t)N;
  const unsigned tag_e = rand_tag(A.domain, ZINC ? 0 : 1, 0);
  const uint32_t ns = slots_of(P, A.n_slots_v, A.stride, A.n_slots, b);
  const double* z = A.slots + b * (A.n_slots_v ? A.stride : A.n_slots);
  // m first (kept apart from the sampler, which would otherwise share the
  // encoder's registers), then m + e once the block's stores are visible
  if (ns) {
    // MS: stored as m + 2^62 (non-negative), read back by the data primes as unsigned
    constexpr i64 off = MS ? (i64)kMsOffset : 0;
    auto st = [&](int k, i64 a, i64 c) {
      me[k] = a + off;
      me[k + n] = c + off;
    };
    encode_core(P, z, ns, re, im, st);
    __syncthreads();
  }
#pragma unroll 2
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const uint4 w = zn_rand(A.seed, (unsigned)k, tag_e, ct);
    if constexpr (MS) {
      if (!ns) {
        me[k] = (i64)kMsOffset;
        me[k + n] = (i64)kMsOffset;
      }
      sp[N + k] = (int8_t)cdt_lookup(w.x, w.y, *cdt);
      sp[N + k + n] = (int8_t)cdt_lookup(w.z, w.w, *cdt);
    } else {
      // m + e with the offset 2^62 (non-negative as an unsigned word; the
      // encryption units remove it with reduce_biased)
      const i64 a = ns ? me[k] : 0, c = ns ? me[k + n] : 0;
      me[k] = (i64)((u64)(a + cdt_lookup(w.x, w.y, *cdt)) + kMsOffset);
      me[k + n] = (i64)((u64)(c + cdt_lookup(w.z, w.w, *cdt)) + kMsOffset);
    }
  }
  if constexpr (!ZINC) {
    int8_t* e1p = sp + (MS ? 2 : 1) * (size_t)N;
    const unsigned tag_u = rand_tag(A.domain, 0, 0), tag_1 = rand_tag(A.domain, 2, 0);
#pragma unroll 2
    for (int blk = threadIdx.x; blk < N / 4; blk += blockDim.x) {
      const uint4 w = zn_rand(A.seed, (unsigned)blk, tag_u, ct);
      sp[blk] = (int8_t)ternary_of(w.x);
      sp[blk + N / 4] = (int8_t)ternary_of(w.y);
      sp[blk + N / 2] = (int8_t)ternary_of(w.z);
      sp[blk + 3 * N / 4] = (int8_t)ternary_of(w.w);
    }
#pragma unroll 2
    for (int blk = threadIdx.x; blk < n; blk += blockDim.x) {
      const uint4 w = zn_rand(A.seed, (unsigned)blk, tag_1, ct);
      e1p[blk] = (int8_t)cdt_lookup(w.x, w.y, *cdt);
      e1p[blk + n] = (int8_t)cdt_lookup(w.z, w.w, *cdt);
    }
  } else {
    const unsigned tag_2 = rand_tag(A.domain, 1, 0);
#pragma unroll 2
    for (int blk = threadIdx.x; blk < n; blk += blockDim.x) {
      const uint4 w = zn_rand(A.seed, (unsigned)blk, tag_2, ct);
      sp[blk] = (int8_t)cdt_lookup(w.x, w.y, *cdt);
      sp[blk + n] = (int8_t)cdt_lookup(w.z, w.w, *cdt);
    }
  }
}


// TB threads per block: 512 (two blocks per SM up to 2^14), or 1024 at
// 2^15, where the encoder's 128 KiB of shared memory allows one block per
// SM and the wider block doubles the warps that hide its latency (64
// registers either way).
template <bool ZINC, bool MS = false, int TB = 512>
__global__ void __launch_bounds__(TB, 1024 / TB) k_prep_smem(DevParams P, PrepArgs A) {
  extern __shared__ i64 smi[];
  __shared__ CdtTab s_cdt;
  stage_cdt_tab(P.cdt, s_cdt);
  const int h = 1 << (P.log_n - 2);
  prep_one<ZINC, MS>(P, A, blockIdx.x, smi, smi + h, &s_cdt);
}

// Persistent prep over a mixed work list: blocks take the next ciphertext
// from a global counter (zero at launch); each holds the encoder FFT of the
// batch's largest ring (4N bytes of shared memory: two 512-thread blocks per
// SM up to 2^14, one 1024-thread block at 2^15).
template <int TB>
__global__ void __launch_bounds__(TB, 1024 / TB) k_batch_prep(const JobDesc* __restrict__ jobs,
                                                       const PrepUnit* __restrict__ units, int n_units, int* counter) {
  extern __shared__ i64 smi[];
  __shared__ int s_next;
  __shared__ CdtTab s_cdt;
  for (;;) {
    if (threadIdx.x == 0) s_next = atomicAdd(counter, 1);
    __syncthreads();
    const int p = s_next;
    __syncthreads();
    if (p >= n_units) break;
    const PrepUnit u = units[p];
    const JobDesc& J = jobs[u.job];
    const int h = 1 << (J.P.log_n - 2);
    stage_cdt_tab(J.P.cdt, s_cdt);
    if (J.zinc) prep_one<true>(J.P, J.Pr, u.b, smi, smi + h, &s_cdt);
    else prep_one<false>(J.P, J.Pr, u.b, smi, smi + h, &s_cdt);
    __syncthreads();
  }
}

// ------------------------------------------------------------ inverse NTT
// Gentleman-Sande, bit-reversed input -> natural order, times N^-1; one
// block per polynomial, in shared memory or in place in global memory.
__device__ void intt_block(const DevParams& P, int i, u64* a) {
  const int log_n = P.log_n, N = 1 << log_n;
  const u64 q = P.q[i];
  const u64* itw = P.itw + (size_t)i * N;
  const u64* itws = P.itws + (size_t)i * N;
  for (int lt = 0; lt < log_n; ++lt) {
    const int t = 1 << lt, m = N >> (lt + 1);
    for (int id = threadIdx.x; id < N / 2; id += blockDim.x) {
      const int g = id >> lt, j = id & (t - 1);
      const int j1 = 2 * g * t + j;
      const u64 w = __ldg(itw + m + g), ws = __ldg(itws + m + g);
      const u64 U = a[j1], V = a[j1 + t];
      u64 s = U + V;
      if (s >= q) s -= q;
      const u64 d = U >= V ? U - V : U + q - V;
      u64 r = mul_shoup(d, w, ws, q);
      if (r >= q) r -= q;
      a[j1] = s;
      a[j1 + t] = r;
    }
    __syncthreads();
  }
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    const u64 r = mul_shoup(a[k], P.ninv[i], P.ninvs[i], q);
    a[k] = r >= q ? r - q : r;
  }
  __syncthreads();
}

__global__ void k_ntt_inv(DevParams P, u64* data, int use_smem) {
  extern __shared__ u64 sm[];
  const int i = blockIdx.x, N = 1 << P.log_n;
  u64* a = data + ((size_t)blockIdx.y * P.L + i) * N;
  if (use_smem) {
    for (int k = threadIdx.x; k < N; k += blockDim.x) sm[k] = a[k];
    __syncthreads();
    intt_block(P, i, sm);
    for (int k = threadIdx.x; k < N; k += blockDim.x) a[k] = sm[k];
  } else {
    intt_block(P, i, a);
  }
}

// -------------------------------------------------------------- decryption
// d = c0 + c1 * s-hat (NTT domain) per prime -> out [B][L][N]
__global__ void k_dec_mul(DevParams P, const u64* __restrict__ ct, const u64* __restrict__ sk, uint32_t batch,
                          u64* __restrict__ out) {
  const int N = 1 << P.log_n, L = P.L;
  const size_t total = (size_t)batch * L * N;
  for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < total; x += (size_t)gridDim.x * blockDim.x) {
    const size_t b = x / ((size_t)L * N), rem = x % ((size_t)L * N);
    const int i = (int)(rem / N);
    const u64 q = P.q[i];
    const u64 c0 = ct[b * 2 * L * N + rem], c1 = ct[b * 2 * L * N + (size_t)L * N + rem];
    const u64 p = mulmod_slow(c1, sk[rem], q);
    u64 s = c0 + p;
    if (s >= q) s -= q;
    out[x] = s;
  }
}

// CRT over the first two primes (or one), centred, then
// z_j = Delta^-1 m(zeta^(5^j)); one block per ciphertext.
__global__ void k_decode(DevParams P, const u64* __restrict__ coeffs, uint32_t n_slots, double* __restrict__ out,
                         double* __restrict__ work) {
  const int log_n = P.log_n, N = 1 << log_n, n = N >> 1, L = P.L;
  const size_t b = blockIdx.x;
  double* re = work + b * 2 * (size_t)n;
  double* im = re + n;
  const u64* r0 = coeffs + b * (size_t)L * N;
  const u64* r1 = r0 + N;
  const u64 q0 = P.q[0];
  const double* twr = P.etw;
  const double* twi = P.etw + N;
  auto coef = [&](int k) -> double {
    if (L == 1) {
      const u64 x = r0[k];
      return x > q0 / 2 ? -(double)(q0 - x) : (double)x;
    }
    const u64 q1 = P.q[1];
    const u64 a = r0[k], c = r1[k];
    const u64 am = a % q1;
    const u64 d = c >= am ? c - am : c + q1 - am;
    const u64 y = mulmod_slow(d, P.q0inv_mod_q1, q1);
    const u128 x = (u128)a + (u128)q0 * y;   // in [0, q0 q1)
    const u128 Q = (u128)q0 * q1;
    if (x > Q / 2) return -(double)(Q - x);
    return (double)x;
  };
  // w'_k = (m_k + i m_{k+n}) * conj(T[k]), placed bit-reversed
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const double mr = coef(k), mi = coef(k + n);
    const double wr = twr[k], wi = -twi[k];
    const int r = brv_bits(k, log_n - 1);
    re[r] = mr * wr - mi * wi;
    im[r] = mr * wi + mi * wr;
  }
  __syncthreads();
  fft_dit(re, im, log_n - 1, log_n, P.etw, true);
  const double inv_delta = ldexp(1.0, -P.log2_delta);
  // slot j sits at t_j = (5^j mod 2N - 1)/4; slot_of_t is the inverse map
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const int j = P.slot_of_t[t];
    if (j < (int)n_slots) out[b * n_slots + j] = re[t] * inv_delta;
  }
}

// ----------------------------------------------------------------- helpers
__global__ void k_add(DevParams P, const u64* a, const u64* b, uint32_t batch, u64* out) {
  const int N = 1 << P.log_n, L = P.L;
  const size_t total = (size_t)batch * 2 * L * N;
  for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < total; x += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)((x / N) % L);
    const u64 q = P.q[i];
    const u64 s = a[x] + b[x];
    out[x] = s >= q ? s - q : s;
  }
}

// Shoup companions: ws[x] = floor(w[x] 2^64 / q) for `polys` polynomials [polys][L][N]
__global__ void k_shoup(DevParams P, const u64* w, u64* ws, uint32_t polys) {
  const int N = 1 << P.log_n, L = P.L;
  const size_t total = (size_t)polys * L * N;
  for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < total; x += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)((x / N) % L);
    ws[x] = shoup_of(w[x], P.q[i]);
  }
}

// secret-key coefficients (int8) -> residues [L][N]
__global__ void k_sk_residues(DevParams P, const int8_t* s, u64* out) {
  const int N = 1 << P.log_n, L = P.L;
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < L * N; x += gridDim.x * blockDim.x)
    out[x] = small_res(s[x % N], P.q[x / N]);
}

// ================================================================ launchers

static unsigned grid_for(size_t total, int block) {
  size_t g = (total + block - 1) / block;
  return (unsigned)(g > 152 * 64 ? 152 * 64 : (g < 1 ? 1 : g));
}

cudaError_t launch_encode(const DevParams& P, const double* slots, uint32_t n_slots, uint32_t batch, i64* out,
                          cudaStream_t st) {
  if (batch == 0) return cudaSuccess;
  const int h = 1 << (P.log_n - 2);
  const int block = h / 2 < 512 ? (h / 2 < 32 ? 32 : h / 2) : 512;
  const size_t smem = 2 * sizeof(i64) * (size_t)h;
  cudaError_t e = cudaFuncSetAttribute(k_encode_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_encode_smem<<<batch, block, smem, st>>>(P, slots, n_slots, nullptr, 0, out);
  return cudaGetLastError();
}

cudaError_t launch_encode_ragged(const DevParams& P, const double* slots, const uint32_t* nv, uint32_t stride,
                                 uint32_t batch, i64* out, cudaStream_t st) {
  if (batch == 0) return cudaSuccess;
  const int h = 1 << (P.log_n - 2);
  const int block = h / 2 < 512 ? (h / 2 < 32 ? 32 : h / 2) : 512;
  const size_t smem = 2 * sizeof(i64) * (size_t)h;
  cudaError_t e = cudaFuncSetAttribute(k_encode_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_encode_smem<<<batch, block, smem, st>>>(P, slots, 0, nv, stride, out);
  return cudaGetLastError();
}

template <bool ZINC, bool MS = false>
static cudaError_t prep_launch(const DevParams& P, const PrepArgs& A, uint32_t batch, cudaStream_t st) {
  const int h = 1 << (P.log_n - 2);
  const bool wide = P.log_n >= 15;
  const int block = wide ? 1024 : h / 2 < 512 ? (h / 2 < 32 ? 32 : h / 2) : 512;
  const size_t smem = (A.n_slots || A.n_slots_v) ? 2 * sizeof(i64) * (size_t)h : 0;
  auto kern = wide ? k_prep_smem<ZINC, MS, 1024> : k_prep_smem<ZINC, MS>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<batch, block, smem, st>>>(P, A);
  return cudaGetLastError();
}

cudaError_t launch_prep(const DevParams& P, const PrepArgs& A, bool zinc, uint32_t batch, cudaStream_t st) {
  if (batch == 0) return cudaSuccess;
  return zinc ? prep_launch<true>(P, A, batch, st) : prep_launch<false>(P, A, batch, st);
}

cudaError_t launch_prep_ms(const DevParams& P, const PrepArgs& A, uint32_t batch, cudaStream_t st) {
  if (batch == 0) return cudaSuccess;
  return prep_launch<false, true>(P, A, batch, st);
}

// 1024-thread blocks when the largest ring is 2^15 (more than 64 KiB each).
static bool batch_prep_wide(size_t smem) { return smem > (size_t)(64 << 10); }

cudaError_t launch_batch_prep(const JobDesc* jobs, const PrepUnit* units, int n_units, int* counter, int grid,
                              size_t smem, cudaStream_t st) {
  if (batch_prep_wide(smem)) k_batch_prep<1024><<<grid, 1024, smem, st>>>(jobs, units, n_units, counter);
  else k_batch_prep<512><<<grid, 512, smem, st>>>(jobs, units, n_units, counter);
  return cudaGetLastError();
}

// Blocks of the persistent prep that fit on one SM with `smem` bytes of
// dynamic shared memory (the attribute must be set first); at least 1.
cudaError_t batch_prep_blocks_per_sm(size_t smem, int* blocks) {
  int n = 0;
  const cudaError_t e = batch_prep_wide(smem)
                            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_prep<1024>, 1024, smem)
                            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_prep<512>, 512, smem);
  *blocks = n > 0 ? n : 1;
  return e;
}

cudaError_t batch_set_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_batch_prep<512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(sizeof(i64) << 14));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_batch_prep<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(sizeof(i64) << 14));
  if (e != cudaSuccess) return e;
  return batch_encrypt_attributes();
}

cudaError_t launch_ntt_inv(const DevParams& P, u64* data, uint32_t batch, cudaStream_t st) {
  if (batch == 0) return cudaSuccess;
  const int N = 1 << P.log_n;
  const int use_smem = P.log_n <= 14;
  const size_t smem = use_smem ? sizeof(u64) * N : 0;
  cudaError_t e = cudaFuncSetAttribute(k_ntt_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int block = N / 2 < 512 ? (N / 2 < 32 ? 32 : N / 2) : 512;
  k_ntt_inv<<<dim3(P.L, batch), block, smem, st>>>(P, data, use_smem);
  return cudaGetLastError();
}

cudaError_t launch_dec_mul(const DevParams& P, const u64* ct, const u64* sk, uint32_t batch, u64* out,
                           cudaStream_t st) {
  const size_t total = (size_t)batch * P.L << P.log_n;
  k_dec_mul<<<grid_for(total, 256), 256, 0, st>>>(P, ct, sk, batch, out);
  return cudaGetLastError();
}

cudaError_t launch_decode(const DevParams& P, const u64* coeffs, uint32_t batch, uint32_t n_slots, double* out,
                          double* work, cudaStream_t st) {
  if (batch == 0) return cudaSuccess;
  const int n = 1 << (P.log_n - 1);
  const int block = n / 2 < 256 ? (n / 2 < 32 ? 32 : n / 2) : 256;
  k_decode<<<batch, block, 0, st>>>(P, coeffs, n_slots, out, work);
  return cudaGetLastError();
}

cudaError_t launch_add(const DevParams& P, const u64* a, const u64* b, uint32_t batch, u64* out, cudaStream_t st) {
  const size_t total = (size_t)batch * 2 * P.L << P.log_n;
  k_add<<<grid_for(total, 256), 256, 0, st>>>(P, a, b, batch, out);
  return cudaGetLastError();
}

cudaError_t launch_shoup(const DevParams& P, const u64* w, u64* ws, uint32_t polys, cudaStream_t st) {
  const size_t total = (size_t)polys * P.L << P.log_n;
  k_shoup<<<grid_for(total, 256), 256, 0, st>>>(P, w, ws, polys);
  return cudaGetLastError();
}

cudaError_t launch_sk_residues(const DevParams& P, const int8_t* s, u64* out, cudaStream_t st) {
  const size_t total = (size_t)P.L << P.log_n;
  k_sk_residues<<<grid_for(total, 256), 256, 0, st>>>(P, s, out);
  return cudaGetLastError();
}

}  // namespace zn
