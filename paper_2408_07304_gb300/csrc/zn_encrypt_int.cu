// BFV (paper Eq. 12) and BGV (Eq. 13) public-key encryption and their Zinc
// forms (Section "Scheme Flexibility"), for coefficient plaintexts m in
// R_t = Z_t[X]/(X^N + 1):
//   BFV vanilla:  c0 = pk0 u + e0 + Delta m,   c1 = pk1 u + e1      Delta = floor(Q/t)
//   BFV Zinc:     c0 = z0 + Delta m + e1',     c1 = z1 + e2'        z: CKKS's cached Enc(0)
//   BGV vanilla:  c0 = pk0 u + t e0 + m,       c1 = pk1 u + t e1    pk0 = -a s + t e
//   BGV Zinc:     c0 = z0 + m + t e1',         c1 = z1 + t e2'      z: a BGV Enc(0)
// The units are the functor-driven ones of zn_encrypt_fn.cuh: Delta m and
// t e are one Shoup product by a per-prime constant (Delta mod q_i, t mod
// q_i); BGV's m + t e_a is one int64 per coefficient from the prep kernel.
// Decryption: Dec (Eq. 10) per prime, inverse NTT, then the scale-and-round
// (BFV) or centred reduction (BGV) from the residues (k_int_decode).
// Rings 2^10..2^15, in the launch shapes of the plain encryption's default
// kernels.
#include "zn_encrypt_fn.cuh"
#include "zn_pair.cuh"
#include "zn_quarter.cuh"

namespace zn {

// -------------------------------------------------------------------- prep
// One block per ciphertext.  Sampling tags as the CKKS path: vanilla u
// (poly 0), e0 (poly 1), e1 (poly 2); Zinc e1' (poly 0), e2' (poly 1).
template <bool BGV, bool ZINC>
__global__ void __launch_bounds__(256) k_prep_int(DevParams P, IntPrepArgs A) {
  __shared__ CdtTab s_cdt;
  stage_cdt_tab(P.cdt, s_cdt);
  __syncthreads();
  const int N = 1 << P.log_n, n = N >> 1;
  const size_t b = blockIdx.x;
  const u64 ct = A.ct_index ? A.ct_index[b] : A.ct_index0 + b;
  const i64 t = (i64)A.t;
  i64* me = A.me + b * N;
  int8_t* sp = A.small + b * (ZINC ? 2 : 3) * (size_t)N;
  int8_t* ea = sp + (ZINC ? 0 : N);
  int8_t* eb = sp + (ZINC ? N : 2 * (size_t)N);
  const i64* m = A.m ? A.m + b * N : nullptr;
  const unsigned tag_a = rand_tag(A.domain, ZINC ? 0 : 1, 0), tag_b = rand_tag(A.domain, ZINC ? 1 : 2, 0);
  auto mod_t = [&](i64 x) {
    i64 r = x % t;
    return r < 0 ? r + t : r;
  };
#pragma unroll 1
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const uint4 w = zn_rand(A.seed, (unsigned)k, tag_a, ct);
    const int a0 = cdt_lookup(w.x, w.y, s_cdt), a1 = cdt_lookup(w.z, w.w, s_cdt);
    ea[k] = (int8_t)a0;
    ea[k + n] = (int8_t)a1;
    const i64 m0 = m ? mod_t(__ldg(m + k)) : 0, m1 = m ? mod_t(__ldg(m + k + n)) : 0;
    me[k] = BGV ? m0 + t * a0 : m0;
    me[k + n] = BGV ? m1 + t * a1 : m1;
  }
#pragma unroll 1
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const uint4 w = zn_rand(A.seed, (unsigned)k, tag_b, ct);
    eb[k] = (int8_t)cdt_lookup(w.x, w.y, s_cdt);
    eb[k + n] = (int8_t)cdt_lookup(w.z, w.w, s_cdt);
  }
  if constexpr (!ZINC) {
    const unsigned tag_u = rand_tag(A.domain, 0, 0);
#pragma unroll 1
    for (int blk = threadIdx.x; blk < N / 4; blk += blockDim.x) {
      const uint4 w = zn_rand(A.seed, (unsigned)blk, tag_u, ct);
      sp[blk] = (int8_t)ternary_of(w.x);
      sp[blk + N / 4] = (int8_t)ternary_of(w.y);
      sp[blk + N / 2] = (int8_t)ternary_of(w.z);
      sp[blk + 3 * N / 4] = (int8_t)ternary_of(w.w);
    }
  }
}

// ------------------------------------------------------------ unit inputs
// First component's input, in [0, 2q): BFV Delta m + e_a (me = m mod t < t),
// BGV m + t e_a (me, a signed int64).
template <bool BGV>
struct IntV0 {
  const i64* me;
  const int8_t* e;
  u64 q, mu, f, fs;
  __device__ __forceinline__ u64 operator()(int k) const {
    if constexpr (BGV) {
      return reduce_signed(__ldg(me + k), q, mu);
    } else {
      u64 x = mul_shoup((u64)__ldg(me + k), f, fs, q) + small_res(__ldg(e + k), q);   // [0, 3q)
      return x >= 2 * q ? x - q : x;
    }
  }
};

// Second component's input: BFV e_b, BGV t e_b.
template <bool BGV>
struct IntV1 {
  const int8_t* e;
  u64 q, f, fs;
  __device__ __forceinline__ u64 operator()(int k) const {
    const u64 x = small_res(__ldg(e + k), q);
    if constexpr (BGV) return mul_shoup(x, f, fs, q);
    return x;
  }
};

template <bool BGV, bool ZINC>
__device__ __forceinline__ void int_inputs(const DevParams& P, const IntArgs& A, int i, size_t b, int N,
                                           IntV0<BGV>& v0, IntV1<BGV>& v1) {
  const int8_t* sp = A.small + b * (ZINC ? 2 : 3) * (size_t)N;
  const int8_t* ea = sp + (ZINC ? 0 : N);
  const int8_t* eb = sp + (ZINC ? N : 2 * (size_t)N);
  v0 = IntV0<BGV>{A.me + b * N, ea, P.q[i], P.mu[i], A.f[i], A.fs[i]};
  v1 = IntV1<BGV>{eb, P.q[i], A.f[i], A.fs[i]};
}

template <int LOGN, int LOGPER, bool RELAX, int KM, bool BGV, bool ZINC>
__device__ __forceinline__ void int_unit_q(const DevParams& P, const IntArgs& A, int i, size_t b, u64* sm, int t) {
  constexpr int N = 1 << LOGN;
  const int L = P.L;
  FnLimb o;
  o.c0 = A.out + (b * 2 * L + i) * N;
  o.c1 = o.c0 + (size_t)L * N;
  o.k0 = A.key + (size_t)i * N;
  o.k1 = o.k0 + (size_t)L * N;
  o.k0s = ZINC ? nullptr : A.keys + (size_t)i * N;
  o.k1s = ZINC ? nullptr : o.k0s + (size_t)L * N;
  o.u = A.small + b * 3 * N;
  IntV0<BGV> v0;
  IntV1<BGV> v1;
  int_inputs<BGV, ZINC>(P, A, i, b, N, v0, v1);
  fn_unit_q<LOGN, LOGPER, RELAX, KM, ZINC, false>(P.twp + (size_t)i * N, P.q[i], o, v0, v1, sm, t);
}


// N = 2^15: output quarter j of prime i on a four-CTA cluster (zn_quarter.cuh).
template <bool RELAX, bool BGV, bool ZINC>
__device__ __forceinline__ void int_quarter_unit_q(const DevParams& P, const IntArgs& A, int i, unsigned j, size_t b,
                                                   u64* sm, int t) {
  using namespace quarter;
  const int L = P.L;
  const u64 q = P.q[i];
  const size_t off = (size_t)j * kQ;
  FnLimb o;
  o.c0 = A.out + (b * 2 * L + i) * kN + off;
  o.c1 = o.c0 + (size_t)L * kN;
  o.k0 = A.key + (size_t)i * kN + off;
  o.k1 = o.k0 + (size_t)L * kN;
  o.k0s = ZINC ? nullptr : A.keys + (size_t)i * kN + off;
  o.k1s = ZINC ? nullptr : o.k0s + (size_t)L * kN;
  o.u = A.small + b * 3 * kN;
  IntV0<BGV> v0;
  IntV1<BGV> v1;
  int_inputs<BGV, ZINC>(P, A, i, b, kN, v0, v1);
  const ulonglong2* tw = P.twp + (size_t)i * kN;
  auto gu = [&] { gen_i8<RELAX, true>(sm, t, j, o.u, tw, q); };
  auto g0 = [&] { gen_val<RELAX>(sm, t, j, v0, tw, q); };
  auto g1 = [&] { gen_val<RELAX>(sm, t, j, v1, tw, q); };
  unit<ZINC, RELAX>(sm, t, j, tw, q, o, gu, g0, g1);
}

// N = 2^14: output half h of prime i on a two-CTA cluster (zn_pair.cuh);
// vanilla writes its finished words with streaming stores (DRAM traffic
// 1.41x -> 1.10x of the ciphertext bytes, the same launch time).
template <bool RELAX, bool BGV, bool ZINC>
__device__ __forceinline__ void int_pair_unit_q(const DevParams& P, const IntArgs& A, int i, unsigned h, size_t b,
                                                u64* sm, int t) {
  using namespace pair;
  const int L = P.L;
  const u64 q = P.q[i];
  const size_t off = (size_t)h * kH;
  FnLimb o;
  o.c0 = A.out + (b * 2 * L + i) * kN + off;
  o.c1 = o.c0 + (size_t)L * kN;
  o.k0 = A.key + (size_t)i * kN + off;
  o.k1 = o.k0 + (size_t)L * kN;
  o.k0s = ZINC ? nullptr : A.keys + (size_t)i * kN + off;
  o.k1s = ZINC ? nullptr : o.k0s + (size_t)L * kN;
  o.u = A.small + b * 3 * kN;
  IntV0<BGV> v0;
  IntV1<BGV> v1;
  int_inputs<BGV, ZINC>(P, A, i, b, kN, v0, v1);
  const ulonglong2* tw = P.twp + (size_t)i * kN;
  auto gu = [&] { gen_i8<RELAX, true>(sm, t, h, o.u, tw, q); };
  auto g0 = [&] { gen_val<RELAX>(sm, t, h, v0, tw, q); };
  auto g1 = [&] { gen_val<RELAX>(sm, t, h, v1, tw, q); };
  unit<ZINC, RELAX, !ZINC>(sm, t, h, tw, q, o, gu, g0, g1);
}

// grid (2L, B), or (2B, L) when A.swap; cluster rank h owns half h
template <bool BGV, bool ZINC>
__global__ void __launch_bounds__(pair::kT, 3) k_encrypt_int_pair(DevParams P, IntArgs A) {
  extern __shared__ u64 sm[];
  const unsigned h = cluster::cluster_rank();
  const int i = A.swap ? (int)blockIdx.y : (int)(blockIdx.x >> 1);
  const size_t b = A.swap ? (size_t)(blockIdx.x >> 1) : blockIdx.y;
  if (P.q[i] < kRelaxLimit) int_pair_unit_q<true, BGV, ZINC>(P, A, i, h, b, sm, threadIdx.x);
  else int_pair_unit_q<false, BGV, ZINC>(P, A, i, h, b, sm, threadIdx.x);
}

// grid (4L, B), or (4B, L) when A.swap; cluster rank j owns quarter j
template <bool BGV, bool ZINC>
__global__ void __launch_bounds__(quarter::kT, 3) k_encrypt_int_quarter(DevParams P, IntArgs A) {
  extern __shared__ u64 sm[];
  const unsigned j = quarter::cluster_rank();
  const int i = A.swap ? (int)blockIdx.y : (int)(blockIdx.x >> 2);
  const size_t b = A.swap ? (size_t)(blockIdx.x >> 2) : blockIdx.y;
  if (P.q[i] < kRelaxLimit) int_quarter_unit_q<true, BGV, ZINC>(P, A, i, j, b, sm, threadIdx.x);
  else int_quarter_unit_q<false, BGV, ZINC>(P, A, i, j, b, sm, threadIdx.x);
}

// grid (L, B), or (B, L) when A.swap
template <int LOGN, int LOGPER, int MINB, int KM, bool BGV, bool ZINC>
__global__ void __launch_bounds__(NttShape<LOGN, LOGPER>::T, MINB) k_encrypt_int(DevParams P, IntArgs A) {
  extern __shared__ u64 sm[];
  const int i = A.swap ? blockIdx.y : blockIdx.x;
  const size_t b = A.swap ? blockIdx.x : blockIdx.y;
  if (P.q[i] < kRelaxLimit) int_unit_q<LOGN, LOGPER, true, KM, BGV, ZINC>(P, A, i, b, sm, threadIdx.x);
  else int_unit_q<LOGN, LOGPER, false, KM, BGV, ZINC>(P, A, i, b, sm, threadIdx.x);
}


// ------------------------------------------------------------- decoding
// x_i = coefficient residues of c0 + c1 s.  With Q/q_i and y_i = (Q/q_i)^-1 mod q_i:
//   BFV: t x / Q = sum_i x_i (I_i + r_i / q_i) (mod t), t y_i = I_i q_i + r_i, and
//        x_i r_i = A_i q_i + B_i, so m = sum_i (x_i I_i + A_i) + round(sum_i B_i / q_i) mod t;
//   BGV: v_i = x_i y_i mod q_i, the centred x = sum_i v_i Q/q_i - alpha Q with
//        alpha = round(sum_i v_i / q_i), so m = sum_i v_i (Q/q_i mod t) - alpha (Q mod t) mod t.
// The sums of fractions (below L) are taken in FP64; their rounding is
// unambiguous while the decryption noise leaves a margin (a tie cannot occur
// exactly: 2 t x = (2k + 1) Q has no solution for odd Q).
template <bool BGV>
__global__ void k_int_decode(DevParams P, IntDec D, const u64* __restrict__ x, uint32_t batch, i64* __restrict__ m) {
  const int N = 1 << P.log_n, L = P.L;
  const u64 t = D.t;
  const size_t total = (size_t)batch * N;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
    const size_t b = g / N;
    const int k = (int)(g % N);
    u64 acc = 0;
    double frac = 0.0;
    for (int i = 0; i < L; ++i) {
      const u64 q = P.q[i];
      const u64 xi = x[(b * L + i) * N + k];
      if constexpr (BGV) {
        const u64 v = mulmod_slow(xi, D.y[i], q);
        acc = (u64)(((u128)acc + (u128)(v % t) * D.Qit[i]) % t);
        frac += (double)v / (double)q;
      } else {
        const u128 pr = (u128)xi * D.r[i];
        const u64 Ai = (u64)(pr / q), Bi = (u64)(pr % q);
        acc = (u64)(((u128)acc + (u128)xi * D.It[i] + Ai % t) % t);
        frac += (double)Bi / (double)q;
      }
    }
    const u64 rnd = (u64)floor(frac + 0.5);
    u64 r;
    if constexpr (BGV) r = (acc + t - (u64)(((u128)(rnd % t) * D.Qt) % t)) % t;
    else r = (acc + rnd % t) % t;
    m[g] = (i64)r;
  }
}

__global__ void k_bgv_key(DevParams P, u64 t, const u64* __restrict__ ehat, u64* pk, u64* pks) {
  const int N = 1 << P.log_n, L = P.L;
  for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < (size_t)L * N; x += (size_t)gridDim.x * blockDim.x) {
    const u64 q = P.q[x / N];
    u64 v = pk[x] + mulmod_slow(ehat[x], (t - 1) % q, q);
    if (v >= q) v -= q;
    pk[x] = v;
    pks[x] = shoup_of(v, q);
  }
}

__global__ void k_residues(DevParams P, const i64* __restrict__ v, u64* out) {
  const int N = 1 << P.log_n, L = P.L;
  for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < (size_t)L * N; x += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(x / N);
    out[x] = reduce_signed(v[x % N], P.q[i], P.mu[i]);
  }
}

// ------------------------------------------------------------- launchers

static unsigned grid_of(size_t total) {
  size_t g = (total + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  return (unsigned)(g < 1 ? 1 : g);
}

template <bool BGV, bool ZINC>
static cudaError_t prep_int(const DevParams& P, const IntPrepArgs& A, uint32_t batch, cudaStream_t st) {
  k_prep_int<BGV, ZINC><<<batch, 256, 0, st>>>(P, A);
  return cudaGetLastError();
}

cudaError_t launch_prep_int(const DevParams& P, const IntPrepArgs& A, bool bgv, bool zinc, uint32_t batch,
                            cudaStream_t st) {
  if (batch == 0) return cudaSuccess;
  if (bgv) return zinc ? prep_int<true, true>(P, A, batch, st) : prep_int<true, false>(P, A, batch, st);
  return zinc ? prep_int<false, true>(P, A, batch, st) : prep_int<false, false>(P, A, batch, st);
}

template <int LOGN, int LOGPER, int MINB, int KM, bool BGV, bool ZINC>
static cudaError_t int_full(const DevParams& P, const IntArgs& A, uint32_t batch, cudaStream_t st) {
  using S = NttShape<LOGN, LOGPER>;
  const size_t smem = sizeof(u64) * S::N;
  auto kern = k_encrypt_int<LOGN, LOGPER, MINB, KM, BGV, ZINC>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 grid = A.swap ? dim3(batch, P.L) : dim3(P.L, batch);
  kern<<<grid, S::T, smem, st>>>(P, A);
  return cudaGetLastError();
}


template <bool BGV, bool ZINC>
static cudaError_t int_pair(const DevParams& P, const IntArgs& A, uint32_t batch, cudaStream_t st) {
  if ((!A.swap && batch > 65535u) || (A.swap && 2ull * batch > 0x7fffffffull)) return cudaErrorInvalidValue;
  const dim3 grid = A.swap ? dim3(2 * batch, P.L) : dim3(2 * P.L, batch);
  return pair::launch(k_encrypt_int_pair<BGV, ZINC>, grid, st, P, A);
}

template <bool BGV, bool ZINC>
static cudaError_t int_quarter(const DevParams& P, const IntArgs& A, uint32_t batch, cudaStream_t st) {
  if ((!A.swap && batch > 65535u) || (A.swap && 4ull * batch > 0x7fffffffull)) return cudaErrorInvalidValue;
  const dim3 grid = A.swap ? dim3(4 * batch, P.L) : dim3(4 * P.L, batch);
  return quarter::launch(k_encrypt_int_quarter<BGV, ZINC>, grid, st, P, A);
}

template <bool BGV, bool ZINC>
static cudaError_t int_dispatch(const DevParams& P, const IntArgs& A, uint32_t batch, cudaStream_t st) {
  switch (P.log_n) {
    case 10: return int_full<10, 5, 24, 3, BGV, ZINC>(P, A, batch, st);
    case 11: return int_full<11, 5, 12, 3, BGV, ZINC>(P, A, batch, st);
    case 12: return int_full<12, 5, 6, 3, BGV, ZINC>(P, A, batch, st);
    case 13: return int_full<13, 5, 3, 3, BGV, ZINC>(P, A, batch, st);
    case 14: return int_pair<BGV, ZINC>(P, A, batch, st);
    case 15: return int_quarter<BGV, ZINC>(P, A, batch, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_encrypt_int(const DevParams& P, const IntArgs& A, bool bgv, bool zinc, uint32_t batch,
                               cudaStream_t st) {
  if (batch == 0) return cudaSuccess;
  if (bgv) return zinc ? int_dispatch<true, true>(P, A, batch, st) : int_dispatch<true, false>(P, A, batch, st);
  return zinc ? int_dispatch<false, true>(P, A, batch, st) : int_dispatch<false, false>(P, A, batch, st);
}

cudaError_t launch_int_decode(const DevParams& P, const IntDec& D, bool bgv, const u64* x, uint32_t batch, i64* m,
                              cudaStream_t st) {
  if (batch == 0) return cudaSuccess;
  const unsigned g = grid_of((size_t)batch << P.log_n);
  if (bgv) k_int_decode<true><<<g, 256, 0, st>>>(P, D, x, batch, m);
  else k_int_decode<false><<<g, 256, 0, st>>>(P, D, x, batch, m);
  return cudaGetLastError();
}

cudaError_t launch_bgv_key(const DevParams& P, u64 t, const u64* ehat, u64* pk, u64* pks, cudaStream_t st) {
  k_bgv_key<<<grid_of((size_t)P.L << P.log_n), 256, 0, st>>>(P, t, ehat, pk, pks);
  return cudaGetLastError();
}

cudaError_t launch_residues(const DevParams& P, const i64* v, u64* out, cudaStream_t st) {
  k_residues<<<grid_of((size_t)P.L << P.log_n), 256, 0, st>>>(P, v, out);
  return cudaGetLastError();
}

}  // namespace zn
