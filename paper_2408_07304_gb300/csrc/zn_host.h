// Host-side parameter tables (see zn_host.cpp).
#pragma once
#include <cstdint>

namespace zn {
typedef uint64_t u64;

u64 powmod(u64 b, u64 e, u64 q);
bool is_prime(u64 n);
int gen_primes(uint32_t log_n, const uint32_t* bits, uint32_t count, u64* out);
u64 find_psi(u64 q, uint32_t log_n);
u64 shoup(u64 w, u64 q);
void ntt_tables(u64 q, u64 psi, uint32_t log_n, u64* tw, u64* tws, u64* itw, u64* itws);
int encoder_twiddles(uint32_t log_n, double* re, double* im);
int encoder_twiddles_q62(uint32_t log_n, int64_t* c, int64_t* s);
int cdt_thresholds(u64 out[38]);
}  // namespace zn
