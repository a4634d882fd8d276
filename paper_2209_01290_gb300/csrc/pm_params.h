// pm_params.h -- host-side number theory and table construction for plans.
#pragma once
#include <cstdint>

#include "pm_types.h"

namespace pm {
namespace host {

uint64_t pow_mod(uint64_t base, uint64_t exp, uint64_t q);
bool is_prime_u64(uint64_t n);
uint32_t bit_length(uint64_t x);
// The `count` largest primes q < 2^qbits with q = 1 (mod 2N), descending.
// Returns how many were found.
int largest_ntt_primes(uint32_t log2n, uint32_t qbits, uint32_t count, uint64_t* out);
// psi for q by the fixed search rule; 0 if q is not = 1 mod 2N or none found.
uint64_t default_psi(uint64_t q, uint32_t log2n);
// Limb constants and twiddle tables (host arrays of N entries).
// halving: the inverse table holds Psi^-1_br[i] / 2 (per-stage halving of
// Sec. III-A); otherwise Psi^-1_br[i] and 1/N is folded into the last stage.
void build_limb(uint32_t log2n, uint64_t q, uint64_t psi, bool halving, LimbConst* lc,
                TwPair* twf, TwPair* twi);
// Constants for the fused polynomial multiplication (Algorithm 8): its pair
// step already carries the 1/2 of the omitted first GS stage, so the scale
// folded into the last stage becomes 2/N (N^-1 and Psi^-1_br[1] N^-1 times 2).
void fused_limb(const LimbConst& in, LimbConst* out);
// The same for 32-bit words (q < 2^30; companions floor(w * 2^32 / q)).
void build_limb32(uint32_t log2n, uint64_t q, uint64_t psi, bool halving, LimbConst32* lc,
                  TwPair32* twf, TwPair32* twi);
void fused_limb32(const LimbConst32& in, LimbConst32* out);

}  // namespace host
}  // namespace pm
