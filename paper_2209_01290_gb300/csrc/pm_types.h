// pm_types.h -- plain data shared by host and device code.
#pragma once
#include <cstdint>

namespace pm {

// Per-limb constants, 64 bytes, read through the read-only path.
struct alignas(64) LimbConst {
  uint64_t q;        // modulus
  uint64_t two_q;    // 2q
  uint64_t half_q1;  // (q + 1) / 2: the odd-case addend of x/2 mod q (Sec. III-A)
  uint64_t mu;       // Algorithm 4: floor(2^(2m+1) / q)
  uint32_t m;        // len(q), bit length
  uint32_t sh1;      // m - 2   (Algorithm 4, step 1 shift)
  uint32_t sh2;      // m + 3   (Algorithm 4, step 2 shift)
  uint32_t halving;  // 1: the inverse table holds w/2 and every GS butterfly halves
  uint64_t ninv;     // N^-1 mod q            (1/N folded into the last GS stage)
  uint64_t ninv_p;   //   its Shoup companion
  uint64_t w1ninv;   // Psi^-1_br[1] * N^-1 mod q
  uint64_t w1ninv_p; //   its Shoup companion
};

// Twiddle factor with its Shoup companion floor(w * 2^64 / q), 16 bytes.
struct alignas(16) TwPair {
  uint64_t w;
  uint64_t wp;
};

// 32-bit words (moduli q < 2^30, Algorithm 4 with beta = 32): the same
// constants in 32-bit fields.  mu = floor(2^(2m+1) / q) < 2^(m+2) <= 2^32.
struct alignas(64) LimbConst32 {
  uint32_t q;
  uint32_t two_q;
  uint32_t half_q1;
  uint32_t mu;
  uint32_t m;
  uint32_t sh1;
  uint32_t sh2;
  uint32_t halving;
  uint32_t ninv;
  uint32_t ninv_p;
  uint32_t w1ninv;
  uint32_t w1ninv_p;
};

// 32-bit twiddle with its Shoup companion floor(w * 2^32 / q), 8 bytes.
struct alignas(8) TwPair32 {
  uint32_t w;
  uint32_t wp;
};

}  // namespace pm
