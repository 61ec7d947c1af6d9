// Modular arithmetic over GF(p), 2 <= p < 2^31, for the device kernels.
//
// Residues are stored as uint32 in [0, p).  Products use Montgomery's
// reduction (P. L. Montgomery, "Modular multiplication without trial
// division", Math. Comp. 44, 1985) with R = 2^32: for t < p R,
// REDC(t) = t R^{-1} mod p.  A multiplier kept in Montgomery form (c R mod p)
// times a plain residue w gives REDC(cR * w) = c w mod p with one reduction.
// p = 2 (even, no Montgomery inverse) is handled by bit operations.
#pragma once
#include <stdint.h>

struct FieldP {
  uint32_t p;
  uint32_t pneg_inv;  // -p^{-1} mod 2^32 (odd p), 0 for p = 2
  uint32_t r2;        // 2^64 mod p
  uint32_t is2;       // p == 2
};

__host__ inline FieldP make_field(uint32_t p) {
  FieldP F;
  F.p = p;
  F.is2 = (p == 2);
  if (p == 2) {
    F.pneg_inv = 0;
    F.r2 = 0;
    return F;
  }
  // Newton iteration for p^{-1} mod 2^32: x <- x (2 - p x), 5 steps from x = p.
  uint32_t x = p;
  for (int i = 0; i < 5; ++i) x *= 2u - p * x;
  F.pneg_inv = 0u - x;
  uint64_t r = ((uint64_t)1 << 32) % p;
  F.r2 = (uint32_t)((unsigned __int128)r * r % p);
  return F;
}

__device__ __forceinline__ uint32_t f_redc(uint64_t t, const FieldP& F) {
  uint32_t m = (uint32_t)t * F.pneg_inv;
  uint64_t u = (t + (uint64_t)m * F.p) >> 32;
  uint32_t r = (uint32_t)u;
  return r >= F.p ? r - F.p : r;
}

// c -> c R mod p
__device__ __forceinline__ uint32_t f_to_mont(uint32_t c, const FieldP& F) {
  if (F.is2) return c & 1u;
  return f_redc((uint64_t)c * F.r2, F);
}

// (cR) * w -> c w mod p ; cm in Montgomery form, w plain
__device__ __forceinline__ uint32_t f_mul_mont(uint32_t cm, uint32_t w, const FieldP& F) {
  if (F.is2) return cm & w;
  return f_redc((uint64_t)cm * w, F);
}

// a * b mod p, both plain
__device__ __forceinline__ uint32_t f_mul(uint32_t a, uint32_t b, const FieldP& F) {
  if (F.is2) return a & b;
  return f_redc((uint64_t)f_redc((uint64_t)a * b, F) * F.r2, F);
}

__device__ __forceinline__ uint32_t f_sub(uint32_t a, uint32_t b, const FieldP& F) {
  return a >= b ? a - b : a + F.p - b;
}

__device__ __forceinline__ uint32_t f_add(uint32_t a, uint32_t b, const FieldP& F) {
  uint32_t s = a + b;  // < 2^32 since a, b < 2^31
  return s >= F.p ? s - F.p : s;
}

// x mod p for any 64-bit x (slow path; used once per output element).
__device__ __forceinline__ uint32_t f_reduce64(uint64_t x, const FieldP& F) {
  return (uint32_t)(x % F.p);
}

// Inverse of a in [1, p) by the extended Euclidean algorithm.
__device__ inline uint32_t f_inv_euclid(uint32_t a, uint32_t p) {
  int64_t t0 = 0, t1 = 1;
  uint32_t r0 = p, r1 = a;
  while (r1 != 0) {
    uint32_t q = r0 / r1;
    uint32_t rr = r0 - q * r1;
    r0 = r1;
    r1 = rr;
    int64_t tt = t0 - (int64_t)q * t1;
    t0 = t1;
    t1 = tt;
  }
  return (uint32_t)(t0 < 0 ? t0 + (int64_t)p : t0);
}

// Inverse through the per-p table when one exists (p below the table limit),
// else by Euclid.
__device__ __forceinline__ uint32_t f_inv(uint32_t a, const FieldP& F, const uint32_t* table) {
  if (F.is2) return 1u;
  if (table) return __ldg(table + a);
  return f_inv_euclid(a, F.p);
}
