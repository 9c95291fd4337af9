// Modular arithmetic over Z_p for 31-bit primes p in (2^30, 2^31).
//
// Montgomery multiplication (P. L. Montgomery, "Modular multiplication
// without trial division", Math. Comp. 44, 1985) with R = 2^32: a residue a
// is held as aR mod p and REDC(t) = t R^{-1} mod p for 0 <= t < p R.  Because
// p < 2^31, a sum of two products of reduced residues, a b + c d < 2 p^2,
// stays below p R, so one REDC finishes a two-term dot product ("lazy"
// reduction).  Every helper returns a fully reduced value in [0, p).
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define RS_HD __host__ __device__ __forceinline__
#else
#define RS_HD inline
#endif

struct ModP {
  uint32_t p;     // the prime
  uint32_t pinv;  // -p^{-1} mod 2^32
  uint32_t r1;    // R mod p      (Montgomery form of 1)
  uint32_t r2;    // R^2 mod p    (converts a plain residue to Montgomery form)
};

RS_HD uint32_t rs_umin(uint32_t a, uint32_t b) { return a < b ? a : b; }

// REDC for 0 <= t < p * 2^32.
RS_HD uint32_t redc(uint64_t t, uint32_t p, uint32_t pinv) {
  uint32_t m = (uint32_t)t * pinv;
  uint64_t s = t + (uint64_t)m * p;  // low word is zero; s < 2 p 2^32 < 2^64
  uint32_t u = (uint32_t)(s >> 32);  // u < 2p
  return rs_umin(u, u - p);
}

RS_HD uint32_t mmul(uint32_t a, uint32_t b, const ModP &m) {
  return redc((uint64_t)a * b, m.p, m.pinv);
}

// a*b + c*d, one reduction (all inputs in [0, p)).
RS_HD uint32_t mmul2(uint32_t a, uint32_t b, uint32_t c, uint32_t d, const ModP &m) {
  return redc((uint64_t)a * b + (uint64_t)c * d, m.p, m.pinv);
}

RS_HD uint32_t madd(uint32_t a, uint32_t b, uint32_t p) {
  uint32_t s = a + b;  // < 2p < 2^32
  return rs_umin(s, s - p);
}

RS_HD uint32_t msub(uint32_t a, uint32_t b, uint32_t p) {
  uint32_t d = a - b;
  return rs_umin(d, d + p);
}

RS_HD uint32_t mneg(uint32_t a, uint32_t p) { return a ? p - a : 0u; }

// Plain residue (any 32-bit value) -> Montgomery form.
RS_HD uint32_t to_mont(uint32_t a, const ModP &m) {
  return redc((uint64_t)a * m.r2, m.p, m.pinv);  // a < 2^32, r2 < p: a r2 < p 2^32
}

RS_HD uint32_t from_mont(uint32_t a, const ModP &m) { return redc((uint64_t)a, m.p, m.pinv); }

// a^e in Montgomery form (a in Montgomery form).
RS_HD uint32_t mpow(uint32_t a, uint32_t e, const ModP &m) {
  uint32_t r = m.r1;
  while (e) {
    if (e & 1u) r = mmul(r, a, m);
    a = mmul(a, a, m);
    e >>= 1;
  }
  return r;
}

// Inverse by Fermat's little theorem, a^(p-2); a != 0 (Montgomery form in/out).
RS_HD uint32_t minv(uint32_t a, const ModP &m) { return mpow(a, m.p - 2u, m); }

// -p^{-1} mod 2^32 by Newton's iteration x <- x (2 - p x) (p odd; x = p is
// correct to 3 bits and every step doubles the correct bits).
RS_HD uint32_t neg_inv32(uint32_t p) {
  uint32_t x = p;
  for (int i = 0; i < 4; ++i) x *= 2u - p * x;
  return 0u - x;
}

RS_HD ModP make_modp(uint32_t p) {
  ModP m;
  m.p = p;
  m.pinv = neg_inv32(p);
  uint64_t r1 = (((uint64_t)1) << 32) % p;
  m.r1 = (uint32_t)r1;
  m.r2 = (uint32_t)((r1 * r1) % p);
  return m;
}

#if defined(__CUDACC__)
// acc + a b for signed 32-bit a, b: one wide multiply-add.
__device__ __forceinline__ int64_t rs_mac_s32(int64_t acc, int32_t a, int32_t b) {
  asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(acc) : "r"(a), "r"(b));
  return acc;
}

// hi 2^32 + lo -> hi c + lo for s = hi 2^32 + lo (c = 2^32 mod p, |c| < 2^31):
// congruent mod p, and |result| < 2^31 |c| + 2^32.
__device__ __forceinline__ int64_t rs_fold64(int64_t s, uint32_t c) {
  int64_t r;
  asm("{\n\t.reg .b32 lo, hi;\n\t.reg .s64 l64;\n\t"
      "mov.b64 {lo, hi}, %1;\n\t"
      "cvt.u64.u32 l64, lo;\n\t"
      "mad.wide.s32 %0, hi, %2, l64;\n\t}"
      : "=l"(r)
      : "l"(s), "r"(c));
  return r;
}
#endif
