// Shared pieces of the tcgen05 kernels (G2 products, CRT digits): PTX
// wrappers for mbarriers, bulk copies, tensor memory and kind::f16 MMAs, the
// no-swizzle K-major operand layout, and exact residue products through bf16
// digits (four balanced base-256 digits per residue, seven digit-weight
// classes accumulated in separate fp32 TMEM columns, read out every 64 inputs).
// Included by each kernel file inside its anonymous namespace, after
// rs_internal.cuh (ModP, redc, rs_fold64).
#pragma once

constexpr uint64_t kWaitNs = 1000000000ull;    // a wait gives up after a second
// kind::f16 instruction descriptor: fp32 accumulator (bits 4-5 = 1), bf16 A
// and B (bits 7-9, 10-12 = 1), both K-major, N = 128 (bits 17-22: N / 8),
// M = 128 (bits 24-28: M / 16).
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(128 >> 3) << 17) |
                            ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(bar),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase of the given parity.  Gives up when another
// thread of the block gave up (abort), or after kWaitNs: then it raises the
// block's abort flag and the error word.
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort, int32_t *err, bool watch = true) {
  uint64_t t0 = 0;
  for (uint32_t it = 1;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if (it > 8) __nanosleep(32);  // a longer wait yields the issue slots to the warps doing the work
    if ((it & 63) == 0) {
      if (watch && *abort) return false;
      const uint64_t now = globaltimer();
      if (t0 == 0) {
        t0 = now;
      } else if (now - t0 > kWaitNs) {
        *abort = 1;
        atomicExch(err, 1);
        return false;
      }
    }
  }
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: start address / 16 (bits 0-13), leading
// byte offset / 16 (bits 16-29: 128 B between core matrices along K), stride
// byte offset / 16 (bits 32-45: 512 B between 8-row groups), descriptor
// version 1 (bit 46), no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(512 >> 4) << 32) |
         (1ull << 46);
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}


// 16 consecutive TMEM columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t *v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}

// Orders later uses of 16 loaded registers after a tcgen05.wait::ld.
__device__ __forceinline__ void tmem_hold16(uint32_t *v) {
  asm volatile(""
               : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7]),
                 "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]), "+r"(v[14]),
                 "+r"(v[15])::"memory");
}

__device__ __forceinline__ void tmem_zero32(uint32_t taddr) {
  const uint32_t z = 0;
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, "
      "%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1};" ::"r"(taddr),
      "r"(z)
      : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Read-out of the digit-weight classes.  With digits |d_0..d_2| <= 128 and
// |d_3| <= 64, one input adds at most 2^14, 2^15, 3 2^14, 3 2^14, 2^15, 2^14,
// 2^12 to classes 0..6, so over 64 inputs |c_s| <= 2^20, 2^21, 3 2^20,
// 3 2^20, 2^21, 2^20, 2^18.  For an fp32 integer c and a magic constant
// m = 1.5 2^23 + delta with |c + delta| <= 2^22, c + m lies in [2^23, 2^24],
// where the spacing is 1: its bit pattern is 0x4B400000 + delta + c.  With
// delta = 0 for even classes and delta = -0xB4000 for odd ones (within the
// bounds above), the 32-bit combination b_even + 256 b_odd equals
// c_even + 256 c_odd + 2^31 exactly (|c_even + 256 c_odd| < 2^30), so each
// class costs one FADD and each pair one IMAD; the constant biases are
// removed once per output at the end.
constexpr float kMagEven = 12582912.0f;           // 1.5 2^23
constexpr float kMagOdd = 12582912.0f - 737280.0f;  // 1.5 2^23 - 0xB4000
constexpr uint32_t kBias6 = 0x4B400000u;           // class 6 pattern offset

__device__ __forceinline__ uint32_t mag(uint32_t v, float m) { return __float_as_uint(__uint_as_float(v) + m); }

__device__ __forceinline__ int32_t signed_rep_t(uint32_t v, uint32_t p) {
  return v > (p >> 1) ? (int32_t)v - (int32_t)p : (int32_t)v;
}

// Balanced base-256 digits of |v| < 2^30 as bf16 bit patterns (a digit has at
// most 8 significant bits, so the top half of its fp32 pattern is exact).
__device__ __forceinline__ void digits4(int32_t v, uint32_t (&bits)[4]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int32_t d = (int32_t)(int8_t)(v & 0xff);
    bits[i] = __float_as_uint((float)d) >> 16;
    v = (v - d) >> 8;
  }
  bits[3] = __float_as_uint((float)v) >> 16;
}

// Element offset of (row, input s, digit 0) in a row tile's operand layout;
// digit i is 4096 elements further.  s0 a multiple of 8 addresses 8 inputs.
__device__ __forceinline__ int64_t xoff(int row, int s) {
  return (int64_t)(s >> 6) * 32768 + ((s >> 5) & 1) * 16384 + (row >> 3) * 256 + ((s & 31) >> 3) * 64 +
         (row & 7) * 8 + (s & 7);
}

// The digits of 8 consecutive inputs s0..s0+7 of one row: four 16-byte stores.
__device__ __forceinline__ void store_digits8(uint16_t *x, int row, int s0, const int32_t (&v)[8]) {
  uint32_t w[4][4];
#pragma unroll
  for (int e = 0; e < 8; e += 2) {
    uint32_t lo[4], hi[4];
    digits4(v[e], lo);
    digits4(v[e + 1], hi);
#pragma unroll
    for (int i = 0; i < 4; ++i) w[i][e >> 1] = lo[i] | (hi[i] << 16);
  }
  uint16_t *p = x + xoff(row, s0);
#pragma unroll
  for (int i = 0; i < 4; ++i)
    *reinterpret_cast<uint4 *>(p + i * 4096) = make_uint4(w[i][0], w[i][1], w[i][2], w[i][3]);
}

__device__ __forceinline__ int64_t fold64_t(int64_t s, uint32_t c32) { return rs_fold64(s, c32); }

__device__ __forceinline__ uint32_t finish64_t(int64_t s, const ModP &m) {
  const uint64_t t = (uint64_t)(s + ((int64_t)m.p << 22));  // |s| < 2^53: 0 <= t < 2^54 < p 2^32
  return redc(t, m.p, m.pinv);
}
