// CRT digits on the tensor cores.  Paper, Section 4.1: R^{(y)} is recovered
// from its residues by Chinese remaindering; here through Garner's mixed-radix
// digits
//   v_k = (r_k - sum_{l<k} v_l W[k][l]) c_k  mod p_k,  W[k][l] = p_0 ... p_{l-1} mod p_k,
// c_k = (p_0 ... p_{k-1})^{-1} mod p_k, each v_k in the symmetric range (the
// CUDA-core forms are in kernels_g3.cu).  For a block of 64 primes
// [k0, k0 + 64) the contribution of every earlier digit,
//   A[j][k] = sum_{l < k0} v_l(j) W[k][l],
// is a dense product of a coefficients x earlier-digits matrix and a slice of
// W, the same for every coefficient: one thread block owns 128 coefficients
// of one pair (the rows) and walks the digit blocks in order; block kb is a
// product over its kb 64-digit chunks, computed exactly on the tensor cores
// as in kernels_g2t.cu (signed residues as four bf16 digits, seven
// digit-weight classes in fp32 TMEM columns), except that each output column
// k is reduced modulo its own prime p_k and the classes are read out once
// per window of up to four chunks (exact integers below 2^24, decoded by
// cvt.rni).  The block splits into halves of 32 primes: warps 0-3 finish the
// first 32 digits from the triangle of W inside their half on the CUDA
// cores and write them as operand digits; the products of those digits with
// W[k0 + 32 + t][k0 + e] (the block's "rect") then go to half 1's
// accumulator on the tensor cores like one more 32-input chunk, and warps
// 4-7 finish the last 32 digits from their own triangle.  Warps 0-3 read out
// both halves' accumulators (and pass half 1's sums on through spare TMEM
// columns), so the products of the next block's chunks go on while warps
// 4-7 are busy with this block.  The digits are
// written over the residues and, as bf16 digits in the tensor cores'
// layout, to the tile's operand buffer, from which later blocks (and the
// tensor-core limb kernel) copy them.
//
// Operands: the tile's digit rows
//   [64-digit chunk][32-digit stage][digit i][row/8][l/8][row%8][l%8]
// (zero where no digit is written); per (block kb, chunk c < kb) a 32 KB
// tile of W, [stage u][half h][(4 digits x 32 primes)/8][l/8][n%8][l%8] with
// W[64 kb + 32 h + t][64 c + 32 u + e], at index kb (kb - 1) / 2 + c; and per
// block an 8 KB rect tile in the layout of one (stage, half).
// Threads: warp 9 copies (the newest chunk of a block only after the
// previous block's digits are written and fenced for the async proxy, a
// block's rect only after its first 32 digits are), warp 8 issues the MMAs,
// warps 0-3 read out both halves and compute the digits of half 0 (primes
// k0 .. k0 + 31), warps 4-7 those of half 1 (k0 + 32 .. k0 + 63).  Every wait is bounded (about a
// second) and reports through the status word.
#include <algorithm>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "../../include/rs.h"
#include "rs_internal.cuh"

namespace {

#include "tcdigits.cuh"

constexpr int kBlkK = 64;                               // primes per digit block
constexpr int kHalf = 32;                               // primes per accumulator half
constexpr int kAStage = 4 * 128 * 32 * 2;               // 32 KB: four digit tiles of 128 rows x 32 digits
constexpr int kBStage = 2 * 4 * kHalf * 32 * 2;         // 16 KB: two halves
constexpr int kBHalf = kBStage / 2;                     // 8 KB: one half's W digit tile of one stage
constexpr int kAChunk = 2 * kAStage;                    // 64 KB
constexpr int kBuf = kAChunk + 2 * kBStage;             // 96 KB
constexpr int kHalfCols = 7 * kHalf;                    // 224 TMEM columns per half
constexpr int kDigStride = kBlkK + 1;                   // shared digits of the block, per row
constexpr int kSmem = 2 * kBuf + 128 * kDigStride * 4;  // 192 KB + 33 KB
constexpr int kThreads = 384;
constexpr int kWin = 4;                                 // 64-digit chunks per read-out window

struct ColConst {  // per prime of the current block (20 bytes: shared memory is tight)
  uint32_t p, pinv, r1;  // the prime, -p^{-1} mod 2^32, 2^32 mod p
  uint32_t w48;          // 2^48 mod p
  uint32_t c;            // (p_0 ... p_{k-1})^{-1} mod p_k (Montgomery)
};

__device__ __forceinline__ ModP mod_of(const ColConst &c) {
  ModP m;
  m.p = c.p;
  m.pinv = c.pinv;
  m.r1 = c.r1;
  m.r2 = 0u;  // not used by the reductions here
  return m;
}

// Named barrier of one half's four warps (ids 2 and 3; 0 is __syncthreads).
__device__ __forceinline__ void half_sync(int h) {
  if (h == 0)
    asm volatile("bar.sync 2, 128;" ::: "memory");
  else
    asm volatile("bar.sync 3, 128;" ::: "memory");
}

// 8 consecutive TMEM columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t *v) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(taddr));
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t *v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
               "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
               : "memory");
}

__device__ __forceinline__ void tmem_hold8(uint32_t *v) {
  asm volatile(""
               : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7])::"memory");
}

// Read-out windows of block kb: ceil(kb / kWin) over its earlier chunks; half
// 1 also takes the products of the block's first 32 digits (its "rect"),
// appended to its last window (alone when kb = 0), when the block has primes
// in half 1.
__device__ __forceinline__ int nwin_of(int kb) { return (kb + kWin - 1) / kWin; }
__device__ __forceinline__ bool rect_of(int kb, int K) { return K - kBlkK * kb > kHalf; }

__global__ void __launch_bounds__(kThreads, 1) g3m_kernel(G3mArgs a) {
  extern __shared__ __align__(1024) uint8_t sm[];
  // full[2], empty[2], accfull[2], accfree[2], drain, digits, digits of half 0,
  // half 1's sums handed over
  __shared__ __align__(8) uint64_t bar[12];
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  // Constants of the block's primes: half 0's 32 (used by half 0 only) and
  // half 1's 32 by block parity (half 0 fills them for the next block while
  // half 1 still uses this block's).
  __shared__ ColConst cc0[kHalf];
  __shared__ ColConst cc1[2][kHalf];
  const int2 task = a.tasks[blockIdx.x];
  const PairDesc pd = a.pairs[task.x];
  const int K = pd.K, N = pd.N, S = pd.NI, j0 = task.y;
  const int KB = (K + kBlkK - 1) / kBlkK;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t *col = a.coef + pd.img_off;  // residue, then digit, of (k, j) at col[k S + j]
  uint16_t *xd = a.xdig + a.xoff[blockIdx.x];
  int32_t *dig = reinterpret_cast<int32_t *>(sm + 2 * kBuf);  // [row][kDigStride]: the block's digits
  const uint32_t sbase = smem_u32(sm);
  const uint32_t b_full = smem_u32(&bar[0]), b_empty = smem_u32(&bar[2]);
  const uint32_t b_accfull = smem_u32(&bar[4]), b_accfree = smem_u32(&bar[6]);
  const uint32_t b_drain = smem_u32(&bar[8]), b_dig = smem_u32(&bar[9]), b_dig0 = smem_u32(&bar[10]);
  const uint32_t b_a1 = smem_u32(&bar[11]);
  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int i = 0; i < 2; ++i) {
      mbar_init(b_full + 8 * i, 1);
      mbar_init(b_empty + 8 * i, 1);
      mbar_init(b_accfull + 8 * i, 1);
      mbar_init(b_accfree + 8 * i, 4);
    }
    mbar_init(b_drain, 1);
    mbar_init(b_dig, 8);   // one arrival per digit warp
    mbar_init(b_dig0, 4);  // one arrival per warp of half 0
    mbar_init(b_a1, 4);    // one arrival per warp of half 0
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 8) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_slot;

  // Register split (launch: 168 per thread, 64,512 in all): the control
  // warpgroup gives back down to 72, the draining warpgroups take 216 each
  // (2 x 128 x 216 + 128 x 72 = 64,512; per SMSP 216 + 216 + 72 per lane).
  // Copies in order: block kb = 0 .. KB - 1 takes its chunks c = 0 .. kb - 1
  // (digits 64 c .. 64 c + 63; the newest only once the previous block's
  // digits are written), then its rect (its own first 32 digits, once half
  // 0 wrote them, with the 8 KB tile of W[64 kb + 32 + t][64 kb + e]); g
  // counts the copies and picks the buffer (g & 1) and the barrier phases.
  if (warp >= 8) {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 72;" ::: "memory");
    if (warp == 9 && lane == 0) {  // producer
      const uint8_t *xa = reinterpret_cast<const uint8_t *>(xd);
      const uint8_t *rt = reinterpret_cast<const uint8_t *>(a.rtiles);
      int g = 0, issued = 0;
      bool ok = *a.stall == 0;  // test hook: no copies, so every consumer's wait runs out
      for (int kb = 0; kb < KB && ok; ++kb) {
        const uint8_t *wt = reinterpret_cast<const uint8_t *>(a.wtiles) + (size_t)(kb * (kb - 1) / 2) * 2 * kBStage;
        for (int c = 0; c < kb; ++c, ++g) {
          const int buf = g & 1;
          if (g >= 2 && !mbar_wait(b_empty + 8 * buf, ((g - 2) >> 1) & 1, &abort_flag, a.err)) {
            ok = false;
            break;
          }
          // the newest chunk holds the previous block's digits: wait until they are written
          if (c == kb - 1 && !mbar_wait(b_dig, (kb - 1) & 1, &abort_flag, a.err)) {
            ok = false;
            break;
          }
          const uint32_t dst = sbase + buf * kBuf, fb = b_full + 8 * buf;
          mbar_expect_tx(fb, kBuf);
          bulk_load(dst, xa + (size_t)c * kAChunk, kAChunk, fb);
          bulk_load(dst + kAChunk, wt + (size_t)c * 2 * kBStage, 2 * kBStage, fb);
          issued = g + 1;
        }
        if (!ok || !rect_of(kb, K)) continue;
        const int buf = g & 1;
        if (g >= 2 && !mbar_wait(b_empty + 8 * buf, ((g - 2) >> 1) & 1, &abort_flag, a.err)) break;
        if (!mbar_wait(b_dig0, kb & 1, &abort_flag, a.err)) break;
        const uint32_t dst = sbase + buf * kBuf, fb = b_full + 8 * buf;
        mbar_expect_tx(fb, kAStage + kBHalf);
        bulk_load(dst, xa + (size_t)kb * kAChunk, kAStage, fb);  // stage 0 of chunk kb: half 0's digits
        bulk_load(dst + kAChunk + kBHalf, rt + (size_t)kb * kBHalf, kBHalf, fb);  // where half 1's W tile sits
        issued = ++g;
      }
      for (int q = issued > 2 ? issued - 2 : 0; q < issued; ++q)
        mbar_wait(b_full + 8 * (q & 1), (q >> 1) & 1, &abort_flag, a.err, false);
    }
    if (warp == 8 && lane == 0) {  // MMA issuer
      // wh0, wh1: windows issued into half 0, 1 (the phase of its accfree
      // wait).  A window's first MMA overwrites classes 0-3 (the drain zeroed
      // 4-6 after the previous read-out); the rest accumulate.
      int g = 0, wh0 = 0, wh1 = 0;
      bool ok = true;
      for (int kb = 0; kb < KB && ok; ++kb) {
        const bool rect = rect_of(kb, K);
        for (int c = 0; c < kb && ok; ++c, ++g) {
          const int buf = g & 1;
          if (!mbar_wait(b_full + 8 * buf, (g >> 1) & 1, &abort_flag, a.err)) {
            ok = false;
            break;
          }
          const bool first = c % kWin == 0, last = c % kWin == kWin - 1 || c == kb - 1;
          const uint32_t abase = sbase + buf * kBuf, bbase = abase + kAChunk;
          for (int h = 0; h < 2 && ok; ++h) {
            if (first && !mbar_wait(b_accfree + 8 * h, (h ? wh1 : wh0) & 1, &abort_flag, a.err)) {
              ok = false;
              break;
            }
            tc_fence_after();
#pragma unroll
            for (int u = 0; u < 2; ++u)
#pragma unroll
              for (int ks = 0; ks < 2; ++ks)
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                  const uint64_t ad = sdesc(abase + u * kAStage + i * 8192 + ks * 256);
                  const uint64_t bd = sdesc(bbase + u * kBStage + h * kBHalf + ks * 256);
                  tc_mma(tbase + h * kHalfCols + i * kHalf, ad, bd, !first || (u | ks | i) != 0);
                }
            if (last && !(h == 1 && rect && c == kb - 1)) {  // half 1's last window waits for the rect
              tc_commit(b_accfull + 8 * h);
              if (h)
                ++wh1;
              else
                ++wh0;
            }
          }
          if (!ok) break;
          tc_commit(b_empty + 8 * buf);
        }
        if (!ok || !rect) continue;
        const int buf = g & 1;
        if (!mbar_wait(b_full + 8 * buf, (g >> 1) & 1, &abort_flag, a.err)) break;
        if (kb == 0 && !mbar_wait(b_accfree + 8, wh1 & 1, &abort_flag, a.err)) break;
        tc_fence_after();
        const uint32_t abase = sbase + buf * kBuf, bbase = abase + kAChunk;
#pragma unroll
        for (int ks = 0; ks < 2; ++ks)
#pragma unroll
          for (int i = 0; i < 4; ++i)
            tc_mma(tbase + kHalfCols + i * kHalf, sdesc(abase + i * 8192 + ks * 256),
                   sdesc(bbase + kBHalf + ks * 256), kb != 0 || (ks | i) != 0);
        tc_commit(b_accfull + 8);
        ++wh1;
        tc_commit(b_empty + 8 * buf);
        ++g;
      }
      tc_commit(b_drain);
      mbar_wait(b_drain, 0, &abort_flag, a.err, false);
    }
    __syncwarp();
  } else {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 216;" ::: "memory");
    // Warps 0-3 (half 0) read out both halves' accumulators (a warp reaches
    // the TMEM lanes of its quarter, rows 32 q .. 32 q + 31, in any column),
    // so the windows of the next block's chunks go on while warps 4-7 (half 1)
    // finish this block's last 32 digits; half 1's sums of a block reach its
    // threads through TMEM columns 448 + 32 (kb & 1) .. + 31 of their rows
    // (half 0 accumulates them there; the same lane quarter).  The constants of the
    // block's primes alternate between two buffers by block parity: half 0
    // fills them, half 1 reads them after the hand-over.  A failed wait sets
    // ok = false; the warp then skips the work but keeps arriving, so no other
    // warp is left waiting for it.
    const int h = warp >> 2, q = warp & 3, row = 32 * q + lane, j = j0 + row;
    const uint32_t tq = tbase + ((uint32_t)(32 * q) << 16);
    int32_t *drow = dig + row * kDigStride;
    if (h == 0) {
#pragma unroll
      for (int hh = 0; hh < 2; ++hh)
#pragma unroll
        for (int z = 0; z < 3; ++z) tmem_zero32(tq + hh * kHalfCols + 128 + 32 * z);
      tmem_wait_st();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(b_accfree);
        mbar_arrive(b_accfree + 8);
      }
    }
    bool ok = true;
    int rc0 = 0, rc1 = 0;  // read-outs of half 0's / half 1's accumulator so far (by half 0)
    for (int kb = 0; kb < KB; ++kb) {
      const int k0 = kb * kBlkK, bk = min(kBlkK, K - k0);
      ColConst *const c1 = cc1[kb & 1];
      ColConst *const cown = h ? c1 : cc0;  // this half's primes
      const bool rect = rect_of(kb, K);
      // This half's residues of the block, all 32 loads in flight at once and
      // parked in the thread's digit row until the triangle (loaded at their
      // use they came one miss after another: by then the copies of the
      // operand chunks have pushed them out of L2).
      const size_t base = (size_t)k0 * S + j;
      {
        uint32_t res[32];
#pragma unroll
        for (int t = 0; t < 32; ++t)
          res[t] = (kHalf * h + t < bk && j < N) ? col[base + (size_t)(kHalf * h + t) * S] : 0u;
#pragma unroll
        for (int t = 0; t < 32; ++t) drow[kHalf * h + t] = (int32_t)res[t];
      }
      // a0: this half's sums A[j][k] (half 1: handed over); half 1's sums
      // gather in TMEM columns ta1 .. ta1 + 31 (kept by half 0)
      const uint32_t ta1 = tq + 448 + 32 * (kb & 1);
      uint32_t a0[32];
#pragma unroll
      for (int t = 0; t < 32; ++t) a0[t] = 0u;
      // The block: half 0 reads half 0's and half 1's windows in turn (tri
      // read-outs), finishes its digits, then reads half 1's last window,
      // which holds the rect; half 1 only finishes its digits.
      int tri = 0;  // half 0's read-outs before its triangle
      if (h == 0) {
        half_sync(0);  // half 0's readers of this buffer (two blocks back) are done; half 1's too (see the hand-over)
        if (threadIdx.x < bk) {
          const ModP m = a.mods[k0 + threadIdx.x];
          ColConst &cq = (threadIdx.x < kHalf ? cc0 : c1)[threadIdx.x & 31];
          cq.p = m.p;
          cq.pinv = m.pinv;
          cq.r1 = m.r1;
          cq.w48 = (uint32_t)(((uint64_t)m.r1 << 16) % m.p);
          cq.c = a.crt[k0 + threadIdx.x];
        }
        half_sync(0);
        // this parity's hand-over columns were last read by half 1 two blocks
        // back, before it wrote that block out (waited for at the last hand-over)
        tmem_zero32(ta1);
        tmem_wait_st();
        const int nw = nwin_of(kb);
        tri = rect ? max(2 * nw - 1, 0) : 2 * nw;
      } else {
        ok = ok && mbar_wait(b_a1, kb & 1, &abort_flag, a.err);
        tc_fence_after();
        tmem_ld16(ta1, a0);
        tmem_ld16(ta1 + 16, a0 + 16);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        tmem_hold16(a0);
        tmem_hold16(a0 + 16);
        tc_fence_before();
      }
      auto readout = [&](const int hh) {
        // One window of half hh's accumulator: each class an exact integer
        // below 13.5 2^20 (at most 4.5 chunks of 64 inputs), taken by
        // cvt.rni and combined with its weight 256^s (2^32 = r1 <= 2^21,
        // 2^48 = w48 mod p) into one int64 term below 2^52.3, reduced at
        // once (REDC, as every window's) and added mod p.
        ok = ok && mbar_wait(b_accfull + 8 * hh, (hh ? rc1 : rc0) & 1, &abort_flag, a.err);
        if (hh)
          ++rc1;
        else
          ++rc0;
        if (!ok) return;
        tc_fence_after();
        const uint32_t tl = tq + hh * kHalfCols;
#pragma unroll
        for (int grp = 0; grp < 4; ++grp) {
          uint32_t v[7][8], s8[8];
#pragma unroll
          for (int k = 0; k < 7; ++k) tmem_ld8(tl + 32 * k + 8 * grp, v[k]);
          if (hh) tmem_ld8(ta1 + 8 * grp, s8);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int k = 0; k < 7; ++k) tmem_hold8(v[k]);
          tmem_hold8(s8);
          if (grp == 3) {  // every class of the window is in registers: free the half
#pragma unroll
            for (int z = 0; z < 3; ++z) tmem_zero32(tl + 128 + 32 * z);
            tmem_wait_st();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(b_accfree + 8 * hh);
          }
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            const ColConst &cq = (hh ? c1 : cc0)[8 * grp + t];
            int32_t c[7];
#pragma unroll
            for (int k = 0; k < 7; ++k) c[k] = __float2int_rn(__uint_as_float(v[k][t]));
            const int64_t lo = (int64_t)c[0] + (int64_t)c[1] * 256 + (int64_t)c[2] * 65536 +
                               (int64_t)c[3] * 16777216;
            const int64_t mid = (int64_t)c[4] + (int64_t)c[5] * 256;
            const int64_t x = lo + mid * (int64_t)cq.r1 + (int64_t)c[6] * (int64_t)cq.w48;
            const uint32_t val = finish64_t(x, mod_of(cq));
            if (hh)
              s8[t] = madd(s8[t], val, cq.p);
            else
              a0[8 * grp + t] = madd(a0[8 * grp + t], val, cq.p);
          }
          if (hh) tmem_st8(ta1 + 8 * grp, s8);
        }
        if (hh) tmem_wait_st();
      };
      for (int st = 0; st < tri; ++st) readout(st & 1);  // half 0 only (tri = 0 for half 1)
      // The half's digits.  D_k = r_k - A[j][k] mod p_k (plain residues: W
      // is in Montgomery form, the final reduction removes R); for half 1,
      // A includes the block's first 32 digits (the rect).  The W values of
      // the half's triangle, spread over the lanes by column: lane e holds
      // wtri[t] = W[k0 + 32 h + t][k0 + 32 h + e] (e < t); each row t is one
      // coalesced load, and W[row][l] is read back by a shuffle from lane l.
      int32_t wtri[32];
#pragma unroll
      for (int t = 0; t < 32; ++t) {
        const int kr = k0 + kHalf * h + t;
        wtri[t] = (kHalf * h + t < bk && lane < t) ? __ldg(a.wtab + (size_t)kr * (kr - 1) / 2 + k0 + kHalf * h + lane) : 0;
      }
      // Right-looking: sa[t] starts at (p - D_k) (2^32 mod p), congruent to
      // -D_k R (|.| < 2^52), and collects sum_l W[k][l] v_l for
      // k = k0 + 32 h + t over this half's earlier digits; each new digit is
      // added into every later sum at once (independent products), so a
      // digit waits only for its own reduction: v_k = -REDC(sa[t]) c_k.
      int64_t sa[32];
#pragma unroll
      for (int t = 0; t < 32; ++t) {
        const int kk = kHalf * h + t;
        sa[t] = 0;
        if (kk < bk) {
          const ColConst &cq = cown[t];
          sa[t] = (int64_t)(cq.p - msub((uint32_t)drow[kk], a0[t], cq.p)) * cq.r1;
        }
      }
#pragma unroll
      for (int l = 0; l < 32; ++l) {
        const int kl = kHalf * h + l;
        int32_t vl = 0;
        if (kl < bk) {
          const ColConst &cq = cown[l];
          const ModP m = mod_of(cq);
          const int64_t s2 = rs_fold64(sa[l], cq.r1);
          const uint32_t vv = mmul(mneg(finish64_t(s2, m), cq.p), cq.c, m);
          vl = signed_rep_t(vv, cq.p);
          drow[kl] = vl;
        }
#pragma unroll
        for (int t = l + 1; t < 32; ++t) sa[t] = rs_mac_s32(sa[t], __shfl_sync(0xffffffffu, wtri[t], l), vl);
        if (l % 7 == 6) {
#pragma unroll
          for (int t = l + 1; t < 32; ++t)
            if (kHalf * h + t < bk) sa[t] = rs_fold64(sa[t], cown[t].r1);
        }
      }
      // Write the half's digits over the residues and, as operand digits,
      // into stage h of chunk kb (every block, the last too: the limb kernel
      // reads them all); then fence them for the copies (async proxy).
      if (ok) {
#pragma unroll
        for (int t = 0; t < 32; ++t) {
          const int kk = kHalf * h + t;
          if (kk < bk && j < N) col[base + (size_t)kk * S] = (uint32_t)drow[kk];
        }
#pragma unroll
        for (int e8 = 0; e8 < 4; ++e8) {
          int32_t v8[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int kk = kHalf * h + 8 * e8 + e;
            v8[e] = kk < bk ? drow[kk] : 0;
          }
          store_digits8(xd, row, k0 + kHalf * h + 8 * e8, v8);
        }
      }
      asm volatile("fence.proxy.async;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(b_dig);
        if (h == 0) mbar_arrive(b_dig0);
      }
      if (h == 0 && rect) readout(1);  // half 1's last window, with the rect
      if (h == 0) {
        // Hand half 1's sums over (they are in TMEM), after half 1 has written
        // out the previous block: by then it has read the other parity's
        // hand-over columns and constants buffer for the last time, which
        // the next block reuses.
        if (kb > 0) ok = ok && mbar_wait(b_dig, (kb - 1) & 1, &abort_flag, a.err);
        tc_fence_after();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(b_a1);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 8) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tbase) : "memory");
  }
}

// W digit tiles for blocks kb < KB: tile kb (kb - 1) / 2 + c (c < kb) holds
// W[64 kb + 32 h + t][64 c + 32 u + e] (always l < k) as digit j, zero for
// rows k >= K.  One thread per 16-byte row segment.
__global__ void g3m_wtile_kernel(const int32_t *wtab, int K, int64_t ntiles, uint16_t *out) {
  const int64_t total = ntiles * 2048;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < total; v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ti = v >> 11;
    int kb = (int)((1.0 + sqrt(1.0 + 8.0 * (double)ti)) * 0.5);
    while ((int64_t)kb * (kb - 1) / 2 > ti) --kb;
    while ((int64_t)(kb + 1) * kb / 2 <= ti) ++kb;
    const int c = (int)(ti - (int64_t)kb * (kb - 1) / 2);
    const int w = (int)(v & 2047), u = w >> 10, rest = w & 1023;
    const int h = rest >> 9, ngp = (rest >> 5) & 15, kc = (rest >> 3) & 3, r = rest & 7;
    const int n = ngp * 8 + r, jd = n >> 5, t = n & 31;
    const int k = kBlkK * kb + kHalf * h + t, l0 = kBlkK * c + 32 * u + 8 * kc;
    uint32_t word[4];
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
      uint32_t lo[4], hi[4];
      digits4(k < K ? wtab[(size_t)k * (k - 1) / 2 + l0 + e] : 0, lo);
      digits4(k < K ? wtab[(size_t)k * (k - 1) / 2 + l0 + e + 1] : 0, hi);
      const uint32_t x = jd == 0 ? lo[0] : jd == 1 ? lo[1] : jd == 2 ? lo[2] : lo[3];
      const uint32_t y = jd == 0 ? hi[0] : jd == 1 ? hi[1] : jd == 2 ? hi[2] : hi[3];
      word[e >> 1] = x | (y << 16);
    }
    *reinterpret_cast<uint4 *>(out + v * 8) = make_uint4(word[0], word[1], word[2], word[3]);
  }
}

// Rect tiles, one per block kb < KB: the 8 KB tile of W[64 kb + 32 + t][64 kb + e]
// (e < 32: the block's first 32 primes against its last 32) as digit j, in
// the layout of one (stage, half) of the tiles above; zero for rows k >= K.
__global__ void g3m_rtile_kernel(const int32_t *wtab, int K, int KB, uint16_t *out) {
  const int total = KB * 512;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < total; v += gridDim.x * blockDim.x) {
    const int kb = v >> 9, w = v & 511;
    const int ngp = w >> 5, kc = (w >> 3) & 3, r = w & 7;
    const int n = ngp * 8 + r, jd = n >> 5, t = n & 31;
    const int k = kBlkK * kb + kHalf + t, l0 = kBlkK * kb + 8 * kc;
    uint32_t word[4];
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
      uint32_t lo[4], hi[4];
      digits4(k < K ? wtab[(size_t)k * (k - 1) / 2 + l0 + e] : 0, lo);
      digits4(k < K ? wtab[(size_t)k * (k - 1) / 2 + l0 + e + 1] : 0, hi);
      const uint32_t x = jd == 0 ? lo[0] : jd == 1 ? lo[1] : jd == 2 ? lo[2] : lo[3];
      const uint32_t y = jd == 0 ? hi[0] : jd == 1 ? hi[1] : jd == 2 ? hi[2] : hi[3];
      word[e >> 1] = x | (y << 16);
    }
    *reinterpret_cast<uint4 *>(out + (size_t)v * 8) = make_uint4(word[0], word[1], word[2], word[3]);
  }
}

}  // namespace

int64_t g3m_rtile_elems(int KB) { return (int64_t)KB * (kBHalf / 2); }

cudaError_t launch_g3m_rtiles(const int32_t *wtab, int K, int KB, uint16_t *out, cudaStream_t s) {
  if (KB <= 0) return cudaSuccess;
  const int total = KB * 512;
  g3m_rtile_kernel<<<(total + 255) / 256, 256, 0, s>>>(wtab, K, KB, out);
  return cudaGetLastError();
}

cudaError_t g3m_prepare() {
  return cudaFuncSetAttribute(g3m_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
}

int64_t g3m_wtile_elems(int KB) { return KB > 1 ? (int64_t)KB * (KB - 1) / 2 * (2 * kBStage / 2) : 0; }

int64_t g3m_tile_elems(int K) { return (int64_t)((K + kBlkK - 1) / kBlkK) * (kAChunk / 2); }

cudaError_t launch_g3m_wtiles(const int32_t *wtab, int K, int KB, uint16_t *out, cudaStream_t s) {
  const int64_t ntiles = KB > 1 ? (int64_t)KB * (KB - 1) / 2 : 0;
  if (ntiles == 0) return cudaSuccess;
  const int64_t total = ntiles * 2048;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 65535);
  g3m_wtile_kernel<<<blocks, 256, 0, s>>>(wtab, K, ntiles, out);
  return cudaGetLastError();
}

cudaError_t launch_g3m(int ntiles, const G3mArgs &a, cudaStream_t s) {
  if (ntiles > 0) g3m_kernel<<<ntiles, kThreads, kSmem, s>>>(a);
  return cudaGetLastError();
}
