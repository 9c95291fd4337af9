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
// digit-weight classes in fp32 TMEM columns, read out every 64 inputs),
// except that each output column k is reduced modulo its own prime p_k.
// The 64 digits of the block then follow on the CUDA cores from the triangle
// of W inside the block (warps 0-3: the first 32, then warps 4-7: the last
// 32), are written over the residues and, as bf16 digits in the tensor
// cores' layout, to the tile's operand buffer, from which later blocks (and
// the tensor-core limb kernel) copy them.
//
// Operands: the tile's digit rows
//   [64-digit chunk][32-digit stage][digit i][row/8][l/8][row%8][l%8]
// (zero where no digit is written), and per (block kb, chunk c < kb) a 32 KB
// tile of W, [stage u][half h][(4 digits x 32 primes)/8][l/8][n%8][l%8] with
// W[64 kb + 32 h + t][64 c + 32 u + e], at index kb (kb - 1) / 2 + c.
// Threads: warp 9 copies chunks (the newest chunk of a block only after the
// previous block's digits are written and fenced for the async proxy), warp 8
// issues the MMAs, warps 0-3 / 4-7 drain the two halves (primes
// k0 .. k0 + 31 / k0 + 32 .. k0 + 63) and compute the digits.  Every wait is
// bounded (about a second) and reports through the status word.
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
constexpr int kAChunk = 2 * kAStage;                    // 64 KB
constexpr int kBuf = kAChunk + 2 * kBStage;             // 96 KB
constexpr int kHalfCols = 7 * kHalf;                    // 224 TMEM columns per half
constexpr int kDigStride = kBlkK + 1;                   // shared digits of the block, per row
constexpr int kSmem = 2 * kBuf + 128 * kDigStride * 4;  // 192 KB + 33 KB
constexpr int kThreads = 384;

struct ColConst {  // per prime of the current block
  ModP m;
  uint32_t w48;  // 2^48 mod p
  uint32_t c;    // (p_0 ... p_{k-1})^{-1} mod p_k (Montgomery)
};

__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

__global__ void __launch_bounds__(kThreads, 1) g3m_kernel(G3mArgs a) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ __align__(8) uint64_t bar[11];  // full[2], empty[2], accfull[2], accfree[2], drain, digits
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  __shared__ ColConst cc[kBlkK];
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
  const uint32_t b_drain = smem_u32(&bar[8]), b_dig = smem_u32(&bar[9]);
  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int i = 0; i < 2; ++i) {
      mbar_init(b_full + 8 * i, 1);
      mbar_init(b_empty + 8 * i, 1);
      mbar_init(b_accfull + 8 * i, 1);
      mbar_init(b_accfree + 8 * i, 4);
    }
    mbar_init(b_drain, 1);
    mbar_init(b_dig, 8);  // one arrival per digit warp
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
  // Chunks in order: block kb = 1 .. KB - 1 takes chunks c = 0 .. kb - 1
  // (digits 64 c .. 64 c + 63); g counts them over the whole tile and picks
  // the buffer (g & 1) and the barrier phases.
  if (warp >= 8) {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 72;" ::: "memory");
    if (warp == 9 && lane == 0) {  // producer
      const uint8_t *xa = reinterpret_cast<const uint8_t *>(xd);
      int g = 0, issued = 0;
      bool ok = *a.stall == 0;  // test hook: no copies, so every consumer's wait runs out
      for (int kb = 1; kb < KB && ok; ++kb) {
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
      }
      for (int q = issued > 2 ? issued - 2 : 0; q < issued; ++q)
        mbar_wait(b_full + 8 * (q & 1), (q >> 1) & 1, &abort_flag, a.err, false);
    }
    if (warp == 8 && lane == 0) {  // MMA issuer
      int g = 0;
      bool ok = true;
      for (int kb = 1; kb < KB && ok; ++kb) {
        for (int c = 0; c < kb; ++c, ++g) {
          const int buf = g & 1;
          if (!mbar_wait(b_full + 8 * buf, (g >> 1) & 1, &abort_flag, a.err)) {
            ok = false;
            break;
          }
          const uint32_t abase = sbase + buf * kBuf, bbase = abase + kAChunk;
          for (int h = 0; h < 2 && ok; ++h) {
            if (!mbar_wait(b_accfree + 8 * h, g & 1, &abort_flag, a.err)) {
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
                  const uint64_t bd = sdesc(bbase + u * kBStage + h * 8192 + ks * 256);
                  tc_mma(tbase + h * kHalfCols + i * kHalf, ad, bd, (u | ks | i) != 0);
                }
            tc_commit(b_accfull + 8 * h);
          }
          if (!ok) break;
          tc_commit(b_empty + 8 * buf);
        }
      }
      tc_commit(b_drain);
      mbar_wait(b_drain, 0, &abort_flag, a.err, false);
    }
    __syncwarp();
  } else {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 216;" ::: "memory");
    // Warps 0-3 drain half 0 (primes k0 .. k0 + 31), warps 4-7 half 1; a warp
    // reads the TMEM lanes of its quarter: rows (coefficients) 32 q .. 32 q + 31.
    // A failed wait sets ok = false; the warp then skips the work but keeps
    // passing the named barriers, so no digit warp waits there for a warp that left.
    const int h = warp >> 2, q = warp & 3, row = 32 * q + lane, j = j0 + row;
    const uint32_t tl = tbase + ((uint32_t)(32 * q) << 16) + h * kHalfCols;
    int32_t *drow = dig + row * kDigStride;
#pragma unroll
    for (int z = 0; z < 3; ++z) tmem_zero32(tl + 128 + 32 * z);
    tmem_wait_st();
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(b_accfree + 8 * h);
    bool ok = true;
    int g = 0;
    for (int kb = 0; kb < KB; ++kb) {
      const int k0 = kb * kBlkK, bk = min(kBlkK, K - k0);
      // The residues of this block reach L2 while its products are read out.
      if (j < N) {
#pragma unroll
        for (int t = 0; t < 32; ++t)
          if (kHalf * h + t < bk)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(col + (size_t)(k0 + kHalf * h + t) * S + j));
      }
      epi_sync();  // the previous block's readers of cc are done
      if (threadIdx.x < bk) {
        const ModP m = a.mods[k0 + threadIdx.x];
        cc[threadIdx.x].m = m;
        cc[threadIdx.x].w48 = (uint32_t)(((uint64_t)m.r1 << 16) % m.p);
        cc[threadIdx.x].c = a.crt[k0 + threadIdx.x];
      }
      epi_sync();
      uint64_t acc[32];
#pragma unroll
      for (int t = 0; t < 32; ++t) acc[t] = 0;
      for (int c = 0; c < kb; ++c, ++g) {
        ok = ok && mbar_wait(b_accfull + 8 * h, g & 1, &abort_flag, a.err);
        if (!ok) continue;
        tc_fence_after();
#pragma unroll
        for (int grp = 0; grp < 2; ++grp) {
          uint32_t v[7][16];
#pragma unroll
          for (int k = 0; k < 7; ++k) tmem_ld16(tl + 32 * k + 16 * grp, v[k]);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int k = 0; k < 7; ++k) tmem_hold16(v[k]);
          if (grp == 1) {  // every class of the chunk is in registers: free the half
#pragma unroll
            for (int z = 0; z < 3; ++z) tmem_zero32(tl + 128 + 32 * z);
            tmem_wait_st();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(b_accfree + 8 * h);
          }
#pragma unroll
          for (int t = 0; t < 16; ++t) {
            const ColConst &cq = cc[kHalf * h + 16 * grp + t];
            const uint32_t u = mag(v[0][t], kMagEven) + 256u * mag(v[1][t], kMagOdd);
            const uint32_t w = mag(v[2][t], kMagEven) + 256u * mag(v[3][t], kMagOdd);
            const uint32_t hh = mag(v[4][t], kMagEven) + 256u * mag(v[5][t], kMagOdd);
            const uint32_t b6 = mag(v[6][t], kMagEven);
            uint64_t x = acc[16 * grp + t] + u;
            x += (uint64_t)w << 16;
            x += (uint64_t)hh * cq.m.r1;
            x += (uint64_t)b6 * cq.w48;
            acc[16 * grp + t] = x;
          }
        }
      }
      // D_k = r_k - A[j][k] mod p_k for this half's primes (plain residues:
      // W is in Montgomery form, the final reduction removes R).  The W values
      // of the block's triangle come in meanwhile, spread over the lanes by
      // column: lane e holds wtri[t] = W[k0 + 32 h + t][k0 + 32 h + e] (e < t)
      // and, for half 1, wrect[t] = W[k0 + 32 + t][k0 + e]; each row t is one
      // coalesced load, and W[row][l] is read back by a shuffle from lane l.
      int32_t wtri[32];
#pragma unroll
      for (int t = 0; t < 32; ++t) {
        const int kr = k0 + kHalf * h + t;
        wtri[t] = (kHalf * h + t < bk && lane < t) ? __ldg(a.wtab + (size_t)kr * (kr - 1) / 2 + k0 + kHalf * h + lane) : 0;
      }
      // The block's digits, right-looking: sa[t] starts at (p - D_k) (2^32 mod p),
      // congruent to -D_k R (|.| < 2^52), and collects sum_l W[k][l] v_l for
      // this half's k = k0 + 32 h + t; each new digit is added into every
      // later sum at once (independent products), so a digit waits only for
      // its own reduction: v_k = -REDC(sa[t]) c_k.  Half 1 first adds the 32
      // digits of half 0.
      const size_t base = (size_t)k0 * S + j;
      int64_t sa[32];
#pragma unroll
      for (int t = 0; t < 32; ++t) {
        const int kk = kHalf * h + t;
        sa[t] = 0;
        if (kk < bk) {
          const ColConst &cq = cc[kk];
          const uint32_t r = j < N ? col[base + (size_t)kk * S] : 0u;
          const uint64_t bias =
              (uint64_t)kb * ((1ull << 31) + (1ull << 47) + (1ull << 31) * cq.m.r1 + (uint64_t)kBias6 * cq.w48);
          const uint32_t A = kb ? finish64_t(fold64_t((int64_t)(acc[t] - bias), cq.m.r1), cq.m) : 0u;
          sa[t] = (int64_t)(cq.m.p - msub(r, A, cq.m.p)) * cq.m.r1;
        }
      }
      auto fold_from = [&](int t0) {
#pragma unroll
        for (int t = 0; t < 32; ++t)
          if (t >= t0 && kHalf * h + t < bk) sa[t] = rs_fold64(sa[t], cc[kHalf * h + t].m.r1);
      };
      auto triangle = [&]() {
#pragma unroll
        for (int l = 0; l < 32; ++l) {
          const int kl = kHalf * h + l;
          int32_t vl = 0;
          if (kl < bk) {
            const ColConst &cq = cc[kl];
            const int64_t s2 = rs_fold64(sa[l], cq.m.r1);
            const uint32_t vv = mmul(mneg(finish64_t(s2, cq.m), cq.m.p), cq.c, cq.m);
            vl = signed_rep_t(vv, cq.m.p);
            drow[kl] = vl;
          }
#pragma unroll
          for (int t = l + 1; t < 32; ++t) sa[t] = rs_mac_s32(sa[t], __shfl_sync(0xffffffffu, wtri[t], l), vl);
          if (l % 7 == 6) fold_from(l + 1);
        }
      };
      // Half 0 runs its triangle while half 1 loads its rectangle of W; then
      // half 1 adds half 0's digits (a rolled loop over them: straight-line
      // code executed once per block would stream through the instruction
      // cache) and runs its own triangle.  One call site for the triangle.
      int32_t wrect[32];
      if (h == 1) {
#pragma unroll
        for (int t = 0; t < 32; ++t) {
          const int kr = k0 + kHalf + t;
          wrect[t] = kHalf + t < bk ? __ldg(a.wtab + (size_t)kr * (kr - 1) / 2 + k0 + lane) : 0;
        }
      }
#pragma unroll 1
      for (int pass = 0; pass < 2; ++pass) {
        if (pass == h) {
          if (h == 1) {
#pragma unroll 1
            for (int l = 0; l < 32; ++l) {
              const int32_t vl = drow[l];
#pragma unroll
              for (int t = 0; t < 32; ++t) sa[t] = rs_mac_s32(sa[t], __shfl_sync(0xffffffffu, wrect[t], l), vl);
              if (l % 7 == 6) fold_from(0);
            }
            fold_from(0);
          }
          triangle();
        }
        epi_sync();
      }
      // Write this half's digits over the residues and, for later blocks, as
      // operand digits; then fence them for the copies (async proxy).
      if (ok) {
#pragma unroll
        for (int t = 0; t < 32; ++t) {
          const int kk = kHalf * h + t;
          if (kk < bk && j < N) col[base + (size_t)kk * S] = (uint32_t)drow[kk];
        }
        {  // every block, the last too: the limb kernel reads them all
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
      }
      asm volatile("fence.proxy.async;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(b_dig);
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

}  // namespace

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
