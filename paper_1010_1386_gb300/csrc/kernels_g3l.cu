// CRT limbs on the tensor cores.  Paper, Section 4.1: R^{(y)} is recovered
// from its residues by Chinese remaindering; in Garner's mixed-radix form the
// coefficient is
//   R_j = sum_k v_k(j) P_k,   P_k = p_0 ... p_{k-1},
// with the signed digits |v_k| < p_k / 2 of the digit kernels.  Over the
// balanced base-256 digits of both factors (v_k = sum_a x_a 256^a with
// |x_a| <= 128, |x_3| <= 64; P_k = sum_b B_k[b] 256^b with |B_k[b]| <= 128)
// the byte column t of R_j collects
//   S_t(j) = sum_k sum_{a<4} x_a(j, k) B_k[t - a],
// a dense product of the coefficients x (prime, digit) matrix and, per digit
// a, the prefix-product bytes shifted by a.  One thread block owns 128
// coefficients of one pair (the rows) and one unit of 256 byte columns
// (64 output limbs); it walks the 64-prime blocks whose prefix products reach
// the unit (the others only arrive through carries) and accumulates the
// exact column sums in fp32 TMEM columns (M = 128, N = 256, bf16 operands).
//
// Exactness: one 64-prime block adds at most 64 * 128 * (3 * 128 + 64) =
// 3,670,016 to a column.  The accumulator has two buffers of 256 columns,
// taking windows of kWin blocks in turn; after a window, unless it was that
// buffer's last, its warpgroup splits every column s = 256 q + r (q = rint(s
// / 256), |r| <= 128) and writes back r + q_prev (the carry of the column
// below; column 255's carry is kept per row), so a buffer never holds more
// than 65,664 + kWin * 3,670,016 < 2^23 in magnitude, where fp32 sums of
// integers are exact.  At the end warps 0-3 add both buffers per column and
// fold the columns into 32-bit limbs with a carry chain; the unit's top
// carry goes to the limb chunk carries that the output kernel adds (the
// digits are signed, so no offset is removed there).
//
// Operands: the digit rows of the tensor-core digit kernel,
//   [64-prime chunk][32-prime stage][digit][row/8][l/8][row%8][l%8],
// and a table of prefix-product tiles per (chunk c, unit u): 128 KB,
//   [stage][digit a][column/8][l/8][column%8][l%8]  = B_k[256 u + column - a],
// k = 64 c + 32 stage + l, at block cbase[c] + u (units u <= the highest that
// chunk c reaches; the layout of a chunk does not change when more chunks are
// added).  Threads: warp 9 copies (48 KB stages: two digits of A, the two
// matching shifted tiles of B), warp 8 issues the MMAs, warps 0-3 / 4-7 keep
// buffers 0 / 1.  Every wait is bounded (about a second) and reports through
// the status word.
#include <algorithm>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rs.h"
#include "rs_internal.cuh"

namespace {

#include "tcdigits.cuh"

constexpr int kBlkK = 64;                         // primes per chunk
constexpr int kAStage = 2 * 128 * 32 * 2;         // 16 KB: two digits of 128 rows x 32 primes
constexpr int kBTile = 256 * 32 * 2;              // 16 KB: one shifted tile, 256 columns x 32 primes
constexpr int kBStage = 2 * kBTile;               // 32 KB
constexpr int kStage = kAStage + kBStage;         // 48 KB
constexpr int kStages = 4;
constexpr int kSmem = kStages * kStage;           // 192 KB
constexpr int kBBlock = 8 * kBTile;               // 128 KB of table per (chunk, unit)
constexpr int kWin = 2;                           // chunks per exact accumulation window
constexpr int kThreads = 320;
// kind::f16, fp32 accumulator, bf16 A and B, both K-major, N = 256, M = 128.
constexpr uint32_t kIdesc256 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(256 >> 3) << 17) |
                               ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ void mma256(uint32_t d, uint64_t a, uint64_t b) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, 1, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(kIdesc256)
      : "memory");
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t *v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15, %16};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]),
      "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
      : "memory");
}

__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

__global__ void __launch_bounds__(kThreads, 1) g3l_kernel(G3lArgs a) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ __align__(8) uint64_t bar[13];  // full[4], empty[4], accfull[2], accfree[2], done
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  __shared__ int32_t qs[128];  // buffer 1's carries out of column 255, per row
  const int4 lt = a.ltasks[blockIdx.x];
  const int2 task = a.tasks[lt.x];
  const PairDesc pd = a.pairs[task.x];
  const int u = lt.y, lo = lt.z, N = pd.N;
  const int KB = (pd.K + kBlkK - 1) / kBlkK;
  const int nch = KB > lo ? KB - lo : 0;
  const int nwin = (nch + kWin - 1) / kWin;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t sbase = smem_u32(sm);
  const uint32_t b_full = smem_u32(&bar[0]), b_empty = smem_u32(&bar[4]);
  const uint32_t b_accfull = smem_u32(&bar[8]), b_accfree = smem_u32(&bar[10]), b_done = smem_u32(&bar[12]);
  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int i = 0; i < kStages; ++i) {
      mbar_init(b_full + 8 * i, 1);
      mbar_init(b_empty + 8 * i, 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(b_accfull + 8 * i, 1);
      mbar_init(b_accfree + 8 * i, 4);
    }
    mbar_init(b_done, 1);
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

  // Sub-stages in order: chunk lo + ci, stage s = 2 (32-prime half) + digit
  // pair; g counts them and picks the buffer (g % 4) and the phases.
  if (warp >= 8) {
    if (warp == 9 && lane == 0) {  // producer
      const uint8_t *xa = reinterpret_cast<const uint8_t *>(a.xdig + a.xoff[lt.x]);
      const uint8_t *bt = reinterpret_cast<const uint8_t *>(a.btiles);
      int g = 0, issued = 0;
      bool ok = *a.stall == 0;  // test hook: no copies, so every consumer's wait runs out
      for (int c = lo; c < KB && ok; ++c) {
        const uint8_t *bblk = bt + ((size_t)__ldg(a.cbase + c) + u) * kBBlock;
        for (int s = 0; s < 4; ++s, ++g) {
          const int buf = g & (kStages - 1);
          if (g >= kStages && !mbar_wait(b_empty + 8 * buf, ((g >> 2) - 1) & 1, &abort_flag, a.err)) {
            ok = false;
            break;
          }
          const uint32_t dst = sbase + buf * kStage, fb = b_full + 8 * buf;
          mbar_expect_tx(fb, kStage);
          bulk_load(dst, xa + (size_t)c * (2 * 2 * kAStage) + s * kAStage, kAStage, fb);
          bulk_load(dst + kAStage, bblk + s * kBStage, kBStage, fb);
          issued = g + 1;
        }
      }
      for (int q = issued > kStages ? issued - kStages : 0; q < issued; ++q)
        mbar_wait(b_full + 8 * (q & (kStages - 1)), (q >> 2) & 1, &abort_flag, a.err, false);
    }
    if (warp == 8 && lane == 0) {  // MMA issuer
      int g = 0;
      bool ok = true;
      for (int w = 0; w < nwin && ok; ++w) {
        const int bb = w & 1;
        if (!mbar_wait(b_accfree + 8 * bb, (w >> 1) & 1, &abort_flag, a.err)) break;
        tc_fence_after();
        const uint32_t dcol = tbase + 256 * bb;
        const int c1 = min(nch, (w + 1) * kWin);
        for (int ci = w * kWin; ci < c1 && ok; ++ci) {
          for (int s = 0; s < 4; ++s, ++g) {
            const int buf = g & (kStages - 1);
            if (!mbar_wait(b_full + 8 * buf, (g >> 2) & 1, &abort_flag, a.err)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t ab = sbase + buf * kStage, bbase = ab + kAStage;
#pragma unroll
            for (int d = 0; d < 2; ++d)
#pragma unroll
              for (int ks = 0; ks < 2; ++ks)
                mma256(dcol, sdesc(ab + d * 8192 + ks * 256), sdesc(bbase + d * kBTile + ks * 256));
            tc_commit(b_empty + 8 * buf);
          }
        }
        if (ok && w + 2 < nwin) tc_commit(b_accfull + 8 * bb);
      }
      tc_commit(b_done);
      mbar_wait(b_done, 0, &abort_flag, a.err, false);  // no MMA in flight when the block frees TMEM
    }
    __syncwarp();
  } else {
    // Warps 4 grp .. 4 grp + 3 keep buffer grp; a warp reaches the TMEM lanes
    // of its quarter: rows (coefficients) 32 q .. 32 q + 31.  A failed wait
    // sets ok = false; the warp then skips the work but keeps arriving, so no
    // other warp is left waiting for it.
    const int grp = warp >> 2, q = warp & 3, row = 32 * q + lane, j = task.y + row;
    const uint32_t tl = tbase + ((uint32_t)(32 * q) << 16) + 256 * grp;
#pragma unroll
    for (int z = 0; z < 8; ++z) tmem_zero32(tl + 32 * z);
    tmem_wait_st();
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(b_accfree + 8 * grp);
    bool ok = true;
    int32_t Q = 0;  // carries out of column 255 of this buffer
    for (int w = grp; w + 2 < nwin; w += 2) {
      ok = ok && mbar_wait(b_accfull + 8 * grp, (w >> 1) & 1, &abort_flag, a.err);
      if (ok) {
        tc_fence_after();
        float qprev = 0.f;
#pragma unroll 1
        for (int g32 = 0; g32 < 8; ++g32) {
          uint32_t v[2][16];
          tmem_ld16(tl + 32 * g32, v[0]);
          tmem_ld16(tl + 32 * g32 + 16, v[1]);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          tmem_hold16(v[0]);
          tmem_hold16(v[1]);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
#pragma unroll
            for (int t = 0; t < 16; ++t) {
              const float x = __uint_as_float(v[h][t]);
              const float qf = rintf(x * 0.00390625f);
              const float r = fmaf(qf, -256.f, x);
              v[h][t] = __float_as_uint(r + qprev);
              qprev = qf;
            }
            tmem_st16(tl + 32 * g32 + 16 * h, v[h]);
          }
        }
        Q += (int32_t)qprev;
        tmem_wait_st();
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(b_accfree + 8 * grp);
    }
    if (grp == 1) qs[row] = Q;
    epi_sync();
    if (grp == 0) {
      ok = ok && mbar_wait(b_done, 0, &abort_flag, a.err);
      tc_fence_after();
      const bool live = ok && j < N;
      const int chunks = (pd.Lout + 15) / 16, L16 = 16 * chunks;
      uint32_t *xl = a.xl + pd.xl_off + j;
      int64_t carry = 0;
#pragma unroll 1
      for (int g16 = 0; g16 < 16; ++g16) {
        uint32_t v0[16], v1[16];
        tmem_ld16(tl + 16 * g16, v0);
        tmem_ld16(tl + 256 + 16 * g16, v1);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        tmem_hold16(v0);
        tmem_hold16(v1);
#pragma unroll
        for (int l4 = 0; l4 < 4; ++l4) {
          int64_t s = carry;
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int32_t cv = __float2int_rn(__uint_as_float(v0[4 * l4 + i])) +
                               __float2int_rn(__uint_as_float(v1[4 * l4 + i]));
            s += (int64_t)cv * (int64_t)(1u << (8 * i));
          }
          const int limb = 64 * u + 4 * g16 + l4;
          if (live && limb < L16) xl[(size_t)limb * N] = (uint32_t)s;
          carry = s >> 32;
        }
      }
      const int64_t top = carry + Q + qs[row];
#pragma unroll
      for (int s4 = 0; s4 < 4; ++s4) {
        const int cc = 4 * u + s4;
        if (live && cc < chunks) a.carry[pd.cy_off + (size_t)cc * N + j] = s4 == 3 ? top : 0;
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

// Byte b of P_k in balanced base 256 (digits in [-128, 128)), from the row of
// 16-bit digits (nbytes bytes reserved, zero above P_k).  The carry into byte
// b is 1 exactly when byte b - 1 plus its own carry is at least 128, so the
// first byte below b that is not 0x7f decides it (0x80 or more: 1).
__device__ int bal_byte(const uint16_t *row, int nbytes, int b) {
  if (b < 0) return 0;
  auto byte = [&](int i) -> int { return i < nbytes ? (int)((row[i >> 1] >> (8 * (i & 1))) & 0xffu) : 0; };
  int c = 0;
  for (int i = b - 1; i >= 0; --i) {
    const int x = byte(i);
    if (x != 0x7f) {
      c = x > 0x7f;
      break;
    }
  }
  const int d = byte(b) + c;
  return d >= 128 ? d - 256 : d;
}

// Prefix-product tiles of chunks c < KB: block cbase[c] + u holds, for
// stage s and shift a, tile 4 s + a with B_k[256 u + column - a] at
// (column, l), k = 64 c + 32 s + l (zero for k > K, where the table has no
// row).  One thread per 16-byte segment (8 consecutive l of one column).
__global__ void g3l_btile_kernel(const uint16_t *p16, const int32_t *poff, int K, const int32_t *cbase, int KB,
                                 int64_t nseg, uint16_t *out) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nseg; v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t blk = v >> 13;  // 8 tiles x 1024 segments per block
    int lo = 0, hi = KB - 1;      // the chunk c with cbase[c] <= blk < cbase[c + 1]
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (cbase[mid] <= blk)
        lo = mid;
      else
        hi = mid - 1;
    }
    const int c = lo, u = (int)(blk - cbase[c]);
    const int w = (int)(v & 8191), tile = w >> 10, seg = w & 1023;
    const int s = tile >> 2, sh = tile & 3;
    const int col = ((seg >> 5) << 3) | (seg & 7), l0 = ((seg >> 3) & 3) * 8;
    const int b = 256 * u + col - sh;
    uint32_t word[4];
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
      uint32_t bits[2];
#pragma unroll
      for (int f = 0; f < 2; ++f) {
        const int k = kBlkK * c + 32 * s + l0 + e + f;
        int d = 0;
        if (k <= K) {
          const int o = poff[k];
          d = bal_byte(p16 + o, 2 * (poff[k + 1] - o), b);
        }
        bits[f] = __float_as_uint((float)d) >> 16;
      }
      word[e >> 1] = bits[0] | (bits[1] << 16);
    }
    *reinterpret_cast<uint4 *>(out + v * 8) = make_uint4(word[0], word[1], word[2], word[3]);
  }
}

}  // namespace

cudaError_t g3l_prepare() {
  return cudaFuncSetAttribute(g3l_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
}

int64_t g3l_block_elems() { return kBBlock / 2; }

cudaError_t launch_g3l_btiles(const uint16_t *p16, const int32_t *poff, int K, const int32_t *cbase, int KB,
                              int64_t nblocks, uint16_t *out, cudaStream_t s) {
  if (nblocks <= 0) return cudaSuccess;
  const int64_t nseg = nblocks * 8192;
  const int blocks = (int)std::min<int64_t>((nseg + 255) / 256, 65535);
  g3l_btile_kernel<<<blocks, 256, 0, s>>>(p16, poff, K, cbase, KB, nseg, out);
  return cudaGetLastError();
}

cudaError_t launch_g3l(int ntasks, const G3lArgs &a, cudaStream_t s) {
  if (ntasks > 0) g3l_kernel<<<ntasks, kThreads, kSmem, s>>>(a);
  return cudaGetLastError();
}
