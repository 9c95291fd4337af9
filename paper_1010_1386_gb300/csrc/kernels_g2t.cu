// G2 on the tensor cores.  Paper, Section 4.1: R^{(y)} is interpolated over
// Z_p from its images; on the geometric points x_i = q^i the Vandermonde solve
// factors into two convolutions with the chirp sequence b_t of prime p (the
// derivation is in kernels_g23.cu).  For one prime every pair of a batch
// convolves with the same b, so the convolutions of all pairs are one matrix
// product Y = X T with the lower-triangular Toeplitz matrix T[s][t] = b_{t-s}:
// rows are (pair, part) for the even part E and the odd part O of each pair,
// columns are output indices.  This file computes those products exactly on
// tcgen05 tensor cores.
//
// Exactness.  Residues enter as signed representatives |v| < 2^30 and are
// split into four balanced base-256 digits v = sum_i d_i 256^i, d_0..d_2 in
// [-128, 127], |d_3| <= 64; each digit is exact in bf16.  The product of two
// residues is the sum over digit pairs (i, j) of d_i e_j 256^(i+j): seven
// digit-weight classes s = i + j.  One MMA multiplies the i-th digit tile of X
// (128 rows x 16 inputs) by all four digit tiles of T laid side by side
// (16 inputs x 4 x 32 outputs) and accumulates into TMEM columns starting at
// class i, so class s of every output lands in its own fp32 column block.  A
// class sums at most 4 x 64 products of magnitude <= 2^14 per 64 inputs, so
// every partial sum is an integer below 2^22 in magnitude: exact in fp32.
// After each 64 inputs the classes are read out, recombined with weights
// 256^s mod p into an int64 per output (|sum| < 2^54 per 64 inputs, < 2^61 for
// up to 8192 inputs), and the upper class columns are cleared.  The final
// Montgomery reduction gives exactly the residue the direct convolution
// computes (sum_s x_s b_{t-s} R^{-1} mod p, both operands in Montgomery form).
//
// Data movement.  Operands live in global memory already in the tensor
// cores' shared-memory layout (no swizzle, K-major 8 x 16-byte core matrices,
// 128 bytes between core matrices along K, 512 bytes between 8-row groups), so
// every stage is a plain bulk copy (cp.async.bulk) completing on an mbarrier:
//   X of a row tile: [64-input chunk][32-input stage][digit i][row/8][in/8][row%8][in%8];
//   T of a prime: one 16 KB tile per diagonal offset D = t0 - s0 (a multiple
//     of 32, from -32): [half h][(4 digits x 32 outputs)/8][in/8][n%8][in%8].
// One thread block per work item (row tile, 64 outputs t0..t0+63): in the
// third warpgroup warp 9 loads 96 KB chunks into two buffers and warp 8
// issues the MMAs (its issue blocks while the tensor pipe's queue is full,
// so the copies have a warp of their own); warps 0-3 and 4-7
// drain the two accumulator halves (outputs t0..t0+31 and t0+32..t0+63), so
// one half's read-out overlaps the other half's MMAs.  Every wait is bounded
// (about a second); a wait that runs out sets the error word and the block
// drains its copies and MMAs, frees its tensor memory and returns.
#include <algorithm>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rs.h"
#include "blockinv.cuh"
#include "rs_internal.cuh"

namespace {

#include "tcdigits.cuh"

constexpr int kRows = 128;                     // MMA M: 64 pairs x {E, O}
constexpr int kHalfT = 32;                     // outputs per accumulator half
constexpr int kStageS = 32;                    // inputs per stage
constexpr int kChunkS = 64;                    // inputs per exact accumulation
constexpr int kAStageBytes = 4 * kRows * kStageS * 2;     // 32 KB: four digit tiles
constexpr int kBStageBytes = 2 * 4 * kHalfT * kStageS * 2;  // 16 KB: two halves
constexpr int kAChunkBytes = 2 * kAStageBytes;
constexpr int kBufBytes = kAChunkBytes + 2 * kBStageBytes;  // 96 KB
constexpr int kGemmSmem = 2 * kBufBytes;
constexpr int kHalfCols = 7 * kHalfT;          // TMEM columns of one half: 7 classes x 32
constexpr int kThreads = 384;  // warpgroups 0, 1: accumulator halves; 2: warp 8 issues, warp 9 loads

// ------------------------------------------------------------- products
//
// Block for item (rt, t0): Y[row][t] = sum_{s <= t} X[row][s] b_{t-s} mod p
// for t in [t0, t0 + 64), over the 64-input chunks c = 0 .. t0 / 64.  Chunk c,
// stage u (u = 0, 1) covers inputs s0 = 64 c + 32 u .. s0 + 31 and uses the
// Toeplitz tile of diagonal offset t0 - s0, index (t0 - s0) / 32 + 1.
__global__ void __launch_bounds__(kThreads, 1) g2t_gemm_kernel(G2tArgs a) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ __align__(8) uint64_t bar[10];  // full[2], empty[2], accfull[2], accfree[2], drain
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  const G2tItem it = a.items[blockIdx.x];
  const G2tRowTile rt = a.rts[it.rt];
  const ModP m = a.mods[rt.prime];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nc = it.t0 / kChunkS + 1;
  const uint32_t sbase = smem_u32(sm);
  const uint32_t b_full = smem_u32(&bar[0]), b_empty = smem_u32(&bar[2]);
  const uint32_t b_accfull = smem_u32(&bar[4]), b_accfree = smem_u32(&bar[6]), b_drain = smem_u32(&bar[8]);
  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int i = 0; i < 2; ++i) {
      mbar_init(b_full + 8 * i, 1);
      mbar_init(b_empty + 8 * i, 1);
      mbar_init(b_accfull + 8 * i, 1);
      mbar_init(b_accfree + 8 * i, 4);  // one arrival per draining warp
    }
    mbar_init(b_drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 8) {  // 512 columns: two halves of 7 x 32
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_slot;

  // Register split (launch: 168 per thread, 64,512 in all): the control
  // warpgroup gives back down to 88, the two draining warpgroups take 208
  // each (2 x 128 x 208 + 128 x 88 = 64,512; per SMSP 208 + 208 + 88 per
  // lane, within its 16,384).
  if (warp >= 8) {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 88;" ::: "memory");
    if (warp == 9 && lane == 0) {
      // Producer: chunk c goes into buffer c & 1 once the MMAs of chunk c - 2
      // (the buffer's previous contents) have completed.
      const uint8_t *xa = reinterpret_cast<const uint8_t *>(a.x + rt.x_off);
      const uint8_t *bt = reinterpret_cast<const uint8_t *>(a.btile + (size_t)rt.prime * a.bt_tiles * 8192);
      int issued = 0;
      const int ncopy = *a.stall ? 0 : nc;  // test hook: no copies, so every consumer's wait runs out
      for (int c = 0; c < ncopy; ++c) {
        const int buf = c & 1;
        if (c >= 2 && !mbar_wait(b_empty + 8 * buf, ((c - 2) >> 1) & 1, &abort_flag, a.err)) break;
        const uint32_t dst = sbase + buf * kBufBytes, fb = b_full + 8 * buf;
        const int d0 = (it.t0 - kChunkS * c) / kStageS + 1;  // tile of stage 0; stage 1 takes d0 - 1
        mbar_expect_tx(fb, kBufBytes);
        bulk_load(dst, xa + (size_t)c * kAChunkBytes, kAChunkBytes, fb);
        bulk_load(dst + kAChunkBytes, bt + (size_t)d0 * kBStageBytes, kBStageBytes, fb);
        bulk_load(dst + kAChunkBytes + kBStageBytes, bt + (size_t)(d0 - 1) * kBStageBytes, kBStageBytes, fb);
        issued = c + 1;
      }
      // The last copies into each buffer (no later phase follows them) must
      // have landed before the block exits.
      for (int c = issued > 2 ? issued - 2 : 0; c < issued; ++c)
        mbar_wait(b_full + 8 * (c & 1), (c >> 1) & 1, &abort_flag, a.err, false);
    }
    if (warp == 8 && lane == 0) {
      // MMA issuer.
      for (int c = 0; c < nc; ++c) {
        const int buf = c & 1;
        if (!mbar_wait(b_full + 8 * buf, (c >> 1) & 1, &abort_flag, a.err)) break;
        const uint32_t abase = sbase + buf * kBufBytes, bbase = abase + kAChunkBytes;
        bool ok = true;
        for (int h = 0; h < 2; ++h) {
          if (!mbar_wait(b_accfree + 8 * h, c & 1, &abort_flag, a.err)) {
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
                const uint64_t ad = sdesc(abase + u * kAStageBytes + i * 8192 + ks * 256);
                const uint64_t bd = sdesc(bbase + u * kBStageBytes + h * 8192 + ks * 256);
                tc_mma(tbase + h * kHalfCols + i * kHalfT, ad, bd, (u | ks | i) != 0);
              }
          tc_commit(b_accfull + 8 * h);
        }
        if (!ok) break;
        tc_commit(b_empty + 8 * buf);
      }
      // Drain every MMA this thread issued.
      tc_commit(b_drain);
      mbar_wait(b_drain, 0, &abort_flag, a.err, false);
    }
    __syncwarp();
  } else {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 208;" ::: "memory");
    // Warps 0-3 drain half 0 (outputs t0 .. t0 + 31), warps 4-7 half 1; a
    // warp reads the TMEM lanes of its quarter: rows 32 q .. 32 q + 31.
    const int h = warp >> 2, q = warp & 3, row = 32 * q + lane;
    const uint32_t tl = tbase + ((uint32_t)(32 * q) << 16) + h * kHalfCols;
    const uint32_t c32 = m.r1;                                             // 2^32 mod p < 2^21
    const uint32_t w48 = (uint32_t)(((uint64_t)c32 << 16) % m.p);          // 2^48 mod p
    // Classes 4..6 start cleared; classes 0..3 are written by each chunk's first MMA.
#pragma unroll
    for (int z = 0; z < 3; ++z) tmem_zero32(tl + 128 + 32 * z);
    tmem_wait_st();
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(b_accfree + 8 * h);
    // acc = sum over chunks of u + 2^16 w + c32 hh + w48 b6 (mod 2^64), each
    // term carrying its constant bias; |true sum| < 2^60.
    uint64_t acc[32];
#pragma unroll
    for (int t = 0; t < 32; ++t) acc[t] = 0;
    bool ok = true;
    for (int c = 0; c < nc; ++c) {
      if (!mbar_wait(b_accfull + 8 * h, c & 1, &abort_flag, a.err)) {
        ok = false;
        break;
      }
      tc_fence_after();
#pragma unroll
      for (int grp = 0; grp < 2; ++grp) {
        uint32_t v[7][16];
#pragma unroll
        for (int k = 0; k < 7; ++k) tmem_ld16(tl + 32 * k + 16 * grp, v[k]);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int k = 0; k < 7; ++k) tmem_hold16(v[k]);
        if (grp == 1) {  // every class of the chunk is in registers: free the accumulator half
          if (c + 1 < nc) {
#pragma unroll
            for (int z = 0; z < 3; ++z) tmem_zero32(tl + 128 + 32 * z);
            tmem_wait_st();
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(b_accfree + 8 * h);
        }
#pragma unroll
        for (int t = 0; t < 16; ++t) {
          const uint32_t u = mag(v[0][t], kMagEven) + 256u * mag(v[1][t], kMagOdd);
          const uint32_t w = mag(v[2][t], kMagEven) + 256u * mag(v[3][t], kMagOdd);
          const uint32_t hh = mag(v[4][t], kMagEven) + 256u * mag(v[5][t], kMagOdd);
          const uint32_t b6 = mag(v[6][t], kMagEven);
          uint64_t x = acc[16 * grp + t] + u;
          x += (uint64_t)w << 16;
          x += (uint64_t)hh * c32;
          x += (uint64_t)b6 * w48;
          acc[16 * grp + t] = x;
        }
      }
    }
    if (ok && row < rt.rows) {
      const uint64_t bias =
          (uint64_t)nc * ((1ull << 31) + (1ull << 47) + (1ull << 31) * c32 + (uint64_t)kBias6 * w48);
      uint32_t *y = a.y + rt.y_off + (size_t)row * rt.mt + it.t0 + kHalfT * h;
#pragma unroll
      for (int t = 0; t < 32; t += 4) {
        uint4 o;
        o.x = finish64_t(fold64_t((int64_t)(acc[t] - bias), c32), m);
        o.y = finish64_t(fold64_t((int64_t)(acc[t + 1] - bias), c32), m);
        o.z = finish64_t(fold64_t((int64_t)(acc[t + 2] - bias), c32), m);
        o.w = finish64_t(fold64_t((int64_t)(acc[t + 3] - bias), c32), m);
        *reinterpret_cast<uint4 *>(y + t) = o;
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

// ------------------------------------------------- element-wise steps

// Images -> operand digits.  One block per (pair, prime): the same fractions
// as the direct form (z+ +- z-, over the paired denominators inverted
// together), scaled by 1 / (2 F_i) for E and by 1 / (2 q^i F_i) for O.
// Shared memory: 4 M words.
__global__ void g2t_prep_kernel(G2tArgs a) {
  extern __shared__ __align__(16) uint32_t sw[];
  __shared__ uint32_t scratch[128];
  const G2tTask tk = a.tasks[blockIdx.x];
  const PairDesc pd = a.pairs[tk.pair];
  const ModP m = a.mods[tk.prime];
  const int NI = pd.NI, M = NI >> 1, T = blockDim.x, tid = threadIdx.x;
  const size_t base = (size_t)pd.img_off + (size_t)tk.prime * NI;
  const size_t tb = (size_t)tk.prime * a.tab_stride;
  const uint32_t *finv = a.finv + tb, *hq = a.hq + tb;
  uint32_t *dens = sw, *inv = sw + M;
  int32_t *xe = reinterpret_cast<int32_t *>(sw + 2 * M), *xo = xe + M;
  for (int i = tid; i < M; i += T) dens[i] = mmul(a.den[base + 2 * i], a.den[base + 2 * i + 1], m);
  __syncthreads();
  batch_invert(dens, inv, M, m, scratch);
  __syncthreads();
  for (int i = tid; i < M; i += T) {
    const uint32_t np = a.num[base + 2 * i], dp = a.den[base + 2 * i];
    const uint32_t nm = a.num[base + 2 * i + 1], dm = a.den[base + 2 * i + 1];
    const uint32_t e = mmul(mmul2(np, dm, nm, dp, m), inv[i], m);             // z+ + z-
    const uint32_t o = mmul(mmul2(np, dm, mneg(nm, m.p), dp, m), inv[i], m);  // z+ - z-
    xe[i] = signed_rep_t(mmul(mmul(e, hq[0], m), finv[i], m), m.p);
    xo[i] = signed_rep_t(mmul(mmul(o, hq[i], m), finv[i], m), m.p);
  }
  __syncthreads();
  uint16_t *x = a.x + a.rts[tk.rt].x_off;
  const int ng = (M + 7) >> 3;
  for (int w = tid; w < 2 * ng; w += T) {
    const int part = w >= ng, g = w - part * ng;
    const int32_t *src = part ? xo : xe;
    int32_t v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = 8 * g + e < M ? src[8 * g + e] : 0;
    store_digits8(x, 2 * tk.slot + part, 8 * g, v);
  }
}

// First products -> reversed operand: X'[s] = Y[D - s] Q^{-C(D-s,2)} F_{D-s}
// for s <= D = M - 1 (the Newton coefficients times F, reversed).
__global__ void g2t_mid_kernel(G2tArgs a) {
  const G2tTask tk = a.tasks[blockIdx.x];
  const PairDesc pd = a.pairs[tk.pair];
  const ModP m = a.mods[tk.prime];
  const G2tRowTile rt = a.rts[tk.rt];
  const int M = pd.NI >> 1, D = M - 1;
  const uint32_t *gt = a.gtab + (size_t)tk.prime * a.tab_stride;
  const int ng = (M + 7) >> 3;
  for (int w = threadIdx.x; w < 2 * ng; w += blockDim.x) {
    const int part = w >= ng, g = w - part * ng, row = 2 * tk.slot + part;
    const uint32_t *y = a.y + rt.y_off + (size_t)row * rt.mt;
    int32_t v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int s = 8 * g + e;
      v[e] = s < M ? signed_rep_t(mmul(y[D - s], gt[D - s], m), m.p) : 0;
    }
    store_digits8(a.x + rt.x_off, row, 8 * g, v);
  }
}

// Second products -> coefficients: R_{2i + part} = Y'[D - i] / F_i (plain).
__global__ void g2t_post_kernel(G2tArgs a) {
  const G2tTask tk = a.tasks[blockIdx.x];
  const PairDesc pd = a.pairs[tk.pair];
  const ModP m = a.mods[tk.prime];
  const G2tRowTile rt = a.rts[tk.rt];
  const int N = pd.N, M = pd.NI >> 1, D = M - 1;
  const size_t base = (size_t)pd.img_off + (size_t)tk.prime * pd.NI;
  const uint32_t *finv = a.finv + (size_t)tk.prime * a.tab_stride;
  const uint32_t *y0 = a.y + rt.y_off + (size_t)(2 * tk.slot) * rt.mt;
  for (int c = threadIdx.x; c < N; c += blockDim.x) {
    const int i = c >> 1, part = c & 1;
    a.coef[base + c] = from_mont(mmul(y0[(size_t)part * rt.mt + D - i], finv[i], m), m);
  }
}

// Toeplitz digit tiles: tile d of prime k holds T[s][t] = b_{D + t - s},
// D = 32 (d - 1), for inputs s < 32 and outputs t < 64 (two halves of 32),
// b_u = 0 for u < 0 or u >= nvalid.  One thread per 16-byte row segment.
__global__ void g2t_btile_kernel(const int32_t *btab, int tab_stride, int nvalid, int K, int ntiles,
                                 uint16_t *out) {
  const int64_t total = (int64_t)K * ntiles * 1024;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < total; v += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(v / ((int64_t)ntiles * 1024));
    const int rem = (int)(v - (int64_t)k * ntiles * 1024);
    const int d = rem >> 10, w = rem & 1023;
    const int h = w >> 9, ngp = (w >> 5) & 15, kc = (w >> 3) & 3, r = w & 7;
    const int n = ngp * 8 + r, j = n >> 5, tt = n & 31;
    const int u0 = 32 * (d - 1) + 32 * h + tt - 8 * kc;  // input e of the segment reads b_{u0 - e}
    uint32_t word[4];
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
      uint32_t lo[4], hi[4];
      const int ua = u0 - e, ub = u0 - e - 1;
      digits4(ua >= 0 && ua < nvalid ? btab[(size_t)k * tab_stride + ua] : 0, lo);
      digits4(ub >= 0 && ub < nvalid ? btab[(size_t)k * tab_stride + ub] : 0, hi);
      const uint32_t l = j == 0 ? lo[0] : j == 1 ? lo[1] : j == 2 ? lo[2] : lo[3];
      const uint32_t u = j == 0 ? hi[0] : j == 1 ? hi[1] : j == 2 ? hi[2] : hi[3];
      word[e >> 1] = l | (u << 16);
    }
    *reinterpret_cast<uint4 *>(out + v * 8) = make_uint4(word[0], word[1], word[2], word[3]);
  }
}

}  // namespace

cudaError_t g2t_prepare() {
  cudaError_t e = cudaFuncSetAttribute(g2t_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(g2t_prep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 4 * RS_G2T_MAX_M * 4);
  return e;
}

cudaError_t launch_g2t_btile(const int32_t *btab, int tab_stride, int nvalid, int K, int ntiles, uint16_t *out,
                             cudaStream_t s) {
  const int64_t total = (int64_t)K * ntiles * 1024;
  if (total <= 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 65535);
  g2t_btile_kernel<<<blocks, 256, 0, s>>>(btab, tab_stride, nvalid, K, ntiles, out);
  return cudaGetLastError();
}

cudaError_t launch_g2t(int ntasks, int nitems, int maxM, const G2tArgs &a, cudaStream_t s) {
  if (ntasks <= 0) return cudaSuccess;
  g2t_prep_kernel<<<ntasks, 256, (size_t)4 * maxM * 4, s>>>(a);
  g2t_gemm_kernel<<<nitems, kThreads, kGemmSmem, s>>>(a);
  g2t_mid_kernel<<<ntasks, 256, 0, s>>>(a);
  g2t_gemm_kernel<<<nitems, kThreads, kGemmSmem, s>>>(a);
  g2t_post_kernel<<<ntasks, 256, 0, s>>>(a);
  return cudaGetLastError();
}
