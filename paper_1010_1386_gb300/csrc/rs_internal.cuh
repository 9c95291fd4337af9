// Internal layout shared by the host engine and the kernels of librs.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rs.h"
#include "modarith.cuh"

#define RS_VT_STRIDE (RS_MAX_LIMBS + 1)  // V[k][l] = 2^(32 l) R^2 mod p_k, l = 0..RS_MAX_LIMBS
#define RS_G1_MAX_STAGED_WORDS (48 * 1024)  // staged residues + meta per G1 tile
#define RS_G1_MAX_SMEM_BYTES (RS_G1_MAX_STAGED_WORDS * 4)
#define RS_G2_PAD 8          // zero words around each G2 shared-memory region
#define RS_CONV_R 7          // G2 outputs per register block; odd, so lanes hit distinct banks
#define RS_G2_MAX_SMEM_BYTES (4 * (8192 + 2 * RS_G2_PAD) * 4)  // four regions of M <= 8192 pairs
#define RS_NTT_LGMAX 13      // G2 transforms up to 2^13 points (N <= 2^12)
#define RS_G2N_MAX_SMEM_BYTES ((4 * 4096 + 2 * (1 << RS_NTT_LGMAX)) * 4)

// Stage counters written by the kernels (detection of unlucky / degenerate cases).
enum { ST_UNLUCKY_POINTS = 0, ST_DEGENERATE = 1, ST_UNLUCKY_PRIMES = 2, ST_COUNT = 4 };

// One resultant of a batch, as the kernels see it.  Degrees are trimmed.
struct PairDesc {
  int32_t my, ny;      // actual y-degrees of f and g
  int32_t N;           // coefficients = degree bound D + 1
  // Points come in pairs +-q^i, i < M = ceil(N / 2); the images of prime k are
  // [k NI, k NI + NI), NI = 2 M, image 2 i + s at x = (-1)^s q^i, and the
  // interpolated residues (then the CRT digits) keep that stride.
  int32_t K;           // primes
  int32_t Lf, Lg;      // input limbs per coefficient
  int32_t fstride, gstride;  // input row stride in coefficients (= array deg_y + 1)
  int32_t fnc, gnc;    // coefficients kept (sum over j of deg_x f_j + 1)
  int32_t Lout;        // output limbs per coefficient
  int32_t mxf, mxg;    // x-degrees of f and g
  int32_t NI;          // images per prime (2 M)
  int64_t f_off, g_off;  // word offsets of the input limb arrays
  int64_t meta_off;      // int2 offset: (my+1) entries for f then (ny+1) for g
  int64_t img_off;       // offset of the K*NI image block (prime-major)
  int64_t out_off;       // offset of the N*Lout output block (coefficient-major)
  int64_t xl_off;        // offset of the CRT digit scratch: N * 16 * ceil(Lout/16) words
  int64_t cy_off;        // offset of the CRT chunk carries: N * ceil(Lout/16) int64
};

// G1 work item: point pairs [x0, x0 + n) of one (pair, prime), two threads
// (the images at +q^i and -q^i) per pair.
struct Tile {
  int32_t pair;
  int32_t prime;
  int32_t x0;
  int32_t n;
};

struct G1Args {
  const PairDesc *pairs;
  const Tile *tiles;
  int32_t ntiles;
  int32_t persistent;
  int32_t *counter;        // persistent tile counter (zeroed before launch)
  const uint32_t *limbs;   // batch input limbs
  const int2 *meta;        // per-j (start in the staged residue array, x-degree or -1)
  const ModP *mods;
  const int32_t *qc;       // [prime][tstride] Q^{C(t,2)}, Q = q^2, signed representative (Montgomery)
  const uint32_t *qn;      // [prime][tstride] Q^{-C(t,2)} (Montgomery)
  const uint32_t *qp;      // [prime][tstride] q^t (Montgomery)
  int32_t tstride;
  const uint32_t *vtab;    // [prime][RS_VT_STRIDE]
  uint32_t *num;           // numerators  (Montgomery form, sign applied)
  uint32_t *den;           // denominators (Montgomery form, non-zero)
  unsigned long long *stats;
};

// Schur variant of G1 (kernels_schur.cu): the same tiles, points and image
// layout; images whose recurrence meets a zero pivot are listed as (tile,
// image within the tile) for the elimination fallback.
struct G1sArgs {
  const PairDesc *pairs;
  const Tile *tiles;
  const uint32_t *limbs;
  const ModP *mods;
  const uint32_t *vtab;
  const uint32_t *qp;      // [prime][tstride] q^t (Montgomery)
  int32_t tstride;
  uint32_t *num, *den;
  int2 *fail;              // capacity: every image of the batch
  int32_t *fail_count;     // zeroed before the launch
  unsigned long long *stats;
};

#define RS_G1S_MAX_SLOTS 5  // Schur variant: m_y + n_y <= 32 x this

// Triangular-factorisation variant of G2 (kernels_schur.cu): one block per
// (pair, prime), shared memory 4 N + 97 words.
struct G2sArgs {
  const PairDesc *pairs;
  const int2 *tasks;       // (pair, prime)
  const ModP *mods;
  const uint32_t *num, *den;
  uint32_t *coef;          // out: R mod p (plain), may alias num
  const uint32_t *qp;      // [prime][tstride] q^t (Montgomery)
  int32_t tstride;
};

struct G2Args {
  const PairDesc *pairs;
  const int2 *tasks;       // (pair, prime)
  const ModP *mods;
  const uint32_t *num;     // in: numerators
  const uint32_t *den;     // in: denominators
  uint32_t *coef;          // out: R mod p coefficients, plain form (may alias num)
  const uint32_t *finv;    // [prime][tab_stride] 1 / F_t, F_t = prod_{s<=t} (Q^s - 1)  (Montgomery)
  const uint32_t *gtab;    // [prime][tab_stride] Q^{-C(t,2)} F_t   (Montgomery)
  const int32_t *btab;     // [prime][tab_stride] (-1)^t Q^{C(t,2)} / F_t, signed representative
  const uint32_t *hq;      // [prime][tab_stride] 1 / (2 q^t)  (Montgomery)
  int32_t tab_stride;
};

// Tensor-core G2 (kernels_g2t.cu).  For one prime, the rows of a row tile
// are 64 (pair, prime) tasks x {E, O}; their inputs are zero beyond each
// pair's point-pair count M, and the tile's length mt (a multiple of 64)
// covers its largest M.
struct G2tRowTile {
  int64_t x_off;  // element offset of the tile's operand digits (64 KB per 64 inputs)
  int64_t y_off;  // word offset of the tile's products, [128 rows][mt]
  int32_t prime;
  int32_t mt;
  int32_t rows;   // rows in use (2 x tasks)
  int32_t pad;
};

struct G2tItem {  // one block: outputs t0 .. t0 + 63 of a row tile
  int32_t rt;
  int32_t t0;
};

struct G2tTask {  // one (pair, prime): rows 2 slot (E) and 2 slot + 1 (O) of row tile rt
  int32_t pair, prime, rt, slot;
};

struct G2tArgs {
  const PairDesc *pairs;
  const G2tTask *tasks;
  const G2tRowTile *rts;
  const G2tItem *items;
  const ModP *mods;
  const uint32_t *num, *den;
  uint32_t *coef;             // out: R mod p (plain), may alias num
  const uint32_t *finv, *gtab, *hq;  // as in G2Args
  int32_t tab_stride;
  const uint16_t *btile;      // [prime][bt_tiles][8192] Toeplitz digit tiles (bf16 patterns)
  int32_t bt_tiles;           // tiles per prime: diagonal offsets -32, 0, 32, ...
  uint16_t *x;                // operand digits of every row tile
  uint32_t *y;                // products of every row tile
  int32_t *err;               // set to 1 by a block whose bounded wait ran out
  const int32_t *stall;       // test hook: non-zero = the copy warp issues nothing
};

#define RS_G2T_MAX_M 4096  // point pairs per (pair, prime) the tensor-core form takes

#ifndef RS_G3M_MIN_K
#define RS_G3M_MIN_K 128  // largest prime count from which a batch's digits take the tensor cores
#endif
#ifndef RS_G3M_WIDE_K
#define RS_G3M_WIDE_K 1024  // ... and from which they do so even with few coefficient tiles
#endif

// Tensor-core CRT digits (kernels_g3m.cu): one block per 128 coefficients of
// one pair (the output kernel's tasks), over 64-prime digit blocks.
struct G3mArgs {
  const PairDesc *pairs;
  const int2 *tasks;        // (pair, first coefficient), coefficients in steps of 128
  const ModP *mods;
  const uint32_t *crt;      // (p_0 ... p_{k-1})^{-1} mod p_k, Montgomery form
  const int32_t *wtab;      // triangular W[k][l] (signed Montgomery), as for the other digit kernels
  const uint16_t *wtiles;   // W digit tiles per (block, chunk)
  const uint16_t *rtiles;   // per block: W of its last 32 primes against its first 32, as digits
  uint32_t *coef;           // in: R mod p_k (plain); overwritten by the digits
  uint16_t *xdig;           // operand digits of every tile (zeroed once)
  const int64_t *xoff;      // per task: element offset of its operand digits
  int32_t *err;             // status word (a bounded wait ran out)
  const int32_t *stall;     // test hook: non-zero = the copy warp issues nothing
};

// Tensor-core CRT limbs (kernels_g3l.cu): one block per (128 coefficients of
// a pair, unit of 64 output limbs), over the 64-prime chunks whose prefix
// products reach the unit; reads the digit rows the tensor-core digit kernel
// wrote and writes limb chunks and carries for the output kernel.
struct G3lArgs {
  const PairDesc *pairs;
  const int2 *tasks;        // the digit kernel's tasks: (pair, first coefficient)
  const int4 *ltasks;       // (digit task, unit, first chunk, -) per block
  const uint16_t *xdig;     // operand digits of every digit task
  const int64_t *xoff;      // per digit task: element offset of its operand digits
  const uint16_t *btiles;   // prefix-product tiles, block cbase[c] + u per (chunk c, unit u)
  const int32_t *cbase;     // per chunk: its first table block
  uint32_t *xl;             // out: limbs [16 chunk + w][N] per pair
  int64_t *carry;           // out: chunk carries [chunk][N] per pair
  int32_t *err;             // status word (a bounded wait ran out)
  const int32_t *stall;     // test hook: non-zero = the copy warp issues nothing
};

// The three NTT primes P0 < P1 < P2 of the transform-based G2 (each
// c 2^k + 1 with k >= 25, in (2^30, 2^31)) and their Garner constants.
struct NttConst {
  ModP m[3];
  uint32_t c01;    // P0^-1 mod P1, Montgomery form
  uint32_t p0_m2;  // P0 R mod P2 (mmul(v, p0_m2) = v P0 mod P2)
  uint32_t c012;   // (P0 P1)^-1 mod P2, Montgomery form
};

struct G2nArgs {
  const PairDesc *pairs;
  const int2 *tasks;       // (pair, prime), all with transform length 2^lg
  const ModP *mods;
  const uint32_t *num, *den;
  uint32_t *coef;          // out (may alias num)
  const uint32_t *finv, *gtab, *hq;  // as in G2Args
  int32_t tab_stride;
  const uint2 *tw;         // [q][forward, inverse][2^RS_NTT_LGMAX]: rows of 2^(lg-1) twiddles
                           // (w_L^j, Shoup quotient), L = 2^lg, starting at 2^(lg-1) - 1
  const uint32_t *bhat;    // [prime][q][2^lg] transformed interpolation kernel / 2^lg (Montgomery mod P_q)
  NttConst nc;
  int32_t lg;
};

// Square-free factorisation mod p keeps its two scratch polynomials in
// shared memory up to this size (2 x the scratch stride in words).
#define RS_YUN_MAX_SMEM_BYTES (96 * 1024)

// Square-free factorisation of R mod p (kernels_yun.cu), one task per
// (pair, prime) after G2: output layout documented there.
struct YunArgs {
  const PairDesc *pairs;
  const int2 *tasks;       // (pair, prime)
  const ModP *mods;
  const uint32_t *coef;    // G2's residues of R (plain), stride NI per prime
  uint32_t *out;           // [task][ostride]
  uint32_t *work;          // [task][8][wstride] scratch
  int64_t ostride, wstride;
  int32_t maxm;            // largest multiplicity reported
  int32_t shared_scratch;  // set by launch_yun: the two scratch polynomials in shared memory
};

struct G3Args {
  const PairDesc *pairs;
  const int2 *tasks;       // (pair, first coefficient) per block (digit tiles of 32 coefficients)
  const int4 *ctasks;      // (pair, first coefficient, chunk, -) per limb-chunk block
  const ModP *mods;
  const uint32_t *crt;     // (p_0 ... p_{k-1})^{-1} mod p_k, Montgomery form
  const int32_t *wtab;     // triangular: W[k][l] = p_0 ... p_{l-1} mod p_k (Montgomery, signed)
  const uint16_t *p16;     // prefix products p_0 ... p_{k-1} in 16-bit digits
  const int32_t *poff;     // row offsets into p16 (u16 units, multiples of 32)
  const int32_t *nh;       // digits of each prefix product
  uint32_t *coef;          // in: R mod p_k (plain); overwritten by mixed-radix digits
  uint32_t *xl;            // 16-bit digit pairs of R_j, [16 chunk + w][N] per pair
  int64_t *carry;          // chunk carries [chunk][N] per pair
  uint32_t *out;           // out: [coefficient][limb]
  int32_t *shape;          // out: per pair (1 + degree, limbs needed), zeroed before the launch
  int32_t kmax;            // largest K of the batch
  int32_t signed_digits = 0;  // 1: the limbs come from the signed digits (no floor(P / 2) to remove)
};

// Launchers (kernels_*.cu).  Each returns the cudaGetLastError() of its launch.
cudaError_t launch_g1(int cap, int threads, int blocks, size_t smem, const G1Args &a, cudaStream_t s);
int g1_supported_cap(int cap);           // smallest compiled register capacity >= cap, or 0
cudaError_t g1_prepare(int cap, int threads, size_t smem, int *max_blocks_per_sm);
cudaError_t launch_g2(int threads, int blocks, size_t smem, const G2Args &a, cudaStream_t s);
cudaError_t g2_prepare(size_t smem);
cudaError_t g2n_prepare();
cudaError_t launch_g2n(int blocks, size_t smem, const G2nArgs &a, cudaStream_t s);
// Tensor-core G2: kernel attributes once; the Toeplitz digit tiles of K
// primes (ntiles per prime, entries t < nvalid of btab); the five launches of
// one class (images -> E/O digits, products, reversed scaled digits,
// products, coefficients), maxM its largest point-pair count.
cudaError_t g2t_prepare();
cudaError_t launch_g2t_btile(const int32_t *btab, int tab_stride, int nvalid, int K, int ntiles, uint16_t *out,
                             cudaStream_t s);
cudaError_t launch_g2t(int ntasks, int nitems, int maxM, const G2tArgs &a, cudaStream_t s);
// Tensor-core CRT digits: kernel attributes; the W digit tiles of blocks
// kb < KB (g3m_wtile_elems(KB) elements); per-tile operand size for K primes.
cudaError_t g3m_prepare();
int64_t g3m_wtile_elems(int KB);
int64_t g3m_tile_elems(int K);
cudaError_t launch_g3m_wtiles(const int32_t *wtab, int K, int KB, uint16_t *out, cudaStream_t s);
int64_t g3m_rtile_elems(int KB);
cudaError_t launch_g3m_rtiles(const int32_t *wtab, int K, int KB, uint16_t *out, cudaStream_t s);
cudaError_t launch_g3m(int ntiles, const G3mArgs &a, cudaStream_t s);
cudaError_t g3l_prepare();
int64_t g3l_block_elems();  // bf16 elements of one (chunk, unit) block of prefix-product tiles
cudaError_t launch_g3l_btiles(const uint16_t *p16, const int32_t *poff, int K, const int32_t *cbase, int KB,
                              int64_t nblocks, uint16_t *out, cudaStream_t s);
cudaError_t launch_g3l(int ntasks, const G3lArgs &a, cudaStream_t s);
cudaError_t launch_bhat(const int32_t *btab, int tab_stride, int nb, int K, int lg, const uint2 *tw,
                        const NttConst &nc, uint32_t *bhat, cudaStream_t s);
// CRT digits by tiles of jt (32 or 16) coefficients (tasks step by jt), any
// prime count.
cudaError_t launch_g3t(int nt, const G3Args &a, const int2 *ttasks, cudaStream_t s, int jt = 32);
// CRT digits with one thread per coefficient (tasks: (pair, first
// coefficient) per block of 128 coefficients, the output kernel's tasks).
cudaError_t launch_g3p(int nt, const G3Args &a, const int2 *tasks, cudaStream_t s);
// Coefficients per SM from which a batch takes the one-thread-per-coefficient
// digit kernel.
#ifndef RS_G3P_MIN_COEF_PER_SM
#define RS_G3P_MIN_COEF_PER_SM 1024
#endif
cudaError_t launch_yun(int ntasks, const YunArgs &a, cudaStream_t s);
// Schur variant of G1: one block per tile, `slots` = ceil((m_y + n_y) / 32)
// over the batch, smem = staged residues of the largest pair; then the
// elimination fallback over the listed images (grid-stride).
cudaError_t launch_g1s(int slots, int ntiles, size_t smem, const G1sArgs &a, cudaStream_t s);
cudaError_t launch_g1s_fallback(int blocks, size_t smem, const G1sArgs &a, cudaStream_t s);
cudaError_t launch_g2s(int ntasks, size_t smem, const G2sArgs &a, cudaStream_t s);
cudaError_t launch_g3bc(int nb, int nc, const G3Args &a, const int2 *otasks, cudaStream_t s);
// Residues of one lifted factor divided by an integer g, prime by prime:
// out[dst_off + k n + j] = in[src_off + k src_stride + j] * (g mod p_k)^{-1}
// mod p_k for k < this factor's primes, j < n; g's 32-bit limbs (least
// significant first) at gw[g_off .. g_off + g_len).
struct ScaleDesc {
  int64_t src_off, dst_off, g_off;
  int32_t src_stride, n, k, g_len;
};
cudaError_t launch_scale(const ScaleDesc *sd, int nf, int kmax, const ModP *mods, const uint32_t *gw,
                         const uint32_t *in, uint32_t *out, cudaStream_t s);
cudaError_t launch_crt_tables(const ModP *mods, int K, int32_t *wtab, cudaStream_t s);
cudaError_t launch_init_primes(const uint32_t *primes, int n, ModP *mods, uint32_t *vtab,
                               uint32_t *crt, uint32_t *qbase, cudaStream_t s);
cudaError_t launch_tables(const ModP *mods, const uint32_t *qbase, int K, int N, int stride,
                          uint32_t *finv, uint32_t *gtab, int32_t *btab, uint32_t *hq, int32_t *qc,
                          uint32_t *qn, uint32_t *qp, cudaStream_t s);
// z[k N + x] and the point of image x for x < N, from images of stride NI.
cudaError_t launch_finalize_images(const ModP *mods, const uint32_t *qbase, const uint32_t *num,
                                   const uint32_t *den, uint32_t *z, uint32_t *points, int K, int N,
                                   int NI, cudaStream_t s);
