// G2 by number-theoretic transforms: the two convolutions of the geometric-
// point interpolation (Section 4.1; see kernels_g23.cu for the formulas)
// computed exactly over Z with three NTT primes and Chinese remaindering,
// then reduced mod the resultant's prime p.
//
// The convolution S_k = sum_{j<=k} x_j b_{k-j}, k < n, of signed residues
// |x_j|, |b_t| < 2^30 satisfies |S_k| < n 2^60 <= 2^72 (n <= 2^12), and the
// three primes below multiply to more than 2^92, so S_k is recovered exactly
// in the symmetric range.  A cyclic transform of length L >= 2n - 1 holds the
// linear convolution without wrap-around when b is truncated to t < L/2
// (terms with t >= n only reach outputs k >= n, which are discarded).
//
// Transforms: forward decimation in frequency (natural order in,
// bit-reversed out), inverse decimation in time (bit-reversed in, natural
// out), so the pointwise product needs no reordering.  Twiddle products use
// Shoup's precomputed quotient w' = floor(w 2^32 / P) (V. Shoup, NTL;
// D. Harvey, "Faster arithmetic for number-theoretic transforms", J. Symb.
// Comput. 60, 2014): for a < 2^32 and w < P, a w - floor(a w' / 2^32) P lies
// in [0, 2P).
#include "../../include/rs.h"
#include "blockinv.cuh"
#include "rs_internal.cuh"

namespace {

__device__ __forceinline__ uint32_t shoup_mul(uint32_t a, uint2 w, uint32_t P) {
  const uint32_t q = __umulhi(a, w.y);
  const uint32_t r = a * w.x - q * P;  // in [0, 2P)
  return rs_umin(r, r - P);
}

__device__ __forceinline__ uint32_t add_p(uint32_t a, uint32_t b, uint32_t P) {
  const uint32_t s = a + b;  // < 2P < 2^32
  return rs_umin(s, s - P);
}

// A twiddle pair of stage row l (w_{2^l}^j): shared-memory rows 1 .. lg-1,
// the top row lg from global memory.
__device__ __forceinline__ uint2 twiddle(const uint2 *rows, const uint2 *top, int l, int lg, int j) {
  return l == lg ? __ldg(top + j) : rows[(1 << (l - 1)) - 1 + j];
}

// A 16-entry group of shared memory in registers and back.  Thread t moves
// its group's four 16-byte chunks starting with chunk (t / 2) mod 4, so the
// eight threads of a quarter warp (groups 64 bytes apart) always touch eight
// different 16-byte bank groups.
#ifndef RS_G2N_ROTATE
#define RS_G2N_ROTATE 1
#endif
#ifndef RS_G2N_MINB
#define RS_G2N_MINB 3  // resident blocks per SM requested from ptxas (caps registers at 85)
#endif

__device__ __forceinline__ void load16(const uint32_t *g, uint32_t (&x)[16]) {
  const int h = RS_G2N_ROTATE ? (threadIdx.x >> 1) & 3 : 0;
  const uint4 *g4 = reinterpret_cast<const uint4 *>(g);
  uint4 v[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) v[q] = g4[(q + h) & 3];
#pragma unroll
  for (int c = 0; c < 4; ++c) {  // chunk c is v[(c - h) mod 4]
    const uint4 a0 = v[(c + 4) & 3], a1 = v[(c + 3) & 3], a2 = v[(c + 2) & 3], a3 = v[(c + 1) & 3];
    const uint4 u = h == 0 ? a0 : h == 1 ? a1 : h == 2 ? a2 : a3;
    x[4 * c] = u.x;
    x[4 * c + 1] = u.y;
    x[4 * c + 2] = u.z;
    x[4 * c + 3] = u.w;
  }
}

__device__ __forceinline__ void store16(uint32_t *g, const uint32_t (&x)[16]) {
  const int h = RS_G2N_ROTATE ? (threadIdx.x >> 1) & 3 : 0;
  uint4 *g4 = reinterpret_cast<uint4 *>(g);
#pragma unroll
  for (int q = 0; q < 4; ++q) {  // chunk (q + h) mod 4
    const uint4 c0 = make_uint4(x[(4 * q) & 15], x[(4 * q + 1) & 15], x[(4 * q + 2) & 15], x[(4 * q + 3) & 15]);
    const uint4 c1 = make_uint4(x[(4 * q + 4) & 15], x[(4 * q + 5) & 15], x[(4 * q + 6) & 15], x[(4 * q + 7) & 15]);
    const uint4 c2 = make_uint4(x[(4 * q + 8) & 15], x[(4 * q + 9) & 15], x[(4 * q + 10) & 15], x[(4 * q + 11) & 15]);
    const uint4 c3 = make_uint4(x[(4 * q + 12) & 15], x[(4 * q + 13) & 15], x[(4 * q + 14) & 15], x[(4 * q + 15) & 15]);
    g4[(q + h) & 3] = h == 0 ? c0 : h == 1 ? c1 : h == 2 ? c2 : c3;
  }
}

// The two radix-4 passes with the smallest strides (quarter sizes 4 and 1)
// only combine entries inside aligned groups of 16, so one thread takes a
// whole group: four 16-byte shared loads, both passes in registers with the
// 14 twiddles every group shares, four 16-byte stores.  (Done pass by pass,
// those strides made 2- to 4-way shared-memory bank conflicts.)
__device__ __forceinline__ void dif16_tail(uint32_t *a, int lg, const uint2 *rows, const uint2 *top, uint32_t P) {
  uint2 w16[8], w8[4];
#pragma unroll
  for (int j = 0; j < 8; ++j) w16[j] = twiddle(rows, top, 4, lg, j);
#pragma unroll
  for (int j = 0; j < 4; ++j) w8[j] = twiddle(rows, top, 3, lg, j);
  const uint2 w4a = twiddle(rows, top, 2, lg, 0), w4b = twiddle(rows, top, 2, lg, 1);
  const uint2 w2 = twiddle(rows, top, 1, lg, 0);
  const int groups = 1 << (lg - 4);
  for (int gi = threadIdx.x; gi < groups; gi += blockDim.x) {
    uint32_t x[16];
    load16(a + 16 * gi, x);
#pragma unroll
    for (int j = 0; j < 4; ++j) {  // half-sizes 8 and 4: entries j, j + 4, j + 8, j + 12
      const uint32_t x0 = x[j], x1 = x[j + 4], x2 = x[j + 8], x3 = x[j + 12];
      const uint32_t y0 = add_p(x0, x2, P), y1 = add_p(x1, x3, P);
      const uint32_t y2 = shoup_mul(x0 + P - x2, w16[j], P);
      const uint32_t y3 = shoup_mul(x1 + P - x3, w16[j + 4], P);
      x[j] = add_p(y0, y1, P);
      x[j + 4] = shoup_mul(y0 + P - y1, w8[j], P);
      x[j + 8] = add_p(y2, y3, P);
      x[j + 12] = shoup_mul(y2 + P - y3, w8[j], P);
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) {  // half-sizes 2 and 1: entries 4 m .. 4 m + 3
      const uint32_t x0 = x[4 * m], x1 = x[4 * m + 1], x2 = x[4 * m + 2], x3 = x[4 * m + 3];
      const uint32_t y0 = add_p(x0, x2, P), y1 = add_p(x1, x3, P);
      const uint32_t y2 = shoup_mul(x0 + P - x2, w4a, P);
      const uint32_t y3 = shoup_mul(x1 + P - x3, w4b, P);
      x[4 * m] = add_p(y0, y1, P);
      x[4 * m + 1] = shoup_mul(y0 + P - y1, w2, P);
      x[4 * m + 2] = add_p(y2, y3, P);
      x[4 * m + 3] = shoup_mul(y2 + P - y3, w2, P);
    }
    store16(a + 16 * gi, x);
  }
  __syncthreads();
}

// The inverse's first two passes (quarter sizes 1 and 4) the same way.
__device__ __forceinline__ void dit16_head(uint32_t *a, int lg, const uint2 *irows, const uint2 *top, uint32_t P) {
  uint2 w16[8], w8[4];
#pragma unroll
  for (int j = 0; j < 8; ++j) w16[j] = twiddle(irows, top, 4, lg, j);
#pragma unroll
  for (int j = 0; j < 4; ++j) w8[j] = twiddle(irows, top, 3, lg, j);
  const uint2 w4a = twiddle(irows, top, 2, lg, 0), w4b = twiddle(irows, top, 2, lg, 1);
  const uint2 w2 = twiddle(irows, top, 1, lg, 0);
  const int groups = 1 << (lg - 4);
  for (int gi = threadIdx.x; gi < groups; gi += blockDim.x) {
    uint32_t x[16];
    load16(a + 16 * gi, x);
#pragma unroll
    for (int m = 0; m < 4; ++m) {  // half-sizes 1 and 2: entries 4 m .. 4 m + 3
      const uint32_t v1 = shoup_mul(x[4 * m + 1], w2, P), v3 = shoup_mul(x[4 * m + 3], w2, P);
      const uint32_t x0 = x[4 * m], x2 = x[4 * m + 2];
      const uint32_t y0 = add_p(x0, v1, P), y1 = x0 + P - v1;
      const uint32_t y2 = add_p(x2, v3, P), y3 = x2 + P - v3;
      const uint32_t u2 = shoup_mul(y2, w4a, P);
      const uint32_t u3 = shoup_mul(y3, w4b, P);
      const uint32_t z1 = rs_umin(y1, y1 - P);
      x[4 * m] = add_p(y0, u2, P);
      x[4 * m + 2] = y0 + P - u2 - (y0 + P - u2 >= P ? P : 0);
      x[4 * m + 1] = add_p(z1, u3, P);
      x[4 * m + 3] = z1 + P - u3 - (z1 + P - u3 >= P ? P : 0);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {  // half-sizes 4 and 8: entries j, j + 4, j + 8, j + 12
      const uint32_t v1 = shoup_mul(x[j + 4], w8[j], P), v3 = shoup_mul(x[j + 12], w8[j], P);
      const uint32_t x0 = x[j], x2 = x[j + 8];
      const uint32_t y0 = add_p(x0, v1, P), y1 = x0 + P - v1;
      const uint32_t y2 = add_p(x2, v3, P), y3 = x2 + P - v3;
      const uint32_t u2 = shoup_mul(y2, w16[j], P);
      const uint32_t u3 = shoup_mul(y3, w16[j + 4], P);
      const uint32_t z1 = rs_umin(y1, y1 - P);
      x[j] = add_p(y0, u2, P);
      x[j + 8] = y0 + P - u2 - (y0 + P - u2 >= P ? P : 0);
      x[j + 4] = add_p(z1, u3, P);
      x[j + 12] = z1 + P - u3 - (z1 + P - u3 >= P ? P : 0);
    }
    store16(a + 16 * gi, x);
  }
  __syncthreads();
}

// Forward transform of a[0, L), L = 2^lg, in shared memory: decimation in
// frequency, two stages per pass (radix 4) plus one radix-2 pass when lg is
// odd.  Twiddle row l holds (w_{2^l}^j, Shoup quotient) for j < 2^(l-1); a
// stage reads its own row, so neighbouring lanes read neighbouring entries.
// rows: rows 1 .. lg-1 staged in shared memory (row l at 2^(l-1) - 1); top:
// row lg, read by one pass only, from global memory (coalesced).
__device__ void ntt_dif(uint32_t *a, int lg, const uint2 *rows, const uint2 *top, uint32_t P) {
  const int L = 1 << lg;
  int s = lg - 1;  // half-size of the next stage is 2^s
  if (lg & 1) {    // radix-2 pass: h = L/2, twiddle w^j
    const int h = L >> 1;
    for (int j = threadIdx.x; j < h; j += blockDim.x) {
      const uint32_t u = a[j], v = a[j + h];
      a[j] = add_p(u, v, P);
      a[j + h] = shoup_mul(u + P - v, __ldg(top + j), P);
    }
    __syncthreads();
    --s;
  }
  const int s_end = lg >= 4 ? 3 : 0;  // with lg >= 4 the last two passes run as 16-entry groups
  for (; s > s_end; s -= 2) {  // stages with half-sizes h = 2^s and q = h/2
    const int q = 1 << (s - 1), h = q << 1;
    const bool gtop = s + 1 == lg;  // w_{2h}^j from the global top row (block-uniform)
    const uint2 *r1 = rows + (h - 1), *r0 = rows + (q - 1);  // w_{2h}^j and w_h^j in shared memory
    for (int t = threadIdx.x; t < (L >> 2); t += blockDim.x) {
      const int j = t & (q - 1), base = (t >> (s - 1)) << (s + 1);
      uint32_t *x = a + base + j;
      const uint32_t x0 = x[0], x1 = x[q], x2 = x[h], x3 = x[h + q];
      const uint32_t y0 = add_p(x0, x2, P), y1 = add_p(x1, x3, P);
      const uint2 wa = gtop ? __ldg(top + j) : r1[j], wb = gtop ? __ldg(top + j + q) : r1[j + q];
      const uint32_t y2 = shoup_mul(x0 + P - x2, wa, P);
      const uint32_t y3 = shoup_mul(x1 + P - x3, wb, P);
      const uint2 w = r0[j];
      x[0] = add_p(y0, y1, P);
      x[q] = shoup_mul(y0 + P - y1, w, P);
      x[h] = add_p(y2, y3, P);
      x[h + q] = shoup_mul(y2 + P - y3, w, P);
    }
    __syncthreads();
  }
  if (lg >= 4) dif16_tail(a, lg, rows, top, P);
}

// Inverse transform (without the 1/L factor) of a bit-reversed a: decimation
// in time, radix-4 passes plus one radix-2 pass when lg is odd; irows and
// top as in ntt_dif with the inverse roots.
__device__ void ntt_dit_inv(uint32_t *a, int lg, const uint2 *irows, const uint2 *top, uint32_t P) {
  const int L = 1 << lg;
  int s = 0;
  if (lg >= 4) {  // the first two passes as 16-entry groups
    dit16_head(a, lg, irows, top, P);
    s = 4;
  }
  for (; s + 1 < lg; s += 2) {  // stages with half-sizes q = 2^s and h = 2q
    const int q = 1 << s, h = q << 1;
    const bool gtop = s + 2 == lg;  // w_{4q}^-j from the global top row (block-uniform)
    const uint2 *r1 = irows + (q - 1), *r2 = irows + (h - 1);  // w_{2q}^-j, w_{4q}^-j in shared memory
    for (int t = threadIdx.x; t < (L >> 2); t += blockDim.x) {
      const int j = t & (q - 1), base = (t >> s) << (s + 2);
      uint32_t *x = a + base + j;
      const uint2 w = r1[j];
      const uint32_t v1 = shoup_mul(x[q], w, P), v3 = shoup_mul(x[h + q], w, P);
      const uint32_t x0 = x[0], x2 = x[h];
      const uint32_t y0 = add_p(x0, v1, P), y1 = x0 + P - v1;
      const uint32_t y2 = add_p(x2, v3, P), y3 = x2 + P - v3;
      const uint2 wa = gtop ? __ldg(top + j) : r2[j], wb = gtop ? __ldg(top + j + q) : r2[j + q];
      const uint32_t u2 = shoup_mul(y2, wa, P);
      const uint32_t u3 = shoup_mul(y3, wb, P);
      const uint32_t z1 = rs_umin(y1, y1 - P);
      x[0] = add_p(y0, u2, P);
      x[h] = y0 + P - u2 - (y0 + P - u2 >= P ? P : 0);
      x[q] = add_p(z1, u3, P);
      x[h + q] = z1 + P - u3 - (z1 + P - u3 >= P ? P : 0);
    }
    __syncthreads();
  }
  if (s < lg) {  // radix-2 pass: h = L/2, twiddle w^-j
    const int h = L >> 1;
    for (int j = threadIdx.x; j < h; j += blockDim.x) {
      const uint32_t u = a[j], v = shoup_mul(a[j + h], __ldg(top + j), P);
      a[j] = add_p(u, v, P);
      const uint32_t d = u + P - v;
      a[j + h] = rs_umin(d, d - P);
    }
    __syncthreads();
  }
}

// Stage the twiddle rows 1 .. lg-1 (2^(lg-1) - 1 entries, contiguous at the
// start of the compact table) into shared memory.
__device__ __forceinline__ void stage_twiddles(uint2 *dst, const uint2 *table, int lg) {
  const int n = (1 << (lg - 1)) - 1;
#pragma unroll 4
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = __ldg(table + i);
}

__device__ __forceinline__ uint32_t lift(int32_t v, uint32_t P) { return v < 0 ? (uint32_t)(v + (int32_t)P) : (uint32_t)v; }

// out[k] = S_k R^-1 mod p for k < N (the Montgomery form of the convolution
// of Montgomery-form inputs, as the direct kernel produces).  bhat: this
// prime's three transformed kernels [3][L] (Montgomery form, 1/L folded in).
// W holds L words, TWS L/2 twiddles, V0 and V1 N words each; out may alias V0.
__device__ void conv_ntt(const int32_t *x, int N, int lg, const uint32_t *bhat, const G2nArgs &a, uint32_t *W,
                         uint2 *TWS, uint32_t *V0, uint32_t *V1, uint32_t *out, const ModP &m, uint32_t cp0,
                         uint32_t cp01, uint32_t cneg) {
  const int L = 1 << lg, T = blockDim.x;
  constexpr int TWROW = 1 << RS_NTT_LGMAX;  // compact twiddle rows of one (prime, direction)
  for (int q = 0; q < 3; ++q) {
    const ModP P = a.nc.m[q];
    for (int i = threadIdx.x; i < L; i += T) W[i] = i < N ? lift(x[i], P.p) : 0u;
    const uint2 *fw = a.tw + (size_t)(2 * q) * TWROW, *iw = a.tw + (size_t)(2 * q + 1) * TWROW;
    stage_twiddles(TWS, fw, lg);
    __syncthreads();
    ntt_dif(W, lg, TWS, fw + ((L >> 1) - 1), P.p);
    const uint32_t *bh = bhat + (size_t)q * L;
#pragma unroll 4
    for (int i = threadIdx.x; i < L; i += T) W[i] = mmul(W[i], __ldg(bh + i), P);
    stage_twiddles(TWS, iw, lg);
    __syncthreads();
    ntt_dit_inv(W, lg, TWS, iw + ((L >> 1) - 1), P.p);
    // Garner over (P0, P1, P2), P0 < P1 < P2 < p: S = v0 + v1 P0 + v2 P0 P1,
    // negative when v2 > P2 / 2.
    for (int i = threadIdx.x; i < N; i += T) {
      if (q == 0) {
        V0[i] = W[i];
      } else if (q == 1) {
        V1[i] = mmul(msub(W[i], V0[i], P.p), a.nc.c01, P);
      } else {
        const uint32_t v0 = V0[i], v1 = V1[i];
        const uint32_t t = mmul(v1, a.nc.p0_m2, P);
        const uint32_t v2 = mmul(msub(msub(W[i], v0, P.p), t, P.p), a.nc.c012, P);
        uint32_t r = madd(madd(redc((uint64_t)v0, m.p, m.pinv), mmul(v1, cp0, m), m.p), mmul(v2, cp01, m), m.p);
        if (v2 > (P.p >> 1)) r = msub(r, cneg, m.p);
        out[i] = r;
      }
    }
    __syncthreads();
  }
}

__device__ __forceinline__ int32_t srep(uint32_t v, uint32_t p) {
  return v > (p >> 1) ? (int32_t)v - (int32_t)p : (int32_t)v;
}

// One block per (pair, prime) whose transform length is 2^lg (2^lg >= 2M - 1
// for the M = NI / 2 point pairs).  As in the direct kernel, the paired
// images give E(Q^i) and O(Q^i), interpolated in turn into the even and the
// odd coefficients.  Shared memory: X, V0, V1, Oh (M words each), W (2^lg
// words), twiddle rows 1 .. lg-1 (2^(lg-1) - 1 pairs).
__global__ void __launch_bounds__(256, RS_G2N_MINB) g2n_kernel(G2nArgs a) {
  extern __shared__ __align__(16) uint32_t sm[];
  __shared__ uint32_t scratch[128];
  const int2 task = a.tasks[blockIdx.x];
  const PairDesc pd = a.pairs[task.x];
  const ModP m = a.mods[task.y];
  const int N = pd.N, NI = pd.NI, M = NI >> 1, D = M - 1, T = blockDim.x, tid = threadIdx.x;
  const int Mp = (M + 3) & ~3;
  int32_t *X = reinterpret_cast<int32_t *>(sm);
  uint32_t *V0 = reinterpret_cast<uint32_t *>(X + Mp);
  uint32_t *V1 = V0 + Mp;
  uint32_t *Oh = V1 + Mp;
  uint32_t *W = Oh + Mp;
  uint2 *TWS = reinterpret_cast<uint2 *>(W + (1 << a.lg));
  const size_t base = (size_t)pd.img_off + (size_t)task.y * NI;
  const size_t tb = (size_t)task.y * a.tab_stride;
  const uint32_t *finv = a.finv + tb, *gt = a.gtab + tb, *hq = a.hq + tb;
  const uint32_t *bhat = a.bhat + (size_t)task.y * 3 * ((size_t)1 << a.lg);
  // P0 < p, so P0 mod p = P0; P0 P1 mod p and P0 P1 P2 mod p once per block.
  const uint32_t cp0 = a.nc.m[0].p;
  const uint32_t cp01 = (uint32_t)(((uint64_t)a.nc.m[0].p * a.nc.m[1].p) % m.p);
  const uint32_t cneg = redc((uint64_t)(((uint64_t)cp01 * a.nc.m[2].p) % m.p), m.p, m.pinv);  // P R^-1 mod p

  for (int i = tid; i < M; i += T) V0[i] = mmul(a.den[base + 2 * i], a.den[base + 2 * i + 1], m);
  __syncthreads();
  batch_invert(V0, V1, M, m, scratch);
  __syncthreads();
  for (int i = tid; i < M; i += T) {
    const uint32_t np = a.num[base + 2 * i], dp = a.den[base + 2 * i];
    const uint32_t nm = a.num[base + 2 * i + 1], dm = a.den[base + 2 * i + 1];
    const uint32_t e = mmul(mmul2(np, dm, nm, dp, m), V1[i], m);             // z+ + z-
    const uint32_t o = mmul(mmul2(np, dm, mneg(nm, m.p), dp, m), V1[i], m);  // z+ - z-
    X[i] = srep(mmul(mmul(e, hq[0], m), finv[i], m), m.p);  // (E / F_i); hq[0] = 1/2
    Oh[i] = mmul(mmul(o, hq[i], m), finv[i], m);             // (O / F_i)
  }
  __syncthreads();
  for (int half = 0; half < 2; ++half) {  // E: even coefficients, then O: odd ones
    conv_ntt(X, M, a.lg, bhat, a, W, TWS, V0, V1, V0, m, cp0, cp01, cneg);  // V0[k] = Q^{C(k,2)} c_k
    for (int k = tid; k < M; k += T) X[D - k] = srep(mmul(V0[k], gt[k], m), m.p);  // c_k F_k reversed
    __syncthreads();
    conv_ntt(X, M, a.lg, bhat, a, W, TWS, V0, V1, V0, m, cp0, cp01, cneg);
    for (int i = tid; i < M; i += T) {
      const int c = 2 * i + half;
      if (c < N) a.coef[base + c] = from_mont(mmul(V0[D - i], finv[i], m), m);
    }
    if (half == 0) {
      for (int i = tid; i < M; i += T) X[i] = srep(Oh[i], m.p);
      __syncthreads();
    }
  }
}

// bhat[k][q][i] for prime k < K and NTT prime q: the forward transform of
// b_t mod P_q (t < min(L/2, nb), zero beyond) times 1/L, in Montgomery form
// mod P_q.  One block per (k, q); shared memory 2^lg words.
__global__ void __launch_bounds__(256) bhat_kernel(const int32_t *btab, int tab_stride, int nb, int K, int lg,
                                                   const uint2 *tw, NttConst nc, uint32_t *bhat) {
  extern __shared__ __align__(16) uint32_t sm[];
  const int k = blockIdx.x / 3, q = blockIdx.x - 3 * (blockIdx.x / 3);
  if (k >= K) return;
  const ModP P = nc.m[q];
  const int L = 1 << lg, lim = min(L / 2, nb);
  uint2 *TWS = reinterpret_cast<uint2 *>(sm + L);  // twiddle rows 1 .. lg-1
  const int32_t *b = btab + (size_t)k * tab_stride;
  for (int i = threadIdx.x; i < L; i += blockDim.x) sm[i] = i < lim ? lift(b[i], P.p) : 0u;
  const uint2 *fw = tw + (size_t)(2 * q) * (1 << RS_NTT_LGMAX);
  stage_twiddles(TWS, fw, lg);
  __syncthreads();
  ntt_dif(sm, lg, TWS, fw + ((L >> 1) - 1), P.p);
  // 1/L = -(P - 1)/L mod P (L divides P - 1); times R^2 so that mmul gives (bhat / L) R
  const uint32_t linv = P.p - (P.p - 1u) / (uint32_t)L;
  const uint32_t sc = to_mont(to_mont(linv, P), P);
  uint32_t *out = bhat + ((size_t)k * 3 + q) * L;
  for (int i = threadIdx.x; i < L; i += blockDim.x) out[i] = mmul(sm[i], sc, P);
}

}  // namespace

cudaError_t g2n_prepare() {
  return cudaFuncSetAttribute(g2n_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, RS_G2N_MAX_SMEM_BYTES);
}

cudaError_t launch_g2n(int blocks, size_t smem, const G2nArgs &a, cudaStream_t s) {
  g2n_kernel<<<blocks, 256, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_bhat(const int32_t *btab, int tab_stride, int nb, int K, int lg, const uint2 *tw,
                        const NttConst &nc, uint32_t *bhat, cudaStream_t s) {
  const size_t smem = ((size_t)1 << lg) * 8;  // data and twiddle rows
  cudaError_t e = cudaFuncSetAttribute(bhat_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  bhat_kernel<<<3 * K, 256, smem, s>>>(btab, tab_stride, nb, K, lg, tw, nc, bhat);
  return cudaGetLastError();
}
