// G1: fused modular reduction + evaluation + univariate resultant, one
// thread per modular image (pair, prime p, point x_i).  Paper, Section 4.1:
// Collins' algorithm maps f, g to Z_p and evaluates them at points x_i
// (steps 1-2), then takes z_i^{(p)} = res(f(x_i, y), g(x_i, y), y) in Z_p.
// The points come in pairs +-q^i (q of multiplicative order above the
// largest point count, chosen per prime).  With f_j(x) = E_j(x^2) + x O_j(x^2)
// (even and odd parts), both images of a pair need E_j(Q^i) and x O_j(Q^i)
// only, Q = q^2, x = q^i: the sums of f_{j,k} q^{ik} over the even and over
// the odd k.  The two threads of a pair each take one parity, as a
// correlation of chirp-scaled coefficients with the sequence q^{C(t,2)}
// (accumulated without per-term reduction), and exchange it with a shuffle:
// f_j(+-q^i) = E_j(Q^i) +- q^i O_j(Q^i).  G2 splits the images back into
// E and O and interpolates each with two convolutions.
//
// The univariate resultant keeps the formal degrees (a, b) = (m_y, n_y) of
// the Sylvester matrix of Section 3.1, so z_i^{(p)} = R^{(y)}(x_i) mod p for
// every prime and point.  It is computed by a division-free remainder
// sequence on the two coefficient vectors held in registers, top-aligned
// (index 0 = leading coefficient), with one final inversion left to G2:
//
//   a >= b, l_B != 0:  A' = l_B A - l_A y^(a-b) B  (top term cancels, formal
//                      degree a-1);  Res_{a,b}(A,B) l_B^{b-1} = (-1)^b Res_{a-1,b}(A',B)
//   a <  b, l_A != 0:  B' = l_A B - l_B y^(b-a) A;  Res_{a,b}(A,B) l_A^{a-1} = Res_{a,b-1}(A,B')
//   a >= b, l_B == 0:  Res_{a,b}(A,B) = l_A Res_{a,b-1}(A, B without its zero top)
//   a <  b, l_A == 0:  Res_{a,b}(A,B) = (-1)^b l_B Res_{a-1,b}(A without its zero top, B)
//   Res_{0,b}(A,B) = A_0^b,  Res_{a,0}(A,B) = B_0^a
//
// (each identity is a row operation on the Sylvester matrix followed by a
// cofactor expansion along its first column).  The pivot powers
// prod_t c_t^{e_t}, e_t = deg(pivot_t) - 1, are non-increasing in t, so they
// are accumulated by Abel summation: with Q_t = c_1 ... c_t,
// prod_t c_t^{e_t} = prod_t Q_t^{e_t - e_{t+1}}: one product per step into Q
// and one into the denominator whenever e drops.
//
// Register arrays have a compile-time capacity C; once both degrees fit in
// C - 8 entries the state moves to arrays of C - 8 (registers are renamed,
// nothing is copied), so the unrolled update loops shrink with the degrees.
#include "rs_internal.cuh"

#ifndef RS_G1_PSTEP
#define RS_G1_PSTEP 12  // register capacity dropped per phase
#endif
// Minimum resident 128-thread blocks per SM requested from ptxas per register
// capacity (caps registers at 65536 / (128 * MINB) per thread).
#if defined(RS_G1_MINB_AT) && defined(RS_G1_MINB_SET) && RS_G1_MINB_AT == RS_G1_CAP
#define RS_G1_MINB RS_G1_MINB_SET  // tuning override for one capacity
#endif
#ifndef RS_G1_MINB
#define RS_G1_MINB (RS_G1_CAP <= 24 ? 6 : RS_G1_CAP <= 48 ? 4 : 3)
#endif

namespace {

struct Prs {
  int a, b;        // formal degrees of A and B
  uint32_t num;    // numerator (Montgomery form)
  uint32_t den;    // accumulated pivot powers (Montgomery form)
  uint32_t Q;      // running product of pivots
  int eprev;       // exponent of the previous pivot
  uint32_t sign;   // parity of the accumulated (-1) factors
  uint32_t degen;  // a zero pivot was met
};

__device__ __forceinline__ void settle(Prs &s, int e, uint32_t c, const ModP &m) {
  while (s.eprev > e) {
    s.den = mmul(s.den, s.Q, m);
    --s.eprev;
  }
  s.Q = mmul(s.Q, c, m);
  s.eprev = e;
}

// Entries I .. C - 2 of a reduction whose result has `live` entries: entry
// I is computed while I < live, entry `live` (the old constant term shifted
// out) becomes zero, and the zero padding beyond it is left alone.  The
// degrees are the same for every image of a tile, so these branches are
// uniform across the warp and skip the padding instead of multiplying zeros.
template <int C, int I>
__device__ __forceinline__ void reduce_tail(uint32_t (&P)[C], const uint32_t (&V)[C], uint32_t w1, uint32_t w2,
                                            const ModP &m, int live) {
  if constexpr (I < C - 1) {
    if (live > I) {
      P[I] = mmul2(P[I + 1], w1, V[I + 1], w2, m);
      reduce_tail<C, I + 1>(P, V, w1, w2, m, live);
    } else {
      P[I] = 0u;
    }
  }
}

// P[i] <- w1 P[i+1] + w2 V[i+1] for i < live (the reduced polynomial's
// entries); the top entry (which cancels) is dropped.  Every caller reduces
// an array whose degree is at least C - 8 (the phase condition), so the
// first C - 8 entries are always live and only the last 7 are checked.
template <int C>
__device__ __forceinline__ void reduce_into(uint32_t (&P)[C], const uint32_t (&V)[C], uint32_t w1,
                                            uint32_t w2, const ModP &m, int live) {
  constexpr int H = C > RS_G1_PSTEP ? C - RS_G1_PSTEP : 0;
#pragma unroll
  for (int i = 0; i < H; ++i) P[i] = mmul2(P[i + 1], w1, V[i + 1], w2, m);
  reduce_tail<C, H>(P, V, w1, w2, m, live);
  P[C - 1] = 0u;
}

template <int C>
__device__ __forceinline__ void drop_top(uint32_t (&P)[C]) {
#pragma unroll
  for (int i = 0; i < C - 1; ++i) P[i] = P[i + 1];
  P[C - 1] = 0u;
}

// One normal step on A (a >= b, l_B != 0) or on B (a < b, l_A != 0).
template <int C>
__device__ __forceinline__ void step_a(uint32_t (&A)[C], const uint32_t (&B)[C], Prs &s, const ModP &m) {
  const uint32_t lb = B[0], la = A[0];
  settle(s, s.b - 1, lb, m);
  reduce_into<C>(A, B, lb, mneg(la, m.p), m, s.a);
  s.sign ^= (uint32_t)(s.b & 1);
  --s.a;
}

template <int C>
__device__ __forceinline__ void step_b(const uint32_t (&A)[C], uint32_t (&B)[C], Prs &s, const ModP &m) {
  const uint32_t la = A[0], lb = B[0];
  settle(s, s.a - 1, la, m);
  reduce_into<C>(B, A, la, mneg(lb, m.p), m, s.b);
  --s.b;
}

template <int C>
__device__ __forceinline__ void prs_run(uint32_t (&A)[C], uint32_t (&B)[C], Prs &s, const ModP &m) {
  // invariant: a, b <= C - 1
  constexpr int S = RS_G1_PSTEP;
  // Fast path for the normal sequence, with a fixed role for each array in
  // every loop (no data-dependent choice of which array to update): first
  // reduce the larger degree down to the smaller, then alternate A, B.
  while (s.a > s.b && s.b > 0 && B[0] != 0u && (C <= S || s.a > C - S - 1)) step_a<C>(A, B, s, m);
  while (s.b > s.a && s.a > 0 && A[0] != 0u && (C <= S || s.b > C - S - 1)) step_b<C>(A, B, s, m);
  while (s.a == s.b && s.a > 1 && B[0] != 0u && (C <= S || s.a > C - S - 1)) {
    step_a<C>(A, B, s, m);  // (a, a) -> (a - 1, a)
    if (A[0] == 0u) break;
    step_b<C>(A, B, s, m);  // (a - 1, a) -> (a - 1, a - 1)
  }
  // General steps: zero pivots, the last steps, and the phase boundary.
  while (s.a > 0 && s.b > 0 && (C <= S || s.a > C - S - 1 || s.b > C - S - 1)) {
    if (s.a >= s.b) {
      const uint32_t lb = B[0];
      if (lb != 0u) {
        const uint32_t la = A[0];
        settle(s, s.b - 1, lb, m);
        reduce_into<C>(A, B, lb, mneg(la, m.p), m, s.a);
        s.sign ^= (uint32_t)(s.b & 1);
        --s.a;
      } else {
        s.num = mmul(s.num, A[0], m);
        drop_top<C>(B);
        --s.b;
        s.degen = 1u;
      }
    } else {
      const uint32_t la = A[0];
      if (la != 0u) {
        const uint32_t lb = B[0];
        settle(s, s.a - 1, la, m);
        reduce_into<C>(B, A, la, mneg(lb, m.p), m, s.b);
        --s.b;
      } else {
        s.num = mmul(s.num, B[0], m);
        s.sign ^= (uint32_t)(s.b & 1);
        drop_top<C>(A);
        --s.a;
        s.degen = 1u;
      }
    }
  }
  if constexpr (C > S) {
    if (s.a > 0 && s.b > 0) {
      uint32_t A2[C - S], B2[C - S];
#pragma unroll
      for (int i = 0; i < C - S; ++i) {
        A2[i] = A[i];
        B2[i] = B[i];
      }
      prs_run<C - S>(A2, B2, s, m);
      return;
    }
  }
  if (s.a == 0)
    s.num = mmul(s.num, mpow(A[0], (uint32_t)s.b, m), m);
  else
    s.num = mmul(s.num, mpow(B[0], (uint32_t)s.a, m), m);
}

// Montgomery form of a two's-complement limb integer:
// sum_l limb_l 2^(32 l) R - [negative] 2^(32 L) R, with V[l] = 2^(32 l) R^2.
__device__ __forceinline__ uint32_t reduce_coef(const uint32_t *src, int L, const uint32_t *V,
                                                const ModP &m) {
  uint32_t acc = 0u;
  for (int l = 0; l < L; ++l) acc = madd(acc, redc((uint64_t)src[l] * V[l], m.p, m.pinv), m.p);
  if (src[L - 1] >> 31) acc = msub(acc, redc((uint64_t)V[L], m.p, m.pinv), m.p);
  return acc;
}

__device__ __forceinline__ int32_t signed_rep(uint32_t v, uint32_t p) {
  return v > (p >> 1) ? (int32_t)v - (int32_t)p : (int32_t)v;
}

// Evaluation of the sum over the k of parity par (0 even, 1 odd) at x = q^i
// by the chirp identity i k = C(i+k,2) - C(i,2) - C(k,2):
//   sum_{k = par mod 2} f_{j,k} q^{ik} = q^{-C(i,2)} sum_{k = par mod 2} (f_{j,k} q^{-C(k,2)}) q^{C(i+k,2)},
// which is E_j(Q^i) for par = 0 and x O_j(Q^i) for par = 1.  The factor
// w_i = q^{-C(i,2)} is the same for every coefficient of f and g at the point
// pair, and the Sylvester determinant is homogeneous of degree n_y in the
// f-entries and m_y in the g-entries, so the coefficients are left without
// it and the image is multiplied by w_i^(m_y + n_y) at the end.  The staged
// coefficients a[k][r] = f_{deg-r,k} q^{-C(k,2)} (top-aligned in r, zero past
// the degree) and the window w[t] = q^{C(x0+t,2)} are signed representatives
// (|v| < 2^30): 7 products accumulate exactly in an int64, then one fold
// S = hi 2^32 + lo -> hi (2^32 mod p) + lo keeps |S| < 2^53.
__device__ __forceinline__ int64_t fold64(int64_t s, uint32_t c32) { return rs_fold64(s, c32); }

__device__ __forceinline__ uint32_t finish64(int64_t s, const ModP &m) {
  return redc((uint64_t)(s + ((int64_t)m.p << 22)), m.p, m.pinv);  // 0 <= . < 2^54 < p 2^32
}

template <int C>
__device__ __forceinline__ void eval_chirp(uint32_t (&P)[C], const int32_t *sa, const int2 *meta,
                                           int deg, const int32_t *win, int par, const ModP &m) {
  const uint32_t c32 = m.r1;  // 2^32 mod p (<= 2^21 for every table prime)
#pragma unroll
  for (int r0 = 0; r0 < C; r0 += 8) {
    int64_t acc[8];
#pragma unroll
    for (int rr = 0; rr < 8; ++rr) acc[rr] = 0;
    int kmax = -1;
#pragma unroll
    for (int rr = 0; rr < 8; ++rr)
      if (deg - (r0 + rr) >= 0) kmax = max(kmax, meta[deg - (r0 + rr)].y);
    auto step = [&](int k) {
      const int32_t c = win[k];
      const int4 lo = *reinterpret_cast<const int4 *>(sa + k * C + r0);
      const int4 hi = *reinterpret_cast<const int4 *>(sa + k * C + r0 + 4);
      acc[0] = rs_mac_s32(acc[0], lo.x, c);
      acc[1] = rs_mac_s32(acc[1], lo.y, c);
      acc[2] = rs_mac_s32(acc[2], lo.z, c);
      acc[3] = rs_mac_s32(acc[3], lo.w, c);
      acc[4] = rs_mac_s32(acc[4], hi.x, c);
      acc[5] = rs_mac_s32(acc[5], hi.y, c);
      acc[6] = rs_mac_s32(acc[6], hi.z, c);
      acc[7] = rs_mac_s32(acc[7], hi.w, c);
    };
    // rows par, par + 2, ... (window entry k): full groups of 7 products per
    // fold unrolled, then the rest
    int k = par;
#pragma unroll 1
    for (; k + 12 <= kmax; k += 14) {
#pragma unroll
      for (int u = 0; u < 7; ++u) step(k + 2 * u);
#pragma unroll
      for (int rr = 0; rr < 8; ++rr) acc[rr] = fold64(acc[rr], c32);
    }
#pragma unroll 1
    for (; k <= kmax; k += 2) step(k);
#pragma unroll
    for (int rr = 0; rr < 8; ++rr) acc[rr] = fold64(acc[rr], c32);
#pragma unroll
    for (int rr = 0; rr < 8; ++rr) P[r0 + rr] = kmax >= 0 ? finish64(acc[rr], m) : 0u;
  }
}

// f_j(+-x) = E_j +- x O_j from the partner lane's part: lane par = 0 holds
// E_j and keeps +x, lane par = 1 holds x O_j and takes -x.
template <int C>
__device__ __forceinline__ void combine_pm(uint32_t (&P)[C], int par, const ModP &m) {
#pragma unroll
  for (int r = 0; r < C; ++r) {
    const uint32_t other = __shfl_xor_sync(0xffffffffu, P[r], 1);
    const uint32_t e = par ? other : P[r], o = par ? P[r] : other;
    P[r] = par ? msub(e, o, m.p) : madd(e, o, m.p);
  }
}

// a[k][r] for k <= dx (the largest x-degree), r < C; qn[t] = q^{-C(t,2)}.
template <int C>
__device__ __forceinline__ void stage_chirp(int32_t *sa, const int2 *smeta, int deg, int dx,
                                            const uint32_t *limbs, int stride, int L,
                                            const uint32_t *V, const uint32_t *qn, const ModP &m) {
  const int n = (dx + 1) * C;
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
    const int k = idx / C, r = idx - k * C, j = deg - r;
    int32_t v = 0;
    if (j >= 0 && k <= smeta[j].y)
      v = signed_rep(mmul(reduce_coef(limbs + ((size_t)k * stride + j) * L, L, V, m), qn[k], m), m.p);
    sa[idx] = v;
  }
}

template <int C>
__global__ void __launch_bounds__(128, RS_G1_MINB) g1_kernel(G1Args a) {
  extern __shared__ __align__(16) uint32_t sm[];
  __shared__ int s_tile;
  bool first = true;
  for (;;) {
    int t;
    if (a.persistent) {
      if (threadIdx.x == 0) s_tile = atomicAdd(a.counter, 1);
      __syncthreads();
      t = s_tile;
    } else {
      t = first ? (int)blockIdx.x : a.ntiles;
    }
    first = false;
    if (t >= a.ntiles) return;

    const Tile tl = a.tiles[t];
    const PairDesc pd = a.pairs[tl.pair];
    const ModP m = a.mods[tl.prime];
    const uint32_t *V = a.vtab + (size_t)tl.prime * RS_VT_STRIDE;
    const int nmeta = pd.my + pd.ny + 2;
    const int dxm = max(pd.mxf, pd.mxg);
    int2 *smeta = reinterpret_cast<int2 *>(sm);
    int32_t *saf = reinterpret_cast<int32_t *>(sm) + ((2 * nmeta + 7) & ~7);  // 32-byte aligned
    int32_t *sag = saf + (pd.mxf + 1) * C;
    int32_t *swin = sag + (pd.mxg + 1) * C;
    const size_t tb = (size_t)tl.prime * a.tstride;

    for (int i = threadIdx.x; i < nmeta; i += blockDim.x) smeta[i] = a.meta[pd.meta_off + i];
    __syncthreads();
    stage_chirp<C>(saf, smeta, pd.my, pd.mxf, a.limbs + pd.f_off, pd.fstride, pd.Lf, V, a.qn + tb, m);
    stage_chirp<C>(sag, smeta + pd.my + 1, pd.ny, pd.mxg, a.limbs + pd.g_off, pd.gstride, pd.Lg, V,
                   a.qn + tb, m);
    __syncthreads();

    if (tl.x0 == 0 && threadIdx.x == 0) {  // unlucky prime: a leading coefficient vanishes mod p
      bool zf = true, zg = true;
      for (int k = 0; k <= pd.mxf; ++k) zf = zf && saf[k * C] == 0;
      for (int k = 0; k <= pd.mxg; ++k) zg = zg && sag[k * C] == 0;
      if (zf || zg) atomicAdd(a.stats + ST_UNLUCKY_PRIMES, 1ull);
    }

    // The work item's point pairs [x0, x0 + n) in chunks of blockDim / 2: the
    // staged coefficients serve every chunk, only the window is reloaded.
    const int ti = (int)threadIdx.x >> 1, par = (int)threadIdx.x & 1;
    const int half = (int)(blockDim.x >> 1);
    for (int cx = tl.x0; cx < tl.x0 + tl.n; cx += half) {
      const int nn = min(half, tl.x0 + tl.n - cx);
      for (int t = threadIdx.x; t < half + dxm + 1; t += blockDim.x) swin[t] = a.qc[tb + cx + t];
      __syncthreads();
      uint32_t unlucky = 0u, degen = 0u;
      const int i = cx + ti;  // point pair: this thread's image is at (-1)^par q^i
      // every thread evaluates (the shuffles need the whole warp); only the
      // threads of the chunk's pairs run the remainder sequence
      uint32_t A[C], B[C];
      eval_chirp<C>(A, saf, smeta, pd.my, swin + ti, par, m);
      eval_chirp<C>(B, sag, smeta + pd.my + 1, pd.ny, swin + ti, par, m);
      combine_pm<C>(A, par, m);
      combine_pm<C>(B, par, m);
      if (ti < nn) {
        unlucky = (A[0] == 0u || B[0] == 0u) ? 1u : 0u;
        Prs s;
        s.a = pd.my;
        s.b = pd.ny;
        s.num = s.den = s.Q = m.r1;
        s.eprev = max(min(pd.my, pd.ny) - 1, 0);
        s.sign = 0u;
        s.degen = 0u;
        prs_run<C>(A, B, s, m);
        // the chirp factor left out of the coefficients (reloaded: no register held through the sequence)
        s.num = mmul(s.num, mpow(a.qn[tb + i], (uint32_t)(pd.my + pd.ny), m), m);
        while (s.eprev > 0) {
          s.den = mmul(s.den, s.Q, m);
          --s.eprev;
        }
        const size_t idx = (size_t)pd.img_off + (size_t)tl.prime * pd.NI + 2 * i + par;
        a.num[idx] = s.sign ? mneg(s.num, m.p) : s.num;
        a.den[idx] = s.den;
        degen = s.degen;
      }
      const unsigned bu = __ballot_sync(0xffffffffu, unlucky);
      const unsigned bd = __ballot_sync(0xffffffffu, degen);
      if ((threadIdx.x & 31) == 0) {
        if (bu) atomicAdd(a.stats + ST_UNLUCKY_POINTS, (unsigned long long)__popc(bu));
        if (bd) atomicAdd(a.stats + ST_DEGENERATE, (unsigned long long)__popc(bd));
      }
      __syncthreads();  // the next chunk reloads the window (the next item restages everything)
    }
  }
}

}  // namespace

#ifndef RS_G1_CAP
#error "compile this file once per register capacity with -DRS_G1_CAP=<8..72>"
#endif
#define RS_CAT2(a, b) a##b
#define RS_CAT(a, b) RS_CAT2(a, b)

cudaError_t RS_CAT(rs_g1_launch_, RS_G1_CAP)(int threads, int blocks, size_t smem, const G1Args &a,
                                            cudaStream_t s) {
  g1_kernel<RS_G1_CAP><<<blocks, threads, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t RS_CAT(rs_g1_prepare_, RS_G1_CAP)(int threads, size_t smem, int *mb) {
  const size_t smem_used = smem;
  // The attribute is per kernel, not per launch: always allow the largest
  // staging any plan may request so that batches prepared earlier with more
  // shared memory keep working.
  (void)smem;
  cudaError_t e = cudaFuncSetAttribute(g1_kernel<RS_G1_CAP>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       RS_G1_MAX_SMEM_BYTES);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(mb, g1_kernel<RS_G1_CAP>, threads, smem_used);
}
