// G3: Chinese remaindering (paper, Section 4.1: the residues R mod p are
// combined into the integer result by the Chinese remainder theorem).
//
// Garner's mixed-radix form R_j = v_0 + p_0 (v_1 + p_1 (v_2 + ...)) with
// digits v_k in the symmetric range (-p_k/2, p_k/2) gives the symmetric
// representative of R_j mod p_0 ... p_{K-1} directly.  Digit k is
//   v_k = (r_k - sum_{l<k} v_l W[k][l]) c_k  (mod p_k),
//   W[k][l] = p_0 ... p_{l-1} mod p_k,  c_k = (p_0 ... p_{k-1})^{-1} mod p_k,
// and the integer is R_j = sum_k v_k P_k with P_k = p_0 ... p_{k-1}.
//
// G3t: the digits, in tiles of 32 coefficients by blocks of 64 digits (a
//      rectangular update from the earlier digits, then a small triangular
//      solve), every dot product lazily accumulated in int64.
// G3b: one thread per (coefficient, chunk of 16 limbs of R_j) accumulates
//      sum_k w_k P_k[h] with the offset digits w_k = v_k + (p_k - 1)/2 >= 0
//      in 96-bit carry chains and normalises the chunk, keeping its carry.
// G3c: one block per 128 coefficients ripples the chunk carries, subtracts
//      floor(P/2) = sum_k (p_k - 1)/2 P_k and writes the two's-complement
//      32-bit limbs through shared memory in coalesced runs.
#include <algorithm>

#include "../../include/rs.h"
#include "rs_internal.cuh"

namespace {

__device__ __forceinline__ int32_t signed_rep3(uint32_t v, uint32_t p) {
  return v > (p >> 1) ? (int32_t)v - (int32_t)p : (int32_t)v;
}

__device__ __forceinline__ uint32_t finish64_3(int64_t s, const ModP &m) {
  return redc((uint64_t)(s + ((int64_t)m.p << 22)), m.p, m.pinv);  // 0 <= . < 2^54 < p 2^32
}

#define G3T_BK 64  // digits per digit block
#ifndef RS_G3T_LS16
#define RS_G3T_LS16 1  // thread groups per 16-coefficient tile (1 or 2)
#endif
#define G3T_LC 32  // earlier digits per staged chunk

// Digits by tiles: a block of 256 threads owns JT (32, or 16 when there are
// few coefficients to spread over the SMs) consecutive coefficients of one
// pair and produces their digits 64 at a time.  For the digit block
// [k0, k0 + 64) the contribution of every earlier digit,
//   A[k][j] = sum_{l < k0} W[k][l] v_l(j),
// is the product of a 64 x k0 slice of W and a k0 x 32 slice of digits:
// chunks of both are staged in shared memory and each thread accumulates a
// 4 x JT/16 block lazily in int64 (a fold with its row's 2^32 mod p_k every 7
// products).  The 64 digits of the block then follow one by one (JT lanes of
// one warp, lane = coefficient) from the triangle of W inside the block, with the
// residues, constants and that triangle prefetched into shared memory.
// The work per coefficient is still K^2 / 2 products, but W and the digits
// come from shared memory, each value reused 32 and 64 times.
template <int JT, int LS>
__global__ void __launch_bounds__(256 * LS, 4 / LS) g3t_kernel(G3Args a) {
  constexpr int CJ = JT / 16;  // columns per thread
  // LS thread groups of 256 share the earlier-digit chunks of a digit block
  // (group q takes chunks q, q + LS, ...) and their partial sums are added
  // through shared memory; with few tiles per SM this multiplies the warps
  // without changing each thread's 4 x CJ register block.
  // W[k0 + r][l0 + c] at Ws[q][c][r]: rows of 68 words keep each thread's four
  // consecutive r 16-byte aligned, so they come in one shared load
  __shared__ __align__(16) int32_t Ws[LS][G3T_LC][G3T_BK + 4];
  __shared__ int32_t Vs[LS][G3T_LC][JT];                        // digit l0 + c of coefficient j0 + jj
  __shared__ int32_t Wt[G3T_BK][G3T_BK + 1];                    // W[k0 + r][k0 + c], c < r
  __shared__ uint32_t Ds[G3T_BK][JT];                           // r_k(j) - A[k][j] mod p_k
  __shared__ int32_t Vb[G3T_BK][JT];                            // the block's digits
  __shared__ ModP Ms[G3T_BK];
  __shared__ uint32_t Cs[G3T_BK];
  static_assert(LS == 1 || (size_t)(LS - 1) * 256 * 4 * CJ * 8 <= sizeof(Ws), "partial sums fit in Ws");
  const int2 task = a.tasks[blockIdx.x];
  const PairDesc pd = a.pairs[task.x];
  const int K = pd.K, N = pd.N, S = pd.NI, j0 = task.y, tid = threadIdx.x;
  const int grp = tid >> 8, ltid = tid & 255;
  const int rg = ltid >> 4, cg = ltid & 15;  // rows 4 rg .. 4 rg + 3, columns CJ cg .. CJ cg + CJ - 1
  uint32_t *col = a.coef + pd.img_off;       // residue, then digit, of (k, j) at col[k S + j]
  for (int k0 = 0; k0 < K; k0 += G3T_BK) {
    const int bk = min(G3T_BK, K - k0);
    for (int r = tid; r < bk; r += blockDim.x) {
      Ms[r] = a.mods[k0 + r];
      Cs[r] = a.crt[k0 + r];
    }
    __syncthreads();
    uint32_t c32[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) c32[i] = 4 * rg + i < bk ? Ms[4 * rg + i].r1 : 0u;
    int64_t acc[4][CJ];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int c = 0; c < CJ; ++c) acc[i][c] = 0;
    // Chunks of W (8 values per thread) and digits are loaded into registers
    // one chunk ahead, so their latency overlaps the products.
    constexpr int NW = G3T_LC * G3T_BK / 256, NV = G3T_LC * JT / 256;
    int32_t wreg[NW], vreg[NV];
    auto fetch = [&](int l0) {
#pragma unroll
      for (int q = 0; q < NW; ++q) {
        const int e = ltid + 256 * q, r = e >> 5, c = e & 31, k = k0 + r;
        wreg[q] = r < bk ? __ldg(a.wtab + (size_t)k * (k - 1) / 2 + l0 + c) : 0;
      }
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        const int e = ltid + 256 * q, c = e / JT, jj = e % JT, j = j0 + jj;
        vreg[q] = j < N ? (int32_t)col[(size_t)(l0 + c) * S + j] : 0;
      }
    };
    const int nch = k0 / G3T_LC;  // k0 is a multiple of G3T_LC: full chunks
    if (grp < nch) fetch(grp * G3T_LC);
    for (int it = 0; it * LS < nch; ++it) {
      const int ch = it * LS + grp, l0 = ch * G3T_LC;
      const bool act = ch < nch;
      if (act) {
#pragma unroll
        for (int q = 0; q < NW; ++q) {
          const int e = ltid + 256 * q;
          Ws[grp][e & 31][e >> 5] = wreg[q];
        }
#pragma unroll
        for (int q = 0; q < NV; ++q) {
          const int e = ltid + 256 * q;
          Vs[grp][e / JT][e % JT] = vreg[q];
        }
      }
      __syncthreads();
      if (ch + LS < nch) fetch(l0 + LS * G3T_LC);
      if (act) {
        // |acc| < 2^53 after a fold and each product is below 2^60 in size, so
        // 7 products may follow a fold: four groups of 7 steps and one of 4.
        auto steps = [&](int c0, int n) {
#pragma unroll
          for (int c = c0; c < c0 + 7; ++c) {
            if (c - c0 >= n) break;
            const int4 w4 = *reinterpret_cast<const int4 *>(&Ws[grp][c][4 * rg]);
            const int32_t w[4] = {w4.x, w4.y, w4.z, w4.w};
            int32_t v[CJ];
#pragma unroll
            for (int cc = 0; cc < CJ; ++cc) v[cc] = Vs[grp][c][CJ * cg + cc];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
              for (int cc = 0; cc < CJ; ++cc) acc[i][cc] = rs_mac_s32(acc[i][cc], w[i], v[cc]);
          }
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int cc = 0; cc < CJ; ++cc) acc[i][cc] = rs_fold64(acc[i][cc], c32[i]);
        };
#pragma unroll 1
        for (int c0 = 0; c0 < 28; c0 += 7) steps(c0, 7);
        steps(28, G3T_LC - 28);
      }
      __syncthreads();
    }
    if constexpr (LS > 1) {  // the other groups' partial sums, through the (now unused) staging buffer
      int64_t *part = reinterpret_cast<int64_t *>(&Ws[0][0][0]);
      if (grp > 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int c = 0; c < CJ; ++c)
            part[(((size_t)(grp - 1) * 256 + ltid) * 4 + i) * CJ + c] = rs_fold64(acc[i][c], c32[i]);
      }
      __syncthreads();
      if (grp == 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int c = 0; c < CJ; ++c) {
            int64_t sum = rs_fold64(acc[i][c], c32[i]);  // |.| < 2^53 each: LS of them stay below 2^63
            for (int q = 1; q < LS; ++q) sum += part[(((size_t)(q - 1) * 256 + ltid) * 4 + i) * CJ + c];
            acc[i][c] = sum;
          }
      }
    }
    // D = r - A mod p_k (plain: W is in Montgomery form, the finish removes R)
    if (grp == 0) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = 4 * rg + i;
        if (r >= bk) continue;
        const ModP m = Ms[r];
#pragma unroll
        for (int c = 0; c < CJ; ++c) {
          const int jj = CJ * cg + c, j = j0 + jj;
          const uint32_t tA = finish64_3(rs_fold64(acc[i][c], m.r1), m);
          const uint32_t res = j < N ? col[(size_t)(k0 + r) * S + j] : 0u;
          Ds[r][jj] = msub(res, tA, m.p);
        }
      }
    }
    for (int e = tid; e < G3T_BK * G3T_BK; e += blockDim.x) {
      const int r = e >> 6, c = e & 63, k = k0 + r;
      Wt[r][c] = (c < r && r < bk) ? __ldg(a.wtab + (size_t)k * (k - 1) / 2 + k0 + c) : 0;
    }
    __syncthreads();
    if (tid < JT) {  // the block's digits in order, lane = coefficient
      const int jj = tid, j = j0 + jj;
      for (int r = 0; r < bk; ++r) {
        const ModP m = Ms[r];
        int64_t s0 = 0, s1 = 0;
        int n = 0;
        for (int c = 0; c + 1 < r; c += 2) {
          s0 = rs_mac_s32(s0, Wt[r][c], Vb[c][jj]);
          s1 = rs_mac_s32(s1, Wt[r][c + 1], Vb[c + 1][jj]);
          if (++n == 7) {
            s0 = rs_fold64(s0, m.r1);
            s1 = rs_fold64(s1, m.r1);
            n = 0;
          }
        }
        if (r & 1) s0 = rs_mac_s32(s0, Wt[r][r - 1], Vb[r - 1][jj]);
        const int64_t s = rs_fold64(rs_fold64(s0, m.r1) + rs_fold64(s1, m.r1), m.r1);
        const uint32_t v = mmul(msub(Ds[r][jj], finish64_3(s, m), m.p), Cs[r], m);
        const int32_t vs = signed_rep3(v, m.p);
        Vb[r][jj] = vs;
        if (j < N) col[(size_t)(k0 + r) * S + j] = (uint32_t)vs;
      }
    }
    __syncthreads();  // this block's digits are read by the next digit blocks
  }
}

#define G3P_G 4     // digit rows per group
#define G3P_LC 128  // earlier digits per staged chunk of W

// Digits, one thread per coefficient: a block of 128 threads owns 128
// consecutive coefficients of one pair (the same tasks as the output
// kernel) and walks the digits in groups of 4 rows.  For the group
// [k0, k0 + 4) each thread accumulates A[k0 + i] = sum_{l < k0} W[k0 + i][l] v_l
// over its own earlier digits (re-read from the residue array they
// overwrote, where they stay in L1) with the four W values of each l
// broadcast from shared memory (one 16-byte load per l), lazily in int64 (a
// fold every 7 products); then it finishes the group's four digits in turn
// from the 4 x 4 triangle of W.  No warp waits for another: this is the form
// for batches with many coefficients, where one thread per coefficient
// fills the GPU (the tiled kernel serves batches with few coefficients and
// many primes).
__global__ void __launch_bounds__(128) g3p_kernel(G3Args a) {
  __shared__ __align__(16) int32_t Ws[G3P_LC][G3P_G];  // W[k0 + i][l0 + c] at Ws[c][i]
  __shared__ int32_t Wt[G3P_G][G3P_G];                 // W[k0 + i][k0 + c], c < i
  __shared__ ModP Ms[G3P_G];
  __shared__ uint32_t Cs[G3P_G];
  const int2 task = a.tasks[blockIdx.x];
  const PairDesc pd = a.pairs[task.x];
  const int K = pd.K, N = pd.N, S = pd.NI, t = (int)threadIdx.x, j = task.y + t;
  const bool live = j < N;
  uint32_t *col = a.coef + pd.img_off + (live ? j : 0);  // residue, then digit, of row k at col[k S]
  for (int k0 = 0; k0 < K; k0 += G3P_G) {
    const int g = min(G3P_G, K - k0);
    __syncthreads();  // the previous group's constants and triangle are no longer read
    if (t < G3P_G) {
      Ms[t] = a.mods[k0 + min(t, g - 1)];
      Cs[t] = a.crt[k0 + min(t, g - 1)];
    }
    if (t < G3P_G * G3P_G) {
      const int i = t >> 2, c = t & 3, k = k0 + i;
      Wt[i][c] = (c < i && i < g) ? __ldg(a.wtab + (size_t)k * (k - 1) / 2 + k0 + c) : 0;
    }
    int64_t acc[G3P_G] = {0, 0, 0, 0};
    uint32_t c32[G3P_G];
    for (int l0 = 0; l0 < k0; l0 += G3P_LC) {
      const int lc = min(G3P_LC, k0 - l0);
      if (l0 > 0) __syncthreads();  // the previous chunk is no longer read
#pragma unroll
      for (int i = 0; i < G3P_G; ++i) {  // row k0 + i, entries l0 + t
        const int k = k0 + i;
        Ws[t][i] = (t < lc && i < g) ? __ldg(a.wtab + (size_t)k * (k - 1) / 2 + l0 + t) : 0;
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < G3P_G; ++i) c32[i] = Ms[i].r1;
      int c = 0;
      while (c < lc) {
        const int cend = min(c + 7, lc);  // 7 products per fold
#pragma unroll 7
        for (; c < cend; ++c) {
          const int32_t v = live ? (int32_t)col[(size_t)(l0 + c) * S] : 0;
          const int4 w = *reinterpret_cast<const int4 *>(&Ws[c][0]);
          acc[0] = rs_mac_s32(acc[0], w.x, v);
          acc[1] = rs_mac_s32(acc[1], w.y, v);
          acc[2] = rs_mac_s32(acc[2], w.z, v);
          acc[3] = rs_mac_s32(acc[3], w.w, v);
        }
#pragma unroll
        for (int i = 0; i < G3P_G; ++i) acc[i] = rs_fold64(acc[i], c32[i]);
      }
    }
    __syncthreads();  // Ms, Cs, Wt of this group are in place
    int32_t vg[G3P_G];
#pragma unroll
    for (int i = 0; i < G3P_G; ++i) {
      if (i >= g) break;
      const ModP m = Ms[i];
      int64_t s2 = rs_fold64(acc[i], m.r1);  // |s2| < 2^53
#pragma unroll
      for (int c = 0; c < i; ++c) s2 = rs_mac_s32(s2, Wt[i][c], vg[c]);  // + at most 3 products < 2^60
      s2 = rs_fold64(s2, m.r1);                                          // |s2| < 2^53 again
      const uint32_t r = live ? col[(size_t)(k0 + i) * S] : 0u;
      const uint32_t v = mmul(msub(r, finish64_3(s2, m), m.p), Cs[i], m);
      vg[i] = signed_rep3(v, m.p);
      if (live) col[(size_t)(k0 + i) * S] = (uint32_t)vg[i];
    }
  }
}

#ifndef RS_G3B_UNROLL
#define RS_G3B_UNROLL 4
#endif
constexpr int kG3bUnroll = RS_G3B_UNROLL;  // prime rows of the limb kernel per loop iteration

// a2:a1:a0 += x * y (96-bit accumulator, one carry chain).
__device__ __forceinline__ void mac96(uint32_t &a0, uint32_t &a1, uint32_t &a2, uint32_t x, uint32_t y) {
  asm("mad.lo.cc.u32 %0, %3, %4, %0;\n\t"
      "madc.hi.cc.u32 %1, %3, %4, %1;\n\t"
      "addc.u32 %2, %2, 0;"
      : "+r"(a0), "+r"(a1), "+r"(a2)
      : "r"(x), "r"(y));
}

// Limb chunks: blockDim = 128 coefficients of one pair, one chunk of 16
// output limbs.  With the offset digits w_k = v_k + (p_k - 1)/2 in [0, p_k)
// the limb sums S[h] = sum_k w_k P_k[16 c + h] (P_k's 32-bit limbs) are
// unsigned and below K 2^63, so each is kept in a 96-bit carry chain; the
// chunk is then normalised into 16 limbs and a carry (< 2^47).  Only primes
// whose prefix product reaches this chunk contribute to it directly; lower
// terms arrive through the previous chunk's carry.
__global__ void __launch_bounds__(128) g3b_kernel(G3Args a) {
  const int4 task = a.ctasks[blockIdx.x];
  const PairDesc pd = a.pairs[task.x];
  const int c = task.z;
  const int j = task.y + (int)threadIdx.x;
  if (j >= pd.N) return;
  const int K = pd.K, N = pd.N;
  // first k whose prefix product has a limb in this chunk (nh is increasing)
  int lo = 0, hi = K;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a.nh[mid] > 32 * c)
      hi = mid;
    else
      lo = mid + 1;
  }
  uint32_t a0[16], a1[16], a2[16];
#pragma unroll
  for (int h = 0; h < 16; ++h) a0[h] = a1[h] = a2[h] = 0u;
  const uint32_t *col = a.coef + pd.img_off + j;
#pragma unroll kG3bUnroll
  for (int k = lo; k < K; ++k) {
    const uint32_t half = (__ldg(&a.mods[k].p) - 1u) >> 1;
    const uint32_t w = (uint32_t)((int32_t)col[(size_t)k * pd.NI] + (int32_t)half);
    const uint4 *row = reinterpret_cast<const uint4 *>(a.p16 + __ldg(a.poff + k) + 32 * c);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint4 l4 = __ldg(row + q);
      mac96(a0[4 * q], a1[4 * q], a2[4 * q], w, l4.x);
      mac96(a0[4 * q + 1], a1[4 * q + 1], a2[4 * q + 1], w, l4.y);
      mac96(a0[4 * q + 2], a1[4 * q + 2], a2[4 * q + 2], w, l4.z);
      mac96(a0[4 * q + 3], a1[4 * q + 3], a2[4 * q + 3], w, l4.w);
    }
  }
  uint64_t carry = 0;
  uint32_t *xl = a.xl + pd.xl_off + j;
#pragma unroll
  for (int h = 0; h < 16; ++h) {
    const uint64_t lo64 = ((uint64_t)a1[h] << 32) | a0[h];
    const uint64_t t = lo64 + carry;
    const uint64_t ovf = t < lo64 ? 1u : 0u;
    xl[(size_t)(16 * c + h) * N] = (uint32_t)t;
    carry = (t >> 32) + (((uint64_t)a2[h] + ovf) << 32);
  }
  a.carry[pd.cy_off + (size_t)c * N + j] = (int64_t)carry;
}

// Carries and output: one thread per coefficient adds the chunk carries to
// the chunk limbs and subtracts floor(P / 2), P = p_0 ... p_{K-1} (the offset
// digits added sum_k (p_k - 1)/2 P_k = (P - 1)/2; limbs summed from the
// signed digits already have the symmetric value), giving the symmetric
// representative in two's complement; only the Lout low limbs are formed,
// which is exact because the result fits in them.  Each chunk's 16 limbs of
// the block's 128 coefficients are staged in shared memory and written back
// as runs of 16 consecutive limbs of one coefficient (out is
// [coefficient][limb], so a warp's store covers two 64-byte runs instead of
// 32 words Lout apart).  Also records the shape of each pair's result:
// shape[2 pair] = 1 + the largest index of a non-zero coefficient (0 for
// R = 0) and shape[2 pair + 1] = the most two's-complement limbs any
// coefficient needs (both by atomicMax on zeroed words).
__global__ void __launch_bounds__(128) g3c_kernel(G3Args a) {
  __shared__ uint32_t T[128 * 17];  // T[t * 17 + w]: limb 16 c + w of coefficient j0 + t
  const int2 task = a.tasks[blockIdx.x];
  const PairDesc pd = a.pairs[task.x];
  const int t = (int)threadIdx.x, j0 = task.y, j = j0 + t;
  const bool live = j < pd.N;
  const int N = pd.N, L = pd.Lout, C = (L + 15) / 16;
  const uint32_t *xl = a.xl + pd.xl_off + j;
  const int p0 = __ldg(a.poff + pd.K);
  const uint32_t *PK = reinterpret_cast<const uint32_t *>(a.p16 + p0);  // P's 32-bit limbs
  // limbs from the signed digits (tensor-core limb kernel) need no offset: P = 0 here
  const int plen = a.signed_digits ? 0 : (__ldg(a.poff + pd.K + 1) - p0) / 2;
  uint32_t *o = a.out + pd.out_off;
  int64_t r = 0;
  int last_nz = -1, last_nf = -1;  // last limb != 0, last limb != 0xffffffff
  uint32_t top_nz = 0u, top_nf = 0u, top = 0u;
  // A chunk's loads (its limbs, P's limbs, its carry) are independent of the
  // carry chain: chunk c + 1's are issued before chunk c's chain and stores,
  // so a chunk does not wait a memory latency after the previous one.
  auto load = [&](int c, uint32_t (&x)[16], uint32_t (&pkv)[17], int64_t &cyv) {
#pragma unroll
    for (int w = 0; w < 16; ++w) x[w] = xl[(size_t)(16 * c + w) * N];
#pragma unroll
    for (int w = 0; w < 17; ++w) pkv[w] = 16 * c + w < plen ? __ldg(PK + 16 * c + w) : 0u;
    cyv = a.carry[pd.cy_off + (size_t)c * N + j];
  };
  uint32_t xw[16], pk[17];
  int64_t cy = 0;
  if (live && C > 0) load(0, xw, pk, cy);
  for (int c = 0; c < C; ++c) {
    uint32_t xn[16], pn[17];
    int64_t cn = 0;
#pragma unroll
    for (int w = 0; w < 16; ++w) xn[w] = 0u;
#pragma unroll
    for (int w = 0; w < 17; ++w) pn[w] = 0u;
    if (live && c + 1 < C) load(c + 1, xn, pn, cn);
    if (live) {
#pragma unroll
      for (int w = 0; w < 16; ++w) {
        const int l = 16 * c + w;
        const uint32_t h = (pk[w] >> 1) | (pk[w + 1] << 31);
        const int64_t v = (int64_t)xw[w] + r - (int64_t)h;
        const uint32_t limb = (uint32_t)v;
        r = v >> 32;
        T[t * 17 + w] = limb;
        if (l < L) {
          if (limb != 0u) {
            last_nz = l;
            top_nz = limb;
          }
          if (limb != 0xffffffffu) {
            last_nf = l;
            top_nf = limb;
          }
          top = limb;
        }
      }
      r += cy;
    }
    __syncthreads();
    const int nl = min(16, L - 16 * c);  // limbs of this chunk that exist
#pragma unroll 4
    for (int q = 0; q < 16; ++q) {
      const int e = q * 128 + t, jj = e >> 4, w = e & 15;
      if (j0 + jj < N && w < nl) o[(size_t)(j0 + jj) * L + 16 * c + w] = T[jj * 17 + w];
    }
    __syncthreads();
#pragma unroll
    for (int w = 0; w < 16; ++w) xw[w] = xn[w];
#pragma unroll
    for (int w = 0; w < 17; ++w) pk[w] = pn[w];
    cy = cn;
  }
  if (!live) return;
  // fewest limbs whose two's-complement value is this coefficient
  const bool neg = (top >> 31) != 0u;
  if (!neg && last_nz < 0) return;  // a zero coefficient
  int need = neg ? last_nf + 1 + ((top_nf >> 31) ? 0 : 1) : last_nz + 1 + ((top_nz >> 31) ? 1 : 0);
  need = max(1, min(need, L));
  atomicMax(a.shape + 2 * task.x, j + 1);
  atomicMax(a.shape + 2 * task.x + 1, need);
}

// W[k][l] = p_0 ... p_{l-1} mod p_k (Montgomery form, signed), one thread per k.
__global__ void crt_w_kernel(const ModP *mods, int K, int32_t *wtab) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  const ModP m = mods[k];
  int32_t *w = wtab + (size_t)k * (k - 1) / 2;
  uint32_t acc = m.r1;
  for (int l = 0; l < k; ++l) {
    w[l] = signed_rep3(acc, m.p);
    acc = mmul(acc, to_mont(mods[l].p - m.p, m), m);  // p_l mod p_k (the table is descending)
  }
}

// One warp per (factor, prime): g mod p by Horner over g's limbs
// (r <- r 2^32 + limb, with 2^32 = R mod p taken as mmul by R^2 mod p), its
// inverse by Fermat, then the factor's residues times that inverse (plain
// residues times a Montgomery-form value stay plain).  g = 0 mod p gives 0.
__global__ void scale_kernel(const ScaleDesc *sd, int nf, int kmax, const ModP *mods, const uint32_t *gw,
                             const uint32_t *in, uint32_t *out) {
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= (int64_t)nf * kmax) return;
  const int fi = (int)(warp / kmax), k = (int)(warp - (int64_t)fi * kmax);
  const ScaleDesc d = sd[fi];
  if (k >= d.k) return;
  const ModP m = mods[k];
  uint32_t r = 0u;
  for (int l = d.g_len - 1; l >= 0; --l) {
    uint32_t limb = gw[d.g_off + l];  // < 2^32 < 4p
    while (limb >= m.p) limb -= m.p;
    r = madd(mmul(r, m.r2, m), limb, m.p);
  }
  const uint32_t inv = minv(to_mont(r, m), m);
  const uint32_t *src = in + d.src_off + (int64_t)k * d.src_stride;
  uint32_t *dst = out + d.dst_off + (int64_t)k * d.n;
  for (int j = lane; j < d.n; j += 32) dst[j] = mmul(src[j], inv, m);
}

}  // namespace

cudaError_t launch_scale(const ScaleDesc *sd, int nf, int kmax, const ModP *mods, const uint32_t *gw,
                         const uint32_t *in, uint32_t *out, cudaStream_t s) {
  const int64_t warps = (int64_t)nf * kmax;
  if (warps > 0) scale_kernel<<<(unsigned)((warps + 3) / 4), 128, 0, s>>>(sd, nf, kmax, mods, gw, in, out);
  return cudaGetLastError();
}

cudaError_t launch_g3t(int nt, const G3Args &a, const int2 *ttasks, cudaStream_t s, int jt) {
  G3Args at = a;
  at.tasks = ttasks;
  if (nt) {
    if (jt == 16)
      g3t_kernel<16, RS_G3T_LS16><<<nt, 256 * RS_G3T_LS16, 0, s>>>(at);
    else
      g3t_kernel<32, 1><<<nt, 256, 0, s>>>(at);
  }
  return cudaGetLastError();
}

cudaError_t launch_g3p(int nt, const G3Args &a, const int2 *tasks, cudaStream_t s) {
  G3Args at = a;
  at.tasks = tasks;
  if (nt) g3p_kernel<<<nt, 128, 0, s>>>(at);
  return cudaGetLastError();
}

cudaError_t launch_g3bc(int nb, int nc, const G3Args &a, const int2 *otasks, cudaStream_t s) {
  if (nb) g3b_kernel<<<nb, 128, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  G3Args ao = a;
  ao.tasks = otasks;
  if (nc) g3c_kernel<<<nc, 128, 0, s>>>(ao);
  return cudaGetLastError();
}

cudaError_t launch_crt_tables(const ModP *mods, int K, int32_t *wtab, cudaStream_t s) {
  crt_w_kernel<<<(K + 63) / 64, 64, 0, s>>>(mods, K, wtab);
  return cudaGetLastError();
}
