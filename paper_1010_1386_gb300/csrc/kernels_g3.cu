// G3: Chinese remaindering (paper, Section 4.1: the residues R mod p are
// "lifted to an integer solution via Chinese remaindering").
//
// Garner's mixed-radix form R_j = v_0 + p_0 (v_1 + p_1 (v_2 + ...)) with
// digits v_k in the symmetric range (-p_k/2, p_k/2) gives the symmetric
// representative of R_j mod p_0 ... p_{K-1} directly.  Digit k is
//   v_k = (r_k - sum_{l<k} v_l W[k][l]) c_k  (mod p_k),
//   W[k][l] = p_0 ... p_{l-1} mod p_k,  c_k = (p_0 ... p_{k-1})^{-1} mod p_k,
// and the integer is R_j = sum_k v_k P_k with P_k = p_0 ... p_{k-1}.
//
// G3a: the digits, each dot product over the previous digits lazily
//      accumulated in int64: one thread per coefficient when a batch has many
//      coefficients and few primes, one warp per coefficient otherwise.
// G3b: one thread per (coefficient, chunk of 32 sixteen-bit digits of R_j)
//      accumulates sum_k v_k P_k[h] exactly in int64 (|v_k P_k[h]| < 2^46)
//      and normalises the chunk, keeping its carry.
// G3c: one thread per coefficient ripples the chunk carries and writes the
//      two's-complement 32-bit limbs.
#include "../../include/rs.h"
#include "rs_internal.cuh"

namespace {

__device__ __forceinline__ int32_t signed_rep3(uint32_t v, uint32_t p) {
  return v > (p >> 1) ? (int32_t)v - (int32_t)p : (int32_t)v;
}

__device__ __forceinline__ uint32_t finish64_3(int64_t s, const ModP &m) {
  return redc((uint64_t)(s + ((int64_t)m.p << 22)), m.p, m.pinv);  // 0 <= . < 2^54 < p 2^32
}

// Digits: one thread per coefficient, blockDim = T consecutive coefficients
// of one pair; each thread keeps its digits in shared memory (digit l of
// thread t at sdig[l T + t], conflict-free) and reads W[k][l] as a broadcast.
__global__ void g3a_kernel(G3Args a) {
  extern __shared__ int32_t sdig[];
  const int2 task = a.tasks[blockIdx.x];
  const PairDesc pd = a.pairs[task.x];
  const int T = blockDim.x, tid = threadIdx.x;
  const int j = task.y + tid;
  if (j >= pd.N) return;
  const int K = pd.K, N = pd.N;
  uint32_t *col = a.coef + pd.img_off + j;  // residue, then digit, k at col[k N]
  for (int k = 0; k < K; ++k) {
    const ModP mk = a.mods[k];
    const int32_t *wk = a.wtab + (size_t)k * (k - 1) / 2;
    int64_t acc = 0;
    int l = 0;
    while (l < k) {
      const int lend = min(l + 7, k);
      if (a.digits_in_smem)
        for (; l < lend; ++l) acc = rs_mac_s32(acc, sdig[l * T + tid], __ldg(wk + l));
      else
        for (; l < lend; ++l) acc = rs_mac_s32(acc, (int32_t)col[(size_t)l * N], __ldg(wk + l));
      acc = rs_fold64(acc, mk.r1);
    }
    const uint32_t t = finish64_3(acc, mk);  // sum_l v_l W[k][l] (plain: W is in Montgomery form)
    const uint32_t v = mmul(msub(col[(size_t)k * N], t, mk.p), a.crt[k], mk);  // plain, [0, p_k)
    const int32_t vs = signed_rep3(v, mk.p);
    if (a.digits_in_smem) sdig[k * T + tid] = vs;
    col[(size_t)k * N] = (uint32_t)vs;
  }
}

// Digits, one warp per coefficient (for many primes or few coefficients):
// blockDim = 64 (two coefficients), dynamic shared memory 2 * kmax words.
// Each dot product is split over the 32 lanes, lazily accumulated, folded,
// reduced and summed with shuffles.
__global__ void g3w_kernel(G3Args a) {
  extern __shared__ int32_t sdig_w[];
  const int2 task = a.tasks[blockIdx.x];
  const PairDesc pd = a.pairs[task.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = task.y + warp;
  if (j >= pd.N) return;  // the whole warp leaves together
  const int K = pd.K, N = pd.N;
  int32_t *sd = sdig_w + warp * a.kmax;
  uint32_t *col = a.coef + pd.img_off + j;
  for (int k = 0; k < K; ++k) {
    const ModP mk = a.mods[k];
    const int32_t *wk = a.wtab + (size_t)k * (k - 1) / 2;
    int64_t acc = 0;
    int cnt = 0;
    for (int l = lane; l < k; l += 32) {
      acc = rs_mac_s32(acc, sd[l], __ldg(wk + l));
      if (++cnt == 7) {
        acc = rs_fold64(acc, mk.r1);
        cnt = 0;
      }
    }
    acc = rs_fold64(acc, mk.r1);
    uint32_t t = finish64_3(acc, mk);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t = madd(t, __shfl_xor_sync(0xffffffffu, t, off), mk.p);
    const uint32_t v = mmul(msub(col[(size_t)k * N], t, mk.p), a.crt[k], mk);
    const int32_t vs = signed_rep3(v, mk.p);
    if (lane == 0) {
      sd[k] = vs;
      col[(size_t)k * N] = (uint32_t)vs;
    }
    __syncwarp();
  }
}

// Limb chunks: blockDim = 128 coefficients of one pair, one 32-digit chunk.
__global__ void g3b_kernel(G3Args a) {
  const int4 task = a.ctasks[blockIdx.x];
  const PairDesc pd = a.pairs[task.x];
  const int c = task.z;
  const int j = task.y + (int)threadIdx.x;
  if (j >= pd.N) return;
  const int K = pd.K, N = pd.N;
  // first k whose prefix product has a digit in this chunk (nh is increasing)
  int lo = 0, hi = K;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a.nh[mid] > 32 * c)
      hi = mid;
    else
      lo = mid + 1;
  }
  int64_t acc[32];
#pragma unroll
  for (int h = 0; h < 32; ++h) acc[h] = 0;
  const uint32_t *col = a.coef + pd.img_off + j;
  for (int k = lo; k < K; ++k) {
    const int32_t v = (int32_t)col[(size_t)k * N];
    const uint4 *row = reinterpret_cast<const uint4 *>(a.p16 + a.poff[k] + 32 * c);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint4 w = row[q];
      const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        acc[8 * q + 2 * e] = rs_mac_s32(acc[8 * q + 2 * e], v, (int32_t)(ws[e] & 0xffffu));
        acc[8 * q + 2 * e + 1] = rs_mac_s32(acc[8 * q + 2 * e + 1], v, (int32_t)(ws[e] >> 16));
      }
    }
  }
  int64_t carry = 0;
  uint32_t *xl = a.xl + pd.xl_off + j;
#pragma unroll
  for (int w = 0; w < 16; ++w) {
    const int64_t t0 = acc[2 * w] + carry;
    const uint32_t d0 = (uint32_t)t0 & 0xffffu;
    carry = (t0 - (int64_t)d0) >> 16;
    const int64_t t1 = acc[2 * w + 1] + carry;
    const uint32_t d1 = (uint32_t)t1 & 0xffffu;
    carry = (t1 - (int64_t)d1) >> 16;
    xl[(size_t)(16 * c + w) * N] = d0 | (d1 << 16);
  }
  a.carry[pd.cy_off + (size_t)c * N + j] = carry;
}

// Carries and output: one thread per coefficient.
__global__ void g3c_kernel(G3Args a) {
  const int2 task = a.tasks[blockIdx.x];
  const PairDesc pd = a.pairs[task.x];
  const int j = task.y + (int)threadIdx.x;
  if (j >= pd.N) return;
  const int N = pd.N, L = pd.Lout, C = (L + 15) / 16;
  const uint32_t *xl = a.xl + pd.xl_off + j;
  uint32_t *o = a.out + pd.out_off + (size_t)j * L;
  int64_t r = 0;
  for (int c = 0; c < C; ++c) {
    for (int w = 0; w < 16; ++w) {
      const uint32_t word = xl[(size_t)(16 * c + w) * N];
      const int64_t t0 = (int64_t)(word & 0xffffu) + r;
      const uint32_t e0 = (uint32_t)t0 & 0xffffu;
      r = (t0 - (int64_t)e0) >> 16;
      const int64_t t1 = (int64_t)(word >> 16) + r;
      const uint32_t e1 = (uint32_t)t1 & 0xffffu;
      r = (t1 - (int64_t)e1) >> 16;
      const int l = 16 * c + w;
      if (l < L) o[l] = e0 | (e1 << 16);
    }
    r += a.carry[pd.cy_off + (size_t)c * N + j];
  }
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

// Prefix products P_k = p_0 ... p_{k-1} as 16-bit digits, row k at poff[k]
// (zero padded to its reserved length), nh[k] = digits up to the top
// non-zero one.  A single thread: P_{k+1} = P_k p_k on 32-bit limbs.
__global__ void crt_p16_kernel(const ModP *mods, int K, const int32_t *poff, uint16_t *p16, int32_t *nh,
                               uint32_t *limbs) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  int n = 1;
  limbs[0] = 1u;
  for (int k = 0; k < K; ++k) {
    uint16_t *row = p16 + poff[k];
    const int reserved = poff[k + 1] - poff[k];
    int top = 0;
    for (int i = 0; i < reserved; ++i) {
      const int li = i >> 1;
      const uint32_t d = li < n ? ((i & 1) ? (limbs[li] >> 16) : (limbs[li] & 0xffffu)) : 0u;
      row[i] = (uint16_t)d;
      if (d) top = i + 1;
    }
    nh[k] = top;
    const uint64_t p = mods[k].p;
    uint64_t carry = 0;
    for (int i = 0; i < n; ++i) {
      const uint64_t t = (uint64_t)limbs[i] * p + carry;
      limbs[i] = (uint32_t)t;
      carry = t >> 32;
    }
    if (carry) limbs[n++] = (uint32_t)carry;
  }
}

}  // namespace

cudaError_t launch_g3a(int nd, int dthreads, int kd, const G3Args &a, const int2 *dtasks, cudaStream_t s) {
  G3Args ad = a;
  ad.tasks = dtasks;
  ad.kmax = kd;
  ad.digits_in_smem = (size_t)dthreads * kd * 4 <= 200 * 1024;
  if (nd) g3a_kernel<<<nd, dthreads, ad.digits_in_smem ? (size_t)dthreads * kd * 4 : 0, s>>>(ad);
  return cudaGetLastError();
}

cudaError_t launch_g3w(int nw, int kw, const G3Args &a, const int2 *wtasks, cudaStream_t s) {
  G3Args aw = a;
  aw.tasks = wtasks;
  aw.kmax = kw;
  if (nw) g3w_kernel<<<nw, 64, (size_t)2 * kw * 4, s>>>(aw);
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

int g3_digit_threads(int kmax) {
  int t = 128;
  while (t > 32 && (size_t)t * kmax * 4 > 96 * 1024) t >>= 1;
  return t;
}

cudaError_t g3_prepare(int kmax) {
  (void)kmax;  // beyond 200 KB of digits per block the kernel reads them from global memory
  cudaError_t e = cudaFuncSetAttribute(g3a_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(g3w_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

cudaError_t launch_crt_tables(const ModP *mods, int K, const int32_t *poff, int32_t *wtab, uint16_t *p16,
                              int32_t *nh, uint32_t *limbs, cudaStream_t s) {
  crt_w_kernel<<<(K + 63) / 64, 64, 0, s>>>(mods, K, wtab);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  crt_p16_kernel<<<1, 1, 0, s>>>(mods, K, poff, p16, nh, limbs);
  return cudaGetLastError();
}
