// Block-wide modular helpers shared by the interpolation kernels (G2):
// prefix/suffix products across a thread block and Montgomery's
// simultaneous inversion (P. L. Montgomery, "Speeding the Pollard and
// elliptic curve methods of factorization", Math. Comp. 48, 1987).
#pragma once
#include "modarith.cuh"

namespace {

// Block-wide exclusive prefix / suffix products of one value per thread
// (warp shuffles, then one warp over the warp totals).  scratch >= 97 words.
__device__ __forceinline__ void block_scan_mul(uint32_t v, uint32_t &pre, uint32_t &suf,
                                               uint32_t &total, const ModP &m, uint32_t *scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  uint32_t ip = v, is = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t up = __shfl_up_sync(0xffffffffu, ip, off);
    const uint32_t dn = __shfl_down_sync(0xffffffffu, is, off);
    if (lane >= off) ip = mmul(ip, up, m);
    if (lane + off < 32) is = mmul(is, dn, m);
  }
  uint32_t ep = __shfl_up_sync(0xffffffffu, ip, 1);
  uint32_t es = __shfl_down_sync(0xffffffffu, is, 1);
  if (lane == 0) ep = m.r1;
  if (lane == 31) es = m.r1;
  if (lane == 31) scratch[warp] = ip;
  __syncthreads();
  if (warp == 0) {
    uint32_t t = lane < nw ? scratch[lane] : m.r1;
    uint32_t wp = t, ws = t;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t up = __shfl_up_sync(0xffffffffu, wp, off);
      const uint32_t dn = __shfl_down_sync(0xffffffffu, ws, off);
      if (lane >= off) wp = mmul(wp, up, m);
      if (lane + off < 32) ws = mmul(ws, dn, m);
    }
    uint32_t xp = __shfl_up_sync(0xffffffffu, wp, 1);
    uint32_t xs = __shfl_down_sync(0xffffffffu, ws, 1);
    if (lane == 0) xp = m.r1;
    if (lane == 31) xs = m.r1;
    scratch[32 + lane] = xp;
    scratch[64 + lane] = xs;
    if (lane == 31) scratch[96] = wp;
  }
  __syncthreads();
  pre = mmul(scratch[32 + warp], ep, m);
  suf = mmul(scratch[64 + warp], es, m);
  total = scratch[96];
  __syncthreads();  // scratch may be reused right after
}

// out[i] = d[i]^{-1} for i < n (Montgomery's simultaneous inversion: one
// Fermat inverse of the product, prefix and suffix products for the rest).
__device__ void batch_invert(const uint32_t *d, uint32_t *out, int n, const ModP &m,
                             uint32_t *scratch) {
  const int T = blockDim.x;
  const int E = (n + T - 1) / T;
  const int beg = min((int)threadIdx.x * E, n), end = min(beg + E, n);
  uint32_t v = m.r1;
  for (int i = beg; i < end; ++i) v = mmul(v, d[i], m);
  uint32_t pre, suf, total;
  block_scan_mul(v, pre, suf, total, m, scratch);
  const uint32_t itot = minv(total, m);
  uint32_t r = pre;
  for (int i = beg; i < end; ++i) {
    out[i] = r;
    r = mmul(r, d[i], m);
  }
  uint32_t s = suf;
  for (int i = end - 1; i >= beg; --i) {
    out[i] = mmul(mmul(out[i], s, m), itot, m);
    s = mmul(s, d[i], m);
  }
}

}  // namespace
