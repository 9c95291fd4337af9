// G2 (interpolation mod p), G3 (Garner CRT) and the per-prime constant
// tables.  Paper, Section 4.1: "the resultant polynomial R^{(y)}(x) is
// interpolated over the prime field Z_p and eventually lifted to an integer
// solution via Chinese remaindering"; interpolation is the Vandermonde solve
// on the points x_i, here the points 0, 1, ..., D, in Newton form.
#include "rs_internal.cuh"

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

// One block per (pair, prime): images z_i = num_i / den_i at x_i = i, then
// Newton divided differences c_k (x_i - x_{i-k} = k), then the Newton form
// c_0 + x (c_1 + (x - 1) (c_2 + ...)) expanded to monomials.
__global__ void g2_kernel(G2Args a) {
  extern __shared__ __align__(16) uint32_t sm[];
  __shared__ uint32_t scratch[128];
  const int2 task = a.tasks[blockIdx.x];
  const PairDesc pd = a.pairs[task.x];
  const ModP m = a.mods[task.y];
  const int N = pd.N, D = N - 1, T = blockDim.x, tid = threadIdx.x;
  uint32_t *B0 = sm, *B1 = sm + N, *B2 = sm + 2 * N;
  const size_t base = (size_t)pd.img_off + (size_t)task.y * N;

  for (int i = tid; i < N; i += T) {
    B0[i] = a.num[base + i];
    B1[i] = a.den[base + i];
  }
  __syncthreads();
  batch_invert(B1, B2, N, m, scratch);
  __syncthreads();
  for (int i = tid; i < N; i += T) {
    B0[i] = mmul(B0[i], B2[i], m);  // z_i
    B1[i] = i ? to_mont((uint32_t)i, m) : m.r1;
  }
  __syncthreads();
  batch_invert(B1, B2, N, m, scratch);  // B2[k] = 1/k
  __syncthreads();

  for (int lev = 1; lev <= D; ++lev) {
    const uint32_t *src = (lev & 1) ? B0 : B1;
    uint32_t *dst = (lev & 1) ? B1 : B0;
    const uint32_t ik = B2[lev];
    for (int i = lev + tid; i <= D; i += T) dst[i] = mmul(msub(src[i], src[i - 1], m.p), ik, m);
    __syncthreads();
  }
  for (int i = tid; i < N; i += T) B2[i] = (i & 1) ? B1[i] : B0[i];  // c_i
  __syncthreads();

  uint32_t *cur = B0, *nxt = B1;
  if (tid == 0) cur[0] = B2[D];
  __syncthreads();
  for (int k = D - 1; k >= 0; --k) {
    const uint32_t nk = mneg(to_mont((uint32_t)k, m), m.p);
    const int len = D - k + 1;  // coefficients of the new polynomial
    for (int j = tid; j < len; j += T) {
      const uint32_t lo = j > 0 ? cur[j - 1] : 0u;
      const uint32_t hi = j < len - 1 ? cur[j] : 0u;
      uint32_t v = mmul2(lo, m.r1, hi, nk, m);  // lo - k hi
      if (j == 0) v = madd(v, B2[k], m.p);
      nxt[j] = v;
    }
    __syncthreads();
    uint32_t *t = cur;
    cur = nxt;
    nxt = t;
  }
  for (int j = tid; j < N; j += T) a.coef[base + j] = from_mont(cur[j], m);
}

// One thread per output coefficient: Garner's mixed-radix digits in the
// symmetric range, R_j = v_0 + p_0 (v_1 + p_1 (v_2 + ...)), then the limbs.
__global__ void g3_kernel(G3Args a) {
  const int2 task = a.tasks[blockIdx.x];
  const PairDesc pd = a.pairs[task.x];
  const int j = task.y + (int)threadIdx.x;
  if (j >= pd.N) return;
  const int K = pd.K, N = pd.N, L = pd.Lout;
  uint32_t *col = a.coef + pd.img_off + j;  // residue / digit k at col[k N]

  for (int k = 0; k < K; ++k) {
    const ModP mk = a.mods[k];
    uint32_t t = 0u;
    if (k > 0) {
      const int32_t vp = (int32_t)col[(size_t)(k - 1) * N];
      t = vp < 0 ? (uint32_t)(vp + (int32_t)mk.p) : (uint32_t)vp;
      for (int l = k - 2; l >= 0; --l) {
        const uint32_t ym = to_mont(a.mods[l].p - mk.p, mk);  // p_l mod p_k (table is descending)
        const int32_t vl = (int32_t)col[(size_t)l * N];
        const uint32_t vr = vl < 0 ? (uint32_t)(vl + (int32_t)mk.p) : (uint32_t)vl;
        t = madd(mmul(t, ym, mk), vr, mk.p);  // plain t times Montgomery y -> plain
      }
    }
    const uint32_t rk = col[(size_t)k * N];
    const uint32_t v = mmul(msub(rk, t, mk.p), a.crt[k], mk);  // plain digit in [0, p_k)
    const int32_t vs = v > (mk.p - 1u) / 2u ? (int32_t)v - (int32_t)mk.p : (int32_t)v;
    col[(size_t)k * N] = (uint32_t)vs;
  }

  uint32_t *xl = a.xl + pd.out_off + j;  // limb l at xl[l N]
  int act = 1;
  xl[0] = col[(size_t)(K - 1) * N];
  for (int k = K - 2; k >= 0; --k) {
    int need = (31 * (K - k) + 1 + 31) / 32 + 1;
    if (need > L) need = L;
    if (need > act) {
      const uint32_t ext = (xl[(size_t)(act - 1) * N] >> 31) ? 0xffffffffu : 0u;
      for (int l = act; l < need; ++l) xl[(size_t)l * N] = ext;
      act = need;
    }
    const uint64_t p = a.mods[k].p;
    const int32_t vk = (int32_t)col[(size_t)k * N];
    const uint64_t ext = vk < 0 ? 0xffffffffull : 0ull;
    uint64_t c = (uint32_t)vk;
    for (int l = 0; l < act; ++l) {
      const uint64_t t = (uint64_t)xl[(size_t)l * N] * p + c + (l ? ext : 0ull);
      xl[(size_t)l * N] = (uint32_t)t;
      c = t >> 32;
    }
  }
  const uint32_t ext = (xl[(size_t)(act - 1) * N] >> 31) ? 0xffffffffu : 0u;
  uint32_t *o = a.out + pd.out_off + (size_t)j * L;
  for (int l = 0; l < L; ++l) o[l] = l < act ? xl[(size_t)l * N] : ext;
}

// Per prime: Montgomery constants, V[l] = 2^(32 l) R^2 mod p (limb weights
// for the modular reduction of input coefficients) and the Garner constant
// (p_0 ... p_{k-1})^{-1} mod p_k.
__global__ void init_primes_kernel(const uint32_t *primes, int n, ModP *mods, uint32_t *vtab,
                                   uint32_t *crt) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const ModP m = make_modp(primes[k]);
  mods[k] = m;
  uint32_t v = m.r2;
  for (int l = 0; l < RS_VT_STRIDE; ++l) {
    vtab[(size_t)k * RS_VT_STRIDE + l] = v;
    v = mmul(v, m.r2, m);
  }
  uint32_t acc = m.r1;
  for (int l = 0; l < k; ++l) acc = mmul(acc, to_mont(primes[l] - m.p, m), m);
  crt[k] = minv(acc, m);
}

__global__ void finalize_images_kernel(const ModP *mods, const uint32_t *num, const uint32_t *den,
                                       uint32_t *z, int K, int N) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)K * N) return;
  const ModP m = mods[i / N];
  z[i] = from_mont(mmul(num[i], minv(den[i], m), m), m);
}

}  // namespace

cudaError_t g2_prepare(size_t smem) {
  (void)smem;  // per-kernel attribute: allow the largest any plan may need
  return cudaFuncSetAttribute(g2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              RS_G2_MAX_SMEM_BYTES);
}

cudaError_t launch_g2(int threads, int blocks, size_t smem, const G2Args &a, cudaStream_t s) {
  g2_kernel<<<blocks, threads, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_g3(int threads, int blocks, const G3Args &a, cudaStream_t s) {
  g3_kernel<<<blocks, threads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_init_primes(const uint32_t *primes, int n, ModP *mods, uint32_t *vtab,
                               uint32_t *crt, cudaStream_t s) {
  init_primes_kernel<<<(n + 127) / 128, 128, 0, s>>>(primes, n, mods, vtab, crt);
  return cudaGetLastError();
}

cudaError_t launch_finalize_images(const ModP *mods, const uint32_t *num, const uint32_t *den,
                                   uint32_t *z, int K, int N, cudaStream_t s) {
  const size_t n = (size_t)K * N;
  finalize_images_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(mods, num, den, z, K, N);
  return cudaGetLastError();
}
