// Univariate resultants mod p by the generalised Schur algorithm on
// displacement generators: the paper's own GPU kernel (Section 4.1), built
// here as a variant of G1 for comparison with the remainder sequence.
//
// The Sylvester matrix S of Section 3.1 (n_y rows of f, then m_y rows of g,
// coefficients in descending powers) is structured: its transpose M = S^T
// satisfies the displacement equation
//   M - Z M A^T = G B^T,  A = Z_{n_y} (+) Z_{m_y},
// Z the down-shift, with the two-column generators read off by inspection:
// G = [f_{m_y}, ..., f_0, 0, ... | g_{n_y}, ..., g_0, 0, ...] (the first
// columns of the f block and of the g block of M) and B = [e_0 | e_{n_y}].
// One Schur step on generators (G, B) whose row k is (a, b | c, d) takes the
// pivot t = a c + b d (= M_kk of the current Schur complement) and forms
//   G' = [Z (c G_0 + d G_1) | -b G_0 + a G_1],
//   B' = [A (a B_0 + b B_1) | -d B_0 + c B_1],
// the generators of t times the next Schur complement (row k of both
// becomes zero): division-free.  With c_0 = 1, c_{k+1} = c_k t_k the true
// pivots are t_k / c_k, so det M = prod t_k / prod c_k: a numerator and a
// denominator, exactly what G2 takes from G1.
//
// Mapping: one warp per image (the paper uses r threads per resultant); lane
// l holds rows l, l + 32, ... of the four generator columns in registers, the
// pivot row is broadcast by shuffles and the two shifts move values one lane
// up.  A zero pivot (a leading principal minor of M vanishes mod p, e.g. at a
// point where lc_y f vanishes) stops the recurrence: the image goes to a list
// that a second kernel finishes by Gaussian elimination with row pivoting on
// the Sylvester matrix, so every image is exact.
#include "blockinv.cuh"
#include "rs_internal.cuh"

namespace {

constexpr unsigned FULL = 0xffffffffu;

// f_ij mod p (Montgomery form) from two's-complement limbs: sum_l limb_l 2^{32 l}.
__device__ __forceinline__ uint32_t reduce_limbs(const uint32_t *src, int L, const uint32_t *V, const ModP &m) {
  uint32_t acc = 0u;
  for (int l = 0; l < L; ++l) acc = madd(acc, redc((uint64_t)src[l] * V[l], m.p, m.pinv), m.p);
  if (src[L - 1] >> 31) acc = msub(acc, redc((uint64_t)V[L], m.p, m.pinv), m.p);
  return acc;
}

// sum_i c[i] x^i by Horner's rule (Montgomery form).
__device__ __forceinline__ uint32_t horner(const uint32_t *c, int n, uint32_t x, const ModP &m) {
  uint32_t acc = 0u;
  for (int i = n - 1; i >= 0; --i) acc = madd(mmul(acc, x, m), c[i], m.p);
  return acc;
}

// Stage f_ij and g_ij mod p of a pair in shared memory: sf[j (mxf + 1) + i].
__device__ void stage_residues(uint32_t *sf, uint32_t *sg, const PairDesc &pd, const uint32_t *limbs,
                               const uint32_t *V, const ModP &m) {
  const int wf = pd.mxf + 1, wg = pd.mxg + 1;
  for (int e = threadIdx.x; e < (pd.my + 1) * wf; e += blockDim.x) {
    const int j = e / wf, i = e - j * wf;
    sf[e] = reduce_limbs(limbs + pd.f_off + ((size_t)i * pd.fstride + j) * pd.Lf, pd.Lf, V, m);
  }
  for (int e = threadIdx.x; e < (pd.ny + 1) * wg; e += blockDim.x) {
    const int j = e / wg, i = e - j * wg;
    sg[e] = reduce_limbs(limbs + pd.g_off + ((size_t)i * pd.gstride + j) * pd.Lg, pd.Lg, V, m);
  }
}

template <int T>
__device__ __forceinline__ uint32_t pick(const uint32_t (&v)[T], int t) {
  uint32_t r = 0u;
#pragma unroll
  for (int s = 0; s < T; ++s)
    if (s == t) r = v[s];
  return r;
}

// One block per G1 tile (point pairs [x0, x0 + n) of one (pair, prime));
// each warp takes every fourth image of the tile.  T = row slots per lane
// (m_y + n_y <= 32 T).
template <int T>
__global__ void __launch_bounds__(128) g1s_kernel(G1sArgs a) {
  extern __shared__ __align__(16) uint32_t sm[];
  const Tile tl = a.tiles[blockIdx.x];
  const PairDesc pd = a.pairs[tl.pair];
  const ModP m = a.mods[tl.prime];
  const int my = pd.my, ny = pd.ny, r = my + ny;
  const int wf = pd.mxf + 1, wg = pd.mxg + 1;
  uint32_t *sf = sm, *sg = sm + (my + 1) * wf;
  stage_residues(sf, sg, pd, a.limbs, a.vtab + (size_t)tl.prime * RS_VT_STRIDE, m);
  __syncthreads();
  const int lane = (int)(threadIdx.x & 31u), warp = (int)(threadIdx.x >> 5), nw = (int)(blockDim.x >> 5);
  const size_t tb = (size_t)tl.prime * a.tstride;
  unsigned long long n_unlucky = 0, n_degen = 0;
  for (int e = warp; e < 2 * tl.n; e += nw) {
    const int i = tl.x0 + (e >> 1), par = e & 1;
    const uint32_t q = a.qp[tb + i];
    const uint32_t x = par ? mneg(q, m.p) : q;
    const size_t idx = (size_t)pd.img_off + (size_t)tl.prime * pd.NI + 2 * i + par;
    uint32_t G0[T], G1[T], B0[T], B1[T];
#pragma unroll
    for (int t = 0; t < T; ++t) {
      const int k = lane + 32 * t;
      G0[t] = k <= my ? horner(sf + (my - k) * wf, wf, x, m) : 0u;
      G1[t] = k <= ny ? horner(sg + (ny - k) * wg, wg, x, m) : 0u;
      B0[t] = k == 0 ? m.r1 : 0u;
      B1[t] = k == ny ? m.r1 : 0u;
    }
    const uint32_t lcf = __shfl_sync(FULL, G0[0], 0), lcg = __shfl_sync(FULL, G1[0], 0);
    if (lcf == 0u || lcg == 0u) ++n_unlucky;
    uint32_t num = m.r1, den = m.r1;
    bool broke = false;
    if (my == 0 || ny == 0) {  // Res = f_0^{n_y} (m_y = 0) or g_0^{m_y} (n_y = 0)
      num = my == 0 ? mpow(lcf, (uint32_t)ny, m) : mpow(lcg, (uint32_t)my, m);
    } else {
      uint32_t c = m.r1;
      for (int k = 0; k < r; ++k) {
        const int ol = k & 31, os = k >> 5;
        const uint32_t al = __shfl_sync(FULL, pick(G0, os), ol), be = __shfl_sync(FULL, pick(G1, os), ol);
        const uint32_t ga = __shfl_sync(FULL, pick(B0, os), ol), de = __shfl_sync(FULL, pick(B1, os), ol);
        const uint32_t d = mmul2(al, ga, be, de, m);
        if (d == 0u) {  // the same in every lane
          broke = true;
          break;
        }
        num = mmul(num, d, m);
        den = mmul(den, c, m);
        c = mmul(c, d, m);
        const uint32_t nbe = mneg(be, m.p), nde = mneg(de, m.p);
        uint32_t L[T], U[T];
#pragma unroll
        for (int t = 0; t < T; ++t) {
          if (32 * t + 31 < k) {  // every row of the slot is eliminated (zero)
            L[t] = 0u;
            U[t] = 0u;
            continue;
          }
          L[t] = mmul2(ga, G0[t], de, G1[t], m);
          G1[t] = mmul2(nbe, G0[t], al, G1[t], m);
          U[t] = mmul2(al, B0[t], be, B1[t], m);
          B1[t] = mmul2(nde, B0[t], ga, B1[t], m);
        }
        // row j takes row j - 1 (the lane below, or lane 31 of the slot
        // below); the g block of B restarts at row n_y
#pragma unroll
        for (int t = 0; t < T; ++t) {
          const uint32_t lu = __shfl_up_sync(FULL, L[t], 1), uu = __shfl_up_sync(FULL, U[t], 1);
          const uint32_t lp = t ? __shfl_sync(FULL, L[t > 0 ? t - 1 : 0], 31) : 0u;
          const uint32_t up = t ? __shfl_sync(FULL, U[t > 0 ? t - 1 : 0], 31) : 0u;
          G0[t] = lane ? lu : lp;
          B0[t] = (lane + 32 * t == ny) ? 0u : (lane ? uu : up);
        }
      }
    }
    if (lane == 0) {
      if (broke) {
        const int pos = atomicAdd(a.fail_count, 1);
        a.fail[pos] = make_int2((int)blockIdx.x, e);
        ++n_degen;
      } else {
        a.num[idx] = num;
        a.den[idx] = den;
      }
    }
  }
  if (lane == 0) {
    if (n_unlucky) atomicAdd(a.stats + ST_UNLUCKY_POINTS, n_unlucky);
    if (n_degen) atomicAdd(a.stats + ST_DEGENERATE, n_degen);
  }
}

// The images whose Schur recurrence met a zero pivot: det S(x) mod p by
// Gaussian elimination with row pivoting on the Sylvester matrix in shared
// memory (r x r words, then r words of elimination factors), one block per
// listed image, blocks striding over the list.
__global__ void __launch_bounds__(256) g1s_fallback_kernel(G1sArgs a) {
  extern __shared__ __align__(16) uint32_t fm[];
  __shared__ int s_piv;
  const int count = *a.fail_count;
  for (int w = blockIdx.x; w < count; w += gridDim.x) {
    const int2 fl = a.fail[w];
    const Tile tl = a.tiles[fl.x];
    const PairDesc pd = a.pairs[tl.pair];
    const ModP m = a.mods[tl.prime];
    const uint32_t *V = a.vtab + (size_t)tl.prime * RS_VT_STRIDE;
    const int my = pd.my, ny = pd.ny, r = my + ny;
    const int i = tl.x0 + (fl.y >> 1), par = fl.y & 1;
    const uint32_t q = a.qp[(size_t)tl.prime * a.tstride + i];
    const uint32_t x = par ? mneg(q, m.p) : q;
    uint32_t *M = fm, *fac = fm + (size_t)r * r, *fv = fac + r, *gv = fv + my + 1;
    // coefficient values f_j(x), g_j(x) (reduced and evaluated straight from the limbs)
    for (int j = threadIdx.x; j <= my + ny + 1; j += blockDim.x) {
      const bool isf = j <= my;
      const int jj = isf ? j : j - my - 1;
      const int w1 = isf ? pd.mxf + 1 : pd.mxg + 1;
      const uint32_t *base = a.limbs + (isf ? pd.f_off : pd.g_off);
      const int stride = isf ? pd.fstride : pd.gstride, L = isf ? pd.Lf : pd.Lg;
      uint32_t acc = 0u;
      for (int k = w1 - 1; k >= 0; --k)
        acc = madd(mmul(acc, x, m), reduce_limbs(base + ((size_t)k * stride + jj) * L, L, V, m), m.p);
      (isf ? fv : gv)[jj] = acc;
    }
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) M[e] = 0u;
    __syncthreads();
    for (int e = threadIdx.x; e < ny * (my + 1); e += blockDim.x) {  // f rows
      const int row = e / (my + 1), k = e - row * (my + 1);
      M[row * r + row + k] = fv[my - k];
    }
    for (int e = threadIdx.x; e < my * (ny + 1); e += blockDim.x) {  // g rows
      const int row = e / (ny + 1), k = e - row * (ny + 1);
      M[(ny + row) * r + row + k] = gv[ny - k];
    }
    __syncthreads();
    uint32_t det = m.r1;
    bool neg = false;
    for (int c = 0; c < r; ++c) {
      if (threadIdx.x == 0) s_piv = r;
      __syncthreads();
      for (int row = c + (int)threadIdx.x; row < r; row += blockDim.x)
        if (M[row * r + c] != 0u) atomicMin(&s_piv, row);
      __syncthreads();
      const int piv = s_piv;
      __syncthreads();
      if (piv == r) {
        det = 0u;
        break;
      }
      if (piv != c) {
        for (int col = c + (int)threadIdx.x; col < r; col += blockDim.x) {
          const uint32_t t = M[c * r + col];
          M[c * r + col] = M[piv * r + col];
          M[piv * r + col] = t;
        }
        neg = !neg;
        __syncthreads();
      }
      const uint32_t pv = M[c * r + c];
      det = mmul(det, pv, m);
      const uint32_t inv = minv(pv, m);
      for (int row = c + 1 + (int)threadIdx.x; row < r; row += blockDim.x) fac[row] = mmul(M[row * r + c], inv, m);
      __syncthreads();
      const int wdt = r - c - 1;
      for (int e = threadIdx.x; e < wdt * wdt; e += blockDim.x) {
        const int row = c + 1 + e / wdt, col = c + 1 + e % wdt;
        M[row * r + col] = msub(M[row * r + col], mmul(fac[row], M[c * r + col], m), m.p);
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      const size_t idx = (size_t)pd.img_off + (size_t)tl.prime * pd.NI + 2 * i + par;
      a.num[idx] = neg ? mneg(det, m.p) : det;
      a.den[idx] = m.r1;
    }
    __syncthreads();  // the next image reuses shared memory
  }
}

// Interpolation (a5) by the triangular factorisation of the Vandermonde
// system V c = z, V[j][i] = x_j^i (the paper solves it with the Schur
// algorithm, exploiting its structure; this is the comparison variant of
// G2).  The displacement V - D V Z^T (D = diag x_j) has rank one, and its
// Schur recursion yields V's triangular factors; applying their inverses as
// bidiagonal stages is the method of A. Bjorck and V. Pereyra ("Solution of
// Vandermonde systems of equations", Math. Comp. 24, 1970):
//   stage 1 (divided differences): for k = 0 .. N-2, for j > k:
//     c_j <- (c_j - c_{j-1}) / (x_j - x_{j-k-1});
//   stage 2 (Newton to monomial):  for k = N-2 .. 0, for k <= j < N-1:
//     c_j <- c_j - x_k c_{j+1}.
// Each stage is one parallel step over j (O(N) parallel time, O(N^2) work).
// Stage 1 runs on fractions (numerator, denominator), starting from G1's
// num/den images, so no division is taken until one simultaneous inversion
// of the N denominators between the stages.  Thread t owns the contiguous
// indices [t E, t E + E); it walks them downward in stage 1 and upward in
// stage 2, reading the one old value it needs from a neighbour's range
// before the stage's barrier.  Points: the first N images, x_j =
// (-1)^j q^{floor(j/2)}.
__global__ void __launch_bounds__(256) g2s_kernel(G2sArgs a) {
  extern __shared__ __align__(16) uint32_t sv[];
  const int2 task = a.tasks[blockIdx.x];
  const PairDesc pd = a.pairs[task.x];
  const ModP m = a.mods[task.y];
  const int N = pd.N, T = (int)blockDim.x, tid = (int)threadIdx.x;
  uint32_t *A = sv, *Bd = sv + N, *X = sv + 2 * N, *Inv = sv + 3 * N, *scratch = sv + 4 * N;
  const size_t base = (size_t)pd.img_off + (size_t)task.y * pd.NI;
  const uint32_t *qp = a.qp + (size_t)task.y * a.tstride;
  for (int j = tid; j < N; j += T) {
    A[j] = a.num[base + j];
    Bd[j] = a.den[base + j];
    const uint32_t q = qp[j >> 1];
    X[j] = (j & 1) ? mneg(q, m.p) : q;
  }
  __syncthreads();
  const int E = (N + T - 1) / T;
  const int beg = min(tid * E, N), end = min(beg + E, N);
  for (int k = 0; k + 1 < N; ++k) {
    const int lo = max(beg, k + 1);
    uint32_t pa = 0u, pb = 0u;
    if (lo < end) {
      pa = A[lo - 1];
      pb = Bd[lo - 1];
    }
    __syncthreads();
    for (int j = end - 1; j >= lo; --j) {
      const uint32_t aj = A[j], bj = Bd[j];
      const uint32_t am = j > lo ? A[j - 1] : pa, bm = j > lo ? Bd[j - 1] : pb;
      const uint32_t e = msub(X[j], X[j - k - 1], m.p);
      A[j] = mmul2(aj, bm, mneg(am, m.p), bj, m);
      Bd[j] = mmul(mmul(bj, bm, m), e, m);
    }
    __syncthreads();
  }
  batch_invert(Bd, Inv, N, m, scratch);
  __syncthreads();
  for (int j = tid; j < N; j += T) A[j] = mmul(A[j], Inv[j], m);
  __syncthreads();
  for (int k = N - 2; k >= 0; --k) {
    const int lo = max(beg, k), hi = min(end, N - 1);
    const uint32_t nx = lo < hi ? A[hi] : 0u;
    __syncthreads();
    const uint32_t xk = X[k];
    for (int j = lo; j < hi; ++j) {
      const uint32_t cn = j + 1 < hi ? A[j + 1] : nx;
      A[j] = msub(A[j], mmul(xk, cn, m), m.p);
    }
    __syncthreads();
  }
  for (int j = tid; j < N; j += T) a.coef[base + j] = from_mont(A[j], m);
}

}  // namespace

cudaError_t launch_g2s(int ntasks, size_t smem, const G2sArgs &a, cudaStream_t s) {
  if (!ntasks) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(g2s_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  g2s_kernel<<<ntasks, 256, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_g1s(int slots, int ntiles, size_t smem, const G1sArgs &a, cudaStream_t s) {
  if (!ntiles) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  switch (slots) {
#define RS_G1S_CASE(TT)                                                                              \
  case TT:                                                                                           \
    e = cudaFuncSetAttribute(g1s_kernel<TT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    if (e != cudaSuccess) return e;                                                                  \
    g1s_kernel<TT><<<ntiles, 128, smem, s>>>(a);                                                     \
    break;
    RS_G1S_CASE(1)
    RS_G1S_CASE(2)
    RS_G1S_CASE(3)
    RS_G1S_CASE(4)
    RS_G1S_CASE(5)
#undef RS_G1S_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_g1s_fallback(int blocks, size_t smem, const G1sArgs &a, cudaStream_t s) {
  const cudaError_t e = cudaFuncSetAttribute(g1s_fallback_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
  if (e != cudaSuccess) return e;
  g1s_fallback_kernel<<<blocks, 256, smem, s>>>(a);
  return cudaGetLastError();
}
