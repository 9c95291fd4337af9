// Square-free factorisation of R mod p (the paper's solver, Section 5,
// PROJECT: R^{(y)} "and a corresponding square-free factorization"), one
// thread block per (pair, prime), between the interpolation (G2) and the
// Chinese remaindering (G3): Yun's algorithm (D. Y. Y. Yun, SYMSAC 1976) over
// Z_p on the interpolated residues of R,
//   A = gcd(F, F'), B = F / A, C = F' / A, D = C - B';
//   repeat: R_i = gcd(B, D), B = B / R_i, C = D / R_i, D = C - B'
// with monic R_i.  Remainders for the gcds are division-free (X <- lc(Y) X -
// lc(X) x^s Y, the degree drops by one per step; a gcd is only defined up to
// a unit), exact divisions use one inverse of the divisor's leading
// coefficient, and every step is spread over the block's threads with a
// barrier.  The polynomials live in global scratch, except the two that every
// remainder and division step rewrites (the gcd operands and the division
// remainder), which live in shared memory when they fit.
//
// Output per task (word offsets from out + task * ostride):
//   [0]            degree of R mod p (-1 if R = 0 mod p)
//   [1]            1 if the multiplicities exceed maxm, else 0
//   [2 .. 2+maxm)  degree d_i of R_i mod p for i = 1..maxm (0: R_i = 1)
//   then for i = 1..maxm the d_i + 1 coefficients (ascending, plain form) of
//   lc(R) R_i mod p, back to back (the layout the CRT kernels read with
//   stride ostride when every prime has the same degrees).
#include "../../include/rs.h"
#include "rs_internal.cuh"

namespace {

struct Poly {
  uint32_t *c;  // Montgomery form, c[0 .. deg]
  int deg;      // -1 for the zero polynomial
};

// Highest j <= from with p[j] != 0, or -1 (all threads return the same value).
__device__ int top_degree(const uint32_t *p, int from, int *s_min) {
  const int T = blockDim.x;
  for (int hi = from; hi >= 0; hi -= T) {
    const int j = hi - (int)threadIdx.x;
    const bool nz = j >= 0 && p[j] != 0u;
    if (__syncthreads_or(nz)) {
      if (threadIdx.x == 0) *s_min = T;
      __syncthreads();
      if (nz) atomicMin(s_min, (int)threadIdx.x);
      __syncthreads();
      const int r = hi - *s_min;
      __syncthreads();
      return r;
    }
  }
  return -1;
}

__device__ void copy_poly(Poly &dst, const Poly &src) {
  for (int j = threadIdx.x; j <= src.deg; j += blockDim.x) dst.c[j] = src.c[j];
  dst.deg = src.deg;
  __syncthreads();
}

// d = p' (d may not alias p).
__device__ void derivative(Poly &d, const Poly &p, const ModP &m) {
  for (int j = threadIdx.x; j < p.deg; j += blockDim.x) d.c[j] = mmul(p.c[j + 1], to_mont((uint32_t)(j + 1), m), m);
  __syncthreads();
  d.deg = p.deg - 1;
  if (d.deg >= 0) {
    __shared__ int s_min;
    d.deg = top_degree(d.c, d.deg, &s_min);
  }
}

// x <- x - y (in place).
__device__ void sub_in_place(Poly &x, const Poly &y, const ModP &m) {
  const int n = max(x.deg, y.deg);
  for (int j = threadIdx.x; j <= n; j += blockDim.x) {
    const uint32_t a = j <= x.deg ? x.c[j] : 0u, b = j <= y.deg ? y.c[j] : 0u;
    x.c[j] = msub(a, b, m.p);
  }
  __syncthreads();
  __shared__ int s_min;
  x.deg = n >= 0 ? top_degree(x.c, n, &s_min) : -1;
}

// x <- x mod y up to a unit factor (division-free), y non-zero.
__device__ void rem_in_place(Poly &x, const Poly &y, const ModP &m) {
  __shared__ int s_min;
  while (x.deg >= y.deg && x.deg >= 0) {
    const int s = x.deg - y.deg;
    const uint32_t lx = x.c[x.deg], ly = y.c[y.deg];
    __syncthreads();
    const uint32_t nlx = mneg(lx, m.p);
    for (int j = threadIdx.x; j < x.deg; j += blockDim.x)
      x.c[j] = j >= s ? mmul2(ly, x.c[j], nlx, y.c[j - s], m) : mmul(ly, x.c[j], m);
    if (threadIdx.x == 0) x.c[x.deg] = 0u;
    __syncthreads();
    x.deg = x.deg > 0 ? top_degree(x.c, x.deg - 1, &s_min) : -1;
  }
}

__device__ uint32_t block_inverse(uint32_t v, const ModP &m) {
  __shared__ uint32_t s_inv;
  if (threadIdx.x == 0) s_inv = minv(v, m);
  __syncthreads();
  const uint32_t r = s_inv;
  __syncthreads();
  return r;
}

// x <- x / lc(x).
__device__ void make_monic(Poly &x, const ModP &m) {
  if (x.deg < 0) return;
  const uint32_t inv = block_inverse(x.c[x.deg], m);
  for (int j = threadIdx.x; j <= x.deg; j += blockDim.x) x.c[j] = mmul(x.c[j], inv, m);
  __syncthreads();
}

// g <- monic gcd(a, b), copied into g's own buffer; a and b (distinct from
// g) are destroyed.
__device__ void gcd_monic(Poly &g, Poly a, Poly b, const ModP &m) {
  if (a.deg < b.deg) {
    const Poly t = a;
    a = b;
    b = t;
  }
  while (b.deg >= 0) {
    rem_in_place(a, b, m);
    const Poly t = a;
    a = b;
    b = t;
  }
  make_monic(a, m);
  copy_poly(g, a);
}

// q <- x / y exactly (y non-zero and dividing x); r is scratch holding x's copy.
__device__ void divexact(Poly &q, const Poly &x, const Poly &y, Poly &r, const ModP &m) {
  copy_poly(r, x);
  const int dq = x.deg - y.deg;
  const uint32_t inv = block_inverse(y.c[y.deg], m);
  for (int t = dq; t >= 0; --t) {
    const uint32_t qt = mmul(r.c[y.deg + t], inv, m);
    __syncthreads();
    const uint32_t nq = mneg(qt, m.p);
    for (int j = threadIdx.x; j < y.deg; j += blockDim.x) r.c[j + t] = madd(r.c[j + t], mmul(nq, y.c[j], m), m.p);
    if (threadIdx.x == 0) q.c[t] = qt;
    __syncthreads();
  }
  q.deg = max(dq, -1);
}

__global__ void __launch_bounds__(256) yun_kernel(YunArgs a) {
  const int2 task = a.tasks[blockIdx.x];
  const PairDesc pd = a.pairs[task.x];
  const ModP m = a.mods[task.y];
  const int N = pd.N;
  uint32_t *o = a.out + (size_t)blockIdx.x * a.ostride;
  uint32_t *w = a.work + (size_t)blockIdx.x * 8 * (size_t)a.wstride;
  extern __shared__ uint32_t ysm[];
  Poly P[8];
  for (int i = 0; i < 8; ++i) P[i] = Poly{w + (size_t)i * a.wstride, -1};
  if (a.shared_scratch) {
    P[6].c = ysm;
    P[7].c = ysm + a.wstride;
  }
  Poly &F = P[0], &Fd = P[1], &A = P[2], &B = P[3], &C = P[4], &D = P[5], &T1 = P[6], &T2 = P[7];
  const uint32_t *res = a.coef + pd.img_off + (size_t)task.y * pd.NI;
  for (int j = threadIdx.x; j < N; j += blockDim.x) F.c[j] = to_mont(res[j], m);
  __syncthreads();
  __shared__ int s_min;
  F.deg = top_degree(F.c, N - 1, &s_min);
  if (threadIdx.x == 0) {
    o[0] = (uint32_t)F.deg;
    o[1] = 0u;
  }
  for (int i = threadIdx.x; i < a.maxm; i += blockDim.x) o[2 + i] = 0u;
  if (F.deg <= 0) return;  // R = 0 or a constant mod p: no factors
  const uint32_t lcR = F.c[F.deg];
  derivative(Fd, F, m);
  copy_poly(T1, F);
  copy_poly(T2, Fd);
  gcd_monic(A, T1, T2, m);       // A = gcd(F, F')
  divexact(B, F, A, T1, m);      // B = F / A
  divexact(C, Fd, A, T1, m);     // C = F' / A
  derivative(T2, B, m);
  copy_poly(D, C);
  sub_in_place(D, T2, m);        // D = C - B'
  uint32_t *dst = o + 2 + a.maxm;
  int i = 1;
  while (B.deg > 0) {
    if (i > a.maxm) {
      if (threadIdx.x == 0) o[1] = 1u;
      return;
    }
    // R_i = gcd(B, D) into the buffer of F' (free after the first step),
    // on copies of B and D
    Poly &Ri = Fd;
    copy_poly(T1, B);
    copy_poly(T2, D);
    gcd_monic(Ri, T1, T2, m);
    // emit lc(R) R_i (plain) and its degree
    for (int j = threadIdx.x; j <= Ri.deg; j += blockDim.x) dst[j] = from_mont(mmul(Ri.c[j], lcR, m), m);
    if (threadIdx.x == 0) o[1 + i] = (uint32_t)Ri.deg;
    dst += Ri.deg + 1;
    // B = B / R_i, C = D / R_i, D = C - B'
    divexact(A, B, Ri, T1, m);  // A is free now: the new B
    divexact(C, D, Ri, T1, m);
    copy_poly(B, A);
    derivative(T2, B, m);
    copy_poly(D, C);
    sub_in_place(D, T2, m);
    ++i;
  }
}

}  // namespace

cudaError_t launch_yun(int ntasks, const YunArgs &a, cudaStream_t s) {
  if (!ntasks) return cudaSuccess;
  YunArgs b = a;
  const size_t smem = 2 * (size_t)a.wstride * sizeof(uint32_t);
  size_t dyn = 0;
  b.shared_scratch = 0;
  if (smem <= RS_YUN_MAX_SMEM_BYTES) {
    const cudaError_t e = cudaFuncSetAttribute(yun_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dyn = smem;
    b.shared_scratch = 1;
  }
  yun_kernel<<<ntasks, 256, dyn, s>>>(b);
  return cudaGetLastError();
}
