// Square-free factorisation of R mod p (the paper's solver computes R^{(y)}
// together with its square-free factorisation, Section 5, PROJECT), one warp
// per (pair, prime), between the interpolation (G2) and the Chinese
// remaindering (G3): Yun's algorithm (D. Y. Y. Yun, SYMSAC 1976) over Z_p on
// the interpolated residues of R,
//   A = gcd(F, F'), B = F / A, C = F' / A, D = C - B';
//   repeat: R_i = gcd(B, D), B = B / R_i, C = D / R_i, D = C - B'
// with monic R_i.  Remainders for the gcds are division-free (X <- lc(Y) X -
// lc(X) x^s Y, the degree drops by one per step; a gcd is only defined up to
// a unit), exact divisions use one inverse of the divisor's leading
// coefficient.  Each step is spread over the warp's lanes; a remainder step
// reads the new leading coefficient once (it is non-zero unless p divides it,
// and only then is the polynomial scanned for its degree), so a step costs one
// warp barrier.  The polynomials live in global scratch, except two buffers
// in shared memory (when they fit) that hold what every pass touches: the
// gcd operands, then the division remainder and the divisor.
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

constexpr unsigned FULL = 0xffffffffu;

struct Poly {
  uint32_t *c;  // Montgomery form, c[0 .. deg]; words above deg are don't-care
  int deg;      // -1 for the zero polynomial
};

__device__ __forceinline__ int lane_id() { return (int)(threadIdx.x & 31u); }

// Highest j <= from with p[j] != 0, or -1 (the same value in every lane).
__device__ int top_degree(const uint32_t *p, int from) {
  for (int hi = from; hi >= 0; hi -= 32) {
    const int j = hi - lane_id();
    const unsigned m = __ballot_sync(FULL, j >= 0 && p[j] != 0u);
    if (m) return hi - (__ffs(m) - 1);  // the lowest lane holds the highest index
  }
  return -1;
}

__device__ void copy_poly(Poly &dst, const Poly &src) {
  for (int j = lane_id(); j <= src.deg; j += 32) dst.c[j] = src.c[j];
  dst.deg = src.deg;
  __syncwarp();
}

// d = p' (d may not alias p).
__device__ void derivative(Poly &d, const Poly &p, const ModP &m) {
  for (int j = lane_id(); j < p.deg; j += 32) d.c[j] = mmul(p.c[j + 1], to_mont((uint32_t)(j + 1), m), m);
  __syncwarp();
  d.deg = p.deg >= 1 ? top_degree(d.c, p.deg - 1) : -1;
}

// x <- x - y (in place).
__device__ void sub_in_place(Poly &x, const Poly &y, const ModP &m) {
  const int n = max(x.deg, y.deg);
  for (int j = lane_id(); j <= n; j += 32) {
    const uint32_t a = j <= x.deg ? x.c[j] : 0u, b = j <= y.deg ? y.c[j] : 0u;
    x.c[j] = msub(a, b, m.p);
  }
  __syncwarp();
  x.deg = n >= 0 ? top_degree(x.c, n) : -1;
}

// x <- x mod y up to a unit factor (division-free), y non-zero.  A step
// rewrites x[0 .. deg) and never its leading coefficient, and each step ends
// with a warp barrier, so the next step's reads of the leading coefficients
// follow the writes.  In the normal case deg x = deg y + 1 one pass takes two
// division steps at once:
//   x <- lc(y)^2 x - (a t + b) y,  a = lc(y) x_n,  b = lc(y) x_{n-1} - x_n y_{n-2},
// whose coefficients n and n - 1 vanish; otherwise one step
//   x <- lc(y) x - lc(x) t^s y.
__device__ void rem_in_place(Poly &x, const Poly &y, const ModP &m) {
  uint32_t *__restrict__ xc = x.c;
  const uint32_t *__restrict__ yc = y.c;
  const int dy = y.deg;
  const uint32_t ly = yc[dy];
  const uint32_t c2 = mmul(ly, ly, m);
  while (x.deg >= dy) {
    const int n = x.deg, s = n - dy;
    if (s == 1 && dy >= 1) {
      const uint32_t xn = xc[n], xn1 = xc[n - 1];
      const uint32_t na = mneg(mmul(ly, xn, m), m.p);
      const uint32_t nb = msub(mmul(xn, yc[dy - 1], m), mmul(ly, xn1, m), m.p);
      // four coefficients per iteration, loads first
      const int e = n - 1;
      int j = lane_id();
      for (; j + 96 < e; j += 128) {
        uint32_t xv[4], yv[4], zv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          xv[u] = xc[j + 32 * u];
          yv[u] = yc[j + 32 * u];
          zv[u] = (u > 0 || j >= 1) ? yc[j + 32 * u - 1] : 0u;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) xc[j + 32 * u] = madd(mmul2(c2, xv[u], na, zv[u], m), mmul(nb, yv[u], m), m.p);
      }
      for (; j < e; j += 32) {
        const uint32_t t1 = j >= 1 ? mmul2(c2, xc[j], na, yc[j - 1], m) : mmul(c2, xc[j], m);
        xc[j] = madd(t1, mmul(nb, yc[j], m), m.p);
      }
      __syncwarp();
      const int nd = n - 2;
      x.deg = (nd < 0 || xc[nd] != 0u) ? nd : top_degree(xc, nd);
    } else {
      const uint32_t nlx = mneg(xc[n], m.p);
      for (int j = lane_id(); j < n; j += 32)
        xc[j] = j >= s ? mmul2(ly, xc[j], nlx, yc[j - s], m) : mmul(ly, xc[j], m);
      __syncwarp();
      const int nd = n - 1;
      x.deg = (nd < 0 || xc[nd] != 0u) ? nd : top_degree(xc, nd);
    }
  }
}

// x <- x / lc(x).
__device__ void make_monic(Poly &x, const ModP &m) {
  if (x.deg < 0) return;
  const uint32_t inv = minv(x.c[x.deg], m);  // every lane computes the same inverse
  __syncwarp();
  for (int j = lane_id(); j <= x.deg; j += 32) x.c[j] = mmul(x.c[j], inv, m);
  __syncwarp();
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

// q <- x / y exactly (y non-zero and dividing x); r is scratch holding x's
// copy.  One pass takes two quotient coefficients q_t, q_{t-1} (the second
// after the first's correction of r[deg y + t - 1]) and subtracts
// (q_t t^t + q_{t-1} t^{t-1}) y from r; a pass reads the top two words of r,
// which the previous pass wrote, and writes below them, with one barrier per
// pass.
__device__ void divexact(Poly &q, const Poly &x, const Poly &y, Poly &r, const ModP &m) {
  copy_poly(r, x);
  const int dq = x.deg - y.deg, n = y.deg;
  const uint32_t inv = minv(y.c[n], m);
  uint32_t *__restrict__ rc = r.c;
  const uint32_t *__restrict__ yc = y.c;
  q.deg = max(dq, -1);
  if (n == 0) {  // a constant divisor
    for (int t = lane_id(); t <= dq; t += 32) q.c[t] = mmul(rc[t], inv, m);
    __syncwarp();
    return;
  }
  int t = dq;
  for (; t >= 1; t -= 2) {
    const uint32_t qt = mmul(rc[n + t], inv, m);
    const uint32_t qt1 = mmul(msub(rc[n + t - 1], mmul(qt, yc[n - 1], m), m.p), inv, m);
    const uint32_t nq = mneg(qt, m.p), nq1 = mneg(qt1, m.p);
    const int e = n + t - 1;
    int i = t - 1 + lane_id();
    for (; i + 96 < e; i += 128) {  // four coefficients per iteration, loads first
      const int k = i - t;           // y index of the q_t term
      uint32_t rv[4], av[4], bv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        rv[u] = rc[i + 32 * u];
        av[u] = (u > 0 || k >= 0) ? yc[k + 32 * u] : 0u;
        bv[u] = yc[k + 32 * u + 1];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) rc[i + 32 * u] = madd(rv[u], mmul2(nq, av[u], nq1, bv[u], m), m.p);
    }
    for (; i < e; i += 32) {
      const int k = i - t;
      const uint32_t v = k >= 0 ? mmul2(nq, yc[k], nq1, yc[k + 1], m) : mmul(nq1, yc[0], m);
      rc[i] = madd(rc[i], v, m.p);
    }
    if (lane_id() == 0) {
      q.c[t] = qt;
      q.c[t - 1] = qt1;
    }
    __syncwarp();
  }
  if (t == 0) {
    const uint32_t q0 = mmul(rc[n], inv, m);
    if (lane_id() == 0) q.c[0] = q0;
    __syncwarp();
  }
}

__global__ void __launch_bounds__(32) yun_kernel(YunArgs a) {
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
  for (int j = lane_id(); j < N; j += 32) F.c[j] = to_mont(res[j], m);
  __syncwarp();
  F.deg = top_degree(F.c, N - 1);
  if (lane_id() == 0) {
    o[0] = (uint32_t)F.deg;
    o[1] = 0u;
  }
  for (int i = lane_id(); i < a.maxm; i += 32) o[2 + i] = 0u;
  if (F.deg <= 0) return;  // R = 0 or a constant mod p: no factors
  const uint32_t lcR = F.c[F.deg];
  derivative(Fd, F, m);
  copy_poly(T1, F);
  copy_poly(T2, Fd);
  gcd_monic(A, T1, T2, m);       // A = gcd(F, F')
  copy_poly(T2, A);              // the divisor, read by every division pass
  divexact(B, F, T2, T1, m);     // B = F / A
  divexact(C, Fd, T2, T1, m);    // C = F' / A
  derivative(T2, B, m);
  copy_poly(D, C);
  sub_in_place(D, T2, m);        // D = C - B'
  uint32_t *dst = o + 2 + a.maxm;
  int i = 1;
  while (B.deg > 0) {
    if (i > a.maxm) {
      if (lane_id() == 0) o[1] = 1u;
      return;
    }
    // R_i = gcd(B, D) into the buffer of F' (free after the first step),
    // on copies of B and D
    Poly &Ri = Fd;
    copy_poly(T1, B);
    copy_poly(T2, D);
    gcd_monic(Ri, T1, T2, m);
    // emit lc(R) R_i (plain) and its degree
    for (int j = lane_id(); j <= Ri.deg; j += 32) dst[j] = from_mont(mmul(Ri.c[j], lcR, m), m);
    if (lane_id() == 0) o[1 + i] = (uint32_t)Ri.deg;
    dst += Ri.deg + 1;
    // B = B / R_i, C = D / R_i, D = C - B'
    copy_poly(T2, Ri);          // the divisor, read by every division pass
    divexact(A, B, T2, T1, m);  // A is free now: the new B
    divexact(C, D, T2, T1, m);
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
  yun_kernel<<<ntasks, 32, dyn, s>>>(b);
  return cudaGetLastError();
}
