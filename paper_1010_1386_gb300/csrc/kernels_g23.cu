// G2 (interpolation mod p) and the per-prime constant tables.  Paper,
// Section 4.1: R^{(y)} is interpolated over Z_p from the images z_i^{(p)}
// (a Vandermonde solve); the Chinese remaindering is in kernels_g3.cu.
#include "../../include/rs.h"
#include "blockinv.cuh"
#include "rs_internal.cuh"

namespace {

// Interpolation at the geometric points x_i = q^i, i = 0..D (Section 4.1
// asks for the Vandermonde solve; on a geometric progression it factors into
// two convolutions).  With F_t = prod_{s=1}^t (q^s - 1) and
// b_t = (-1)^t q^{C(t,2)} / F_t:
//   Newton coefficients  c_k = q^{-C(k,2)} sum_{j<=k} (z_j / F_j) b_{k-j}
//   (the divided differences on a geometric progression, since
//   prod_{l<=k, l!=j} (q^j - q^l) = q^{C(k,2)} (-1)^{k-j} F_j F_{k-j} / q^{C(k-j,2)}),
//   monomial coefficients R_m = (1 / F_m) sum_{t<=D-m} (c_{m+t} F_{m+t}) b_t
//   (q-binomial expansion of prod_{j<k} (x - q^j)).
// Both sums are the convolution conv(x, b)_k = sum_{j<=k} x_j b_{k-j}, the
// second one on the reversed sequence.  Residues enter it as signed
// representatives |v| < 2^30, so 7 products accumulate exactly in an int64
// and one fold S = hi 2^32 + lo -> hi (2^32 mod p) + lo keeps |S| < 2^53
// (every table prime exceeds 2^31 - 2^20, so 2^32 mod p <= 2^21).


__device__ __forceinline__ int32_t signed_rep(uint32_t v, uint32_t p) {
  return v > (p >> 1) ? (int32_t)v - (int32_t)p : (int32_t)v;
}

__device__ __forceinline__ int64_t fold64(int64_t s, uint32_t c32) { return rs_fold64(s, c32); }

// Reduce a folded accumulator (|s| < 2^53) to [0, p) in Montgomery form.
__device__ __forceinline__ uint32_t finish64(int64_t s, const ModP &m) {
  const uint64_t t = (uint64_t)(s + ((int64_t)m.p << 22));  // 0 <= t < 2^54 < p 2^32
  return redc(t, m.p, m.pinv);
}

// y[k] = sum_{j<=k} x[j] b[k-j] for k < n (Montgomery form, reduced).  x and b
// hold signed representatives and are zero for indices in [-RS_G2_PAD, 0)
// and [n, n + RS_G2_PAD).
//
// Outputs come in blocks of R; block bi needs bi + 1 chunks of R inputs.
// Thread t owns the block pair (pi, nblk - 1 - pi), pi = t, t + T, ..., and
// walks both in one loop of nblk + 1 chunks, so every lane of a warp runs
// the same trip count (no divergence in the multiply-accumulate loop).  In
// the loop's first part neighbouring lanes read b and x R words apart (R odd:
// distinct banks); in its second part every lane reads the same b words (a
// broadcast).
__device__ void conv_lazy(const int32_t *x, const int32_t *b, uint32_t *y, int n, const ModP &m) {
  constexpr int R = RS_CONV_R;
  const uint32_t c32 = m.r1;  // 2^32 mod p
  const int nblk = (n + R - 1) / R;
  const int npair = (nblk + 1) / 2;
  for (int pi = threadIdx.x; pi < npair; pi += blockDim.x) {
    const int hb = nblk - 1 - pi;
    const int steps = hb == pi ? pi + 1 : nblk + 1;  // odd count: the middle block once
    int k0 = pi * R, j0 = 0;
    int64_t acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = 0;
#pragma unroll 1
    for (int c = 0; c < steps; ++c) {
      int32_t bw[2 * R - 1], av[R];
      const int base = k0 - j0 - (R - 1);
#pragma unroll
      for (int i = 0; i < 2 * R - 1; ++i) bw[i] = b[base + i];
#pragma unroll
      for (int i = 0; i < R; ++i) av[i] = x[j0 + i];
#pragma unroll
      for (int r = 0; r < R; ++r) {
#pragma unroll
        for (int jj = 0; jj < R; ++jj) acc[r] = rs_mac_s32(acc[r], av[jj], bw[(R - 1) + r - jj]);
        acc[r] = fold64(acc[r], c32);
      }
      j0 += R;
      if (j0 > k0) {  // block complete: write it and move to the mirror block
#pragma unroll
        for (int r = 0; r < R; ++r) {
          if (k0 + r < n) y[k0 + r] = finish64(acc[r], m);
          acc[r] = 0;
        }
        k0 = hb * R;
        j0 = 0;
      }
    }
  }
}

// One block per (pair, prime).  The images come in pairs z+-_i at +-q^i,
// i < M = NI / 2, with R(x) = E(x^2) + x O(x^2):
//   E(Q^i) = (z+_i + z-_i) / 2,  O(Q^i) = (z+_i - z-_i) / (2 q^i),  Q = q^2,
// and with z = num / den both are fractions over D_i = den+ den-, inverted
// together.  E and O (degrees < M) are then interpolated in turn on the
// geometric points Q^i by the two convolutions above, giving the even and
// the odd coefficients of R.  Shared memory: four regions of M words, each
// with RS_G2_PAD zero words on both sides.
__global__ void g2_kernel(G2Args a) {
  extern __shared__ __align__(16) uint32_t sm[];
  __shared__ uint32_t scratch[128];
  const int2 task = a.tasks[blockIdx.x];
  const PairDesc pd = a.pairs[task.x];
  const ModP m = a.mods[task.y];
  const int N = pd.N, NI = pd.NI, M = NI >> 1, D = M - 1, T = blockDim.x, tid = threadIdx.x;
  const int W = M + 2 * RS_G2_PAD;
  int32_t *X = reinterpret_cast<int32_t *>(sm) + RS_G2_PAD;
  int32_t *Bs = X + W;
  uint32_t *Y = reinterpret_cast<uint32_t *>(Bs + W);
  uint32_t *Oh = Y + W;  // O's interpolation input while E is interpolated
  const size_t base = (size_t)pd.img_off + (size_t)task.y * NI;
  const size_t tb = (size_t)task.y * a.tab_stride;
  const uint32_t *finv = a.finv + tb, *gt = a.gtab + tb, *hq = a.hq + tb;
  const int32_t *bt = a.btab + tb;

  uint32_t *dens = reinterpret_cast<uint32_t *>(Bs);
  for (int i = tid; i < M; i += T) dens[i] = mmul(a.den[base + 2 * i], a.den[base + 2 * i + 1], m);
  __syncthreads();
  batch_invert(dens, Y, M, m, scratch);
  __syncthreads();
  for (int i = tid; i < M; i += T) {
    const uint32_t np = a.num[base + 2 * i], dp = a.den[base + 2 * i];
    const uint32_t nm = a.num[base + 2 * i + 1], dm = a.den[base + 2 * i + 1];
    const uint32_t e = mmul(mmul2(np, dm, nm, dp, m), Y[i], m);             // z+ + z-
    const uint32_t o = mmul(mmul2(np, dm, mneg(nm, m.p), dp, m), Y[i], m);  // z+ - z-
    X[i] = signed_rep(mmul(mmul(e, hq[0], m), finv[i], m), m.p);  // (E / F_i); hq[0] = 1/2
    Oh[i] = mmul(mmul(o, hq[i], m), finv[i], m);                   // (O / F_i)
  }
  __syncthreads();
  for (int i = tid; i < M; i += T) Bs[i] = bt[i];
  for (int i = tid; i < RS_G2_PAD; i += T) {
    X[-1 - i] = 0;
    X[M + i] = 0;
    Bs[-1 - i] = 0;
    Bs[M + i] = 0;
  }
  __syncthreads();
  for (int half = 0; half < 2; ++half) {  // E: even coefficients, then O: odd ones
    conv_lazy(X, Bs, Y, M, m);  // Y[k] = Q^{C(k,2)} c_k
    __syncthreads();
    for (int k = tid; k < M; k += T) X[D - k] = signed_rep(mmul(Y[k], gt[k], m), m.p);  // c_k F_k reversed
    __syncthreads();
    conv_lazy(X, Bs, Y, M, m);  // Y[D - t] = sum_s c_{t+s} F_{t+s} b_s
    __syncthreads();
    for (int i = tid; i < M; i += T) {
      const int c = 2 * i + half;
      if (c < N) a.coef[base + c] = from_mont(mmul(Y[D - i], finv[i], m), m);
    }
    if (half == 0) {
      for (int i = tid; i < M; i += T) X[i] = signed_rep(Oh[i], m.p);
      __syncthreads();
    }
  }
}

// Per prime k < K, with q its point base and Q = q^2: for t < stride the
// chirp tables Q^{C(t,2)} (signed representative) and Q^{-C(t,2)} and the
// powers q^t (evaluation in G1), and for t < N the interpolation tables
// 1 / F_t, Q^{-C(t,2)} F_t, the signed (-1)^t Q^{C(t,2)} / F_t,
// F_t = prod_{s=1}^t (Q^s - 1), and 1 / (2 q^t) (G2; finv may be NULL when
// only the chirp tables are wanted).  One thread per prime.
__global__ void tables_kernel(const ModP *mods, const uint32_t *qbase, int K, int N, int stride,
                              uint32_t *finv, uint32_t *gtab, int32_t *btab, uint32_t *hqt, int32_t *qct,
                              uint32_t *qnt, uint32_t *qpt) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  const ModP m = mods[k];
  const uint32_t qb = qbase[k], qbi = minv(qb, m);
  const uint32_t q = mmul(qb, qb, m), qi = minv(q, m);  // Q and 1/Q
  {
    // the chirp tables of the evaluation, base q: q^{C(t,2)}, q^{-C(t,2)}, and q^t
    uint32_t up = m.r1, dn = m.r1, pw = m.r1, piw = m.r1;  // q^{C(t,2)}, q^{-C(t,2)}, q^t, q^{-t}
    int32_t *qc = qct + (size_t)k * stride;
    uint32_t *qn = qnt + (size_t)k * stride;
    uint32_t *qp = qpt + (size_t)k * stride;
    for (int t = 0; t < stride; ++t) {
      qc[t] = signed_rep(up, m.p);
      qn[t] = dn;
      qp[t] = pw;
      up = mmul(up, pw, m);  // C(t+1,2) = C(t,2) + t
      dn = mmul(dn, piw, m);
      pw = mmul(pw, qb, m);
      piw = mmul(piw, qbi, m);
    }
  }
  if (!finv) return;
  uint32_t *fi = finv + (size_t)k * N, *gt = gtab + (size_t)k * N, *hq = hqt + (size_t)k * N;
  int32_t *bt = btab + (size_t)k * N;
  {
    const uint32_t inv2 = minv(madd(m.r1, m.r1, m.p), m);
    uint32_t w = inv2;  // 1 / (2 q^t)
    for (int t = 0; t < N; ++t) {
      hq[t] = w;
      w = mmul(w, qbi, m);
    }
  }
  // forward: F_t (kept in fi for now) and Q^{-C(t,2)} (kept in gt)
  uint32_t F = m.r1, qt = m.r1, qneg = m.r1, qinvt = m.r1;  // Q^t, Q^{-C(t,2)}, Q^{-(t-1)}
  for (int t = 0; t < N; ++t) {
    if (t > 0) {
      qt = mmul(qt, q, m);
      F = mmul(F, msub(qt, m.r1, m.p), m);
      if (t > 1) qinvt = mmul(qinvt, qi, m);
      qneg = mmul(qneg, qinvt, m);
    }
    fi[t] = F;
    gt[t] = qneg;
  }
  // backward: 1 / F_t from 1 / F_{N-1}; Q^{C(t,2)} from Q^{C(N-1,2)}
  uint32_t inv = minv(F, m);
  uint32_t qc = minv(qneg, m);  // Q^{C(N-1,2)}
  uint32_t qm1 = qinvt;         // Q^{-(t-1)} at t = N-1
  for (int t = N - 1; t >= 0; --t) {
    const uint32_t Ft = fi[t];
    fi[t] = inv;
    uint32_t bv = mmul(qc, inv, m);
    if (t & 1) bv = mneg(bv, m.p);
    bt[t] = signed_rep(bv, m.p);
    gt[t] = mmul(gt[t], Ft, m);
    if (t > 0) {
      inv = mmul(inv, msub(qt, m.r1, m.p), m);  // 1/F_{t-1} = (Q^t - 1) / F_t
      qt = mmul(qt, qi, m);
      qc = mmul(qc, qm1, m);                    // Q^{C(t-1,2)} = Q^{C(t,2)} Q^{-(t-1)}
      qm1 = mmul(qm1, q, m);
    }
  }
}

// Per prime: Montgomery constants, V[l] = 2^(32 l) R^2 mod p (limb weights
// for the modular reduction of input coefficients) and the Garner constant
// (p_0 ... p_{k-1})^{-1} mod p_k.
__global__ void init_primes_kernel(const uint32_t *primes, int n, ModP *mods, uint32_t *vtab,
                                   uint32_t *crt, uint32_t *qbase) {
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
  // base of the evaluation points: the smallest q >= 2 whose powers
  // q^1 .. q^RS_MAX_POINTS all differ from 1.  Then the points +-q^i,
  // i < RS_MAX_POINTS / 2, are distinct (q^d = -1 would give q^(2d) = 1 with
  // 2d <= RS_MAX_POINTS) and every Q^t - 1 = q^(2t) - 1, 0 < t <
  // RS_MAX_POINTS / 2, is invertible.
  for (uint32_t c = 2;; ++c) {
    const uint32_t qm = to_mont(c, m);
    uint32_t x = qm;
    int t = 1;
    while (t <= RS_MAX_POINTS && x != m.r1) {
      x = mmul(x, qm, m);
      ++t;
    }
    if (t > RS_MAX_POINTS) {
      qbase[k] = qm;
      break;
    }
  }
}

__global__ void finalize_images_kernel(const ModP *mods, const uint32_t *qbase, const uint32_t *num,
                                       const uint32_t *den, uint32_t *z, uint32_t *points, int K,
                                       int N, int NI) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)K * N) return;
  const int k = (int)(i / N), x = (int)(i % N);
  const ModP m = mods[k];
  const size_t src = (size_t)k * NI + x;
  z[i] = from_mont(mmul(num[src], minv(den[src], m), m), m);
  if (points) {  // image 2 i + s is at (-1)^s q^i
    const uint32_t pw = from_mont(mpow(qbase[k], (uint32_t)(x >> 1), m), m);
    points[i] = (x & 1) ? mneg(pw, m.p) : pw;
  }
}

}  // namespace

cudaError_t launch_tables(const ModP *mods, const uint32_t *qbase, int K, int N, int stride,
                          uint32_t *finv, uint32_t *gtab, int32_t *btab, uint32_t *hq, int32_t *qc,
                          uint32_t *qn, uint32_t *qp, cudaStream_t s) {
  tables_kernel<<<(K + 63) / 64, 64, 0, s>>>(mods, qbase, K, N, stride, finv, gtab, btab, hq, qc, qn, qp);
  return cudaGetLastError();
}

cudaError_t g2_prepare(size_t smem) {
  (void)smem;  // per-kernel attribute: allow the largest any plan may need
  return cudaFuncSetAttribute(g2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              RS_G2_MAX_SMEM_BYTES);
}

cudaError_t launch_g2(int threads, int blocks, size_t smem, const G2Args &a, cudaStream_t s) {
  g2_kernel<<<blocks, threads, smem, s>>>(a);
  return cudaGetLastError();
}


cudaError_t launch_init_primes(const uint32_t *primes, int n, ModP *mods, uint32_t *vtab,
                               uint32_t *crt, uint32_t *qbase, cudaStream_t s) {
  init_primes_kernel<<<(n + 127) / 128, 128, 0, s>>>(primes, n, mods, vtab, crt, qbase);
  return cudaGetLastError();
}

cudaError_t launch_finalize_images(const ModP *mods, const uint32_t *qbase, const uint32_t *num,
                                   const uint32_t *den, uint32_t *z, uint32_t *points, int K, int N,
                                   int NI, cudaStream_t s) {
  const size_t n = (size_t)K * N;
  finalize_images_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(mods, qbase, num, den, z, points,
                                                                      K, N, NI);
  return cudaGetLastError();
}
