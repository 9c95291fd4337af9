// Host-side planning (no device work): see planner.h.
//
// Degree bound (paper, Section 3.1): every term of det S^{(y)} multiplies
// n_y entries of f-rows (x-degree <= m_x) and m_y entries of g-rows
// (x-degree <= n_x), so deg R <= m_x n_y + n_x m_y; the paper also states
// deg R <= m n (total degrees).  D is the smaller of the two.
//
// Coefficient bound: R(x) = det S(x) and |coef_k R| <= max_{|x|=1} |R(x)|.
// An f-row of S at x = e^{it} has squared Euclidean norm
//   T_f(t) = sum_j |f_j(e^{it})|^2 = a_0 + 2 sum_{k>=1} a_k cos(k t),
//   a_k = sum_j sum_i f_{j,i} f_{j,i+k}   (the summed autocorrelation),
// so T_f(t) <= a_0 + 2 sum_{k>=1} |a_k| =: H_f, and Hadamard's inequality on
// the rows of S gives
//   |coef_k R| <= H_f^{n_y/2} H_g^{m_y/2}.
// H_f never exceeds sum_j ||f_j||_1^2 (the bound with |f_j(x)| <= ||f_j||_1,
// ||.||_1 the sum of |coefficients|), which is also computed; the smaller
// is used.  Both are the row-norm idea the paper uses for its inclusion
// predicate (Section 3.2).  Logarithms are taken with upward margins.
#include "planner.h"

#include <math.h>
#include <string.h>

#include <algorithm>

namespace {

// Upper bound of |c| for a two's-complement limb integer: returns the top
// limb position t of the magnitude (-1 for c = 0) and sets hi so that
// |c| <= hi * 2^(32 max(t - 1, 0)): the top two limbs plus one unit for
// everything below them (hi <= 2^64 up to the rounding of one double
// addition).  For c < 0 the magnitude ~c + 1 is bounded from the top limbs
// of ~c alone, so no carry chain is taken.
int abs_upper(const uint32_t *c, int L, double *hi) {
  const bool neg = (c[L - 1] >> 31) != 0;
  const uint32_t x = neg ? 0xffffffffu : 0u;  // limbs of ~c are c ^ x
  int t = L - 1;
  while (t >= 0 && (c[t] ^ x) == 0) --t;
  if (t < 0) {
    if (!neg) return -1;  // c = 0
    *hi = 1.0;            // c = -1
    return 0;
  }
  const double top = (double)(c[t] ^ x);
  if (t == 0) {
    *hi = top + 1.0;
    return 0;
  }
  *hi = top * 4294967296.0 + (double)(c[t - 1] ^ x) + 1.0;
  return t;
}

// log2 of sum_t acc[t] 2^(32 max(t - 1, 0)), rounded up
// by the relative error `rel` of the sums that built acc; -INFINITY if empty.
double log2_scaled_sum(const double *acc, int tmax, double rel) {
  double mx = -INFINITY;
  for (int t = 0; t <= tmax; ++t)
    if (acc[t] > 0.0) mx = std::max(mx, log2(acc[t]) + 32.0 * (t > 0 ? t - 1 : 0));
  if (mx == -INFINITY) return -INFINITY;
  double s = 0.0;
  for (int t = 0; t <= tmax; ++t)
    if (acc[t] > 0.0) s += exp2(log2(acc[t]) + 32.0 * (t > 0 ? t - 1 : 0) - mx);
  return mx + log2(s) * (1.0 + 1e-12) + log2(1.0 + rel) + 1e-12;
}

// log2(sum 2^x_i), upper-rounded a little.
double lse2(const std::vector<double> &xs) {
  double mx = -INFINITY;
  for (double x : xs) mx = std::max(mx, x);
  if (mx == -INFINITY) return -INFINITY;
  double s = 0.0;
  for (double x : xs)
    if (x != -INFINITY) s += exp2(x - mx);
  return mx + log2(s) * (1.0 + 1e-12) + 1e-12;
}

// floor(c / 2^S) for a two's-complement limb integer c whose quotient fits
// in an int64 (an arithmetic shift right by S bits).
int64_t shr_floor(const uint32_t *c, int L, int S) {
  const uint32_t ext = (c[L - 1] >> 31) ? 0xffffffffu : 0u;
  const int w = S >> 5, o = S & 31;
  auto limb = [&](int i) { return i < L ? c[i] : ext; };
  const uint64_t u = ((uint64_t)limb(w + 1) << 32) | limb(w);
  const uint64_t r = o ? (u >> o) | ((uint64_t)limb(w + 2) << (64 - o)) : u;
  return (int64_t)r;
}

// log2 of H_f = a_0 + 2 sum_{k>=1} |a_k| (see the top of this file), rounded
// up.  Every coefficient is cut to a = floor(c / 2^S) with |a| <= 2^20 + 1
// (S from the largest magnitude, 2^maxbits), so c = 2^S (a + r), 0 <= r < 1,
// and each product f_{j,i} f_{j,i+k} differs from 2^{2S} a a' by less than
// 2^{2S} (|a| + |a'| + 1); summed over the products of a_k (weight 2 for
// k >= 1) that is at most 2^{2S} sum_j 2 n_j (2 s_j + n_j) with s_j =
// sum_i |a_{j,i}| and n_j the entries of row j.  Everything up to the final
// logarithm is exact integer arithmetic: products below 2^42, row sums of at
// most 2^14 of them in int64, sums over rows in 128 bits.
double log2_autocorr_bound(const rs_bipoly *f, const std::vector<int> &dx, int maxbits) {
  const int L = f->limbs, ny = f->deg_y + 1, my = (int)dx.size() - 1;
  const int S = std::max(0, maxbits - 20);
  std::vector<int> len(my + 1, 0);  // row j holds f_{j,0..dx_j}
  double work = 0.0;
  int nmax = 0;
  for (int j = 0; j <= my; ++j) {
    len[j] = dx[j] + 1;
    nmax = std::max(nmax, len[j]);
    work += 0.5 * len[j] * len[j];
  }
  // long rows: keep the l1 bound (planning stays near linear in the input)
  if (work > 0x1p27 || nmax > (1 << 14)) return INFINITY;
  // rows padded with at least 4 zeros, so the products run in whole groups of 4
  const int stride = ((nmax + 3) & ~3) + 4;
  std::vector<int32_t> a((size_t)(my + 1) * stride, 0);
  for (int i = 0; i < nmax; ++i)
    for (int j = 0; j <= my; ++j)
      if (i < len[j]) a[(size_t)j * stride + i] = (int32_t)shr_floor(f->coeffs + ((size_t)i * ny + j) * L, L, S);
  std::vector<__int128> ac(nmax, 0);
  __int128 trunc = 0;
  for (int j = 0; j <= my; ++j) {
    const int n = len[j];
    if (n == 0) continue;
    const int32_t *r = &a[(size_t)j * stride];
    int64_t s1 = 0;
    for (int i = 0; i < n; ++i) s1 += r[i] < 0 ? -(int64_t)r[i] : (int64_t)r[i];
    if (S > 0) trunc += (__int128)(2 * (int64_t)n) * (2 * s1 + n);
    for (int k = 0; k < n; ++k) {
      const int m = n - k;  // terms i < m; r[i + k] = 0 for i >= m (padding)
      int64_t u0 = 0, u1 = 0, u2 = 0, u3 = 0;  // four independent chains
      for (int i = 0; i < m; i += 4) {
        u0 += (int64_t)r[i] * r[i + k];
        u1 += (int64_t)r[i + 1] * r[i + 1 + k];
        u2 += (int64_t)r[i + 2] * r[i + 2 + k];
        u3 += (int64_t)r[i + 3] * r[i + 3 + k];
      }
      ac[k] += (__int128)u0 + u1 + u2 + u3;
    }
  }
  __int128 h = ac[0] + trunc;
  for (int k = 1; k < nmax; ++k) h += 2 * (ac[k] < 0 ? -ac[k] : ac[k]);
  if (h <= 0) return -INFINITY;
  // (double) h errs by at most 2^-53 relative: inside the margins below
  return 2.0 * S + log2((double)h) * (1.0 + 1e-12) + 1e-12;
}

int analyze(const rs_bipoly *f, PolyInfo &pi, const char **why) {
  if (!f || !f->coeffs) {
    *why = "NULL polynomial or coefficient pointer";
    return RS_ERR_ARG;
  }
  if (f->deg_x < 0 || f->deg_y < 0) {
    *why = "negative array extent";
    return RS_ERR_ARG;
  }
  if (f->limbs < 1 || f->limbs > RS_MAX_LIMBS) {
    *why = "limbs must be in 1..RS_MAX_LIMBS (128)";
    return RS_ERR_ARG;
  }
  if ((int64_t)(f->deg_x + 1) * (f->deg_y + 1) > ((int64_t)1 << 26)) {
    *why = "input array too large";
    return RS_ERR_LIMIT;
  }
  const int L = f->limbs, nx = f->deg_x + 1, ny = f->deg_y + 1;
  pi = PolyInfo();
  pi.L = L;
  pi.stride = ny;
  std::vector<int> dx(ny, -1);
  // ||f_j||_1 per row j, kept as sums of hi by limb position (hi < 2^64 + 1,
  // at most 2^26 terms: the sums stay far below the double range).
  std::vector<double> acc((size_t)ny * (RS_MAX_LIMBS + 1), 0.0);
  std::vector<int> tmax(ny, -1);
  int maxbits = 0;  // |c| <= 2^maxbits for every coefficient
  for (int i = 0; i < nx; ++i)
    for (int j = 0; j < ny; ++j) {
      const uint32_t *c = f->coeffs + ((size_t)i * ny + j) * L;
      double hi;
      const int t = abs_upper(c, L, &hi);
      if (t < 0) continue;
      int e;  // hi < 2^e (hi >= 1)
      frexp(hi, &e);
      maxbits = std::max(maxbits, 32 * (t > 0 ? t - 1 : 0) + e);
      dx[j] = i;
      pi.mx = std::max(pi.mx, i);
      pi.tdeg = std::max(pi.tdeg, i + j);
      pi.my = std::max(pi.my, j);
      acc[(size_t)j * (RS_MAX_LIMBS + 1) + t] += hi;
      tmax[j] = std::max(tmax[j], t);
    }
  pi.zero = pi.my < 0;
  if (pi.zero) return RS_OK;
  pi.dx.assign(dx.begin(), dx.begin() + pi.my + 1);
  // Each double operation errs by at most 2^-53 relative; a row sum of n
  // terms by at most n 2^-53 (plus the conversions), taken as (n + 4) 2^-52.
  const double rel = ((double)nx + 4.0) * 0x1p-52;
  std::vector<double> rows;
  for (int j = 0; j <= pi.my; ++j) {
    pi.nc += pi.dx[j] + 1;
    if (tmax[j] >= 0) rows.push_back(2.0 * log2_scaled_sum(&acc[(size_t)j * (RS_MAX_LIMBS + 1)], tmax[j], rel));
  }
  pi.log2_rownorm2 = std::min(lse2(rows), log2_autocorr_bound(f, pi.dx, maxbits));
  return RS_OK;
}

}  // namespace

int rs_plan_pair(const rs_bipoly *f, const rs_bipoly *g, const std::vector<double> &log2p,
                 PairPlan &plan, const char **why) {
  static const char *none = "";
  *why = none;
  plan = PairPlan();
  int rc = analyze(f, plan.f, why);
  if (rc == RS_OK) rc = analyze(g, plan.g, why);
  if (rc != RS_OK) return plan.status = rc;
  if (plan.f.zero || plan.g.zero) {
    plan.trivial_zero = true;
    plan.D = -1;
    plan.Lout = 1;
    return RS_OK;
  }
  const int my = plan.f.my, ny = plan.g.my;
  if (my > RS_MAX_DEG_Y || ny > RS_MAX_DEG_Y) {
    *why = "y-degree above RS_MAX_DEG_Y";
    return plan.status = RS_ERR_LIMIT;
  }
  const int64_t d1 = (int64_t)plan.f.mx * ny + (int64_t)plan.g.mx * my;
  const int64_t d2 = (int64_t)plan.f.tdeg * plan.g.tdeg;
  const int64_t D = std::min(d1, d2);
  if (D + 1 > RS_MAX_POINTS) {
    *why = "degree bound above RS_MAX_POINTS - 1";
    return plan.status = RS_ERR_LIMIT;
  }
  plan.D = (int)D;
  plan.N = (int)D + 1;
  const double B = 0.5 * ny * plan.f.log2_rownorm2 + 0.5 * my * plan.g.log2_rownorm2;
  plan.bits = (int)ceil(B * (1.0 + 1e-12) + 1e-6) + 1;
  if (plan.bits < 1) plan.bits = 1;
  const double need = plan.bits + 1 + 1e-6;  // product of primes > 2^(bits+1)
  if (log2p.empty()) {
    plan.K = (int)ceil(need / 30.9992);
  } else {
    double acc = 0.0;
    int k = 0;
    while (k < (int)log2p.size() && acc < need) acc += log2p[k++];
    if (acc < need) {
      *why = "coefficient bound needs more primes than RS_MAX_PRIMES";
      return plan.status = RS_ERR_LIMIT;
    }
    plan.K = k;
  }
  if (plan.K > RS_MAX_PRIMES) {
    *why = "coefficient bound needs more primes than RS_MAX_PRIMES";
    return plan.status = RS_ERR_LIMIT;
  }
  plan.Lout = (plan.bits + 31) / 32;
  plan.cap = std::max(my, ny) + 1;
  plan.staged = rs_g1_staged_words(plan, ((plan.cap + 7) / 8) * 8, 128);
  if (plan.staged > 48 * 1024) {  // RS_G1_MAX_STAGED_WORDS
    *why = "too many coefficients to stage in shared memory";
    return plan.status = RS_ERR_LIMIT;
  }
  return RS_OK;
}

std::vector<uint32_t> rs_prime_table(int count) {
  const uint64_t hi = (uint64_t)1 << 31, lo = hi - ((uint64_t)1 << 20);
  const int lim = 46341;  // > sqrt(2^31)
  std::vector<char> small(lim + 1, 1);
  std::vector<uint32_t> base;
  for (int i = 2; i <= lim; ++i) {
    if (!small[i]) continue;
    base.push_back(i);
    for (int64_t k = (int64_t)i * i; k <= lim; k += i) small[k] = 0;
  }
  std::vector<char> comp(hi - lo, 0);
  for (uint32_t q : base) {
    uint64_t s = ((lo + q - 1) / q) * q;
    for (uint64_t v = s; v < hi; v += q) comp[v - lo] = 1;
  }
  std::vector<uint32_t> out;
  for (uint64_t v = hi - 1; v >= lo && (int)out.size() < count; --v)
    if (!comp[v - lo]) out.push_back((uint32_t)v);
  return out;
}
