// Host-side planning (no device work): see planner.h.
//
// Degree bound (paper, Section 3.1): every term of det S^{(y)} multiplies
// n_y entries of f-rows (x-degree <= m_x) and m_y entries of g-rows
// (x-degree <= n_x), so deg R <= m_x n_y + n_x m_y; the paper also states
// deg R <= m n (total degrees).  D is the smaller of the two.
//
// Coefficient bound: R(x) = det S(x) and |coef_k R| <= max_{|x|=1} |R(x)|.
// On |x| = 1, |f_j(x)| <= ||f_j||_1 (sum of |coefficients|), so by
// Hadamard's inequality on the rows of S,
//   |coef_k R| <= (sum_j ||f_j||_1^2)^{n_y/2} (sum_j ||g_j||_1^2)^{m_y/2}.
// The same row-norm idea is the one the paper uses for its inclusion
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
  for (int i = 0; i < nx; ++i)
    for (int j = 0; j < ny; ++j) {
      const uint32_t *c = f->coeffs + ((size_t)i * ny + j) * L;
      double hi;
      const int t = abs_upper(c, L, &hi);
      if (t < 0) continue;
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
  pi.log2_rownorm2 = lse2(rows);
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
