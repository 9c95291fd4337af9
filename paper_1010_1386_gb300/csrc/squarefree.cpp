// Square-free factorisation of R^{(y)} = res(f, g, y) (the paper's solver
// computes R^{(y)} together with its square-free factorisation, Section 5,
// PROJECT): R = c prod_i R_i^i with R_i primitive, square-free, pairwise
// coprime, leading coefficient > 0.
//
// One batch computes R over K primes chosen for the factors' bound (below),
// and Yun's algorithm mod every prime after G2 (kernels_yun.cu).  A prime is
// used if R keeps its degree mod p and the square-free part mod p has the
// largest degree seen (a smaller one means p divides a discriminant and
// merged factors).  Every R_i divides R in Z[x], so by the Landau-Mignotte
// bound (M. Mignotte, "An inequality about factors of polynomials", Math.
// Comp. 28, 1974: with R = R_i G, M(R_i) = M(R) / M(G) <= M(R) |lc R_i| /
// |lc R| since M(G) >= |lc G|, and ||h||_1 <= 2^{deg h} M(h), M(R) <=
// ||R||_2)  ||R_i||_1 <= 2^{deg R_i} |lc R_i / lc R| ||R||_2.  So
// H_i = lc(R) R_i / lc(R_i), the integer polynomial the residues
// lc(R) monic(R_i mod p) lift to, has ||H_i||_1 <= 2^{deg R_i} ||R||_2
// <= 2^{B + D + log2(D + 1) / 2}, B the resultant's coefficient bits and D its
// degree bound.  The H_i are lifted by the CRT kernels over the first K_H
// primes, then R_i = H_i / content(H_i) on the host (long division and
// Lehmer's gcd), and c = lc(R) / prod_i lc(R_i)^i (an exact division, since
// lc R = c prod_i lc(R_i)^i; the gcd of R's coefficients if it is not).
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <functional>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "engine.h"

namespace {

// ------------------------------------------------------------ big integers
// Magnitudes as little-endian 32-bit limbs without leading zeros (empty = 0).
using Big = std::vector<uint32_t>;

void trim(Big &a) {
  while (!a.empty() && a.back() == 0u) a.pop_back();
}

// Two's-complement limbs -> (magnitude, sign).
Big from_twos(const uint32_t *c, int L, bool *neg) {
  Big m(c, c + L);
  *neg = (c[L - 1] >> 31) != 0;
  if (*neg) {
    uint64_t carry = 1;
    for (uint32_t &v : m) {
      const uint64_t t = (uint64_t)(uint32_t)~v + carry;
      v = (uint32_t)t;
      carry = t >> 32;
    }
  }
  trim(m);
  return m;
}

// (magnitude, sign) -> two's complement in L limbs (the caller made room).
void to_twos(const Big &m, bool neg, uint32_t *out, int L) {
  for (int l = 0; l < L; ++l) out[l] = l < (int)m.size() ? m[l] : 0u;
  if (neg) {
    uint64_t carry = 1;
    for (int l = 0; l < L; ++l) {
      const uint64_t t = (uint64_t)(uint32_t)~out[l] + carry;
      out[l] = (uint32_t)t;
      carry = t >> 32;
    }
  }
}

// Limbs needed for the two's-complement form of +-m.
int twos_limbs(const Big &m, bool neg) {
  if (m.empty()) return 1;
  int L = (int)m.size();
  const uint32_t top = m.back();
  if (top >> 31) {  // needs a sign limb unless it is exactly -2^(32 L - 1)
    bool pow2 = top == 0x80000000u;
    for (int l = 0; l + 1 < L && pow2; ++l) pow2 = m[l] == 0u;
    if (!(neg && pow2)) ++L;
  }
  return L;
}

int cmp(const Big &a, const Big &b) {
  if (a.size() != b.size()) return a.size() < b.size() ? -1 : 1;
  for (size_t i = a.size(); i-- > 0;)
    if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
  return 0;
}

void sub_in_place(Big &a, const Big &b) {  // a >= b
  int64_t borrow = 0;
  for (size_t i = 0; i < a.size(); ++i) {
    int64_t t = (int64_t)a[i] - (i < b.size() ? (int64_t)b[i] : 0) - borrow;
    borrow = t < 0;
    a[i] = (uint32_t)(t + (borrow << 32));
  }
  trim(a);
}

int ctz(const Big &a) {
  for (size_t i = 0; i < a.size(); ++i)
    if (a[i]) return (int)(32 * i) + __builtin_ctz(a[i]);
  return 0;
}

void shr_in_place(Big &a, int bits) {
  const size_t w = (size_t)bits / 32;
  const int r = bits % 32;
  if (w >= a.size()) {
    a.clear();
    return;
  }
  a.erase(a.begin(), a.begin() + w);
  if (r) {
    for (size_t i = 0; i < a.size(); ++i) a[i] = (a[i] >> r) | (i + 1 < a.size() ? a[i + 1] << (32 - r) : 0u);
  }
  trim(a);
}

void shl_in_place(Big &a, int bits) {
  if (a.empty()) return;
  const size_t w = (size_t)bits / 32;
  const int r = bits % 32;
  a.insert(a.begin(), w, 0u);
  if (r) {
    a.push_back(0u);
    for (size_t i = a.size(); i-- > w + 1;) a[i] = (a[i] << r) | (a[i - 1] >> (32 - r));
    a[w] <<= r;
  }
  trim(a);
}

uint32_t mod_small(const Big &a, uint32_t m) {
  uint64_t r = 0;
  for (size_t i = a.size(); i-- > 0;) r = ((r << 32) | a[i]) % m;
  return (uint32_t)r;
}

uint32_t gcd32(uint32_t a, uint32_t b) {
  while (b) {
    const uint32_t t = a % b;
    a = b;
    b = t;
  }
  return a;
}

// Binary gcd (Stein) of magnitudes; a one-limb operand takes a remainder first.
Big big_gcd(Big a, Big b) {
  if (a.empty()) return b;
  if (b.empty()) return a;
  if (a.size() == 1 || b.size() == 1) {
    const uint32_t s = a.size() == 1 ? a[0] : b[0];
    const Big &o = a.size() == 1 ? b : a;
    const uint32_t g = gcd32(s, mod_small(o, s));
    return Big{g};
  }
  const int za = ctz(a), zb = ctz(b), z = std::min(za, zb);
  shr_in_place(a, za);
  shr_in_place(b, zb);
  while (true) {  // both odd
    if (cmp(a, b) < 0) std::swap(a, b);
    sub_in_place(a, b);
    if (a.empty()) break;
    shr_in_place(a, ctz(a));
    if (b.size() == 1) {
      const uint32_t g = gcd32(b[0], mod_small(a, b[0]));
      b = Big{g};
      break;
    }
  }
  shl_in_place(b, z);
  return b;
}

// a * b of magnitudes (schoolbook, 64-bit column sums).
Big big_mul(const Big &a, const Big &b) {
  if (a.empty() || b.empty()) return Big();
  Big r(a.size() + b.size(), 0u);
  for (size_t i = 0; i < a.size(); ++i) {
    uint64_t carry = 0;
    for (size_t j = 0; j < b.size(); ++j) {
      const uint64_t t = (uint64_t)a[i] * b[j] + r[i + j] + carry;
      r[i + j] = (uint32_t)t;
      carry = t >> 32;
    }
    r[i + b.size()] = (uint32_t)carry;
  }
  trim(r);
  return r;
}

// Quotient and remainder of magnitudes, b non-zero (D. E. Knuth, The Art of
// Computer Programming vol. 2, 4.3.1, Algorithm D), on 64-bit limbs with
// 128-bit products: normalise b's top limb, estimate each quotient limb from
// the top two limbs, multiply and subtract, add back when the estimate was one
// too large.
using u64 = uint64_t;
using u128 = unsigned __int128;

std::vector<u64> pack64(const Big &a, size_t extra = 0) {
  std::vector<u64> r((a.size() + 1) / 2 + extra, 0u);
  for (size_t i = 0; i < a.size(); ++i) r[i / 2] |= (u64)a[i] << (32 * (i & 1));
  return r;
}

Big unpack32(const u64 *r, size_t n) {
  Big a(2 * n);
  for (size_t i = 0; i < n; ++i) {
    a[2 * i] = (uint32_t)r[i];
    a[2 * i + 1] = (uint32_t)(r[i] >> 32);
  }
  trim(a);
  return a;
}

Big big_divmod(const Big &a, const Big &b, Big *rem) {
  if (cmp(a, b) < 0) {
    *rem = a;
    return Big();
  }
  if (b.size() == 1) {
    Big q(a.size());
    uint64_t r = 0;
    for (size_t i = a.size(); i-- > 0;) {
      const uint64_t cur = (r << 32) | a[i];
      q[i] = (uint32_t)(cur / b[0]);
      r = cur % b[0];
    }
    trim(q);
    *rem = r ? Big{(uint32_t)r} : Big();
    return q;
  }
  std::vector<u64> v = pack64(b), u = pack64(a, 1);
  while (!v.empty() && v.back() == 0u) v.pop_back();
  const size_t n = v.size();
  size_t ua = u.size() - 1;  // limbs of a
  while (ua > 0 && u[ua - 1] == 0u) --ua;
  u.resize(ua + 1);
  u[ua] = 0u;
  if (n == 1) {  // one 64-bit limb: schoolbook with 128-bit steps
    std::vector<u64> q(ua, 0u);
    u128 r = 0;
    for (size_t i = ua; i-- > 0;) {
      const u128 cur = (r << 64) | u[i];
      q[i] = (u64)(cur / v[0]);
      r = cur % v[0];
    }
    const u64 rr = (u64)r;
    *rem = unpack32(&rr, 1);
    return unpack32(q.data(), q.size());
  }
  const size_t m = ua - n;
  const int s = __builtin_clzll(v.back());
  if (s) {
    for (size_t i = n; i-- > 1;) v[i] = (v[i] << s) | (v[i - 1] >> (64 - s));
    v[0] <<= s;
    u[ua] = u[ua - 1] >> (64 - s);
    for (size_t i = ua; i-- > 1;) u[i] = (u[i] << s) | (u[i - 1] >> (64 - s));
    u[0] <<= s;
  }
  std::vector<u64> q(m + 1, 0u);
  const u64 vt = v[n - 1], vs = v[n - 2];
  for (size_t j = m + 1; j-- > 0;) {
    const u128 num = ((u128)u[j + n] << 64) | u[j + n - 1];
    u128 qh = num / vt, rh = num % vt;
    while ((qh >> 64) != 0 || qh * vs > ((rh << 64) | u[j + n - 2])) {
      --qh;
      rh += vt;
      if ((rh >> 64) != 0) break;
    }
    const u64 q64 = (u64)qh;
    u64 carry = 0, borrow = 0;
    for (size_t i = 0; i < n; ++i) {
      const u128 pr = (u128)q64 * v[i] + carry;
      carry = (u64)(pr >> 64);
      const u64 lo = (u64)pr, x = u[i + j];
      const u64 t = x - lo;
      const u64 b1 = x < lo;
      u[i + j] = t - borrow;
      borrow = b1 + (t < borrow);
    }
    const u128 top = (u128)carry + borrow;
    const bool neg = (u128)u[j + n] < top;
    u[j + n] = (u64)((u128)u[j + n] - top);
    if (neg) {  // the estimate was one too large: add b back
      q[j] = q64 - 1;
      u64 c = 0;
      for (size_t i = 0; i < n; ++i) {
        const u128 sm = (u128)u[i + j] + v[i] + c;
        u[i + j] = (u64)sm;
        c = (u64)(sm >> 64);
      }
      u[j + n] += c;
    } else {
      q[j] = q64;
    }
  }
  std::vector<u64> r(n);
  for (size_t i = 0; i < n; ++i) r[i] = s ? (u[i] >> s) | (u[i + 1] << (64 - s)) : u[i];
  *rem = unpack32(r.data(), n);
  return unpack32(q.data(), q.size());
}

int bitlen(const Big &a) { return a.empty() ? 0 : 32 * ((int)a.size() - 1) + (32 - __builtin_clz(a.back())); }

// Bits [sh, sh + 62) of a (a < 2^(sh + 62)).
u64 top_bits(const Big &a, int sh) {
  const int w = sh / 32, o = sh % 32;
  u128 r = 0;
  for (int k = 3; k >= 0; --k) {
    const size_t i = (size_t)(w + k);
    r = (r << 32) | (i < a.size() ? a[i] : 0u);
  }
  return (u64)(r >> o);
}

// X a + Y b for signed single-word cofactors with X a + Y b >= 0.
Big lin_comb(const Big &a, __int128 X, const Big &b, __int128 Y) {
  const size_t n = std::max(a.size(), b.size()) + 3;
  Big r(n);
  __int128 carry = 0;
  for (size_t i = 0; i < n; ++i) {
    __int128 t = carry;
    if (i < a.size()) t += X * (__int128)a[i];
    if (i < b.size()) t += Y * (__int128)b[i];
    r[i] = (uint32_t)((u128)t & 0xffffffffu);
    carry = t >> 32;  // arithmetic shift (floor division by 2^32)
  }
  trim(r);
  return r;
}

// gcd of magnitudes by Lehmer's method (D. H. Lehmer, "Euclid's algorithm
// for large numbers", Amer. Math. Monthly 45, 1938; Knuth 4.5.2, Algorithm
// L): the leading 62 bits of a and b drive single-precision Euclid steps for
// as long as the quotients are certain (the quotients from (a' + A)/(b' + C)
// and (a' + B)/(b' + D) agree); the accumulated 2x2 matrix is then applied
// to the full numbers at once.  A full division step when no single-precision
// step was certain.
Big big_gcd_lehmer(Big a, Big b) {
  if (cmp(a, b) < 0) std::swap(a, b);
  while (b.size() > 2) {
    const int sh = std::max(0, bitlen(a) - 62);
    __int128 ah = (__int128)top_bits(a, sh), bh = (__int128)top_bits(b, sh);
    __int128 A = 1, B = 0, C = 0, D = 1;
    while (bh + C != 0 && bh + D != 0) {
      const __int128 q1 = (ah + A) / (bh + C), q2 = (ah + B) / (bh + D);
      if (q1 != q2) break;
      __int128 t = A - q1 * C;
      A = C;
      C = t;
      t = B - q1 * D;
      B = D;
      D = t;
      t = ah - q1 * bh;
      ah = bh;
      bh = t;
    }
    if (B == 0) {
      Big r;
      big_divmod(a, b, &r);
      a = std::move(b);
      b = std::move(r);
      continue;
    }
    // a' = A a + B b, b' = C a + D b (both non-negative)
    Big na = lin_comb(a, A, b, B), nb = lin_comb(a, C, b, D);
    a = std::move(na);
    b = std::move(nb);
    if (cmp(a, b) < 0) std::swap(a, b);
  }
  if (b.empty()) return a;
  Big r;  // b has at most two limbs: one division, then the binary gcd
  big_divmod(a, b, &r);
  return big_gcd(b, r);
}

// Content of the integers c[0..n) (magnitudes, c[n-1] non-zero) and, when
// quot is given, every c[j] divided by it.  Starts from |c[n-1]| and takes a
// gcd only when a division leaves a remainder (then the quotients so far are
// recomputed), so a content that is found early costs one long division per
// coefficient.
Big content_of(const std::vector<Big> &c, std::vector<Big> *quot) {
  Big g = c.back();
  if (quot) quot->assign(c.size(), Big());
  for (size_t j = 0; j < c.size(); ++j) {
    if (g.size() == 1 && g[0] == 1u) {
      if (!quot) return g;
      for (size_t k = j; k < c.size(); ++k) (*quot)[k] = c[k];
      return g;
    }
    if (c[j].empty()) continue;
    Big r;
    Big q = big_divmod(c[j], g, &r);
    if (!r.empty()) {
      g = big_gcd_lehmer(g, r);
      if (quot)
        for (size_t k = 0; k < j; ++k) {  // the earlier quotients were by a multiple of g
          Big r2;
          (*quot)[k] = big_divmod(c[k], g, &r2);
        }
      q = big_divmod(c[j], g, &r);
    }
    if (quot) (*quot)[j] = std::move(q);
  }
  return g;
}

}  // namespace

extern "C" int rs_squarefree_batch(rs_ctx *ctx, int32_t n, const rs_bipoly *f, const rs_bipoly *g,
                                   int32_t max_mult, rs_upoly *content, rs_upoly *factors, int32_t *nmult,
                                   int32_t *status) {
  if (!ctx || n < 0 || max_mult < 1 || (n > 0 && (!f || !g || !content || !factors || !nmult)))
    return rs_fail(ctx, RS_ERR_ARG, "NULL argument, negative n or max_mult < 1");
  if (n == 0) return RS_OK;
  const auto t_start = std::chrono::steady_clock::now();
  rs_sqf_info info;
  memset(&info, 0, sizeof(info));
  std::vector<PairPlan> plans;
  int first = RS_OK;
  rs_plan_all(ctx, n, f, g, plans, nullptr, &first);
  std::vector<int> st(n, RS_OK);
  std::vector<std::string> why(n);
  std::vector<int> KH(n, 0), bitsH(n, 0);
  int valid = 0;
  for (int i = 0; i < n; ++i) {
    PairPlan &p = plans[i];
    st[i] = p.status;
    if (st[i] != RS_OK) {
      why[i] = "rejected by the planner";
      continue;
    }
    if (p.trivial_zero) {
      st[i] = RS_ERR_ARG;
      why[i] = "R = 0 has no square-free factorisation";
      p.status = RS_ERR_ARG;
      continue;
    }
    // primes for the factors: coefficients of H_i below 2^bitsH (|coef R| < 2^bits,
    // so ||R||_2 < 2^{bits + log2(D + 1) / 2}; one bit of margin)
    bitsH[i] = p.bits + p.D + (int)std::ceil(0.5 * std::log2((double)p.D + 1.0)) + 1;
    double acc = 0.0;
    while (KH[i] < (int)ctx->log2p.size() && acc < bitsH[i] + 2) acc += ctx->log2p[KH[i]++];
    if (acc < bitsH[i] + 2) {
      st[i] = RS_ERR_LIMIT;
      why[i] = "factor bound needs more primes than RS_MAX_PRIMES";
      p.status = RS_ERR_LIMIT;
      continue;
    }
    p.Kcrt = p.K;  // R itself needs only its own primes
    p.K = std::min((int)ctx->log2p.size(), std::max(p.K, KH[i]) + 4);  // a few spare primes
    ++valid;
  }
  const int M = max_mult;
  std::vector<int> K(n, 0);
  for (int i = 0; i < n; ++i) K[i] = plans[i].K;
  rs_batch *b = nullptr;
  std::vector<uint32_t> hdr;  // per Yun task: deg R mod p, overflow flag, d_1 .. d_M
  const int hw = 2 + M;
  if (valid) {
    RsBatchOpts o;
    o.use_graph = false;
    o.persistent = ctx->cfg.persistent != 0;
    o.fork = true;
    o.yun_maxm = M;
    o.timing = true;
    // the batch of the previous call is reused when every pair has the same shape
    rs_batch *cb = ctx->sqf_cache;
    bool reuse = cb && cb->n == n && cb->opt.yun_maxm == M;
    for (int i = 0; reuse && i < n; ++i) reuse = rs_same_shape(plans[i], cb->plans[i]);
    int rc = RS_OK;
    if (reuse) {
      b = cb;
    } else {
      if (cb) rs_free_batch(cb);
      ctx->sqf_cache = nullptr;
      rc = rs_build_batch(ctx, n, f, g, std::move(plans), o, &b);
      if (rc != RS_OK) return rc;
      ctx->sqf_cache = b;
    }
    DevGuard dg(ctx->device);
    rc = rs_upload(b, f, g);
    if (rc == RS_OK) rc = rs_run(b);
    if (rc == RS_OK) rc = rs_fetch_async(b);
    hdr.resize((size_t)b->nyun * hw);
    info.h2d_bytes += b->in_words * 4;
    info.d2h_bytes += b->out_words * 4 + (int64_t)b->nyun * hw * 4;
    if (rc == RS_OK && b->nyun) {
      cudaError_t e = cudaMemcpy2DAsync(hdr.data(), hw * 4, b->d_yun_out, (size_t)b->yun_ostride * 4, hw * 4,
                                        b->nyun, cudaMemcpyDeviceToHost, b->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
      if (e != cudaSuccess) rc = rs_fail(ctx, RS_ERR_CUDA, std::string("square-free: ") + cudaGetErrorString(e));
    }
    if (rc == RS_OK) rc = rs_batch_info_get(b, &info.batch);
    if (rc != RS_OK) {
      rs_free_batch(b);
      ctx->sqf_cache = nullptr;
      return rc;
    }
    info.yun_tasks = b->nyun;
  }
  const auto t_host0 = std::chrono::steady_clock::now();
  auto put = [&](rs_upoly &out, const std::vector<Big> &mag, const std::vector<char> &neg) -> int {
    int L = 1;
    for (size_t j = 0; j < mag.size(); ++j) L = std::max(L, twos_limbs(mag[j], neg[j] != 0));
    const int deg = (int)mag.size() - 1;
    out.deg = deg;
    out.limbs = L;
    if ((int64_t)(deg + 1) * L > out.capacity_words || (!out.coeffs && deg >= 0)) return RS_ERR_CAPACITY;
    for (int j = 0; j <= deg; ++j) to_twos(mag[j], neg[j] != 0, out.coeffs + (size_t)j * L, L);
    return RS_OK;
  };
  const std::vector<Big> one_m{Big{1u}};
  const std::vector<char> one_s{0};
  // Per pair, on host threads: R, the usable primes and the pattern of
  // factor degrees (R's content is taken later, while the GPU lifts the
  // factors).
  struct PairRes {
    int degR = -1, LR = 1;
    std::vector<uint32_t> Rw;  // R's limbs until its content is taken
    Big lcR;                   // |lc R|
    Big content;
    bool lc_neg = false;
    std::vector<int> pattern;
  };
  std::vector<PairRes> pr(n);
  std::vector<int64_t> t0v(n, 0);
  {
    int64_t task0 = 0;
    for (int i = 0; i < n; ++i)
      if (st[i] == RS_OK) {
        t0v[i] = task0;
        task0 += K[i];
      }
  }
  auto analyse = [&](int i) {
    PairRes &q = pr[i];
    st[i] = rs_unpack_one(b, i, q.Rw, &q.degR, &q.LR);
    if (st[i] != RS_OK) {
      why[i] = "resultant failed";
      return;
    }
    if (q.degR < 0) {
      st[i] = RS_ERR_ARG;
      why[i] = "R = 0 has no square-free factorisation";
      return;
    }
    q.lc_neg = (q.Rw[(size_t)q.degR * q.LR + q.LR - 1] >> 31) != 0;
    {
      bool ng;
      q.lcR = from_twos(&q.Rw[(size_t)q.degR * q.LR], q.LR, &ng);
    }
    if (q.degR == 0) return;
    // usable primes: R keeps its degree mod p, square-free part of largest degree
    auto task = [&](int k) { return &hdr[(size_t)(t0v[i] + k) * hw]; };
    int best_sf = -1;
    for (int k = 0; k < K[i]; ++k) {
      const uint32_t *t = task(k);
      if ((int)t[0] != q.degR || t[1]) continue;
      int sf = 0;
      for (int m = 0; m < M; ++m) sf += (int)t[2 + m];
      best_sf = std::max(best_sf, sf);
    }
    bool over = false;
    for (int k = 0; k < KH[i]; ++k) over = over || ((int)task(k)[0] == q.degR && task(k)[1]);
    if (over) {  // Yun ran past max_mult on a prime that keeps deg R
      st[i] = RS_ERR_CAPACITY;
      why[i] = "a factor's multiplicity exceeds max_mult";
      return;
    }
    q.pattern.assign(M, 0);
    int good = 0;  // length of the prefix of usable primes with the same pattern
    for (int k = 0; k < K[i]; ++k) {
      const uint32_t *t = task(k);
      if ((int)t[0] != q.degR || t[1]) break;
      int sf = 0;
      for (int m = 0; m < M; ++m) sf += (int)t[2 + m];
      if (sf != best_sf) break;
      if (k == 0)
        for (int m = 0; m < M; ++m) q.pattern[m] = (int)t[2 + m];
      bool same = true;
      for (int m = 0; m < M; ++m) same = same && (int)t[2 + m] == q.pattern[m];
      if (!same) break;
      ++good;
    }
    if (good < KH[i]) {
      st[i] = RS_ERR_LIMIT;
      why[i] = "an unlucky prime for the square-free factorisation lies among the first " + std::to_string(KH[i]) +
               " primes (prime index " + std::to_string(good) + ")";
    }
  };
  auto parallel_for = [](int count, const std::function<void(int)> &fn) {
    const int nt = std::max(1, std::min({count, 16, (int)std::thread::hardware_concurrency()}));
    if (nt <= 1) {
      for (int i = 0; i < count; ++i) fn(i);
      return;
    }
    std::atomic<int> next{0};
    std::vector<std::thread> th;
    for (int t = 0; t < nt; ++t)
      th.emplace_back([&] {
        for (int i = next++; i < count; i = next++) fn(i);
      });
    for (auto &x : th) x.join();
  };
  {
    std::vector<int> todo;
    for (int i = 0; i < n; ++i)
      if (st[i] == RS_OK) todo.push_back(i);
    const auto ta = std::chrono::steady_clock::now();
    parallel_for((int)todo.size(), [&](int t) { analyse(todo[t]); });
    info.ms_analyse = (float)std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - ta).count();
  }
  // Outputs that are known now, and the factors to lift.
  struct Lift {
    int pair, mult;
    PairDesc pd;
  };
  std::vector<Lift> lifts;
  int64_t xl = 0, cy = 0, outw = 0;
  int kmax = 0;
  std::vector<int> out_rc(n, RS_OK);
  for (int i = 0; i < n; ++i) {
    if (st[i] != RS_OK) continue;
    const PairRes &q = pr[i];
    for (int m = 0; m < M; ++m) {  // R_i = 1 unless set below
      const int r2 = put(factors[(size_t)i * M + m], one_m, one_s);
      if (out_rc[i] == RS_OK) out_rc[i] = r2;
    }
    nmult[i] = 0;
    if (q.degR == 0) continue;
    // H_m = lc(R) R_m / lc(R_m) over the first KH primes, read in place from
    // the Yun output (stride one task per prime)
    const int LH = (bitsH[i] + 1 + 31) / 32;
    int64_t off = t0v[i] * b->yun_ostride + 2 + M;
    for (int m = 0; m < M; ++m) {
      const int d = q.pattern[m];
      if (d > 0) {
        Lift lf;
        lf.pair = i;
        lf.mult = m;
        PairDesc &pd = lf.pd;
        memset(&pd, 0, sizeof(pd));
        pd.N = d + 1;
        pd.NI = (int32_t)b->yun_ostride;
        pd.K = KH[i];
        pd.Lout = LH;
        pd.img_off = off;
        const int64_t chunks = (LH + 15) / 16;
        pd.xl_off = xl;
        xl += (int64_t)pd.N * 16 * chunks;
        pd.cy_off = cy;
        cy += (int64_t)pd.N * chunks;
        pd.out_off = outw;
        outw += (int64_t)pd.N * LH;
        lifts.push_back(lf);
        kmax = std::max(kmax, KH[i]);
      }
      off += d + 1;
    }
  }
  // R's content as the gcd of its coefficients: the fallback of the content
  // from the factors' leading coefficients (below).
  auto content_by_gcd = [&](PairRes &q) {
    std::vector<Big> Rm(q.degR + 1);
    for (int j = 0; j <= q.degR; ++j) {
      bool ng;
      Rm[j] = from_twos(&q.Rw[(size_t)j * q.LR], q.LR, &ng);
    }
    q.content = content_of(Rm, nullptr);
  };
  // One CRT pass over every factor of every pair.
  const int nf = (int)lifts.size();
  std::vector<uint32_t> hwords((size_t)outw);
  if (nf) {
    // The CRT's digit kernel overwrites its residues with the mixed-radix
    // digits, and the device path of the primitive parts (below) reads the
    // residues of H_m again: the residues are first gathered (scaled by g = 1)
    // into a compact copy, prime-major with stride N, which this pass consumes.
    std::vector<PairDesc> descs(nf);
    std::vector<ScaleDesc> gat(nf);
    int64_t qwA = 0;
    for (int fi = 0; fi < nf; ++fi) {
      const PairDesc &pd = lifts[fi].pd;
      descs[fi] = pd;
      descs[fi].img_off = qwA;
      descs[fi].NI = pd.N;
      ScaleDesc &u = gat[fi];
      u.src_off = pd.img_off;
      u.src_stride = pd.NI;
      u.dst_off = qwA;
      u.n = pd.N;
      u.k = pd.K;
      u.g_off = 0;
      u.g_len = 1;
      qwA += (int64_t)pd.K * pd.N;
    }
    const uint32_t one = 1u;
    std::vector<int2> g3d, g3;
    std::vector<int4> g3b;
    for (int fi = 0; fi < nf; ++fi) {
      const PairDesc &pd = descs[fi];
      for (int j = 0; j < pd.N; j += 32) g3d.push_back(make_int2(fi, j));
      for (int j = 0; j < pd.N; j += 128) g3.push_back(make_int2(fi, j));
      for (int c = 0; c < (pd.Lout + 15) / 16; ++c)
        for (int j = 0; j < pd.N; j += 128) g3b.push_back(make_int4(fi, j, c, 0));
    }
    const int64_t shape_off = outw;
    auto round256 = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t piece[10] = {descs.size() * sizeof(PairDesc), g3d.size() * 8, g3.size() * 8, g3b.size() * 16,
                              (size_t)xl * 4, (size_t)cy * 8, (size_t)(outw + 2 * (int64_t)nf) * 4,
                              (size_t)qwA * 4, gat.size() * sizeof(ScaleDesc), sizeof(one)};
    size_t bytes = 0;
    for (size_t x : piece) bytes += round256(x);
    DevGuard dg(ctx->device);
    cudaError_t e = cudaSuccess;
    if (bytes > ctx->sqf_arena_bytes) {  // grown on demand, kept by the context
      if (ctx->sqf_arena) cudaFree(ctx->sqf_arena);
      ctx->sqf_arena = nullptr;
      ctx->sqf_arena_bytes = 0;
      e = cudaMalloc(&ctx->sqf_arena, bytes);
      if (e == cudaSuccess) ctx->sqf_arena_bytes = bytes;
      else ctx->sqf_arena = nullptr;
    }
    char *cur = static_cast<char *>(ctx->sqf_arena);
    auto carve = [&](size_t x) {
      char *r = cur;
      cur += round256(x);
      return r;
    };
    cudaStream_t s = b->stream;
    cudaEvent_t lev[2] = {nullptr, nullptr};
    for (auto &x : lev)
      if (e == cudaSuccess) e = cudaEventCreate(&x);
    if (e == cudaSuccess) {
      PairDesc *d_desc = (PairDesc *)carve(piece[0]);
      int2 *d_g3d = (int2 *)carve(piece[1]);
      int2 *d_g3 = (int2 *)carve(piece[2]);
      int4 *d_g3b = (int4 *)carve(piece[3]);
      uint32_t *d_xl = (uint32_t *)carve(piece[4]);
      int64_t *d_cy = (int64_t *)carve(piece[5]);
      uint32_t *d_out = (uint32_t *)carve(piece[6]);
      uint32_t *d_qA = (uint32_t *)carve(piece[7]);
      ScaleDesc *d_gat = (ScaleDesc *)carve(piece[8]);
      uint32_t *d_one = (uint32_t *)carve(piece[9]);
      e = cudaMemcpyAsync(d_desc, descs.data(), piece[0], cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(d_gat, gat.data(), piece[8], cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(d_one, &one, piece[9], cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(d_g3d, g3d.data(), piece[1], cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(d_g3, g3.data(), piece[2], cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(d_g3b, g3b.data(), piece[3], cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaMemsetAsync(d_out + shape_off, 0, (size_t)nf * 8, s);
      RsTables tab;
      {
        std::lock_guard<std::mutex> lock(ctx->tab_mu);
        tab = ctx->tab;
      }
      if (e == cudaSuccess) {
        G3Args a3;
        memset(&a3, 0, sizeof(a3));
        a3.pairs = d_desc;
        a3.ctasks = d_g3b;
        a3.mods = ctx->d_mods;
        a3.crt = ctx->d_crt;
        a3.wtab = tab.wtab;
        a3.p16 = tab.p16;
        a3.poff = tab.poff;
        a3.nh = tab.nh;
        a3.coef = d_qA;  // residues of H_m gathered from the Yun output
        a3.xl = d_xl;
        a3.carry = d_cy;
        a3.out = d_out;
        a3.shape = reinterpret_cast<int32_t *>(d_out + shape_off);
        a3.kmax = kmax;
        e = cudaEventRecord(lev[0], s);
        if (e == cudaSuccess) e = launch_scale(d_gat, nf, kmax, ctx->d_mods, d_one, b->d_yun_out, d_qA, s);
        if (e == cudaSuccess) e = launch_g3t((int)g3d.size(), a3, d_g3d, s);
        if (e == cudaSuccess) e = launch_g3bc((int)g3b.size(), (int)g3.size(), a3, d_g3, s);
        if (e == cudaSuccess) e = cudaEventRecord(lev[1], s);
      }
      const auto tf = std::chrono::steady_clock::now();
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(hwords.data(), d_out, (size_t)outw * 4, cudaMemcpyDeviceToHost, s);
      info.h2d_bytes += (int64_t)(piece[0] + piece[1] + piece[2] + piece[3] + piece[8] + piece[9]);
      info.d2h_bytes += (int64_t)outw * 4;
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      info.ms_fetch = (float)std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tf).count();
      if (e == cudaSuccess) e = cudaEventElapsedTime(&info.ms_lift, lev[0], lev[1]);
    }
    for (auto &x : lev)
      if (x) cudaEventDestroy(x);
    if (e != cudaSuccess) {
      rs_free_batch(b);
      ctx->sqf_cache = nullptr;
      return rs_fail(ctx, RS_ERR_CUDA, std::string("square-free CRT: ") + cudaGetErrorString(e));
    }
  }
  // Primitive parts R_m = H_m / content(H_m), first on the device.  g = gcd of
  // lc(H_m) and a few coefficients of H_m is a multiple of content(H_m) and
  // divides lc(H_m) = lc(R), so it is invertible modulo every lifting prime
  // (each keeps deg R).  The device takes V = H_m g^{-1} mod each prime and
  // its CRT in the symmetric range, so g V = H_m (mod P).  Since |H_m| < P/4
  // (the factor bound), |g V| <= P/4 forces g V = H_m: g then divides every
  // coefficient, g = content(H_m) and V = +-R_m.  A factor that fails this
  // check (or any device step) takes the host path: content by running gcd
  // and long division of every coefficient.
  const auto t_prim0 = std::chrono::steady_clock::now();
  std::vector<char> dev_ok(nf, 0);
  std::vector<int> qneed(nf, 0), gbitsv(nf, 0), limP(nf, 0);
  std::vector<int64_t> qoffh(nf, 0);
  std::vector<uint32_t> qh;
  if (nf) {
    std::vector<Big> gc(nf);
    parallel_for(nf, [&](int fi) {
      const PairDesc &pd = lifts[fi].pd;
      auto coef = [&](int j) {
        bool ng;
        return from_twos(&hwords[(size_t)(pd.out_off + (int64_t)j * pd.Lout)], pd.Lout, &ng);
      };
      Big g = coef(pd.N - 1);
      const int picks[8] = {0, 1, 2, pd.N / 4, pd.N / 2, (3 * pd.N) / 4, pd.N - 3, pd.N - 2};
      for (int t = 0; t < 8 && !(g.size() == 1 && g[0] == 1u); ++t) {
        const int j = picks[t];
        if (j < 0 || j >= pd.N - 1) continue;
        const Big c = coef(j);
        if (c.empty()) continue;
        Big r;
        big_divmod(c, g, &r);
        if (!r.empty()) g = big_gcd_lehmer(g, r);
      }
      gc[fi] = std::move(g);
    });
    // second CRT pass over the scaled residues (compact: prime-major, stride N)
    std::vector<PairDesc> dB(nf);
    std::vector<ScaleDesc> sd(nf);
    std::vector<uint32_t> gw;
    int64_t qw = 0, xlB = 0, cyB = 0, outB = 0;
    int kmaxB = 0;
    for (int fi = 0; fi < nf; ++fi) {
      const PairDesc &pd = lifts[fi].pd;
      PairDesc q = pd;
      const int LQ = (31 * pd.K + 31) / 32 + 1;  // any symmetric residue mod P < 2^(31 K)
      const int64_t chunks = (LQ + 15) / 16;
      q.img_off = qw;
      q.NI = pd.N;
      q.Lout = LQ;
      q.xl_off = xlB;
      xlB += (int64_t)pd.N * 16 * chunks;
      q.cy_off = cyB;
      cyB += (int64_t)pd.N * chunks;
      q.out_off = outB;
      outB += (int64_t)pd.N * LQ;
      dB[fi] = q;
      ScaleDesc &u = sd[fi];
      u.src_off = pd.img_off;
      u.src_stride = pd.NI;
      u.dst_off = qw;
      u.n = pd.N;
      u.k = pd.K;
      u.g_off = (int64_t)gw.size();
      u.g_len = (int32_t)gc[fi].size();
      gw.insert(gw.end(), gc[fi].begin(), gc[fi].end());
      qw += (int64_t)pd.K * pd.N;
      kmaxB = std::max(kmaxB, pd.K);
    }
    if (gw.empty()) gw.push_back(0u);
    std::vector<int2> g3dB, g3B;
    std::vector<int4> g3bB;
    for (int fi = 0; fi < nf; ++fi) {
      const PairDesc &q = dB[fi];
      for (int j = 0; j < q.N; j += 32) g3dB.push_back(make_int2(fi, j));
      for (int j = 0; j < q.N; j += 128) g3B.push_back(make_int2(fi, j));
      for (int c = 0; c < (q.Lout + 15) / 16; ++c)
        for (int j = 0; j < q.N; j += 128) g3bB.push_back(make_int4(fi, j, c, 0));
    }
    auto round256 = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t pc[10] = {dB.size() * sizeof(PairDesc), g3dB.size() * 8, g3B.size() * 8, g3bB.size() * 16,
                           (size_t)xlB * 4, (size_t)cyB * 8, (size_t)(outB + 2 * (int64_t)nf) * 4,
                           (size_t)qw * 4, gw.size() * 4, sd.size() * sizeof(ScaleDesc)};
    size_t bytes = 0;
    for (size_t x : pc) bytes += round256(x);
    DevGuard dg(ctx->device);
    cudaError_t e = cudaSuccess;
    if (bytes > ctx->sqf_arena_bytes) {
      if (ctx->sqf_arena) cudaFree(ctx->sqf_arena);
      ctx->sqf_arena = nullptr;
      ctx->sqf_arena_bytes = 0;
      e = cudaMalloc(&ctx->sqf_arena, bytes);
      if (e == cudaSuccess) ctx->sqf_arena_bytes = bytes;
      else ctx->sqf_arena = nullptr;
    }
    cudaStream_t s = b->stream;
    cudaEvent_t qev[2] = {nullptr, nullptr};
    for (auto &x : qev)
      if (e == cudaSuccess) e = cudaEventCreate(&x);
    std::vector<int32_t> shp(2 * (size_t)nf, 0);
    uint32_t *d_outB = nullptr;
    if (e == cudaSuccess) {
      char *cur = static_cast<char *>(ctx->sqf_arena);
      auto carve = [&](size_t x) {
        char *r = cur;
        cur += round256(x);
        return r;
      };
      PairDesc *d_desc = (PairDesc *)carve(pc[0]);
      int2 *d_g3d = (int2 *)carve(pc[1]);
      int2 *d_g3 = (int2 *)carve(pc[2]);
      int4 *d_g3b = (int4 *)carve(pc[3]);
      uint32_t *d_xl = (uint32_t *)carve(pc[4]);
      int64_t *d_cy = (int64_t *)carve(pc[5]);
      d_outB = (uint32_t *)carve(pc[6]);
      uint32_t *d_q = (uint32_t *)carve(pc[7]);
      uint32_t *d_gw = (uint32_t *)carve(pc[8]);
      ScaleDesc *d_sd = (ScaleDesc *)carve(pc[9]);
      e = cudaMemcpyAsync(d_desc, dB.data(), pc[0], cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(d_g3d, g3dB.data(), pc[1], cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(d_g3, g3B.data(), pc[2], cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(d_g3b, g3bB.data(), pc[3], cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(d_gw, gw.data(), pc[8], cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(d_sd, sd.data(), pc[9], cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaMemsetAsync(d_outB + outB, 0, (size_t)nf * 8, s);
      info.h2d_bytes += (int64_t)(pc[0] + pc[1] + pc[2] + pc[3] + pc[8] + pc[9]);
      RsTables tab;
      {
        std::lock_guard<std::mutex> lock(ctx->tab_mu);
        tab = ctx->tab;
      }
      if (e == cudaSuccess) e = cudaEventRecord(qev[0], s);
      if (e == cudaSuccess) e = launch_scale(d_sd, nf, kmaxB, ctx->d_mods, d_gw, b->d_yun_out, d_q, s);
      if (e == cudaSuccess) {
        G3Args a3;
        memset(&a3, 0, sizeof(a3));
        a3.pairs = d_desc;
        a3.ctasks = d_g3b;
        a3.mods = ctx->d_mods;
        a3.crt = ctx->d_crt;
        a3.wtab = tab.wtab;
        a3.p16 = tab.p16;
        a3.poff = tab.poff;
        a3.nh = tab.nh;
        a3.coef = d_q;
        a3.xl = d_xl;
        a3.carry = d_cy;
        a3.out = d_outB;
        a3.shape = reinterpret_cast<int32_t *>(d_outB + outB);
        a3.kmax = kmaxB;
        e = launch_g3t((int)g3dB.size(), a3, d_g3d, s);
        if (e == cudaSuccess) e = launch_g3bc((int)g3bB.size(), (int)g3B.size(), a3, d_g3, s);
      }
      if (e == cudaSuccess) e = cudaEventRecord(qev[1], s);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(shp.data(), d_outB + outB, (size_t)nf * 8, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      float msB = 0.0f;
      if (e == cudaSuccess && cudaEventElapsedTime(&msB, qev[0], qev[1]) == cudaSuccess) info.ms_lift += msB;
    }
    if (e == cudaSuccess) {
      int64_t words = 0;
      for (int fi = 0; fi < nf; ++fi) {
        const PairDesc &q = dB[fi];
        double log2P = 0.0;
        for (int k = 0; k < q.K; ++k) log2P += ctx->log2p[k];
        const int need = shp[2 * (size_t)fi + 1];
        gbitsv[fi] = bitlen(gc[fi]);
        limP[fi] = (int)std::floor(log2P - 1e-6) - 2;  // 2^limP <= P / 4
        // |g V| <= P / 4 holds when gbits + (bits of the largest |V_j|) <= limP,
        // checked exactly on the host once V is read; a coefficient that needs
        // `need` limbs has more than 32 (need - 1) - 1 bits, so this filter
        // only drops factors that would fail
        if (shp[2 * (size_t)fi] == q.N && need >= 1 && need <= q.Lout &&
            gbitsv[fi] + 32 * (need - 1) - 1 <= limP[fi]) {
          dev_ok[fi] = 1;
          qneed[fi] = need;
          qoffh[fi] = words;
          words += (int64_t)q.N * need;
        }
      }
      qh.assign((size_t)std::max<int64_t>(words, 1), 0u);
      for (int fi = 0; fi < nf && e == cudaSuccess; ++fi) {
        if (!dev_ok[fi]) continue;
        const PairDesc &q = dB[fi];
        e = cudaMemcpy2DAsync(qh.data() + qoffh[fi], (size_t)qneed[fi] * 4, d_outB + q.out_off, (size_t)q.Lout * 4,
                              (size_t)qneed[fi] * 4, q.N, cudaMemcpyDeviceToHost, s);
      }
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      info.d2h_bytes += (int64_t)nf * 8 + words * 4;
    }
    for (auto &x : qev)
      if (x) cudaEventDestroy(x);
    if (e != cudaSuccess) {
      cudaGetLastError();  // a non-sticky failure: every factor takes the host path
      std::fill(dev_ok.begin(), dev_ok.end(), 0);
    }
  }
  std::vector<int> lift_rc(nf, RS_OK);
  std::vector<Big> lcq(nf);  // lc of each primitive factor
  std::vector<int> order(nf);  // largest factors first
  for (int fi = 0; fi < nf; ++fi) order[fi] = fi;
  std::sort(order.begin(), order.end(), [&](int x, int y) { return lifts[x].pd.N > lifts[y].pd.N; });
  parallel_for(nf, [&](int t) {
    const int fi = order[t];
    const Lift &lf = lifts[fi];
    const PairDesc &pd = lf.pd;
    std::vector<Big> mag(pd.N), q;
    std::vector<char> neg(pd.N);
    if (dev_ok[fi]) {  // V = +-R_m from the device, if |g V| <= P / 4
      int vbits = 0;
      for (int j = 0; j < pd.N; ++j) {
        bool ng;
        q.push_back(from_twos(&qh[(size_t)(qoffh[fi] + (int64_t)j * qneed[fi])], qneed[fi], &ng));
        neg[j] = ng;
        vbits = std::max(vbits, bitlen(q.back()));
      }
      if (gbitsv[fi] + vbits > limP[fi]) {
        dev_ok[fi] = 0;
        q.clear();
      }
    }
    if (!dev_ok[fi]) {
      for (int j = 0; j < pd.N; ++j) {
        bool ng;
        mag[j] = from_twos(&hwords[(size_t)(pd.out_off + (int64_t)j * pd.Lout)], pd.Lout, &ng);
        neg[j] = ng;
      }
      content_of(mag, &q);
    }
    lcq[fi] = q[pd.N - 1];
    const bool flip = neg[pd.N - 1] != 0;
    for (int j = 0; j < pd.N; ++j) neg[j] = q[j].empty() ? 0 : (char)((neg[j] != 0) != flip);
    lift_rc[fi] = put(factors[(size_t)lf.pair * M + lf.mult], q, neg);
  });
  info.factors_device = (int32_t)std::count(dev_ok.begin(), dev_ok.end(), (char)1);
  std::vector<Big> lcprod(n, Big{1u});  // prod_i lc(R_i)^i per pair
  for (int fi = 0; fi < nf; ++fi) {
    const Lift &lf = lifts[fi];
    if (out_rc[lf.pair] == RS_OK) out_rc[lf.pair] = lift_rc[fi];
    nmult[lf.pair] = std::max(nmult[lf.pair], lf.mult + 1);
    for (int r = 0; r <= lf.mult; ++r) lcprod[lf.pair] = big_mul(lcprod[lf.pair], lcq[fi]);
  }
  const auto t_end = std::chrono::steady_clock::now();
  // R's content: R = c prod_i R_i^i with R_i primitive and lc R_i > 0, so
  // c = lc(R) / prod_i lc(R_i)^i, sign(c) = sign(lc R).  The division must be
  // exact; if it is not (or a factor was not produced), the gcd of R's
  // coefficients is taken instead.
  {
    std::vector<int> todo;
    for (int i = 0; i < n; ++i)
      if (st[i] == RS_OK) todo.push_back(i);
    parallel_for((int)todo.size(), [&](int t) {
      const int i = todo[t];
      PairRes &q = pr[i];
      Big r;
      q.content = out_rc[i] == RS_OK ? big_divmod(q.lcR, lcprod[i], &r) : Big();
      if (out_rc[i] != RS_OK || !r.empty() || q.content.empty()) content_by_gcd(q);
      std::vector<uint32_t>().swap(q.Rw);
    });
    for (int i : todo) {
      const int r2 = put(content[i], {pr[i].content}, {(char)pr[i].lc_neg});
      if (out_rc[i] == RS_OK) out_rc[i] = r2;
    }
  }
  const auto t_end2 = std::chrono::steady_clock::now();
  info.ms_contents = (float)std::chrono::duration<double, std::milli>(t_end2 - t_end).count();
  auto ms = [](std::chrono::steady_clock::time_point a, std::chrono::steady_clock::time_point z) {
    return (float)std::chrono::duration<double, std::milli>(z - a).count();
  };
  info.factors = nf;
  info.ms_primitive = ms(t_prim0, t_end);
  info.ms_host = ms(t_host0, t_end2) - info.ms_lift;
  info.ms_total = ms(t_start, t_end2);
  ctx->sqf_info = info;
  int ret = RS_OK;
  for (int i = 0; i < n; ++i) {
    if (st[i] == RS_OK && out_rc[i] != RS_OK) {
      st[i] = out_rc[i];
      why[i] = "output capacity too small";
    }
    if (status) status[i] = st[i];
    if (st[i] != RS_OK && ret == RS_OK) {
      ret = st[i];
      rs_fail(ctx, st[i], n == 1 ? why[i] : "pair " + std::to_string(i) + ": " + why[i]);
    }
  }
  return ret;
}

extern "C" int rs_squarefree_y(rs_ctx *ctx, const rs_bipoly *f, const rs_bipoly *g, int32_t max_mult,
                               rs_upoly *content, rs_upoly *factors, int32_t *nmult) {
  if (!ctx || !f || !g || !content || !factors || !nmult || max_mult < 1)
    return rs_fail(ctx, RS_ERR_ARG, "NULL argument or max_mult < 1");
  return rs_squarefree_batch(ctx, 1, f, g, max_mult, content, factors, nmult, nullptr);
}

extern "C" int rs_squarefree_info_get(const rs_ctx *ctx, rs_sqf_info *info) {
  if (!ctx || !info) return RS_ERR_ARG;
  *info = ctx->sqf_info;
  return RS_OK;
}
