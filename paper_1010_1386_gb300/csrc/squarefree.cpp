// Square-free factorisation of R^{(y)} = res(f, g, y) (the paper's solver,
// Section 5, PROJECT: R^{(y)} "and a corresponding square-free
// factorization"): R = c prod_i R_i^i with R_i primitive, square-free,
// pairwise coprime, leading coefficient > 0.
//
// One batch computes R over K primes chosen for the factors' bound (below),
// and Yun's algorithm mod every prime after G2 (kernels_yun.cu).  A prime is
// used if R keeps its degree mod p and the square-free part mod p has the
// largest degree seen (a smaller one means p divides a discriminant and
// merged factors).  Every R_i divides F = pp(R), so by Mignotte's bound
// (M. Mignotte, "An inequality about factors of polynomials", Math. Comp. 28,
// 1974) |coef R_i| <= 2^{deg R_i} ||R||_2, and H_i = lc(R) R_i / lc(R_i) (the
// residues lc(R) monic(R_i mod p) lift to it) has coefficients below
// |lc R| 2^{deg R} ||R||_2 <= 2^{2 B + D + log2(D + 1) / 2}, B the resultant's
// coefficient bits and D its degree bound.  The H_i are lifted by the CRT
// kernels over the first K_H primes, then R_i = H_i / content(H_i) on the
// host (binary gcd and exact division by Hensel's method), and c = sign(lc R)
// content(R).
#include <string.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>
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

// a / b for b dividing a exactly (Hensel division from the low limb).
Big big_divexact(Big a, Big b) {
  const int z = ctz(b);
  shr_in_place(a, z);
  shr_in_place(b, z);
  if (b.size() == 1 && b[0] == 1u) return a;
  uint32_t inv = b[0];  // b odd: Newton's iteration for b^-1 mod 2^32
  for (int i = 0; i < 5; ++i) inv *= 2u - b[0] * inv;
  const size_t nq = a.size() >= b.size() ? a.size() - b.size() + 1 : 0;
  Big q(nq, 0u);
  a.resize(std::max(a.size(), nq + b.size()) + 1, 0u);
  for (size_t i = 0; i < nq; ++i) {
    const uint32_t qi = a[i] * inv;
    q[i] = qi;
    uint64_t borrow = 0;  // a -= qi * b << (32 i)
    for (size_t j = 0; j < b.size(); ++j) {
      const uint64_t prod = (uint64_t)qi * b[j] + borrow;
      const uint32_t lo = (uint32_t)prod;
      borrow = (prod >> 32) + (a[i + j] < lo ? 1u : 0u);
      a[i + j] -= lo;
    }
    for (size_t j = i + b.size(); borrow && j < a.size(); ++j) {
      const uint32_t prev = a[j];
      a[j] -= (uint32_t)borrow;
      borrow = prev < (uint32_t)borrow ? 1u : 0u;
    }
  }
  trim(q);
  return q;
}

}  // namespace

extern "C" int rs_squarefree_y(rs_ctx *ctx, const rs_bipoly *f, const rs_bipoly *g, int32_t max_mult,
                               rs_upoly *content, rs_upoly *factors, int32_t *nmult) {
  if (!ctx || !f || !g || !content || !factors || !nmult || max_mult < 1)
    return rs_fail(ctx, RS_ERR_ARG, "NULL argument or max_mult < 1");
  std::vector<PairPlan> plans;
  int first = RS_OK;
  rs_plan_all(ctx, 1, f, g, plans, nullptr, &first);
  if (first != RS_OK) return first;
  PairPlan &p = plans[0];
  if (p.trivial_zero) return rs_fail(ctx, RS_ERR_ARG, "R = 0 has no square-free factorisation");
  // primes for the factors: coefficients of H_i below 2^bitsH
  const int bitsH = 2 * p.bits + p.D + (int)std::ceil(0.5 * std::log2((double)p.D + 1.0)) + 2;
  int KH = 0;
  {
    double acc = 0.0;
    while (KH < (int)ctx->log2p.size() && acc < bitsH + 2) acc += ctx->log2p[KH++];
    if (acc < bitsH + 2) return rs_fail(ctx, RS_ERR_LIMIT, "factor bound needs more primes than RS_MAX_PRIMES");
  }
  const int Kall = std::min((int)ctx->log2p.size(), std::max(p.K, KH) + 4);  // a few spare primes
  p.K = Kall;
  RsBatchOpts o;
  o.use_graph = false;
  o.persistent = ctx->cfg.persistent != 0;
  o.fork = true;
  o.yun_maxm = max_mult;
  rs_batch *b = nullptr;
  int rc = rs_build_batch(ctx, 1, f, g, std::move(plans), o, &b);
  if (rc != RS_OK) return rc;
  DevGuard dg(ctx->device);
  rc = rs_upload(b, f, g);
  if (rc == RS_OK) rc = rs_run(b);
  if (rc == RS_OK) rc = rs_fetch_async(b);
  std::vector<uint32_t> yun((size_t)b->nyun * b->yun_ostride);
  if (rc == RS_OK && !yun.empty()) {
    cudaError_t e = cudaMemcpyAsync(yun.data(), b->d_yun_out, yun.size() * 4, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) rc = rs_fail(ctx, RS_ERR_CUDA, std::string("square-free: ") + cudaGetErrorString(e));
  }
  std::vector<uint32_t> Rw;
  int degR = -1, LR = 1;
  if (rc == RS_OK) rc = rs_unpack_one(b, 0, Rw, &degR, &LR);
  if (rc != RS_OK) {
    rs_free_batch(b);
    return rc;
  }
  if (degR < 0) {
    rs_free_batch(b);
    return rs_fail(ctx, RS_ERR_ARG, "R = 0 has no square-free factorisation");
  }
  // content c = sign(lc R) gcd(coefficients of R)
  Big cg;
  bool lc_neg = false;
  for (int j = 0; j <= degR; ++j) {
    bool neg;
    const Big v = from_twos(&Rw[(size_t)j * LR], LR, &neg);
    if (j == degR) lc_neg = neg;
    cg = big_gcd(cg, v);
  }
  auto put = [&](rs_upoly &out, const std::vector<std::pair<Big, bool>> &coefs) -> int {
    int L = 1;
    for (const auto &cv : coefs) L = std::max(L, twos_limbs(cv.first, cv.second));
    const int deg = (int)coefs.size() - 1;
    out.deg = deg;
    out.limbs = L;
    if ((int64_t)(deg + 1) * L > out.capacity_words || (!out.coeffs && deg >= 0)) return RS_ERR_CAPACITY;
    for (int j = 0; j <= deg; ++j) to_twos(coefs[j].first, coefs[j].second, out.coeffs + (size_t)j * L, L);
    return RS_OK;
  };
  int out_rc = put(*content, {{cg, lc_neg}});
  for (int i = 0; i < max_mult; ++i) {  // R_i = 1 unless set below
    std::vector<std::pair<Big, bool>> one{{Big{1u}, false}};
    const int r2 = put(factors[i], one);
    if (out_rc == RS_OK) out_rc = r2;
  }
  *nmult = 0;
  if (degR <= 0) {
    rs_free_batch(b);
    return out_rc != RS_OK ? rs_fail(ctx, out_rc, "output capacity too small") : RS_OK;
  }
  // usable primes: R keeps its degree mod p, square-free part of largest degree
  const int M = max_mult;
  auto task = [&](int k) { return &yun[(size_t)k * b->yun_ostride]; };
  int best_sf = -1;
  for (int k = 0; k < b->nyun; ++k) {
    const uint32_t *t = task(k);
    if ((int)t[0] != degR || t[1]) continue;
    int sf = 0;
    for (int i = 0; i < M; ++i) sf += (int)t[2 + i];
    best_sf = std::max(best_sf, sf);
  }
  for (int k = 0; k < KH && k < b->nyun; ++k)
    if ((int)task(k)[0] == degR && task(k)[1]) {  // Yun ran past max_mult on a prime that keeps deg R
      rs_free_batch(b);
      return rs_fail(ctx, RS_ERR_CAPACITY, "a factor's multiplicity exceeds max_mult");
    }
  std::vector<int> pattern(M, 0);
  int good = 0;  // length of the prefix of usable primes with the same pattern
  for (int k = 0; k < b->nyun; ++k) {
    const uint32_t *t = task(k);
    if ((int)t[0] != degR || t[1]) break;
    int sf = 0;
    for (int i = 0; i < M; ++i) sf += (int)t[2 + i];
    if (sf != best_sf) break;
    if (k == 0)
      for (int i = 0; i < M; ++i) pattern[i] = (int)t[2 + i];
    bool same = true;
    for (int i = 0; i < M; ++i) same = same && (int)t[2 + i] == pattern[i];
    if (!same) break;
    ++good;
  }
  if (good < KH) {
    rs_free_batch(b);
    return rs_fail(ctx, RS_ERR_LIMIT,
                   "an unlucky prime for the square-free factorisation lies among the first " +
                       std::to_string(KH) + " primes (prime index " + std::to_string(good) + ")");
  }
  // Lift H_i = lc(R) R_i / lc(R_i) over the first KH primes with the CRT kernels.
  std::vector<int> fidx;  // multiplicities with a non-constant factor
  std::vector<PairDesc> descs;
  int64_t off = 2 + M, xl = 0, cy = 0, outw = 0;
  const int LH = (bitsH + 1 + 31) / 32;
  for (int i = 0; i < M; ++i) {
    const int d = pattern[i];
    if (d > 0) {
      PairDesc pd;
      memset(&pd, 0, sizeof(pd));
      pd.N = d + 1;
      pd.NI = (int32_t)b->yun_ostride;
      pd.K = KH;
      pd.Lout = LH;
      pd.img_off = off;
      const int64_t chunks = (LH + 15) / 16;
      pd.xl_off = xl;
      xl += (int64_t)pd.N * 16 * chunks;
      pd.cy_off = cy;
      cy += (int64_t)pd.N * chunks;
      pd.out_off = outw;
      outw += (int64_t)pd.N * LH;
      descs.push_back(pd);
      fidx.push_back(i);
    }
    off += d + 1;
  }
  const int nf = (int)descs.size();
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
  outw += 2 * (int64_t)nf;
  auto round256 = [](size_t n) { return (n + 255) & ~(size_t)255; };
  const size_t piece[7] = {descs.size() * sizeof(PairDesc), g3d.size() * 8, g3.size() * 8, g3b.size() * 16,
                           (size_t)xl * 4, (size_t)cy * 8, (size_t)outw * 4};
  size_t bytes = 0;
  for (size_t n : piece) bytes += round256(n);
  void *arena = nullptr;
  cudaError_t e = cudaMalloc(&arena, bytes);
  char *cur = static_cast<char *>(arena);
  auto carve = [&](size_t n) {
    char *r = cur;
    cur += round256(n);
    return r;
  };
  PairDesc *d_desc = nullptr;
  int2 *d_g3d = nullptr, *d_g3 = nullptr;
  int4 *d_g3b = nullptr;
  uint32_t *d_xl = nullptr, *d_out = nullptr;
  int64_t *d_cy = nullptr;
  if (e == cudaSuccess) {
    d_desc = (PairDesc *)carve(descs.size() * sizeof(PairDesc));
    d_g3d = (int2 *)carve(g3d.size() * 8);
    d_g3 = (int2 *)carve(g3.size() * 8);
    d_g3b = (int4 *)carve(g3b.size() * 16);
    d_xl = (uint32_t *)carve((size_t)xl * 4);
    d_cy = (int64_t *)carve((size_t)cy * 8);
    d_out = (uint32_t *)carve((size_t)outw * 4);
  }
  cudaStream_t s = b->stream;
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_desc, descs.data(), descs.size() * sizeof(PairDesc), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_g3d, g3d.data(), g3d.size() * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_g3, g3.data(), g3.size() * 8, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_g3b, g3b.data(), g3b.size() * 16, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_out + shape_off, 0, (size_t)nf * 8, s);
  RsTables tab;
  {
    std::lock_guard<std::mutex> lock(ctx->tab_mu);
    tab = ctx->tab;
  }
  if (e == cudaSuccess && nf) {
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
    a3.coef = b->d_yun_out;  // the residues, stride yun_ostride per prime (task k = prime k)
    a3.xl = d_xl;
    a3.carry = d_cy;
    a3.out = d_out;
    a3.shape = reinterpret_cast<int32_t *>(d_out + shape_off);
    a3.kmax = KH;
    e = launch_g3t((int)g3d.size(), a3, d_g3d, s);
    if (e == cudaSuccess) e = launch_g3bc((int)g3b.size(), (int)g3.size(), a3, d_g3, s);
  }
  std::vector<uint32_t> hw((size_t)outw);
  if (e == cudaSuccess && outw) e = cudaMemcpyAsync(hw.data(), d_out, (size_t)outw * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (arena) cudaFree(arena);
  rs_free_batch(b);
  if (e != cudaSuccess) return rs_fail(ctx, RS_ERR_CUDA, std::string("square-free CRT: ") + cudaGetErrorString(e));
  // R_i = H_i / content(H_i), leading coefficient made positive
  for (int fi = 0; fi < nf; ++fi) {
    const PairDesc &pd = descs[fi];
    std::vector<std::pair<Big, bool>> co(pd.N);
    Big gg;
    for (int j = 0; j < pd.N; ++j) {
      bool neg;
      co[j].first = from_twos(&hw[(size_t)(pd.out_off + (int64_t)j * LH)], LH, &neg);
      co[j].second = neg;
      gg = big_gcd(gg, co[j].first);
    }
    const bool flip = co[pd.N - 1].second;
    for (auto &cv : co) {
      if (!cv.first.empty()) cv.first = big_divexact(cv.first, gg);
      cv.second = cv.first.empty() ? false : (cv.second != flip);
    }
    const int r2 = put(factors[fidx[fi]], co);
    if (out_rc == RS_OK) out_rc = r2;
    *nmult = std::max(*nmult, fidx[fi] + 1);
  }
  if (out_rc != RS_OK) return rs_fail(ctx, out_rc, "output capacity too small");
  return RS_OK;
}
