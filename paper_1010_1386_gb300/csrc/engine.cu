// Host engine of librs: contexts, prepared batches, CUDA-graph replay and the
// C ABI of include/rs.h.  The host plans (planner.cpp), packs inputs into one
// pinned staging buffer, enqueues G1 (kernels_g1.cu), G2 and G3
// (kernels_g23.cu) on a stream and unpacks the results.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <thread>

#include "engine.h"

namespace {

thread_local std::string g_err;

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// Normal-sequence coefficient updates of the remainder sequence (a4 count).
double prs_updates(int a, int b) {
  double u = 0;
  while (a > 0 && b > 0) {
    if (a >= b) {
      u += a;
      --a;
    } else {
      u += b;
      --b;
    }
  }
  return u;
}

}  // namespace

int rs_cuda_code(cudaError_t e) { return e == cudaErrorMemoryAllocation ? RS_ERR_NOMEM : RS_ERR_CUDA; }

int rs_fail(rs_ctx *c, int code, const std::string &msg) {
  if (c)
    c->err = msg;
  else
    g_err = msg;
  return code;
}

#define RS_CUDA(ctx, call)                                                                         \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess)                                                                         \
      return rs_fail((ctx), rs_cuda_code(e_), std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// ------------------------------------------------------------------ planning

int rs_plan_all(rs_ctx *ctx, int n, const rs_bipoly *f, const rs_bipoly *g,
                std::vector<PairPlan> &plans, int32_t *status, int *first_err) {
  plans.assign(n, PairPlan());
  *first_err = RS_OK;
  std::vector<const char *> why(n, "");
  auto plan_range = [&](int lo, int hi) {
    for (int i = lo; i < hi; ++i) plans[i].status = rs_plan_pair(&f[i], &g[i], ctx->log2p, plans[i], &why[i]);
  };
  // Planning reads every input coefficient once and takes one summed
  // autocorrelation per polynomial ((deg_x + 1)^2 (deg_y + 1) / 2 products);
  // large batches are split over host threads in contiguous ranges of pairs.
  auto sane = [](const rs_bipoly &p) {
    return p.coeffs && p.deg_x >= 0 && p.deg_y >= 0 && p.deg_x < (1 << 26) && p.deg_y < (1 << 26) &&
           p.limbs >= 1 && p.limbs <= RS_MAX_LIMBS;
  };
  int64_t words = 0;  // only steers the thread count
  auto corr = [](const rs_bipoly &p) {  // sane p: (deg_x + 1)^2 (deg_y + 1) < 2^78 would overflow
    const int64_t c = (int64_t)(p.deg_x + 1) * (p.deg_y + 1);
    return c <= ((int64_t)1 << 26) ? c * (p.deg_x + 1) / 16 : 0;
  };
  for (int i = 0; i < n; ++i)
    if (sane(f[i]) && sane(g[i])) words += rs_input_words(f[i]) + rs_input_words(g[i]) + corr(f[i]) + corr(g[i]);
  const int hw = std::max(1, (int)std::thread::hardware_concurrency());
  const int nt = (int)std::min<int64_t>({(int64_t)std::min(hw, 16), (int64_t)n, words / (int64_t(1) << 18) + 1});
  if (nt <= 1) {
    plan_range(0, n);
  } else {
    std::vector<std::thread> th;
    for (int t = 0; t < nt; ++t)
      th.emplace_back(plan_range, (int)((int64_t)n * t / nt), (int)((int64_t)n * (t + 1) / nt));
    for (auto &x : th) x.join();
  }
  for (int i = 0; i < n; ++i) {
    const int rc = plans[i].status;
    if (status) status[i] = rc;
    if (rc != RS_OK && *first_err == RS_OK) {
      *first_err = rc;
      rs_fail(ctx, rc, std::string("pair ") + std::to_string(i) + ": " + why[i]);
    }
  }
  return *first_err;
}

bool rs_same_shape(const PairPlan &a, const PairPlan &b) {
  return a.status == b.status && a.trivial_zero == b.trivial_zero && a.N == b.N && a.K == b.K &&
         a.Kcrt == b.Kcrt &&
         a.Lout == b.Lout && a.f.my == b.f.my && a.g.my == b.g.my && a.f.mx == b.f.mx &&
         a.g.mx == b.g.mx && a.f.L == b.f.L && a.g.L == b.g.L && a.f.stride == b.f.stride &&
         a.g.stride == b.g.stride && a.f.dx == b.f.dx && a.g.dx == b.g.dx;
}

int64_t rs_input_words(const rs_bipoly &p) { return (int64_t)(p.deg_x + 1) * (p.deg_y + 1) * p.limbs; }

// ------------------------------------------------------------------ tables

static void free_tables(RsTables &t) {
  void *p[] = {t.finv, t.gtab, t.qn, t.btab, t.qc, t.qp, t.hq, t.wtab, t.p16, t.poff, t.nh};
  for (void *x : p)
    if (x) cudaFree(x);
  t = RsTables();
}

// Reserved 16-bit digits of row k of the prefix-product table: p_0 ... p_{k-1}
// < 2^(31 k), rounded up to a multiple of 32.
static int p16_row(int k) { return ((31 * k) / 16 + 2 + 31) / 32 * 32; }

// ------------------------------------------------------------ NTT tables

// The three NTT primes c 2^k + 1 (k >= 25) of the transform-based G2, in
// (2^30, 2^31) and ascending; their product exceeds 2^92.
static const uint32_t kNttPrimes[3] = {1811939329u, 2013265921u, 2113929217u};

static uint32_t powmod_u32(uint64_t a, uint64_t e, uint32_t P) {
  uint64_t r = 1;
  a %= P;
  while (e) {
    if (e & 1) r = r * a % P;
    a = a * a % P;
    e >>= 1;
  }
  return (uint32_t)r;
}

// Smallest generator of Z_P^* (P prime): g^((P-1)/r) != 1 for every prime r | P - 1.
static uint32_t generator_of(uint32_t P) {
  std::vector<uint32_t> fac;
  uint32_t n = P - 1;
  for (uint32_t r = 2; (uint64_t)r * r <= n; ++r)
    if (n % r == 0) {
      fac.push_back(r);
      while (n % r == 0) n /= r;
    }
  if (n > 1) fac.push_back(n);
  for (uint32_t g = 2;; ++g) {
    bool ok = true;
    for (uint32_t r : fac) ok = ok && powmod_u32(g, (P - 1) / r, P) != 1;
    if (ok) return g;
  }
}

// Constants and twiddles [q][forward, inverse][2^LGMAX] as (w, floor(w 2^32 / P)):
// for each length 2^lg a row of w_L^j (forward) or w_L^-j (inverse), j < 2^(lg-1),
// starting at 2^(lg-1) - 1.
static void ntt_host_tables(NttConst &nc, std::vector<uint2> &tw) {
  const int ROW = 1 << RS_NTT_LGMAX;
  tw.assign((size_t)6 * ROW, make_uint2(0, 0));
  for (int q = 0; q < 3; ++q) {
    const uint32_t P = kNttPrimes[q];
    nc.m[q] = make_modp(P);
    const uint32_t wmax = powmod_u32(generator_of(P), (P - 1) >> RS_NTT_LGMAX, P);
    for (int lg = 1; lg <= RS_NTT_LGMAX; ++lg) {
      const uint32_t w = powmod_u32(wmax, (uint64_t)1 << (RS_NTT_LGMAX - lg), P);
      const uint32_t wi = powmod_u32(w, P - 2, P);
      const int n = 1 << (lg - 1);
      uint64_t f = 1, b = 1;
      for (int j = 0; j < n; ++j) {
        tw[(size_t)(2 * q) * ROW + (n - 1) + j] = make_uint2((uint32_t)f, (uint32_t)((f << 32) / P));
        tw[(size_t)(2 * q + 1) * ROW + (n - 1) + j] = make_uint2((uint32_t)b, (uint32_t)((b << 32) / P));
        f = f * w % P;
        b = b * wi % P;
      }
    }
  }
  const uint32_t P0 = kNttPrimes[0], P1 = kNttPrimes[1], P2 = kNttPrimes[2];
  const uint64_t R1 = ((uint64_t)1 << 32) % P1, R2 = ((uint64_t)1 << 32) % P2;
  nc.c01 = (uint32_t)((uint64_t)powmod_u32(P0, P1 - 2, P1) * R1 % P1);
  nc.p0_m2 = (uint32_t)((uint64_t)P0 % P2 * R2 % P2);
  const uint32_t p01 = (uint32_t)((uint64_t)P0 * P1 % P2);
  nc.c012 = (uint32_t)((uint64_t)powmod_u32(p01, P2 - 2, P2) * R2 % P2);
}

int rs_g2_len(int N) {
  int lg = 1;
  while ((1 << lg) < 2 * N - 1) ++lg;
  return lg <= RS_NTT_LGMAX ? lg : 0;
}

// Cost per (pair, prime) in direct multiply-accumulate-equivalents of issue
// time: a direct multiply-accumulate issues about 3.8 instructions (two
// convolutions of N^2 / 2 each); the transform form takes 12 transforms of
// (L/2) lg radix-4 butterflies, which timed at about 6.5 such units each on
// GB300 (lengths 2^9 and 2^10 ran 1.08x and 1.44x faster than direct).
double rs_g2_cost(int N, int form) {
  const int lg = rs_g2_len(N);
  if (form == 0 || lg == 0) return 3.8 * (double)N * N;
  return 12.0 * 6.5 * (double)(1 << (lg - 1)) * lg + 60.0 * N;
}

int rs_ensure_bhat(rs_ctx *ctx, int lg, int K) {
  const int L = 1 << lg;
  int rc = rs_ensure_tables(ctx, K, L / 2, 0);  // b_t for every t < L/2
  if (rc != RS_OK) return rc;
  std::lock_guard<std::mutex> lock(ctx->tab_mu);
  if (ctx->bhat_K[lg] >= K) return RS_OK;
  const RsTables &t = ctx->tab;
  DevGuard dg(ctx->device);
  uint32_t *nb = nullptr;
  cudaError_t e = cudaMalloc(&nb, (size_t)t.K * 3 * L * 4);
  if (e == cudaSuccess) e = launch_bhat(t.btab, t.N, t.N, t.K, lg, ctx->d_ntt_tw, ctx->nttc, nb, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    if (nb) cudaFree(nb);
    return rs_fail(ctx, rs_cuda_code(e), std::string("transform tables: ") + cudaGetErrorString(e));
  }
  if (ctx->bhat[lg]) ctx->bhat_retired.push_back(ctx->bhat[lg]);
  ctx->bhat[lg] = nb;
  ctx->bhat_K[lg] = t.K;
  return RS_OK;
}

int rs_ensure_g2t_btile(rs_ctx *ctx, int K, int tiles) {
  std::lock_guard<std::mutex> lock(ctx->tab_mu);
  if (ctx->g2t_K >= K && ctx->g2t_tiles >= tiles) return RS_OK;
  const RsTables &t = ctx->tab;
  const int nK = std::max(K, ctx->g2t_K), nt = std::max(tiles, ctx->g2t_tiles);
  if (t.K < nK)
    return rs_fail(ctx, RS_ERR_STATE, "tensor-core G2 tables: point tables not built for these primes");
  DevGuard dg(ctx->device);
  uint16_t *nb = nullptr;
  cudaError_t e = cudaMalloc(&nb, (size_t)nK * nt * 8192 * sizeof(uint16_t));
  if (e == cudaSuccess) e = launch_g2t_btile(t.btab, t.N, t.N, nK, nt, nb, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    if (nb) cudaFree(nb);
    return rs_fail(ctx, rs_cuda_code(e), std::string("tensor-core G2 tables: ") + cudaGetErrorString(e));
  }
  if (ctx->g2t_bt) ctx->g2t_retired.push_back(ctx->g2t_bt);
  ctx->g2t_bt = nb;
  ctx->g2t_K = nK;
  ctx->g2t_tiles = nt;
  return RS_OK;
}

int rs_ensure_g3m_wtiles(rs_ctx *ctx, int KB) {
  std::lock_guard<std::mutex> lock(ctx->tab_mu);
  if (ctx->g3m_KB >= KB) return RS_OK;
  const RsTables &t = ctx->tab;
  if (t.K < 64 * (KB - 1))
    return rs_fail(ctx, RS_ERR_STATE, "tensor-core CRT tables: CRT tables not built for these primes");
  DevGuard dg(ctx->device);
  uint16_t *nw = nullptr, *nr = nullptr;
  cudaError_t e = cudaMalloc(&nw, (size_t)std::max<int64_t>(1, g3m_wtile_elems(KB)) * sizeof(uint16_t));
  if (e == cudaSuccess) e = cudaMalloc(&nr, (size_t)std::max<int64_t>(1, g3m_rtile_elems(KB)) * sizeof(uint16_t));
  if (e == cudaSuccess) e = launch_g3m_wtiles(t.wtab, t.K, KB, nw, ctx->stream);
  if (e == cudaSuccess) e = launch_g3m_rtiles(t.wtab, t.K, KB, nr, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    if (nw) cudaFree(nw);
    if (nr) cudaFree(nr);
    return rs_fail(ctx, rs_cuda_code(e), std::string("tensor-core CRT tables: ") + cudaGetErrorString(e));
  }
  if (ctx->g3m_wt) ctx->g3m_retired.push_back(ctx->g3m_wt);
  if (ctx->g3m_rt) ctx->g3m_retired.push_back(ctx->g3m_rt);
  ctx->g3m_wt = nw;
  ctx->g3m_rt = nr;
  ctx->g3m_KB = KB;
  return RS_OK;
}

// Chunk c's prefix products reach byte 2 nh[k] (balanced digits of P_k, k
// its last prime's row) and, shifted by up to three digits, column
// 2 nh[k] + 3: units 0 .. (2 nh[k] + 3) / 256 get a block each.
int rs_ensure_g3l_tiles(rs_ctx *ctx, int KB) {
  std::lock_guard<std::mutex> lock(ctx->tab_mu);
  if (ctx->g3l_KB >= KB) return RS_OK;
  const RsTables &t = ctx->tab;
  if (t.K < 64 * (KB - 1) || (int)t.h_nh.size() < t.K + 1)
    return rs_fail(ctx, RS_ERR_STATE, "tensor-core CRT limb tables: CRT tables not built for these primes");
  std::vector<int32_t> cbase(KB + 1, 0);
  for (int c = 0; c < KB; ++c) {
    const int klast = std::min(64 * c + 63, t.K);
    cbase[c + 1] = cbase[c] + (2 * t.h_nh[klast] + 3) / 256 + 1;
  }
  DevGuard dg(ctx->device);
  uint16_t *nw = nullptr;
  int32_t *ncb = nullptr;
  cudaError_t e = cudaMalloc(&nw, (size_t)cbase[KB] * g3l_block_elems() * sizeof(uint16_t));
  if (e == cudaSuccess) e = cudaMalloc(&ncb, cbase.size() * sizeof(int32_t));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ncb, cbase.data(), cbase.size() * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = launch_g3l_btiles(t.p16, t.poff, t.K, ncb, KB, cbase[KB], nw, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    if (nw) cudaFree(nw);
    if (ncb) cudaFree(ncb);
    return rs_fail(ctx, rs_cuda_code(e), std::string("tensor-core CRT limb tables: ") + cudaGetErrorString(e));
  }
  if (ctx->g3l_bt) ctx->g3m_retired.push_back(ctx->g3l_bt);
  if (ctx->g3l_cbase) ctx->g3m_retired.push_back(ctx->g3l_cbase);
  ctx->g3l_bt = nw;
  ctx->g3l_cbase = ncb;
  ctx->h_g3l_cbase = cbase;
  ctx->g3l_KB = KB;
  return RS_OK;
}

int rs_ensure_tables(rs_ctx *ctx, int K, int N, int dx) {
  std::lock_guard<std::mutex> lock(ctx->tab_mu);
  const int need_c = N + 128 + dx + 1;
  RsTables &t = ctx->tab;
  if (K <= t.K && N <= t.N && need_c <= t.cstride) return RS_OK;
  RsTables nt;
  nt.K = std::min((int)ctx->primes.size(), ((std::max(K, t.K) + 63) / 64) * 64);
  nt.N = ((std::max(N, t.N) + 255) / 256) * 256;
  nt.cstride = ((std::max(need_c, t.cstride) + 255) / 256) * 256;
  DevGuard dg(ctx->device);
  const size_t ni = (size_t)nt.K * nt.N * 4, nc = (size_t)nt.K * nt.cstride * 4;
  cudaError_t e = cudaMalloc(&nt.finv, ni);
  if (e == cudaSuccess) e = cudaMalloc(&nt.gtab, ni);
  if (e == cudaSuccess) e = cudaMalloc(&nt.btab, ni);
  if (e == cudaSuccess) e = cudaMalloc(&nt.hq, ni);
  if (e == cudaSuccess) e = cudaMalloc(&nt.qc, nc);
  if (e == cudaSuccess) e = cudaMalloc(&nt.qn, nc);
  if (e == cudaSuccess) e = cudaMalloc(&nt.qp, nc);
  if (e == cudaSuccess)
    e = launch_tables(ctx->d_mods, ctx->d_qbase, nt.K, nt.N, nt.cstride, nt.finv, nt.gtab, nt.btab,
                      nt.hq, nt.qc, nt.qn, nt.qp, ctx->stream);
  // Chinese-remaindering tables for the same primes.
  // Rows 0..K of the prefix products: row K (the product of all K primes of
  // a pair that uses every table prime) gives floor(P / 2) to the limb kernel.
  std::vector<int32_t> poff(nt.K + 2, 0);
  for (int k = 0; k <= nt.K; ++k) poff[k + 1] = poff[k] + p16_row(k);
  if (e == cudaSuccess) e = cudaMalloc(&nt.wtab, std::max<size_t>(1, (size_t)nt.K * (nt.K - 1) / 2) * 4);
  if (e == cudaSuccess) e = cudaMalloc(&nt.p16, (size_t)poff[nt.K + 1] * 2);
  if (e == cudaSuccess) e = cudaMalloc(&nt.poff, (size_t)(nt.K + 2) * 4);
  if (e == cudaSuccess) e = cudaMalloc(&nt.nh, (size_t)(nt.K + 1) * 4);
  // Prefix products P_k = p_0 ... p_{k-1} as 16-bit digits (row k at poff[k],
  // zero padded to its reserved length; read as 32-bit limbs by the limb
  // kernels) and nh[k] = digits up to the top non-zero one, built on the
  // host: P_{k+1} = P_k p_k on 32-bit limbs.
  std::vector<uint16_t> p16((size_t)poff[nt.K + 1], 0);
  std::vector<int32_t> nh(nt.K + 1, 0);
  {
    std::vector<uint32_t> limbs(1, 1u);
    for (int k = 0; k <= nt.K; ++k) {
      uint16_t *row = p16.data() + poff[k];
      const int reserved = poff[k + 1] - poff[k];
      int top = 0;
      for (int i = 0; i < reserved && (i >> 1) < (int)limbs.size(); ++i) {
        const uint32_t d = (i & 1) ? (limbs[i >> 1] >> 16) : (limbs[i >> 1] & 0xffffu);
        row[i] = (uint16_t)d;
        if (d) top = i + 1;
      }
      nh[k] = top;
      if (k == nt.K) break;
      uint64_t carry = 0;
      for (uint32_t &l : limbs) {
        const uint64_t v = (uint64_t)l * ctx->primes[k] + carry;
        l = (uint32_t)v;
        carry = v >> 32;
      }
      if (carry) limbs.push_back((uint32_t)carry);
    }
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(nt.poff, poff.data(), poff.size() * 4, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(nt.p16, p16.data(), p16.size() * 2, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(nt.nh, nh.data(), nh.size() * 4, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = launch_crt_tables(ctx->d_mods, nt.K, nt.wtab, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    free_tables(nt);
    return rs_fail(ctx, rs_cuda_code(e), std::string("point tables: ") + cudaGetErrorString(e));
  }
  nt.h_nh = nh;
  if (t.finv) ctx->retired.push_back(t);
  t = nt;
  return RS_OK;
}

// ------------------------------------------------------------------ batches

void rs_free_batch(rs_batch *b) {
  if (!b) return;
  DevGuard dg(b->ctx->device);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  for (auto &e : b->ev)
    if (e) cudaEventDestroy(e);
  for (auto &e : b->fev)
    if (e) cudaEventDestroy(e);
  for (auto &e : b->jev)
    if (e) cudaEventDestroy(e);
  if (b->arena) {
    if (b->opt.stream_ordered)
      cudaFreeAsync(b->arena, b->stream);
    else
      cudaFree(b->arena);
  }
  if (b->own_host) {
    if (b->h_in) cudaFreeHost(b->h_in);
    if (b->h_out) cudaFreeHost(b->h_out);
  }
  delete b;
}

void rs_batch_sizes(const std::vector<PairPlan> &plans, const rs_bipoly *f, const rs_bipoly *g,
                    int64_t *in_words, int64_t *out_words, int64_t *device_bytes) {
  int64_t in = 0, out = 0, img = 0, meta = 0, tiles = 0, g2 = 0, g3 = 0, xl = 0, cy = 0, g3d = 0, g3b = 0;
  int64_t t_items = 0, t_bytes = 0;  // tensor-core G2 work items and buffers, if every pair takes that form
  for (size_t i = 0; i < plans.size(); ++i) {
    in += rs_input_words(f[i]) + rs_input_words(g[i]);
    const PairPlan &p = plans[i];
    if (p.status != RS_OK || p.trivial_zero) continue;
    const int64_t chunks = (p.Lout + 15) / 16;
    out += (int64_t)p.N * p.Lout + 2;
    xl += (int64_t)p.N * 16 * chunks;
    cy += (int64_t)p.N * chunks;
    img += (int64_t)p.K * 2 * ((p.N + 1) / 2);
    meta += p.f.my + p.g.my + 2;
    tiles += (int64_t)p.K * (((p.N + 1) / 2 + 15) / 16);
    g2 += p.K;
    const int64_t mt = (((p.N + 1) / 2 + 63) / 64) * 64;
    t_items += (int64_t)p.K * (mt / 64);
    t_bytes += (int64_t)p.K * mt * 2 * (4 * 2 + 4);  // two rows: four bf16 digits and one product per input
    t_bytes += (int64_t)((p.N + 127) / 128) * (((p.K + 63) / 64) * 65536 + 8);  // tensor-core CRT digit rows
    g3 += (p.N + 127) / 128;
    g3d += (p.N + 31) / 32;  // digit tiles
    g3b += (p.N + 127) / 128 * chunks;
  }
  // inputs plus room for the static tables (descriptors, tiles, task lists)
  // that rs_build_batch packs behind them in borrowed pinned staging
  const int64_t stat = meta * 2 + (int64_t)plans.size() * (int64_t)(sizeof(PairDesc) / 4) + tiles * 4 +
                       g2 * 2 + g3 * 2 + g3d * 4 + g3b * 4 + 8 * 4 + g2 * 4 + g2 * 8 + t_items * 2;
  *in_words = in + stat;
  *out_words = out + 1;
  *device_bytes = (int64_t)(align_up(in * 4) + align_up(meta * 8) + align_up(plans.size() * sizeof(PairDesc)) +
                            align_up(tiles * sizeof(Tile)) + kAlign + 2 * align_up(img * 4) +
                            align_up(xl * 4) + align_up(out * 4) + align_up(cy * 8) + align_up(g2 * 8) +
                            align_up(g3 * 8) + align_up(g3d * 8) + align_up(g3b * 16) + kAlign +
                            align_up(g2 * 16) + align_up(g2 * 32) + align_up(t_items * 8) + align_up(t_bytes));
}

int rs_build_batch(rs_ctx *ctx, int n, const rs_bipoly *f, const rs_bipoly *g,
                   std::vector<PairPlan> &&plans, const RsBatchOpts &opt, rs_batch **out) {
  rs_batch *b = new rs_batch();
  b->ctx = ctx;
  b->n = n;
  b->opt = opt;
  b->stream = opt.stream ? opt.stream : ctx->stream;
  b->plans = std::move(plans);
  b->dev_index.assign(n, -1);
  memset(&b->info, 0, sizeof(b->info));
  b->info.pairs = n;
  const bool images_only = opt.images_only;

  std::vector<int2> meta;
  std::vector<int> order;
  b->in_f.assign(n, -1);
  b->in_g.assign(n, -1);
  int maxM = 1, maxK = 0, maxDx = 0;  // largest point-pair count, prime count, x-degree
  for (int i = 0; i < n; ++i) {
    b->in_f[i] = b->in_words;
    b->in_words += rs_input_words(f[i]);
    b->in_g[i] = b->in_words;
    b->in_words += rs_input_words(g[i]);
    const PairPlan &p = b->plans[i];
    if (p.status != RS_OK || p.trivial_zero) continue;
    PairDesc d;
    memset(&d, 0, sizeof(d));
    d.my = p.f.my;
    d.ny = p.g.my;
    d.N = p.N;
    d.NI = 2 * ((p.N + 1) / 2);
    d.K = p.Kcrt > 0 ? std::min(p.Kcrt, p.K) : p.K;  // read by the CRT kernels only
    d.Lf = p.f.L;
    d.Lg = p.g.L;
    d.fstride = p.f.stride;
    d.gstride = p.g.stride;
    d.fnc = p.f.nc;
    d.gnc = p.g.nc;
    d.Lout = p.Lout;
    d.mxf = p.f.mx;
    d.mxg = p.g.mx;
    d.f_off = b->in_f[i];
    d.g_off = b->in_g[i];
    d.meta_off = (int64_t)meta.size();
    int start = 0;
    for (int j = 0; j <= p.f.my; ++j) {
      meta.push_back(make_int2(start, p.f.dx[j]));
      start += p.f.dx[j] + 1;
    }
    for (int j = 0; j <= p.g.my; ++j) {
      meta.push_back(make_int2(start, p.g.dx[j]));
      start += p.g.dx[j] + 1;
    }
    d.img_off = b->img_words;
    b->img_words += (int64_t)p.K * d.NI;
    d.out_off = b->out_words;
    b->out_words += (int64_t)p.N * p.Lout;
    const int64_t chunks = (p.Lout + 15) / 16;
    d.xl_off = b->xl_words;
    b->xl_words += (int64_t)p.N * 16 * chunks;
    d.cy_off = b->cy_words;
    b->cy_words += (int64_t)p.N * chunks;
    b->dev_index[i] = (int)b->descs.size();
    b->descs.push_back(d);
    order.push_back(i);
    maxM = std::max(maxM, d.NI / 2);
    maxK = std::max(maxK, p.K);
    maxDx = std::max(maxDx, std::max(p.f.mx, p.g.mx));
    b->info.images += (int64_t)p.K * d.NI;
    b->info.primes_total += p.K;
    b->info.coeffs_total += p.N;
    const double imgs = (double)p.K * d.NI;
    // per image: half of the evaluation (the two images of a point pair share
    // the even and odd parts) plus one product per coefficient to combine them
    if (ctx->cfg.univariate == 1) {  // Schur variant: Horner per coefficient, 4 r (r + 1) products
      const double r = (double)p.f.my + p.g.my;
      b->info.modmul_eval += imgs * ((double)(p.f.my + 1) * (p.f.mx + 1) + (double)(p.g.my + 1) * (p.g.mx + 1));
      b->info.modmul_prs += imgs * 4.0 * r * (r + 1.0);
    } else {
      b->info.modmul_eval += imgs * (0.5 * (p.f.nc + p.g.nc) + (p.f.my + 1) + (p.g.my + 1));
      b->info.modmul_prs += imgs * 2.0 * prs_updates(p.f.my, p.g.my);
    }
    b->info.modmul_interp += (double)p.K * ((double)d.NI * d.NI / 2 + 8.0 * d.NI);  // two interpolations of NI / 2
    b->info.modmul_crt += (double)p.N * ((double)d.K * (d.K - 1) + d.K);
  }
  b->shape_off = b->out_words;  // per pair (1 + degree, limbs), written by the last CRT kernel
  b->status_off = b->shape_off + 2 * (int64_t)b->descs.size();
  if (!images_only) b->out_words += 2 * (int64_t)b->descs.size() + 1;  // + the device status word
  if (images_only) b->out_words = std::max(b->out_words, b->img_words);

  // G1 tiles grouped by register-capacity class; costliest pairs first.
  std::sort(order.begin(), order.end(), [&](int x, int y) {
    const PairPlan &a = b->plans[x], &c = b->plans[y];
    double ca = (double)a.K * a.N * (a.f.nc + a.g.nc + 2.0 * a.f.my * a.g.my);
    double cc = (double)c.K * c.N * (c.f.nc + c.g.nc + 2.0 * c.f.my * c.g.my);
    return ca > cc;
  });
  // Tile width and schedule per class: forced by the options or the context,
  // else the tuner's cached choice (timed now when missing and allowed), else
  // 128 points on a persistent grid.
  std::vector<Tile> tiles;
  for (int cap = 8; cap <= 72; cap += 8) {
    std::vector<int> members;
    int cmaxN = 0;
    int64_t cimages = 0;
    for (int i : order)
      if (g1_supported_cap(b->plans[i].cap) == cap) {
        members.push_back(i);
        cmaxN = std::max(cmaxN, b->plans[i].N);
        cimages += (int64_t)b->plans[i].K * b->plans[i].N;
      }
    if (members.empty()) continue;
    RsG1Choice ch;
    if (opt.g1_threads > 0) {
      ch.threads = opt.g1_threads;
    } else if (ctx->cfg.tile_points > 0) {
      ch.threads = ctx->cfg.tile_points;
    } else {
      const int64_t key = rs_tune_key(ctx->sms, cap, cmaxN, cimages);
      if (!rs_tune_find(key, &ch) && opt.tune && ctx->cfg.autotune && ctx->cfg.univariate == 0) {
        const int rc = rs_tune_g1(ctx, f, g, b->plans, members, key, &ch);
        if (rc != RS_OK) {
          rs_free_batch(b);
          return rc;
        }
      }
    }
    ch.persistent = (ch.persistent && opt.persistent) ? 1 : 0;
    if (opt.g1_threads > 0 || ctx->cfg.tile_points > 0) ch.persistent = opt.persistent ? 1 : 0;
    const int T = ch.threads;
    RsClassLaunch cl;
    cl.cap = cap;
    cl.threads = T;
    cl.persistent = ch.persistent;
    cl.tile_off = (int64_t)tiles.size();
    // Work items of `run` consecutive chunks of T / 2 point pairs: the block
    // stages a (pair, prime)'s coefficients once per item and walks its
    // chunks.  Runs are as long as the class allows while it keeps at least
    // 16 items per SM for the scheduler to balance.
    int64_t chunks = 0;
    for (int i : members) chunks += (int64_t)b->plans[i].K * (((b->plans[i].N + 1) / 2 + T / 2 - 1) / (T / 2));
    const int run = (int)std::max<int64_t>(1, chunks / (16 * (int64_t)ctx->sms));
    for (int i : members) {
      const PairPlan &p = b->plans[i];
      cl.cost += (double)p.K * p.N * (p.f.nc + p.g.nc + 2.0 * p.f.my * p.g.my);
      cl.smem = std::max(cl.smem, (size_t)rs_g1_staged_words(p, cap, T) * 4);
      const int M = (p.N + 1) / 2;  // point pairs: two threads each
      for (int k = 0; k < p.K; ++k) {
        if (ctx->cfg.univariate == 0) {
          for (int x0 = 0; x0 < M; x0 += run * (T / 2))
            tiles.push_back(Tile{b->dev_index[i], k, x0, std::min(run * (T / 2), M - x0)});
        } else {
          for (int x0 = 0; x0 < M; x0 += T / 2) tiles.push_back(Tile{b->dev_index[i], k, x0, std::min(T / 2, M - x0)});
        }
      }
    }
    cl.ntiles = (int)((int64_t)tiles.size() - cl.tile_off);
    if (cl.ntiles > 0) b->classes.push_back(cl);
  }
  std::stable_sort(b->classes.begin(), b->classes.end(),
                   [](const RsClassLaunch &x, const RsClassLaunch &y) { return x.cost > y.cost; });
  if (ctx->cfg.univariate == 1 && !tiles.empty()) {
    b->schur = true;
    b->ntiles_all = (int)tiles.size();
    int rmax = 0;
    size_t staged = 0, fb = 0;
    for (int i : order) {
      const PairPlan &p = b->plans[i];
      const int r = p.f.my + p.g.my;
      rmax = std::max(rmax, r);
      staged = std::max(staged, (size_t)((p.f.my + 1) * (p.f.mx + 1) + (p.g.my + 1) * (p.g.mx + 1)) * 4);
      fb = std::max(fb, (size_t)((size_t)r * r + r + r + 2) * 4);
    }
    b->schur_slots = std::max(1, (rmax + 31) / 32);
    b->schur_smem = staged;
    b->schur_fb_smem = fb;
    if (b->schur_slots > RS_G1S_MAX_SLOTS || staged > 227 * 1024 || fb > 227 * 1024) {
      rs_free_batch(b);
      return rs_fail(ctx, RS_ERR_LIMIT, "Schur variant: m_y + n_y or the staged coefficients exceed its limits");
    }
  }
  std::vector<int2> g2, g3;
  std::vector<int> byN(order);
  std::sort(byN.begin(), byN.end(), [&](int x, int y) { return b->plans[x].N > b->plans[y].N; });
  // G2 launches by point count: each thread owns one pair of output blocks
  // of the convolutions per round; a (pair, prime) gets the fewest rounds
  // with at most 256 threads, and the fewest warps for them, so the threads
  // of a block carry equal work (classes of 32, 64, ..., 256 threads).
  // Pairs whose transform-based G2 is cheaper go to one launch per transform
  // length instead (256 threads, shared memory 3 N + 2^lg words).
  // The form is chosen per transform-length group: forced by the context or
  // the options, else the tuner's cached choice (timed now when missing and
  // allowed; groups with lg < 7, under 64 point pairs, keep the model's
  // choice), else the model.
  std::vector<int> g2lg(n, 0), g2t_lg(n, 0);  // transform / tensor-core length group per pair
  int bhatK[RS_NTT_LGMAX + 1] = {};
  const bool g2tri = ctx->cfg.g2_form == 3;  // triangular factorisation of the Vandermonde system
  if (g2tri && !images_only && !order.empty()) {
    RsG2Class gc;
    gc.lg = -1;
    gc.off = (int64_t)g2.size();
    int cmaxN = 0;
    for (int i : byN) {
      cmaxN = std::max(cmaxN, b->plans[i].N);
      for (int k = 0; k < b->plans[i].K; ++k) g2.push_back(make_int2(b->dev_index[i], k));
    }
    gc.count = (int)((int64_t)g2.size() - gc.off);
    gc.smem = (size_t)(4 * cmaxN + 97) * 4;
    if (gc.smem > 227 * 1024) {
      rs_free_batch(b);
      return rs_fail(ctx, RS_ERR_LIMIT, "g2_form 3: D + 1 above the shared-memory limit of the form (14,000)");
    }
    b->g2cls.push_back(gc);
  }
  if (!images_only && !g2tri) {
    std::vector<std::vector<int>> bylg(RS_NTT_LGMAX + 1);
    for (int i : byN) {
      const int lg = rs_g2_len((b->plans[i].N + 1) / 2);
      if (lg) bylg[lg].push_back(i);
    }
    for (int lg = 1; lg <= RS_NTT_LGMAX; ++lg) {
      if (bylg[lg].empty()) continue;
      double cd = 0.0, cn = 0.0;
      int64_t images = 0;
      for (int i : bylg[lg]) {
        const PairPlan &p = b->plans[i];
        cd += p.K * rs_g2_cost((p.N + 1) / 2, 0);
        cn += p.K * rs_g2_cost((p.N + 1) / 2, 1);
        images += (int64_t)p.K * p.N;
      }
      const int model = cn < cd ? 1 : 0;
      int form = model;
      if (ctx->cfg.g2_form == 1 || ctx->cfg.g2_form == 2 || ctx->cfg.g2_form == 4) {
        form = ctx->cfg.g2_form == 2 ? 1 : ctx->cfg.g2_form == 4 ? 2 : 0;
      } else if (opt.g2_force >= 0) {
        form = opt.g2_force;
      } else if (lg >= 7) {
        const int64_t key = rs_tune_key_g2(ctx->sms, lg, images);
        RsG1Choice c;
        if (rs_tune_find(key, &c)) {
          form = c.threads;
        } else if (opt.tune && ctx->cfg.autotune) {
          const int rc = rs_tune_g2(ctx, f, g, b->plans, bylg[lg], key, model, &form);
          if (rc != RS_OK) {
            rs_free_batch(b);
            return rc;
          }
        }
      }
      if (!form) continue;
      if (form == 2) {
        for (int i : bylg[lg]) g2t_lg[i] = lg;
        continue;
      }
      for (int i : bylg[lg]) {
        g2lg[i] = lg;
        bhatK[lg] = std::max(bhatK[lg], b->plans[i].K);
      }
    }
  }
  // One tensor-core class over every pair whose length group chose that
  // form: for every prime k, the pairs with K > k in decreasing point count
  // (so a tile's rows have similar lengths), 64 to a row tile
  // (rows 2 slot, 2 slot + 1: even and odd part); a tile's length is its
  // first pair's point-pair count rounded up to 64.  Work items: every 64
  // outputs of every tile, tiles by decreasing length, outputs from the top
  // (the longest items first; a tile's items run close together in time,
  // so its operand digits are read from L2).
  std::vector<G2tTask> g2t_tasks;
  std::vector<G2tRowTile> g2t_rts;
  std::vector<G2tItem> g2t_items;
  int64_t g2t_y_words = 0;
  int g2t_kmax = 0, g2t_tiles = 0;
  b->g2t_x_elems = 0;
  std::vector<int> g2t_mem;
  for (int i : byN)
    if (g2t_lg[i] > 0) g2t_mem.push_back(i);
  if (!images_only && !g2tri && !g2t_mem.empty()) {
    const std::vector<int> &mem = g2t_mem;
    RsG2Class gc;
    gc.lg = g2t_lg[mem[0]];
    gc.tensor = true;
    gc.t_task_off = (int64_t)g2t_tasks.size();
    gc.t_item_off = (int64_t)g2t_items.size();
    const int rt0 = (int)g2t_rts.size();
    int kmax = 0;
    for (int i : mem) kmax = std::max(kmax, b->plans[i].K);
    for (int k = 0; k < kmax; ++k) {
      std::vector<int> rows;
      for (int i : mem)
        if (b->plans[i].K > k) rows.push_back(i);
      for (size_t c0 = 0; c0 < rows.size(); c0 += 64) {
        const int cnt = (int)std::min<size_t>(64, rows.size() - c0);
        G2tRowTile rt;
        memset(&rt, 0, sizeof(rt));
        rt.prime = k;
        rt.mt = (((b->plans[rows[c0]].N + 1) / 2 + 63) / 64) * 64;
        rt.rows = 2 * cnt;
        rt.x_off = b->g2t_x_elems;
        rt.y_off = g2t_y_words;
        b->g2t_x_elems += (int64_t)(rt.mt / 64) * 32768;
        g2t_y_words += (int64_t)128 * rt.mt;
        const int rti = (int)g2t_rts.size();
        g2t_rts.push_back(rt);
        for (int sl = 0; sl < cnt; ++sl) {
          G2tTask t;
          t.pair = b->dev_index[rows[c0 + sl]];
          t.prime = k;
          t.rt = rti;
          t.slot = sl;
          g2t_tasks.push_back(t);
          gc.t_maxM = std::max(gc.t_maxM, (b->plans[rows[c0 + sl]].N + 1) / 2);
        }
        g2t_tiles = std::max(g2t_tiles, rt.mt / 32);
      }
    }
    g2t_kmax = std::max(g2t_kmax, kmax);
    std::vector<int> ord;
    for (int r = rt0; r < (int)g2t_rts.size(); ++r) ord.push_back(r);
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return g2t_rts[x].mt > g2t_rts[y].mt; });
    for (int r : ord)
      for (int t0 = g2t_rts[r].mt - 64; t0 >= 0; t0 -= 64) g2t_items.push_back(G2tItem{r, t0});
    gc.t_ntask = (int)((int64_t)g2t_tasks.size() - gc.t_task_off);
    gc.t_nitem = (int)((int64_t)g2t_items.size() - gc.t_item_off);
    gc.count = gc.t_ntask;
    b->g2cls.push_back(gc);
  }
  for (int lg = RS_NTT_LGMAX; lg > 0; --lg) {
    if (!bhatK[lg]) continue;
    RsG2Class gc;
    gc.lg = lg;
    gc.off = (int64_t)g2.size();
    int cmaxN = 0;
    for (int i : byN) {
      if (g2lg[i] != lg) continue;
      cmaxN = std::max(cmaxN, (b->plans[i].N + 1) / 2);  // point pairs
      for (int k = 0; k < b->plans[i].K; ++k) g2.push_back(make_int2(b->dev_index[i], k));
    }
    gc.count = (int)((int64_t)g2.size() - gc.off);
    gc.smem = (size_t)(4 * ((cmaxN + 3) & ~3) + 2 * (1 << lg)) * 4;
    b->g2cls.push_back(gc);
  }
  const int nlg = (int)b->g2cls.size();
  for (int c = 0; c < 8 && !g2tri; ++c) {
    RsG2Class gc;
    gc.threads = 32 * (c + 1);
    gc.off = (int64_t)g2.size();
    int cmaxN = 0;
    for (int i : byN) {
      const PairPlan &p = b->plans[i];
      if (g2lg[i] || g2t_lg[i]) continue;
      const int npair = (((p.N + 1) / 2 + RS_CONV_R - 1) / RS_CONV_R + 1) / 2;  // output-block pairs
      const int rounds = (npair + 255) / 256;
      const int warps = (npair + 32 * rounds - 1) / (32 * rounds);
      if (warps - 1 != c) continue;
      cmaxN = std::max(cmaxN, (p.N + 1) / 2);
      for (int k = 0; k < p.K; ++k) g2.push_back(make_int2(b->dev_index[i], k));
    }
    gc.count = (int)((int64_t)g2.size() - gc.off);
    gc.smem = (size_t)4 * (cmaxN + 2 * RS_G2_PAD) * 4;
    if (gc.count > 0 && !images_only) b->g2cls.insert(b->g2cls.begin() + nlg, gc);  // largest point counts first
  }
  // CRT digits in tiles of 32 coefficients; limbs in blocks of 128
  // coefficients by chunks of 16 output limbs.
  // Digit tiles hold 32 coefficients, or 16 when 32-wide tiles would be
  // fewer than two per SM (few coefficients with many primes each).
  std::vector<int2> g3d;
  std::vector<int4> g3b;  // CRT limb chunks: 128 coefficients x one chunk per block
  // With enough coefficients for one thread each to fill the GPU, the digits
  // take one thread per coefficient (no warp waits on a serial triangle);
  // otherwise the tiled kernel spreads each coefficient's work over a block.
  {
    int64_t nt32 = 0, ncoef = 0;
    for (int i : order) {
      nt32 += (b->plans[i].N + 31) / 32;
      ncoef += b->plans[i].N;
    }
    b->g3_jt = nt32 < 2 * (int64_t)ctx->sms ? 16 : 32;
    b->g3_perthread = ncoef >= (int64_t)RS_G3P_MIN_COEF_PER_SM * ctx->sms;
    // Otherwise the digits go to the tensor cores when a pair has enough
    // primes for the per-block products to matter (two 64-prime blocks) and
    // the 128-coefficient tiles fill half the SMs, or a pair has so many
    // primes that the products dominate; with few tiles and a few hundred
    // primes the CUDA-core tiles of 16 coefficients spread the work wider.
    int64_t nt128 = 0;
    for (int i : order) nt128 += (b->plans[i].N + 127) / 128;
    b->g3_tensor = !b->g3_perthread && !images_only && ctx->cfg.crt_form != 1 &&
                   (ctx->cfg.crt_form == 2 ||
                    (maxK >= RS_G3M_MIN_K && (2 * nt128 >= ctx->sms || maxK >= RS_G3M_WIDE_K)));
  }
  for (int i : order) {
    const PairPlan &p = b->plans[i];
    const int di = b->dev_index[i], chunks = (p.Lout + 15) / 16;
    for (int j = 0; j < p.N; j += 128) g3.push_back(make_int2(di, j));
    for (int j = 0; j < p.N; j += b->g3_jt) g3d.push_back(make_int2(di, j));  // digit tiles
    for (int c = 0; c < chunks; ++c)
      for (int j = 0; j < p.N; j += 128) g3b.push_back(make_int4(di, j, c, 0));
  }
  std::vector<int2> yun;  // square-free factorisation tasks: every (pair, prime), pairs in order
  if (opt.yun_maxm > 0 && !images_only) {
    int maxNp = 1;
    for (int i = 0; i < n; ++i) {
      if (b->dev_index[i] < 0) continue;
      maxNp = std::max(maxNp, b->plans[i].N);
      for (int k = 0; k < b->plans[i].K; ++k) yun.push_back(make_int2(b->dev_index[i], k));
    }
    b->yun_wstride = ((int64_t)maxNp + 3) & ~(int64_t)3;
    b->yun_ostride = ((int64_t)maxNp + 2 * opt.yun_maxm + 2 + 3) & ~(int64_t)3;
  }
  // Tensor-core CRT digits: each task (128 coefficients of a pair) owns its
  // operand digit rows, one 64 KB chunk per 64 of the pair's primes.
  std::vector<int64_t> g3m_xoff;
  b->g3m_x_elems = 0;
  if (b->g3_tensor) {
    for (const int2 &t : g3) {
      g3m_xoff.push_back(b->g3m_x_elems);
      b->g3m_x_elems += g3m_tile_elems(b->descs[t.x].K);
    }
  }
  b->nyun = (int)yun.size();
  b->ng2 = images_only ? 0 : (int)g2.size();
  b->ng3 = images_only ? 0 : (int)g3.size();
  b->ng3d = images_only ? 0 : (int)g3d.size();
  b->ng3b = images_only ? 0 : (int)g3b.size();
  b->kmax = maxK;
  b->g2smem = (size_t)4 * (maxM + 2 * RS_G2_PAD) * 4;
  b->info.input_bytes = b->in_words * 4;
  b->info.output_bytes = b->out_words * 4;
  b->info.kernel_launches = (b->schur ? 2 : (int64_t)b->classes.size()) + (int64_t)b->g2cls.size() + (b->ng3d > 0) +
                            (b->nyun > 0) +
                            (b->ng3b > 0) +
                            (b->ng3 > 0);
  for (const auto &gc : b->g2cls)
    if (gc.tensor) b->info.kernel_launches += 4;  // five launches per tensor-core class

  int rc = RS_OK;
  if (!order.empty()) rc = rs_ensure_tables(ctx, maxK, maxM, maxDx);
  for (int lg = 1; lg <= RS_NTT_LGMAX && rc == RS_OK; ++lg)
    if (bhatK[lg]) rc = rs_ensure_bhat(ctx, lg, bhatK[lg]);
  if (rc == RS_OK && g2t_kmax > 0) rc = rs_ensure_g2t_btile(ctx, g2t_kmax, g2t_tiles);
  if (rc == RS_OK && b->g3_tensor) rc = rs_ensure_g3m_wtiles(ctx, (maxK + 63) / 64);
  if (rc == RS_OK && b->g3_tensor) rc = rs_ensure_g3l_tiles(ctx, (maxK + 63) / 64);
  if (rc == RS_OK && b->g3_tensor) {
    // The limbs then come from the tensor cores too: one task per (digit
    // task, unit of 64 limbs) instead of the limb chunks, with the chunks
    // from the first whose prefix products reach the unit; the longest first.
    std::vector<int32_t> cb;
    {
      std::lock_guard<std::mutex> lock(ctx->tab_mu);
      cb = ctx->h_g3l_cbase;
    }
    const int KBt = (int)cb.size() - 1;
    std::vector<std::pair<int, int4>> lt;
    for (size_t ti = 0; ti < g3.size(); ++ti) {
      const PairDesc &pd = b->descs[g3[ti].x];
      const int KBp = (pd.K + 63) / 64, units = (pd.Lout + 63) / 64;
      int lo = 0;
      for (int u = 0; u < units; ++u) {
        while (lo < KBt && cb[lo + 1] - cb[lo] - 1 < u) ++lo;
        lt.push_back({KBp > lo ? KBp - lo : 0, make_int4((int)ti, u, lo, 0)});
      }
    }
    std::stable_sort(lt.begin(), lt.end(), [](const std::pair<int, int4> &x, const std::pair<int, int4> &y) {
      return x.first > y.first;
    });
    g3b.clear();
    for (const auto &x : lt) g3b.push_back(x.second);
    b->ng3b = (int)g3b.size();
  }
  if (rc != RS_OK) {
    rs_free_batch(b);
    return rc;
  }
  DevGuard dg(ctx->device);
  size_t off = 0;  // one device arena carved into every buffer of the batch
  auto carve = [&](size_t bytes) {
    size_t o = off;
    off += align_up(bytes);
    return o;
  };
  const size_t o_in = carve(b->in_words * 4), o_meta = carve(meta.size() * sizeof(int2)),
               o_pairs = carve(b->descs.size() * sizeof(PairDesc)), o_tiles = carve(tiles.size() * sizeof(Tile)),
               o_cnt = carve(16 * sizeof(int32_t)), o_num = carve(b->img_words * 4), o_den = carve(b->img_words * 4),
               o_xl = carve(std::max(b->xl_words, b->out_words) * 4), o_out = carve(b->out_words * 4),
               o_g2 = carve(g2.size() * sizeof(int2)), o_g3 = carve(g3.size() * sizeof(int2)),
               o_st = carve(ST_COUNT * sizeof(unsigned long long)), o_cy = carve(b->cy_words * 8),
               o_g3d = carve(g3d.size() * sizeof(int2)), o_yt = carve(yun.size() * sizeof(int2)),
               o_yo = carve((size_t)b->nyun * b->yun_ostride * 4), o_yw = carve((size_t)b->nyun * 8 * b->yun_wstride * 4),
               o_g3b = carve(g3b.size() * sizeof(int4)), o_fail = carve(b->schur ? b->img_words * sizeof(int2) : 0),
               o_tt = carve(g2t_tasks.size() * sizeof(G2tTask)), o_trt = carve(g2t_rts.size() * sizeof(G2tRowTile)),
               o_tit = carve(g2t_items.size() * sizeof(G2tItem)), o_tx = carve(b->g2t_x_elems * sizeof(uint16_t)),
               o_ty = carve(g2t_y_words * 4), o_g3mx = carve(b->g3m_x_elems * sizeof(uint16_t)),
               o_g3mo = carve(g3m_xoff.size() * sizeof(int64_t));
  cudaError_t e = opt.stream_ordered ? cudaMallocAsync(&b->arena, off, b->stream) : cudaMalloc(&b->arena, off);
  if (e != cudaSuccess) {
    b->arena = nullptr;
    rs_free_batch(b);
    return rs_fail(ctx, rs_cuda_code(e), std::string("device arena: ") + cudaGetErrorString(e));
  }
  char *base = static_cast<char *>(b->arena);
  b->d_in = (uint32_t *)(base + o_in);
  b->d_meta = (int2 *)(base + o_meta);
  b->d_pairs = (PairDesc *)(base + o_pairs);
  b->d_tiles = (Tile *)(base + o_tiles);
  b->d_counters = (int32_t *)(base + o_cnt);
  b->d_num = (uint32_t *)(base + o_num);
  b->d_den = (uint32_t *)(base + o_den);
  b->d_xl = (uint32_t *)(base + o_xl);
  b->d_out = (uint32_t *)(base + o_out);
  b->d_g2 = (int2 *)(base + o_g2);
  b->d_g3 = (int2 *)(base + o_g3);
  b->d_stats = (unsigned long long *)(base + o_st);
  b->d_cy = (int64_t *)(base + o_cy);
  b->d_g3d = (int2 *)(base + o_g3d);
  b->d_yun_tasks = (int2 *)(base + o_yt);
  b->d_yun_out = (uint32_t *)(base + o_yo);
  b->d_yun_work = (uint32_t *)(base + o_yw);
  b->d_g3b = (int4 *)(base + o_g3b);
  b->d_fail = b->schur ? (int2 *)(base + o_fail) : nullptr;
  b->d_g2t_tasks = (G2tTask *)(base + o_tt);
  b->d_g2t_rts = (G2tRowTile *)(base + o_trt);
  b->d_g2t_items = (G2tItem *)(base + o_tit);
  b->d_g2t_x = (uint16_t *)(base + o_tx);
  b->d_g2t_y = (uint32_t *)(base + o_ty);
  b->d_g3m_x = (uint16_t *)(base + o_g3mx);
  b->d_g3m_xoff = (int64_t *)(base + o_g3mo);
  // Tensor-core operand digits: rows and inputs beyond each pair's points
  // stay zero for the batch's life (the kernels write only inputs < M).
  if (b->g3m_x_elems) e = cudaMemsetAsync(b->d_g3m_x, 0, b->g3m_x_elems * sizeof(uint16_t), b->stream);
  if (e == cudaSuccess && b->g2t_x_elems)
    e = cudaMemsetAsync(b->d_g2t_x, 0, b->g2t_x_elems * sizeof(uint16_t), b->stream);
  if (e != cudaSuccess) {
    rs_free_batch(b);
    return rs_fail(ctx, rs_cuda_code(e), std::string("tensor-core operands: ") + cudaGetErrorString(e));
  }

  if (opt.h_in && opt.h_in_words >= b->in_words && opt.h_out && opt.h_out_words >= b->out_words) {
    b->h_in = opt.h_in;
    b->h_out = opt.h_out;
  } else {
    b->own_host = true;
    if (b->in_words && cudaMallocHost((void **)&b->h_in, b->in_words * 4) != cudaSuccess) rc = RS_ERR_NOMEM;
    if (rc == RS_OK && b->out_words && cudaMallocHost((void **)&b->h_out, b->out_words * 4) != cudaSuccess)
      rc = RS_ERR_NOMEM;
    if (rc != RS_OK) {
      rs_free_batch(b);
      return rs_fail(ctx, rc, "cudaMallocHost (staging)");
    }
  }
  // Static per-batch tables, ordered on the batch stream.  With borrowed
  // pinned staging large enough they are packed behind the inputs and copied
  // without waiting; otherwise they are copied from pageable memory and the
  // stream is synchronised before the host vectors go away.
  struct Piece {
    void *dst;
    const void *src;
    size_t bytes;
  };
  const Piece pieces[] = {{b->d_meta, meta.data(), meta.size() * sizeof(int2)},
                          {b->d_pairs, b->descs.data(), b->descs.size() * sizeof(PairDesc)},
                          {b->d_tiles, tiles.data(), tiles.size() * sizeof(Tile)},
                          {b->d_g2, g2.data(), g2.size() * sizeof(int2)},
                          {b->d_g3, g3.data(), g3.size() * sizeof(int2)},
                          {b->d_g3d, g3d.data(), g3d.size() * sizeof(int2)},
                          {b->d_yun_tasks, yun.data(), yun.size() * sizeof(int2)},
                          {b->d_g3b, g3b.data(), g3b.size() * sizeof(int4)},
                          {b->d_g2t_tasks, g2t_tasks.data(), g2t_tasks.size() * sizeof(G2tTask)},
                          {b->d_g2t_rts, g2t_rts.data(), g2t_rts.size() * sizeof(G2tRowTile)},
                          {b->d_g2t_items, g2t_items.data(), g2t_items.size() * sizeof(G2tItem)},
                          {b->d_g3m_xoff, g3m_xoff.data(), g3m_xoff.size() * sizeof(int64_t)}};
  size_t static_bytes = 0;
  for (const Piece &pc : pieces) static_bytes += (pc.bytes + 15) & ~(size_t)15;
  const bool pinned_static = !b->own_host && (size_t)opt.h_in_words * 4 >= (size_t)b->in_words * 4 + static_bytes;
  char *stage = pinned_static ? reinterpret_cast<char *>(b->h_in + b->in_words) : nullptr;
  for (const Piece &pc : pieces) {
    if (rc != RS_OK || pc.bytes == 0) continue;
    const void *src = pc.src;
    if (stage) {
      memcpy(stage, pc.src, pc.bytes);
      src = stage;
      stage += (pc.bytes + 15) & ~(size_t)15;
    }
    cudaError_t e2 = cudaMemcpyAsync(pc.dst, src, pc.bytes, cudaMemcpyHostToDevice, b->stream);
    if (e2 != cudaSuccess) rc = rs_fail(ctx, RS_ERR_CUDA, std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e2));
  }
  if (rc == RS_OK && !pinned_static) {
    cudaError_t e2 = cudaStreamSynchronize(b->stream);
    if (e2 != cudaSuccess) rc = rs_fail(ctx, RS_ERR_CUDA, std::string("sync: ") + cudaGetErrorString(e2));
  }
  {
    // Kernel attributes and occupancies, once per context.
    std::lock_guard<std::mutex> lock(ctx->prep_mu);
    if (rc == RS_OK && nlg > 0 && !ctx->g2n_ready) {
      cudaError_t e2 = g2n_prepare();
      if (e2 != cudaSuccess) rc = rs_fail(ctx, RS_ERR_CUDA, std::string("G2 set-up: ") + cudaGetErrorString(e2));
      ctx->g2n_ready = e2 == cudaSuccess;
    }
    if (rc == RS_OK && b->g3_tensor && !ctx->g3m_ready) {
      cudaError_t e2 = g3m_prepare();
      if (e2 != cudaSuccess) rc = rs_fail(ctx, RS_ERR_CUDA, std::string("G3 set-up: ") + cudaGetErrorString(e2));
      ctx->g3m_ready = e2 == cudaSuccess;
    }
    if (rc == RS_OK && b->g3_tensor && !ctx->g3l_ready) {
      cudaError_t e2 = g3l_prepare();
      if (e2 != cudaSuccess) rc = rs_fail(ctx, RS_ERR_CUDA, std::string("G3 set-up: ") + cudaGetErrorString(e2));
      ctx->g3l_ready = e2 == cudaSuccess;
    }
    if (rc == RS_OK && g2t_kmax > 0 && !ctx->g2t_ready) {
      cudaError_t e2 = g2t_prepare();
      if (e2 != cudaSuccess) rc = rs_fail(ctx, RS_ERR_CUDA, std::string("G2 set-up: ") + cudaGetErrorString(e2));
      ctx->g2t_ready = e2 == cudaSuccess;
    }
    if (rc == RS_OK && !b->g2cls.empty() && !ctx->g2_ready) {
      cudaError_t e2 = g2_prepare(b->g2smem);
      if (e2 != cudaSuccess) rc = rs_fail(ctx, RS_ERR_CUDA, std::string("G2 set-up: ") + cudaGetErrorString(e2));
      ctx->g2_ready = e2 == cudaSuccess;
    }
    for (auto &cl : b->classes) {
      if (rc != RS_OK) break;
      const int64_t key = ((int64_t)cl.cap << 40) | ((int64_t)cl.threads << 24) | (int64_t)((cl.smem + 1023) / 1024);
      auto it = ctx->g1_occupancy.find(key);
      int mb = 0;
      if (it != ctx->g1_occupancy.end()) {
        mb = it->second;
      } else {
        cudaError_t e2 = g1_prepare(cl.cap, cl.threads, ((cl.smem + 1023) / 1024) * 1024, &mb);
        if (e2 != cudaSuccess) {
          rc = rs_fail(ctx, RS_ERR_CUDA, std::string("G1 set-up: ") + cudaGetErrorString(e2));
          break;
        }
        ctx->g1_occupancy[key] = mb;
      }
      if (mb < 1) mb = 1;
      cl.blocks = cl.persistent ? std::min(cl.ntiles, mb * ctx->sms) : cl.ntiles;
    }
  }
  if (ctx->cfg.timing || opt.timing)
    for (auto &ev : b->ev)
      if (rc == RS_OK && cudaEventCreate(&ev) != cudaSuccess) rc = rs_fail(ctx, RS_ERR_CUDA, "cudaEventCreate");
  if (opt.fork && (b->classes.size() > 1 || b->g2cls.size() > 1)) {
    b->jev.assign(b->classes.size() + b->g2cls.size(), nullptr);
    for (auto &ev : b->fev)
      if (rc == RS_OK && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
        rc = rs_fail(ctx, RS_ERR_CUDA, "cudaEventCreate");
    for (auto &ev : b->jev)
      if (rc == RS_OK && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
        rc = rs_fail(ctx, RS_ERR_CUDA, "cudaEventCreate");
  }
  if (rc != RS_OK) {
    rs_free_batch(b);
    return rc;
  }
  *out = b;
  return RS_OK;
}

int rs_upload(rs_batch *b, const rs_bipoly *f, const rs_bipoly *g) {
  rs_ctx *ctx = b->ctx;
  for (int i = 0; i < b->n; ++i) {
    memcpy(b->h_in + b->in_f[i], f[i].coeffs, rs_input_words(f[i]) * 4);
    memcpy(b->h_in + b->in_g[i], g[i].coeffs, rs_input_words(g[i]) * 4);
  }
  if (b->in_words)
    RS_CUDA(ctx, cudaMemcpyAsync(b->d_in, b->h_in, b->in_words * 4, cudaMemcpyHostToDevice, b->stream));
  return RS_OK;
}

static cudaError_t record(cudaEvent_t e, cudaStream_t s, bool capturing) {
  return capturing ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal) : cudaEventRecord(e, s);
}

// The launches of one stage are independent (disjoint tiles or tasks): with
// fork events they run as parallel branches on the context's side streams
// (inside a captured graph: parallel graph nodes), so the tail of one launch
// overlaps the next instead of idling SMs.  Branch i of the stage uses side
// stream i mod 8 and join event j0 + i.
static cudaStream_t branch_begin(rs_batch *b, int stage, int i, cudaStream_t s, cudaError_t *e) {
  if (!b->fev[stage]) return s;
  cudaStream_t si = b->ctx->side[i % 8];
  if (*e == cudaSuccess && i == 0) *e = cudaEventRecord(b->fev[stage], s);
  if (*e == cudaSuccess) *e = cudaStreamWaitEvent(si, b->fev[stage], 0);
  return si;
}

static void branch_end(rs_batch *b, int stage, int j, cudaStream_t si, cudaError_t *e) {
  if (!b->fev[stage]) return;
  if (*e == cudaSuccess) *e = cudaEventRecord(b->jev[j], si);
}

static void join_all(rs_batch *b, int stage, int j0, int n, cudaStream_t s, cudaError_t *e) {
  if (!b->fev[stage]) return;
  for (int j = j0; j < j0 + n && *e == cudaSuccess; ++j) *e = cudaStreamWaitEvent(s, b->jev[j], 0);
}

static int enqueue(rs_batch *b, bool capturing) {
  rs_ctx *ctx = b->ctx;
  cudaStream_t s = b->stream;
  const bool timing = ctx->cfg.timing != 0 || b->opt.timing;
  RsTables tab;
  {
    std::lock_guard<std::mutex> lock(ctx->tab_mu);
    tab = ctx->tab;
  }
  RS_CUDA(ctx, cudaMemsetAsync(b->d_counters, 0, 16 * sizeof(int32_t), s));
  RS_CUDA(ctx, cudaMemsetAsync(b->d_stats, 0, ST_COUNT * sizeof(unsigned long long), s));
  if (b->g2t_x_elems > 0 || b->g3_tensor)  // the status word only the tensor-core kernels write
    RS_CUDA(ctx, cudaMemsetAsync(b->d_out + b->status_off, 0, sizeof(uint32_t), s));
  if (timing) RS_CUDA(ctx, record(b->ev[0], s, capturing));
  if (b->schur) {  // Schur variant of G1 over every tile, then the elimination fallback
    G1sArgs a;
    a.pairs = b->d_pairs;
    a.tiles = b->d_tiles;
    a.limbs = b->d_in;
    a.mods = ctx->d_mods;
    a.vtab = ctx->d_vtab;
    a.qp = tab.qp;
    a.tstride = tab.cstride;
    a.num = b->d_num;
    a.den = b->d_den;
    a.fail = b->d_fail;
    a.fail_count = b->d_counters + 15;
    a.stats = b->d_stats;
    RS_CUDA(ctx, launch_g1s(b->schur_slots, b->ntiles_all, b->schur_smem, a, s));
    RS_CUDA(ctx, launch_g1s_fallback(2 * ctx->sms, b->schur_fb_smem, a, s));
  }
  int ci = 0;
  for (const auto &cl : b->classes) {
    if (b->schur) break;
    G1Args a;
    a.pairs = b->d_pairs;
    a.tiles = b->d_tiles + cl.tile_off;
    a.ntiles = cl.ntiles;
    a.persistent = cl.persistent;
    a.counter = b->d_counters + (ci++);
    a.limbs = b->d_in;
    a.meta = b->d_meta;
    a.mods = ctx->d_mods;
    a.qc = tab.qc;
    a.qn = tab.qn;
    a.qp = tab.qp;
    a.tstride = tab.cstride;
    a.vtab = ctx->d_vtab;
    a.num = b->d_num;
    a.den = b->d_den;
    a.stats = b->d_stats;
    cudaError_t fe = cudaSuccess;
    cudaStream_t si = branch_begin(b, 0, ci - 1, s, &fe);
    RS_CUDA(ctx, fe);
    RS_CUDA(ctx, launch_g1(cl.cap, cl.threads, cl.blocks, cl.smem, a, si));
    branch_end(b, 0, ci - 1, si, &fe);
    RS_CUDA(ctx, fe);
  }
  {
    cudaError_t fe = cudaSuccess;
    if (!b->schur) join_all(b, 0, 0, (int)b->classes.size(), s, &fe);
    RS_CUDA(ctx, fe);
  }
  if (timing) RS_CUDA(ctx, record(b->ev[1], s, capturing));
  uint32_t *bhat[RS_NTT_LGMAX + 1];
  {
    std::lock_guard<std::mutex> lock(ctx->tab_mu);
    for (int l = 0; l <= RS_NTT_LGMAX; ++l) bhat[l] = ctx->bhat[l];
  }
  uint16_t *g2t_bt = nullptr;
  int g2t_tiles = 0;
  {
    std::lock_guard<std::mutex> lock(ctx->tab_mu);
    g2t_bt = ctx->g2t_bt;
    g2t_tiles = ctx->g2t_tiles;
  }
  int gi = 0;
  for (const auto &gc : b->g2cls) {
    if (gc.tensor) {
      G2tArgs at;
      at.pairs = b->d_pairs;
      at.tasks = b->d_g2t_tasks + gc.t_task_off;
      at.rts = b->d_g2t_rts;
      at.items = b->d_g2t_items + gc.t_item_off;
      at.mods = ctx->d_mods;
      at.num = b->d_num;
      at.den = b->d_den;
      at.coef = b->d_num;
      at.finv = tab.finv;
      at.gtab = tab.gtab;
      at.hq = tab.hq;
      at.tab_stride = tab.N;
      at.btile = g2t_bt;
      at.bt_tiles = g2t_tiles;
      at.x = b->d_g2t_x;
      at.y = b->d_g2t_y;
      at.err = reinterpret_cast<int32_t *>(b->d_out + b->status_off);
      at.stall = ctx->d_stall;
      const int j = (int)b->classes.size() + gi;
      cudaError_t fe = cudaSuccess;
      cudaStream_t si = branch_begin(b, 1, gi, s, &fe);
      RS_CUDA(ctx, fe);
      RS_CUDA(ctx, launch_g2t(gc.t_ntask, gc.t_nitem, gc.t_maxM, at, si));
      branch_end(b, 1, j, si, &fe);
      RS_CUDA(ctx, fe);
      ++gi;
      continue;
    }
    if (gc.lg < 0) {
      G2sArgs as;
      as.pairs = b->d_pairs;
      as.tasks = b->d_g2 + gc.off;
      as.mods = ctx->d_mods;
      as.num = b->d_num;
      as.den = b->d_den;
      as.coef = b->d_num;
      as.qp = tab.qp;
      as.tstride = tab.cstride;
      const int j = (int)b->classes.size() + gi;
      cudaError_t fe = cudaSuccess;
      cudaStream_t si = branch_begin(b, 1, gi, s, &fe);
      RS_CUDA(ctx, fe);
      RS_CUDA(ctx, launch_g2s(gc.count, gc.smem, as, si));
      branch_end(b, 1, j, si, &fe);
      RS_CUDA(ctx, fe);
      ++gi;
      continue;
    }
    if (gc.lg > 0) {
      G2nArgs an;
      an.pairs = b->d_pairs;
      an.tasks = b->d_g2 + gc.off;
      an.mods = ctx->d_mods;
      an.num = b->d_num;
      an.den = b->d_den;
      an.coef = b->d_num;
      an.finv = tab.finv;
      an.hq = tab.hq;
      an.gtab = tab.gtab;
      an.tab_stride = tab.N;
      an.tw = ctx->d_ntt_tw;
      an.bhat = bhat[gc.lg];
      an.nc = ctx->nttc;
      an.lg = gc.lg;
      const int j = (int)b->classes.size() + gi;
      cudaError_t fe = cudaSuccess;
      cudaStream_t si = branch_begin(b, 1, gi, s, &fe);
      RS_CUDA(ctx, fe);
      RS_CUDA(ctx, launch_g2n(gc.count, gc.smem, an, si));
      branch_end(b, 1, j, si, &fe);
      RS_CUDA(ctx, fe);
      ++gi;
      continue;
    }
    G2Args a2;
    a2.pairs = b->d_pairs;
    a2.tasks = b->d_g2 + gc.off;
    a2.mods = ctx->d_mods;
    a2.num = b->d_num;
    a2.den = b->d_den;
    a2.coef = b->d_num;
    a2.finv = tab.finv;
    a2.hq = tab.hq;
    a2.gtab = tab.gtab;
    a2.btab = tab.btab;
    a2.tab_stride = tab.N;
    const int j = (int)b->classes.size() + gi;
    cudaError_t fe = cudaSuccess;
    cudaStream_t si = branch_begin(b, 1, gi, s, &fe);
    RS_CUDA(ctx, fe);
    RS_CUDA(ctx, launch_g2(gc.threads, gc.count, gc.smem, a2, si));
    branch_end(b, 1, j, si, &fe);
    RS_CUDA(ctx, fe);
    ++gi;
  }
  {
    cudaError_t fe = cudaSuccess;
    join_all(b, 1, (int)b->classes.size(), (int)b->g2cls.size(), s, &fe);
    RS_CUDA(ctx, fe);
  }
  if (b->nyun) {  // square-free factorisation of R mod p, before G3 overwrites the residues
    if (timing) RS_CUDA(ctx, record(b->ev[4], s, capturing));
    YunArgs ya;
    ya.pairs = b->d_pairs;
    ya.tasks = b->d_yun_tasks;
    ya.mods = ctx->d_mods;
    ya.coef = b->d_num;
    ya.out = b->d_yun_out;
    ya.work = b->d_yun_work;
    ya.ostride = b->yun_ostride;
    ya.wstride = b->yun_wstride;
    ya.maxm = b->opt.yun_maxm;
    RS_CUDA(ctx, launch_yun(b->nyun, ya, s));
  }
  if (timing) RS_CUDA(ctx, record(b->ev[2], s, capturing));
  if (b->ng3) {
    G3Args a3;
    a3.pairs = b->d_pairs;
    a3.tasks = b->d_g3;
    a3.ctasks = b->d_g3b;
    a3.mods = ctx->d_mods;
    a3.crt = ctx->d_crt;
    a3.wtab = tab.wtab;
    a3.p16 = tab.p16;
    a3.poff = tab.poff;
    a3.nh = tab.nh;
    a3.coef = b->d_num;
    a3.xl = b->d_xl;
    a3.carry = b->d_cy;
    a3.out = b->d_out;
    a3.shape = reinterpret_cast<int32_t *>(b->d_out + b->shape_off);
    RS_CUDA(ctx, cudaMemsetAsync(a3.shape, 0, b->descs.size() * 2 * sizeof(int32_t), s));
    a3.kmax = b->kmax;
    a3.signed_digits = b->g3_tensor ? 1 : 0;
    if (b->g3_perthread) {
      RS_CUDA(ctx, launch_g3p(b->ng3, a3, b->d_g3, s));
    } else if (b->g3_tensor) {
      G3mArgs am;
      am.pairs = b->d_pairs;
      am.tasks = b->d_g3;
      am.mods = ctx->d_mods;
      am.crt = ctx->d_crt;
      am.wtab = tab.wtab;
      {
        std::lock_guard<std::mutex> lock(ctx->tab_mu);
        am.wtiles = ctx->g3m_wt;
        am.rtiles = ctx->g3m_rt;
      }
      am.coef = b->d_num;
      am.xdig = b->d_g3m_x;
      am.xoff = b->d_g3m_xoff;
      am.err = reinterpret_cast<int32_t *>(b->d_out + b->status_off);
      am.stall = ctx->d_stall;
      RS_CUDA(ctx, launch_g3m(b->ng3, am, s));
      G3lArgs al;
      al.pairs = b->d_pairs;
      al.tasks = b->d_g3;
      al.ltasks = b->d_g3b;
      al.xdig = b->d_g3m_x;
      al.xoff = b->d_g3m_xoff;
      {
        std::lock_guard<std::mutex> lock(ctx->tab_mu);
        al.btiles = ctx->g3l_bt;
        al.cbase = ctx->g3l_cbase;
      }
      al.xl = b->d_xl;
      al.carry = b->d_cy;
      al.err = am.err;
      al.stall = ctx->d_stall;
      RS_CUDA(ctx, launch_g3l(b->ng3b, al, s));
    } else {
      RS_CUDA(ctx, launch_g3t(b->ng3d, a3, b->d_g3d, s, b->g3_jt));
    }
    // the output kernel; the limb chunks unless the tensor cores formed the limbs
    RS_CUDA(ctx, launch_g3bc(b->g3_tensor ? 0 : b->ng3b, b->ng3, a3, b->d_g3, s));
  }
  if (timing) RS_CUDA(ctx, record(b->ev[3], s, capturing));
  return RS_OK;
}

int rs_run(rs_batch *b) {
  rs_ctx *ctx = b->ctx;
  DevGuard dg(ctx->device);
  if (b->opt.use_graph && !b->opt.images_only) {
    if (!b->gexec) {
      RS_CUDA(ctx, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
      int rc = enqueue(b, true);
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
      if (rc != RS_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
      }
      if (e != cudaSuccess) return rs_fail(ctx, RS_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
      e = cudaGraphInstantiate(&b->gexec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return rs_fail(ctx, RS_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    RS_CUDA(ctx, cudaGraphLaunch(b->gexec, b->stream));
  } else {
    int rc = enqueue(b, false);
    if (rc != RS_OK) return rc;
  }
  b->ran = true;
  return RS_OK;
}

int rs_fetch_async(rs_batch *b) {
  rs_ctx *ctx = b->ctx;
  if (!b->ran) return rs_fail(ctx, RS_ERR_STATE, "batch has not been run");
  if (b->out_words)
    RS_CUDA(ctx, cudaMemcpyAsync(b->h_out, b->d_out, b->out_words * 4, cudaMemcpyDeviceToHost, b->stream));
  return RS_OK;
}

// Degree and limb count of pair i's result (recorded on the device by the
// last CRT kernel and copied back with the limbs), and its limbs in the host
// staging buffer.
static const uint32_t *result_shape(rs_batch *b, int i, int *deg, int *limbs) {
  const PairPlan &p = b->plans[i];
  *deg = -1;
  *limbs = 1;
  if (p.trivial_zero) return nullptr;
  const int d = b->dev_index[i];
  const int32_t *shape = reinterpret_cast<const int32_t *>(b->h_out + b->shape_off) + 2 * (size_t)d;
  *deg = shape[0] - 1;
  *limbs = std::max(1, (int)shape[1]);
  return b->h_out + b->descs[d].out_off;
}

// The device status word copied back with the results: non-zero when a
// bounded wait of the tensor-core interpolation ran out in the last run.
static int device_status(rs_batch *b) {
  if ((b->g2t_x_elems == 0 && !b->g3_tensor) || b->out_words <= b->status_off || !b->h_out) return RS_OK;
  return b->h_out[b->status_off] ? RS_ERR_TIMEOUT : RS_OK;
}

int rs_unpack_one(rs_batch *b, int i, std::vector<uint32_t> &words, int *deg, int *limbs) {
  const PairPlan &p = b->plans[i];
  if (p.status != RS_OK) return p.status;
  if (device_status(b) != RS_OK) return RS_ERR_TIMEOUT;
  const uint32_t *w = result_shape(b, i, deg, limbs);
  words.assign((size_t)(*deg + 1) * *limbs, 0u);
  for (int j = 0; j <= *deg; ++j)
    memcpy(&words[(size_t)j * *limbs], w + (size_t)j * p.Lout, (size_t)*limbs * 4);
  return RS_OK;
}

static int unpack_pair(rs_batch *b, int i, rs_upoly &o) {
  const PairPlan &p = b->plans[i];
  int rc = p.status;
  if (rc == RS_OK && !o.coeffs && o.capacity_words > 0) rc = RS_ERR_ARG;
  if (rc != RS_OK) return rc;
  int deg, L;
  const uint32_t *w = result_shape(b, i, &deg, &L);
  o.deg = deg;
  o.limbs = L;
  if ((int64_t)(deg + 1) * L > o.capacity_words) return RS_ERR_CAPACITY;
  if (L == p.Lout) {
    if (deg >= 0) memcpy(o.coeffs, w, (size_t)(deg + 1) * L * 4);
  } else {
    for (int j = 0; j <= deg; ++j) memcpy(o.coeffs + (size_t)j * L, w + (size_t)j * p.Lout, (size_t)L * 4);
  }
  return RS_OK;
}

int rs_unpack(rs_batch *b, rs_upoly *out, int32_t *status) {
  rs_ctx *ctx = b->ctx;
  const int n = b->n;
  if (device_status(b) != RS_OK) {
    for (int i = 0; i < n && status; ++i) status[i] = RS_ERR_TIMEOUT;
    return rs_fail(ctx, RS_ERR_TIMEOUT, "tensor-core kernels: a bounded device wait ran out");
  }
  std::vector<int> rcs(n, RS_OK);
  // Large outputs are trimmed and copied by several host threads, each
  // taking a contiguous range of pairs of about equal size.
  const int64_t kWordsPerThread = int64_t(1) << 20;
  const int hw = std::max(1, (int)std::thread::hardware_concurrency());
  const int nt = (int)std::min<int64_t>({(int64_t)std::min(hw, 16), (int64_t)n, b->out_words / kWordsPerThread + 1});
  if (nt <= 1) {
    for (int i = 0; i < n; ++i) rcs[i] = unpack_pair(b, i, out[i]);
  } else {
    std::vector<int> cut(1, 0);
    int64_t acc = 0;
    for (int i = 0; i < n; ++i) {
      const PairPlan &p = b->plans[i];
      if (p.status == RS_OK && !p.trivial_zero) acc += (int64_t)p.N * p.Lout;
      if (acc * nt >= b->out_words * (int64_t)cut.size() && (int)cut.size() < nt) cut.push_back(i + 1);
    }
    while ((int)cut.size() <= nt) cut.push_back(n);
    cut.back() = n;
    std::vector<std::thread> th;
    for (int t = 0; t < nt; ++t)
      th.emplace_back([&, t] {
        for (int i = cut[t]; i < cut[t + 1]; ++i) rcs[i] = unpack_pair(b, i, out[i]);
      });
    for (auto &x : th) x.join();
  }
  int first = RS_OK;
  for (int i = 0; i < n; ++i) {
    const int rc = rcs[i];
    if (status) status[i] = rc;
    if (rc != RS_OK && first == RS_OK) {
      first = rc;
      rs_fail(ctx, rc, std::string("pair ") + std::to_string(i) + ": " + rs_error_string(rc));
    }
  }
  return first;
}

static int fetch(rs_batch *b, rs_upoly *out, int32_t *status) {
  rs_ctx *ctx = b->ctx;
  DevGuard dg(ctx->device);
  int rc = rs_fetch_async(b);
  if (rc != RS_OK) return rc;
  RS_CUDA(ctx, cudaStreamSynchronize(b->stream));
  return rs_unpack(b, out, status);
}

static RsBatchOpts default_opts(rs_ctx *ctx) {
  RsBatchOpts o;
  o.use_graph = ctx->cfg.use_graphs != 0;
  o.persistent = ctx->cfg.persistent != 0;
  return o;
}

// ------------------------------------------------------------------ C ABI

extern "C" {

const char *rs_error_string(int code) {
  switch (code) {
    case RS_OK: return "ok";
    case RS_PENDING: return "pending";
    case RS_ERR_ARG: return "invalid argument";
    case RS_ERR_CAPACITY: return "output capacity too small";
    case RS_ERR_NOMEM: return "out of memory";
    case RS_ERR_CUDA: return "CUDA error";
    case RS_ERR_TIMEOUT: return "wait timed out";
    case RS_ERR_LIMIT: return "input exceeds a library limit";
    case RS_ERR_STATE: return "invalid state";
    default: return "unknown error";
  }
}

const char *rs_last_error(const rs_ctx *ctx) { return ctx ? ctx->err.c_str() : g_err.c_str(); }

int rs_test_stall_tensor_cores(rs_ctx *ctx, int32_t on) {
  if (!ctx) return rs_fail(nullptr, RS_ERR_ARG, "ctx is NULL");
  DevGuard dg(ctx->device);
  const int32_t v = on ? 1 : 0;
  RS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  RS_CUDA(ctx, cudaMemcpy(ctx->d_stall, &v, sizeof(v), cudaMemcpyHostToDevice));
  return RS_OK;
}

int rs_config_default(rs_config *cfg) {
  if (!cfg) return rs_fail(nullptr, RS_ERR_ARG, "cfg is NULL");
  memset(cfg, 0, sizeof(*cfg));
  cfg->device = -1;
  cfg->use_graphs = 1;
  cfg->persistent = 1;
  cfg->autotune = 1;
  return RS_OK;
}

int rs_create(rs_ctx **out, const rs_config *cfg) {
  if (!out) return rs_fail(nullptr, RS_ERR_ARG, "ctx is NULL");
  *out = nullptr;
  rs_config c;
  if (cfg)
    c = *cfg;
  else
    rs_config_default(&c);
  if (c.tile_points != 0 && c.tile_points != 32 && c.tile_points != 64 && c.tile_points != 128)
    return rs_fail(nullptr, RS_ERR_ARG, "tile_points must be 0, 32, 64 or 128");
  if (c.g2_form < 0 || c.g2_form > 4) return rs_fail(nullptr, RS_ERR_ARG, "g2_form must be 0, 1, 2, 3 or 4");
  if (c.univariate < 0 || c.univariate > 1) return rs_fail(nullptr, RS_ERR_ARG, "univariate must be 0 or 1");
  if (c.crt_form < 0 || c.crt_form > 2) return rs_fail(nullptr, RS_ERR_ARG, "crt_form must be 0, 1 or 2");
  int dev = c.device;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0)
    return rs_fail(nullptr, RS_ERR_CUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
  if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) dev = 0;
  if (dev >= ndev) return rs_fail(nullptr, RS_ERR_ARG, "device ordinal out of range");
  if (c.autotune_cache && c.autotune_cache[0]) {
    FILE *probe = fopen(c.autotune_cache, "r");
    if (probe) {
      fclose(probe);
      int rc0 = rs_autotune_load(c.autotune_cache);
      if (rc0 != RS_OK) return rc0;
    }
  }
  rs_ctx *ctx = new rs_ctx();
  ctx->device = dev;
  ctx->cfg = c;
  if (c.autotune_cache) ctx->tune_path = c.autotune_cache;
  ctx->cfg.autotune_cache = nullptr;  // the copy in tune_path is the one kept
  DevGuard dg(dev);
  int rc = RS_OK;
  auto chk = [&](cudaError_t e2, const char *what) {
    if (rc == RS_OK && e2 != cudaSuccess)
      rc = rs_fail(nullptr, rs_cuda_code(e2), std::string(what) + ": " + cudaGetErrorString(e2));
  };
  chk(cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, dev), "device query");
  chk(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking), "cudaStreamCreate");
  for (auto &ss : ctx->side) chk(cudaStreamCreateWithFlags(&ss, cudaStreamNonBlocking), "cudaStreamCreate");
  ctx->primes = rs_prime_table(RS_MAX_PRIMES);
  for (uint32_t p : ctx->primes) ctx->log2p.push_back(log2((double)p) - 1e-12);
  const int np = (int)ctx->primes.size();
  chk(cudaMalloc(&ctx->d_primes, np * 4), "cudaMalloc");
  chk(cudaMalloc(&ctx->d_mods, np * sizeof(ModP)), "cudaMalloc");
  chk(cudaMalloc(&ctx->d_vtab, (size_t)np * RS_VT_STRIDE * 4), "cudaMalloc");
  chk(cudaMalloc(&ctx->d_crt, np * 4), "cudaMalloc");
  chk(cudaMalloc(&ctx->d_qbase, np * 4), "cudaMalloc");
  chk(cudaMalloc(&ctx->d_stall, sizeof(int32_t)), "cudaMalloc");
  if (rc == RS_OK) chk(cudaMemset(ctx->d_stall, 0, sizeof(int32_t)), "cudaMemset");
  if (rc == RS_OK) chk(cudaMemcpy(ctx->d_primes, ctx->primes.data(), np * 4, cudaMemcpyHostToDevice), "cudaMemcpy");
  if (rc == RS_OK)
    chk(launch_init_primes(ctx->d_primes, np, ctx->d_mods, ctx->d_vtab, ctx->d_crt, ctx->d_qbase, ctx->stream),
        "prime tables");
  if (rc == RS_OK) {
    std::vector<uint2> tw;
    ntt_host_tables(ctx->nttc, tw);
    chk(cudaMalloc(&ctx->d_ntt_tw, tw.size() * sizeof(uint2)), "cudaMalloc");
    if (rc == RS_OK) chk(cudaMemcpy(ctx->d_ntt_tw, tw.data(), tw.size() * sizeof(uint2), cudaMemcpyHostToDevice), "cudaMemcpy");
  }
  if (rc == RS_OK) chk(cudaStreamSynchronize(ctx->stream), "prime tables");
  if (rc != RS_OK) {
    rs_destroy(ctx);
    return rc;
  }
  *out = ctx;
  return RS_OK;
}

int rs_destroy(rs_ctx *ctx) {
  if (!ctx) return RS_OK;
  rs_server_shutdown(ctx);
  if (!ctx->tune_path.empty()) rs_autotune_save(ctx->tune_path.c_str());
  {
    DevGuard dg(ctx->device);
    for (rs_batch *b : ctx->batches) rs_free_batch(b);
    if (ctx->cache) rs_free_batch(ctx->cache);
    if (ctx->sqf_cache) rs_free_batch(ctx->sqf_cache);
    if (ctx->sqf_arena) cudaFree(ctx->sqf_arena);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    free_tables(ctx->tab);
    for (auto &t : ctx->retired) free_tables(t);
    for (uint32_t *bh : ctx->bhat)
      if (bh) cudaFree(bh);
    for (void *bh : ctx->bhat_retired) cudaFree(bh);
    if (ctx->g2t_bt) cudaFree(ctx->g2t_bt);
    for (void *bt : ctx->g2t_retired) cudaFree(bt);
    if (ctx->g3m_wt) cudaFree(ctx->g3m_wt);
    if (ctx->g3m_rt) cudaFree(ctx->g3m_rt);
    if (ctx->g3l_bt) cudaFree(ctx->g3l_bt);
    if (ctx->g3l_cbase) cudaFree(ctx->g3l_cbase);
    for (void *wt : ctx->g3m_retired) cudaFree(wt);
    void *dev[] = {ctx->d_primes, ctx->d_mods, ctx->d_vtab, ctx->d_crt, ctx->d_qbase, ctx->d_ntt_tw, ctx->d_stall};
    for (void *p : dev)
      if (p) cudaFree(p);
    for (auto ss : ctx->side)
      if (ss) {
        cudaStreamSynchronize(ss);
        cudaStreamDestroy(ss);
      }
    if (ctx->stream) cudaStreamDestroy(ctx->stream);
  }
  delete ctx;
  return RS_OK;
}

int rs_stream(rs_ctx *ctx, void **stream) {
  if (!ctx || !stream) return rs_fail(ctx, RS_ERR_ARG, "NULL argument");
  *stream = (void *)ctx->stream;
  return RS_OK;
}

int rs_result_bound(const rs_bipoly *f, const rs_bipoly *g, int32_t *deg_bound, int32_t *limbs_bound,
                    int32_t *primes, int32_t *bits) {
  static const std::vector<double> log2p = [] {
    std::vector<double> v;
    for (uint32_t p : rs_prime_table(RS_MAX_PRIMES)) v.push_back(log2((double)p) - 1e-12);
    return v;
  }();
  PairPlan p;
  const char *why = "";
  int rc = rs_plan_pair(f, g, log2p, p, &why);
  if (rc != RS_OK) return rs_fail(nullptr, rc, why);
  if (deg_bound) *deg_bound = p.trivial_zero ? -1 : p.D;
  if (limbs_bound) *limbs_bound = p.Lout;
  if (primes) *primes = p.K;
  if (bits) *bits = p.bits;
  return RS_OK;
}

int rs_batch_create_on(rs_ctx *ctx, int32_t n, const rs_bipoly *f, const rs_bipoly *g, void *stream,
                       rs_batch **batch) {
  if (!ctx || !batch || n < 0 || (n > 0 && (!f || !g))) return rs_fail(ctx, RS_ERR_ARG, "NULL argument or negative n");
  *batch = nullptr;
  std::vector<PairPlan> plans;
  int first = RS_OK;
  rs_plan_all(ctx, n, f, g, plans, nullptr, &first);
  rs_batch *b = nullptr;
  RsBatchOpts o = default_opts(ctx);
  o.stream = static_cast<cudaStream_t>(stream);
  int rc = rs_build_batch(ctx, n, f, g, std::move(plans), o, &b);
  if (rc != RS_OK) return rc;
  DevGuard dg(ctx->device);
  rc = rs_upload(b, f, g);
  if (rc != RS_OK) {
    rs_free_batch(b);
    return rc;
  }
  ctx->batches.push_back(b);
  *batch = b;
  return RS_OK;
}

int rs_batch_create(rs_ctx *ctx, int32_t n, const rs_bipoly *f, const rs_bipoly *g, rs_batch **batch) {
  return rs_batch_create_on(ctx, n, f, g, nullptr, batch);
}

int rs_batch_upload(rs_batch *b, int32_t n, const rs_bipoly *f, const rs_bipoly *g) {
  if (!b || n != b->n || (n > 0 && (!f || !g))) return rs_fail(b ? b->ctx : nullptr, RS_ERR_ARG, "bad arguments");
  std::vector<PairPlan> plans;
  int first = RS_OK;
  rs_plan_all(b->ctx, n, f, g, plans, nullptr, &first);
  for (int i = 0; i < n; ++i)
    if (!rs_same_shape(plans[i], b->plans[i]))
      return rs_fail(b->ctx, RS_ERR_STATE, "inputs do not match the batch's plan (pair " + std::to_string(i) + ")");
  DevGuard dg(b->ctx->device);
  return rs_upload(b, f, g);
}

int rs_batch_run(rs_batch *b) {
  if (!b) return rs_fail(nullptr, RS_ERR_ARG, "batch is NULL");
  return rs_run(b);
}

int rs_batch_sync(rs_batch *b) {
  if (!b) return rs_fail(nullptr, RS_ERR_ARG, "batch is NULL");
  DevGuard dg(b->ctx->device);
  RS_CUDA(b->ctx, cudaStreamSynchronize(b->stream));
  return RS_OK;
}

int rs_batch_results(rs_batch *b, rs_upoly *out, int32_t *status) {
  if (!b || (b->n > 0 && !out)) return rs_fail(b ? b->ctx : nullptr, RS_ERR_ARG, "NULL argument");
  return fetch(b, out, status);
}

int rs_batch_destroy(rs_batch *b) {
  if (!b) return RS_OK;
  auto &v = b->ctx->batches;
  v.erase(std::remove(v.begin(), v.end(), b), v.end());
  rs_free_batch(b);
  return RS_OK;
}

int rs_batch_info_get(rs_batch *b, rs_batch_info *info) {
  if (!b || !info) return rs_fail(b ? b->ctx : nullptr, RS_ERR_ARG, "NULL argument");
  rs_ctx *ctx = b->ctx;
  DevGuard dg(ctx->device);
  *info = b->info;
  info->ms_images = info->ms_interp = info->ms_crt = info->ms_total = -1.0f;
  info->ms_yun = 0.0f;
  info->reserved = 0;
  if (!b->ran) return RS_OK;
  RS_CUDA(ctx, cudaStreamSynchronize(b->stream));
  unsigned long long st[ST_COUNT];
  RS_CUDA(ctx, cudaMemcpy(st, b->d_stats, sizeof(st), cudaMemcpyDeviceToHost));
  info->unlucky_points = (int64_t)st[ST_UNLUCKY_POINTS];
  info->degenerate_images = (int64_t)st[ST_DEGENERATE];
  info->unlucky_primes = (int64_t)st[ST_UNLUCKY_PRIMES];
  if (ctx->cfg.timing) {
    float t = 0;
    if (cudaEventElapsedTime(&t, b->ev[0], b->ev[1]) == cudaSuccess) info->ms_images = t;
    if (!b->opt.images_only) {
      if (cudaEventElapsedTime(&t, b->ev[1], b->ev[b->nyun ? 4 : 2]) == cudaSuccess) info->ms_interp = t;
      if (b->nyun && cudaEventElapsedTime(&t, b->ev[4], b->ev[2]) == cudaSuccess) info->ms_yun = t;
      if (cudaEventElapsedTime(&t, b->ev[2], b->ev[3]) == cudaSuccess) info->ms_crt = t;
      if (cudaEventElapsedTime(&t, b->ev[0], b->ev[3]) == cudaSuccess) info->ms_total = t;
    }
  }
  return RS_OK;
}

int rs_resultant_batch(rs_ctx *ctx, int32_t n, const rs_bipoly *f, const rs_bipoly *g, rs_upoly *out,
                       int32_t *status) {
  if (!ctx || n < 0 || (n > 0 && (!f || !g || !out))) return rs_fail(ctx, RS_ERR_ARG, "NULL argument or negative n");
  if (n == 0) return RS_OK;
  std::vector<PairPlan> plans;
  int first = RS_OK;
  rs_plan_all(ctx, n, f, g, plans, status, &first);
  rs_batch *b = ctx->cache;
  bool reuse = b && b->n == n;
  for (int i = 0; reuse && i < n; ++i) reuse = rs_same_shape(plans[i], b->plans[i]);
  if (!reuse) {
    if (b) rs_free_batch(b);
    ctx->cache = nullptr;
    int rc = rs_build_batch(ctx, n, f, g, std::move(plans), default_opts(ctx), &b);
    if (rc != RS_OK) return rc;
    ctx->cache = b;
  }
  DevGuard dg(ctx->device);
  int rc = rs_upload(b, f, g);
  if (rc == RS_OK) rc = rs_run(b);
  if (rc == RS_OK) rc = fetch(b, out, status);
  return rc != RS_OK ? rc : first;
}

int rs_resultant_y(rs_ctx *ctx, const rs_bipoly *f, const rs_bipoly *g, rs_upoly *out) {
  return rs_resultant_batch(ctx, 1, f, g, out, nullptr);
}

// Copy of p with x and y exchanged (storage in `buf`); an input the planner
// would reject is passed through unchanged so that it fails the same way.
static rs_bipoly transposed(const rs_bipoly &p, std::vector<uint32_t> &buf) {
  if (!p.coeffs || p.deg_x < 0 || p.deg_y < 0 || p.limbs < 1 || p.limbs > RS_MAX_LIMBS ||
      (int64_t)(p.deg_x + 1) * (p.deg_y + 1) > ((int64_t)1 << 26))
    return p;
  const int nx = p.deg_x + 1, ny = p.deg_y + 1, L = p.limbs;
  buf.resize((size_t)nx * ny * L);
  for (int i = 0; i < nx; ++i)
    for (int j = 0; j < ny; ++j)
      memcpy(&buf[((size_t)j * nx + i) * L], p.coeffs + ((size_t)i * ny + j) * L, (size_t)L * 4);
  rs_bipoly t;
  t.deg_x = p.deg_y;
  t.deg_y = p.deg_x;
  t.limbs = L;
  t.coeffs = buf.data();
  return t;
}

int rs_resultant_x(rs_ctx *ctx, const rs_bipoly *f, const rs_bipoly *g, rs_upoly *out) {
  if (!ctx || !f || !g || !out) return rs_fail(ctx, RS_ERR_ARG, "NULL argument");
  std::vector<uint32_t> bf, bg;
  const rs_bipoly ft = transposed(*f, bf), gt = transposed(*g, bg);
  return rs_resultant_batch(ctx, 1, &ft, &gt, out, nullptr);
}

int rs_squarefree_projections(rs_ctx *ctx, int32_t n, const rs_bipoly *f, const rs_bipoly *g, int32_t max_mult,
                              rs_upoly *content_y, rs_upoly *factors_y, int32_t *nmult_y, rs_upoly *content_x,
                              rs_upoly *factors_x, int32_t *nmult_x, int32_t *status) {
  if (!ctx || n < 0 || max_mult < 1 ||
      (n > 0 && (!f || !g || !content_y || !factors_y || !nmult_y || !content_x || !factors_x || !nmult_x)))
    return rs_fail(ctx, RS_ERR_ARG, "NULL argument, negative n or max_mult < 1");
  if (n == 0) return RS_OK;
  const size_t N2 = 2 * (size_t)n, M = (size_t)max_mult;
  std::vector<std::vector<uint32_t>> bufs(N2);
  std::vector<rs_bipoly> F(N2), G(N2);
  std::vector<rs_upoly> C(N2), FA(N2 * M);
  std::vector<int32_t> NM(N2, 0);
  for (int i = 0; i < n; ++i) {
    F[i] = f[i];
    G[i] = g[i];
    F[n + i] = transposed(f[i], bufs[2 * (size_t)i]);
    G[n + i] = transposed(g[i], bufs[2 * (size_t)i + 1]);
    C[i] = content_y[i];
    C[n + i] = content_x[i];
    for (size_t m = 0; m < M; ++m) {
      FA[i * M + m] = factors_y[i * M + m];
      FA[(n + i) * M + m] = factors_x[i * M + m];
    }
  }
  const int rc = rs_squarefree_batch(ctx, 2 * n, F.data(), G.data(), max_mult, C.data(), FA.data(), NM.data(),
                                     status);
  for (int i = 0; i < n; ++i) {  // shapes (and data, through the caller's pointers) back
    content_y[i] = C[i];
    content_x[i] = C[n + i];
    nmult_y[i] = NM[i];
    nmult_x[i] = NM[n + i];
    for (size_t m = 0; m < M; ++m) {
      factors_y[i * M + m] = FA[i * M + m];
      factors_x[i * M + m] = FA[(n + i) * M + m];
    }
  }
  return rc;
}

int rs_projections(rs_ctx *ctx, int32_t n, const rs_bipoly *f, const rs_bipoly *g, rs_upoly *out_y,
                   rs_upoly *out_x, int32_t *status) {
  if (!ctx || n < 0 || (n > 0 && (!f || !g || !out_y || !out_x)))
    return rs_fail(ctx, RS_ERR_ARG, "NULL argument or negative n");
  if (n == 0) return RS_OK;
  std::vector<std::vector<uint32_t>> bufs(2 * (size_t)n);
  std::vector<rs_bipoly> F(2 * (size_t)n), G(2 * (size_t)n);
  std::vector<rs_upoly> O(2 * (size_t)n);
  for (int i = 0; i < n; ++i) {
    F[i] = f[i];
    G[i] = g[i];
    F[n + i] = transposed(f[i], bufs[2 * (size_t)i]);
    G[n + i] = transposed(g[i], bufs[2 * (size_t)i + 1]);
    O[i] = out_y[i];
    O[n + i] = out_x[i];
  }
  const int rc = rs_resultant_batch(ctx, 2 * n, F.data(), G.data(), O.data(), status);
  for (int i = 0; i < n; ++i) {  // deg and limbs are written on success and on RS_ERR_CAPACITY
    out_y[i].deg = O[i].deg;
    out_y[i].limbs = O[i].limbs;
    out_x[i].deg = O[n + i].deg;
    out_x[i].limbs = O[n + i].limbs;
  }
  return rc;
}

int rs_images(rs_ctx *ctx, const rs_bipoly *f, const rs_bipoly *g, int32_t nprimes, int32_t npoints,
              uint32_t *primes_out, uint32_t *points_out, uint32_t *images_out) {
  if (!ctx || !f || !g || !images_out || nprimes < 1 || npoints < 1)
    return rs_fail(ctx, RS_ERR_ARG, "bad arguments");
  if (nprimes > (int)ctx->primes.size() || npoints > RS_MAX_POINTS)
    return rs_fail(ctx, RS_ERR_LIMIT, "nprimes or npoints above the library limits");
  std::vector<PairPlan> plans;
  int first = RS_OK;
  rs_plan_all(ctx, 1, f, g, plans, nullptr, &first);
  if (first != RS_OK) return first;
  DevGuard dg(ctx->device);
  if (plans[0].trivial_zero) {
    memset(images_out, 0, (size_t)nprimes * npoints * 4);
    if (points_out) {
      std::vector<uint32_t> qb(nprimes);
      RS_CUDA(ctx, cudaMemcpy(qb.data(), ctx->d_qbase, (size_t)nprimes * 4, cudaMemcpyDeviceToHost));
      for (int k = 0; k < nprimes; ++k) {
        const ModP m = make_modp(ctx->primes[k]);
        for (int i = 0; i < npoints; ++i) {  // point 2 t + s is (-1)^s q^t
          const uint32_t pw = from_mont(mpow(qb[k], (uint32_t)(i >> 1), m), m);
          points_out[(size_t)k * npoints + i] = (i & 1) ? mneg(pw, m.p) : pw;
        }
      }
    }
  } else {
    plans[0].K = nprimes;
    plans[0].N = npoints;
    plans[0].D = npoints - 1;
    plans[0].Lout = 1;
    plans[0].cap = std::max(plans[0].f.my, plans[0].g.my) + 1;
    RsBatchOpts o = default_opts(ctx);
    o.images_only = true;
    o.use_graph = false;
    o.tune = false;
    rs_batch *b = nullptr;
    int rc = rs_build_batch(ctx, 1, f, g, std::move(plans), o, &b);
    if (rc != RS_OK) return rc;
    rc = rs_upload(b, f, g);
    if (rc == RS_OK) rc = rs_run(b);
    if (rc == RS_OK) {
      uint32_t *d_pts = points_out ? b->d_out : nullptr;  // images-only batches size d_out to K * N
      cudaError_t e = launch_finalize_images(ctx->d_mods, ctx->d_qbase, b->d_num, b->d_den, b->d_xl, d_pts,
                                             nprimes, npoints, b->descs[0].NI, b->stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(images_out, b->d_xl, (size_t)nprimes * npoints * 4, cudaMemcpyDeviceToHost, b->stream);
      if (e == cudaSuccess && points_out)
        e = cudaMemcpyAsync(points_out, d_pts, (size_t)nprimes * npoints * 4, cudaMemcpyDeviceToHost, b->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
      if (e != cudaSuccess) rc = rs_fail(ctx, RS_ERR_CUDA, std::string("images: ") + cudaGetErrorString(e));
    }
    rs_free_batch(b);
    if (rc != RS_OK) return rc;
  }
  if (primes_out) memcpy(primes_out, ctx->primes.data(), (size_t)nprimes * 4);
  return RS_OK;
}

}  // extern "C"
