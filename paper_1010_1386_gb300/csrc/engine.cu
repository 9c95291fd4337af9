// Host engine of librs: contexts, prepared batches, CUDA-graph replay and the
// C ABI of include/rs.h.  The host plans (planner.cpp), packs inputs into one
// pinned staging buffer, enqueues G1 (kernels_g1.cu), G2 and G3
// (kernels_g23.cu) on the context's stream and unpacks the results.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "planner.h"
#include "rs_internal.cuh"

namespace {

thread_local std::string g_err;

struct DevGuard {
  int prev = -1;
  explicit DevGuard(int d) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (d >= 0 && prev != d) cudaSetDevice(d);
  }
  ~DevGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

struct ClassLaunch {
  int cap = 0;
  int threads = 128;
  int blocks = 0;
  int64_t tile_off = 0;
  int ntiles = 0;
  size_t smem = 0;
};

int cuda_code(cudaError_t e) {
  return e == cudaErrorMemoryAllocation ? RS_ERR_NOMEM : RS_ERR_CUDA;
}

}  // namespace

struct rs_ctx {
  int device = 0;
  rs_config cfg;
  cudaStream_t stream = nullptr;
  int sms = 0;
  std::vector<uint32_t> primes;
  std::vector<double> log2p;
  uint32_t *d_primes = nullptr;
  ModP *d_mods = nullptr;
  uint32_t *d_vtab = nullptr;
  uint32_t *d_crt = nullptr;
  uint32_t *d_qbase = nullptr;
  std::string err;
  std::vector<rs_batch *> batches;
  rs_batch *cache = nullptr;
};

struct rs_batch {
  rs_ctx *ctx = nullptr;
  int n = 0;
  bool images_only = false;
  std::vector<PairPlan> plans;
  std::vector<int> dev_index;  // pair -> device pair index, -1 if none
  std::vector<PairDesc> descs;
  std::vector<int64_t> in_f, in_g;  // word offsets of each pair's inputs in the staging buffer
  std::vector<ClassLaunch> classes;
  int64_t in_words = 0, img_words = 0, out_words = 0;
  int ng2 = 0, ng3 = 0;
  size_t g2smem = 0;
  uint32_t *d_in = nullptr;
  int2 *d_meta = nullptr;
  PairDesc *d_pairs = nullptr;
  Tile *d_tiles = nullptr;
  int32_t *d_counters = nullptr;
  uint32_t *d_num = nullptr, *d_den = nullptr, *d_xl = nullptr, *d_out = nullptr;
  int2 *d_g2 = nullptr, *d_g3 = nullptr;
  unsigned long long *d_stats = nullptr;
  uint32_t *d_finv = nullptr, *d_gtab = nullptr;  // interpolation tables [K][tab_stride]
  int32_t *d_btab = nullptr;
  int32_t *d_qc = nullptr;   // chirp tables [K][chirp_stride]
  uint32_t *d_qn = nullptr;
  int tab_k = 0, tab_stride = 0, chirp_stride = 0;
  uint32_t *h_in = nullptr, *h_out = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  bool ran = false;
  rs_batch_info info;
};

static int fail(rs_ctx *c, int code, const std::string &msg) {
  if (c)
    c->err = msg;
  else
    g_err = msg;
  return code;
}

#define RS_CUDA(ctx, call)                                                                \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail((ctx), cuda_code(e_), std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// ------------------------------------------------------------------ helpers

static int plan_all(rs_ctx *ctx, int n, const rs_bipoly *f, const rs_bipoly *g,
                    std::vector<PairPlan> &plans, int32_t *status, int *first_err) {
  plans.assign(n, PairPlan());
  *first_err = RS_OK;
  for (int i = 0; i < n; ++i) {
    const char *why = "";
    int rc = rs_plan_pair(&f[i], &g[i], ctx->log2p, plans[i], &why);
    plans[i].status = rc;
    if (status) status[i] = rc;
    if (rc != RS_OK && *first_err == RS_OK) {
      *first_err = rc;
      fail(ctx, rc, std::string("pair ") + std::to_string(i) + ": " + why);
    }
  }
  return *first_err;
}

static bool same_shape(const PairPlan &a, const PairPlan &b) {
  return a.status == b.status && a.trivial_zero == b.trivial_zero && a.N == b.N && a.K == b.K &&
         a.Lout == b.Lout && a.f.my == b.f.my && a.g.my == b.g.my && a.f.L == b.f.L &&
         a.g.L == b.g.L && a.f.stride == b.f.stride && a.g.stride == b.g.stride &&
         a.f.dx == b.f.dx && a.g.dx == b.g.dx;
}

static int64_t input_words(const rs_bipoly &p) {
  return (int64_t)(p.deg_x + 1) * (p.deg_y + 1) * p.limbs;
}

static void free_batch(rs_batch *b) {
  if (!b) return;
  DevGuard dg(b->ctx->device);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  for (auto &e : b->ev)
    if (e) cudaEventDestroy(e);
  void *dev[] = {b->d_in,  b->d_meta, b->d_pairs, b->d_tiles, b->d_counters, b->d_num,
                 b->d_den, b->d_xl,   b->d_out,   b->d_g2,    b->d_g3,       b->d_stats,
                 b->d_finv, b->d_gtab, b->d_btab, b->d_qc,  b->d_qn};
  for (void *p : dev)
    if (p) cudaFree(p);
  if (b->h_in) cudaFreeHost(b->h_in);
  if (b->h_out) cudaFreeHost(b->h_out);
  delete b;
}

// Normal-sequence coefficient updates of the remainder sequence (a4 count).
static double prs_updates(int a, int b) {
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

static int build_batch(rs_ctx *ctx, int n, const rs_bipoly *f, const rs_bipoly *g,
                       std::vector<PairPlan> &&plans, bool images_only, rs_batch **out) {
  rs_batch *b = new rs_batch();
  b->ctx = ctx;
  b->n = n;
  b->images_only = images_only;
  b->plans = std::move(plans);
  b->dev_index.assign(n, -1);
  memset(&b->info, 0, sizeof(b->info));
  b->info.pairs = n;
  const int T = ctx->cfg.tile_points > 0 ? ctx->cfg.tile_points : 128;

  std::vector<int2> meta;
  std::vector<int> order;
  b->in_f.assign(n, -1);
  b->in_g.assign(n, -1);
  for (int i = 0; i < n; ++i) {
    b->in_f[i] = b->in_words;
    b->in_words += input_words(f[i]);
    b->in_g[i] = b->in_words;
    b->in_words += input_words(g[i]);
    const PairPlan &p = b->plans[i];
    if (p.status != RS_OK || p.trivial_zero) continue;
    PairDesc d;
    memset(&d, 0, sizeof(d));
    d.my = p.f.my;
    d.ny = p.g.my;
    d.N = p.N;
    d.K = p.K;
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
    b->img_words += (int64_t)p.K * p.N;
    d.out_off = b->out_words;
    b->out_words += (int64_t)p.N * p.Lout;
    b->dev_index[i] = (int)b->descs.size();
    b->descs.push_back(d);
    order.push_back(i);
    b->info.images += (int64_t)p.K * p.N;
    b->info.primes_total += p.K;
    b->info.coeffs_total += p.N;
    const double imgs = (double)p.K * p.N;
    b->info.modmul_eval += imgs * (p.f.nc + p.g.nc);
    b->info.modmul_prs += imgs * 2.0 * prs_updates(p.f.my, p.g.my);
    b->info.modmul_interp += (double)p.K * ((double)p.N * p.N + 8.0 * p.N);
    b->info.modmul_crt += (double)p.N * ((double)p.K * (p.K - 1) + p.K);
  }

  // G1 tiles grouped by register-capacity class; costliest pairs first.
  std::sort(order.begin(), order.end(), [&](int x, int y) {
    const PairPlan &a = b->plans[x], &c = b->plans[y];
    double ca = (double)a.K * a.N * (a.f.nc + a.g.nc + 2.0 * a.f.my * a.g.my);
    double cc = (double)c.K * c.N * (c.f.nc + c.g.nc + 2.0 * c.f.my * c.g.my);
    return ca > cc;
  });
  std::vector<Tile> tiles;
  int ncap = 0;
  for (int cap = 8; cap <= 72; cap += 8) {
    ClassLaunch cl;
    cl.cap = cap;
    cl.threads = T;
    cl.tile_off = (int64_t)tiles.size();
    for (int i : order) {
      const PairPlan &p = b->plans[i];
      if (g1_supported_cap(p.cap) != cap) continue;
      cl.smem = std::max(cl.smem, (size_t)rs_g1_staged_words(p, cap, T) * 4);
      for (int k = 0; k < p.K; ++k)
        for (int x0 = 0; x0 < p.N; x0 += T) tiles.push_back(Tile{b->dev_index[i], k, x0, std::min(T, p.N - x0)});
    }
    cl.ntiles = (int)((int64_t)tiles.size() - cl.tile_off);
    if (cl.ntiles > 0) {
      b->classes.push_back(cl);
      ++ncap;
    }
  }
  std::vector<int2> g2, g3;
  std::vector<int> byN(order);
  std::sort(byN.begin(), byN.end(), [&](int x, int y) { return b->plans[x].N > b->plans[y].N; });
  int maxN = 1, maxK = 0, maxDx = 0;
  for (int i : byN) {
    const PairPlan &p = b->plans[i];
    maxN = std::max(maxN, p.N);
    maxK = std::max(maxK, p.K);
    maxDx = std::max(maxDx, std::max(p.f.mx, p.g.mx));
    for (int k = 0; k < p.K; ++k) g2.push_back(make_int2(b->dev_index[i], k));
  }
  for (int i : order) {
    const PairPlan &p = b->plans[i];
    for (int j = 0; j < p.N; j += 128) g3.push_back(make_int2(b->dev_index[i], j));
  }
  b->ng2 = (int)g2.size();
  b->ng3 = (int)g3.size();
  b->g2smem = (size_t)3 * (maxN + 2 * RS_G2_PAD) * 4;
  b->tab_k = maxK;
  b->tab_stride = maxN;
  b->chirp_stride = maxN + T + maxDx + 1;
  b->info.kernel_launches = (int64_t)b->classes.size() + (images_only ? 0 : (b->ng2 > 0) + (b->ng3 > 0));
  b->info.input_bytes = b->in_words * 4;
  b->info.output_bytes = b->out_words * 4;

  DevGuard dg(ctx->device);
  int rc = RS_OK;
  auto alloc = [&](void **p, size_t bytes) {
    if (rc != RS_OK || bytes == 0) return;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) rc = fail(ctx, cuda_code(e), std::string("cudaMalloc: ") + cudaGetErrorString(e));
  };
  alloc((void **)&b->d_in, b->in_words * 4);
  alloc((void **)&b->d_meta, meta.size() * sizeof(int2));
  alloc((void **)&b->d_pairs, b->descs.size() * sizeof(PairDesc));
  alloc((void **)&b->d_tiles, tiles.size() * sizeof(Tile));
  alloc((void **)&b->d_counters, 16 * sizeof(int32_t));
  alloc((void **)&b->d_num, b->img_words * 4);
  alloc((void **)&b->d_den, b->img_words * 4);
  alloc((void **)&b->d_xl, std::max<int64_t>(b->out_words, images_only ? b->img_words : 0) * 4);
  alloc((void **)&b->d_out, std::max<int64_t>(b->out_words, images_only ? b->img_words : 0) * 4);
  alloc((void **)&b->d_g2, g2.size() * sizeof(int2));
  alloc((void **)&b->d_g3, g3.size() * sizeof(int2));
  alloc((void **)&b->d_stats, ST_COUNT * sizeof(unsigned long long));
  if (!images_only) {
    alloc((void **)&b->d_finv, (size_t)b->tab_k * b->tab_stride * 4);
    alloc((void **)&b->d_gtab, (size_t)b->tab_k * b->tab_stride * 4);
    alloc((void **)&b->d_btab, (size_t)b->tab_k * b->tab_stride * 4);
  }
  alloc((void **)&b->d_qc, (size_t)b->tab_k * b->chirp_stride * 4);
  alloc((void **)&b->d_qn, (size_t)b->tab_k * b->chirp_stride * 4);
  if (rc == RS_OK && b->in_words) {
    cudaError_t e = cudaMallocHost((void **)&b->h_in, b->in_words * 4);
    if (e != cudaSuccess) rc = fail(ctx, RS_ERR_NOMEM, "cudaMallocHost (inputs)");
  }
  if (rc == RS_OK && b->out_words) {
    cudaError_t e = cudaMallocHost((void **)&b->h_out, b->out_words * 4);
    if (e != cudaSuccess) rc = fail(ctx, RS_ERR_NOMEM, "cudaMallocHost (outputs)");
  }
  auto h2d = [&](void *dst, const void *src, size_t bytes) {
    if (rc != RS_OK || bytes == 0) return;
    cudaError_t e = cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) rc = fail(ctx, RS_ERR_CUDA, std::string("cudaMemcpy: ") + cudaGetErrorString(e));
  };
  h2d(b->d_meta, meta.data(), meta.size() * sizeof(int2));
  h2d(b->d_pairs, b->descs.data(), b->descs.size() * sizeof(PairDesc));
  h2d(b->d_tiles, tiles.data(), tiles.size() * sizeof(Tile));
  h2d(b->d_g2, g2.data(), g2.size() * sizeof(int2));
  h2d(b->d_g3, g3.data(), g3.size() * sizeof(int2));
  for (auto &cl : b->classes) {
    if (rc != RS_OK) break;
    int mb = 0;
    cudaError_t e = g1_prepare(cl.cap, cl.threads, cl.smem, &mb);
    if (e != cudaSuccess) {
      rc = fail(ctx, RS_ERR_CUDA, std::string("G1 set-up: ") + cudaGetErrorString(e));
      break;
    }
    if (mb < 1) mb = 1;
    cl.blocks = ctx->cfg.persistent ? std::min(cl.ntiles, mb * ctx->sms) : cl.ntiles;
  }
  if (rc == RS_OK && b->tab_k > 0) {
    cudaError_t e = launch_tables(ctx->d_mods, ctx->d_qbase, b->tab_k, b->tab_stride, b->chirp_stride,
                                  b->d_finv, b->d_gtab, b->d_btab, b->d_qc, b->d_qn, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) rc = fail(ctx, RS_ERR_CUDA, std::string("point tables: ") + cudaGetErrorString(e));
  }
  if (rc == RS_OK && b->ng2) {
    cudaError_t e = g2_prepare(b->g2smem);
    if (e != cudaSuccess) rc = fail(ctx, RS_ERR_CUDA, std::string("G2 set-up: ") + cudaGetErrorString(e));
  }
  for (auto &e : b->ev)
    if (rc == RS_OK && cudaEventCreate(&e) != cudaSuccess) rc = fail(ctx, RS_ERR_CUDA, "cudaEventCreate");
  if (rc != RS_OK) {
    free_batch(b);
    return rc;
  }
  *out = b;
  return RS_OK;
}

static int upload(rs_batch *b, const rs_bipoly *f, const rs_bipoly *g) {
  rs_ctx *ctx = b->ctx;
  for (int i = 0; i < b->n; ++i) {
    memcpy(b->h_in + b->in_f[i], f[i].coeffs, input_words(f[i]) * 4);
    memcpy(b->h_in + b->in_g[i], g[i].coeffs, input_words(g[i]) * 4);
  }
  if (b->in_words)
    RS_CUDA(ctx, cudaMemcpyAsync(b->d_in, b->h_in, b->in_words * 4, cudaMemcpyHostToDevice, ctx->stream));
  return RS_OK;
}

static cudaError_t record(cudaEvent_t e, cudaStream_t s, bool capturing) {
  return capturing ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal) : cudaEventRecord(e, s);
}

static int enqueue(rs_batch *b, bool capturing) {
  rs_ctx *ctx = b->ctx;
  cudaStream_t s = ctx->stream;
  const bool timing = ctx->cfg.timing != 0;
  RS_CUDA(ctx, cudaMemsetAsync(b->d_counters, 0, 16 * sizeof(int32_t), s));
  RS_CUDA(ctx, cudaMemsetAsync(b->d_stats, 0, ST_COUNT * sizeof(unsigned long long), s));
  if (timing) RS_CUDA(ctx, record(b->ev[0], s, capturing));
  int ci = 0;
  for (const auto &cl : b->classes) {
    G1Args a;
    a.pairs = b->d_pairs;
    a.tiles = b->d_tiles + cl.tile_off;
    a.ntiles = cl.ntiles;
    a.persistent = ctx->cfg.persistent ? 1 : 0;
    a.counter = b->d_counters + (ci++);
    a.limbs = b->d_in;
    a.meta = b->d_meta;
    a.mods = ctx->d_mods;
    a.qc = b->d_qc;
    a.qn = b->d_qn;
    a.tstride = b->chirp_stride;
    a.vtab = ctx->d_vtab;
    a.num = b->d_num;
    a.den = b->d_den;
    a.stats = b->d_stats;
    RS_CUDA(ctx, launch_g1(cl.cap, cl.threads, cl.blocks, cl.smem, a, s));
  }
  if (timing) RS_CUDA(ctx, record(b->ev[1], s, capturing));
  if (b->images_only) return RS_OK;
  if (b->ng2) {
    G2Args a2;
    a2.pairs = b->d_pairs;
    a2.tasks = b->d_g2;
    a2.mods = ctx->d_mods;
    a2.num = b->d_num;
    a2.den = b->d_den;
    a2.coef = b->d_num;
    a2.finv = b->d_finv;
    a2.gtab = b->d_gtab;
    a2.btab = b->d_btab;
    a2.tab_stride = b->tab_stride;
    RS_CUDA(ctx, launch_g2(256, b->ng2, b->g2smem, a2, s));
  }
  if (timing) RS_CUDA(ctx, record(b->ev[2], s, capturing));
  if (b->ng3) {
    G3Args a3;
    a3.pairs = b->d_pairs;
    a3.tasks = b->d_g3;
    a3.mods = ctx->d_mods;
    a3.crt = ctx->d_crt;
    a3.coef = b->d_num;
    a3.xl = b->d_xl;
    a3.out = b->d_out;
    RS_CUDA(ctx, launch_g3(128, b->ng3, a3, s));
  }
  if (timing) RS_CUDA(ctx, record(b->ev[3], s, capturing));
  return RS_OK;
}

static int run(rs_batch *b) {
  rs_ctx *ctx = b->ctx;
  DevGuard dg(ctx->device);
  if (ctx->cfg.use_graphs && !b->images_only) {
    if (!b->gexec) {
      RS_CUDA(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
      int rc = enqueue(b, true);
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
      if (rc != RS_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
      }
      if (e != cudaSuccess) return fail(ctx, RS_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
      e = cudaGraphInstantiate(&b->gexec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return fail(ctx, RS_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    RS_CUDA(ctx, cudaGraphLaunch(b->gexec, ctx->stream));
  } else {
    int rc = enqueue(b, false);
    if (rc != RS_OK) return rc;
  }
  b->ran = true;
  return RS_OK;
}

static int coef_limbs_needed(const uint32_t *c, int L) {
  const uint32_t ext = (c[L - 1] >> 31) ? 0xffffffffu : 0u;
  int l = L;
  while (l > 1 && c[l - 1] == ext && ((c[l - 2] >> 31) ? 0xffffffffu : 0u) == ext) --l;
  return l;
}

static int fetch(rs_batch *b, rs_upoly *out, int32_t *status) {
  rs_ctx *ctx = b->ctx;
  DevGuard dg(ctx->device);
  if (!b->ran) return fail(ctx, RS_ERR_STATE, "batch has not been run");
  if (b->out_words)
    RS_CUDA(ctx, cudaMemcpyAsync(b->h_out, b->d_out, b->out_words * 4, cudaMemcpyDeviceToHost, ctx->stream));
  RS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  int first = RS_OK;
  for (int i = 0; i < b->n; ++i) {
    const PairPlan &p = b->plans[i];
    int rc = p.status;
    if (rc == RS_OK && !out[i].coeffs && out[i].capacity_words > 0) rc = RS_ERR_ARG;
    if (rc == RS_OK) {
      int deg = -1, L = 1;
      const uint32_t *w = nullptr;
      if (!p.trivial_zero) {
        const PairDesc &d = b->descs[b->dev_index[i]];
        w = b->h_out + d.out_off;
        for (int j = 0; j < p.N; ++j) {
          const uint32_t *c = w + (size_t)j * p.Lout;
          bool nz = false;
          for (int l = 0; l < p.Lout; ++l) nz = nz || c[l];
          if (nz) {
            deg = j;
            L = std::max(L, coef_limbs_needed(c, p.Lout));
          }
        }
      }
      out[i].deg = deg;
      out[i].limbs = L;
      if ((int64_t)(deg + 1) * L > out[i].capacity_words) {
        rc = RS_ERR_CAPACITY;
      } else {
        for (int j = 0; j <= deg; ++j)
          for (int l = 0; l < L; ++l) out[i].coeffs[(size_t)j * L + l] = w[(size_t)j * p.Lout + l];
      }
    }
    if (status) status[i] = rc;
    if (rc != RS_OK && first == RS_OK) {
      first = rc;
      fail(ctx, rc, std::string("pair ") + std::to_string(i) + ": " + rs_error_string(rc));
    }
  }
  return first;
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
    case RS_ERR_TIMEOUT: return "device wait timed out";
    case RS_ERR_LIMIT: return "input exceeds a library limit";
    case RS_ERR_STATE: return "invalid state";
    default: return "unknown error";
  }
}

const char *rs_last_error(const rs_ctx *ctx) { return ctx ? ctx->err.c_str() : g_err.c_str(); }

int rs_config_default(rs_config *cfg) {
  if (!cfg) return fail(nullptr, RS_ERR_ARG, "cfg is NULL");
  memset(cfg, 0, sizeof(*cfg));
  cfg->device = -1;
  cfg->use_graphs = 1;
  cfg->persistent = 1;
  return RS_OK;
}

int rs_create(rs_ctx **out, const rs_config *cfg) {
  if (!out) return fail(nullptr, RS_ERR_ARG, "ctx is NULL");
  *out = nullptr;
  rs_config c;
  if (cfg)
    c = *cfg;
  else
    rs_config_default(&c);
  if (c.tile_points != 0 && c.tile_points != 32 && c.tile_points != 64 && c.tile_points != 128)
    return fail(nullptr, RS_ERR_ARG, "tile_points must be 0, 32, 64 or 128");
  int dev = c.device;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0)
    return fail(nullptr, RS_ERR_CUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
  if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) dev = 0;
  if (dev >= ndev) return fail(nullptr, RS_ERR_ARG, "device ordinal out of range");
  rs_ctx *ctx = new rs_ctx();
  ctx->device = dev;
  ctx->cfg = c;
  DevGuard dg(dev);
  int rc = RS_OK;
  auto chk = [&](cudaError_t e2, const char *what) {
    if (rc == RS_OK && e2 != cudaSuccess) rc = fail(nullptr, cuda_code(e2), std::string(what) + ": " + cudaGetErrorString(e2));
  };
  chk(cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, dev), "device query");
  chk(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking), "cudaStreamCreate");
  ctx->primes = rs_prime_table(RS_MAX_PRIMES);
  for (uint32_t p : ctx->primes) ctx->log2p.push_back(log2((double)p) - 1e-12);
  const int np = (int)ctx->primes.size();
  chk(cudaMalloc(&ctx->d_primes, np * 4), "cudaMalloc");
  chk(cudaMalloc(&ctx->d_mods, np * sizeof(ModP)), "cudaMalloc");
  chk(cudaMalloc(&ctx->d_vtab, (size_t)np * RS_VT_STRIDE * 4), "cudaMalloc");
  chk(cudaMalloc(&ctx->d_crt, np * 4), "cudaMalloc");
  chk(cudaMalloc(&ctx->d_qbase, np * 4), "cudaMalloc");
  if (rc == RS_OK) chk(cudaMemcpy(ctx->d_primes, ctx->primes.data(), np * 4, cudaMemcpyHostToDevice), "cudaMemcpy");
  if (rc == RS_OK) chk(launch_init_primes(ctx->d_primes, np, ctx->d_mods, ctx->d_vtab, ctx->d_crt, ctx->d_qbase, ctx->stream), "prime tables");
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
  {
    DevGuard dg(ctx->device);
    for (rs_batch *b : ctx->batches) free_batch(b);
    if (ctx->cache) free_batch(ctx->cache);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    void *dev[] = {ctx->d_primes, ctx->d_mods, ctx->d_vtab, ctx->d_crt, ctx->d_qbase};
    for (void *p : dev)
      if (p) cudaFree(p);
    if (ctx->stream) cudaStreamDestroy(ctx->stream);
  }
  delete ctx;
  return RS_OK;
}

int rs_stream(rs_ctx *ctx, void **stream) {
  if (!ctx || !stream) return fail(ctx, RS_ERR_ARG, "NULL argument");
  *stream = (void *)ctx->stream;
  return RS_OK;
}

int rs_result_bound(const rs_bipoly *f, const rs_bipoly *g, int32_t *deg_bound, int32_t *limbs_bound,
                    int32_t *primes, int32_t *bits) {
  static std::vector<double> log2p;
  static bool init = false;
  if (!init) {
    for (uint32_t p : rs_prime_table(RS_MAX_PRIMES)) log2p.push_back(log2((double)p) - 1e-12);
    init = true;
  }
  PairPlan p;
  const char *why = "";
  int rc = rs_plan_pair(f, g, log2p, p, &why);
  if (rc != RS_OK) return fail(nullptr, rc, why);
  if (deg_bound) *deg_bound = p.trivial_zero ? -1 : p.D;
  if (limbs_bound) *limbs_bound = p.Lout;
  if (primes) *primes = p.K;
  if (bits) *bits = p.bits;
  return RS_OK;
}

int rs_batch_create(rs_ctx *ctx, int32_t n, const rs_bipoly *f, const rs_bipoly *g, rs_batch **batch) {
  if (!ctx || !batch || n < 0 || (n > 0 && (!f || !g))) return fail(ctx, RS_ERR_ARG, "NULL argument or negative n");
  *batch = nullptr;
  std::vector<PairPlan> plans;
  int first = RS_OK;
  plan_all(ctx, n, f, g, plans, nullptr, &first);
  rs_batch *b = nullptr;
  int rc = build_batch(ctx, n, f, g, std::move(plans), false, &b);
  if (rc != RS_OK) return rc;
  rc = upload(b, f, g);
  if (rc != RS_OK) {
    free_batch(b);
    return rc;
  }
  ctx->batches.push_back(b);
  *batch = b;
  return RS_OK;
}

int rs_batch_upload(rs_batch *b, int32_t n, const rs_bipoly *f, const rs_bipoly *g) {
  if (!b || n != b->n || (n > 0 && (!f || !g))) return fail(b ? b->ctx : nullptr, RS_ERR_ARG, "bad arguments");
  std::vector<PairPlan> plans;
  int first = RS_OK;
  plan_all(b->ctx, n, f, g, plans, nullptr, &first);
  for (int i = 0; i < n; ++i)
    if (!same_shape(plans[i], b->plans[i]))
      return fail(b->ctx, RS_ERR_STATE, "inputs do not match the batch's plan (pair " + std::to_string(i) + ")");
  DevGuard dg(b->ctx->device);
  return upload(b, f, g);
}

int rs_batch_run(rs_batch *b) {
  if (!b) return fail(nullptr, RS_ERR_ARG, "batch is NULL");
  return run(b);
}

int rs_batch_sync(rs_batch *b) {
  if (!b) return fail(nullptr, RS_ERR_ARG, "batch is NULL");
  DevGuard dg(b->ctx->device);
  RS_CUDA(b->ctx, cudaStreamSynchronize(b->ctx->stream));
  return RS_OK;
}

int rs_batch_results(rs_batch *b, rs_upoly *out, int32_t *status) {
  if (!b || (b->n > 0 && !out)) return fail(b ? b->ctx : nullptr, RS_ERR_ARG, "NULL argument");
  return fetch(b, out, status);
}

int rs_batch_destroy(rs_batch *b) {
  if (!b) return RS_OK;
  auto &v = b->ctx->batches;
  v.erase(std::remove(v.begin(), v.end(), b), v.end());
  free_batch(b);
  return RS_OK;
}

int rs_batch_info_get(rs_batch *b, rs_batch_info *info) {
  if (!b || !info) return fail(b ? b->ctx : nullptr, RS_ERR_ARG, "NULL argument");
  rs_ctx *ctx = b->ctx;
  DevGuard dg(ctx->device);
  *info = b->info;
  info->ms_images = info->ms_interp = info->ms_crt = info->ms_total = -1.0f;
  if (!b->ran) return RS_OK;
  RS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  unsigned long long st[ST_COUNT];
  RS_CUDA(ctx, cudaMemcpy(st, b->d_stats, sizeof(st), cudaMemcpyDeviceToHost));
  info->unlucky_points = (int64_t)st[ST_UNLUCKY_POINTS];
  info->degenerate_images = (int64_t)st[ST_DEGENERATE];
  info->unlucky_primes = (int64_t)st[ST_UNLUCKY_PRIMES];
  if (ctx->cfg.timing) {
    float t = 0;
    if (cudaEventElapsedTime(&t, b->ev[0], b->ev[1]) == cudaSuccess) info->ms_images = t;
    if (!b->images_only) {
      if (cudaEventElapsedTime(&t, b->ev[1], b->ev[2]) == cudaSuccess) info->ms_interp = t;
      if (cudaEventElapsedTime(&t, b->ev[2], b->ev[3]) == cudaSuccess) info->ms_crt = t;
      if (cudaEventElapsedTime(&t, b->ev[0], b->ev[3]) == cudaSuccess) info->ms_total = t;
    }
  }
  return RS_OK;
}

int rs_resultant_batch(rs_ctx *ctx, int32_t n, const rs_bipoly *f, const rs_bipoly *g, rs_upoly *out,
                       int32_t *status) {
  if (!ctx || n < 0 || (n > 0 && (!f || !g || !out))) return fail(ctx, RS_ERR_ARG, "NULL argument or negative n");
  if (n == 0) return RS_OK;
  std::vector<PairPlan> plans;
  int first = RS_OK;
  plan_all(ctx, n, f, g, plans, status, &first);
  rs_batch *b = ctx->cache;
  bool reuse = b && b->n == n;
  for (int i = 0; reuse && i < n; ++i) reuse = same_shape(plans[i], b->plans[i]);
  if (!reuse) {
    if (b) free_batch(b);
    ctx->cache = nullptr;
    int rc = build_batch(ctx, n, f, g, std::move(plans), false, &b);
    if (rc != RS_OK) return rc;
    ctx->cache = b;
  }
  DevGuard dg(ctx->device);
  int rc = upload(b, f, g);
  if (rc == RS_OK) rc = run(b);
  if (rc == RS_OK) rc = fetch(b, out, status);
  return rc != RS_OK ? rc : first;
}

int rs_resultant_y(rs_ctx *ctx, const rs_bipoly *f, const rs_bipoly *g, rs_upoly *out) {
  return rs_resultant_batch(ctx, 1, f, g, out, nullptr);
}

int rs_images(rs_ctx *ctx, const rs_bipoly *f, const rs_bipoly *g, int32_t nprimes, int32_t npoints,
              uint32_t *primes_out, uint32_t *points_out, uint32_t *images_out) {
  if (!ctx || !f || !g || !images_out || nprimes < 1 || npoints < 1)
    return fail(ctx, RS_ERR_ARG, "bad arguments");
  if (nprimes > (int)ctx->primes.size() || npoints > RS_MAX_POINTS)
    return fail(ctx, RS_ERR_LIMIT, "nprimes or npoints above the library limits");
  std::vector<PairPlan> plans;
  int first = RS_OK;
  plan_all(ctx, 1, f, g, plans, nullptr, &first);
  if (first != RS_OK) return first;
  if (plans[0].trivial_zero) {
    memset(images_out, 0, (size_t)nprimes * npoints * 4);
    if (points_out) {  // the points are not needed; report them from a host-side run of the table
      std::vector<uint32_t> qb(nprimes);
      DevGuard dg(ctx->device);
      RS_CUDA(ctx, cudaMemcpy(qb.data(), ctx->d_qbase, (size_t)nprimes * 4, cudaMemcpyDeviceToHost));
      for (int k = 0; k < nprimes; ++k) {
        const ModP m = make_modp(ctx->primes[k]);
        for (int i = 0; i < npoints; ++i) points_out[(size_t)k * npoints + i] = from_mont(mpow(qb[k], i, m), m);
      }
    }
  } else {
    plans[0].K = nprimes;
    plans[0].N = npoints;
    plans[0].D = npoints - 1;
    plans[0].Lout = 1;
    plans[0].cap = std::max(plans[0].f.my, plans[0].g.my) + 1;
    rs_batch *b = nullptr;
    int rc = build_batch(ctx, 1, f, g, std::move(plans), true, &b);
    if (rc != RS_OK) return rc;
    DevGuard dg(ctx->device);
    rc = upload(b, f, g);
    if (rc == RS_OK) rc = run(b);
    if (rc == RS_OK) {
      uint32_t *d_pts = points_out ? b->d_out : nullptr;  // images-only batches size d_out to K * N
      cudaError_t e = launch_finalize_images(ctx->d_mods, ctx->d_qbase, b->d_num, b->d_den, b->d_xl, d_pts,
                                             nprimes, npoints, ctx->stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(images_out, b->d_xl, (size_t)nprimes * npoints * 4, cudaMemcpyDeviceToHost, ctx->stream);
      if (e == cudaSuccess && points_out)
        e = cudaMemcpyAsync(points_out, d_pts, (size_t)nprimes * npoints * 4, cudaMemcpyDeviceToHost, ctx->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
      if (e != cudaSuccess) rc = fail(ctx, RS_ERR_CUDA, std::string("images: ") + cudaGetErrorString(e));
    }
    free_batch(b);
    if (rc != RS_OK) return rc;
  }
  if (primes_out) memcpy(primes_out, ctx->primes.data(), (size_t)nprimes * 4);
  return RS_OK;
}

}  // extern "C"
