// Tuner of the G1 launch (tile width and schedule) and of the G2 form
// (direct convolutions, number-theoretic transforms or tensor-core products)
// per workload class, with a process-wide cache and its text file form.  The
// G1 candidates change only how the (pair, prime, point) work list is cut
// into blocks and handed to SMs, and every G2 form computes the same
// residues exactly, so every result is the same under each choice.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "engine.h"

namespace {

std::mutex g_mu;
std::map<int64_t, RsG1Choice> g_cache;

constexpr int64_t kSampleImages = int64_t(1) << 22;  // tuning sample bound
constexpr int kRuns = 3;                             // timed runs per candidate (after one warm-up)
constexpr float kKeepDefault = 1.02f;                // another choice must beat the default by 2%
constexpr int64_t kWholeGroupImages = int64_t(1) << 25;  // G2 forms: groups timed whole up to this

int ilog2(int64_t v) {
  int r = 0;
  while (v > 1) {
    v >>= 1;
    ++r;
  }
  return r;
}

int64_t make_key(int kind, int sms, int cap, int lgN, int lgI) {
  return ((int64_t)kind << 48) | ((int64_t)sms << 32) | ((int64_t)cap << 16) | ((int64_t)lgN << 8) | (int64_t)lgI;
}

void unpack_key(int64_t key, rs_tune_entry &e) {
  e.kind = (int)(key >> 48);
  e.sms = (int)((key >> 32) & 0xffff);
  e.cap = (int)((key >> 16) & 0xffff);
  e.lg_points = (int)((key >> 8) & 0xff);
  e.lg_images = (int)(key & 0xff);
}

bool valid_entry(const rs_tune_entry &e) {
  const bool common = e.sms > 0 && e.sms < 65536 && e.lg_points >= 0 && e.lg_points < 32 && e.lg_images >= 0 &&
                      e.lg_images < 64 && e.ms_best >= 0.f && e.ms_default >= 0.f;
  if (e.kind == RS_TUNE_G1)
    return common && e.cap >= 8 && e.cap <= 72 && e.cap % 8 == 0 &&
           (e.choice == 32 || e.choice == 64 || e.choice == 128) && (e.persistent == 0 || e.persistent == 1);
  if (e.kind == RS_TUNE_G2)
    return common && e.cap == 0 && e.lg_points >= 1 && e.lg_points <= RS_NTT_LGMAX && (e.choice >= 0 && e.choice <= 2) &&
           e.persistent == 0;
  return false;
}

rs_tune_entry to_entry(int64_t key, const RsG1Choice &c) {
  rs_tune_entry e;
  unpack_key(key, e);
  e.choice = c.threads;
  e.persistent = c.persistent;
  e.ms_best = c.ms_best;
  e.ms_default = c.ms_default;
  return e;
}

// G1 time (ms, median of kRuns) of one candidate on the sample.
int time_candidate(rs_ctx *ctx, const std::vector<rs_bipoly> &F, const std::vector<rs_bipoly> &G,
                   const std::vector<PairPlan> &P, int threads, int persistent, float *ms) {
  RsBatchOpts o;
  o.images_only = true;
  o.use_graph = false;
  o.persistent = persistent != 0;
  o.tune = false;
  o.timing = true;
  o.g1_threads = threads;
  std::vector<PairPlan> plans(P);
  rs_batch *b = nullptr;
  const int n = (int)F.size();
  int rc = rs_build_batch(ctx, n, F.data(), G.data(), std::move(plans), o, &b);
  if (rc != RS_OK) return rc;
  rc = rs_upload(b, F.data(), G.data());
  std::vector<float> t;
  for (int r = 0; rc == RS_OK && r <= kRuns; ++r) {
    rc = rs_run(b);
    if (rc != RS_OK) break;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    float v = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&v, b->ev[0], b->ev[1]);
    if (e != cudaSuccess) rc = rs_fail(ctx, RS_ERR_CUDA, std::string("tuner: ") + cudaGetErrorString(e));
    if (r > 0) t.push_back(v);
  }
  rs_free_batch(b);
  if (rc != RS_OK) return rc;
  std::sort(t.begin(), t.end());
  *ms = t[t.size() / 2];
  return RS_OK;
}

}  // namespace

int64_t rs_tune_key(int sms, int cap, int max_points, int64_t images) {
  return make_key(RS_TUNE_G1, sms, cap, ilog2(std::max(max_points, 1)), ilog2(std::max<int64_t>(images, 1)));
}

int64_t rs_tune_key_g2(int sms, int lg, int64_t images) {
  return make_key(RS_TUNE_G2, sms, 0, lg, ilog2(std::max<int64_t>(images, 1)));
}

bool rs_tune_find(int64_t key, RsG1Choice *out) {
  std::lock_guard<std::mutex> lock(g_mu);
  auto it = g_cache.find(key);
  if (it == g_cache.end()) return false;
  *out = it->second;
  return true;
}

int rs_tune_g1(rs_ctx *ctx, const rs_bipoly *f, const rs_bipoly *g, const std::vector<PairPlan> &plans,
               const std::vector<int> &members, int64_t key, RsG1Choice *out) {
  int64_t total = 0;
  for (int i : members) total += (int64_t)plans[i].K * plans[i].N;
  const int64_t stride = std::max<int64_t>(1, (total + kSampleImages - 1) / kSampleImages);
  std::vector<rs_bipoly> F, G;
  std::vector<PairPlan> P;
  for (size_t s = 0; s < members.size(); s += (size_t)stride) {
    const int i = members[s];
    F.push_back(f[i]);
    G.push_back(g[i]);
    P.push_back(plans[i]);
  }
  const int widths[3] = {128, 64, 32};
  RsG1Choice best;
  float ms_default = -1.f, ms_best = -1.f;
  for (int persistent = 1; persistent >= 0; --persistent)
    for (int w : widths) {
      float ms = 0.f;
      int rc = time_candidate(ctx, F, G, P, w, persistent, &ms);
      if (rc != RS_OK) return rc;
      if (w == 128 && persistent == 1) ms_default = ms;
      if (ms_best < 0.f || ms < ms_best) {
        ms_best = ms;
        best.threads = w;
        best.persistent = persistent;
      }
    }
  if (ms_best * kKeepDefault >= ms_default) {
    best.threads = 128;
    best.persistent = 1;
    ms_best = ms_default;
  }
  best.ms_best = ms_best;
  best.ms_default = ms_default;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    g_cache[key] = best;
  }
  *out = best;
  return RS_OK;
}

// G2 time (ms, median of kRuns) of the whole path on the sample with one form.
static int time_g2_form(rs_ctx *ctx, const std::vector<rs_bipoly> &F, const std::vector<rs_bipoly> &G,
                        const std::vector<PairPlan> &P, int form, float *ms) {
  RsBatchOpts o;
  o.use_graph = false;
  o.persistent = ctx->cfg.persistent != 0;
  o.tune = false;
  o.timing = true;
  o.g2_force = form;
  std::vector<PairPlan> plans(P);
  rs_batch *b = nullptr;
  int rc = rs_build_batch(ctx, (int)F.size(), F.data(), G.data(), std::move(plans), o, &b);
  if (rc != RS_OK) return rc;
  rc = rs_upload(b, F.data(), G.data());
  std::vector<float> t;
  for (int r = 0; rc == RS_OK && r <= kRuns; ++r) {
    rc = rs_run(b);
    if (rc != RS_OK) break;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    float v = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&v, b->ev[1], b->ev[2]);
    if (e != cudaSuccess) rc = rs_fail(ctx, RS_ERR_CUDA, std::string("tuner: ") + cudaGetErrorString(e));
    if (r > 0) t.push_back(v);
  }
  rs_free_batch(b);
  if (rc != RS_OK) return rc;
  std::sort(t.begin(), t.end());
  *ms = t[t.size() / 2];
  return RS_OK;
}

int rs_tune_g2(rs_ctx *ctx, const rs_bipoly *f, const rs_bipoly *g, const std::vector<PairPlan> &plans,
               const std::vector<int> &members, int64_t key, int model_form, int *form) {
  int64_t total = 0;
  for (int i : members) total += (int64_t)plans[i].K * plans[i].N;
  // The tensor-core form multiplies all pairs of a prime at once, so a
  // strided sample (fewer pairs per prime) would understate it: groups up to
  // kWholeGroupImages are timed whole.
  const int64_t stride = total <= kWholeGroupImages
                             ? 1
                             : std::max<int64_t>(1, (total + kSampleImages - 1) / kSampleImages);
  std::vector<rs_bipoly> F, G;
  std::vector<PairPlan> P;
  for (size_t s = 0; s < members.size(); s += (size_t)stride) {
    F.push_back(f[members[s]]);
    G.push_back(g[members[s]]);
    P.push_back(plans[members[s]]);
  }
  float ms[3] = {0.f, 0.f, 0.f};  // direct, transforms, tensor cores
  for (int fm = 0; fm < 3; ++fm) {
    const int rc = time_g2_form(ctx, F, G, P, fm, &ms[fm]);
    if (rc != RS_OK) return rc;
  }
  int best = model_form;
  for (int fm = 0; fm < 3; ++fm)
    if (ms[fm] * kKeepDefault < ms[best]) best = fm;
  RsG1Choice c;
  c.threads = best;
  c.persistent = 0;
  c.ms_best = ms[best];
  c.ms_default = ms[model_form];
  {
    std::lock_guard<std::mutex> lock(g_mu);
    g_cache[key] = c;
  }
  *form = best;
  return RS_OK;
}

extern "C" {

int rs_autotune(rs_ctx *ctx, int32_t n, const rs_bipoly *f, const rs_bipoly *g) {
  if (!ctx || n < 0 || (n > 0 && (!f || !g))) return rs_fail(ctx, RS_ERR_ARG, "NULL argument or negative n");
  if (n == 0) return RS_OK;
  std::vector<PairPlan> plans;
  int first = RS_OK;
  rs_plan_all(ctx, n, f, g, plans, nullptr, &first);
  RsBatchOpts o;  // the tuning happens while the batch is built; nothing is run
  o.use_graph = false;
  o.persistent = ctx->cfg.persistent != 0;
  o.tune = true;
  rs_batch *b = nullptr;
  int rc = rs_build_batch(ctx, n, f, g, std::move(plans), o, &b);
  if (rc != RS_OK) return rc;
  rs_free_batch(b);
  return RS_OK;
}

int rs_autotune_entries(rs_tune_entry *out, int32_t cap_entries, int32_t *count) {
  if (!count || cap_entries < 0 || (cap_entries > 0 && !out)) return rs_fail(nullptr, RS_ERR_ARG, "bad arguments");
  std::lock_guard<std::mutex> lock(g_mu);
  int i = 0;
  for (const auto &kv : g_cache) {
    if (i < cap_entries) out[i] = to_entry(kv.first, kv.second);
    ++i;
  }
  *count = (int32_t)g_cache.size();
  return RS_OK;
}

int rs_autotune_save(const char *path) {
  if (!path) return rs_fail(nullptr, RS_ERR_ARG, "path is NULL");
  std::vector<rs_tune_entry> v;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    for (const auto &kv : g_cache) v.push_back(to_entry(kv.first, kv.second));
  }
  const std::string tmp = std::string(path) + ".tmp";
  FILE *fp = fopen(tmp.c_str(), "w");
  if (!fp) return rs_fail(nullptr, RS_ERR_ARG, std::string("cannot write ") + tmp);
  fprintf(fp, "# librs tuner cache: kind sms cap lg_points lg_images choice persistent ms_best ms_default\n");
  for (const rs_tune_entry &e : v)
    fprintf(fp, "%d %d %d %d %d %d %d %.6g %.6g\n", e.kind, e.sms, e.cap, e.lg_points, e.lg_images, e.choice,
            e.persistent, (double)e.ms_best, (double)e.ms_default);
  const bool ok = fclose(fp) == 0;
  if (!ok || rename(tmp.c_str(), path) != 0) return rs_fail(nullptr, RS_ERR_ARG, std::string("cannot write ") + path);
  return RS_OK;
}

int rs_autotune_load(const char *path) {
  if (!path) return rs_fail(nullptr, RS_ERR_ARG, "path is NULL");
  FILE *fp = fopen(path, "r");
  if (!fp) return rs_fail(nullptr, RS_ERR_ARG, std::string("cannot read ") + path);
  std::vector<rs_tune_entry> v;
  char line[512];
  int lineno = 0;
  int rc = RS_OK;
  while (fgets(line, sizeof(line), fp)) {
    ++lineno;
    const char *s = line;
    while (*s == ' ' || *s == '\t') ++s;
    if (*s == '#' || *s == '\n' || *s == '\r' || *s == 0) continue;
    rs_tune_entry e;
    char rest[8];
    const int got = sscanf(s, "%d %d %d %d %d %d %d %f %f %7s", &e.kind, &e.sms, &e.cap, &e.lg_points,
                           &e.lg_images, &e.choice, &e.persistent, &e.ms_best, &e.ms_default, rest);
    if (got != 9 || !valid_entry(e)) {
      rc = rs_fail(nullptr, RS_ERR_ARG, std::string(path) + ":" + std::to_string(lineno) + ": malformed entry");
      break;
    }
    v.push_back(e);
  }
  fclose(fp);
  if (rc != RS_OK) return rc;
  std::lock_guard<std::mutex> lock(g_mu);
  for (const rs_tune_entry &e : v) {
    RsG1Choice c;
    c.threads = e.choice;
    c.persistent = e.persistent;
    c.ms_best = e.ms_best;
    c.ms_default = e.ms_default;
    g_cache[make_key(e.kind, e.sms, e.cap, e.lg_points, e.lg_images)] = c;
  }
  return RS_OK;
}

int rs_autotune_clear(void) {
  std::lock_guard<std::mutex> lock(g_mu);
  g_cache.clear();
  return RS_OK;
}

}  // extern "C"
