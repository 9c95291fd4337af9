// Continuous-batching request server of librs.
//
// Requests (one resultant each) are planned and copied at submission, then a
// scheduler thread admits them in arrival order while their device footprint
// (images K * N, outputs N * Lout, inputs; see rs_batch_sizes) fits the
// memory budget, groups the admitted ones into a micro-batch and runs it on
// one of several CUDA streams with stream-ordered allocation.  Micro-batches
// on different streams overlap on the GPU; a request that arrives while
// others run is admitted as soon as a stream slot and memory are free, so the
// device never waits for a whole "epoch" to drain.  Results stay on the
// device until their micro-batch finishes, then are copied back once.
#include <stdio.h>
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <thread>
#include <unordered_map>

#include "engine.h"

namespace {

using Clock = std::chrono::steady_clock;

enum { REQ_PENDING = 0, REQ_RUNNING = 1, REQ_DONE = 2 };

struct Request {
  uint64_t ticket = 0;
  PairPlan plan;
  std::vector<uint32_t> fl, gl;
  rs_bipoly f, g;
  int64_t footprint = 0;
  int state = REQ_PENDING;
  int status = RS_OK;
  std::vector<uint32_t> words;
  int deg = -1, limbs = 1;
  Clock::time_point t_submit, t_admit, t_done;
  bool admitted = false;
};

struct Flight {
  rs_batch *batch = nullptr;
  std::vector<Request *> reqs;
  cudaEvent_t done = nullptr;
  int64_t bytes = 0;
  int slot = 0;
};

}  // namespace

struct RsServer {
  rs_ctx *ctx = nullptr;
  std::thread th;
  std::mutex mu;
  std::condition_variable cv, cv_done;
  bool stop = false;
  std::deque<Request *> pending;
  std::unordered_map<uint64_t, Request *> reqs;
  uint64_t next_ticket = 1;
  int64_t mem_limit = 0, mem_used = 0;
  int max_inflight = 3, max_batch = 256;
  int min_batch = 32;                                  // launch early once this many wait
  int64_t max_images = int64_t(1) << 22;               // images per micro-batch (about 5 ms of G1)
  std::chrono::microseconds max_wait{1000};            // or once the oldest waited this long
  std::vector<cudaStream_t> streams;
  std::vector<uint32_t *> h_in, h_out;
  std::vector<int64_t> h_in_words, h_out_words;
  std::vector<bool> slot_busy;
  std::vector<Flight> flights;
  rs_server_stats st;
  FILE *log = nullptr;  // one JSON line per finished request (rs_server_set_log)
  Clock::time_point t0 = Clock::now();
};

namespace {

int grow_pinned(uint32_t *&buf, int64_t &have, int64_t need) {
  if (need <= have) return RS_OK;
  if (buf) cudaFreeHost(buf);
  buf = nullptr;
  have = 0;
  const int64_t words = need + need / 4 + 1024;
  if (cudaMallocHost((void **)&buf, words * 4) != cudaSuccess) return RS_ERR_NOMEM;
  have = words;
  return RS_OK;
}

// Called with the lock held when a request is done: its JSON line, times in
// microseconds since the server started (admit_us -1: never admitted).
void log_request(RsServer *s, const Request *r) {
  if (!s->log) return;
  auto us = [&](Clock::time_point t) {
    return (long long)std::chrono::duration_cast<std::chrono::microseconds>(t - s->t0).count();
  };
  fprintf(s->log,
          "{\"ticket\": %llu, \"status\": %d, \"submit_us\": %lld, \"admit_us\": %lld, \"done_us\": %lld, "
          "\"K\": %d, \"D\": %d, \"footprint\": %lld, \"deg\": %d, \"limbs\": %d}\n",
          (unsigned long long)r->ticket, r->status, us(r->t_submit), r->admitted ? us(r->t_admit) : -1LL,
          us(r->t_done), r->plan.K, r->plan.D, (long long)r->footprint, r->deg, r->limbs);
}

// Called with the lock held: finish flights whose event has completed.
void reap(RsServer *s) {
  for (size_t i = 0; i < s->flights.size();) {
    Flight &fl = s->flights[i];
    const cudaError_t q = cudaEventQuery(fl.done);
    if (q == cudaErrorNotReady) {
      ++i;
      continue;
    }
    const auto now = Clock::now();
    for (size_t r = 0; r < fl.reqs.size(); ++r) {
      Request *req = fl.reqs[r];
      req->status = q == cudaSuccess ? rs_unpack_one(fl.batch, (int)r, req->words, &req->deg, &req->limbs)
                                     : RS_ERR_CUDA;
      req->state = REQ_DONE;
      req->t_done = now;
      log_request(s, req);
      if (req->status == RS_OK)
        s->st.completed++;
      else
        s->st.failed++;
    }
    rs_free_batch(fl.batch);
    cudaEventDestroy(fl.done);
    s->mem_used -= fl.bytes;
    s->slot_busy[fl.slot] = false;
    s->flights.erase(s->flights.begin() + i);
    s->cv_done.notify_all();
  }
}

// Called with the lock held; releases it while the micro-batch is built.
void launch(RsServer *s, std::unique_lock<std::mutex> &lk) {
  int slot = -1;
  for (int i = 0; i < (int)s->slot_busy.size(); ++i)
    if (!s->slot_busy[i]) {
      slot = i;
      break;
    }
  if (slot < 0 || s->pending.empty()) return;
  std::vector<Request *> take;
  int64_t bytes = 0, images = 0;
  while (!s->pending.empty() && (int)take.size() < s->max_batch) {
    Request *r = s->pending.front();
    // a micro-batch holds at most max_images images (K N), so that one large
    // request does not hold up many small ones behind it
    const int64_t im = (int64_t)r->plan.K * r->plan.N;
    if (!take.empty() && images + im > s->max_images) break;
    if (r->footprint > s->mem_limit) {  // can never fit: fail it
      s->pending.pop_front();
      r->status = RS_ERR_NOMEM;
      r->state = REQ_DONE;
      r->t_done = Clock::now();
      log_request(s, r);
      s->st.failed++;
      s->cv_done.notify_all();
      continue;
    }
    if (s->mem_used + bytes + r->footprint > s->mem_limit) break;
    bytes += r->footprint;
    images += im;
    take.push_back(r);
    s->pending.pop_front();
  }
  if (take.empty()) return;
  s->slot_busy[slot] = true;
  s->mem_used += bytes;
  const auto t_admit = Clock::now();
  for (Request *r : take) {
    r->state = REQ_RUNNING;
    r->t_admit = t_admit;
    r->admitted = true;
  }
  lk.unlock();

  const int n = (int)take.size();
  std::vector<rs_bipoly> F(n), G(n);
  std::vector<PairPlan> plans(n);
  for (int i = 0; i < n; ++i) {
    F[i] = take[i]->f;
    G[i] = take[i]->g;
    plans[i] = take[i]->plan;
  }
  int64_t in_w = 0, out_w = 0, dev_b = 0;
  rs_batch_sizes(plans, F.data(), G.data(), &in_w, &out_w, &dev_b);
  int rc = grow_pinned(s->h_in[slot], s->h_in_words[slot], in_w);
  if (rc == RS_OK) rc = grow_pinned(s->h_out[slot], s->h_out_words[slot], out_w);
  RsBatchOpts o;
  o.stream = s->streams[slot];
  o.stream_ordered = true;
  o.use_graph = false;
  o.persistent = s->ctx->cfg.persistent != 0;
  o.tune = false;  // cached tuner choices only: timing here would stall the scheduler
  o.fork = false;  // micro-batches already overlap on the server's streams
  o.h_in = s->h_in[slot];
  o.h_out = s->h_out[slot];
  o.h_in_words = s->h_in_words[slot];
  o.h_out_words = s->h_out_words[slot];
  rs_batch *b = nullptr;
  if (rc == RS_OK) rc = rs_build_batch(s->ctx, n, F.data(), G.data(), std::move(plans), o, &b);
  if (rc == RS_OK) rc = rs_upload(b, F.data(), G.data());
  if (rc == RS_OK) rc = rs_run(b);
  if (rc == RS_OK) rc = rs_fetch_async(b);
  cudaEvent_t ev = nullptr;
  if (rc == RS_OK && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) rc = RS_ERR_CUDA;
  if (rc == RS_OK && cudaEventRecord(ev, o.stream) != cudaSuccess) rc = RS_ERR_CUDA;

  lk.lock();
  if (rc != RS_OK) {
    if (ev) cudaEventDestroy(ev);
    if (b) {
      cudaStreamSynchronize(o.stream);
      rs_free_batch(b);
    }
    for (Request *r : take) {
      r->status = rc;
      r->state = REQ_DONE;
      r->t_done = Clock::now();
      log_request(s, r);
      s->st.failed++;
    }
    s->mem_used -= bytes;
    s->slot_busy[slot] = false;
    s->cv_done.notify_all();
    return;
  }
  Flight fl;
  fl.batch = b;
  fl.reqs = std::move(take);
  fl.done = ev;
  fl.bytes = bytes;
  fl.slot = slot;
  s->flights.push_back(fl);
  s->st.batches++;
  s->st.kernel_launches += b->info.kernel_launches;
  s->st.running = 0;
  for (auto &f2 : s->flights) s->st.running += (int64_t)f2.reqs.size();
  if ((int64_t)s->flights.size() > s->st.peak_inflight_batches) s->st.peak_inflight_batches = (int64_t)s->flights.size();
  if (s->st.running > s->st.peak_running) s->st.peak_running = s->st.running;
}

void loop(RsServer *s) {
  cudaSetDevice(s->ctx->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    reap(s);
    // Launch when a stream is free and either the GPU is idle, enough
    // requests have accumulated for a full micro-batch share, or the oldest
    // pending request has waited max_wait: larger micro-batches while the
    // GPU is busy, no waiting when it is idle.
    bool can_launch = !s->pending.empty() && (int)s->flights.size() < s->max_inflight;
    if (can_launch && !s->flights.empty()) {
      const auto age = Clock::now() - s->pending.front()->t_submit;
      can_launch = (int)s->pending.size() >= s->min_batch || age >= s->max_wait;
    }
    if (can_launch) {
      const size_t before = s->pending.size();
      launch(s, lk);
      if (s->pending.size() != before) continue;  // launched or failed something: look again
    }
    if (s->stop && s->pending.empty() && s->flights.empty()) break;
    if (!s->flights.empty())
      s->cv.wait_for(lk, std::chrono::microseconds(20));
    else
      s->cv.wait(lk);
  }
}

int start(rs_ctx *ctx, int32_t max_inflight, int32_t max_batch, int64_t mem_limit) {
  if (ctx->server) return RS_OK;
  RsServer *s = new RsServer();
  s->ctx = ctx;
  memset(&s->st, 0, sizeof(s->st));
  s->max_inflight = max_inflight > 0 ? max_inflight : 3;
  s->max_batch = max_batch > 0 ? max_batch : 256;
  s->min_batch = std::max(1, std::min(32, s->max_batch / 4));
  if (mem_limit <= 0) mem_limit = ctx->cfg.mem_limit_bytes;
  if (mem_limit <= 0) {
    size_t fr = 0, tot = 0;
    cudaSetDevice(ctx->device);
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) fr = (size_t)1 << 30;
    mem_limit = (int64_t)(fr / 2);
  }
  s->mem_limit = mem_limit;
  s->st.mem_limit = mem_limit;
  cudaSetDevice(ctx->device);
  for (int i = 0; i < s->max_inflight; ++i) {
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      for (auto x : s->streams) cudaStreamDestroy(x);
      delete s;
      return rs_fail(ctx, RS_ERR_CUDA, "server: cudaStreamCreate");
    }
    s->streams.push_back(st);
  }
  s->h_in.assign(s->max_inflight, nullptr);
  s->h_out.assign(s->max_inflight, nullptr);
  s->h_in_words.assign(s->max_inflight, 0);
  s->h_out_words.assign(s->max_inflight, 0);
  s->slot_busy.assign(s->max_inflight, false);
  ctx->server = s;
  s->th = std::thread(loop, s);
  return RS_OK;
}

int take_result(RsServer *s, Request *r, rs_upoly *out, double *latency_ms) {
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  int rc = r->status;
  if (rc == RS_OK) {
    if (!out) return RS_ERR_ARG;
    out->deg = r->deg;
    out->limbs = r->limbs;
    if ((int64_t)r->words.size() > out->capacity_words) return RS_ERR_CAPACITY;  // keep the ticket
    if (!r->words.empty()) {
      if (!out->coeffs) return RS_ERR_ARG;
      memcpy(out->coeffs, r->words.data(), r->words.size() * 4);
    }
  }
  s->reqs.erase(r->ticket);
  delete r;
  return rc;
}

}  // namespace

void rs_server_shutdown(rs_ctx *ctx) {
  RsServer *s = ctx->server;
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->th.joinable()) s->th.join();
  cudaSetDevice(ctx->device);
  for (auto st : s->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  for (auto p : s->h_in)
    if (p) cudaFreeHost(p);
  for (auto p : s->h_out)
    if (p) cudaFreeHost(p);
  for (auto &kv : s->reqs) delete kv.second;
  if (s->log) fclose(s->log);
  delete s;
  ctx->server = nullptr;
}

extern "C" {

int rs_server_start(rs_ctx *ctx, int32_t max_inflight, int32_t max_batch, int64_t mem_limit_bytes) {
  if (!ctx || max_inflight < 0 || max_batch < 0) return rs_fail(ctx, RS_ERR_ARG, "bad arguments");
  return start(ctx, max_inflight, max_batch, mem_limit_bytes);
}

int rs_server_submit(rs_ctx *ctx, const rs_bipoly *f, const rs_bipoly *g, uint64_t *ticket) {
  if (!ctx || !f || !g || !ticket) return rs_fail(ctx, RS_ERR_ARG, "NULL argument");
  if (!ctx->server) {
    int rc = start(ctx, 0, 0, 0);
    if (rc != RS_OK) return rc;
  }
  RsServer *s = ctx->server;
  Request *r = new Request();
  r->t_submit = Clock::now();
  const char *why = "";
  int rc = rs_plan_pair(f, g, ctx->log2p, r->plan, &why);
  if (rc != RS_OK) {
    delete r;
    return rs_fail(ctx, rc, why);
  }
  r->fl.assign(f->coeffs, f->coeffs + rs_input_words(*f));
  r->gl.assign(g->coeffs, g->coeffs + rs_input_words(*g));
  r->f = *f;
  r->f.coeffs = r->fl.data();
  r->g = *g;
  r->g.coeffs = r->gl.data();
  int64_t in_w, out_w, dev_b;
  std::vector<PairPlan> one(1, r->plan);
  rs_batch_sizes(one, &r->f, &r->g, &in_w, &out_w, &dev_b);
  r->footprint = dev_b;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->ticket = s->next_ticket++;
    s->reqs[r->ticket] = r;
    s->pending.push_back(r);
    s->st.submitted++;
  }
  s->cv.notify_all();
  *ticket = r->ticket;
  return RS_OK;
}

int rs_server_poll(rs_ctx *ctx, uint64_t ticket, rs_upoly *out, double *latency_ms) {
  if (!ctx || !ctx->server) return rs_fail(ctx, RS_ERR_STATE, "server not running");
  RsServer *s = ctx->server;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return rs_fail(ctx, RS_ERR_ARG, "unknown ticket");
  if (it->second->state != REQ_DONE) return RS_PENDING;
  return take_result(s, it->second, out, latency_ms);
}

int rs_server_wait(rs_ctx *ctx, uint64_t ticket, rs_upoly *out, double *latency_ms, int64_t timeout_us) {
  if (!ctx || !ctx->server) return rs_fail(ctx, RS_ERR_STATE, "server not running");
  RsServer *s = ctx->server;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return rs_fail(ctx, RS_ERR_ARG, "unknown ticket");
  Request *r = it->second;
  const auto pred = [&] { return r->state == REQ_DONE; };
  if (timeout_us < 0)
    s->cv_done.wait(lk, pred);
  else if (!s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), pred))
    return RS_ERR_TIMEOUT;
  return take_result(s, r, out, latency_ms);
}

int rs_server_stats_get(rs_ctx *ctx, rs_server_stats *out) {
  if (!ctx || !out) return rs_fail(ctx, RS_ERR_ARG, "NULL argument");
  if (!ctx->server) {
    memset(out, 0, sizeof(*out));
    return RS_OK;
  }
  RsServer *s = ctx->server;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->st;
  out->pending = (int64_t)s->pending.size();
  out->inflight_batches = (int64_t)s->flights.size();
  out->mem_used = s->mem_used;
  out->running = 0;
  for (auto &f : s->flights) out->running += (int64_t)f.reqs.size();
  return RS_OK;
}

int rs_server_set_log(rs_ctx *ctx, const char *path) {
  if (!ctx) return rs_fail(ctx, RS_ERR_ARG, "NULL argument");
  RsServer *s = ctx->server;
  if (!s) return rs_fail(ctx, RS_ERR_STATE, "no server running");
  FILE *f = nullptr;
  if (path && !(f = fopen(path, "w"))) return rs_fail(ctx, RS_ERR_ARG, std::string("cannot open ") + path);
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->log) fclose(s->log);
  s->log = f;
  return RS_OK;
}

int rs_server_stop(rs_ctx *ctx) {
  if (!ctx) return rs_fail(ctx, RS_ERR_ARG, "NULL argument");
  rs_server_shutdown(ctx);
  return RS_OK;
}

}  // extern "C"
