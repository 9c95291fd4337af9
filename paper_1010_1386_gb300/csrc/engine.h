// Internal host-side structures of librs shared by engine.cu (contexts,
// batches, C ABI) and server.cu (continuous-batching request server).
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "planner.h"
#include "rs_internal.cuh"

struct RsServer;  // server.cu

// Makes device d current for the scope and restores the previous device.
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

// Point and interpolation tables per prime, shared by every batch of a
// context and grown on demand (old allocations are kept until the context is
// destroyed, so captured graphs stay valid).
struct RsTables {
  int K = 0;        // primes covered
  int N = 0;        // interpolation stride (point pairs covered)
  int cstride = 0;  // chirp stride (point pair + x-degree + tile window covered)
  uint32_t *finv = nullptr, *gtab = nullptr, *hq = nullptr, *qn = nullptr, *qp = nullptr;
  int32_t *btab = nullptr, *qc = nullptr;
  // Chinese-remaindering tables for the first K primes.
  int32_t *wtab = nullptr;   // triangular p_0 ... p_{l-1} mod p_k
  uint16_t *p16 = nullptr;   // prefix products in 16-bit digits
  int32_t *poff = nullptr;   // K + 1 row offsets into p16
  int32_t *nh = nullptr;     // digits per prefix product
  std::vector<int32_t> h_nh;  // the same counts on the host
};

struct rs_ctx {
  int device = 0;
  rs_config cfg;
  rs_sqf_info sqf_info{};  // the last square-free call
  cudaStream_t stream = nullptr;
  int sms = 0;
  std::vector<uint32_t> primes;
  std::vector<double> log2p;
  uint32_t *d_primes = nullptr;
  int32_t *d_stall = nullptr;  // test hook read by the tensor-core kernels' copy warps (0 = normal)
  ModP *d_mods = nullptr;
  uint32_t *d_vtab = nullptr;
  uint32_t *d_crt = nullptr;
  uint32_t *d_qbase = nullptr;
  std::string err;
  std::vector<rs_batch *> batches;
  rs_batch *cache = nullptr;
  rs_batch *sqf_cache = nullptr;  // the last square-free batch, reused for the same shapes
  void *sqf_arena = nullptr;      // the factor CRT's device arena, grown on demand
  size_t sqf_arena_bytes = 0;
  std::mutex tab_mu;
  RsTables tab;
  std::vector<RsTables> retired;
  RsServer *server = nullptr;
  std::mutex prep_mu;  // kernel attributes and the occupancy cache below
  bool g2_ready = false;
  std::map<int64_t, int> g1_occupancy;  // (capacity, threads, staged KiB) -> blocks per SM
  std::string tune_path;                 // autotune cache file written at rs_destroy ("" = none)
  cudaStream_t side[8] = {};             // branches of the fork-join stage launches
  // Transform-based G2: NTT primes and twiddles, and per transform length 2^lg
  // the transformed interpolation kernels of the first bhat_K[lg] primes
  // (guarded by tab_mu; grown tables keep their old allocation until the
  // context is destroyed).
  NttConst nttc;
  uint2 *d_ntt_tw = nullptr;
  uint32_t *bhat[RS_NTT_LGMAX + 1] = {};
  int bhat_K[RS_NTT_LGMAX + 1] = {};
  std::vector<void *> bhat_retired;
  bool g2n_ready = false;
  // Tensor-core G2: the Toeplitz digit tiles of the first g2t_K primes,
  // g2t_tiles per prime (guarded by tab_mu; replaced tables are kept until
  // the context is destroyed, as graphs may still read them).
  uint16_t *g2t_bt = nullptr;
  int g2t_K = 0, g2t_tiles = 0;
  std::vector<void *> g2t_retired;
  bool g2t_ready = false;
  // Tensor-core CRT digits: W digit tiles of the digit blocks kb < g3m_KB
  // (same lifetime rules as above).
  uint16_t *g3m_wt = nullptr;
  uint16_t *g3m_rt = nullptr;  // per block: the rect digit tile (W of its last 32 primes on its first 32)
  int g3m_KB = 0;
  std::vector<void *> g3m_retired;
  bool g3m_ready = false;
  // Tensor-core CRT limbs: prefix-product tiles of the chunks c < g3l_KB,
  // block g3l_cbase[c] + u for the units u that chunk c reaches (host and
  // device copies of cbase; same lifetime rules, kept in g3m_retired).
  uint16_t *g3l_bt = nullptr;
  int32_t *g3l_cbase = nullptr;
  std::vector<int32_t> h_g3l_cbase;
  int g3l_KB = 0;
  bool g3l_ready = false;
};

struct RsClassLaunch {
  int cap = 0;
  int threads = 128;
  int persistent = 1;
  double cost = 0.0;  // modular products of the class (launch order: costliest first)
  int blocks = 0;
  int64_t tile_off = 0;
  int ntiles = 0;
  size_t smem = 0;
};

struct RsG2Class {
  int lg = 0;  // > 0: transform-based (or tensor-core) G2 of length group 2^lg; 0: direct convolutions
  bool tensor = false;  // tensor-core products over row tiles (kernels_g2t.cu)
  int64_t t_task_off = 0, t_item_off = 0;  // first task / work item of the class in the batch lists
  int t_ntask = 0, t_nitem = 0, t_maxM = 0;
  int threads = 256;
  int64_t off = 0;  // first task of the class in the G2 task list
  int count = 0;
  size_t smem = 0;
};

struct RsBatchOpts {
  bool images_only = false;
  cudaStream_t stream = nullptr;  // NULL: the context's stream
  bool stream_ordered = false;    // allocate with cudaMallocAsync on `stream`
  uint32_t *h_in = nullptr;       // borrowed pinned staging (NULL: allocate)
  uint32_t *h_out = nullptr;
  int64_t h_in_words = 0, h_out_words = 0;
  bool use_graph = true;
  bool persistent = true;
  bool fork = true;     // run the launches of a stage (capacity / G2 classes) as parallel branches
  bool tune = true;     // time G1 choices for classes missing from the tuner cache
  bool timing = false;  // record stage events even when the context does not time
  int g1_threads = 0;   // > 0: force this tile width (and opt.persistent) for every class
  int g2_force = -1;    // 0: direct G2 for every pair, 1: transforms, 2: tensor cores wherever possible, -1: choose
  int yun_maxm = 0;     // > 0: square-free factorisation of R mod every prime after G2 (up to this multiplicity)
};

struct rs_batch {
  rs_ctx *ctx = nullptr;
  int n = 0;
  RsBatchOpts opt;
  cudaStream_t stream = nullptr;
  std::vector<PairPlan> plans;
  std::vector<int> dev_index;  // pair -> device pair index, -1 if none
  std::vector<PairDesc> descs;
  std::vector<int64_t> in_f, in_g;  // word offsets of each pair's inputs in the staging buffer
  std::vector<RsClassLaunch> classes;
  std::vector<RsG2Class> g2cls;
  // Schur variant of G1 (rs_config.univariate = 1): one launch over every
  // tile, then the elimination fallback over the listed images.
  bool schur = false;
  int schur_slots = 0, ntiles_all = 0;
  size_t schur_smem = 0, schur_fb_smem = 0;
  int2 *d_fail = nullptr;
  int64_t in_words = 0, img_words = 0, out_words = 0;
  int64_t shape_off = 0;  // word offset of the per-pair result shapes in the output buffer
  int64_t status_off = 0; // word offset of the device status word (0 = every bounded wait completed)
  int ng2 = 0, ng3 = 0, g2_threads = 256;
  int ng3d = 0, ng3b = 0, kmax = 0;  // CRT digit tiles, limb chunks, largest K
  int g3_jt = 32;                    // coefficients per CRT digit tile (32 or 16)
  bool g3_perthread = false;         // CRT digits with one thread per coefficient
  bool g3_tensor = false;            // CRT digits on the tensor cores (kernels_g3m.cu)
  int64_t g3m_x_elems = 0;           // their operand digits
  uint16_t *d_g3m_x = nullptr;
  int64_t *d_g3m_xoff = nullptr;
  int64_t xl_words = 0, cy_words = 0;
  int2 *d_g3d = nullptr;
  int nyun = 0;                         // square-free tasks (pair, prime)
  int64_t yun_ostride = 0, yun_wstride = 0;
  int2 *d_yun_tasks = nullptr;
  uint32_t *d_yun_out = nullptr, *d_yun_work = nullptr;
  int4 *d_g3b = nullptr;
  // Tensor-core G2: tasks, row tiles, work items, operand digits and products.
  G2tTask *d_g2t_tasks = nullptr;
  G2tRowTile *d_g2t_rts = nullptr;
  G2tItem *d_g2t_items = nullptr;
  uint16_t *d_g2t_x = nullptr;
  uint32_t *d_g2t_y = nullptr;
  int64_t g2t_x_elems = 0;
  int64_t *d_cy = nullptr;
  size_t g2smem = 0;
  void *arena = nullptr;  // one device allocation carved into the buffers below
  uint32_t *d_in = nullptr;
  int2 *d_meta = nullptr;
  PairDesc *d_pairs = nullptr;
  Tile *d_tiles = nullptr;
  int32_t *d_counters = nullptr;
  uint32_t *d_num = nullptr, *d_den = nullptr, *d_xl = nullptr, *d_out = nullptr;
  int2 *d_g2 = nullptr, *d_g3 = nullptr;
  unsigned long long *d_stats = nullptr;
  uint32_t *h_in = nullptr, *h_out = nullptr;
  bool own_host = false;
  cudaGraphExec_t gexec = nullptr;
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // stage bounds; [4] before Yun
  cudaEvent_t fev[2] = {nullptr, nullptr};  // fork points of the G1 and G2 stages
  std::vector<cudaEvent_t> jev;             // joins of the branches (one per launch of a forked stage)
  bool ran = false;
  rs_batch_info info;
};

int rs_fail(rs_ctx *c, int code, const std::string &msg);
int rs_cuda_code(cudaError_t e);
int rs_plan_all(rs_ctx *ctx, int n, const rs_bipoly *f, const rs_bipoly *g,
                std::vector<PairPlan> &plans, int32_t *status, int *first_err);
bool rs_same_shape(const PairPlan &a, const PairPlan &b);
int64_t rs_input_words(const rs_bipoly &p);
int rs_ensure_tables(rs_ctx *ctx, int K, int N, int dx);
// Transformed interpolation kernels of length 2^lg for at least K primes.
int rs_ensure_bhat(rs_ctx *ctx, int lg, int K);
// Toeplitz digit tiles of the tensor-core G2 for at least K primes and
// `tiles` diagonal offsets per prime (the point tables must cover K first).
int rs_ensure_g2t_btile(rs_ctx *ctx, int K, int tiles);
// W digit tiles of the tensor-core CRT digits for digit blocks kb < KB.
int rs_ensure_g3m_wtiles(rs_ctx *ctx, int KB);
int rs_ensure_g3l_tiles(rs_ctx *ctx, int KB);
// log2 of the G2 transform length for N points (2^lg >= 2N - 1), 0 when
// above the transform limit; model cost of a form (0 direct, 1 transforms).
int rs_g2_len(int N);
double rs_g2_cost(int N, int form);
int rs_build_batch(rs_ctx *ctx, int n, const rs_bipoly *f, const rs_bipoly *g,
                   std::vector<PairPlan> &&plans, const RsBatchOpts &opt, rs_batch **out);
// Byte sizes a batch of these plans needs (device arena, host staging in/out).
void rs_batch_sizes(const std::vector<PairPlan> &plans, const rs_bipoly *f, const rs_bipoly *g,
                    int64_t *in_words, int64_t *out_words, int64_t *device_bytes);
int rs_upload(rs_batch *b, const rs_bipoly *f, const rs_bipoly *g);
int rs_run(rs_batch *b);
int rs_fetch_async(rs_batch *b);                                // enqueue the result copy
int rs_unpack(rs_batch *b, rs_upoly *out, int32_t *status);     // after the copy completed
// Unpack pair i into a freshly sized host vector (deg, limbs); returns status.
int rs_unpack_one(rs_batch *b, int i, std::vector<uint32_t> &words, int *deg, int *limbs);
void rs_free_batch(rs_batch *b);
void rs_server_shutdown(rs_ctx *ctx);  // server.cu

// G1 launch tuner (autotune.cu).  A workload class is (SM count, register
// capacity, floor(log2 of its largest point count), floor(log2 of its images));
// the process-wide cache maps it to a tile width and a schedule.
struct RsG1Choice {
  int threads = 128;  // G2 entries: the form (1 = transforms, 0 = direct)
  int persistent = 1;
  float ms_best = 0.f, ms_default = 0.f;
};
int64_t rs_tune_key(int sms, int cap, int max_points, int64_t images);
int64_t rs_tune_key_g2(int sms, int lg, int64_t images);
// Time the whole path on (a sample of) a transform-length group with each G2
// form and cache the faster (the model's form unless the other wins by 2%).
int rs_tune_g2(rs_ctx *ctx, const rs_bipoly *f, const rs_bipoly *g, const std::vector<PairPlan> &plans,
               const std::vector<int> &members, int64_t key, int model_form, int *form);
bool rs_tune_find(int64_t key, RsG1Choice *out);
// Time every candidate on (a sample of) the class's pairs and cache the fastest.
int rs_tune_g1(rs_ctx *ctx, const rs_bipoly *f, const rs_bipoly *g, const std::vector<PairPlan> &plans,
               const std::vector<int> &members, int64_t key, RsG1Choice *out);
