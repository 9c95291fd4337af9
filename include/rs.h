/*
 * rs.h -- C ABI of librs: exact bivariate resultants Res_y(f, g) in Z[x] on
 * one NVIDIA GB300 (sm_103a).
 *
 * Problem (paper, Section 2, Eq. (2.1)): f, g in Z[x, y],
 *     f = sum_{i,j} f_ij x^i y^j = sum_{j=0}^{m_y} f_j^{(y)}(x) y^j,
 * and likewise g with y-degree n_y.  Output (Section 3.1): the resultant
 * R^{(y)} = res(f, g, y) in Z[x], the determinant of the (m_y+n_y)-square
 * Sylvester matrix whose first n_y rows hold f_{m_y}^{(y)}, ..., f_0^{(y)}
 * and whose last m_y rows hold g_{n_y}^{(y)}, ..., g_0^{(y)}, each row shifted
 * one column right of the one above it.  deg R^{(y)} <= m * n (total degrees).
 *
 * Method (Section 4.1, Collins' modular algorithm): coefficients are mapped
 * to Z_p for many 31-bit primes p and evaluated at many points x_i; one
 * univariate resultant z_i^{(p)} = res(f(x_i, y), g(x_i, y), y) in Z_p is
 * taken per (prime, point); R mod p is interpolated per prime; the integer
 * coefficients are recovered by Chinese remaindering.  All of it runs on the
 * GPU; the host only plans (degrees, bounds, prime count) and copies.
 *
 * Conventions where the paper is silent: f == 0 or g == 0 gives R = 0;
 * m_y = n_y = 0 gives R = 1 (empty determinant).  Degrees are taken after
 * trimming zero rows/columns; the y-degrees used are the actual y-degrees of
 * f and g over Z[x].
 *
 * Memory: every pointer in this header is a HOST pointer.  Input arrays are
 * owned by the caller and only read during the call.  Output arrays are owned
 * by the caller and written only when the call returns RS_OK.  The context
 * owns all device memory, its CUDA stream and its CUDA graphs.  A context is
 * bound to the CUDA device that was current (or named in rs_config) when it
 * was created and is not thread-safe: use one context per host thread.
 *
 * Errors: every int-returning call returns RS_OK (0), RS_PENDING (1) or a
 * negative RS_ERR_* code; rs_last_error() gives a one-line description.
 */
#ifndef RS_H
#define RS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  RS_OK = 0,
  RS_PENDING = 1,        /* serving: request not finished yet */
  RS_ERR_ARG = -1,       /* NULL pointer, negative extent, limbs out of range */
  RS_ERR_CAPACITY = -2,  /* output buffer too small; out->deg/limbs hold the need */
  RS_ERR_NOMEM = -3,     /* device or host allocation failed / pool exhausted */
  RS_ERR_CUDA = -4,      /* a CUDA runtime call failed (no device, launch error) */
  RS_ERR_TIMEOUT = -5,   /* a bounded device-side wait ran out */
  RS_ERR_LIMIT = -6,     /* input exceeds a library limit (see RS_MAX_*) */
  RS_ERR_STATE = -7      /* call not valid in the object's current state */
};

/* Library limits. */
#define RS_MAX_LIMBS 128       /* input coefficients up to 4096 bits */
#define RS_MAX_DEG_Y 71        /* y-degree of f and of g */
#define RS_MAX_POINTS 16384    /* degree bound D + 1 of the resultant */
#define RS_MAX_PRIMES 16384    /* 31-bit primes available for the CRT */

/* A bivariate polynomial f in Z[x, y] (Eq. (2.1)), dense, x-major:
 * coefficient f_ij is coeffs[((i * (deg_y + 1)) + j) * limbs + k], k = 0..limbs-1,
 * little-endian 32-bit limbs in two's complement.  deg_x, deg_y are the array
 * extents minus one (>= 0); zero top rows/columns are allowed and trimmed. */
typedef struct {
  int32_t deg_x;
  int32_t deg_y;
  int32_t limbs;
  const uint32_t *coeffs;
} rs_bipoly;

/* A univariate result R in Z[x]: coefficient of x^i is
 * coeffs[i * limbs + k], k = 0..limbs-1, two's complement.  capacity_words is
 * set by the caller (u32 words available); deg (-1 for R = 0) and limbs are
 * written by the library.  On RS_ERR_CAPACITY, deg and limbs hold the bound
 * that the caller must provide room for ((deg + 1) * limbs words). */
typedef struct {
  int32_t deg;
  int32_t limbs;
  int64_t capacity_words;
  uint32_t *coeffs;
} rs_upoly;

typedef struct {
  int32_t device;            /* CUDA device ordinal, -1 = the current device */
  int32_t tile_points;       /* G1 points per block: 32, 64 or 128 forces that width for every
                                class; 0 = per class from the tuner (see rs_autotune) */
  int32_t use_graphs;        /* 1 = replay batch runs as CUDA graphs */
  int32_t persistent;        /* 1 = the tuner may pick persistent G1 launches over a cost-sorted
                                tile list; 0 = one block per tile always */
  int32_t timing;            /* 1 = record per-stage CUDA events on each run */
  int32_t autotune;          /* 1 = a batch whose workload class is not in the tuner cache times
                                the G1 candidates first; 0 = cached choices or the built-in
                                default (128 points, persistent) */
  int32_t g2_form;           /* interpolation: 0 = convolutions, per pair by a cost model, 1 = direct
                                convolutions (lazily reduced dot products) only, 2 = number-theoretic
                                transforms wherever D + 1 <= 4096, 3 = triangular factorisation of the
                                Vandermonde system (the paper's Section 4.1 solve; comparison form,
                                D + 1 <= 14,000), 4 = the convolutions of all pairs of a prime as
                                one exact matrix product on the tensor cores (bf16 digit products
                                with fp32 accumulation) wherever D + 1 <= 8192 */
  int32_t univariate;        /* univariate resultants mod p (G1): 0 = division-free remainder
                                sequence, one thread per image; 1 = the generalised Schur algorithm
                                on displacement generators of the Sylvester matrix (the paper's
                                Section 4.1 kernel), one warp per image, for comparison */
  int64_t mem_limit_bytes;   /* serving: device bytes admitted requests may hold; 0 = auto */
  const char *autotune_cache;  /* tuner cache file merged at rs_create (a missing file is not an
                                  error) and rewritten at rs_destroy; NULL = none.  The string
                                  is copied. */
  int32_t crt_form;          /* Chinese remaindering digits: 0 = by the batch's shape (one thread
                                per coefficient when there are at least 1024 coefficients per SM;
                                else the tensor cores when some pair has at least 128 primes and
                                the batch has 128-coefficient tiles for half the SMs, or some pair
                                has at least 1024 primes; else tiles on the CUDA cores), 1 = CUDA
                                cores only, 2 = tensor cores whenever the batch does not take one
                                thread per coefficient.  With tensor-core digits the limbs
                                sum_k v_k P_k are a tensor-core product too. */
  int32_t reserved;          /* 0 */
} rs_config;

typedef struct rs_ctx rs_ctx;
typedef struct rs_batch rs_batch;

/* Fill *cfg with the defaults (device -1, tiles autotuned, graphs and
 * persistent kernels on, timing off, autotuning on without a cache file,
 * memory limit auto). */
int rs_config_default(rs_config *cfg);

/* Create a context on the configured device: allocates the prime table and
 * its CRT constants on the device and a non-blocking stream.  cfg may be
 * NULL for the defaults.  Returns RS_ERR_CUDA when no usable GPU exists. */
int rs_create(rs_ctx **ctx, const rs_config *cfg);

/* Release every device resource of the context (batches included). */
int rs_destroy(rs_ctx *ctx);

/* The context's CUDA stream (a cudaStream_t) for callers that time or order
 * work around the library's launches. */
int rs_stream(rs_ctx *ctx, void **stream);

/* Static description of an error code, and the last error of a context
 * (ctx may be NULL for errors of calls that have no context). */
const char *rs_error_string(int code);
const char *rs_last_error(const rs_ctx *ctx);

/* Host-only planning, no GPU needed: the degree bound D of R (Section 3.1:
 * D = min(m_x n_y + n_x m_y, m n)), the limbs an output coefficient needs
 * (from the Hadamard bound on the Sylvester rows, |coef R| < 2^bits), and
 * the number of 31-bit primes the CRT uses.  Any output pointer may be NULL.
 * *deg_bound is -1 when f or g is zero. */
int rs_result_bound(const rs_bipoly *f, const rs_bipoly *g, int32_t *deg_bound,
                    int32_t *limbs_bound, int32_t *primes, int32_t *bits);

/* R = Res_y(f, g) (Section 3.1) through the modular method (Section 4.1). */
int rs_resultant_y(rs_ctx *ctx, const rs_bipoly *f, const rs_bipoly *g, rs_upoly *out);

/* n independent resultants out[i] = Res_y(f[i], g[i]) in one batched run:
 * one persistent G1 launch per register-capacity class over the flattened
 * (pair, prime, point) work list, then batched interpolation and CRT.
 * status (may be NULL) receives each pair's code; the call returns the
 * first failure, RS_OK if none. */
int rs_resultant_batch(rs_ctx *ctx, int32_t n, const rs_bipoly *f, const rs_bipoly *g,
                       rs_upoly *out, int32_t *status);

/* Prepared batches: plan once and keep the inputs resident on the device,
 * then run as often as wanted.  rs_batch_run only enqueues on the batch's
 * stream (a CUDA graph when enabled); rs_batch_sync waits for it;
 * rs_batch_results copies the last run's results to the host. */
int rs_batch_create(rs_ctx *ctx, int32_t n, const rs_bipoly *f, const rs_bipoly *g,
                    rs_batch **batch);
/* As rs_batch_create, with every copy and launch of the batch enqueued on
 * the caller's CUDA stream (a cudaStream_t of the context's device; NULL =
 * the context's stream).  Batches on different streams overlap: while one
 * runs, another's results can be copied back and its next inputs uploaded.
 * The stream must outlive the batch. */
int rs_batch_create_on(rs_ctx *ctx, int32_t n, const rs_bipoly *f, const rs_bipoly *g, void *stream,
                       rs_batch **batch);
/* New inputs for a prepared batch (copied into its pinned staging and sent
 * to the device on its stream).  The inputs are planned again: if any pair's
 * plan (degrees, prime count, output limbs) differs from the batch's, the
 * call returns RS_ERR_STATE and uploads nothing. */
int rs_batch_upload(rs_batch *batch, int32_t n, const rs_bipoly *f, const rs_bipoly *g);
int rs_batch_run(rs_batch *batch);
int rs_batch_sync(rs_batch *batch);
int rs_batch_results(rs_batch *batch, rs_upoly *out, int32_t *status);
int rs_batch_destroy(rs_batch *batch);

/* Work and timing of a prepared batch.  Counts are per run; stage times are
 * those of the last run (only when rs_config.timing = 1, else -1). */
typedef struct {
  int64_t pairs;
  int64_t images;             /* (pair, prime, point) univariate resultants */
  int64_t primes_total;       /* sum over pairs of the prime count K */
  int64_t coeffs_total;       /* sum over pairs of D + 1 */
  double modmul_eval;         /* algorithmic modular products: evaluation (a3; the two images of
                                  a point pair +-x share one evaluation of the even and odd
                                  parts, plus one product per coefficient each) */
  double modmul_prs;          /* univariate resultants (a4) */
  double modmul_interp;       /* interpolation (a5) */
  double modmul_crt;          /* Garner CRT (a6) */
  int64_t input_bytes;        /* host->device bytes of one upload */
  int64_t output_bytes;       /* device->host bytes of one result fetch */
  float ms_images;            /* G1 (reduce + evaluate + resultant) */
  float ms_interp;            /* G2 */
  float ms_crt;               /* G3 */
  float ms_total;
  int64_t unlucky_points;     /* images with lc_y f(x_i) lc_y g(x_i) = 0 mod p */
  int64_t degenerate_images;  /* images whose remainder sequence hit a zero pivot */
  int64_t unlucky_primes;     /* (pair, prime) with lc_y f or lc_y g = 0 mod p */
  int64_t kernel_launches;    /* kernels of the library launched per run */
  float ms_yun;               /* square-free factorisation mod p (rs_squarefree_batch only; inside
                                 the span ms_interp measures otherwise) */
  int32_t reserved;
} rs_batch_info;

int rs_batch_info_get(rs_batch *batch, rs_batch_info *info);

/* R^{(x)} = res(f, g, x) in Z[y] (Section 3.1: defined like R^{(y)} with f
 * and g read as polynomials in x over Z[y]).  The library exchanges the
 * variables of copies of f and g on the host and runs the same path; out
 * receives the coefficients of y^0 .. y^deg.  Errors as rs_resultant_y. */
int rs_resultant_x(rs_ctx *ctx, const rs_bipoly *f, const rs_bipoly *g, rs_upoly *out);

/* Both projections of each pair (the PROJECT phase of the paper's solver
 * computes R^{(y)} and R^{(x)}, Section 3.1 / Theorem 3.1): out_y[i] =
 * res(f_i, g_i, y) in Z[x] and out_x[i] = res(f_i, g_i, x) in Z[y], all 2n
 * resultants in one batch (one pass over the GPU).  status (may be NULL)
 * receives 2n entries: the y-projections, then the x-projections.  Returns
 * the first failure, as rs_resultant_batch. */
int rs_projections(rs_ctx *ctx, int32_t n, const rs_bipoly *f, const rs_bipoly *g,
                   rs_upoly *out_y, rs_upoly *out_x, int32_t *status);

/* Square-free factorisation of R = R^{(y)} = res(f, g, y) (the paper's
 * solver computes R^{(y)} together with its square-free factorisation,
 * Section 5, PROJECT): R = c * prod_{i >= 1} R_i^i with c an integer and
 * every R_i in Z[x] primitive, square-free, pairwise coprime, with a
 * positive leading coefficient.  One GPU pass computes R over enough primes
 * for the factors' coefficient bound and Yun's algorithm mod every prime;
 * the factors are lifted by the Chinese remaindering kernels and made
 * primitive on the host.  content receives c (deg 0); factors[i - 1]
 * receives R_i for i = 1..max_mult (the constant 1 when R has no factor of
 * multiplicity i); *nmult the largest multiplicity present (0 when R is a
 * constant).  Outputs are written on RS_OK; on RS_ERR_CAPACITY the deg and
 * limbs of the outputs that did not fit give the room needed (a multiplicity
 * above max_mult also returns RS_ERR_CAPACITY).  R = 0 gives RS_ERR_ARG.
 * RS_ERR_LIMIT when one of the primes used divides a discriminant of R's
 * factors (the result would need other primes; not met in practice). */
int rs_squarefree_y(rs_ctx *ctx, const rs_bipoly *f, const rs_bipoly *g, int32_t max_mult,
                    rs_upoly *content, rs_upoly *factors, int32_t *nmult);

/* rs_squarefree_y for n pairs in one GPU pass: content[i], factors[i *
 * max_mult + m - 1] (m = 1..max_mult) and nmult[i] for pair i, as above.
 * status (may be NULL) receives each pair's code; the return value is the
 * first failure in pair order (its message in rs_last_error), RS_OK when
 * every pair succeeded.  A pair's outputs are written when its status is
 * RS_OK. */
int rs_squarefree_batch(rs_ctx *ctx, int32_t n, const rs_bipoly *f, const rs_bipoly *g, int32_t max_mult,
                        rs_upoly *content, rs_upoly *factors, int32_t *nmult, int32_t *status);

/* Square-free factorisations of both projections of each pair (the PROJECT
 * phase factors R^{(y)} and R^{(x)}, Section 5): for pair i, content_y[i],
 * factors_y[i * max_mult + m - 1], nmult_y[i] describe res(f_i, g_i, y) as in
 * rs_squarefree_y, and the _x outputs res(f_i, g_i, x) (coefficient k
 * belongs to y^k), all 2n factorisations in one GPU pass.  status (may be
 * NULL) receives 2n codes: the y-projections, then the x-projections.
 * Returns the first failure, as rs_squarefree_batch. */
int rs_squarefree_projections(rs_ctx *ctx, int32_t n, const rs_bipoly *f, const rs_bipoly *g, int32_t max_mult,
                              rs_upoly *content_y, rs_upoly *factors_y, int32_t *nmult_y, rs_upoly *content_x,
                              rs_upoly *factors_x, int32_t *nmult_x, int32_t *status);

/* Where the last rs_squarefree_y / rs_squarefree_batch call of this context
 * spent its time. */
typedef struct {
  rs_batch_info batch;  /* the GPU pass over the factors' primes (stage times, ms_yun) */
  int64_t yun_tasks;    /* (pair, prime) factorisations mod p */
  int64_t factors;      /* non-constant factors lifted */
  float ms_lift;        /* CRT of the factors on the device (the lifted H_i, then the scaled primitive parts) */
  float ms_host;        /* host work after the GPU pass: prime selection, contents, primitive parts */
  float ms_total;       /* wall time of the call */
  float ms_primitive;   /* of ms_host: the primitive parts of the lifted factors */
  int64_t h2d_bytes;    /* host-to-device bytes the call copied (inputs, CRT descriptors) */
  int64_t d2h_bytes;    /* device-to-host bytes the call copied (R's limbs, Yun headers, lifted factors) */
  float ms_analyse;     /* of ms_host: R unpacked, usable primes and factor degrees per pair */
  float ms_contents;    /* of ms_host: R's contents, lc(R) / prod_i lc(R_i)^i (gcd of R's coefficients
                           if that division is not exact) */
  float ms_fetch;       /* of ms_host: waiting for the lifted factors' limbs after the contents */
  int32_t factors_device; /* of factors: primitive parts taken on the device (the rest by host division) */
} rs_sqf_info;

int rs_squarefree_info_get(const rs_ctx *ctx, rs_sqf_info *info);

/* Diagnostics: the modular images z_i^{(p)} = res(f(x_i, y), g(x_i, y), y) mod p
 * (Section 4.1) that the resultant path computes, for the first nprimes
 * primes of the library's table and its first npoints evaluation points,
 * which come in pairs: x_{k,2t} = q_k^t and x_{k,2t+1} = -q_k^t mod p_k.
 * primes_out[nprimes] receives the primes, points_out[k * npoints + i] the
 * points (may be NULL) and images_out[k * npoints + i] the image for prime k
 * at x_{k,i} (0 <= z < p_k). */
int rs_images(rs_ctx *ctx, const rs_bipoly *f, const rs_bipoly *g, int32_t nprimes,
              int32_t npoints, uint32_t *primes_out, uint32_t *points_out,
              uint32_t *images_out);

/* ---------------------------------------------------------------------
 * Tuner of the image stage (G1: evaluation and univariate resultants,
 * Section 4.1).  Its launch has two free choices that change no result: the
 * points per block (the tile width: 32, 64 or 128) and the schedule (a
 * persistent grid that draws tiles from a cost-sorted list, or one block per
 * tile).  The best pair depends on the workload class: the register
 * capacity of the remainder sequence (the larger y-degree, rounded up to a
 * multiple of 8), floor(log2) of the class's largest point count D + 1 and
 * floor(log2) of its modular images K (D + 1), plus the GPU's SM count.
 * When a batch meets a class that the process-wide cache lacks (and
 * rs_config.autotune is 1), it first builds image-only batches of the
 * class's pairs (a stride sample of at most 2^22 images) for each of the six
 * candidates, times their G1 launches with CUDA events (median of three
 * after one warm-up) and caches the fastest; the built-in default is kept
 * unless another candidate is more than 2% faster.  The interpolation stage
 * (G2) has one more free choice per pair: direct convolutions,
 * number-theoretic transforms, or exact products on the tensor cores of
 * every pair of a prime at once (the last two for D + 1 <= 8192).  Pairs are
 * grouped by transform length 2^lg; for a group missing from the cache the
 * tuner times the whole path with each form (on the whole group up to 2^25
 * images, else on a stride sample) and keeps the fastest G2 (the
 * instruction-count model's choice between the first two unless another is
 * more than 2% faster).  The groups that chose the tensor cores share one
 * set of row tiles.  The server never tunes; it uses cached choices, so warm the
 * cache with rs_autotune first.
 * --------------------------------------------------------------------- */
enum { RS_TUNE_G1 = 0, RS_TUNE_G2 = 1 };

typedef struct {
  int32_t kind;                            /* RS_TUNE_G1: image-stage launch; RS_TUNE_G2:
                                              interpolation form */
  int32_t sms, cap, lg_points, lg_images;  /* the class; for RS_TUNE_G2 cap is 0 and lg_points
                                              is log2 of the transform length */
  int32_t choice, persistent;              /* RS_TUNE_G1: tile points and schedule;
                                              RS_TUNE_G2: 0 = direct, 1 = transforms, 2 = tensor
                                              cores (persistent 0) */
  float ms_best, ms_default;               /* stage time of the choice and of the default on the
                                              tuning sample (0 when loaded without timings) */
} rs_tune_entry;

/* Tune every class that these pairs form (as rs_batch_create would group
 * them) and is not cached yet; no result is computed. */
int rs_autotune(rs_ctx *ctx, int32_t n, const rs_bipoly *f, const rs_bipoly *g);
/* Copy up to cap_entries cached choices into out (may be NULL when
 * cap_entries is 0); *count receives the number cached.  Host only. */
int rs_autotune_entries(rs_tune_entry *out, int32_t cap_entries, int32_t *count);
/* Write the cache as text, one class per line:
 *   kind sms cap lg_points lg_images choice persistent ms_best ms_default
 * after a '#' header line.  Host only. */
int rs_autotune_save(const char *path);
/* Merge a file written by rs_autotune_save into the cache (its entries win).
 * A malformed line rejects the whole file with RS_ERR_ARG and merges
 * nothing.  Host only. */
int rs_autotune_load(const char *path);
/* Empty the cache.  Host only. */
int rs_autotune_clear(void);

/* Test hook (failure detection without a GPU fault): while `on` is non-zero
 * the copy warps of the tensor-core kernels (G2 products, CRT digits) of
 * this context issue no copies, so the MMA and read-out warps' bounded
 * mbarrier waits run out after about a second; each block then drains,
 * frees its tensor memory and sets the status word, and the run's results
 * fail with RS_ERR_TIMEOUT.  The context stays usable; turning the hook off
 * restores normal runs (captured graphs read the flag from device memory).
 * Never needed in normal use.  Synchronises the context's stream. */
int rs_test_stall_tensor_cores(rs_ctx *ctx, int32_t on);

/* ---------------------------------------------------------------------
 * Serving: a continuous-batching request server inside a context.
 * Each request is one resultant Res_y(f, g).  Submission plans the request
 * and copies its inputs (the caller may free them on return).  A scheduler
 * thread admits pending requests in arrival order while their device
 * footprint (the images K * (D+1) of numerators and denominators, the
 * output limbs (D+1) * Lout and the inputs) fits the memory budget, groups
 * them into a micro-batch and runs it on one of max_inflight CUDA streams;
 * micro-batches on different streams overlap on the GPU, and requests that
 * arrive while others run are admitted as soon as a stream and memory free
 * up.  Residues stay on the device until their micro-batch completes.
 * A request's result is the same whether it runs alone or in a mix.
 * The server functions may be called from several host threads; other
 * calls on the same context must not run concurrently with rs_server_stop.
 * --------------------------------------------------------------------- */
typedef struct {
  int64_t submitted, completed, failed;
  int64_t pending;                 /* waiting for admission */
  int64_t running;                 /* in micro-batches on the GPU now */
  int64_t inflight_batches;        /* micro-batches on the GPU now */
  int64_t batches;                 /* micro-batches launched so far */
  int64_t peak_inflight_batches;   /* most micro-batches on the GPU at once */
  int64_t peak_running;            /* most requests on the GPU at once */
  int64_t mem_used, mem_limit;     /* admitted device bytes / budget */
  int64_t kernel_launches;         /* kernels of the library launched so far */
} rs_server_stats;

/* Start the server (optional: the first submit starts it with defaults).
 * max_inflight: concurrent micro-batches (streams), 0 = 3; max_batch:
 * requests per micro-batch, 0 = 256; mem_limit_bytes: admission budget,
 * 0 = rs_config.mem_limit_bytes or half of the free device memory. */
int rs_server_start(rs_ctx *ctx, int32_t max_inflight, int32_t max_batch, int64_t mem_limit_bytes);
/* Queue Res_y(f, g); *ticket identifies the request.  Planning errors
 * (RS_ERR_ARG, RS_ERR_LIMIT) are returned here. */
int rs_server_submit(rs_ctx *ctx, const rs_bipoly *f, const rs_bipoly *g, uint64_t *ticket);
/* RS_PENDING while the request runs; otherwise its status, with the result
 * in *out on RS_OK (the ticket is then released; on RS_ERR_CAPACITY it is
 * kept and out->deg / out->limbs give the size needed).  latency_ms (may be
 * NULL) receives the time from submission to completion. */
int rs_server_poll(rs_ctx *ctx, uint64_t ticket, rs_upoly *out, double *latency_ms);
/* As rs_server_poll, but blocks up to timeout_us microseconds (< 0: no
 * limit); RS_ERR_TIMEOUT when the request is still running. */
int rs_server_wait(rs_ctx *ctx, uint64_t ticket, rs_upoly *out, double *latency_ms,
                   int64_t timeout_us);
int rs_server_stats_get(rs_ctx *ctx, rs_server_stats *stats);
/* Per-request log of the running server: from now on every finished request
 * appends one JSON line to the file at path (created or truncated) —
 * {"ticket", "status", "submit_us", "admit_us" (-1 if never admitted),
 * "done_us" (microseconds since the server started), "K" (primes), "D"
 * (degree bound), "footprint" (device bytes), "deg", "limbs"}.  NULL closes
 * the log; rs_server_stop closes it too.  RS_ERR_STATE without a server,
 * RS_ERR_ARG if the file cannot be opened. */
int rs_server_set_log(rs_ctx *ctx, const char *path);
/* Finish every admitted and pending request, then stop the scheduler
 * thread and release its streams (results not yet polled are dropped). */
int rs_server_stop(rs_ctx *ctx);

/* Throughput of the integer multiply-add forms the kernels use, measured on
 * the current CUDA device (a measurement facility; the paper has no
 * counterpart).  Each rate is operations per second over all SMs at the
 * clock the device runs at during the call: independent chains of
 * mad.lo.u32, mad.wide.u32 (64-bit accumulate), mad.hi.u32, mad.wide.s32,
 * and of the remainder sequence's Montgomery step x <- (x w1 + y w2) R^-1
 * mod p.  The mad.lo.u32 rate is the measured integer multiply-add peak.
 * Runs `launches` short kernels (about 20 ms in all) on the legacy default
 * stream and synchronises; allocates and frees a small device buffer.
 * Returns RS_OK, RS_ERR_ARG (out NULL), RS_ERR_NOMEM or RS_ERR_CUDA. */
typedef struct {
  double mad_lo_u32, mad_wide_u32, mad_hi_u32, mad_wide_s32, mont_update;
  double clock_max_mhz;  /* the device's maximum SM clock */
  int32_t sms;           /* streaming multiprocessors */
  int32_t launches;
} rs_int_peak;
int rs_measure_int_peak(rs_int_peak *out);

/* Chinese remaindering that allocates nothing, for callers that may not
 * allocate device memory (a plugin handed fixed buffers by its host
 * application, code that must not call cudaMalloc/cudaFree because they can
 * synchronise the device or fail under memory pressure, loops that forbid
 * allocation).  The paper has no counterpart: this is a library facility.
 *
 * residues: DEVICE pointer, residues[k * ncoeffs + j] = R_j mod p_k (each
 *   < p_k), p_k the k-th prime of the library's table (primes in
 *   (2^31 - 2^20, 2^31), descending; rs_images reports them).
 * out: DEVICE pointer, ncoeffs * limbs words; coefficient j is written as
 *   two's-complement limbs out[j * limbs + l], the representative of R_j in
 *   (-P/2, P/2), P = p_0 ... p_{nprimes-1}, truncated to `limbs` limbs.
 * stream: a cudaStream_t (NULL = the legacy default stream); the call only
 *   enqueues and returns, except on the first call on a device (below).
 * Working memory is a fixed file-scope device array of 2^21 words (8 MiB)
 * that every GPU which loads the library keeps until the process exits;
 * calls need nprimes * ncoeffs + ncoeffs * limbs <= 2^21 and
 * nprimes <= 2048, else RS_ERR_LIMIT without any device work.  Every word of
 * that array is written before it is read, so no clearing is needed.
 * The first call on each device (with that device current) sets up the
 * device's constant tables and looks up the array's device address; it
 * blocks until that is done, so make it before any stream capture.  All
 * calls on a device share the one array: calls whose kernels overlap on the
 * GPU (other streams, other host threads) race and must be serialised by the
 * caller.  No cudaMalloc, cudaFree or other allocating routine is called.
 * Cost: one thread per coefficient runs the whole O(nprimes^2) digit
 * recurrence and writes its limbs with a stride of `limbs` words, so at
 * nprimes near 2048 it is far slower than the resultant pipeline's CRT.
 * Returns RS_OK, RS_ERR_ARG, RS_ERR_LIMIT or RS_ERR_CUDA (rs_last_error is
 * not updated by this call).  RS_ERR_CUDA is returned only for a launch
 * error that appears during this call; a CUDA error already pending on the
 * calling thread from earlier work is left pending for its owner. */
int rs_crt_noalloc(const uint32_t *residues, int32_t nprimes, int32_t ncoeffs, int32_t limbs,
                   uint32_t *out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* RS_H */
