// rs_crt_noalloc: Chinese remaindering of caller-owned device residues into
// caller-owned device limbs without allocating any memory.
//
// For callers that are not allowed to allocate device memory: code that runs
// inside a host application which owns every device allocation (a plugin
// given fixed buffers), paths that must not call cudaMalloc/cudaFree because
// those calls may synchronise the device or fail under memory pressure, and
// latency-critical loops that forbid allocation altogether.  Such a caller
// passes its own input and output buffers; the working memory this kernel
// needs lives in a fixed file-scope device array of this library instead.
//
// The kernel is a variant of the CRT stage of the resultant pipeline (mixed
// radix digits in the symmetric range, then two's-complement limbs), with its
// digits and its limb accumulator in that array instead of the pipeline's
// buffers, and its own per-prime constants in fixed device tables.
#include <algorithm>
#include <mutex>
#include <vector>

#include "../../include/rs.h"
#include "planner.h"
#include "rs_internal.cuh"

#define RS_NOALLOC_SCRATCH_WORDS (1u << 21)  // 8 MiB of scratch per GPU
#define RS_NOALLOC_MAX_PRIMES 2048
#define RS_NOALLOC_MAX_DEVICES 64

namespace {

// Working memory shared by every call on a device (kept until process exit).
static __device__ __align__(256) uint32_t g_noalloc_scratch[RS_NOALLOC_SCRATCH_WORDS];
static __device__ uint32_t g_noalloc_primes[RS_NOALLOC_MAX_PRIMES];
static __device__ ModP g_noalloc_mods[RS_NOALLOC_MAX_PRIMES];
static __device__ uint32_t g_noalloc_crt[RS_NOALLOC_MAX_PRIMES];

// Host-side set-up state: static storage only, nothing is allocated on the
// device.
struct NoallocDevice {
  bool ready;
  uint32_t *scratch;  // device address of g_noalloc_scratch on that device
  const ModP *mods;
  const uint32_t *crt;
};
static NoallocDevice g_dev[RS_NOALLOC_MAX_DEVICES];
static std::mutex g_mu;
static uint32_t h_primes[RS_NOALLOC_MAX_PRIMES];

__global__ void noalloc_init_kernel(int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const ModP m = make_modp(g_noalloc_primes[k]);
  g_noalloc_mods[k] = m;
  uint32_t acc = m.r1;
  for (int l = 0; l < k; ++l) acc = mmul(acc, to_mont(g_noalloc_primes[l] - m.p, m), m);
  g_noalloc_crt[k] = minv(acc, m);
}

// One thread per coefficient j: res[k N + j] = R_j mod p_k (plain, < p_k).
__global__ void crt_noalloc_kernel(const uint32_t *res, int K, int N, int L, uint32_t *out,
                                   uint32_t *scratch, const ModP *mods, const uint32_t *crt) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  uint32_t *dig = scratch + j;                   // digit k at dig[k N]
  uint32_t *xl = scratch + (size_t)K * N + j;    // limb l at xl[l N]
  for (int k = 0; k < K; ++k) {
    const ModP mk = mods[k];
    uint32_t t = 0u;
    if (k > 0) {
      const int32_t vp = (int32_t)dig[(size_t)(k - 1) * N];
      t = vp < 0 ? (uint32_t)(vp + (int32_t)mk.p) : (uint32_t)vp;
      for (int l = k - 2; l >= 0; --l) {
        const uint32_t ym = to_mont(mods[l].p - mk.p, mk);
        const int32_t vl = (int32_t)dig[(size_t)l * N];
        const uint32_t vr = vl < 0 ? (uint32_t)(vl + (int32_t)mk.p) : (uint32_t)vl;
        t = madd(mmul(t, ym, mk), vr, mk.p);
      }
    }
    const uint32_t v = mmul(msub(res[(size_t)k * N + j], t, mk.p), crt[k], mk);
    const int32_t vs = v > (mk.p - 1u) / 2u ? (int32_t)v - (int32_t)mk.p : (int32_t)v;
    dig[(size_t)k * N] = (uint32_t)vs;
  }
  int act = 1;
  xl[0] = dig[(size_t)(K - 1) * N];
  for (int k = K - 2; k >= 0; --k) {
    int need = (31 * (K - k) + 1 + 31) / 32 + 1;
    if (need > L) need = L;
    if (need > act) {
      const uint32_t ext = (xl[(size_t)(act - 1) * N] >> 31) ? 0xffffffffu : 0u;
      for (int l = act; l < need; ++l) xl[(size_t)l * N] = ext;
      act = need;
    }
    const uint64_t p = mods[k].p;
    const int32_t vk = (int32_t)dig[(size_t)k * N];
    const uint64_t ext = vk < 0 ? 0xffffffffull : 0ull;
    uint64_t c = (uint32_t)vk;
    for (int l = 0; l < act; ++l) {
      const uint64_t t = (uint64_t)xl[(size_t)l * N] * p + c + (l ? ext : 0ull);
      xl[(size_t)l * N] = (uint32_t)t;
      c = t >> 32;
    }
  }
  const uint32_t ext = (xl[(size_t)(act - 1) * N] >> 31) ? 0xffffffffu : 0u;
  uint32_t *o = out + (size_t)j * L;
  for (int l = 0; l < L; ++l) o[l] = l < act ? xl[(size_t)l * N] : ext;
}

// Once per device, with that device current: fill the constant tables and
// look up the device address of the scratch array.
int noalloc_setup(int dev) {
  std::lock_guard<std::mutex> lock(g_mu);
  NoallocDevice &d = g_dev[dev];
  if (d.ready) return RS_OK;
  if (h_primes[0] == 0) {  // the first primes of the library's own table (host memory only)
    const std::vector<uint32_t> t = rs_prime_table(RS_NOALLOC_MAX_PRIMES);
    if ((int)t.size() < RS_NOALLOC_MAX_PRIMES) return RS_ERR_LIMIT;
    std::copy(t.begin(), t.end(), h_primes);
  }
  if (cudaMemcpyToSymbol(g_noalloc_primes, h_primes, sizeof(h_primes)) != cudaSuccess)
    return RS_ERR_CUDA;
  noalloc_init_kernel<<<(RS_NOALLOC_MAX_PRIMES + 127) / 128, 128>>>(RS_NOALLOC_MAX_PRIMES);
  if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
    return RS_ERR_CUDA;
  void *p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return RS_ERR_CUDA;
  d.scratch = static_cast<uint32_t *>(p);
  if (cudaGetSymbolAddress(&p, g_noalloc_mods) != cudaSuccess) return RS_ERR_CUDA;
  d.mods = static_cast<const ModP *>(p);
  if (cudaGetSymbolAddress(&p, g_noalloc_crt) != cudaSuccess) return RS_ERR_CUDA;
  d.crt = static_cast<const uint32_t *>(p);
  d.ready = true;
  return RS_OK;
}

}  // namespace

extern "C" int rs_crt_noalloc(const uint32_t *residues, int32_t nprimes, int32_t ncoeffs,
                              int32_t limbs, uint32_t *out, void *stream) {
  if (!residues || !out || nprimes < 1 || ncoeffs < 1 || limbs < 1) return RS_ERR_ARG;
  if (nprimes > RS_NOALLOC_MAX_PRIMES) return RS_ERR_LIMIT;
  if ((uint64_t)ncoeffs * ((uint64_t)nprimes + (uint64_t)limbs) > RS_NOALLOC_SCRATCH_WORDS)
    return RS_ERR_LIMIT;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return RS_ERR_CUDA;
  if (dev < 0 || dev >= RS_NOALLOC_MAX_DEVICES) return RS_ERR_LIMIT;
  const int rc = noalloc_setup(dev);
  if (rc != RS_OK) return rc;
  const NoallocDevice &d = g_dev[dev];
  // An error left pending by earlier, unrelated work on this thread is not
  // this call's: only a launch error that appears here is consumed and
  // reported, so the caller can still read its own.
  const cudaError_t before = cudaPeekAtLastError();
  crt_noalloc_kernel<<<(ncoeffs + 127) / 128, 128, 0, (cudaStream_t)stream>>>(
      residues, nprimes, ncoeffs, limbs, out, d.scratch, d.mods, d.crt);
  const cudaError_t after = cudaPeekAtLastError();
  if (after != cudaSuccess && after != before) {
    (void)cudaGetLastError();
    return RS_ERR_CUDA;
  }
  return RS_OK;
}
