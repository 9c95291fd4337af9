// rs_measure_int_peak: throughput of the integer multiply-add forms the
// kernels are built from, measured on the current device.
//
// Each thread runs 8 independent dependency chains of one instruction form
// for a fixed number of iterations (operands come from memory, results are
// written back, so nothing folds away); the rate is the operation count over
// the CUDA-event time of the launch, best of several launches of a grid of
// 8 blocks of 256 threads per SM.  The forms:
//   mad.lo.u32     x <- x y + z              (32-bit result)
//   mad.wide.u32   s <- a b + s              (64-bit accumulate)
//   mad.hi.u32     x <- hi(x y) + z
//   mad.wide.s32   s <- a b + s (signed)     (the evaluation's accumulate)
//   update         x <- (x w1 + y w2) R^-1 mod p, Montgomery with R = 2^32
//                  (the remainder sequence's per-coefficient step)
// The result feeds the roofline of the bench: the mad.lo.u32 rate is the
// measured integer multiply-add peak.
#include <algorithm>

#include "../../include/rs.h"
#include "modarith.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kIters = 2048;
constexpr int kThreads = 256;

template <int KIND>
__global__ void __launch_bounds__(kThreads) probe_kernel(const uint32_t *in, uint32_t *out, uint32_t p) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t y = in[0] + (uint32_t)t, z = in[1] ^ (uint32_t)t;
  uint32_t x[kChains];
  uint64_t s[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    x[c] = in[2 + c] + (uint32_t)t;
    s[c] = (uint64_t)x[c] << 7;
  }
  if (KIND == 4) {  // Montgomery update: values below p
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] %= p;
  }
  const uint32_t pinv = neg_inv32(p);
  const uint32_t w1 = y % p, w2 = z % p;
  ModP m;
  m.p = p;
  m.pinv = pinv;
  for (int it = 0; it < kIters; ++it) {
    uint32_t prev[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) prev[c] = x[c];
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      if (KIND == 0) {
        asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x[c]) : "r"(y), "r"(z));
      } else if (KIND == 1) {
        asm volatile("{\n\t.reg .b32 lo, hi;\n\tmov.b64 {lo, hi}, %0;\n\tmad.wide.u32 %0, lo, %1, %0;\n\t}"
                     : "+l"(s[c]) : "r"(y));
      } else if (KIND == 2) {
        asm volatile("mad.hi.u32 %0, %0, %1, %2;" : "+r"(x[c]) : "r"(y), "r"(z));
      } else if (KIND == 3) {
        asm volatile("{\n\t.reg .b32 lo, hi;\n\tmov.b64 {lo, hi}, %0;\n\tmad.wide.s32 %0, lo, %1, %0;\n\t}"
                     : "+l"(s[c]) : "r"(y));
      } else {  // each step reads the previous step's values, as the remainder sequence does
        x[c] = mmul2(prev[c], w1, prev[(c + 1) % kChains], w2, m);
      }
    }
  }
  uint64_t acc = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc += (uint64_t)x[c] + s[c];
  out[t] = (uint32_t)acc ^ (uint32_t)(acc >> 32);
}

template <int KIND>
cudaError_t run_probe(int blocks, const uint32_t *in, uint32_t *out, uint32_t p, float *ms) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  float best = 1e30f;
  for (int r = 0; r < 4 && e == cudaSuccess; ++r) {  // the first launch warms up
    cudaEventRecord(e0);
    probe_kernel<KIND><<<blocks, kThreads>>>(in, out, p);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (r > 0) best = std::min(best, t);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = best;
  return e;
}

}  // namespace

extern "C" int rs_measure_int_peak(rs_int_peak *out) {
  if (!out) return RS_ERR_ARG;
  int dev = 0, sms = 0, khz = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) != cudaSuccess)
    return RS_ERR_CUDA;
  const int blocks = 8 * sms;
  const size_t nthreads = (size_t)blocks * kThreads;
  uint32_t *d = nullptr;
  if (cudaMalloc(&d, (nthreads + 16) * sizeof(uint32_t)) != cudaSuccess) return RS_ERR_NOMEM;
  const uint32_t seed[10] = {0x9e3779b9u, 0x7f4a7c15u, 3u, 5u, 7u, 11u, 13u, 17u, 19u, 23u};
  cudaError_t e = cudaMemcpy(d, seed, sizeof(seed), cudaMemcpyHostToDevice);
  uint32_t *o = d + 16;
  const uint32_t p = 2147483647u;  // the first table prime
  float ms[5] = {0, 0, 0, 0, 0};
  if (e == cudaSuccess) e = run_probe<0>(blocks, d, o, p, &ms[0]);
  if (e == cudaSuccess) e = run_probe<1>(blocks, d, o, p, &ms[1]);
  if (e == cudaSuccess) e = run_probe<2>(blocks, d, o, p, &ms[2]);
  if (e == cudaSuccess) e = run_probe<3>(blocks, d, o, p, &ms[3]);
  if (e == cudaSuccess) e = run_probe<4>(blocks, d, o, p, &ms[4]);
  cudaFree(d);
  if (e != cudaSuccess) return RS_ERR_CUDA;
  const double ops = (double)nthreads * kIters * kChains;
  out->mad_lo_u32 = ops / (ms[0] * 1e-3);
  out->mad_wide_u32 = ops / (ms[1] * 1e-3);
  out->mad_hi_u32 = ops / (ms[2] * 1e-3);
  out->mad_wide_s32 = ops / (ms[3] * 1e-3);
  out->mont_update = ops / (ms[4] * 1e-3);
  out->sms = sms;
  out->launches = 20;
  out->clock_max_mhz = khz / 1000.0;
  return RS_OK;
}
