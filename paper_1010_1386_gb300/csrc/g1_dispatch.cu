// Dispatch of G1 over the register capacities compiled (one translation unit
// of kernels_g1.cu per capacity, so they build in parallel).
#include "rs_internal.cuh"

#define RS_G1_CASES(X) X(8) X(16) X(24) X(32) X(40) X(48) X(56) X(64) X(72)

#define RS_DECL(c)                                                                       \
  cudaError_t rs_g1_launch_##c(int threads, int blocks, size_t smem, const G1Args &a,    \
                               cudaStream_t s);                                          \
  cudaError_t rs_g1_prepare_##c(int threads, size_t smem, int *mb);
RS_G1_CASES(RS_DECL)
#undef RS_DECL

int g1_supported_cap(int cap) {
  if (cap < 1) cap = 1;
  const int c = ((cap + 7) / 8) * 8;
  return c <= 72 ? c : 0;
}

cudaError_t launch_g1(int cap, int threads, int blocks, size_t smem, const G1Args &a,
                      cudaStream_t s) {
  switch (cap) {
#define RS_CASE(c) \
  case c:          \
    return rs_g1_launch_##c(threads, blocks, smem, a, s);
    RS_G1_CASES(RS_CASE)
#undef RS_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t g1_prepare(int cap, int threads, size_t smem, int *max_blocks_per_sm) {
  switch (cap) {
#define RS_CASE(c) \
  case c:          \
    return rs_g1_prepare_##c(threads, smem, max_blocks_per_sm);
    RS_G1_CASES(RS_CASE)
#undef RS_CASE
    default:
      return cudaErrorInvalidValue;
  }
}
