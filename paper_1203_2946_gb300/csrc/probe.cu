// Diagnostic: the cost floor of a product whose x reads are gathers.
//
// Section 6.3 reads a low eta_+ as the sign that x is fetched many times over;
// for a matrix with random columns that is the whole story, and the question
// is how far a kernel is from the rate at which this GPU can gather at all.
// k_gather_dot streams a CRS column array and its FP32 values once, in order,
// with the streaming cache hints of the SpMV kernels, gathers x at every
// column and sums the products -- an SpMV with the row structure taken away
// (no row bounds, no per-row sums, no y).  Its time on a matrix's own column
// array is the floor a row-aware kernel is judged against.
#include <algorithm>

#include "common.cuh"

namespace cmrs {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeU = 8;  // entries in flight per thread

__global__ void __launch_bounds__(kProbeThreads) k_gather_dot(long long nnz, uint32_t cols,
                                                              const int32_t *__restrict__ col,
                                                              const float *__restrict__ val,
                                                              const float *__restrict__ x, float *out) {
  const uint64_t pol = policy_evict_first();
  const long long stride = (long long)gridDim.x * kProbeThreads * kProbeU;
  float s = 0.f;
  for (long long k0 = (long long)blockIdx.x * kProbeThreads * kProbeU + threadIdx.x; k0 < nnz; k0 += stride) {
    uint32_t c[kProbeU];
    float v[kProbeU], xv[kProbeU];
#pragma unroll
    for (int u = 0; u < kProbeU; ++u) {
      const long long k = k0 + (long long)u * kProbeThreads;
      c[u] = k < nnz ? ld_stream(reinterpret_cast<const uint32_t *>(col) + k, pol) : 0u;
      v[u] = k < nnz ? (val ? ld_stream(val + k, pol) : 1.f) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < kProbeU; ++u) xv[u] = ld_x(x + min(c[u], cols - 1));  // stays inside x
#pragma unroll
    for (int u = 0; u < kProbeU; ++u) s = fmaf(v[u], xv[u], s);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

}  // namespace
}  // namespace cmrs

using namespace cmrs;

extern "C" int cmrs_gather_probe(int nnz, int cols, const int32_t *col, const float *val, const float *x, float *out,
                                 void *stream) {
  CMRS_TRACE();
  if (nnz < 0 || cols < 0 || !out || (nnz > 0 && (!col || !x || cols == 0))) return CMRS_ERR_ARG;
  cudaStream_t st = as_stream(stream);
  CMRS_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(float), st));
  if (nnz == 0) return CMRS_OK;
  int per_sm = 0;
  CMRS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gather_dot, kProbeThreads, 0));
  const long long need = ceil_div(nnz, (long long)kProbeThreads * kProbeU);
  const int grid = (int)std::min<long long>(need, (long long)std::max(per_sm, 1) * sm_count());
  k_gather_dot<<<grid, kProbeThreads, 0, st>>>(nnz, (uint32_t)cols, col, val, x, out);
  CMRS_LAUNCH_CHECK();
  return CMRS_OK;
}
