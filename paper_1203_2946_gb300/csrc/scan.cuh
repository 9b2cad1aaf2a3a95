// Exclusive prefix sums of int32 counts into an int32 pointer array
// (out[0] = 0, out[i+1] = mult * (counts[0] + ... + counts[i])), in int64 with
// an overflow flag: block-local scans, one block scanning the block totals,
// then a finishing pass.  Used for the padded StripPtr (mult 32: passes of 32
// items) and the row pointer of a row-permuted matrix (mult 1).
#pragma once
#include "common.cuh"

namespace cmrs {
namespace {

constexpr int kScanThreads = 1024;
constexpr uint32_t ST_SCAN_OVERFLOW = 1u;

// Block-local inclusive scan (int64) of counts, block totals into aux.
__global__ void __launch_bounds__(kScanThreads) k_scan_blocks(int n, const int32_t *__restrict__ in,
                                                               long long *__restrict__ incl,
                                                               long long *__restrict__ aux) {
  __shared__ long long wsum[kScanThreads / 32];
  const int i = blockIdx.x * kScanThreads + threadIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  long long v = i < n ? in[i] : 0;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) wsum[w] = v;
  __syncthreads();
  if (w == 0) {
    long long t = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long u = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += u;
    }
    wsum[lane] = t;
  }
  __syncthreads();
  if (w > 0) v += wsum[w - 1];
  if (i < n) incl[i] = v;
  if (threadIdx.x == kScanThreads - 1) aux[blockIdx.x] = v;
}

// Exclusive scan of the block totals, in place, by one block.
__global__ void __launch_bounds__(kScanThreads) k_scan_aux(int nb, long long *__restrict__ aux) {
  __shared__ long long wsum[kScanThreads / 32];
  __shared__ long long carry;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int b0 = 0; b0 < nb; b0 += kScanThreads) {
    const int i = b0 + threadIdx.x;
    const long long x = i < nb ? aux[i] : 0;
    long long v = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long t = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += t;
    }
    if (lane == 31) wsum[w] = v;
    __syncthreads();
    if (w == 0) {
      long long t = wsum[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const long long u = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += u;
      }
      wsum[lane] = t;
    }
    __syncthreads();
    if (w > 0) v += wsum[w - 1];
    const long long c = carry;
    if (i < nb) aux[i] = c + v - x;
    __syncthreads();
    if (threadIdx.x == kScanThreads - 1) carry = c + v;
    __syncthreads();
  }
}

__global__ void k_scan_finish(int n, const long long *__restrict__ incl, const long long *__restrict__ aux, int mult,
                              int32_t *__restrict__ out, uint32_t *status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) out[0] = 0;
  if (i >= n) return;
  const long long v = (long long)mult * (incl[i] + aux[i / kScanThreads]);
  if (v > 0x7fffffffLL) {
    atomicOr(status, ST_SCAN_OVERFLOW);
    out[i + 1] = 0x7fffffff;
  } else {
    out[i + 1] = (int32_t)v;
  }
}

// Workspace bytes for the scan of n counts: counts int32[n], incl int64[n], aux int64[blocks].
inline size_t scan_ws_bytes(int n) {
  const size_t m = (size_t)(n > 0 ? n : 1);
  return align256(m * 4) + align256(m * 8) + align256((size_t)ceil_div((long long)m, kScanThreads) * 8);
}

// Enqueues the scan of counts (already written at `ws`) into out[n + 1].
inline int scan_counts(int n, char *ws, int mult, int32_t *out, uint32_t *status, cudaStream_t st) {
  const size_t m = (size_t)(n > 0 ? n : 1);
  int32_t *counts = reinterpret_cast<int32_t *>(ws);
  long long *incl = reinterpret_cast<long long *>(ws + align256(m * 4));
  long long *aux = reinterpret_cast<long long *>(ws + align256(m * 4) + align256(m * 8));
  const int nb = (int)ceil_div(n, kScanThreads);
  k_scan_blocks<<<nb, kScanThreads, 0, st>>>(n, counts, incl, aux);
  CMRS_LAUNCH_CHECK();
  k_scan_aux<<<1, kScanThreads, 0, st>>>(nb, aux);
  CMRS_LAUNCH_CHECK();
  k_scan_finish<<<(int)ceil_div(n, 256), 256, 0, st>>>(n, incl, aux, mult, out, status);
  CMRS_LAUNCH_CHECK();
  return CMRS_OK;
}

}  // namespace
}  // namespace cmrs
