// Shared device helpers of libcmrs (sm_103a): inline-PTX wrappers for the
// Blackwell bulk-copy engine (cp.async.bulk + mbarrier), cache-hinted loads,
// the storage-form decoders and host-side error plumbing.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "../../include/cmrs.h"

namespace cmrs {

// ------------------------------------------------------------------ host side
int set_cuda_error(cudaError_t e);  // records e, returns CMRS_ERR_CUDA (or OK)

// An NVTX range named after the entry point, open on the calling thread while
// the entry point runs (it spans the host work and the launches, not the
// kernels' device time).  Profilers select kernels by it, for example
// `ncu --nvtx --nvtx-include "cmrs_spmv/"`.  With no tool attached a push or a
// pop is one call to an empty stub.
struct TraceRange {
  explicit TraceRange(const char *name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange &) = delete;
  TraceRange &operator=(const TraceRange &) = delete;
};
#define CMRS_TRACE() ::cmrs::TraceRange cmrs_trace_range_(__func__)

#define CMRS_CUDA_TRY(expr)                                  \
  do {                                                       \
    cudaError_t _e = (expr);                                 \
    if (_e != cudaSuccess) return ::cmrs::set_cuda_error(_e); \
  } while (0)

#define CMRS_LAUNCH_CHECK() CMRS_CUDA_TRY(cudaGetLastError())

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

int sm_count();  // multiprocessors of the current device (cached per device)
// bytes of workspace the MERGE mapping needs for nnz entries of value form dtype
size_t merge_workspace_bytes(int nnz, int dtype);

// Programmatic dependent launch: `kernel` may begin while the kernel before
// it in the stream is still running, once every block of that kernel has
// executed pdl_launch_dependents() (or exited).  The kernel launched this way
// must call pdl_wait() before it touches anything the earlier kernel writes;
// what it does before (issuing copies of read-only inputs, say) overlaps the
// earlier kernel's tail and the launch gap.
template <typename... KArgs, typename... Args>
int launch_pdl(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t st,
               Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return set_cuda_error(cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...));
}

// Status word bits written by kernels (device side) and read by the host.
enum : uint32_t {
  ST_BAD_ROWPTR = 1u,
  ST_BAD_COL = 2u,
  ST_BAD_RIS = 4u,
  ST_TIMEOUT = 8u,
  ST_BAD_PAD = 16u,  // a padded strip not made of whole 32-item passes
};

// ------------------------------------------------------------------ device side
// The two halves of a programmatic dependent launch (see launch_pdl).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" :::); }

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// L2 policy for data read exactly once (the nonzero streams): evict first, so
// that x and y keep their lines.
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Arrive (count 1) and add `bytes` to the transaction count of this phase.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait on an mbarrier phase.  Each try_wait blocks for a bounded,
// implementation-defined time (a failed try took 3.8 us on a GB300, measured
// with cmrs_wait_probe); after `limit` failed tries the wait gives up and
// returns false so the caller can record a timeout and leave.  The default,
// 2^18 tries, gives up after about one second; the waits it bounds are for
// one bulk copy of a few KB or one stage's FMAs, microseconds each.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint32_t limit = (1u << 18)) {
  for (uint32_t i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// One bulk copy global -> shared (Blackwell/Hopper bulk-copy engine), its
// completion counted in bytes on `bar`.  src, dst and bytes must be multiples
// of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar,
                                         uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}

// Streaming loads for data touched once: skip L1, evict-first in L2.
__device__ __forceinline__ uint32_t ld_stream(const uint32_t *p, uint64_t pol) {
  uint32_t v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ double ld_stream(const double *p, uint64_t pol) {
  double v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ float ld_stream(const float *p, uint64_t pol) {
  float v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ uint16_t ld_stream(const uint16_t *p, uint64_t pol) {
  uint16_t v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.u16 %0, [%1], %2;" : "=h"(v) : "l"(p), "l"(pol));
  return v;
}

// The input vector: read-only path, kept in L1/L2.
template <typename T>
__device__ __forceinline__ T ld_x(const T *p) {
  return __ldg(p);
}

__device__ __forceinline__ float bf16_bits_to_float(uint16_t h) { return __uint_as_float(uint32_t(h) << 16); }

// ------------------------------------------------------------------ storage forms
// Traits per storage form: element type in memory, x/y/accumulator type, and
// how a stored entry becomes an accumulator-typed value.
template <int DT>
struct Form;

template <>
struct Form<CMRS_F64> {
  typedef double Stored;
  typedef double Acc;
  static constexpr int kBytes = 8;
  __device__ __forceinline__ static Acc value(const Stored *v, const Stored *, int64_t k) { return v[k]; }
};
template <>
struct Form<CMRS_F32> {
  typedef float Stored;
  typedef float Acc;
  static constexpr int kBytes = 4;
  __device__ __forceinline__ static Acc value(const Stored *v, const Stored *, int64_t k) { return v[k]; }
};
template <>
struct Form<CMRS_BF16> {
  typedef uint16_t Stored;
  typedef float Acc;
  static constexpr int kBytes = 2;
  __device__ __forceinline__ static Acc value(const Stored *v, const Stored *, int64_t k) {
    return bf16_bits_to_float(v[k]);
  }
};
// Split pair: hi + lo is exact in FP32 (hi has 8 significant bits, lo starts
// at least 8 binades lower with 8 more), so the recombination costs one add.
template <>
struct Form<CMRS_BF16X2> {
  typedef uint16_t Stored;
  typedef float Acc;
  static constexpr int kBytes = 4;
  __device__ __forceinline__ static Acc value(const Stored *hi, const Stored *lo, int64_t k) {
    return bf16_bits_to_float(hi[k]) + bf16_bits_to_float(lo[k]);
  }
};

__device__ __forceinline__ double fma_acc(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_acc(float a, float b, float c) { return fmaf(a, b, c); }

}  // namespace cmrs
