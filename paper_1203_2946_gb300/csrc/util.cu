// Host-side utilities of libcmrs: status strings, the packing-bits rule,
// storage-form sizes and a per-device multiprocessor count cache.
#include <mutex>

#include "common.cuh"

namespace cmrs {

static thread_local int g_last_cuda_error = 0;

int set_cuda_error(cudaError_t e) {
  if (e == cudaSuccess) return CMRS_OK;
  g_last_cuda_error = static_cast<int>(e);
  return CMRS_ERR_CUDA;
}

int sm_count() {
  static std::mutex mu;
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
  std::lock_guard<std::mutex> lk(mu);
  if (cache[dev] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
    cache[dev] = n;
  }
  return cache[dev];
}

}  // namespace cmrs

extern "C" const char *cmrs_error_string(int status) {
  switch (status) {
    case CMRS_OK: return "CMRS_OK";
    case CMRS_ERR_ARG: return "CMRS_ERR_ARG: invalid argument";
    case CMRS_ERR_HEIGHT: return "CMRS_ERR_HEIGHT: strip height must be in 1..32";
    case CMRS_ERR_COL_OVERFLOW: return "CMRS_ERR_COL_OVERFLOW: column index does not fit beside RowInStrip";
    case CMRS_ERR_CSR_INVALID: return "CMRS_ERR_CSR_INVALID: invalid CRS row pointer or column index";
    case CMRS_ERR_CUDA: return "CMRS_ERR_CUDA: a CUDA runtime call failed";
    case CMRS_ERR_UNSUPPORTED: return "CMRS_ERR_UNSUPPORTED: request not supported by this variant";
    case CMRS_ERR_WORKSPACE: return "CMRS_ERR_WORKSPACE: workspace missing, misaligned or too small";
    case CMRS_ERR_TIMEOUT: return "CMRS_ERR_TIMEOUT: a bounded device wait gave up";
    default: return "CMRS: unknown status";
  }
}

extern "C" int cmrs_last_cuda_error(void) { return cmrs::g_last_cuda_error; }

// Section 4 packs RowInStrip into CMRS_BITS = 4 low bits (heights <= 16);
// heights 17..32 take a fifth bit.
extern "C" int cmrs_bits_for_height(int height) {
  if (height < 1 || height > 32) return -1;
  int bits = 0;
  while ((1 << bits) < height) ++bits;
  return bits < 4 ? 4 : bits;
}

extern "C" int64_t cmrs_pad8(int64_t nnz) { return (nnz + 7) & ~int64_t(7); }

extern "C" int64_t cmrs_val_bytes(int64_t nnz, int dtype) {
  if (nnz < 0) return -1;
  switch (dtype) {
    case CMRS_F64: return nnz * 8;
    case CMRS_F32: return nnz * 4;
    case CMRS_BF16: return nnz * 2;
    case CMRS_BF16X2: return 2 * cmrs_pad8(nnz) + 2 * nnz;
    default: return -1;
  }
}
