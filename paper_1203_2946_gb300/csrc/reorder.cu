// Row reordering, the off-line optimisation the paper recommends for CMRS
// (Section 7; Section 6.3 reads a low eta_+ as the cue): rows of similar
// length placed in the same strip, so that the modified form of Section 6.6
// needs fewer zero items.  Order: inside each window of `window` consecutive
// rows, rows by length, longest first, equal lengths in their original
// order.  One CTA sorts one window's (length, index) keys in shared memory
// with a bitonic network.  The permuted CRS (row i = original row perm[i])
// is built by a length gather, a scan and a warp-per-row copy; the SpMV then
// writes y[perm[i]] (cmrs_spmv_rows), so y comes out in the original order.
#include <algorithm>

#include "common.cuh"
#include "scan.cuh"

namespace cmrs {
namespace {

constexpr int kOrderMax = 4096;
constexpr uint32_t ST_PERM_BAD = 2u;

__global__ void __launch_bounds__(1024) k_row_order(int rows, int window, int P, const int32_t *__restrict__ row_ptr,
                                                    int32_t *__restrict__ perm) {
  __shared__ unsigned long long key[kOrderMax];
  const long long w0 = (long long)blockIdx.x * window;
  const int n = (int)min((long long)window, rows - w0);
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    if (i < n) {
      const unsigned len = (unsigned)(row_ptr[w0 + i + 1] - row_ptr[w0 + i]);
      key[i] = ((unsigned long long)(0x7fffffffu - min(len, 0x7fffffffu)) << 32) | (unsigned)i;
    } else {
      key[i] = ~0ull;
    }
  }
  __syncthreads();
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const unsigned long long a = key[i], b = key[l];
          if ((a > b) == ((i & k) == 0)) {
            key[i] = b;
            key[l] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) perm[w0 + i] = (int32_t)(w0 + (long long)(key[i] & 0xffffffffull));
}

// Length of each permuted row; counts how often each original row is named.
// A row outside [0, rows) or a row whose pointers leave [0, nnz] is flagged
// and counted as empty, so nothing later reads outside the arrays.
__global__ void k_perm_lengths(int rows, int nnz, const int32_t *__restrict__ row_ptr,
                               const int32_t *__restrict__ perm, int32_t *__restrict__ counts,
                               int32_t *__restrict__ seen, uint32_t *status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows) return;
  const int r = perm[i];
  if (r < 0 || r >= rows) {
    atomicOr(status, ST_PERM_BAD);
    counts[i] = 0;
    return;
  }
  const int a = row_ptr[r], b = row_ptr[r + 1];
  if (a < 0 || b < a || b > nnz) {
    atomicOr(status, ST_PERM_BAD);
    counts[i] = 0;
  } else {
    counts[i] = b - a;
  }
  atomicAdd(&seen[r], 1);
}

__global__ void k_perm_check(int rows, const int32_t *__restrict__ seen, uint32_t *status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < rows && seen[i] != 1) atomicOr(status, ST_PERM_BAD);
}

template <typename V>
__global__ void k_perm_copy(int rows, const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col_ind,
                            const V *__restrict__ val, const int32_t *__restrict__ perm,
                            const int32_t *__restrict__ row_ptr_out, int32_t *__restrict__ col_out,
                            V *__restrict__ val_out) {
  const int lane = threadIdx.x & 31;
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long i = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < rows; i += nw) {
    const int r = perm[i];
    const int a = row_ptr[r], len = row_ptr[r + 1] - a, o = row_ptr_out[i];
    for (int j = lane; j < len; j += 32) {
      col_out[o + j] = col_ind[a + j];
      if (val) val_out[o + j] = val[a + j];
    }
  }
}

size_t perm_ws_bytes(int rows) { return 256 + align256((size_t)(rows > 0 ? rows : 1) * 4) + scan_ws_bytes(rows); }

}  // namespace
}  // namespace cmrs

using namespace cmrs;

extern "C" int cmrs_row_order(int rows, const int32_t *row_ptr, int window, int32_t *perm_out, void *stream) {
  CMRS_TRACE();
  if (rows < 0 || window < 1 || window > kOrderMax) return CMRS_ERR_ARG;
  if (rows == 0) return CMRS_OK;
  if (!row_ptr || !perm_out) return CMRS_ERR_ARG;
  int P = 1;
  while (P < window) P <<= 1;
  const int threads = std::min(1024, std::max(32, P));
  const long long blocks = ceil_div(rows, window);
  if (blocks > 0x7fffffffLL) return CMRS_ERR_ARG;
  k_row_order<<<(int)blocks, threads, 0, as_stream(stream)>>>(rows, window, P, row_ptr, perm_out);
  CMRS_LAUNCH_CHECK();
  return CMRS_OK;
}

extern "C" int cmrs_permute_csr_workspace(int rows, size_t *bytes) {
  if (!bytes || rows < 0) return CMRS_ERR_ARG;
  *bytes = perm_ws_bytes(rows);
  return CMRS_OK;
}

extern "C" int cmrs_permute_csr(int rows, int nnz, const int32_t *row_ptr, const int32_t *col_ind, const void *val,
                                int val_dtype, const int32_t *perm, int32_t *row_ptr_out, int32_t *col_ind_out,
                                void *val_out, void *workspace, size_t workspace_bytes, void *stream) {
  CMRS_TRACE();
  if (rows < 0 || nnz < 0) return CMRS_ERR_ARG;
  if (val && val_dtype != CMRS_F64 && val_dtype != CMRS_F32) return CMRS_ERR_ARG;
  if (!row_ptr || !row_ptr_out || (rows > 0 && !perm)) return CMRS_ERR_ARG;
  if (nnz > 0 && (!col_ind || !col_ind_out || (val && !val_out))) return CMRS_ERR_ARG;
  if (!workspace || workspace_bytes < perm_ws_bytes(rows) || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return CMRS_ERR_WORKSPACE;
  cudaStream_t st = as_stream(stream);
  char *ws = reinterpret_cast<char *>(workspace);
  uint32_t *status = reinterpret_cast<uint32_t *>(ws);
  int32_t *seen = reinterpret_cast<int32_t *>(ws + 256);
  char *scan = ws + 256 + align256((size_t)(rows > 0 ? rows : 1) * 4);
  int32_t *counts = reinterpret_cast<int32_t *>(scan);
  CMRS_CUDA_TRY(cudaMemsetAsync(status, 0, 4, st));
  if (rows == 0) {
    CMRS_CUDA_TRY(cudaMemsetAsync(row_ptr_out, 0, 4, st));
    return CMRS_OK;
  }
  CMRS_CUDA_TRY(cudaMemsetAsync(seen, 0, (size_t)rows * 4, st));
  const int blocks = (int)ceil_div(rows, 256);
  k_perm_lengths<<<blocks, 256, 0, st>>>(rows, nnz, row_ptr, perm, counts, seen, status);
  CMRS_LAUNCH_CHECK();
  k_perm_check<<<blocks, 256, 0, st>>>(rows, seen, status);
  CMRS_LAUNCH_CHECK();
  int rc = scan_counts(rows, scan, 1, row_ptr_out, status, st);
  if (rc) return rc;
  uint32_t host[2] = {0, 0};
  CMRS_CUDA_TRY(cudaMemcpyAsync(&host[0], status, 4, cudaMemcpyDeviceToHost, st));
  CMRS_CUDA_TRY(cudaMemcpyAsync(&host[1], row_ptr_out + rows, 4, cudaMemcpyDeviceToHost, st));
  CMRS_CUDA_TRY(cudaStreamSynchronize(st));
  if (host[0] & ST_PERM_BAD) return CMRS_ERR_ARG;           // not a permutation, or a bad row pointer
  if (host[0] & ST_SCAN_OVERFLOW || (int)host[1] != nnz) return CMRS_ERR_CSR_INVALID;  // RowPtr ends off nnz
  const int grid = (int)std::min<long long>(ceil_div(rows, 8), (long long)sm_count() * 16);
  if (!val || val_dtype == CMRS_F64)
    k_perm_copy<double><<<grid, 256, 0, st>>>(rows, row_ptr, col_ind, reinterpret_cast<const double *>(val), perm,
                                              row_ptr_out, col_ind_out, reinterpret_cast<double *>(val_out));
  else
    k_perm_copy<float><<<grid, 256, 0, st>>>(rows, row_ptr, col_ind, reinterpret_cast<const float *>(val), perm,
                                             row_ptr_out, col_ind_out, reinterpret_cast<float *>(val_out));
  CMRS_LAUNCH_CHECK();
  return CMRS_OK;
}
