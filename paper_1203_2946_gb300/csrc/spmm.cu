// Multi-right-hand-side SpMM Y = A X on CMRS matrices, for one matrix or a
// batch of uneven matrices in one persistent launch replayed from a CUDA
// graph.  Not in the paper; it applies the strip layout of Section 3 to k
// right-hand sides at once, so that each gathered row of X (k contiguous
// values) is shared by k accumulators.
//
// Thread mapping: a group of G lanes owns one row.  When k is a multiple of 4
// and X, Y are 16-byte aligned, lane g accumulates the four columns
// 4 (c0 + g) .. 4 (c0 + g) + 3 from one 16-byte gather of X (G =
// min(32, next_pow2(k / 4))): a k = 32 row takes 8 lanes and a warp works
// four rows at once.  Otherwise lane g accumulates column c0 + g (G =
// min(32, next_pow2(k))).  Columns beyond the group are done in further
// passes over the row; each column's sum is one FMA chain in entry order
// either way.  Row bounds inside a strip come from binary
// searches on RowInStrip (unsorted strips).  A warp takes 32 / G rows at a
// time.  Work units (matrix, row range) are fetched by warps from a device
// queue (one atomic per unit), which balances uneven matrices.
#include <algorithm>
#include <chrono>
#include <mutex>
#include <new>
#include <vector>

#include "common.cuh"

namespace cmrs {
namespace {

constexpr int kSpmmThreads = 256;
constexpr int kSpmmCH = 2;  // entries whose gathers are in flight together (8 raised registers to 64 and was slower)
#ifndef CMRS_SPMM_CH4
#define CMRS_SPMM_CH4 2  // 16-byte gathers in flight per lane (measured 6.45 ms per batch; 1: 6.72, 3: 7.06, 4: 7.07, 8: 7.73)
#endif
constexpr int kSpmmCH4 = CMRS_SPMM_CH4;  // the same for the 16-byte gathers
#ifndef CMRS_SPMM_MINB
#define CMRS_SPMM_MINB 5  // resident CTAs per SM asked of the register allocator (48 registers)
#endif
#ifndef CMRS_SPMM_PREFETCH
#define CMRS_SPMM_PREFETCH 1  // next batch's column words loaded during this batch's gathers
#endif

struct Desc {
  int32_t rows, height, bits, k, vec, pad;
  const int32_t *sp;
  const uint32_t *packed;
  const float *val;
  const float *X;
  float *Y;
};

struct Unit {
  int32_t mat, row0, row1, pad;
};

struct QueueHead {
  unsigned int next;
  unsigned int pad[63];
};

__device__ __forceinline__ int lb_ris_g(const uint32_t *__restrict__ cp, int lo, int hi, uint32_t r, uint32_t mask) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if ((__ldg(cp + mid) & mask) < r) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Lanes that share one row: 16-byte columns when d.vec, else single ones.
__host__ __device__ __forceinline__ int spmm_lanes(int k, int vec) {
  const int c = vec ? k / 4 : k;
  int G = 1;
  while (G < c && G < 32) G <<= 1;
  return G;
}

// Row bounds inside the strip (binary searches on RowInStrip).
__device__ __forceinline__ void spmm_bounds(const Desc &d, int row, int &k0, int &k1) {
  const uint32_t mask = (1u << d.bits) - 1;
  const int s = row / d.height;
  const uint32_t r = (uint32_t)(row - s * d.height);
  const int sa = __ldg(d.sp + s), sb = __ldg(d.sp + s + 1);
  k0 = sa;
  k1 = sb;
  if (d.height > 1) {
    k0 = lb_ris_g(d.packed, sa, sb, r, mask);
    k1 = lb_ris_g(d.packed, k0, sb, r + 1, mask);
  }
}

// Rows [row0, row1) of matrix d, four columns per lane (d.vec).
__device__ __forceinline__ void spmm_rows4(const Desc &d, int row0, int row1, int lane) {
  const int kv = d.k >> 2;
  const int G = spmm_lanes(d.k, 1);
  const int per = 32 / G;
  const int g = lane & (G - 1);
  const int sub = lane / G;
  const float4 *X4 = reinterpret_cast<const float4 *>(d.X);
  float4 *Y4 = reinterpret_cast<float4 *>(d.Y);
  for (int rb = row0; rb < row1; rb += per) {
    const int row = rb + sub;
    const bool active = row < row1;
    int k0 = 0, k1 = 0;
    if (active) spmm_bounds(d, row, k0, k1);
    for (int c0 = 0; c0 < kv; c0 += G) {
      const int col = c0 + g;
      if (active && col < kv) {
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        // The column words and values of the next batch are loaded while this
        // batch's X gathers are in flight: a gather waits for its column word,
        // so without this every batch pays two memory round trips in a row.
        uint32_t pn[kSpmmCH4];
        float vn[kSpmmCH4];
#pragma unroll
        for (int u = 0; u < kSpmmCH4; ++u)
          if (k0 + u < k1) {
            pn[u] = __ldg(d.packed + k0 + u);
            vn[u] = __ldg(d.val + k0 + u);
          }
        for (int j = k0; j < k1; j += kSpmmCH4) {
          float4 xv[kSpmmCH4];
          float vv[kSpmmCH4];
#pragma unroll
          for (int u = 0; u < kSpmmCH4; ++u) {
            vv[u] = vn[u];
            if (j + u < k1) xv[u] = __ldg(X4 + (size_t)(pn[u] >> d.bits) * kv + col);
          }
          if (CMRS_SPMM_PREFETCH) {
#pragma unroll
            for (int u = 0; u < kSpmmCH4; ++u)
              if (j + kSpmmCH4 + u < k1) {
                pn[u] = __ldg(d.packed + j + kSpmmCH4 + u);
                vn[u] = __ldg(d.val + j + kSpmmCH4 + u);
              }
          }
#pragma unroll
          for (int u = 0; u < kSpmmCH4; ++u)
            if (j + u < k1) {
              acc.x = fmaf(vv[u], xv[u].x, acc.x);
              acc.y = fmaf(vv[u], xv[u].y, acc.y);
              acc.z = fmaf(vv[u], xv[u].z, acc.z);
              acc.w = fmaf(vv[u], xv[u].w, acc.w);
            }
          if (!CMRS_SPMM_PREFETCH) {
#pragma unroll
            for (int u = 0; u < kSpmmCH4; ++u)
              if (j + kSpmmCH4 + u < k1) {
                pn[u] = __ldg(d.packed + j + kSpmmCH4 + u);
                vn[u] = __ldg(d.val + j + kSpmmCH4 + u);
              }
          }
        }
        Y4[(size_t)row * kv + col] = acc;
      }
    }
  }
}

// Rows [row0, row1) of matrix d, processed by one warp.
__device__ __forceinline__ void spmm_rows(const Desc &d, int row0, int row1, int lane) {
  if (d.vec) {
    spmm_rows4(d, row0, row1, lane);
    return;
  }
  const int k = d.k;
  const int G = spmm_lanes(k, 0);
  const int per = 32 / G;
  const int g = lane & (G - 1);
  const int sub = lane / G;
  const uint32_t mask = (1u << d.bits) - 1;
  for (int rb = row0; rb < row1; rb += per) {
    const int row = rb + sub;
    const bool active = row < row1;
    int k0 = 0, k1 = 0;
    if (active) {
      const int s = row / d.height;
      const uint32_t r = (uint32_t)(row - s * d.height);
      const int sa = __ldg(d.sp + s), sb = __ldg(d.sp + s + 1);
      k0 = sa;
      k1 = sb;
      if (d.height > 1) {
        k0 = lb_ris_g(d.packed, sa, sb, r, mask);
        k1 = lb_ris_g(d.packed, k0, sb, r + 1, mask);
      }
    }
    for (int c0 = 0; c0 < k; c0 += G) {
      const int col = c0 + g;
      if (active && col < k) {
        // kSpmmCH entries per batch: their column words, values and X gathers
        // are all issued before the FMAs that use them
        float acc = 0.f;
        for (int j = k0; j < k1; j += kSpmmCH) {
          float xv[kSpmmCH], vv[kSpmmCH];
#pragma unroll
          for (int u = 0; u < kSpmmCH; ++u) {
            if (j + u < k1) {
              const uint32_t p = __ldg(d.packed + j + u);
              vv[u] = __ldg(d.val + j + u);
              xv[u] = __ldg(d.X + (size_t)(p >> d.bits) * k + col);
            }
          }
#pragma unroll
          for (int u = 0; u < kSpmmCH; ++u)
            if (j + u < k1) acc = fmaf(vv[u], xv[u], acc);
        }
        d.Y[(size_t)row * k + col] = acc;
      }
    }
  }
}

__global__ void __launch_bounds__(kSpmmThreads, CMRS_SPMM_MINB) k_spmm_queue(const Desc *__restrict__ descs,
                                                             const Unit *__restrict__ units, int nunits,
                                                             QueueHead *q) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    unsigned int u = 0;
    if (lane == 0) u = atomicAdd(&q->next, 1u);
    u = __shfl_sync(0xffffffffu, u, 0);
    if (u >= (unsigned)nunits) break;
    const Unit un = units[u];
    const Desc d = descs[un.mat];
    spmm_rows(d, un.row0, un.row1, lane);
  }
}

// One matrix, no queue: warp w takes rows [w*rpw, (w+1)*rpw).
__global__ void __launch_bounds__(kSpmmThreads, CMRS_SPMM_MINB) k_spmm_one(Desc d, int rows_per_warp) {
  const int lane = threadIdx.x & 31;
  const long long w = ((long long)blockIdx.x * kSpmmThreads + threadIdx.x) >> 5;
  const long long r0 = w * rows_per_warp;
  if (r0 >= d.rows) return;
  const int r1 = (int)std::min<long long>(r0 + rows_per_warp, d.rows);
  spmm_rows(d, (int)r0, r1, lane);
}

int check_item(const cmrs_matrix *A, int k, const float *X, float *Y) {
  if (!A || k < 1) return CMRS_ERR_ARG;
  if (A->dtype != CMRS_F32) return CMRS_ERR_UNSUPPORTED;
  if (A->flags & (CMRS_SORTED | CMRS_PADDED)) return CMRS_ERR_UNSUPPORTED;
  if (cmrs_bits_for_height(A->height) != A->bits) return CMRS_ERR_HEIGHT;
  if (A->rows < 0 || A->nnz < 0 || A->strips != ceil_div(A->rows, A->height)) return CMRS_ERR_ARG;
  if (A->rows > 0 && (!A->strip_ptr || !Y)) return CMRS_ERR_ARG;
  if (A->nnz > 0 && (!A->col_packed || !A->val || !X)) return CMRS_ERR_ARG;
  return CMRS_OK;
}

Desc make_desc(const cmrs_matrix *A, int k, const float *X, float *Y) {
  Desc d;
  d.rows = A->rows;
  d.height = A->height;
  d.bits = A->bits;
  d.k = k;
  d.sp = A->strip_ptr;
  d.packed = A->col_packed;
  d.val = reinterpret_cast<const float *>(A->val);
  d.X = X;
  d.Y = Y;
  d.vec = (k % 4 == 0) && !((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(Y)) & 15);
  d.pad = 0;
  return d;
}

int rows_per_unit(const cmrs_matrix *A, int k, int vec, int work_target) {
  // work of a row ~ (nnz/rows) * k entry-columns; keep units near work_target
  const double mu = A->rows > 0 ? (double)A->nnz / A->rows : 1.0;
  const int per = 32 / spmm_lanes(k, vec);
  double r = work_target / std::max(1.0, mu * k);
  int ri = (int)std::max<double>(per, std::min<double>(r, 1 << 20));
  ri = (ri + per - 1) / per * per;
  return ri;
}

}  // namespace
}  // namespace cmrs

using namespace cmrs;

// Plan: host-side object holding the schedule layout and the captured graph.
struct cmrs_spmm_plan {
  int batch = 0, nunits = 0, work_target = 0;
  Desc *d_desc = nullptr;
  Unit *d_units = nullptr;
  QueueHead *d_q = nullptr;
  int grid = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

extern "C" int cmrs_spmm(const cmrs_matrix *A, int k, const float *X, float *Y, void *stream) {
  CMRS_TRACE();
  int rc = check_item(A, k, X, Y);
  if (rc) return rc;
  if (A->rows == 0) return CMRS_OK;
  cudaStream_t st = as_stream(stream);
  if (A->nnz == 0) {
    CMRS_CUDA_TRY(cudaMemsetAsync(Y, 0, (size_t)A->rows * k * sizeof(float), st));
    return CMRS_OK;
  }
  const Desc d = make_desc(A, k, X, Y);
  const int rpw = 32 / spmm_lanes(k, d.vec);
  const long long warps = ceil_div(A->rows, rpw);
  const int grid = (int)ceil_div(warps * 32, kSpmmThreads);
  k_spmm_one<<<grid, kSpmmThreads, 0, st>>>(d, rpw);
  CMRS_LAUNCH_CHECK();
  return CMRS_OK;
}

static int build_units(int batch, const cmrs_matrix *const *A, const int32_t *k, int work_target,
                       std::vector<Unit> &units) {
  units.clear();
  for (int b = 0; b < batch; ++b) {
    const int rpu = rows_per_unit(A[b], k[b], k[b] % 4 == 0, work_target);
    for (int r0 = 0; r0 < A[b]->rows; r0 += rpu) {
      Unit u;
      u.mat = b;
      u.row0 = r0;
      u.row1 = std::min(A[b]->rows, r0 + rpu);
      u.pad = 0;
      units.push_back(u);
    }
  }
  // heaviest units first, so the queue ends on small ones
  std::stable_sort(units.begin(), units.end(), [&](const Unit &x, const Unit &y) {
    auto w = [&](const Unit &u) {
      const cmrs_matrix *m = A[u.mat];
      const double mu = m->rows ? (double)m->nnz / m->rows : 0.0;
      return (double)(u.row1 - u.row0) * mu * k[u.mat];
    };
    return w(x) > w(y);
  });
  return CMRS_OK;
}

extern "C" int cmrs_spmm_plan_workspace(int batch, const cmrs_matrix *const *A, const int32_t *k, int work_target,
                                        size_t *bytes) {
  if (batch < 0 || !bytes || (batch > 0 && (!A || !k)) || work_target < 1) return CMRS_ERR_ARG;
  std::vector<Unit> units;
  for (int b = 0; b < batch; ++b)
    if (!A[b] || k[b] < 1) return CMRS_ERR_ARG;
  build_units(batch, A, k, work_target, units);
  *bytes = align256(sizeof(QueueHead)) + align256(sizeof(Desc) * (size_t)std::max(1, batch)) +
           align256(sizeof(Unit) * std::max<size_t>(1, units.size()));
  return CMRS_OK;
}

extern "C" int cmrs_spmm_plan_create(int batch, const cmrs_matrix *const *A, const int32_t *k, const float *const *X,
                                     float *const *Y, int work_target, int use_graph, void *workspace,
                                     size_t workspace_bytes, void *stream, cmrs_spmm_plan **out) {
  CMRS_TRACE();
  if (!out) return CMRS_ERR_ARG;
  *out = nullptr;
  if (batch < 1 || !A || !k || !X || !Y || work_target < 1) return CMRS_ERR_ARG;
  for (int b = 0; b < batch; ++b) {
    int rc = check_item(A[b], k[b], X[b], Y[b]);
    if (rc) return rc;
  }
  size_t need = 0;
  int rc = cmrs_spmm_plan_workspace(batch, A, k, work_target, &need);
  if (rc) return rc;
  if (!workspace || workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255)) return CMRS_ERR_WORKSPACE;
  std::vector<Unit> units;
  build_units(batch, A, k, work_target, units);
  std::vector<Desc> descs(batch);
  for (int b = 0; b < batch; ++b) descs[b] = make_desc(A[b], k[b], X[b], Y[b]);
  cmrs_spmm_plan *p = new (std::nothrow) cmrs_spmm_plan();
  if (!p) return CMRS_ERR_ARG;
  char *ws = reinterpret_cast<char *>(workspace);
  p->batch = batch;
  p->nunits = (int)units.size();
  p->work_target = work_target;
  p->d_q = reinterpret_cast<QueueHead *>(ws);
  p->d_desc = reinterpret_cast<Desc *>(ws + align256(sizeof(QueueHead)));
  p->d_units = reinterpret_cast<Unit *>(ws + align256(sizeof(QueueHead)) + align256(sizeof(Desc) * batch));
  cudaStream_t st = as_stream(stream);
  // Host -> device copies of the schedule; synchronised here because the host
  // vectors go out of scope (plan creation is not on the hot path).
  cudaError_t e = cudaMemcpyAsync(p->d_desc, descs.data(), sizeof(Desc) * batch, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !units.empty())
    e = cudaMemcpyAsync(p->d_units, units.data(), sizeof(Unit) * units.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    delete p;
    return set_cuda_error(e);
  }
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spmm_queue, kSpmmThreads, 0);
  p->grid = std::max(1, per_sm) * sm_count();
  if (use_graph) {
    // the graph holds the queue reset and the persistent launch; replaying it
    // costs one graph launch per batch
    cudaStream_t cap = nullptr;
    e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaMemsetAsync(p->d_q, 0, sizeof(unsigned int), cap);
      k_spmm_queue<<<p->grid, kSpmmThreads, 0, cap>>>(p->d_desc, p->d_units, p->nunits, p->d_q);
      e = cudaStreamEndCapture(cap, &p->graph);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, p->graph, 0);
    if (cap) cudaStreamDestroy(cap);
    if (e != cudaSuccess) {
      if (p->exec) cudaGraphExecDestroy(p->exec);
      if (p->graph) cudaGraphDestroy(p->graph);
      delete p;
      return set_cuda_error(e);
    }
  }
  *out = p;
  return CMRS_OK;
}

extern "C" int cmrs_spmm_batched(cmrs_spmm_plan *p, void *stream) {
  CMRS_TRACE();
  if (!p) return CMRS_ERR_ARG;
  cudaStream_t st = as_stream(stream);
  if (p->exec) {
    CMRS_CUDA_TRY(cudaGraphLaunch(p->exec, st));
  } else {
    CMRS_CUDA_TRY(cudaMemsetAsync(p->d_q, 0, sizeof(unsigned int), st));
    k_spmm_queue<<<p->grid, kSpmmThreads, 0, st>>>(p->d_desc, p->d_units, p->nunits, p->d_q);
    CMRS_LAUNCH_CHECK();
  }
  return CMRS_OK;
}

extern "C" int cmrs_spmm_plan_info(const cmrs_spmm_plan *p, int *nunits, int *grid, int *work_target) {
  if (!p) return CMRS_ERR_ARG;
  if (nunits) *nunits = p->nunits;
  if (grid) *grid = p->grid;
  if (work_target) *work_target = p->work_target;
  return CMRS_OK;
}

extern "C" int cmrs_spmm_plan_destroy(cmrs_spmm_plan *p) {
  if (!p) return CMRS_OK;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  delete p;
  return CMRS_OK;
}

// Autotuner for the batch schedule: builds a plan per candidate unit size,
// times `reps` graph replays of each with CUDA events and keeps the fastest.
extern "C" int cmrs_spmm_autotune(int batch, const cmrs_matrix *const *A, const int32_t *k, const float *const *X,
                                  float *const *Y, const int *candidates, int ncand, int reps, void *workspace,
                                  size_t workspace_bytes, void *stream, int *best_target, float *best_ms) {
  CMRS_TRACE();
  if (!candidates || ncand < 1 || reps < 1 || !best_target) return CMRS_ERR_ARG;
  cudaStream_t st = as_stream(stream);
  cudaEvent_t e0, e1;
  CMRS_CUDA_TRY(cudaEventCreate(&e0));
  CMRS_CUDA_TRY(cudaEventCreate(&e1));
  float best = 1e30f;
  int bt = candidates[0];
  int rc = CMRS_OK;
  for (int c = 0; c < ncand && rc == CMRS_OK; ++c) {
    cmrs_spmm_plan *p = nullptr;
    rc = cmrs_spmm_plan_create(batch, A, k, X, Y, candidates[c], 1, workspace, workspace_bytes, stream, &p);
    if (rc) break;
    for (int w = 0; w < 2 && rc == CMRS_OK; ++w) rc = cmrs_spmm_batched(p, stream);
    cudaEventRecord(e0, st);
    for (int r = 0; r < reps && rc == CMRS_OK; ++r) rc = cmrs_spmm_batched(p, stream);
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess && rc == CMRS_OK) rc = set_cuda_error(e);
    cmrs_spmm_plan_destroy(p);
    ms /= reps;
    if (rc == CMRS_OK && ms < best) {
      best = ms;
      bt = candidates[c];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  *best_target = bt;
  if (best_ms) *best_ms = best;
  return CMRS_OK;
}
