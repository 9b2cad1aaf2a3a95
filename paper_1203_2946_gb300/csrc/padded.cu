// Modified CMRS (Section 6.6): strips rearranged into 32-item warp passes that
// hold at most M contiguous items of any one row (M = slots, 1..8; the
// paper's is 8), filled with zero items, so that the SpMV kernel can add
// each product into slot (lane mod M) of its row's buffer without two lanes
// of a pass meeting in one slot.  With M = 1 and height 32 every pass holds
// exactly one item (or zero item) of each row, row r at lane r.
//
// One warp per strip, lane r owning row r.  Each pass is planned from the
// items each row has left: C = max(ceil(total / 32), ceil(longest / M))
// passes remain; every row first takes max(0, left - M (C - 1)) items (what
// the remaining C - 1 passes cannot hold), free room then goes to the rows
// with most items left (ties: lower row) up to min(left, M) each, and room
// still free becomes zero items, rows 0 upwards, each row topped up to M.
// Inside a pass the rows appear in ascending order, each one run.
//
// The plan always ends after exactly C0 = max(ceil(T / 32), ceil(L / M))
// passes (T the strip's items, L its longest row), the fewest any arrangement
// can have: with C passes left every row holds at most M C items, so each
// forced take max(0, left - M (C - 1)) is at most left / C and together they
// fit in one pass; the pass then takes min(32, sum of min(left, M)) items,
// which is at least total - 32 (C - 1) because left - min(left, M) <=
// left (C - 1) / C; so after it both the total and the longest row fit in
// C - 1 passes.  The layout pass therefore counts C0 per strip from T and L
// alone; a scan turns the counts into the padded StripPtr; the fill pass runs
// the plan and writes, never more passes than the layout gave the strip.
#include <algorithm>

#include "common.cuh"
#include "scan.cuh"

namespace cmrs {
namespace {

constexpr int kPadWarps = 8;
constexpr uint32_t kFull = 0xffffffffu;
constexpr uint32_t ST_PAD_PLAN = 2u;

__device__ __forceinline__ int warp_excl_scan(int v, int lane) {
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += t;
  }
  return incl - v;
}

// First item of row `lane` of strip [sa, sb) (RowInStrip is non-decreasing
// in an unsorted strip) and its item count; lanes at or past the height get 0.
__device__ __forceinline__ int row_span(int sa, int sb, int height, uint32_t mask,
                                        const uint32_t *__restrict__ packed, int lane, int *first) {
  int start = sa;
  if (lane > 0 && lane < height) {
    int lo = sa, hi = sb;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if ((packed[mid] & mask) < (uint32_t)lane) lo = mid + 1;
      else hi = mid;
    }
    start = lo;
  }
  int end = __shfl_down_sync(kFull, start, 1);
  if (lane == height - 1) end = sb;
  *first = start;
  return lane < height ? end - start : 0;
}

// Runs the plan of strip s and writes its passes from out0 on, at most
// `limit` of them.  Returns false if the plan does not fit (a pass
// overflowing, or more passes than `limit`), which a valid unsorted strip
// never does; the writes stay inside the strip's limit either way.
template <typename S, bool kSplit>
__device__ bool pad_strip_fill(int sa, int sb, int height, int bits, int slots, long long limit,
                               const uint32_t *__restrict__ packed, const S *__restrict__ vh,
                               const S *__restrict__ vl, long long out0, uint32_t *__restrict__ pk_out,
                               S *__restrict__ vo_h, S *__restrict__ vo_l) {
  const int lane = threadIdx.x & 31;
  const uint32_t mask = (1u << bits) - 1;
  int next;
  int left = row_span(sa, sb, height, mask, packed, lane, &next);
  if (left < 0) left = 0;  // a corrupt strip: what is left unwritten is reported below
  long long passes = 0;
  for (;;) {
    const int total = (int)__reduce_add_sync(kFull, (unsigned)left);
    if (total == 0) break;
    if (passes == limit) return false;
    const int longest = (int)__reduce_max_sync(kFull, (unsigned)left);
    const int C = max((total + 31) / 32, (longest + slots - 1) / slots);
    int take = max(0, left - slots * (C - 1));
    int room = 32 - (int)__reduce_add_sync(kFull, (unsigned)take);
    if (room < 0) return false;
    // free room: rows with most items left first, lower row on ties
    const int want = min(left, slots) - take;
    const int wanted = (int)__reduce_add_sync(kFull, (unsigned)max(want, 0));
    int extra;
    if (wanted <= room) {
      extra = max(want, 0);  // every row gets what it wants
    } else {
      // before = the want of the rows ranked ahead (more items left, or as
      // many and a lower row), one distinct count of items left at a time,
      // largest first, until the free room is given out
      const int lv = want > 0 ? left - take : 0;  // >= 1 for a row that wants
      unsigned rem = __ballot_sync(kFull, want > 0);
      int before = room, done = 0;
      while (rem && done < room) {
        const int v = (int)__reduce_max_sync(kFull, (rem >> lane) & 1u ? (unsigned)lv : 0u);
        const unsigned g = __ballot_sync(kFull, ((rem >> lane) & 1u) && lv == v);
        const int wg = (g >> lane) & 1u ? want : 0;
        const int below = warp_excl_scan(wg, lane);  // want of the group's lower rows
        if ((g >> lane) & 1u) before = done + below;
        done += (int)__reduce_add_sync(kFull, (unsigned)wg);
        rem &= ~g;
      }
      extra = want > 0 ? max(0, min(want, room - before)) : 0;
    }
    take += extra;
    room -= (int)__reduce_add_sync(kFull, (unsigned)extra);
    // zero items: rows 0 upwards, each topped up to `slots`
    const int zcap = lane < height ? slots - take : 0;
    const int zero = max(0, min(zcap, room - warp_excl_scan(zcap, lane)));
    const int len = take + zero;
    const int off = warp_excl_scan(len, lane);
    const long long base = out0 + passes * 32 + off;
#pragma unroll
    for (int j = 0; j < 8; ++j) {  // slots <= 8 items of a row per pass
      if (j < take) {
        pk_out[base + j] = packed[next + j];
        vo_h[base + j] = vh[next + j];
        if (kSplit) vo_l[base + j] = vl[next + j];
      } else if (j < len) {
        pk_out[base + j] = (uint32_t)lane;  // column 0, this row
        vo_h[base + j] = S(0);
        if (kSplit) vo_l[base + j] = S(0);
      }
    }
    next += take;
    left -= take;
    ++passes;
  }
  return passes == limit;
}

// Passes of each strip: max(ceil(T / 32), ceil(L / M)), 0 for an empty strip.
__global__ void __launch_bounds__(kPadWarps * 32) k_pad_count(int strips, int height, int bits, int slots,
                                                             const int32_t *__restrict__ sp,
                                                             const uint32_t *__restrict__ packed,
                                                             int32_t *__restrict__ counts, uint32_t *status) {
  const int nw = gridDim.x * kPadWarps;
  const int lane = threadIdx.x & 31;
  const uint32_t mask = (1u << bits) - 1;
  for (int s = blockIdx.x * kPadWarps + (threadIdx.x >> 5); s < strips; s += nw) {
    const int sa = sp[s], sb = sp[s + 1];
    int first;
    const int len = row_span(sa, sb, height, mask, packed, lane, &first);
    const bool bad = __any_sync(kFull, len < 0) || sb < sa;
    const int longest = (int)__reduce_max_sync(kFull, (unsigned)max(len, 0));
    if (lane == 0) {
      if (bad) atomicOr(status, ST_PAD_PLAN);
      const long long T = bad ? 0 : sb - sa;
      const long long c = std::max((T + 31) / 32, ((long long)longest + slots - 1) / slots);
      counts[s] = bad ? 0 : (int32_t)std::min<long long>(c, 0x7fffffffLL);
    }
  }
}

// M = 1 (so height 32): every row with items left takes exactly one per pass
// (the forced takes and the free room together never turn a row away), so
// pass p holds item p of row r at position r, or a zero item of row r once
// the row has run out; the strip has max(row length) passes.  No plan to run:
// each lane copies its own row, kPadFillU passes' loads in flight.
constexpr int kPadFillU = 8;
template <typename S, bool kSplit>
__device__ bool pad_strip_fill_m1(int sa, int sb, int bits, long long limit, const uint32_t *__restrict__ packed,
                                  const S *__restrict__ vh, const S *__restrict__ vl, long long out0,
                                  uint32_t *__restrict__ pk_out, S *__restrict__ vo_h, S *__restrict__ vo_l) {
  const int lane = threadIdx.x & 31;
  int next;
  int left = row_span(sa, sb, 32, (1u << bits) - 1, packed, lane, &next);
  if (left < 0) left = 0;
  for (long long p = 0; p < limit; p += kPadFillU) {
    uint32_t c[kPadFillU];
    S h[kPadFillU], l[kPadFillU];
#pragma unroll
    for (int u = 0; u < kPadFillU; ++u) {
      c[u] = (uint32_t)lane;  // a zero item: column 0, this row
      h[u] = S(0);
      l[u] = S(0);
      if (p + u < left) {
        c[u] = packed[next + p + u];
        h[u] = vh[next + p + u];
        if (kSplit) l[u] = vl[next + p + u];
      }
    }
#pragma unroll
    for (int u = 0; u < kPadFillU; ++u)
      if (p + u < limit) {
        const long long o = out0 + (p + u) * 32 + lane;
        pk_out[o] = c[u];
        vo_h[o] = h[u];
        if (kSplit) vo_l[o] = l[u];
      }
  }
  return __all_sync(kFull, left <= limit);
}

template <typename S, bool kSplit>
__global__ void __launch_bounds__(kPadWarps * 32, 4) k_pad_fill(int strips, int height, int bits, int slots,
                                                            const int32_t *__restrict__ sp,
                                                            const uint32_t *__restrict__ packed,
                                                            const S *__restrict__ vh, const S *__restrict__ vl,
                                                            const int32_t *__restrict__ sp_out,
                                                            uint32_t *__restrict__ pk_out, S *__restrict__ vo_h,
                                                            S *__restrict__ vo_l) {
  const int nw = gridDim.x * kPadWarps;
  for (int s = blockIdx.x * kPadWarps + (threadIdx.x >> 5); s < strips; s += nw) {
    const long long o0 = sp_out[s], o1 = sp_out[s + 1];
    const long long limit = o1 > o0 ? (o1 - o0) / 32 : 0;
    if (slots == 1)
      pad_strip_fill_m1<S, kSplit>(sp[s], sp[s + 1], bits, limit, packed, vh, vl, o0, pk_out, vo_h, vo_l);
    else
      pad_strip_fill<S, kSplit>(sp[s], sp[s + 1], height, bits, slots, limit, packed, vh, vl, o0, pk_out, vo_h,
                                vo_l);
  }
}

size_t pad_ws_bytes(int strips) { return 256 + scan_ws_bytes(strips); }

int slots_log2(int slots) {
  for (int k = 0; k <= 3; ++k)
    if (slots == (1 << k)) return k;
  return -1;
}

int check_pad_input(const cmrs_matrix *A, int slots) {
  if (slots_log2(slots) < 0) return CMRS_ERR_ARG;
  if (!A) return CMRS_ERR_ARG;
  if (A->rows < 0 || A->cols < 0 || A->nnz < 0) return CMRS_ERR_ARG;
  const int bits = cmrs_bits_for_height(A->height);
  if (bits < 0) return CMRS_ERR_HEIGHT;
  if (A->bits != bits || A->strips != ceil_div(A->rows, A->height)) return CMRS_ERR_ARG;
  if (A->dtype < CMRS_F64 || A->dtype > CMRS_BF16X2) return CMRS_ERR_ARG;
  if (A->flags & ~(CMRS_SORTED | CMRS_PADDED | CMRS_PAD_SLOTS_MASK)) return CMRS_ERR_ARG;
  if (A->flags) return CMRS_ERR_UNSUPPORTED;  // sorted strips, or already padded
  if (A->height * slots < 32) return CMRS_ERR_HEIGHT;
  if (A->rows > 0 && !A->strip_ptr) return CMRS_ERR_ARG;
  if (A->nnz > 0 && (!A->col_packed || !A->val)) return CMRS_ERR_ARG;
  return CMRS_OK;
}

int pad_grid(int strips) {
  static int sms = 0;
  if (sms == 0) sms = sm_count();
  return (int)std::min<long long>(ceil_div(strips, kPadWarps), (long long)sms * 8);
}

template <typename S, bool kSplit>
int launch_fill(const cmrs_matrix *A, int slots, const int32_t *sp_out, int nnz_padded, uint32_t *pk_out,
                void *val_out, cudaStream_t st) {
  const S *vh = reinterpret_cast<const S *>(A->val);
  const S *vl = kSplit ? vh + cmrs_pad8(A->nnz) : nullptr;
  S *oh = reinterpret_cast<S *>(val_out);
  S *ol = kSplit ? oh + cmrs_pad8(nnz_padded) : nullptr;
  k_pad_fill<S, kSplit><<<pad_grid(A->strips), kPadWarps * 32, 0, st>>>(A->strips, A->height, A->bits, slots,
                                                                        A->strip_ptr, A->col_packed, vh, vl, sp_out,
                                                                        pk_out, oh, ol);
  CMRS_LAUNCH_CHECK();
  return CMRS_OK;
}

}  // namespace
}  // namespace cmrs

using namespace cmrs;

extern "C" int cmrs_pad_workspace(const cmrs_matrix *A, int slots, size_t *bytes) {
  if (!bytes) return CMRS_ERR_ARG;
  const int rc = check_pad_input(A, slots);
  if (rc) return rc;
  *bytes = pad_ws_bytes(A->strips);
  return CMRS_OK;
}

extern "C" int cmrs_pad_layout(const cmrs_matrix *A, int slots, int32_t *strip_ptr_padded, int32_t *nnz_padded,
                               void *workspace, size_t workspace_bytes, void *stream) {
  CMRS_TRACE();
  int rc = check_pad_input(A, slots);
  if (rc) return rc;
  if (!strip_ptr_padded || !nnz_padded) return CMRS_ERR_ARG;
  if (!workspace || workspace_bytes < pad_ws_bytes(A->strips) || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return CMRS_ERR_WORKSPACE;
  cudaStream_t st = as_stream(stream);
  char *ws = reinterpret_cast<char *>(workspace);
  uint32_t *status = reinterpret_cast<uint32_t *>(ws);
  int32_t *counts = reinterpret_cast<int32_t *>(ws + 256);
  CMRS_CUDA_TRY(cudaMemsetAsync(status, 0, 4, st));
  const int S = A->strips;
  if (S == 0) {
    CMRS_CUDA_TRY(cudaMemsetAsync(strip_ptr_padded, 0, 4, st));
    *nnz_padded = 0;
    CMRS_CUDA_TRY(cudaStreamSynchronize(st));
    return CMRS_OK;
  }
  k_pad_count<<<pad_grid(S), kPadWarps * 32, 0, st>>>(S, A->height, A->bits, slots, A->strip_ptr, A->col_packed,
                                                      counts, status);
  CMRS_LAUNCH_CHECK();
  rc = scan_counts(S, ws + 256, 32, strip_ptr_padded, status, st);
  if (rc) return rc;
  uint32_t host[2] = {0, 0};
  CMRS_CUDA_TRY(cudaMemcpyAsync(&host[0], status, 4, cudaMemcpyDeviceToHost, st));
  CMRS_CUDA_TRY(cudaMemcpyAsync(&host[1], strip_ptr_padded + S, 4, cudaMemcpyDeviceToHost, st));
  CMRS_CUDA_TRY(cudaStreamSynchronize(st));
  if (host[0] & ST_PAD_PLAN) return CMRS_ERR_CSR_INVALID;
  if (host[0] & ST_SCAN_OVERFLOW) return CMRS_ERR_ARG;
  *nnz_padded = (int32_t)host[1];
  return CMRS_OK;
}

extern "C" int cmrs_pad_fill(const cmrs_matrix *A, int slots, const int32_t *strip_ptr_padded, int32_t nnz_padded,
                             uint32_t *col_packed_out, void *val_out, void *stream, cmrs_matrix *out) {
  CMRS_TRACE();
  int rc = check_pad_input(A, slots);
  if (rc) return rc;
  if (!out || nnz_padded < 0 || (nnz_padded & 31)) return CMRS_ERR_ARG;
  if (A->rows > 0 && !strip_ptr_padded) return CMRS_ERR_ARG;
  if (nnz_padded > 0 && (!col_packed_out || !val_out)) return CMRS_ERR_ARG;
  if ((reinterpret_cast<uintptr_t>(col_packed_out) | reinterpret_cast<uintptr_t>(val_out)) & 15) return CMRS_ERR_ARG;
  cudaStream_t st = as_stream(stream);
  if (A->strips > 0 && nnz_padded > 0) {
    switch (A->dtype) {
      case CMRS_F64: rc = launch_fill<double, false>(A, slots, strip_ptr_padded, nnz_padded, col_packed_out, val_out, st); break;
      case CMRS_F32: rc = launch_fill<float, false>(A, slots, strip_ptr_padded, nnz_padded, col_packed_out, val_out, st); break;
      case CMRS_BF16: rc = launch_fill<uint16_t, false>(A, slots, strip_ptr_padded, nnz_padded, col_packed_out, val_out, st); break;
      default: rc = launch_fill<uint16_t, true>(A, slots, strip_ptr_padded, nnz_padded, col_packed_out, val_out, st); break;
    }
    if (rc) return rc;
  }
  *out = *A;
  out->nnz = nnz_padded;
  out->flags = CMRS_PADDED | ((uint32_t)slots_log2(slots) << CMRS_PAD_SLOTS_SHIFT);
  out->max_strip_nnz = -1;
  out->strip_ptr = strip_ptr_padded;
  out->col_packed = col_packed_out;
  out->val = val_out;
  return CMRS_OK;
}
