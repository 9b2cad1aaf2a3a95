// CRS <-> CMRS conversion kernels (Section 3; packing and the in-strip sort of
// Section 4) and their C-ABI entry points.
#include <algorithm>

#include "common.cuh"

namespace cmrs {
namespace {

constexpr int kSortShortCap = 1024;  // strips up to this length: warp bitonic sort in shared memory
constexpr int kSortMergeRows = 8;    // heights up to this: rows already in column order are merged
constexpr int kSortBatch = 4;        // independent loads each lane issues before using them
constexpr int kSortWarps = 4;
constexpr int kRadixThreads = 128;   // CTA radix sort for longer strips
constexpr int kRadixWarps = kRadixThreads / 32;

struct StatusBlock {
  uint32_t status;
  int32_t max_strip;
  uint32_t pad[62];
};

// ---------------------------------------------------------------- validation
// Section 2.3: RowPtr[0] = 0, RowPtr[rows] = nnz, row lengths >= 0.
__global__ void k_validate_rowptr(int rows, int nnz, const int32_t *__restrict__ row_ptr, StatusBlock *st) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t bad = 0;
  for (; i < rows; i += gridDim.x * blockDim.x) {
    int32_t a = row_ptr[i], b = row_ptr[i + 1];
    if (a < 0 || b < a || b > nnz) bad = 1;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && (row_ptr[0] != 0 || row_ptr[rows] != nnz)) bad = 1;
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&st->status, ST_BAD_ROWPTR);
}

// ---------------------------------------------------------------- StripPtr
// Section 3: StripPtr[j] = RowPtr[j * height] for j < strips, StripPtr[strips]
// = nnz.  Also records the longest strip.
__global__ void k_strip_ptr(int rows, int nnz, int height, int strips, const int32_t *__restrict__ row_ptr,
                            int32_t *__restrict__ strip_ptr, StatusBlock *st) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  int len = 0;
  if (j <= strips) {
    int32_t v = j < strips ? row_ptr[(int64_t)j * height] : nnz;
    strip_ptr[j] = v;
    if (j < strips) {
      int64_t e = std::min<int64_t>((int64_t)(j + 1) * height, rows);
      len = row_ptr[e] - v;
    }
  }
  for (int o = 16; o > 0; o >>= 1) len = max(len, __shfl_xor_sync(0xffffffffu, len, o));
  if ((threadIdx.x & 31) == 0 && len > 0) atomicMax(&st->max_strip, len);
}

// ---------------------------------------------------------------- value forms
// F32: IEEE round to nearest even.  BF16: round to nearest even of the FP32
// value.  BF16X2: hi = BF16(v), lo = BF16(v - hi), the difference taken in
// double.
template <int DT>
struct Encode;
template <>
struct Encode<CMRS_F64> {
  typedef double Out;
  __device__ static void put(double v, Out *hi, Out *, int64_t k) { hi[k] = v; }
};
template <>
struct Encode<CMRS_F32> {
  typedef float Out;
  __device__ static void put(double v, Out *hi, Out *, int64_t k) { hi[k] = __double2float_rn(v); }
};
template <>
struct Encode<CMRS_BF16> {
  typedef uint16_t Out;
  __device__ static void put(double v, Out *hi, Out *, int64_t k) {
    hi[k] = __bfloat16_as_ushort(__float2bfloat16_rn(__double2float_rn(v)));
  }
};
template <>
struct Encode<CMRS_BF16X2> {
  typedef uint16_t Out;
  __device__ static void put(double v, Out *hi, Out *lo, int64_t k) {
    uint16_t h = __bfloat16_as_ushort(__float2bfloat16_rn(__double2float_rn(v)));
    double rest = __dsub_rn(v, (double)bf16_bits_to_float(h));
    hi[k] = h;
    lo[k] = __bfloat16_as_ushort(__float2bfloat16_rn(__double2float_rn(rest)));
  }
};

// ---------------------------------------------------------------- packing
// Section 4: packed = (col << bits) | (row mod height).  A warp takes 32
// consecutive rows at a time: their entries are one contiguous CRS range,
// walked with coalesced loads, kPackU batches of 32 in flight per lane; an
// entry finds its row among the 32 row starts (held one per lane) by a
// five-step shuffle search.  A group of rows with an invalid RowPtr range is
// skipped (the validation kernel has flagged it), so no access leaves the
// arrays.
constexpr int kPackU = 4;
template <typename In, int DT>
__global__ void k_pack(int rows, int cols, int nnz, int height, int bits, const int32_t *__restrict__ row_ptr,
                       const int32_t *__restrict__ col_ind, const In *__restrict__ val_in,
                       uint32_t *__restrict__ packed, typename Encode<DT>::Out *__restrict__ vhi,
                       typename Encode<DT>::Out *__restrict__ vlo, StatusBlock *st) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  const long long groups = ((long long)rows + 31) / 32;
  uint32_t bad = 0;
  for (long long g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < groups; g += warps) {
    const long long r0 = g * 32;
    const long long r = r0 + lane;
    // row `lane` of the group: [start, end); rows past the matrix are empty
    const int32_t start = r < rows ? row_ptr[r] : 0;
    const int32_t last = row_ptr[min(r0 + 32, (long long)rows)];
    int32_t end = __shfl_down_sync(0xffffffffu, start, 1);
    if (lane == 31 || r + 1 >= rows) end = last;
    const bool ok = r >= rows || (start >= 0 && end >= start && end <= nnz);
    if (!__all_sync(0xffffffffu, ok)) continue;
    const int32_t e0 = __shfl_sync(0xffffffffu, start, 0);
    const int32_t e1 = last;
    const int nrows = (int)min(32LL, rows - r0);
    const int32_t key = lane < nrows ? start : e1;  // empty tail rows sort last
    const uint32_t ris_lane = (uint32_t)(r % height);
    for (int32_t k0 = e0; k0 < e1; k0 += 32 * kPackU) {
      int32_t c[kPackU];
      In v[kPackU];
#pragma unroll
      for (int u = 0; u < kPackU; ++u) {
        const int32_t k = k0 + 32 * u + lane;
        if (k < e1) {
          c[u] = col_ind[k];
          v[u] = val_in[k];
        }
      }
#pragma unroll
      for (int u = 0; u < kPackU; ++u) {
        const int32_t k = k0 + 32 * u + lane;
        // the row holding k: the last of the group's rows starting at or before k
        int j = 0;
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
          const int32_t sj = __shfl_sync(0xffffffffu, key, j + step);
          if (sj <= k) j += step;
        }
        const uint32_t ris = __shfl_sync(0xffffffffu, ris_lane, j);
        if (k < e1) {
          int32_t col = c[u];
          if (col < 0 || col >= cols) {
            bad = 1;
            col = 0;
          }
          packed[k] = ((uint32_t)col << bits) | ris;
          Encode<DT>::put((double)v[u], vhi, vlo, k);
        }
      }
    }
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&st->status, ST_BAD_COL);
}

// ---------------------------------------------------------------- in-strip sort
// Section 4, fourth optimisation: each strip's entries ordered by column,
// ties kept in CRS order.  Short strips, one warp each.  When the strip's
// rows are each already in column order (the usual CRS) and the height is at
// most kSortMergeRows, the stable order is a merge of the rows: an entry's
// place is its index in its row plus, for every other row, the number of
// that row's entries before it (earlier rows: columns <= its column; later
// rows: columns <), found by binary search.  Otherwise the warp sorts unique
// 64-bit keys (column << 32 | position in strip) with a bitonic network in
// shared memory, which makes the order stable, and gathers the payload by
// position.
template <int DT>
__global__ void __launch_bounds__(kSortWarps * 32) k_sort_short(int strips, int height, int bits,
                                                                 const int32_t *__restrict__ sp,
                                                                 const uint32_t *__restrict__ pin,
                                                                 const typename Encode<DT>::Out *__restrict__ hin,
                                                                 const typename Encode<DT>::Out *__restrict__ lin,
                                                                 uint32_t *__restrict__ pout,
                                                                 typename Encode<DT>::Out *__restrict__ hout,
                                                                 typename Encode<DT>::Out *__restrict__ lout) {
  __shared__ uint64_t keys_all[kSortWarps][kSortShortCap];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint64_t *keys = keys_all[w];
  const int nw = gridDim.x * kSortWarps;
  typedef typename Encode<DT>::Out Out;
  const uint32_t mask = (1u << bits) - 1;
  int s = blockIdx.x * kSortWarps + w;
  int32_t na = s < strips ? sp[s] : 0, nb = s < strips ? sp[s + 1] : 0;
  for (; s < strips; s += nw) {
    const int32_t a = na, len = nb - na;
    if (s + nw < strips) {  // the next strip's bounds, loaded ahead
      na = sp[s + nw];
      nb = sp[s + nw + 1];
    }
    if (len > kSortShortCap || len <= 0) continue;
    if (height <= kSortMergeRows) {
      // the strip's packed words, staged in this warp's shared buffer for the searches
      uint32_t *w32 = reinterpret_cast<uint32_t *>(keys);
      for (int i0 = 0; i0 < len; i0 += 32 * kSortBatch) {
        uint32_t v[kSortBatch];
#pragma unroll
        for (int u = 0; u < kSortBatch; ++u) {
          const int i = i0 + 32 * u + lane;
          v[u] = i < len ? pin[a + i] : 0u;
        }
#pragma unroll
        for (int u = 0; u < kSortBatch; ++u) {
          const int i = i0 + 32 * u + lane;
          if (i < len) w32[i] = v[u];
        }
      }
      __syncwarp();
      // first entry of row `lane` (RowInStrip is non-decreasing in an unsorted strip)
      int start = 0;
      if (lane > 0 && lane < height) {
        int lo = 0, hi = len;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if ((w32[mid] & mask) < (uint32_t)lane) lo = mid + 1;
          else hi = mid;
        }
        start = lo;
      }
      int end = __shfl_down_sync(0xffffffffu, start, 1);
      if (lane == height - 1) end = len;
      bool unordered = false;
      for (int i = lane + 1; i < len; i += 32) {
        const uint32_t p = w32[i], q = w32[i - 1];
        if ((p & mask) == (q & mask) && (p >> bits) < (q >> bits)) unordered = true;
      }
      int rs[kSortMergeRows], re[kSortMergeRows];
#pragma unroll
      for (int r = 0; r < kSortMergeRows; ++r) {
        rs[r] = __shfl_sync(0xffffffffu, start, r);
        re[r] = __shfl_sync(0xffffffffu, end, r);
      }
      if (!__any_sync(0xffffffffu, unordered)) {
        for (int i0 = 0; i0 < len; i0 += 32 * kSortBatch) {
          Out hv[kSortBatch], lv[kSortBatch];
#pragma unroll
          for (int u = 0; u < kSortBatch; ++u) {
            const int i = i0 + 32 * u + lane;
            if (i < len) {
              hv[u] = hin[a + i];
              if (DT == CMRS_BF16X2) lv[u] = lin[a + i];
            }
          }
#pragma unroll
          for (int u = 0; u < kSortBatch; ++u) {
            const int i = i0 + 32 * u + lane;
            if (i >= len) continue;
            const uint32_t p = w32[i];
            const int r = (int)(p & mask);
            const uint32_t c = p >> bits;
            int rank = 0;
#pragma unroll
            for (int q = 0; q < kSortMergeRows; ++q) {
              if (q >= height) break;
              if (q == r) {
                rank += i - rs[q];
              } else {
                int lo = rs[q], hi = re[q];
                while (lo < hi) {
                  const int mid = (lo + hi) >> 1;
                  const uint32_t cm = w32[mid] >> bits;
                  if (q < r ? cm <= c : cm < c) lo = mid + 1;
                  else hi = mid;
                }
                rank += lo - rs[q];
              }
            }
            pout[a + rank] = p;
            hout[a + rank] = hv[u];
            if (DT == CMRS_BF16X2) lout[a + rank] = lv[u];
          }
        }
        __syncwarp();  // the buffer is reused by the next strip
        continue;
      }
      __syncwarp();  // the bitonic path below overwrites the staged words
    }
    int n2 = 1;
    while (n2 < len) n2 <<= 1;
    for (int i0 = 0; i0 < n2; i0 += 32 * kSortBatch) {
      uint32_t v[kSortBatch];
#pragma unroll
      for (int u = 0; u < kSortBatch; ++u) {
        const int i = i0 + 32 * u + lane;
        v[u] = i < len ? pin[a + i] : 0u;
      }
#pragma unroll
      for (int u = 0; u < kSortBatch; ++u) {
        const int i = i0 + 32 * u + lane;
        if (i < n2) keys[i] = i < len ? ((uint64_t)(v[u] >> bits) << 32) | (uint32_t)i : ~0ull;
      }
    }
    __syncwarp();
    for (int k = 2; k <= n2; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = lane; i < n2; i += 32) {
          int ixj = i ^ j;
          if (ixj > i) {
            uint64_t u = keys[i], v = keys[ixj];
            bool up = (i & k) == 0;
            if ((u > v) == up) {
              keys[i] = v;
              keys[ixj] = u;
            }
          }
        }
        __syncwarp();
      }
    }
    for (int i0 = 0; i0 < len; i0 += 32 * kSortBatch) {
      uint32_t pv[kSortBatch];
      Out hv[kSortBatch], lv[kSortBatch];
#pragma unroll
      for (int u = 0; u < kSortBatch; ++u) {
        const int i = i0 + 32 * u + lane;
        if (i < len) {
          const int32_t src = a + (int32_t)(keys[i] & 0xffffffffu);
          pv[u] = pin[src];
          hv[u] = hin[src];
          if (DT == CMRS_BF16X2) lv[u] = lin[src];
        }
      }
#pragma unroll
      for (int u = 0; u < kSortBatch; ++u) {
        const int i = i0 + 32 * u + lane;
        if (i < len) {
          pout[a + i] = pv[u];
          hout[a + i] = hv[u];
          if (DT == CMRS_BF16X2) lout[a + i] = lv[u];
        }
      }
    }
    __syncwarp();
  }
}

// Long strips: one CTA per strip, stable least-significant-digit radix sort of
// (column, position) pairs through two global ping-pong buffers, 8 bits per
// pass.  Each pass: digit histogram, exclusive scan into bucket bases, then a
// stable scatter of 128-entry chunks ranked per warp with match_any and across
// warps by a per-digit prefix.
template <int DT>
__global__ void __launch_bounds__(kRadixThreads) k_sort_long(int strips, int bits, int col_bits,
                                                             const int32_t *__restrict__ sp,
                                                             const uint32_t *__restrict__ pin,
                                                             const typename Encode<DT>::Out *__restrict__ hin,
                                                             const typename Encode<DT>::Out *__restrict__ lin,
                                                             uint32_t *__restrict__ pout,
                                                             typename Encode<DT>::Out *__restrict__ hout,
                                                             typename Encode<DT>::Out *__restrict__ lout,
                                                             uint32_t *__restrict__ keyA, uint32_t *__restrict__ posA,
                                                             uint32_t *__restrict__ keyB, uint32_t *__restrict__ posB,
                                                             const StatusBlock *__restrict__ stb) {
  __shared__ int hist[256];
  if (stb->max_strip <= kSortShortCap) return;  // no long strip: nothing to do
  __shared__ int base[256];
  __shared__ int ccount[256];
  __shared__ int wcnt[kRadixWarps][257];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  for (int s = blockIdx.x; s < strips; s += gridDim.x) {
    const int32_t a = sp[s], len = sp[s + 1] - a;
    if (len <= kSortShortCap) continue;
    for (int i = tid; i < len; i += kRadixThreads) {
      keyA[a + i] = pin[a + i] >> bits;
      posA[a + i] = (uint32_t)i;
    }
    uint32_t *ks = keyA, *ps = posA, *kd = keyB, *pd = posB;
    __syncthreads();
    for (int shift = 0; shift < col_bits; shift += 8) {
      for (int d = tid; d < 256; d += kRadixThreads) hist[d] = 0;
      for (int d = tid; d < kRadixWarps * 257; d += kRadixThreads) (&wcnt[0][0])[d] = 0;
      __syncthreads();
      for (int i = tid; i < len; i += kRadixThreads) atomicAdd(&hist[(ks[a + i] >> shift) & 255], 1);
      __syncthreads();
      if (tid == 0) {
        int run = 0;
        for (int d = 0; d < 256; ++d) {
          base[d] = run;
          run += hist[d];
        }
      }
      __syncthreads();
      for (int c0 = 0; c0 < len; c0 += kRadixThreads) {
        const int i = c0 + tid;
        const bool valid = i < len;
        uint32_t key = 0, pos = 0;
        int d = 256;
        if (valid) {
          key = ks[a + i];
          pos = ps[a + i];
          d = (key >> shift) & 255;
        }
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & ((1u << lane) - 1));
        if (valid && (__ffs(peers) - 1) == lane) wcnt[w][d] = __popc(peers);
        __syncthreads();
        for (int dd = tid; dd < 256; dd += kRadixThreads) {
          int run = 0;
          for (int ww = 0; ww < kRadixWarps; ++ww) {
            int t = wcnt[ww][dd];
            wcnt[ww][dd] = run;
            run += t;
          }
          ccount[dd] = run;
        }
        __syncthreads();
        if (valid) {
          int dst = base[d] + wcnt[w][d] + rank;
          kd[a + dst] = key;
          pd[a + dst] = pos;
        }
        __syncthreads();
        for (int dd = tid; dd < 256; dd += kRadixThreads) {
          base[dd] += ccount[dd];
          for (int ww = 0; ww < kRadixWarps; ++ww) wcnt[ww][dd] = 0;
        }
        __syncthreads();
      }
      uint32_t *t;
      t = ks; ks = kd; kd = t;
      t = ps; ps = pd; pd = t;
      __syncthreads();
    }
    for (int i = tid; i < len; i += kRadixThreads) {
      int32_t src = a + (int32_t)ps[a + i];
      pout[a + i] = pin[src];
      hout[a + i] = hin[src];
      if (DT == CMRS_BF16X2) lout[a + i] = lin[src];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- CMRS -> CRS
// One warp per strip.  Pass 1 counts entries per RowInStrip; an exclusive scan
// over the strip's rows gives RowPtr[s*h + r] = StripPtr[s] + #(RIS < r).
// Pass 2 scatters each entry to RowPtr[row] + (its rank among the strip's
// entries of the same row, in strip order), a stable counting sort.
// Unsorted strips (kSorted false) already hold their entries in CRS order:
// the entry arrays are copied with the row bits dropped (coalesced, kPackU
// batches in flight per lane) and RowPtr[s*h + r] is the first entry of
// row r, found by a binary search of RowInStrip.
template <typename V, bool kSorted>
__global__ void k_to_csr(int rows, int nnz, int height, int bits, int strips, const int32_t *__restrict__ sp,
                         const uint32_t *__restrict__ packed, const V *__restrict__ vin, const V *__restrict__ vin_lo,
                         int32_t *__restrict__ row_ptr, int32_t *__restrict__ col_out, V *__restrict__ vout,
                         V *__restrict__ vout_lo, uint32_t *status) {
  __shared__ int cnt_all[8][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int *cnt = cnt_all[w];
  const uint32_t mask = (1u << bits) - 1;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  uint32_t bad = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) row_ptr[rows] = nnz;
  for (int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < strips; s += nw) {
    const int32_t a = sp[s], b = sp[s + 1];
    const int64_t row0 = (int64_t)s * height;
    const int nrow = (int)std::min<int64_t>(height, rows - row0);
    if (!kSorted) {
      int32_t start = a;
      if (lane > 0 && lane < nrow) {
        int32_t lo = a, hi = b;
        while (lo < hi) {
          const int32_t mid = lo + ((hi - lo) >> 1);
          if ((packed[mid] & mask) < (uint32_t)lane) lo = mid + 1;
          else hi = mid;
        }
        start = lo;
      }
      if (lane < nrow) row_ptr[row0 + lane] = start;
      for (int32_t i0 = a; i0 < b; i0 += 32 * kPackU) {
        uint32_t p[kPackU];
        V v[kPackU], vl[kPackU];
#pragma unroll
        for (int u = 0; u < kPackU; ++u) {
          const int32_t i = i0 + 32 * u + lane;
          if (i < b) {
            p[u] = packed[i];
            if (vout) {
              v[u] = vin[i];
              if (vout_lo) vl[u] = vin_lo[i];
            }
          }
        }
#pragma unroll
        for (int u = 0; u < kPackU; ++u) {
          const int32_t i = i0 + 32 * u + lane;
          if (i < b) {
            if ((p[u] & mask) >= (uint32_t)nrow) bad = 1;
            col_out[i] = (int32_t)(p[u] >> bits);
            if (vout) {
              vout[i] = v[u];
              if (vout_lo) vout_lo[i] = vl[u];
            }
          }
        }
      }
      continue;
    }
    cnt[lane] = 0;
    __syncwarp();
    for (int32_t i = a + lane; i < b; i += 32) {
      int r = (int)(packed[i] & mask);
      if (r >= nrow) bad = 1;
      else atomicAdd(&cnt[r], 1);
    }
    __syncwarp();
    int v = lane < nrow ? cnt[lane] : 0;
    int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    int base = a + incl - v;
    if (lane < nrow) row_ptr[row0 + lane] = base;
    __syncwarp();
    cnt[lane] = base;  // running insertion point of row `lane`
    __syncwarp();
    for (int32_t i0 = a; i0 < b; i0 += 32) {
      const int32_t i = i0 + lane;
      int r = 32;
      uint32_t p = 0;
      if (i < b) {
        p = packed[i];
        r = (int)(p & mask);
        if (r >= nrow) r = 32;
      }
      const uint32_t peers = __match_any_sync(0xffffffffu, r);
      const int rank = __popc(peers & ((1u << lane) - 1));
      if (r < 32) {
        int dst = cnt[r] + rank;
        col_out[dst] = (int32_t)(p >> bits);
        if (vout) {
          vout[dst] = vin[i];
          if (vout_lo) vout_lo[dst] = vin_lo[i];
        }
      }
      __syncwarp();
      if (r < 32 && (__ffs(peers) - 1) == lane) cnt[r] += __popc(peers);
      __syncwarp();
    }
  }
  if (status && __any_sync(0xffffffffu, bad) && lane == 0) atomicOr(status, ST_BAD_RIS);
}

// ---------------------------------------------------------------- host glue
struct FromCsrLayout {
  size_t status = 0, ptmp = 0, vtmp = 0, keyA = 0, posA = 0, keyB = 0, posB = 0, total = 0;
};

FromCsrLayout from_csr_layout(int nnz, int dtype, uint32_t flags) {
  FromCsrLayout L;
  size_t off = align256(sizeof(StatusBlock));
  if (flags & CMRS_SORTED) {
    L.ptmp = off;
    off += align256((size_t)nnz * 4);
    L.vtmp = off;
    off += align256((size_t)cmrs_val_bytes(nnz, dtype));
    L.keyA = off;
    off += align256((size_t)nnz * 4);
    L.posA = off;
    off += align256((size_t)nnz * 4);
    L.keyB = off;
    off += align256((size_t)nnz * 4);
    L.posB = off;
    off += align256((size_t)nnz * 4);
  }
  L.total = off;
  return L;
}

template <typename In, int DT>
int from_csr_impl(int rows, int cols, int nnz, int height, int bits, uint32_t flags, const int32_t *row_ptr,
                  const int32_t *col_ind, const In *val_in, int32_t *strip_ptr, uint32_t *packed, void *val_out,
                  char *ws, const FromCsrLayout &L, cudaStream_t st, int *max_strip) {
  typedef typename Encode<DT>::Out Out;
  StatusBlock *sb = reinterpret_cast<StatusBlock *>(ws + L.status);
  const int strips = (int)ceil_div(rows, height);
  CMRS_CUDA_TRY(cudaMemsetAsync(sb, 0, sizeof(StatusBlock), st));
  const int sms = sm_count();
  {
    int g = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(rows, 256), sms * 8));
    k_validate_rowptr<<<g, 256, 0, st>>>(rows, nnz, row_ptr, sb);
    CMRS_LAUNCH_CHECK();
  }
  k_strip_ptr<<<(int)ceil_div(strips + 1, 256), 256, 0, st>>>(rows, nnz, height, strips, row_ptr, strip_ptr, sb);
  CMRS_LAUNCH_CHECK();
  const bool sorted = (flags & CMRS_SORTED) != 0;
  uint32_t *pk = sorted ? reinterpret_cast<uint32_t *>(ws + L.ptmp) : packed;
  Out *vh = sorted ? reinterpret_cast<Out *>(ws + L.vtmp) : reinterpret_cast<Out *>(val_out);
  Out *vl = DT == CMRS_BF16X2 ? vh + cmrs_pad8(nnz) : nullptr;
  if (rows > 0 && nnz > 0) {
    int g = (int)std::min<int64_t>(ceil_div((int64_t)rows, 256), (int64_t)sms * 16);  // 8 warps x 32 rows
    k_pack<In, DT><<<g, 256, 0, st>>>(rows, cols, nnz, height, bits, row_ptr, col_ind, val_in, pk, vh, vl, sb);
    CMRS_LAUNCH_CHECK();
  }
  if (sorted && nnz > 0 && strips > 0) {
    Out *oh = reinterpret_cast<Out *>(val_out);
    Out *ol = DT == CMRS_BF16X2 ? oh + cmrs_pad8(nnz) : nullptr;
    int per_sm = 0;  // one resident wave: every warp walks the same number of strips
    CMRS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sort_short<DT>, kSortWarps * 32, 0));
    int gs = (int)std::min<int64_t>(ceil_div(strips, kSortWarps), (int64_t)sms * std::max(1, per_sm));
    k_sort_short<DT><<<gs, kSortWarps * 32, 0, st>>>(strips, height, bits, strip_ptr, pk, vh, vl, packed, oh, ol);
    CMRS_LAUNCH_CHECK();
    int col_bits = 1;
    while (col_bits < 31 && ((int64_t)1 << col_bits) < (int64_t)cols) ++col_bits;
    int gl = (int)std::min<int64_t>(strips, (int64_t)sms * 4);
    k_sort_long<DT><<<gl, kRadixThreads, 0, st>>>(strips, bits, col_bits, strip_ptr, pk, vh, vl, packed, oh, ol,
                                                  reinterpret_cast<uint32_t *>(ws + L.keyA),
                                                  reinterpret_cast<uint32_t *>(ws + L.posA),
                                                  reinterpret_cast<uint32_t *>(ws + L.keyB),
                                                  reinterpret_cast<uint32_t *>(ws + L.posB), sb);
    CMRS_LAUNCH_CHECK();
  }
  StatusBlock host;
  CMRS_CUDA_TRY(cudaMemcpyAsync(&host, sb, 8, cudaMemcpyDeviceToHost, st));
  CMRS_CUDA_TRY(cudaStreamSynchronize(st));
  *max_strip = host.max_strip;
  if (host.status & (ST_BAD_ROWPTR | ST_BAD_COL)) return CMRS_ERR_CSR_INVALID;
  return CMRS_OK;
}

template <typename In>
int from_csr_dispatch(int dtype, int rows, int cols, int nnz, int height, int bits, uint32_t flags,
                      const int32_t *row_ptr, const int32_t *col_ind, const In *val_in, int32_t *strip_ptr,
                      uint32_t *packed, void *val_out, char *ws, const FromCsrLayout &L, cudaStream_t st,
                      int *max_strip) {
  switch (dtype) {
    case CMRS_F64:
      return from_csr_impl<In, CMRS_F64>(rows, cols, nnz, height, bits, flags, row_ptr, col_ind, val_in, strip_ptr,
                                         packed, val_out, ws, L, st, max_strip);
    case CMRS_F32:
      return from_csr_impl<In, CMRS_F32>(rows, cols, nnz, height, bits, flags, row_ptr, col_ind, val_in, strip_ptr,
                                         packed, val_out, ws, L, st, max_strip);
    case CMRS_BF16:
      return from_csr_impl<In, CMRS_BF16>(rows, cols, nnz, height, bits, flags, row_ptr, col_ind, val_in, strip_ptr,
                                          packed, val_out, ws, L, st, max_strip);
    case CMRS_BF16X2:
      return from_csr_impl<In, CMRS_BF16X2>(rows, cols, nnz, height, bits, flags, row_ptr, col_ind, val_in,
                                            strip_ptr, packed, val_out, ws, L, st, max_strip);
  }
  return CMRS_ERR_ARG;
}

}  // namespace
}  // namespace cmrs

using namespace cmrs;

extern "C" int cmrs_from_csr_workspace(int rows, int nnz, int height, uint32_t flags, int dtype, size_t *bytes) {
  if (!bytes || rows < 0 || nnz < 0 || dtype < CMRS_F64 || dtype > CMRS_BF16X2) return CMRS_ERR_ARG;
  if (cmrs_bits_for_height(height) < 0) return CMRS_ERR_HEIGHT;
  *bytes = from_csr_layout(nnz, dtype, flags).total;
  return CMRS_OK;
}

extern "C" int cmrs_from_csr(int rows, int cols, int nnz, const int32_t *row_ptr, const int32_t *col_ind,
                             const void *val_in, int val_in_dtype, int height, uint32_t flags, int dtype,
                             int32_t *strip_ptr_out, uint32_t *col_packed_out, void *val_out, void *workspace,
                             size_t workspace_bytes, void *stream, cmrs_matrix *out) {
  CMRS_TRACE();
  if (rows < 0 || cols < 0 || nnz < 0) return CMRS_ERR_ARG;
  if (dtype < CMRS_F64 || dtype > CMRS_BF16X2) return CMRS_ERR_ARG;
  if (val_in_dtype != CMRS_F64 && val_in_dtype != CMRS_F32) return CMRS_ERR_ARG;
  if (flags & ~CMRS_SORTED) return CMRS_ERR_ARG;
  const int bits = cmrs_bits_for_height(height);
  if (bits < 0) return CMRS_ERR_HEIGHT;
  if ((uint64_t)cols > ((uint64_t)1 << (32 - bits))) return CMRS_ERR_COL_OVERFLOW;
  if (!row_ptr || !strip_ptr_out) return CMRS_ERR_ARG;
  if (nnz > 0 && (!col_ind || !val_in || !col_packed_out || !val_out)) return CMRS_ERR_ARG;
  const FromCsrLayout L = from_csr_layout(nnz, dtype, flags);
  if (!workspace || workspace_bytes < L.total || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return CMRS_ERR_WORKSPACE;
  int max_strip = 0;
  cudaStream_t st = as_stream(stream);
  char *ws = reinterpret_cast<char *>(workspace);
  int rc = val_in_dtype == CMRS_F64
               ? from_csr_dispatch<double>(dtype, rows, cols, nnz, height, bits, flags, row_ptr, col_ind,
                                           reinterpret_cast<const double *>(val_in), strip_ptr_out, col_packed_out,
                                           val_out, ws, L, st, &max_strip)
               : from_csr_dispatch<float>(dtype, rows, cols, nnz, height, bits, flags, row_ptr, col_ind,
                                          reinterpret_cast<const float *>(val_in), strip_ptr_out, col_packed_out,
                                          val_out, ws, L, st, &max_strip);
  if (rc != CMRS_OK) return rc;
  if (out) {
    out->rows = rows;
    out->cols = cols;
    out->nnz = nnz;
    out->height = height;
    out->strips = (int32_t)ceil_div(rows, height);
    out->bits = bits;
    out->flags = flags;
    out->dtype = dtype;
    out->max_strip_nnz = max_strip;
    out->strip_ptr = strip_ptr_out;
    out->col_packed = col_packed_out;
    out->val = val_out;
  }
  return CMRS_OK;
}

extern "C" int cmrs_to_csr_workspace(const cmrs_matrix *A, size_t *bytes) {
  if (!A || !bytes) return CMRS_ERR_ARG;
  *bytes = 256;
  return CMRS_OK;
}

template <typename V>
void launch_to_csr(bool sorted, int g, cudaStream_t st, const cmrs_matrix *A, const V *vin, const V *vin_lo,
                   int32_t *row_ptr, int32_t *col_out, V *vout, V *vout_lo, uint32_t *status) {
  if (sorted)
    k_to_csr<V, true><<<g, 256, 0, st>>>(A->rows, A->nnz, A->height, A->bits, A->strips, A->strip_ptr,
                                         A->col_packed, vin, vin_lo, row_ptr, col_out, vout, vout_lo, status);
  else
    k_to_csr<V, false><<<g, 256, 0, st>>>(A->rows, A->nnz, A->height, A->bits, A->strips, A->strip_ptr,
                                          A->col_packed, vin, vin_lo, row_ptr, col_out, vout, vout_lo, status);
}

extern "C" int cmrs_to_csr(const cmrs_matrix *A, int32_t *row_ptr_out, int32_t *col_ind_out, void *val_out,
                           void *workspace, size_t workspace_bytes, void *stream) {
  CMRS_TRACE();
  if (!A || !row_ptr_out || A->rows < 0 || A->nnz < 0) return CMRS_ERR_ARG;
  if (cmrs_bits_for_height(A->height) != A->bits) return CMRS_ERR_HEIGHT;
  if (A->strips != ceil_div(A->rows, A->height)) return CMRS_ERR_ARG;
  if (A->nnz > 0 && (!A->col_packed || !col_ind_out || !A->strip_ptr)) return CMRS_ERR_ARG;
  if (A->dtype < CMRS_F64 || A->dtype > CMRS_BF16X2) return CMRS_ERR_ARG;
  if (A->flags & CMRS_PADDED) return CMRS_ERR_UNSUPPORTED;  // zero items are not told apart from entries
  uint32_t *status = (workspace && workspace_bytes >= 256) ? reinterpret_cast<uint32_t *>(workspace) : nullptr;
  cudaStream_t st = as_stream(stream);
  const int sms = sm_count();
  if (A->strips == 0) {
    CMRS_CUDA_TRY(cudaMemsetAsync(row_ptr_out, 0, sizeof(int32_t), st));
    return CMRS_OK;
  }
  int g = (int)std::min<int64_t>(ceil_div((int64_t)A->strips * 32, 256), (int64_t)sms * 8);
  const int64_t lo_off = cmrs_pad8(A->nnz);
  const bool sorted = (A->flags & CMRS_SORTED) != 0;
  switch (A->dtype) {
    case CMRS_F64:
      launch_to_csr<double>(sorted, g, st, A, (const double *)A->val, nullptr, row_ptr_out, col_ind_out,
                            (double *)val_out, nullptr, status);
      break;
    case CMRS_F32:
      launch_to_csr<float>(sorted, g, st, A, (const float *)A->val, nullptr, row_ptr_out, col_ind_out,
                           (float *)val_out, nullptr, status);
      break;
    case CMRS_BF16:
      launch_to_csr<uint16_t>(sorted, g, st, A, (const uint16_t *)A->val, nullptr, row_ptr_out, col_ind_out,
                              (uint16_t *)val_out, nullptr, status);
      break;
    case CMRS_BF16X2:
      launch_to_csr<uint16_t>(sorted, g, st, A, (const uint16_t *)A->val, (const uint16_t *)A->val + lo_off,
                              row_ptr_out, col_ind_out, (uint16_t *)val_out,
                              val_out ? (uint16_t *)val_out + lo_off : nullptr, status);
      break;
  }
  CMRS_LAUNCH_CHECK();
  return CMRS_OK;
}
