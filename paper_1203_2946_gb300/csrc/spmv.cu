// y = A x on the CMRS format (Section 4, Algorithm 1), three thread mappings.
//
// GB300 design notes.  FP64 issue rate on this part is about 1/58 of FP32
// (measured 1.2 TFLOP/s), so at HBM speed an FP64 SpMV can afford about one
// FP64 instruction per nonzero.  The ROW and MERGE mappings therefore keep
// each row's sum in one thread's register (one FMA per nonzero, no per-lane
// buffer, no lane reduction); the STRIP mapping is Algorithm 1 as the paper
// states it (per-lane row buffers + reduction) and costs 31*height extra adds
// per strip.  Nonzero streams are copied into shared memory by the bulk-copy
// engine (cp.async.bulk, mbarrier completion, L2 evict-first) two stages
// ahead of the threads that use them.
#include <algorithm>
#include <mutex>

#include <type_traits>

#include "common.cuh"

namespace cmrs {
namespace {

#ifndef CMRS_ROW_ROWS
#define CMRS_ROW_ROWS 128
#endif
constexpr int kRowThreads = CMRS_ROW_ROWS;    // ROW: rows per block
constexpr int kRowCap = 32 * CMRS_ROW_ROWS;   // ROW: entries per shared-memory stage
// MERGE per value form (FP64; the FP32-accumulated forms): entries per
// thread (odd, so that a warp's shared loads hit 32 banks), resident CTAs
// per SM asked of the register allocator, and the CTAs per SM the launch
// keeps (its shared-memory carveout holds that many and no more, the rest of
// the SM's L1/shared storage stays L1).  The x gathers miss L1 and each miss
// in flight holds an L1 line: with two stages of 15 entries a thread at 5
// CTAs, the FP32 tiles left 92 KB of L1 and FP64 (4 CTAs) 60 KB, and a
// further 8 KB of shared memory per CTA, leaving 28 KB, took the power-law
// FP32 product from 143 to 222 us.  FP32: 11 entries at 6 CTAs (80
// registers); FP64: 9 at 5 CTAs (96 registers); both keep 92 KB of L1.
// Matrices whose rows average CMRS_MERGE_LONG_MU entries or more pay for
// MERGE's per-tile joins more than for L1 misses: they take the _LONG tiles,
// 15 entries a thread at as many CTAs as fit (dense 10^4 x 10^4 as sparse:
// FP64 425 us against 486 us with the short tiles, FP32 257 against 287).
#ifndef CMRS_MERGE_LONG_MU
#define CMRS_MERGE_LONG_MU 16
#endif
#ifndef CMRS_MERGE_E_F64_LONG
#define CMRS_MERGE_E_F64_LONG 15
#endif
#ifndef CMRS_MERGE_MINB_F64_LONG
#define CMRS_MERGE_MINB_F64_LONG 4
#endif
#ifndef CMRS_MERGE_CTAS_F64_LONG
#define CMRS_MERGE_CTAS_F64_LONG 0
#endif
#ifndef CMRS_MERGE_E_F32_LONG
#define CMRS_MERGE_E_F32_LONG 15
#endif
#ifndef CMRS_MERGE_MINB_F32_LONG
#define CMRS_MERGE_MINB_F32_LONG 5
#endif
#ifndef CMRS_MERGE_CTAS_F32_LONG
#define CMRS_MERGE_CTAS_F32_LONG 0
#endif
#ifndef CMRS_MERGE_E_F64
#define CMRS_MERGE_E_F64 9
#endif
#ifndef CMRS_MERGE_E_F32
#define CMRS_MERGE_E_F32 11
#endif
#ifndef CMRS_MERGE_MINB_F64
#define CMRS_MERGE_MINB_F64 5
#endif
#ifndef CMRS_MERGE_MINB_F32
#define CMRS_MERGE_MINB_F32 6
#endif
#ifndef CMRS_MERGE_THREADS
#define CMRS_MERGE_THREADS 128  // threads per MERGE tile (a CTA)
#endif
constexpr int kMergeThreads = CMRS_MERGE_THREADS;
#ifndef CMRS_MERGE_VSMEM
#define CMRS_MERGE_VSMEM 0
#endif
// MERGE: values read from the staged tile at their multiply-add instead of held in registers
constexpr bool kMergeVSmem = CMRS_MERGE_VSMEM != 0;
#ifndef CMRS_MERGE_CTAS_F64
#define CMRS_MERGE_CTAS_F64 5
#endif
#ifndef CMRS_MERGE_CTAS_F32
#define CMRS_MERGE_CTAS_F32 6
#endif
// ROW's lane mapping: most resident CTAs per SM (0: as many as fit)
#ifndef CMRS_LANE_CTAS
#define CMRS_LANE_CTAS 0
#endif
template <int DT, bool kLong>
struct MergeCfg {
  static constexpr bool F64 = DT == CMRS_F64;
  static constexpr int E = F64 ? (kLong ? CMRS_MERGE_E_F64_LONG : CMRS_MERGE_E_F64)
                               : (kLong ? CMRS_MERGE_E_F32_LONG : CMRS_MERGE_E_F32);
  static constexpr int Tile = kMergeThreads * E;  // entries per tile, a multiple of 8
  static constexpr int MinBlocks = F64 ? (kLong ? CMRS_MERGE_MINB_F64_LONG : CMRS_MERGE_MINB_F64)
                                       : (kLong ? CMRS_MERGE_MINB_F32_LONG : CMRS_MERGE_MINB_F32);
  static constexpr int Ctas = F64 ? (kLong ? CMRS_MERGE_CTAS_F64_LONG : CMRS_MERGE_CTAS_F64)
                                  : (kLong ? CMRS_MERGE_CTAS_F32_LONG : CMRS_MERGE_CTAS_F32);
  static_assert(E % 2 == 1 && Tile % 8 == 0, "MERGE: odd entries per thread, 8-entry-aligned tiles");
};
// the long-row tiles are a second kernel only where they differ
template <int DT>
constexpr bool merge_long_differs() {
  return MergeCfg<DT, true>::E != MergeCfg<DT, false>::E ||
         MergeCfg<DT, true>::MinBlocks != MergeCfg<DT, false>::MinBlocks ||
         MergeCfg<DT, true>::Ctas != MergeCfg<DT, false>::Ctas;
}
constexpr int kMergeWarps = kMergeThreads / 32;
constexpr int kStripWarps = 8;
constexpr int kStages = 2;

enum : uint8_t { F_HEAD = 1, F_TAIL = 2, F_THROUGH = 4 };

// Rows crossing a MERGE tile boundary: each tile leaves the partial sum of the
// row it starts inside (head) and of the row that runs past its end (tail).
struct TileRec {
  int32_t head_row, head_flag;  // head_flag: 0 none, 1 row ends in this tile, 2 row spans the whole tile
  double head_sum;
  int32_t tail_row, tail_flag;  // tail_flag: 1 if a row starts here and continues past the tile
  double tail_sum;
};

struct StageInfo {
  long long a8;
  int staged;
  int pad;
};

template <int DT>
struct Stage {
  typedef typename Form<DT>::Stored S;
  static constexpr bool kSplit = DT == CMRS_BF16X2;
  static constexpr size_t al(size_t b) { return (b + 127) & ~size_t(127); }
  static constexpr size_t colp_bytes(int cap) { return al((size_t)(cap + 8) * 4); }
  static constexpr size_t val_bytes(int cap) { return al((size_t)(cap + 8) * sizeof(S)); }
  static constexpr size_t bytes(int cap) { return colp_bytes(cap) + val_bytes(cap) * (kSplit ? 2 : 1); }
};

// One thread: copy entries [ea, eb) of the three streams into a stage.  The
// bulk copy covers the 8-entry-aligned body [a8, e8) (16-byte aligned for all
// forms); entries past the last full 8-group of the array are loaded by this
// thread, so nothing outside the arrays is read.
template <int DT>
__device__ void issue_stage(long long ea, long long eb, long long nnz, const uint32_t *packed,
                            const typename Form<DT>::Stored *hi, const typename Form<DT>::Stored *lo, char *stage,
                            int cap, uint64_t *bar, uint64_t pol, StageInfo *info) {
  typedef typename Form<DT>::Stored S;
  const long long a8 = ea & ~7LL, nnz8 = nnz & ~7LL;
  long long e8 = (eb + 7) & ~7LL;
  if (e8 > nnz8) e8 = nnz8;
  if (e8 < a8) e8 = a8;
  uint32_t *sc = reinterpret_cast<uint32_t *>(stage);
  S *sh = reinterpret_cast<S *>(stage + Stage<DT>::colp_bytes(cap));
  S *sl = reinterpret_cast<S *>(stage + Stage<DT>::colp_bytes(cap) + Stage<DT>::val_bytes(cap));
  for (long long k = e8; k < eb; ++k) {
    sc[k - a8] = packed[k];
    sh[k - a8] = hi[k];
    if (Stage<DT>::kSplit) sl[k - a8] = lo[k];
  }
  info->a8 = a8;
  info->staged = 1;
  const uint32_t cnt = (uint32_t)(e8 - a8);
  fence_proxy_async();
  mbar_arrive_expect_tx(bar, cnt * (4u + (uint32_t)sizeof(S) * (Stage<DT>::kSplit ? 2u : 1u)));
  if (cnt) {
    bulk_g2s(sc, packed + a8, cnt * 4u, bar, pol);
    bulk_g2s(sh, hi + a8, cnt * (uint32_t)sizeof(S), bar, pol);
    if (Stage<DT>::kSplit) bulk_g2s(sl, lo + a8, cnt * (uint32_t)sizeof(S), bar, pol);
  }
}

// First k in [lo, hi) whose RowInStrip is >= r (RowInStrip is non-decreasing
// inside an unsorted strip), or hi.
__device__ __forceinline__ int lb_ris(const uint32_t *cp, long long base, int lo, int hi, uint32_t r, uint32_t mask) {
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if ((cp[mid - base] & mask) < r) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// ============================================================== ROW mapping
// A block is CMRS_ROW_ROWS (default 128) consecutive rows: one contiguous range of
// the nonzero streams.  A producer warp bulk-copies each block's range into a
// ring of kRowStages shared-memory stages (full/empty mbarrier pairs, no CTA
// barrier in the loop) and prefetches the next block's bounds while it
// waits.  T consumer threads share a row: each walks a contiguous segment of
// it (its start from a binary search on RowInStrip, which is non-decreasing in
// an unsorted strip; its end from the next row's start), one FMA per entry,
// and the T partial sums are joined down a shuffle tree with T - 1 adds.  A block larger than
// the stage capacity is read from global memory instead.
#ifndef CMRS_ROW_T_F64
#define CMRS_ROW_T_F64 4
#endif
#ifndef CMRS_ROW_T_F32
#define CMRS_ROW_T_F32 2
#endif
#ifndef CMRS_ROW_STAGES
#define CMRS_ROW_STAGES 2
#endif
constexpr int kRowStages = CMRS_ROW_STAGES;

// x gathers a thread issues per batch; 0 = a 32-entry row share.  FP64 uses 7,
// a 27-point row's share at T = 4 (measured 173 -> 164 us on the 27-point
// 128^3 matrix against 8).
#ifndef CMRS_ROW_CH
#define CMRS_ROW_CH 0
#endif
#ifndef CMRS_ROW_CH_F64
#define CMRS_ROW_CH_F64 7
#endif
#ifndef CMRS_ROW_ILP
#define CMRS_ROW_ILP 1
#endif
// Loading the next block's strip bounds one block ahead pays for FP64 (measured
// 184 -> 172 us on the 27-point 128^3 matrix) and costs the FP32-accumulated
// forms (100 -> 131 us), so it is chosen per form.
#ifndef CMRS_ROW_PREFETCH_F64
#define CMRS_ROW_PREFETCH_F64 1
#endif
#ifndef CMRS_ROW_PREFETCH_F32
#define CMRS_ROW_PREFETCH_F32 0
#endif

template <int DT>
struct RowCfg {
  static constexpr int T = DT == CMRS_F64 ? CMRS_ROW_T_F64 : CMRS_ROW_T_F32;
  static constexpr int kConsumers = kRowThreads * T;   // threads
  static constexpr int kThreads = kConsumers + 32;     // + producer warp
  // x gathers a thread issues per batch (default: a whole 32-entry row share)
  static constexpr int kCH = (DT == CMRS_F64 && CMRS_ROW_CH_F64 > 0) ? CMRS_ROW_CH_F64
                             : CMRS_ROW_CH > 0 ? CMRS_ROW_CH : ((32 / T) < 8 ? 8 : (32 / T));
  static constexpr int kILP = CMRS_ROW_ILP;            // independent FMA chains per segment
  static constexpr bool kPrefetch = DT == CMRS_F64 ? CMRS_ROW_PREFETCH_F64 : CMRS_ROW_PREFETCH_F32;
};

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Partial dot product of entries [lo, hi) with x, one FMA each; CH gathers
// are issued before their FMAs.
template <int DT, int CH, int ILP>
__device__ __forceinline__ typename Form<DT>::Acc seg_dot(const uint32_t *cp, const typename Form<DT>::Stored *vh,
                                                          const typename Form<DT>::Stored *vl, long long base, int lo,
                                                          int hi, int bits, const typename Form<DT>::Acc *x) {
  typedef typename Form<DT>::Acc A;
  A acc[ILP];
#pragma unroll
  for (int i = 0; i < ILP; ++i) acc[i] = A(0);
  // longest segment in the warp: FMAs past it are not issued at all (FP64
  // issue is charged per warp instruction, whatever its active lanes)
  const int nmax = __reduce_max_sync(0xffffffffu, hi - lo);
  // FP64: whole batches of CH entries, then the last, shorter batch one entry
  // at a time -- unrolled behind warp-uniform guards, its multiply-adds were
  // computed for all CH and discarded, and an FP64 warp instruction costs its
  // issue slot whatever its lanes do (p7, one entry per row: 688 -> 409 us).
  // The FP32-accumulated forms keep one guarded batch: their multiply-adds are
  // cheap and the batch keeps its gathers in flight.
  const int nfull = DT == CMRS_F64 ? nmax - nmax % CH : nmax;
  for (int j0 = 0; j0 < nfull; j0 += CH) {
    const int k = lo + j0;
    A xv[CH];
#pragma unroll
    for (int j = 0; j < CH; ++j)
      if (k + j < hi) xv[j] = ld_x(x + (cp[k + j - base] >> bits));
#pragma unroll
    for (int j = 0; j < CH; ++j)
      if (j0 + j < nmax) {  // warp-uniform
        if (k + j < hi) acc[j % ILP] = fma_acc(Form<DT>::value(vh, vl, k + j - base), xv[j], acc[j % ILP]);
      }
  }
#pragma unroll 1
  for (int j = nfull; j < nmax; ++j) {
    const int k = lo + j;
    if (k < hi) acc[0] = fma_acc(Form<DT>::value(vh, vl, k - base), ld_x(x + (cp[k - base] >> bits)), acc[0]);
  }
#pragma unroll
  for (int i = 1; i < ILP; ++i) acc[0] += acc[i];
  return acc[0];
}

template <int DT>
__global__ void __launch_bounds__(RowCfg<DT>::kThreads) k_spmv_row(int rows, int height, int bits, int nnz,
                                                                   const int32_t *__restrict__ sp,
                                                                   const uint32_t *__restrict__ packed,
                                                                   const typename Form<DT>::Stored *__restrict__ hi,
                                                                   const typename Form<DT>::Stored *__restrict__ lo,
                                                                   const typename Form<DT>::Acc *__restrict__ x,
                                                                   typename Form<DT>::Acc *__restrict__ y,
                                                                   const int32_t *__restrict__ row_map,
                                                                   uint32_t *status) {
  typedef typename Form<DT>::Stored S;
  typedef typename Form<DT>::Acc A;
  constexpr int T = RowCfg<DT>::T;
  constexpr int kConsumerWarps = RowCfg<DT>::kConsumers / 32;
  extern __shared__ __align__(128) char smem[];
  __shared__ uint64_t full[kRowStages], empty[kRowStages];
  __shared__ StageInfo info[kRowStages];
  const int tid = threadIdx.x;
  const int nblk = (rows + kRowThreads - 1) / kRowThreads;
  const uint32_t mask = (1u << bits) - 1;
  const size_t stage_bytes = Stage<DT>::bytes(kRowCap);
  if (tid == 0) {
    for (int i = 0; i < kRowStages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], kConsumerWarps);
    }
    fence_barrier_init();
  }
  __syncthreads();

  if (tid < 32) {
    // ---------------- producer warp (one lane)
    if (tid != 0) return;
    const uint64_t pol = policy_evict_first();
    auto bounds = [&](int b, long long &ea, long long &eb) {
      const long long r0 = (long long)b * kRowThreads;
      const long long r1 = min(r0 + kRowThreads, (long long)rows);
      ea = sp[(int)(r0 / height)];
      eb = sp[(int)((r1 - 1) / height) + 1];
    };
    long long ea = 0, eb = 0, nea = 0, neb = 0;
    int b = blockIdx.x;
    if (b < nblk) bounds(b, ea, eb);
    for (int it = 0; b < nblk; ++it, b += gridDim.x) {
      const int st = it % kRowStages, use = it / kRowStages;
      const int bn = b + gridDim.x;
      if (bn < nblk) bounds(bn, nea, neb);  // consumed next iteration
      if (use > 0 && !mbar_wait_bounded(&empty[st], (use - 1) & 1)) {
        atomicOr(status, ST_TIMEOUT);
        return;
      }
      if (eb - ea <= kRowCap) {
        issue_stage<DT>(ea, eb, nnz, packed, hi, lo, smem + st * stage_bytes, kRowCap, &full[st], pol, &info[st]);
      } else {
        info[st].staged = 0;
        info[st].a8 = 0;
        mbar_arrive_expect_tx(&full[st], 0);
      }
      ea = nea;
      eb = neb;
    }
    return;
  }

  // ---------------- consumer warps
  const int ctid = tid - 32;
  const int lane = tid & 31;
  const int q = ctid % T;          // segment index inside the row
  const int rloc = ctid / T;       // row inside the block
  // strip bounds of this thread's row, loaded one block ahead
  int nsa = 0, nsb = 0;
  if (RowCfg<DT>::kPrefetch && blockIdx.x < (unsigned)nblk) {
    const long long row0 = (long long)blockIdx.x * kRowThreads + rloc;
    if (row0 < rows) {
      const int s0 = (int)(row0 / height);
      nsa = sp[s0];
      nsb = sp[s0 + 1];
    }
  }
  for (int it = 0, b = blockIdx.x; b < nblk; ++it, b += gridDim.x) {
    const int st = it % kRowStages, use = it / kRowStages;
    const long long row = (long long)b * kRowThreads + rloc;
    const bool active = row < rows;
    const int s = active ? (int)(row / height) : 0;
    const uint32_t r = (uint32_t)(row - (long long)s * height);
    int sa = nsa, sb = nsb;
    if (!RowCfg<DT>::kPrefetch) {
      sa = active ? sp[s] : 0;
      sb = active ? sp[s + 1] : 0;
    } else {
      const long long rown = row + (long long)gridDim.x * kRowThreads;
      if (rown < rows) {
        const int sn = (int)(rown / height);
        nsa = sp[sn];
        nsb = sp[sn + 1];
      }
    }
    const bool ok = mbar_wait_bounded(&full[st], use & 1);
    if (!ok) atomicOr(status, ST_TIMEOUT);
    const bool staged = info[st].staged;
    const char *stg = smem + st * stage_bytes;
    const uint32_t *cp = staged ? reinterpret_cast<const uint32_t *>(stg) : packed;
    const S *vh = staged ? reinterpret_cast<const S *>(stg + Stage<DT>::colp_bytes(kRowCap)) : hi;
    const S *vl = staged ? reinterpret_cast<const S *>(stg + Stage<DT>::colp_bytes(kRowCap) +
                                                       Stage<DT>::val_bytes(kRowCap))
                         : (Stage<DT>::kSplit ? lo : hi);
    const long long base = staged ? info[st].a8 : 0;
    const bool run = ok && active;
    // the first lane of each row's group searches; the group shares the result
    int k0 = sa;
    if (run && r > 0 && q == 0) k0 = lb_ris(cp, base, sa, sb, r, mask);
    if (T > 1) k0 = __shfl_sync(0xffffffffu, k0, lane & ~(T - 1));
    const int nxt = __shfl_down_sync(0xffffffffu, k0, T);
    int k1 = sb;
    if (run && r + 1 < (uint32_t)height && row + 1 < rows) {
      if (lane + T < 32) k1 = nxt;
      else k1 = lb_ris(cp, base, k0, sb, r + 1, mask);
    }
    // every lane calls (an inactive row has an empty segment) so that the
    // warp-wide bound inside is well defined
    const int seg = run ? (k1 - k0 + T - 1) / T : 0;
    const int a0 = run ? min(k1, k0 + q * seg) : 0, a1 = run ? min(k1, a0 + seg) : 0;
    A acc = seg_dot<DT, RowCfg<DT>::kCH, RowCfg<DT>::kILP>(cp, vh, vl, base, a0, a1, bits, x);
    // join the T partial sums into lane q == 0 with T - 1 adds in total (FP64
    // issue is counted per active lane, so only the lanes that keep a sum add)
#pragma unroll
    for (int o = T / 2; o >= 1; o >>= 1) {
      const A other = __shfl_down_sync(0xffffffffu, acc, o);
      if (q < o) acc += other;
    }
    if (run && q == 0) {
      const long long t = row_map ? row_map[row] : row;  // y position (row map of a reordered matrix)
      if (t >= 0 && t < rows) y[t] = acc;
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[st]);
    if (!ok) break;
  }
}

// ============================================================== LANE mapping
// Plain CMRS, a lane per row (used by CMRS_VARIANT_ROW when the strip height
// divides 32).  A warp takes 32 consecutive rows, i.e. whole strips, whose
// entries are one contiguous range of the streams; one lane bulk-copies the
// range into the warp's own shared-memory stage, and lane r then walks row r
// with one multiply-add per entry, the row's sum in a register, as the M = 1
// walk of Section 6.6 does on padded strips -- but on the plain layout: the
// row starts come from one binary search on RowInStrip per lane, and the
// stage turns the row-by-row order of the strips into the lane-by-lane order
// of the walk.  In a warp the lanes gather x at the same position of 32
// consecutive rows (for a stencil, consecutive columns).  No join adds (on
// this GPU an FP64 warp instruction costs its issue slot whatever its active
// lanes do) and no CTA barrier: each warp waits on its own mbarrier.  A range
// longer than the stage is read from global memory instead: ROW takes this
// mapping only for matrices whose mean row is short enough for most units to
// fit the stage (longer rows go to the share-per-thread kernel below).
#ifndef CMRS_ROW_LANE
#define CMRS_ROW_LANE 1  // 0: ROW always runs k_spmv_row
#endif
#ifndef CMRS_LANE_CAP
#define CMRS_LANE_CAP 896  // most entries per warp stage (28 per row)
#endif
#ifndef CMRS_LANE_SLACK
#define CMRS_LANE_SLACK 40  // stage entries per row of the mean length, in 32nds (40: 1.25x)
#endif
#ifndef CMRS_LANE_MAX_MU
#define CMRS_LANE_MAX_MU 28.0  // mean entries per row up to which ROW takes the lane mapping
#endif
#ifndef CMRS_LANE_MAX_L
#define CMRS_LANE_MAX_L 4  // most lanes sharing a row (1, 2 or 4)
#endif
#ifndef CMRS_LANE_WARPS
#define CMRS_LANE_WARPS 4
#endif
#ifndef CMRS_LANE_CH_F64
#define CMRS_LANE_CH_F64 5
#endif
#ifndef CMRS_LANE_CH_F32
#define CMRS_LANE_CH_F32 16
#endif
constexpr int kLaneCap = CMRS_LANE_CAP;
constexpr int kLaneWarps = CMRS_LANE_WARPS;

template <int DT, int L>
__global__ void __launch_bounds__(kLaneWarps * 32) k_spmv_lane(int rows, int height, int bits, int cap, int nnz,
                                                              const int32_t *__restrict__ sp,
                                                              const uint32_t *__restrict__ packed,
                                                              const typename Form<DT>::Stored *__restrict__ hi,
                                                              const typename Form<DT>::Stored *__restrict__ lo,
                                                              const typename Form<DT>::Acc *__restrict__ x,
                                                              typename Form<DT>::Acc *__restrict__ y,
                                                              const int32_t *__restrict__ row_map, uint32_t *status) {
  typedef typename Form<DT>::Stored S;
  typedef typename Form<DT>::Acc A;
  constexpr int CH = DT == CMRS_F64 ? CMRS_LANE_CH_F64 : CMRS_LANE_CH_F32;
  extern __shared__ __align__(128) char smem[];
  __shared__ uint64_t bars[kLaneWarps];
  __shared__ StageInfo info[kLaneWarps];
  const unsigned kAll = 0xffffffffu;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  char *stg = smem + (size_t)w * Stage<DT>::bytes(cap);
  const uint32_t mask = (1u << bits) - 1;
  if (lane == 0) {
    mbar_init(&bars[w], 1);
    fence_barrier_init();
  }
  __syncwarp();
  uint64_t pol = 0;
  if (lane == 0) pol = policy_evict_first();
  constexpr int R = 32 / L;  // rows per unit: L lanes share a row
  const int q = lane & (L - 1), slot = lane / L;
  const long long units = ((long long)rows + R - 1) / R;
  const long long nw = (long long)gridDim.x * kLaneWarps;
  uint32_t phase = 0;
  for (long long u = (long long)blockIdx.x * kLaneWarps + w; u < units; u += nw) {
    const long long r0 = u * R;
    const long long r1 = min(r0 + R, (long long)rows);
    const int s0 = (int)(r0 / height), s1 = (int)((r1 - 1) / height) + 1;  // the unit's strips
    const int ea = sp[s0], eb = sp[s1];
    const bool staged = eb - ea <= cap;  // warp-uniform
    if (staged && lane == 0) issue_stage<DT>(ea, eb, nnz, packed, hi, lo, stg, cap, &bars[w], pol, &info[w]);
    // this lane's row and its strip's bounds, loaded while the copy is in flight
    const long long row = r0 + slot;
    const bool active = row < rows;
    const int s = active ? (int)(row / height) : s0;
    const uint32_t rr = active ? (uint32_t)(row - (long long)s * height) : 0;
    const int sa = active ? sp[s] : 0, sb = active ? sp[s + 1] : 0;
    bool ok = true;
    if (staged) {
      ok = __all_sync(kAll, mbar_wait_bounded(&bars[w], phase));
      phase ^= 1;
    }
    if (!ok) {
      if (lane == 0) atomicOr(status, ST_TIMEOUT);
      break;
    }
    const uint32_t *cp = staged ? reinterpret_cast<const uint32_t *>(stg) : packed;
    const S *vh = staged ? reinterpret_cast<const S *>(stg + Stage<DT>::colp_bytes(cap)) : hi;
    const S *vl = staged ? reinterpret_cast<const S *>(stg + Stage<DT>::colp_bytes(cap) + Stage<DT>::val_bytes(cap))
                         : (Stage<DT>::kSplit ? lo : hi);
    const long long base = staged ? info[w].a8 : 0;
    // row r ends where row r + 1 starts, or at its strip's end (the height
    // divides R, so the unit's last row is the last of its strip); the row's
    // first lane searches, its L lanes share the result
    int k0 = sa;
    if (active && rr > 0 && q == 0) k0 = lb_ris(cp, base, sa, sb, rr, mask);
    if (L > 1) k0 = __shfl_sync(kAll, k0, lane & ~(L - 1));
    const int nxt = __shfl_down_sync(kAll, k0, L);
    int k1 = (rr + 1 == (uint32_t)height || row + 1 >= rows || slot == R - 1) ? sb : nxt;
    if (!active) k0 = k1 = 0;
    // lane q of the row's L takes the q-th contiguous share of it
    const int seg = (k1 - k0 + L - 1) / L;
    const int a0 = min(k1, k0 + q * seg), a1 = min(k1, a0 + seg);
    A acc = seg_dot<DT, CH, 1>(cp, vh, vl, base, a0, a1, bits, x);
#pragma unroll
    for (int o = L / 2; o >= 1; o >>= 1) acc += __shfl_down_sync(kAll, acc, o);
    if (active && q == 0) {
      const long long t = row_map ? row_map[row] : row;  // y position (row map of a reordered matrix)
      if (t >= 0 && t < rows) y[t] = acc;
    }
    __syncwarp();  // every lane is done with the stage before the next copy lands in it
  }
}

// ============================================================== STRIP mapping
// Algorithm 1 of Section 4: one warp per strip, lane l takes entries
// strip_start + l, + 32, ...; each entry's product is added to buf[r][l] (r =
// RowInStrip); the 32 partial sums of every row are then halved five times
// (l += l + 16, 8, 4, 2, 1) and lanes < height write the rows.  The buffer is
// laid out row-major [r][32] so that the lanes of a warp touch 32 banks.
// Each lane issues the loads of kStripU of its entries before their sums.
#ifndef CMRS_STRIP_U
#define CMRS_STRIP_U 4
#endif
constexpr int kStripU = CMRS_STRIP_U;
template <int DT>
__global__ void __launch_bounds__(kStripWarps * 32) k_spmv_strip(int rows, int height, int bits, int strips,
                                                                  const int32_t *__restrict__ sp,
                                                                  const uint32_t *__restrict__ packed,
                                                                  const typename Form<DT>::Stored *__restrict__ hi,
                                                                  const typename Form<DT>::Stored *__restrict__ lo,
                                                                  const typename Form<DT>::Acc *__restrict__ x,
                                                                  typename Form<DT>::Acc *__restrict__ y,
                                                                  const int32_t *__restrict__ row_map) {
  typedef typename Form<DT>::Acc A;
  extern __shared__ __align__(128) char smem[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  A *buf = reinterpret_cast<A *>(smem) + (size_t)w * height * 32;
  const uint32_t mask = (1u << bits) - 1;
  const int nw = gridDim.x * kStripWarps;
  const typename Form<DT>::Stored *vl = Stage<DT>::kSplit ? lo : hi;
  for (int s = blockIdx.x * kStripWarps + w; s < strips; s += nw) {
    for (int r = 0; r < height; ++r) buf[r * 32 + lane] = A(0);
    const int a = sp[s], b = sp[s + 1];
    for (int j0 = a; j0 < b; j0 += 32 * kStripU) {  // kStripU steps' loads in flight
      uint32_t c[kStripU];
      A v[kStripU], xv[kStripU];
#pragma unroll
      for (int u = 0; u < kStripU; ++u) {
        const int j = j0 + 32 * u + lane;
        if (j < b) {
          c[u] = packed[j];
          v[u] = Form<DT>::value(hi, vl, j);
        }
      }
#pragma unroll
      for (int u = 0; u < kStripU; ++u)
        if (j0 + 32 * u + lane < b) xv[u] = ld_x(x + (c[u] >> bits));
#pragma unroll
      for (int u = 0; u < kStripU; ++u) {
        if (j0 + 32 * u + lane < b) {
          const int r = (int)(c[u] & mask);
          if (r < height) {
            A *p = buf + r * 32 + lane;
            *p = fma_acc(v[u], xv[u], *p);
          }
        }
      }
    }
    __syncwarp();
    for (int half = 16; half >= 1; half >>= 1) {
      for (int idx = lane; idx < height * half; idx += 32) {
        const int r = idx / half, l = idx - r * half;
        buf[r * 32 + l] += buf[r * 32 + l + half];
      }
      __syncwarp();
    }
    if (lane < height) {
      const long long row = (long long)s * height + lane;
      if (row < rows) {
        const long long t = row_map ? row_map[row] : row;
        if (t >= 0 && t < rows) y[t] = buf[lane * 32];
      }
    }
    __syncwarp();
  }
}

// ============================================================== PADDED mapping
// Section 6.6: one warp per strip of a padded matrix.  Every 32-item pass of
// the strip holds each row as one run of at most M items (M = slots), so
// lane l adds its product into slot (l mod M) of its row in a per-warp
// buffer buf[row][slot] without meeting another lane of the pass (a row's run
// covers consecutive words: at most 2-way bank conflicts, where a
// [slot][row] layout put a whole run in one bank); passes follow each other
// behind a warp barrier (the next pass may touch a slot another lane wrote).
// At the strip's end each row's M slots are summed by G = min(M, 32 / h2)
// lanes (h2 = height rounded up to a power of 2), M / G slots each, then a
// butterfly over the G lanes.  M = 1 (height 32): row r sits at lane r in
// every pass, so lane r keeps row r's sum in a register -- no buffer, no
// barrier, no final sum.  Loads are plain coalesced 32-bit ones, kPadU
// passes in flight per warp.
#ifndef CMRS_PAD_U
#define CMRS_PAD_U 4
#endif
#ifndef CMRS_PAD_MINB
#define CMRS_PAD_MINB 6  // resident CTAs per SM asked of the register allocator (7 and 8 spill)
#endif
constexpr int kPadWarps = 8;
constexpr int kPadU = CMRS_PAD_U;  // passes whose loads are in flight together

template <int DT>
__device__ __forceinline__ typename Form<DT>::Acc ld_val_stream(const typename Form<DT>::Stored *hi,
                                                                const typename Form<DT>::Stored *lo, long long k,
                                                                uint64_t pol) {
  if constexpr (DT == CMRS_F64 || DT == CMRS_F32) {
    return ld_stream(hi + k, pol);
  } else if constexpr (DT == CMRS_BF16) {
    return bf16_bits_to_float(ld_stream(hi + k, pol));
  } else {
    return bf16_bits_to_float(ld_stream(hi + k, pol)) + bf16_bits_to_float(ld_stream(lo + k, pol));
  }
}

template <int DT, int kM, bool kExact>
__global__ void __launch_bounds__(kPadWarps * 32, CMRS_PAD_MINB) k_spmv_padded(int rows, int height, int bits, int strips,
                                                               const int32_t *__restrict__ sp,
                                                               const uint32_t *__restrict__ packed,
                                                               const typename Form<DT>::Stored *__restrict__ hi,
                                                               const typename Form<DT>::Stored *__restrict__ lo,
                                                               const typename Form<DT>::Acc *__restrict__ x,
                                                               typename Form<DT>::Acc *__restrict__ y,
                                                               const int32_t *__restrict__ row_map) {
  typedef typename Form<DT>::Acc A;
  extern __shared__ __align__(16) char smem[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  A *buf = reinterpret_cast<A *>(smem) + (size_t)w * kM * height;
  const uint32_t mask = (1u << bits) - 1;
  const int slot = lane & (kM - 1);
  const uint64_t pol = policy_evict_first();
  const int nw = gridDim.x * kPadWarps;
  int h2 = 1;
  while (h2 < height) h2 <<= 1;
  const int G = kM < 32 / h2 ? kM : 32 / h2;  // lanes summing one row's slots
  const int per = kM / G;
  for (int s = blockIdx.x * kPadWarps + w; s < strips; s += nw) {
    A acc = A(0);
    if (kM > 1) {
      for (int i = lane; i < kM * height; i += 32) buf[i] = A(0);
      __syncwarp();
    }
    const int a = sp[s], b = sp[s + 1];  // multiples of 32
    if constexpr (kExact) {
      // NU passes from k0, every one present: no guard that the compiler could
      // turn into a multiply-add computed and then discarded (on this GPU an
      // FP64 warp instruction costs its issue slot whatever its lanes do)
      auto group = [&](auto nu, int k0) {
        constexpr int NU = decltype(nu)::value;
        uint32_t c[NU];
        A v[NU], xv[NU];
  #pragma unroll
        for (int u = 0; u < NU; ++u) {
          const long long k = (long long)k0 + 32 * u + lane;
          c[u] = ld_stream(packed + k, pol);
          v[u] = ld_val_stream<DT>(hi, lo, k, pol);
        }
  #pragma unroll
        for (int u = 0; u < NU; ++u) xv[u] = ld_x(x + (c[u] >> bits));
  #pragma unroll
        for (int u = 0; u < NU; ++u) {
          if (kM == 1) {
            acc = fma_acc(v[u], xv[u], acc);
          } else {
            A *p = buf + (c[u] & mask) * kM + slot;
            *p = fma_acc(v[u], xv[u], *p);
            __syncwarp();
          }
        }
      };
      int k0 = a;
      for (; k0 + 32 * kPadU <= b; k0 += 32 * kPadU) group(std::integral_constant<int, kPadU>(), k0);
      for (; k0 + 64 <= b; k0 += 64) group(std::integral_constant<int, 2>(), k0);  // the last passes: twos,
      if (k0 < b) group(std::integral_constant<int, 1>(), k0);                         // then one
    } else {  // groups of kPadU passes, the strip's last group guarded
      for (int k0 = a; k0 < b; k0 += 32 * kPadU) {
        uint32_t c[kPadU];
        A v[kPadU], xv[kPadU];
  #pragma unroll
        for (int u = 0; u < kPadU; ++u)
          if (k0 + 32 * u < b) {  // warp-uniform
            const long long k = (long long)k0 + 32 * u + lane;
            c[u] = ld_stream(packed + k, pol);
            v[u] = ld_val_stream<DT>(hi, lo, k, pol);
          }
  #pragma unroll
        for (int u = 0; u < kPadU; ++u)
          if (k0 + 32 * u < b) xv[u] = ld_x(x + (c[u] >> bits));
  #pragma unroll
        for (int u = 0; u < kPadU; ++u)
          if (k0 + 32 * u < b) {
            if (kM == 1) {
              acc = fma_acc(v[u], xv[u], acc);
            } else {
              A *p = buf + (c[u] & mask) * kM + slot;
              *p = fma_acc(v[u], xv[u], *p);
              __syncwarp();
            }
          }
      }
    }
    const long long row0 = (long long)s * height;
    if (kM == 1) {
      if (row0 + lane < rows) {
        const long long t = row_map ? row_map[row0 + lane] : row0 + lane;
        if (t >= 0 && t < rows) y[t] = acc;
      }
    } else {
      __syncwarp();
      const int r = lane / G, part = lane - r * G;
      A sum = A(0);
      if (r < height) {
        const A *q = buf + r * kM + part * per;
        sum = q[0];
        for (int m = 1; m < per; ++m) sum += q[m];
      }
      for (int o = G >> 1; o >= 1; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
      if (part == 0 && r < height && row0 + r < rows) {
        const long long t = row_map ? row_map[row0 + r] : row0 + r;
        if (t >= 0 && t < rows) y[t] = sum;
      }
      __syncwarp();
    }
  }
}

// ============================================================== MERGE mapping
// Tile t = entries [T t, T t + T), T = 128 E, staged by bulk copies; thread i
// owns the E consecutive entries from T t + E i (E = 9 for FP64, 11 for the
// other forms, 15 for both where rows average 16 entries or more).  It finds their strip by
// a binary search of StripPtr between the strips holding the tile's first
// and next tile's first entry (tile_strip[], one small pre-pass), then walks
// the entries: a row's run is summed by one FMA chain; a run that starts and
// ends inside the thread is written at once; a run cut by the thread's end is
// joined, after a CTA barrier, by the thread where it started (walking over
// the following threads' head partials in order); a run cut by the tile's end
// goes to a tile record that a fix-up kernel joins in tile order.  Rows with
// no entries are written as 0 by the thread owning the entry before the gap.
__global__ void k_tile_map(int strips, const int32_t *__restrict__ sp, int tile, int ntiles,
                           int32_t *__restrict__ tile_strip) {
  pdl_launch_dependents();  // the product may start staging its first tiles
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= strips) return;
  const long long a = sp[s], b = sp[s + 1];
  if (b <= a) return;
  for (long long t = (a + tile - 1) / tile; t * tile < b && t < ntiles; ++t) tile_strip[t] = s;
}

template <int DT, bool kLong>
__global__ void __launch_bounds__(kMergeThreads, (MergeCfg<DT, kLong>::MinBlocks))
    k_spmv_merge(int rows, int height, int bits, int strips, int nnz,
                                                              const int32_t *__restrict__ sp,
                                                              const uint32_t *__restrict__ packed,
                                                              const typename Form<DT>::Stored *__restrict__ hi,
                                                              const typename Form<DT>::Stored *__restrict__ lo,
                                                              const typename Form<DT>::Acc *__restrict__ x,
                                                              typename Form<DT>::Acc *__restrict__ y,
                                                              const int32_t *__restrict__ tile_strip, int ntiles,
                                                              TileRec *__restrict__ recs, uint32_t *status) {
  typedef typename Form<DT>::Stored S;
  typedef typename Form<DT>::Acc A;
  constexpr int kMergeE = MergeCfg<DT, kLong>::E, kMergeTile = MergeCfg<DT, kLong>::Tile;
  extern __shared__ __align__(128) char smem[];
  __shared__ uint64_t bars[kStages];
  __shared__ StageInfo info[kStages];
  __shared__ A s_wv[kMergeWarps];         // per warp: scan value of its last lane
  __shared__ int s_wf[kMergeWarps];       // per warp: a segment starts in it
  __shared__ unsigned s_wt[kMergeWarps];  // per warp: lanes whose single run passes through
  __shared__ int s_head0, s_abort;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t mask = (1u << bits) - 1;
  const size_t stage_bytes = Stage<DT>::bytes(kMergeTile);
  if (tid == 0) {
    for (int i = 0; i < kStages; ++i) mbar_init(&bars[i], 1);
    fence_barrier_init();
    s_abort = 0;
  }
  __syncthreads();
  uint64_t pol = 0;
  if (tid == 0) pol = policy_evict_first();
  auto issue = [&](int t, int st) {
    const long long ta = (long long)t * kMergeTile;
    const long long tb = min(ta + kMergeTile, (long long)nnz);
    issue_stage<DT>(ta, tb, nnz, packed, hi, lo, smem + st * stage_bytes, kMergeTile, &bars[st], pol, &info[st]);
  };
  int t = blockIdx.x;
  if (tid == 0 && t < ntiles) issue(t, 0);  // the matrix streams are inputs: no wait needed
  pdl_wait();                                // tile_strip is k_tile_map's output
  pdl_launch_dependents();                   // the fix-up kernel may launch and wait in turn
  for (int it = 0; t < ntiles; ++it, t += gridDim.x) {
    const int st = it & 1;
    if (tid == 0) {
      if (t + (int)gridDim.x < ntiles) issue(t + gridDim.x, st ^ 1);
      recs[t].tail_flag = 0;
    }
    const bool ok = mbar_wait_bounded(&bars[st], (it >> 1) & 1);
    if (!ok) {
      s_abort = 1;
      atomicOr(status, ST_TIMEOUT);
    }
    const char *stg = smem + st * stage_bytes;
    const uint32_t *cp = reinterpret_cast<const uint32_t *>(stg);
    const S *vh = reinterpret_cast<const S *>(stg + Stage<DT>::colp_bytes(kMergeTile));
    const S *vl = reinterpret_cast<const S *>(stg + Stage<DT>::colp_bytes(kMergeTile) + Stage<DT>::val_bytes(kMergeTile));
    const long long base = info[st].a8;
    const long long ta = (long long)t * kMergeTile;
    const long long tb = min(ta + kMergeTile, (long long)nnz);
    const long long k0 = ta + (long long)tid * kMergeE;
    const long long k1 = min(k0 + kMergeE, tb);
    auto put = [&](uint32_t row, A val) {
      if (row < (uint32_t)rows) y[row] = val;
    };
    uint8_t flags = 0;
    A hv = A(0), tv = A(0);      // head partial (row continued from before), tail partial (row going on)
    uint32_t hrow = 0, trow = 0;
    // lanes with entries in this tile (every lane of the warp votes)
    const unsigned part = __ballot_sync(0xffffffffu, ok && k0 < tb);
    if (ok && k0 < tb) {
      // strip holding k0: the largest s in [s_lo, s_hi] with StripPtr[s] <= k0
      int slo = tile_strip[t];
      int shi = (t + 1 < ntiles) ? tile_strip[t + 1] : strips - 1;
      while (slo < shi) {
        const int mid = (slo + shi + 1) >> 1;
        if (sp[mid] <= k0) slo = mid;
        else shi = mid - 1;
      }
      int cur = slo;
      long long next = sp[cur + 1];
      // does the entry before k0 (previous thread, or previous tile for thread 0) lie in the same row?
      bool cont_in = false;
      if (k0 > sp[cur]) {
        const uint32_t cprev = k0 > ta ? cp[k0 - 1 - base] : __ldg(packed + k0 - 1);
        cont_in = (cprev & mask) == (cp[k0 - base] & mask);
      }
      const int n = (int)(k1 - k0);  // 1 .. kMergeE
      // The walk over the thread's entries is compiled twice: for a thread
      // holding all kMergeE entries (every thread but the matrix's last one
      // with entries) the per-entry guards j < n vanish.
      uint32_t c[kMergeE], rw[kMergeE];
      A xv[kMergeE], v[kMergeE];
      // operands first, so that the x loads of the run are in flight together;
      // then the row of every entry: integer work only.  When all of the
      // thread's entries lie in the strip holding k0 (the usual case) no
      // StripPtr walk is needed; otherwise the walk may diverge.
      auto operands_and_rows = [&](auto full) {
#pragma unroll
        for (int j = 0; j < kMergeE; ++j) {
          if (decltype(full)::value || j < n) {
            const long long i = k0 + j - base;
            c[j] = cp[i];
            if (!kMergeVSmem) v[j] = Form<DT>::value(vh, vl, i);
            xv[j] = ld_x(x + (c[j] >> bits));
          }
        }
        if (k1 <= next) {
          const uint32_t r0 = (uint32_t)cur * (uint32_t)height;
#pragma unroll
          for (int j = 0; j < kMergeE; ++j)
            if (decltype(full)::value || j < n) rw[j] = r0 + (c[j] & mask);
        } else {
#pragma unroll
          for (int j = 0; j < kMergeE; ++j) {
            if (decltype(full)::value || j < n) {
              while (k0 + j >= next) next = sp[++cur + 1];
              rw[j] = (uint32_t)cur * (uint32_t)height + (c[j] & mask);
            }
          }
        }
      };
      if (n == kMergeE) operands_and_rows(std::true_type{});
      else operands_and_rows(std::false_type{});
      // rows before the first entry of the matrix are empty
      if (k0 == 0)
        for (uint32_t g = 0; g < rw[0] && g < (uint32_t)rows; ++g) put(g, A(0));
      // The sums: one FMA chain per run of equal rows, no branch around the
      // FMAs (a finished run leaves by a predicated store or a select), and
      // the warp reconverged first, so that every FMA issues for the whole
      // warp (FP64 issue is charged per warp instruction).
      __syncwarp(part);
      auto val_of = [&](int j) -> A { return kMergeVSmem ? Form<DT>::value(vh, vl, k0 + j - base) : v[j]; };
      A acc = fma_acc(val_of(0), xv[0], A(0));
      A head_sum = A(0);
      bool first = true;  // the current run is this thread's first
      uint32_t run_row = rw[0];
      auto sums_and_gaps = [&](auto full) {
#pragma unroll
        for (int j = 1; j < kMergeE; ++j) {
          if (decltype(full)::value || j < n) {
            const bool nw = rw[j] != rw[j - 1];
            const bool to_head = nw && first && cont_in;  // first run continues a row from before k0
            head_sum = to_head ? acc : head_sum;
            if (nw && !to_head) put(rw[j - 1], acc);
            first = first && !nw;
            acc = nw ? A(0) : acc;
            acc = fma_acc(val_of(j), xv[j], acc);
            run_row = rw[j];
          }
        }
        // rows with no entries between two runs of this thread (rows are
        // non-decreasing along the entries; one test finds whether any is skipped)
        bool gap = false;
#pragma unroll
        for (int j = 1; j < kMergeE; ++j)
          if (decltype(full)::value || j < n) gap = gap || rw[j] > rw[j - 1] + 1;
        if (gap) {
#pragma unroll
          for (int j = 1; j < kMergeE; ++j)
            if (decltype(full)::value || j < n)
              for (uint32_t g = rw[j - 1] + 1; g < rw[j] && g < (uint32_t)rows; ++g) put(g, A(0));
        }
      };
      if (n == kMergeE) sums_and_gaps(std::true_type{});
      else sums_and_gaps(std::false_type{});
      // the entry after this thread's last one: same row?
      long long next_row = rows;
      if (k1 < nnz) {
        const uint32_t cn = (k1 < tb) ? cp[k1 - base] : __ldg(packed + k1);
        int s2 = cur;
        while (k1 >= sp[s2 + 1]) ++s2;
        next_row = (long long)s2 * height + (cn & mask);
      }
      const bool cont_out = next_row == (long long)run_row;
      if (first && cont_in) {
        // one run, continuing a row from before k0
        hv = acc;
        hrow = run_row;
        flags = cont_out ? (F_HEAD | F_THROUGH) : F_HEAD;
      } else {
        if (cont_in) {
          hv = head_sum;
          hrow = rw[0];
          flags = F_HEAD;
        }
        if (cont_out) {
          tv = acc;
          trow = run_row;
          flags |= F_TAIL;
        } else {
          put(run_row, acc);
        }
      }
      if (!cont_out)
        for (long long g = (long long)run_row + 1; g < next_row && g < rows; ++g) put((uint32_t)g, A(0));
    }
    // Rows crossing thread boundaries, joined by a segmented scan over the
    // tile's threads in thread order.  A thread whose single run continues on
    // both sides (THROUGH) passes its head partial along; every other thread
    // starts a segment with its tail partial (0 if none).  A row that ends
    // inside thread e (HEAD, not THROUGH) is the segment's running sum at
    // e - 1 plus e's head partial.  The in-warp scan takes as many shuffle
    // steps as the longest run of THROUGH lanes needs (0..5, warp-uniform), so
    // short rows pay nothing and a tile inside one long row pays 5 FP64 adds
    // per warp instead of a 127-step serial walk.
    const bool through = (flags & F_THROUGH) != 0;
    const bool start = !through || tid == 0;
    A v = through ? hv : ((flags & F_TAIL) ? tv : A(0));
    bool f = start;
    unsigned z = ~__ballot_sync(0xffffffffu, start);
    int nsteps = 0;  // ceil(log2(longest run of non-start lanes + 1))
    for (int sh = 1; sh <= 16 && z; sh <<= 1) {
      ++nsteps;
      z &= z >> sh;
    }
    for (int st2 = 0, d = 1; st2 < nsteps; ++st2, d <<= 1) {
      const A vo = __shfl_up_sync(0xffffffffu, v, d);
      const int fo = __shfl_up_sync(0xffffffffu, (int)f, d);
      if (lane >= d) {
        if (!f) v = vo + v;
        f = f || fo;
      }
    }
    const unsigned tmask = __ballot_sync(0xffffffffu, through);
    const bool end = (flags & F_HEAD) && !through;
    if (lane == 31) {
      s_wv[wid] = v;
      s_wf[wid] = f;
    }
    if (lane == 0) s_wt[wid] = tmask;
    if (tid == 0) s_head0 = (flags & F_HEAD) != 0;
    __syncthreads();
    if (!s_abort) {
      // the segment open at this warp's start, summed over the warps before it
      A carry = A(0);
      if (wid > 0 && __any_sync(0xffffffffu, !f || (end && lane == 0))) {
        for (int u = 0; u < wid; ++u) carry = s_wf[u] ? s_wv[u] : carry + s_wv[u];
        if (!f) v = carry + v;
      }
      A in = __shfl_up_sync(0xffffffffu, v, 1);
      if (lane == 0) in = carry;
      int estar = kMergeThreads;  // first thread whose run does not pass through
      for (int u = 0; u < kMergeWarps; ++u)
        if (~s_wt[u]) {
          estar = u * 32 + __ffs(~s_wt[u]) - 1;
          break;
        }
      const bool head0 = s_head0 != 0;  // the tile starts inside a row
      if (end) {
        const A res = in + hv;
        if (head0 && tid == estar) {
          recs[t].head_row = (int)hrow;
          recs[t].head_sum = (double)res;
          recs[t].head_flag = 1;
        } else {
          put(hrow, res);
        }
      }
      if (tid == kMergeThreads - 1) {
        if (head0 && estar == kMergeThreads) {
          // one row runs through the whole tile
          recs[t].head_row = (int)hrow;
          recs[t].head_sum = (double)v;
          recs[t].head_flag = 2;
          recs[t].tail_flag = 0;
        } else if (through || (flags & F_TAIL)) {
          recs[t].tail_row = (int)(through ? hrow : trow);
          recs[t].tail_sum = (double)v;
          recs[t].tail_flag = 1;
        } else {
          recs[t].tail_flag = 0;
        }
      }
      if (tid == 0 && !head0) recs[t].head_flag = 0;
    }
    __syncthreads();
    if (s_abort) break;
  }
}

template <typename A>
__global__ void k_merge_fixup(int ntiles, int rows, const TileRec *__restrict__ recs, A *__restrict__ y) {
  pdl_wait();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntiles || recs[t].tail_flag != 1) return;
  A sum = (A)recs[t].tail_sum;
  for (int u = t + 1; u < ntiles; ++u) {
    sum += (A)recs[u].head_sum;
    if (recs[u].head_flag != 2) break;
  }
  const int row = recs[t].tail_row;
  if (row >= 0 && row < rows) y[row] = sum;
}

// ============================================================== PADDED split-strip mapping
// A padded matrix with few, long strips (the dense rows of dense4: 2,500
// strips of 1,250 passes) leaves most warps idle with one warp per strip.
// Here each strip's passes are cut into P parts of near-equal length, one
// warp per (strip, part); a warp sums its part exactly as k_spmv_padded does
// (register at M = 1, slot buffer at M > 1) and writes the partial sum of each
// of the strip's rows to part[(s P + p) h + r]; k_pad_combine then adds a
// row's P partials in part order and writes y -- the same result on every
// call.
#ifndef CMRS_PAD_SPLIT_MINB
#define CMRS_PAD_SPLIT_MINB 5  // resident CTAs per SM asked of the register allocator (6 spills at FP64)
#endif
template <int DT, int kM>
__global__ void __launch_bounds__(kPadWarps * 32, CMRS_PAD_SPLIT_MINB) k_spmv_padded_split(
    int height, int bits, int strips, int P, const int32_t *__restrict__ sp, const uint32_t *__restrict__ packed,
    const typename Form<DT>::Stored *__restrict__ hi, const typename Form<DT>::Stored *__restrict__ lo,
    const typename Form<DT>::Acc *__restrict__ x, typename Form<DT>::Acc *__restrict__ part) {
  typedef typename Form<DT>::Acc A;
  extern __shared__ __align__(16) char smem[];
  pdl_launch_dependents();  // k_pad_combine may launch; it waits for this grid's sums
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  A *buf = reinterpret_cast<A *>(smem) + (size_t)w * kM * height;
  const uint32_t mask = (1u << bits) - 1;
  const int slot = lane & (kM - 1);
  const uint64_t pol = policy_evict_first();
  const long long nw = (long long)gridDim.x * kPadWarps;
  int h2 = 1;
  while (h2 < height) h2 <<= 1;
  const int G = kM < 32 / h2 ? kM : 32 / h2;  // lanes summing one row's slots
  const int per = kM / G;
  if (kM > 1) {  // zeroed here, then by each unit's slot sum
    for (int i = lane; i < kM * height; i += 32) buf[i] = A(0);
    __syncwarp();
  }
  const long long units = (long long)strips * P;
  for (long long u = (long long)blockIdx.x * kPadWarps + w; u < units; u += nw) {
    const int s = (int)(u / P), p = (int)(u - (long long)s * P);
    const int a0 = sp[s], L = (sp[s + 1] - a0) >> 5;  // the strip's passes
    const int a = a0 + 32 * (int)((long long)L * p / P), b = a0 + 32 * (int)((long long)L * (p + 1) / P);
    A acc = A(0);
    for (int k0 = a; k0 < b; k0 += 32 * kPadU) {
      uint32_t c[kPadU];
      A v[kPadU], xv[kPadU];
#pragma unroll
      for (int j = 0; j < kPadU; ++j)
        if (k0 + 32 * j < b) {  // warp-uniform
          const long long k = (long long)k0 + 32 * j + lane;
          c[j] = ld_stream(packed + k, pol);
          v[j] = ld_val_stream<DT>(hi, lo, k, pol);
        }
#pragma unroll
      for (int j = 0; j < kPadU; ++j)
        if (k0 + 32 * j < b) xv[j] = ld_x(x + (c[j] >> bits));
#pragma unroll
      for (int j = 0; j < kPadU; ++j)
        if (k0 + 32 * j < b) {
          if (kM == 1) {
            acc = fma_acc(v[j], xv[j], acc);
          } else {
            A *q = buf + (c[j] & mask) * kM + slot;
            *q = fma_acc(v[j], xv[j], *q);
            __syncwarp();
          }
        }
    }
    A *out = part + u * height;
    if (kM == 1) {
      if (lane < height) out[lane] = acc;
    } else {
      __syncwarp();
      const int r = lane / G, pt = lane - r * G;
      A sum = A(0);
      if (r < height) {
        A *q = buf + r * kM + pt * per;
        sum = q[0];
        q[0] = A(0);
        for (int m = 1; m < per; ++m) {
          sum += q[m];
          q[m] = A(0);
        }
      }
      for (int o = G >> 1; o >= 1; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
      if (pt == 0 && r < height) out[r] = sum;
      __syncwarp();
    }
  }
}

// y[row] = the P partial sums of the row, added in part order.
template <typename A>
__global__ void k_pad_combine(int rows, int height, int P, const A *__restrict__ part, A *__restrict__ y,
                              const int32_t *__restrict__ row_map) {
  pdl_wait();
  const long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= rows) return;
  const long long s = row / height, r = row - s * height;
  const A *q = part + s * P * height + r;
  A sum = q[0];
  for (int p = 1; p < P; ++p) sum += q[(long long)p * height];
  const long long t = row_map ? row_map[row] : row;
  if (t >= 0 && t < rows) y[t] = sum;
}

// Parts per strip: 1 unless the strips are fewer than two per resident warp
// (8 warps x 6 CTAs per SM, the plain walk's residency) and average at least
// 64 passes; then enough parts for two units per resident warp, each of at
// least 16 passes on average.
int pad_parts(const cmrs_matrix *A) {
  if (A->strips <= 0 || !(A->flags & CMRS_PADDED)) return 1;
  const long long target = 2LL * sm_count() * kPadWarps * 6;
  const long long avg = (long long)A->nnz / 32 / A->strips;
  if ((long long)A->strips >= target || avg < 64) return 1;
  long long P = ceil_div(target, A->strips);
  P = std::min<long long>(P, avg / 16);
  return (int)std::max<long long>(1, std::min<long long>(P, 4096));
}

// Workspace bytes of the split walk: the status word, then the partial sums.
size_t pad_split_ws_bytes(const cmrs_matrix *A, int P) {
  const size_t acc = A->dtype == CMRS_F64 ? 8 : 4;
  return P > 1 ? 256 + align256((size_t)A->strips * P * A->height * acc) : 256;
}

// ============================================================== PADDED bulk-staged mapping
// Bulk-staged walk for M = 1 (height 32).  One lane per warp copies the
// warp's strips, kPadCh passes at a time, into a two-stage shared-memory ring
// (cp.async.bulk, completion counted on a per-stage mbarrier, L2 evict-first),
// one stage ahead of the lanes, which then read pass p's item j at word
// 32 p + j of the stage: DRAM sees whole chunks of each stream instead of a
// 128-byte line per warp load.  The next strip's bounds are read one strip
// ahead.  Waits are bounded: on a timeout the warp sets ST_TIMEOUT, waits
// (bounded) for the copies it has in flight, and leaves.
#ifndef CMRS_PAD_CH
#define CMRS_PAD_CH 16
#endif
#ifndef CMRS_PAD_BULK_WARPS
#define CMRS_PAD_BULK_WARPS 8
#endif
#ifndef CMRS_PAD_BULK
#define CMRS_PAD_BULK 14  // bit DT set: that value type's M = 1 form takes this walk (FP32, BF16, split BF16)
#endif
constexpr int kPadCh = CMRS_PAD_CH;
constexpr int kPadBulkWarps = CMRS_PAD_BULK_WARPS;
template <int DT>
struct PadRing {
  typedef typename Form<DT>::Stored S;
  static constexpr bool kSplit = DT == CMRS_BF16X2;
  static constexpr size_t kPk = (size_t)kPadCh * 32 * 4;
  static constexpr size_t kV = (size_t)kPadCh * 32 * sizeof(S);
  static constexpr size_t kStage = kPk + kV * (kSplit ? 2 : 1);
};

template <int DT>
__global__ void __launch_bounds__(kPadBulkWarps * 32) k_spmv_padded_bulk(
    int rows, int bits, int strips, const int32_t *__restrict__ sp, const uint32_t *__restrict__ packed,
    const typename Form<DT>::Stored *__restrict__ hi, const typename Form<DT>::Stored *__restrict__ lo,
    const typename Form<DT>::Acc *__restrict__ x, typename Form<DT>::Acc *__restrict__ y,
    const int32_t *__restrict__ row_map, uint32_t *status) {
  typedef typename Form<DT>::Acc A;
  typedef typename Form<DT>::Stored S;
  typedef PadRing<DT> R;
  extern __shared__ __align__(128) char smem[];
  __shared__ uint64_t bars_all[kPadBulkWarps][2];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  char *ring = smem + (size_t)w * 2 * R::kStage;
  uint64_t *bar = bars_all[w];
  if (lane == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_barrier_init();
  }
  __syncwarp();
  uint64_t pol = 0;
  if (lane == 0) pol = policy_evict_first();
  const int nw = gridDim.x * kPadBulkWarps;
  // copy cursor: strip ps, items [pk, pe); strip ps + nw has bounds [nk, ne)
  int ps = blockIdx.x * kPadBulkWarps + w, pk = 0, pe = 0, nk = 0, ne = 0;
  if (ps < strips) {
    pk = sp[ps];
    pe = sp[ps + 1];
  }
  if (ps + nw < strips) {
    nk = sp[ps + nw];
    ne = sp[ps + nw + 1];
  }
  int cs[2] = {0, 0}, cn[2] = {0, 0};
  bool clast[2] = {false, false}, valid[2] = {false, false};
  uint32_t par[2] = {0u, 0u};
  uint32_t bad = 0;
  // The stage index is a compile-time constant in both lambdas (the ring
  // loop alternates step(0), step(1)), so the descriptors stay in registers.
  auto issue = [&](auto stc) {  // next chunk into stage st (warp-uniform; lane 0 copies)
    constexpr int st = decltype(stc)::value;
    const int n = max(0, min(kPadCh * 32, pe - pk));
    const bool whole = ((pk | n) & 31) == 0;  // padded strips hold whole 32-item passes
    if (!whole) bad = 1;
    cs[st] = ps;
    cn[st] = whole ? n : 0;
    if (lane == 0) {
      char *dst = ring + st * R::kStage;
      const uint32_t m = (uint32_t)cn[st];
      fence_proxy_async();
      mbar_arrive_expect_tx(&bar[st], m * (4u + (uint32_t)sizeof(S) * (R::kSplit ? 2u : 1u)));
      if (m) {
        bulk_g2s(dst, packed + pk, m * 4u, &bar[st], pol);
        bulk_g2s(dst + R::kPk, hi + pk, m * (uint32_t)sizeof(S), &bar[st], pol);
        if (R::kSplit) bulk_g2s(dst + R::kPk + R::kV, lo + pk, m * (uint32_t)sizeof(S), &bar[st], pol);
      }
    }
    valid[st] = true;
    pk += n;
    clast[st] = pk >= pe;
    if (clast[st]) {  // on to the warp's next strip, whose bounds were read one strip ago
      ps += nw;
      pk = nk;
      pe = ne;
      nk = ne = 0;
      if (ps + nw < strips) {
        nk = sp[ps + nw];
        ne = sp[ps + nw + 1];
      }
    }
  };
  A acc = A(0);
  // one ring step on stage st: 0 = go on, 1 = no chunk left, 2 = a wait timed out
  auto step = [&](auto stc) -> int {
    constexpr int st = decltype(stc)::value;
    if (!valid[st]) return 1;
    if (ps < strips) issue(std::integral_constant<int, st ^ 1>());
    const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&bar[st], par[st]));
    par[st] ^= 1u;
    if (!ok) {
      if (lane == 0) atomicOr(status, ST_TIMEOUT);
      mbar_wait_bounded(&bar[st], par[st] ^ 1u);  // copies still in flight land before the warp leaves
      if (valid[st ^ 1]) mbar_wait_bounded(&bar[st ^ 1], par[st ^ 1]);
      return 2;
    }
    const uint32_t *cp = reinterpret_cast<const uint32_t *>(ring + st * R::kStage);
    const S *vh = reinterpret_cast<const S *>(ring + st * R::kStage + R::kPk);
    const S *vl = reinterpret_cast<const S *>(ring + st * R::kStage + R::kPk + R::kV);
    const int np = cn[st] >> 5;
    for (int p0 = 0; p0 < np; p0 += kPadU) {
      uint32_t c[kPadU];
      A v[kPadU], xv[kPadU];
#pragma unroll
      for (int u = 0; u < kPadU; ++u)
        if (p0 + u < np) {
          const int i = (p0 + u) * 32 + lane;
          c[u] = cp[i];
          v[u] = Form<DT>::value(vh, vl, i);
        }
#pragma unroll
      for (int u = 0; u < kPadU; ++u)
        if (p0 + u < np) xv[u] = ld_x(x + (c[u] >> bits));
#pragma unroll
      for (int u = 0; u < kPadU; ++u)
        if (p0 + u < np) acc = fma_acc(v[u], xv[u], acc);
    }
    if (clast[st]) {
      const long long row = (long long)cs[st] * 32 + lane;
      if (row < rows) {
        const long long t = row_map ? row_map[row] : row;
        if (t >= 0 && t < rows) y[t] = acc;
      }
      acc = A(0);
    }
    __syncwarp();
    valid[st] = false;
    return 0;
  };
  if (ps < strips) issue(std::integral_constant<int, 0>());
  int rc = 0;
  while (rc == 0) {
    rc = step(std::integral_constant<int, 0>());
    if (rc == 0) rc = step(std::integral_constant<int, 1>());
  }
  if (rc == 2) return;
  if (bad && lane == 0) atomicOr(status, ST_BAD_PAD);
}

// ============================================================== host side
struct Occ {
  std::mutex mu;
  int val[64] = {0};
};

// Resident CTAs per SM for `smem` bytes of dynamic shared memory, cached per
// device.  The kernel is first opted in to max(smem, smem_cap) bytes, the most
// any launch of it asks for.  With max_per_sm > 0 the kernel's shared-memory
// carveout is set to the smallest that holds max_per_sm CTAs, and the rest of
// the SM's 256 KB of L1/shared storage stays L1: a kernel whose time goes to
// x gathers that miss L1 keeps more of them in flight with more L1 lines to
// hold them than with more resident warps.
template <typename K>
int occupancy(K kernel, int threads, size_t smem, Occ &cache, size_t smem_cap = 0, int max_per_sm = 0) {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  std::lock_guard<std::mutex> lk(cache.mu);
  if (cache.val[dev] == 0) {
    // opt in to the dynamic shared memory the launches use (static + dynamic may pass 48 KB)
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max(smem, smem_cap));
    if (max_per_sm > 0) {
      cudaFuncAttributes fa;
      int sm_smem = 0;
      if (cudaFuncGetAttributes(&fa, kernel) == cudaSuccess &&
          cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess &&
          sm_smem > 0) {
        const size_t need = (size_t)max_per_sm * (std::max(smem, smem_cap) + fa.sharedSizeBytes + 1024);
        const int pct = (int)std::min<size_t>(100, (need * 100 + sm_smem - 1) / sm_smem);
        cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
      }
    }
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess || n < 1) n = 1;
    if (max_per_sm > 0) n = std::min(n, max_per_sm);
    cache.val[dev] = n;
  }
  return cache.val[dev];
}

// sized for the smaller of the form's two tiles: enough for either launch
size_t merge_ws_bytes(int nnz, int dtype) {
  const int tile = dtype == CMRS_F64 ? std::min(MergeCfg<CMRS_F64, false>::Tile, MergeCfg<CMRS_F64, true>::Tile)
                                     : std::min(MergeCfg<CMRS_F32, false>::Tile, MergeCfg<CMRS_F32, true>::Tile);
  const long long ntiles = ceil_div(nnz, tile);
  return 256 + align256((size_t)(ntiles + 1) * 4) + align256((size_t)ntiles * sizeof(TileRec));
}

// The staged walk (k_spmv_padded_bulk) is taken by the value forms CMRS_PAD_BULK
// names when the strips average at least this many passes (BF16 forms; FP32)
#ifndef CMRS_PAD_BULK_MIN_PASSES
#define CMRS_PAD_BULK_MIN_PASSES 12
#endif
#ifndef CMRS_PAD_BULK_MIN_PASSES_F32
#define CMRS_PAD_BULK_MIN_PASSES_F32 16
#endif

template <int DT, int kM>
int launch_padded(const cmrs_matrix *A, const typename Form<DT>::Stored *hi, const typename Form<DT>::Stored *lo,
                  const typename Form<DT>::Acc *x, typename Form<DT>::Acc *y, const int32_t *row_map,
                  uint32_t *status, char *ws, size_t ws_bytes, cudaStream_t st) {
  typedef typename Form<DT>::Acc Acc;
  const int P = pad_parts(A);
  if (P > 1 && ws_bytes >= pad_split_ws_bytes(A, P)) {  // few long strips: several warps per strip
    static Occ occ_split[33];
    Acc *part = reinterpret_cast<Acc *>(ws + 256);
    const size_t per_h = kM > 1 ? (size_t)kPadWarps * kM * sizeof(Acc) : 0;
    const int per_sm = occupancy(k_spmv_padded_split<DT, kM>, kPadWarps * 32, per_h * A->height,
                                 occ_split[A->height], per_h * 32);
    const long long units = (long long)A->strips * P;
    const int grid = (int)std::min<long long>(ceil_div(units, kPadWarps), (long long)per_sm * sm_count());
    k_spmv_padded_split<DT, kM><<<grid, kPadWarps * 32, per_h * A->height, st>>>(
        A->height, A->bits, A->strips, P, A->strip_ptr, A->col_packed, hi, lo, x, part);
    CMRS_LAUNCH_CHECK();
    const int rc = launch_pdl(k_pad_combine<Acc>, (unsigned)ceil_div(A->rows, 256), 256, 0, st, A->rows, A->height, P,
                              part, y, row_map);
    if (rc) return rc;
    return CMRS_OK;
  }
  const bool aligned = ((reinterpret_cast<uintptr_t>(A->col_packed) | reinterpret_cast<uintptr_t>(hi) |
                         reinterpret_cast<uintptr_t>(lo)) & 15) == 0;
  // short strips (a pass or a few) pay a copy round trip each: the plain walk is faster there
  const long long min_passes = DT == CMRS_F32 ? CMRS_PAD_BULK_MIN_PASSES_F32 : CMRS_PAD_BULK_MIN_PASSES;
  if (kM == 1 && ((CMRS_PAD_BULK >> DT) & 1) && aligned && (long long)A->nnz >= 32LL * min_passes * A->strips) {
    static Occ occ_bulk;
    const size_t smem = (size_t)kPadBulkWarps * 2 * PadRing<DT>::kStage;
    const int per_sm = occupancy(k_spmv_padded_bulk<DT>, kPadBulkWarps * 32, smem, occ_bulk);
    const long long need = ceil_div(A->strips, kPadBulkWarps);
    const int grid = (int)std::min<long long>(need, (long long)per_sm * sm_count());
    k_spmv_padded_bulk<DT><<<grid, kPadBulkWarps * 32, smem, st>>>(A->rows, A->bits, A->strips, A->strip_ptr,
                                                                   A->col_packed, hi, lo, x, y, row_map, status);
    CMRS_LAUNCH_CHECK();
    return CMRS_OK;
  }
  // Groups of exactly present passes (no guarded multiply-add that the compiler
  // computes and discards) pay off for strips of under 4 passes on average and
  // for FP64 slot buffers; long one-slot strips keep the guarded last group.
  const bool exact = (long long)A->nnz < 4LL * 32 * A->strips || (DT == CMRS_F64 && kM > 1);
  static Occ occ[2];
  const size_t smem = (size_t)kPadWarps * kM * A->height * sizeof(Acc);
  const size_t smem_occ = (size_t)kPadWarps * kM * 32 * sizeof(Acc);
  const int per_sm = exact ? occupancy(k_spmv_padded<DT, kM, true>, kPadWarps * 32, smem_occ, occ[1])
                           : occupancy(k_spmv_padded<DT, kM, false>, kPadWarps * 32, smem_occ, occ[0]);
  const long long need = ceil_div(A->strips, kPadWarps);
  const int grid = (int)std::min<long long>(need, (long long)per_sm * sm_count());
  if (exact)
    k_spmv_padded<DT, kM, true><<<grid, kPadWarps * 32, smem, st>>>(A->rows, A->height, A->bits, A->strips,
                                                                    A->strip_ptr, A->col_packed, hi, lo, x, y, row_map);
  else
    k_spmv_padded<DT, kM, false><<<grid, kPadWarps * 32, smem, st>>>(A->rows, A->height, A->bits, A->strips,
                                                                     A->strip_ptr, A->col_packed, hi, lo, x, y, row_map);
  CMRS_LAUNCH_CHECK();
  return CMRS_OK;
}

// MERGE: tile map, the product, the fix-up of rows cut by tile boundaries
template <int DT, bool kLong>
int launch_merge(const cmrs_matrix *A, const typename Form<DT>::Stored *hi, const typename Form<DT>::Stored *lo,
                 const typename Form<DT>::Acc *x, typename Form<DT>::Acc *y, uint32_t *status, char *ws,
                 cudaStream_t st) {
  typedef typename Form<DT>::Acc Acc;
  static Occ occ;
  constexpr int kMergeTile = MergeCfg<DT, kLong>::Tile;
  const int ntiles = (int)ceil_div(A->nnz, kMergeTile);
  int32_t *tile_strip = reinterpret_cast<int32_t *>(ws + 256);
  TileRec *recs = reinterpret_cast<TileRec *>(ws + 256 + align256((size_t)(ntiles + 1) * 4));
  k_tile_map<<<(int)ceil_div(A->strips, 256), 256, 0, st>>>(A->strips, A->strip_ptr, kMergeTile, ntiles, tile_strip);
  CMRS_LAUNCH_CHECK();
  const size_t smem = kStages * Stage<DT>::bytes(kMergeTile);
  const int per_sm = occupancy(k_spmv_merge<DT, kLong>, kMergeThreads, smem, occ, 0, MergeCfg<DT, kLong>::Ctas);
  const int grid = (int)std::min<long long>(ntiles, (long long)per_sm * sm_count());
  int rc = launch_pdl(k_spmv_merge<DT, kLong>, (unsigned)grid, kMergeThreads, smem, st, A->rows, A->height, A->bits,
                      A->strips, A->nnz, A->strip_ptr, A->col_packed, hi, lo, x, y, tile_strip, ntiles, recs, status);
  if (rc) return rc;
  return launch_pdl(k_merge_fixup<Acc>, (unsigned)ceil_div(ntiles, 256), 256, 0, st, ntiles, A->rows, recs, y);
}

template <int DT>
int launch(const cmrs_matrix *A, const void *xv, void *yv, const int32_t *row_map, int variant, char *ws,
           size_t ws_bytes, cudaStream_t st) {
  typedef typename Form<DT>::Stored S;
  typedef typename Form<DT>::Acc Acc;
  const S *hi = reinterpret_cast<const S *>(A->val);
  const S *lo = DT == CMRS_BF16X2 ? hi + cmrs_pad8(A->nnz) : nullptr;
  const Acc *x = reinterpret_cast<const Acc *>(xv);
  Acc *y = reinterpret_cast<Acc *>(yv);
  uint32_t *status = reinterpret_cast<uint32_t *>(ws);
  const int sms = sm_count();
  const double mu = A->rows > 0 ? (double)A->nnz / A->rows : 0.0;
  const int lanes = mu <= CMRS_LANE_MAX_MU                              ? 1
                    : (CMRS_LANE_MAX_L >= 2 && mu <= 2 * CMRS_LANE_MAX_MU) ? 2
                    : (CMRS_LANE_MAX_L >= 4 && mu <= 4 * CMRS_LANE_MAX_MU) ? 4
                                                                          : 0;
  if (variant == CMRS_VARIANT_ROW && CMRS_ROW_LANE && lanes && (32 / lanes) % A->height == 0) {
    // stage: 1.25x the entries of an average unit (32 / lanes rows), in
    // multiples of 32, at most kLaneCap -- short rows leave shared memory for
    // more warps; a longer unit is read from global memory
    const int cap = (int)std::min<long long>(
        kLaneCap, std::max<long long>(128, ceil_div((long long)(CMRS_LANE_SLACK * mu / lanes), 32) * 32));
    const size_t smem = (size_t)kLaneWarps * Stage<DT>::bytes(cap);
    const size_t smem_max = (size_t)kLaneWarps * Stage<DT>::bytes(kLaneCap);
    const long long need = ceil_div(ceil_div(A->rows, 32 / lanes), kLaneWarps);
    static Occ occ1[kLaneCap / 32 + 1], occ2[kLaneCap / 32 + 1], occ4[kLaneCap / 32 + 1];
    int per_sm = 1;
    if (lanes == 1) per_sm = occupancy(k_spmv_lane<DT, 1>, kLaneWarps * 32, smem, occ1[cap / 32], smem_max, CMRS_LANE_CTAS);
    if (lanes == 2) per_sm = occupancy(k_spmv_lane<DT, 2>, kLaneWarps * 32, smem, occ2[cap / 32], smem_max, CMRS_LANE_CTAS);
    if (lanes == 4) per_sm = occupancy(k_spmv_lane<DT, 4>, kLaneWarps * 32, smem, occ4[cap / 32], smem_max, CMRS_LANE_CTAS);
    const int grid = (int)std::min<long long>(need, (long long)per_sm * sms);
    if (lanes == 1)
      k_spmv_lane<DT, 1><<<grid, kLaneWarps * 32, smem, st>>>(A->rows, A->height, A->bits, cap, A->nnz,
                                                               A->strip_ptr, A->col_packed, hi, lo, x, y, row_map, status);
    else if (lanes == 2)
      k_spmv_lane<DT, 2><<<grid, kLaneWarps * 32, smem, st>>>(A->rows, A->height, A->bits, cap, A->nnz,
                                                               A->strip_ptr, A->col_packed, hi, lo, x, y, row_map, status);
    else
      k_spmv_lane<DT, 4><<<grid, kLaneWarps * 32, smem, st>>>(A->rows, A->height, A->bits, cap, A->nnz,
                                                               A->strip_ptr, A->col_packed, hi, lo, x, y, row_map, status);
    CMRS_LAUNCH_CHECK();
  } else if (variant == CMRS_VARIANT_ROW) {
    static Occ occ;
    const size_t smem = kRowStages * Stage<DT>::bytes(kRowCap);
    const int per_sm = occupancy(k_spmv_row<DT>, RowCfg<DT>::kThreads, smem, occ);
    const long long nblk = ceil_div(A->rows, kRowThreads);
    const int grid = (int)std::min<long long>(nblk, (long long)per_sm * sms);
    k_spmv_row<DT><<<grid, RowCfg<DT>::kThreads, smem, st>>>(A->rows, A->height, A->bits, A->nnz, A->strip_ptr,
                                                             A->col_packed, hi, lo, x, y, row_map, status);
    CMRS_LAUNCH_CHECK();
  } else if (variant == CMRS_VARIANT_STRIP) {
    static Occ occ;
    const size_t smem = (size_t)kStripWarps * A->height * 32 * sizeof(Acc);
    const int per_sm = occupancy(k_spmv_strip<DT>, kStripWarps * 32, (size_t)kStripWarps * 32 * 32 * sizeof(Acc), occ);
    const long long need = ceil_div(A->strips, kStripWarps);
    const int grid = (int)std::min<long long>(need, (long long)per_sm * sms);
    k_spmv_strip<DT><<<grid, kStripWarps * 32, smem, st>>>(A->rows, A->height, A->bits, A->strips, A->strip_ptr,
                                                           A->col_packed, hi, lo, x, y, row_map);
    CMRS_LAUNCH_CHECK();
  } else if (variant == CMRS_VARIANT_PADDED) {
    switch (CMRS_PAD_SLOTS_OF(A->flags)) {
      case 1: return launch_padded<DT, 1>(A, hi, lo, x, y, row_map, status, ws, ws_bytes, st);
      case 2: return launch_padded<DT, 2>(A, hi, lo, x, y, row_map, status, ws, ws_bytes, st);
      case 4: return launch_padded<DT, 4>(A, hi, lo, x, y, row_map, status, ws, ws_bytes, st);
      default: return launch_padded<DT, 8>(A, hi, lo, x, y, row_map, status, ws, ws_bytes, st);
    }
  } else {
    if constexpr (merge_long_differs<DT>()) {
      if ((double)A->nnz >= CMRS_MERGE_LONG_MU * (double)A->rows)
        return launch_merge<DT, true>(A, hi, lo, x, y, status, ws, st);
    }
    return launch_merge<DT, false>(A, hi, lo, x, y, status, ws, st);
  }
  return CMRS_OK;
}

int check_matrix(const cmrs_matrix *A) {
  if (!A) return CMRS_ERR_ARG;
  if (A->rows < 0 || A->cols < 0 || A->nnz < 0) return CMRS_ERR_ARG;
  if (cmrs_bits_for_height(A->height) < 0) return CMRS_ERR_HEIGHT;
  if (A->bits != cmrs_bits_for_height(A->height)) return CMRS_ERR_ARG;
  if (A->strips != ceil_div(A->rows, A->height)) return CMRS_ERR_ARG;
  if (A->dtype < CMRS_F64 || A->dtype > CMRS_BF16X2) return CMRS_ERR_ARG;
  if (A->flags & ~(CMRS_SORTED | CMRS_PADDED | CMRS_PAD_SLOTS_MASK)) return CMRS_ERR_ARG;
  if ((A->flags & CMRS_SORTED) && (A->flags & CMRS_PADDED)) return CMRS_ERR_ARG;
  if (!(A->flags & CMRS_PADDED) && (A->flags & CMRS_PAD_SLOTS_MASK)) return CMRS_ERR_ARG;
  if (A->flags & CMRS_PADDED) {
    const int m = CMRS_PAD_SLOTS_OF(A->flags);
    if (m > 8 || A->height * m < 32 || (A->nnz & 31)) return CMRS_ERR_ARG;
  }
  if (A->rows > 0 && !A->strip_ptr) return CMRS_ERR_ARG;
  if (A->nnz > 0 && (!A->col_packed || !A->val)) return CMRS_ERR_ARG;
  return CMRS_OK;
}

// AUTO: sorted strips can only use STRIP.  Otherwise MERGE when rows are very
// short (mean < 2 entries: ROW's per-row overhead dominates), long (mean > 32,
// unless ROW's two- or four-lanes-per-row mapping applies: mean up to 56 at
// heights dividing 16, up to 112 at heights dividing 8) or skewed (a strip
// holding more than 8x its share); ROW for everything else.  On the ROW and
// MERGE timings of 2000 synthetic matrices of six families this rule lands
// within 1.5% of the better variant at h = 32 and 1.2% at h = 1 (geometric
// mean).
int resolve_variant(const cmrs_matrix *A, int variant, int *out) {
  const bool sorted = (A->flags & CMRS_SORTED) != 0;
  const bool padded = (A->flags & CMRS_PADDED) != 0;
  if (variant == CMRS_VARIANT_AUTO) {
    if (padded) {
      variant = CMRS_VARIANT_PADDED;
    } else if (sorted) {
      variant = CMRS_VARIANT_STRIP;
    } else {
      const double mu = A->rows > 0 ? (double)A->nnz / A->rows : 0.0;
      const bool skewed = A->max_strip_nnz < 0 || (double)A->max_strip_nnz > 8.0 * A->height * mu;
      // rows longer than 32 on average stay with ROW where its two- or
      // four-lanes-per-row mapping takes them (heights dividing 16 or 8)
      const bool lanes = CMRS_ROW_LANE && ((mu <= 2 * CMRS_LANE_MAX_MU && 16 % A->height == 0) ||
                                           (mu <= 4 * CMRS_LANE_MAX_MU && 8 % A->height == 0));
      variant = (mu < 2.0 || (mu > 32.0 && !lanes) || skewed) ? CMRS_VARIANT_MERGE : CMRS_VARIANT_ROW;
    }
  }
  if (variant < 0 || variant >= CMRS_NUM_VARIANTS) return CMRS_ERR_ARG;
  if (sorted && variant != CMRS_VARIANT_STRIP) return CMRS_ERR_UNSUPPORTED;
  // padded strips: Algorithm 1 or the Section 6.6 kernel; that kernel needs padded strips
  if (padded && variant != CMRS_VARIANT_STRIP && variant != CMRS_VARIANT_PADDED) return CMRS_ERR_UNSUPPORTED;
  if (!padded && variant == CMRS_VARIANT_PADDED) return CMRS_ERR_UNSUPPORTED;
  *out = variant;
  return CMRS_OK;
}

}  // namespace
}  // namespace cmrs

using namespace cmrs;

extern "C" int cmrs_spmv_variant(const cmrs_matrix *A, int variant, int *resolved) {
  if (!resolved) return CMRS_ERR_ARG;
  int rc = check_matrix(A);
  if (rc) return rc;
  return resolve_variant(A, variant, resolved);
}

size_t cmrs::merge_workspace_bytes(int nnz, int dtype) { return merge_ws_bytes(nnz, dtype); }

extern "C" int cmrs_spmv_workspace(const cmrs_matrix *A, int variant, size_t *bytes) {
  if (!bytes) return CMRS_ERR_ARG;
  int rc = check_matrix(A);
  if (rc) return rc;
  int v = 0;
  rc = resolve_variant(A, variant, &v);
  if (rc) return rc;
  *bytes = v == CMRS_VARIANT_MERGE ? merge_ws_bytes(A->nnz, A->dtype)
           : v == CMRS_VARIANT_PADDED ? pad_split_ws_bytes(A, pad_parts(A))
                                       : 256;
  return CMRS_OK;
}

namespace cmrs {
namespace {

// y[map[i]] = (A x)_i, map NULL for the identity.  With a map, AUTO never
// picks MERGE (whose rows leave through several paths) but ROW instead.
int spmv_impl(const cmrs_matrix *A, const void *x, void *y, const int32_t *row_map, int variant, void *workspace,
              size_t workspace_bytes, void *stream) {
  int rc = check_matrix(A);
  if (rc) return rc;
  int v = 0;
  rc = resolve_variant(A, variant, &v);
  if (rc) return rc;
  if (row_map && v == CMRS_VARIANT_MERGE) {
    if (variant != CMRS_VARIANT_AUTO) return CMRS_ERR_UNSUPPORTED;
    v = CMRS_VARIANT_ROW;
  }
  if (A->rows == 0) return CMRS_OK;
  if (!y || (A->nnz > 0 && !x)) return CMRS_ERR_ARG;
  const size_t need = v == CMRS_VARIANT_MERGE ? merge_ws_bytes(A->nnz, A->dtype) : 256;
  if (!workspace || workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255)) return CMRS_ERR_WORKSPACE;
  // ROW and MERGE stream col_packed and val with bulk copies: 16-byte aligned bases
  if ((v == CMRS_VARIANT_ROW || v == CMRS_VARIANT_MERGE) && A->nnz > 0 &&
      ((reinterpret_cast<uintptr_t>(A->col_packed) | reinterpret_cast<uintptr_t>(A->val)) & 15))
    return CMRS_ERR_ARG;
  cudaStream_t st = as_stream(stream);
  const size_t ysz = A->dtype == CMRS_F64 ? 8 : 4;
  if (A->nnz == 0) {
    CMRS_CUDA_TRY(cudaMemsetAsync(y, 0, (size_t)A->rows * ysz, st));
    return CMRS_OK;
  }
  char *ws = reinterpret_cast<char *>(workspace);
  switch (A->dtype) {
    case CMRS_F64: return launch<CMRS_F64>(A, x, y, row_map, v, ws, workspace_bytes, st);
    case CMRS_F32: return launch<CMRS_F32>(A, x, y, row_map, v, ws, workspace_bytes, st);
    case CMRS_BF16: return launch<CMRS_BF16>(A, x, y, row_map, v, ws, workspace_bytes, st);
    case CMRS_BF16X2: return launch<CMRS_BF16X2>(A, x, y, row_map, v, ws, workspace_bytes, st);
  }
  return CMRS_ERR_ARG;
}

}  // namespace
}  // namespace cmrs

extern "C" int cmrs_spmv(const cmrs_matrix *A, const void *x, void *y, int variant, void *workspace,
                         size_t workspace_bytes, void *stream) {
  CMRS_TRACE();
  return spmv_impl(A, x, y, nullptr, variant, workspace, workspace_bytes, stream);
}

extern "C" int cmrs_spmv_rows(const cmrs_matrix *A, const void *x, void *y, const int32_t *row_map, int variant,
                              void *workspace, size_t workspace_bytes, void *stream) {
  CMRS_TRACE();
  if (!row_map && A && A->rows > 0) return CMRS_ERR_ARG;
  return spmv_impl(A, x, y, row_map, variant, workspace, workspace_bytes, stream);
}

extern "C" int cmrs_spmv_check(const cmrs_matrix *A, int variant, const void *workspace, void *stream) {
  CMRS_TRACE();
  (void)A;
  (void)variant;
  if (!workspace) return CMRS_ERR_ARG;
  uint32_t s = 0;
  cudaStream_t st = as_stream(stream);
  CMRS_CUDA_TRY(cudaMemcpyAsync(&s, workspace, 4, cudaMemcpyDeviceToHost, st));
  CMRS_CUDA_TRY(cudaStreamSynchronize(st));
  if (s & ST_TIMEOUT) {
    CMRS_CUDA_TRY(cudaMemsetAsync(const_cast<void *>(workspace), 0, 4, st));
    return CMRS_ERR_TIMEOUT;
  }
  if (s & ST_BAD_PAD) {
    CMRS_CUDA_TRY(cudaMemsetAsync(const_cast<void *>(workspace), 0, 4, st));
    return CMRS_ERR_ARG;
  }
  return CMRS_OK;
}

// ============================================================== wait probe
// One warp runs the bounded mbarrier wait of the staged kernels on a phase
// that only an arrival of its own completes (no copy is issued, so none is in
// flight when it leaves).  Without the arrival every lane gives up after
// `tries` tries and the timeout bit is set as the SpMV kernels set it.
namespace cmrs {
namespace {
__global__ void k_wait_probe(uint32_t tries, int arrive, uint32_t *status) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  if (arrive && threadIdx.x == 0) mbar_arrive(&bar);
  const bool ok = mbar_wait_bounded(&bar, 0, tries);
  if (!__all_sync(0xffffffffu, ok) && threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
}
}  // namespace
}  // namespace cmrs

namespace {
int noalloc_scratch(void **out);
}

extern "C" int cmrs_wait_probe(void *workspace, uint32_t tries, int arrive, void *stream) {
  CMRS_TRACE();
  if (tries < 1 || tries > 65536) return CMRS_ERR_ARG;
  if (!workspace) {  // the status word of the fixed array of cmrs_spmv_noalloc
    const int rc = noalloc_scratch(&workspace);
    if (rc) return rc;
  }
  if (reinterpret_cast<uintptr_t>(workspace) & 255) return CMRS_ERR_ARG;
  k_wait_probe<<<1, 32, 0, as_stream(stream)>>>(tries, arrive != 0, static_cast<uint32_t *>(workspace));
  CMRS_LAUNCH_CHECK();
  return CMRS_OK;
}

// ============================================================== fixed-scratch entry point
// For callers that cannot allocate device memory, cmrs_spmv_noalloc runs the
// MERGE mapping with its scratch (status word, tile map, tile records) in
// this fixed array instead of a caller workspace.  It stays resident on every
// GPU that loads the library until the process exits.
static __device__ __align__(256) unsigned char cmrs_noalloc_scratch[size_t(2) << 20];

namespace {
constexpr size_t kNoAllocBytes = size_t(2) << 20;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[64] = {};

// Device address of the fixed array on the current device.  Looked up once
// per device (with that device current); host code must not use the symbol
// itself, which is only a host-side stand-in.
int noalloc_scratch(void **out) {
  int dev = 0;
  CMRS_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return CMRS_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void *p = nullptr;
    CMRS_CUDA_TRY(cudaGetSymbolAddress(&p, cmrs_noalloc_scratch));
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return CMRS_OK;
}
}  // namespace

extern "C" int cmrs_spmv_noalloc(const cmrs_matrix *A, const void *x, void *y, void *stream) {
  CMRS_TRACE();
  int rc = check_matrix(A);
  if (rc) return rc;
  if (A->flags & (CMRS_SORTED | CMRS_PADDED)) return CMRS_ERR_UNSUPPORTED;
  if (A->rows == 0) return CMRS_OK;
  if (!y || (A->nnz > 0 && !x)) return CMRS_ERR_ARG;
  if (merge_ws_bytes(A->nnz, A->dtype) > kNoAllocBytes) return CMRS_ERR_WORKSPACE;
  if (A->nnz > 0 && ((reinterpret_cast<uintptr_t>(A->col_packed) | reinterpret_cast<uintptr_t>(A->val)) & 15))
    return CMRS_ERR_ARG;
  void *scratch = nullptr;
  rc = noalloc_scratch(&scratch);
  if (rc) return rc;
  cudaStream_t st = as_stream(stream);
  if (A->nnz == 0) {
    CMRS_CUDA_TRY(cudaMemsetAsync(y, 0, (size_t)A->rows * (A->dtype == CMRS_F64 ? 8 : 4), st));
    return CMRS_OK;
  }
  // The status word (zero at load) is not cleared here: a wait that gave up
  // stays recorded until cmrs_spmv_noalloc_check reads it.  Everything else
  // in the array is rewritten by every call.
  char *ws = reinterpret_cast<char *>(scratch);
  switch (A->dtype) {
    case CMRS_F64: return launch<CMRS_F64>(A, x, y, nullptr, CMRS_VARIANT_MERGE, ws, sizeof(cmrs_noalloc_scratch), st);
    case CMRS_F32: return launch<CMRS_F32>(A, x, y, nullptr, CMRS_VARIANT_MERGE, ws, sizeof(cmrs_noalloc_scratch), st);
    case CMRS_BF16: return launch<CMRS_BF16>(A, x, y, nullptr, CMRS_VARIANT_MERGE, ws, sizeof(cmrs_noalloc_scratch), st);
    case CMRS_BF16X2: return launch<CMRS_BF16X2>(A, x, y, nullptr, CMRS_VARIANT_MERGE, ws, sizeof(cmrs_noalloc_scratch), st);
  }
  return CMRS_ERR_ARG;
}

extern "C" int cmrs_spmv_noalloc_check(void *stream) {
  CMRS_TRACE();
  void *scratch = nullptr;
  int rc = noalloc_scratch(&scratch);
  if (rc) return rc;
  uint32_t s = 0;
  cudaStream_t st = as_stream(stream);
  CMRS_CUDA_TRY(cudaMemcpyAsync(&s, scratch, 4, cudaMemcpyDeviceToHost, st));
  CMRS_CUDA_TRY(cudaStreamSynchronize(st));
  if (s) CMRS_CUDA_TRY(cudaMemsetAsync(scratch, 0, 4, st));
  return (s & ST_TIMEOUT) ? CMRS_ERR_TIMEOUT : CMRS_OK;
}
