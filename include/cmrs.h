/*
 * cmrs.h -- C ABI of libcmrs, Compressed Multi-Row Storage (CMRS) sparse
 * matrix-vector products on NVIDIA GB300 (sm_103a).
 *
 * Method: Koza, Matyka, Szkoda, Miroslaw, "Compressed Multi-Row Storage
 * Format for Sparse Matrices on Graphics Processing Units" (arXiv:1203.2946).
 *
 * Conventions for every entry point
 *   - Return value: CMRS_OK (0) or one of the CMRS_ERR_* codes below;
 *     cmrs_error_string() names it.  No C++ exception, abort or exit crosses
 *     this boundary.
 *   - Memory: the caller owns every array.  Pointers documented as "device"
 *     must point to device memory of the current CUDA device (for example
 *     torch tensors); pointers documented as "host" to host memory.  The
 *     library never allocates user-visible arrays and never frees anything it
 *     did not allocate; scratch space ("workspace") is a device buffer the
 *     caller provides, sized by the matching *_workspace query.
 *   - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy
 *     default stream).  Work is enqueued asynchronously on it; an entry point
 *     synchronises only where its comment says so.
 *   - Sizes and indices are int32; rows, cols and nnz must be < 2^31.
 *   - A workspace must not be used by two calls that may run at the same time
 *     (for example on two streams); results are then undefined.
 */
#ifndef CMRS_H
#define CMRS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define CMRS_OK 0
#define CMRS_ERR_ARG 1          /* null pointer, negative size, bad enum, etc. */
#define CMRS_ERR_HEIGHT 2       /* strip height outside 1..32 */
#define CMRS_ERR_COL_OVERFLOW 3 /* cols > 2^(32 - bits): column does not fit the packed word */
#define CMRS_ERR_CSR_INVALID 4  /* RowPtr not a valid CRS row pointer, or a column outside [0, cols) */
#define CMRS_ERR_CUDA 5         /* a CUDA runtime call failed; cmrs_last_cuda_error() has the code */
#define CMRS_ERR_UNSUPPORTED 6  /* valid request this library does not implement (e.g. variant on sorted strips) */
#define CMRS_ERR_WORKSPACE 7    /* workspace pointer null/misaligned or smaller than its query returned */
#define CMRS_ERR_TIMEOUT 8      /* a bounded in-kernel wait gave up; the output is not valid */

/* ---- value storage forms ------------------------------------------------
 * CMRS_F64    double Val[nnz]
 * CMRS_F32    float Val[nnz] (round to nearest even from the input)
 * CMRS_BF16   uint16 Val[nnz]: BF16 = round-to-nearest-even of the FP32 value
 * CMRS_BF16X2 split pair: hi[nnz] = BF16(v) at byte 0, lo[nnz] = BF16(v - hi)
 *             at byte 2 * cmrs_pad8(nnz); the represented value is hi + lo.
 * The paper stores float or double (Section 6.2); the BF16 forms are this
 * library's own and cut the bytes streamed per entry.  SpMV with CMRS_F64
 * takes double x and y and accumulates in double; every other form takes
 * float x and y and accumulates in float. */
#define CMRS_F64 0
#define CMRS_F32 1
#define CMRS_BF16 2
#define CMRS_BF16X2 3

/* ---- flags --------------------------------------------------------------- */
/* Section 4, fourth optimisation: entries of each strip ordered by column
 * (stable: equal columns keep their CRS order). */
#define CMRS_SORTED 1u
/* Section 6.6 ("modified CMRS"): strips rearranged into 32-item warp passes
 * holding at most M items of any one row, stored contiguously, filled with
 * explicit zero items (column 0, value +0); every strip holds a multiple of
 * 32 items.  M (slots) is 1, 2, 4 or 8, kept as log2(M) in flag bits 8..10;
 * the paper's M is 8.  Made by cmrs_pad_layout + cmrs_pad_fill. */
#define CMRS_PADDED 2u
#define CMRS_PAD_SLOTS 8 /* the paper's M */
#define CMRS_PAD_SLOTS_SHIFT 8
#define CMRS_PAD_SLOTS_MASK (7u << CMRS_PAD_SLOTS_SHIFT)
#define CMRS_PAD_SLOTS_OF(flags) (1 << (((flags) & CMRS_PAD_SLOTS_MASK) >> CMRS_PAD_SLOTS_SHIFT))

/* ---- SpMV kernel variants -------------------------------------------------
 * Every variant computes the same y = A x; they differ in how threads are
 * mapped onto strips (Section 4 gives one warp per strip).
 *   CMRS_VARIANT_ROW    mean rows of at most 28, 56 or 112 entries and a
 *                       height dividing 32, 16 or 8: L = 1, 2 or 4 lanes per
 *                       row -- a warp bulk-copies the entries of 32 / L
 *                       consecutive rows (whole strips) into its own
 *                       shared-memory stage and the row's L lanes sum it in
 *                       registers (a range longer than the stage, sized from
 *                       the mean row length, is read from global memory).
 *                       Otherwise: a few threads per row (4 for CMRS_F64, 2
 *                       for the other forms), each summing a contiguous
 *                       share, a CTA staging the strips of 128 consecutive
 *                       rows.  Needs unsorted strips.  Best for regular rows.
 *   CMRS_VARIANT_STRIP  Algorithm 1 of Section 4: one warp per strip, lanes
 *                       stride through the strip and accumulate per-row
 *                       partial sums in a shared-memory buffer buf[row][lane],
 *                       then a lane reduction.  Works on sorted strips.
 *   CMRS_VARIANT_MERGE  equal-work tiles of nonzeros: each thread owns a run
 *                       of consecutive entries, rows that cross thread or
 *                       tile boundaries are joined afterwards in a fixed
 *                       order.  Needs unsorted strips.  Best for skewed rows.
 *   CMRS_VARIANT_PADDED the Section 6.6 kernel, only for CMRS_PADDED
 *                       matrices: one warp per strip, lane l adds each
 *                       product into slot (l mod M) of its row in a per-warp
 *                       shared buffer, the slots of each row are summed at
 *                       the strip's end (M = 1: lane r keeps row r's sum in a
 *                       register, no buffer).  Fully coalesced 32-bit loads,
 *                       no search for row starts.  The FP32 and BF16 forms at
 *                       M = 1 with long strips stream them through a
 *                       shared-memory ring of bulk copies; few long strips
 *                       are split over several warps (see
 *                       cmrs_spmv_workspace).
 *   CMRS_VARIANT_AUTO   (-1) PADDED for padded strips, STRIP for sorted
 *                       strips.  Otherwise, with
 *                       mu = nnz / rows: MERGE if mu < 2, or mu > 32 (except
 *                       mu <= 56 at heights dividing 16 and mu <= 112 at
 *                       heights dividing 8, where ROW runs two or four lanes
 *                       per row), or max_strip_nnz > 8 * height * mu (or
 *                       unknown, -1); ROW for the rest.  cmrs_spmv_variant
 *                       reports the choice. */
#define CMRS_VARIANT_AUTO (-1)
#define CMRS_VARIANT_ROW 0
#define CMRS_VARIANT_STRIP 1
#define CMRS_VARIANT_MERGE 2
#define CMRS_VARIANT_PADDED 3
#define CMRS_NUM_VARIANTS 4

/* A CMRS matrix: a view of caller-owned device arrays (Section 3).
 *   strips     = ceil(rows / height)
 *   strip_ptr  [strips + 1] device int32: StripPtr, StripPtr[strips] = nnz
 *   col_packed [nnz] device uint32: (column << bits) | RowInStrip (Section 4);
 *              bits = cmrs_bits_for_height(height)
 *   val        device array of the storage form `dtype`
 *   max_strip_nnz  longest strip, or -1 if unknown (cmrs_from_csr fills it) */
typedef struct cmrs_matrix {
  int32_t rows, cols, nnz, height, strips, bits;
  uint32_t flags;
  int32_t dtype;
  int32_t max_strip_nnz;
  const int32_t *strip_ptr;
  const uint32_t *col_packed;
  const void *val;
} cmrs_matrix;

/* Name of a status code (static string, never NULL). */
const char *cmrs_error_string(int status);

/* The cudaError_t of the last CUDA failure seen by this thread (0 if none). */
int cmrs_last_cuda_error(void);

/* Bits of RowInStrip packed under the column: the paper uses 4 for heights up
 * to 16 (Section 4); heights 17..32 need 5.  Returns max(4, ceil(log2 h)), or
 * -1 for h outside 1..32.  Host only, pure. */
int cmrs_bits_for_height(int height);

/* Byte offset of the lo half of a CMRS_BF16X2 array: 2 * cmrs_pad8(nnz). */
int64_t cmrs_pad8(int64_t nnz);

/* Bytes of a value array of `nnz` entries in storage form `dtype`, or -1. */
int64_t cmrs_val_bytes(int64_t nnz, int dtype);

/* ---- conversion CRS -> CMRS (Section 3, packing Section 4) ---------------
 * Inputs (device): row_ptr[rows+1], col_ind[nnz] (int32), val_in[nnz] of type
 * val_in_dtype (CMRS_F64 or CMRS_F32).
 * Computes StripPtr[j] = RowPtr[j*height] (j < strips), StripPtr[strips] =
 * nnz; packed[k] = (col << bits) | (row(k) mod height); the values converted
 * to `dtype`; with CMRS_SORTED each strip is stably sorted by column.
 * Outputs (device): strip_ptr_out[strips+1], col_packed_out[nnz],
 * val_out (cmrs_val_bytes(nnz, dtype) bytes).  If `out` is not NULL it is
 * filled with a view of the outputs (host struct).
 * Validation: height 1..32 (CMRS_ERR_HEIGHT), cols <= 2^(32-bits)
 * (CMRS_ERR_COL_OVERFLOW) on the host; RowPtr monotone with RowPtr[0] = 0 and
 * RowPtr[rows] = nnz and 0 <= col < cols on the device (CMRS_ERR_CSR_INVALID).
 * Invalid input never makes a kernel read or write outside the given arrays.
 * Synchronises `stream` once, at the end, to read the device status word.
 * workspace: >= cmrs_from_csr_workspace() bytes, 256-byte aligned. */
int cmrs_from_csr_workspace(int rows, int nnz, int height, uint32_t flags, int dtype, size_t *bytes);
int cmrs_from_csr(int rows, int cols, int nnz, const int32_t *row_ptr, const int32_t *col_ind,
                  const void *val_in, int val_in_dtype, int height, uint32_t flags, int dtype,
                  int32_t *strip_ptr_out, uint32_t *col_packed_out, void *val_out,
                  void *workspace, size_t workspace_bytes, void *stream, cmrs_matrix *out);

/* ---- conversion CMRS -> CRS (the inverse "to and from" of Section 3) -----
 * RowPtr[s*height + r] = StripPtr[s] + #{entries of strip s with RowInStrip
 * < r}, RowPtr[rows] = nnz; within a row, entries keep their strip order (for
 * a sorted matrix each row comes out in column order); col = packed >> bits.
 * Outputs (device): row_ptr_out[rows+1], col_ind_out[nnz], val_out in A's
 * storage form (may be NULL to skip values).  Asynchronous; an entry whose
 * RowInStrip names a row >= rows sets a status the next call does not read:
 * pass a CMRS matrix built by cmrs_from_csr or one that is valid.
 * workspace: >= cmrs_to_csr_workspace() bytes (may be 0 and NULL). */
int cmrs_to_csr_workspace(const cmrs_matrix *A, size_t *bytes);
int cmrs_to_csr(const cmrs_matrix *A, int32_t *row_ptr_out, int32_t *col_ind_out, void *val_out,
                void *workspace, size_t workspace_bytes, void *stream);

/* ---- modified CMRS (Section 6.6) ------------------------------------------
 * Rearranges an unsorted CMRS matrix A (not itself padded) into the padded
 * form with M = slots in {1, 2, 4, 8} (height * slots >= 32, else
 * CMRS_ERR_HEIGHT; bad slots: CMRS_ERR_ARG).  Each strip becomes
 * C = max(ceil(items / 32), ceil(longest row / M)) passes of 32 items -- the
 * fewest possible.  Per pass, every row first takes the items it must for
 * the rest to fit in the passes left, then free room goes to rows with the
 * most items left (ties: lower row); rows appear in ascending order, each as
 * one run of at most M items (its next items in A's order, then its zero
 * items); free room after that is zero items, rows 0 upwards, each topped up
 * to M.  With M = 1 (so height 32) every pass holds one item of each row,
 * row r at position r: the SpMV kernel then keeps each row's sum in a
 * register.  A smaller M shortens the kernel's final slot sums but pads rows
 * longer than M * (items / 32) -- fit for regular rows, not skewed ones.
 * Same storage form as A (BF16X2: hi then lo at 2 * cmrs_pad8(nnz_padded)
 * bytes).
 *
 * A must be a valid unsorted CMRS matrix (RowInStrip non-decreasing within
 * each strip, as cmrs_from_csr writes it).
 * cmrs_pad_layout: writes the padded StripPtr (device, [strips+1], multiples
 * of 32) and the padded item count (host *nnz_padded).  Synchronises
 * `stream` once to read the count.  CMRS_ERR_ARG if the count reaches 2^31,
 * CMRS_ERR_UNSUPPORTED for sorted or padded input, CMRS_ERR_HEIGHT for
 * height < 4, CMRS_ERR_CSR_INVALID for a strip whose row bounds it finds out
 * of order.  workspace: >= cmrs_pad_workspace() bytes, 256-byte aligned.
 * cmrs_pad_fill: writes col_packed_out[nnz_padded] and val_out (device,
 * cmrs_val_bytes(nnz_padded, A->dtype) bytes, 16-byte aligned) and *out (a
 * view of strip_ptr_padded, col_packed_out and val_out with CMRS_PADDED set).
 * Asynchronous; it writes no more passes per strip than the layout gave it.
 * A padded matrix multiplies x[0] by zero in its zero items:
 * x must be finite there.  cmrs_to_csr does not accept padded matrices. */
int cmrs_pad_workspace(const cmrs_matrix *A, int slots, size_t *bytes);
int cmrs_pad_layout(const cmrs_matrix *A, int slots, int32_t *strip_ptr_padded, int32_t *nnz_padded,
                    void *workspace, size_t workspace_bytes, void *stream);
int cmrs_pad_fill(const cmrs_matrix *A, int slots, const int32_t *strip_ptr_padded, int32_t nnz_padded,
                  uint32_t *col_packed_out, void *val_out, void *stream, cmrs_matrix *out);

/* ---- row reordering (Section 7 outlook; Section 6.3: a low eta_+ is the cue)
 * An off-line optimisation of CRS input: rows of similar length placed in the
 * same strip, so that the modified form of Section 6.6 needs fewer zero
 * items.  The product of the reordered matrix P A is returned in the original
 * order by cmrs_spmv_rows with row_map = perm.
 *
 * cmrs_row_order: perm_out[i] (device int32 [rows]) = the original row placed
 * at position i.  Inside each window of `window` consecutive rows (1..4096;
 * the last window may be shorter), rows by length, longest first, equal
 * lengths in their original order; rows never leave their window, so a
 * window that is a multiple of the strip height keeps strips local.  row_ptr:
 * device CRS row pointer.  Asynchronous; no workspace.  CMRS_ERR_ARG for a
 * window outside 1..4096.
 *
 * cmrs_permute_csr: CRS of P A (row i = original row perm[i], entries in their
 * original order) into row_ptr_out [rows+1], col_ind_out [nnz] and val_out
 * (val may be NULL: columns only; val_dtype CMRS_F64 or CMRS_F32).  Checks on
 * the device that perm names every row exactly once and that the row pointer
 * stays inside [0, nnz] (CMRS_ERR_ARG), and that RowPtr[rows] = nnz
 * (CMRS_ERR_CSR_INVALID), before writing any column: synchronises `stream`
 * once.  workspace: >= cmrs_permute_csr_workspace() bytes, 256-byte aligned. */
int cmrs_row_order(int rows, const int32_t *row_ptr, int window, int32_t *perm_out, void *stream);
int cmrs_permute_csr_workspace(int rows, size_t *bytes);
int cmrs_permute_csr(int rows, int nnz, const int32_t *row_ptr, const int32_t *col_ind, const void *val,
                     int val_dtype, const int32_t *perm, int32_t *row_ptr_out, int32_t *col_ind_out,
                     void *val_out, void *workspace, size_t workspace_bytes, void *stream);

/* ---- SpMV, y = A x (Section 4, Algorithm 1) ------------------------------
 * x: device [cols], y: device [rows], double for CMRS_F64 else float.  y is
 * overwritten (rows without entries get 0).  A's arrays are trusted (as built
 * by cmrs_from_csr): no validation of their contents and no synchronisation;
 * writes are still kept inside y.  variant: CMRS_VARIANT_*.  ROW and MERGE
 * need col_packed and val 16-byte aligned (CMRS_ERR_ARG otherwise).
 * workspace: >= cmrs_spmv_workspace() bytes, 256-byte aligned (may be NULL
 * when the query returns 0).  For a padded matrix of few long strips (fewer
 * than two per resident warp, at least 64 passes each on average) the query
 * includes room for per-part row sums: each strip is then split over several
 * warps and a second kernel adds each row's parts in order; with a workspace
 * of only 256 bytes the one-warp-per-strip walk runs instead.  The result
 * depends only on A, x, the variant and (padded matrices) whether the
 * workspace holds the part sums and the device's SM count: fixed summation
 * order, no atomics on values, so repeated calls give bit-identical y. */
int cmrs_spmv_workspace(const cmrs_matrix *A, int variant, size_t *bytes);

/* The kernel variant cmrs_spmv runs for `variant` (resolves
 * CMRS_VARIANT_AUTO by the rule above; checks that an explicit variant suits
 * the matrix).  *resolved receives CMRS_VARIANT_ROW, _STRIP or _MERGE.  Host
 * only: reads the fields of *A, never its device arrays.  Errors as
 * cmrs_spmv_workspace (CMRS_ERR_UNSUPPORTED: ROW or MERGE on sorted strips). */
int cmrs_spmv_variant(const cmrs_matrix *A, int variant, int *resolved);
int cmrs_spmv(const cmrs_matrix *A, const void *x, void *y, int variant,
              void *workspace, size_t workspace_bytes, void *stream);

/* y[row_map[i]] = (A x)_i: the product of a row-reordered matrix (A = P B,
 * row_map = the perm of cmrs_row_order) written in the original row order.
 * row_map: device int32 [rows], a permutation of 0..rows-1 (entries outside
 * that range are skipped; a map that is not a permutation leaves some of y
 * unwritten).  Same arguments, workspace and errors as cmrs_spmv; variants
 * ROW, STRIP and PADDED (explicit MERGE: CMRS_ERR_UNSUPPORTED; AUTO picks ROW
 * where cmrs_spmv would pick MERGE).  Costs 4 bytes per row of map reads.
 * Asynchronous. */
int cmrs_spmv_rows(const cmrs_matrix *A, const void *x, void *y, const int32_t *row_map, int variant,
                   void *workspace, size_t workspace_bytes, void *stream);

/* SpMV that allocates nothing, for callers that cannot allocate device
 * memory at all: code that runs inside an allocator or memory-pool callback,
 * under a pool that forbids growth, or in a runtime that owns every device
 * buffer and hands out no scratch.  (The paper has no counterpart; this entry
 * point belongs to the library.)  It computes y = A x exactly as cmrs_spmv
 * with CMRS_VARIANT_MERGE, same arguments without the workspace, but takes
 * its scratch from one fixed 2 MiB array compiled into the library (a
 * file-scope __device__ array, resident on every GPU that loads the library
 * until the process exits).  Limit: 58,240 MERGE tiles, i.e. A->nnz <=
 * 67,092,480 for CMRS_F64 (tiles of 1,152 entries) and <= 82,001,920 for the
 * other forms (1,408 entries); larger matrices return CMRS_ERR_WORKSPACE
 * before any device work.  Unsorted, unpadded strips only
 * (CMRS_ERR_UNSUPPORTED otherwise).  No cudaMalloc, cudaFree or other
 * allocating call is made.  The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress, with that device current)
 * and keeps it for the later calls.
 * Every call shares the one array, which keeps the last call's contents:
 * calls that may overlap on the GPU (two streams, two host threads) race and
 * their results are undefined.  The cached address belongs to the device's
 * current context: do not use this entry point after cudaDeviceReset in the
 * same process.  Asynchronous on `stream`.
 * The MERGE kernel's bounded waits record a give-up in a status word inside
 * the array; the word is not cleared by the calls, so it holds every give-up
 * since it was last read.  cmrs_spmv_noalloc_check reads and clears it for
 * the current device (synchronising `stream`): CMRS_ERR_TIMEOUT means that
 * some call since the last check left its y invalid. */
int cmrs_spmv_noalloc(const cmrs_matrix *A, const void *x, void *y, void *stream);
int cmrs_spmv_noalloc_check(void *stream);

/* Error status the SpMV kernels left in the status word inside `workspace`,
 * then cleared: CMRS_ERR_TIMEOUT if a bounded in-kernel wait gave up,
 * CMRS_ERR_ARG if a padded strip was not a whole number of 32-item passes
 * (a matrix not made by cmrs_pad_fill; that strip's rows are not valid),
 * else CMRS_OK.  Reads device memory synchronously on `stream`. */
int cmrs_spmv_check(const cmrs_matrix *A, int variant, const void *workspace, void *stream);

/* Diagnostic, not in the paper: exercises the timeout report of the staged
 * kernels without a fault.  One warp waits, with the bounded mbarrier wait
 * those kernels use for their bulk copies, on a phase that only an arrival of
 * its own completes; arrive != 0 makes that arrival first, arrive == 0 leaves
 * the phase open, so every lane gives up after `tries` tries (1..65536) and
 * the kernel sets the timeout bit of the status word at the start of
 * `workspace` (device, caller-owned, >= 256 bytes, 256-byte aligned) and
 * returns.  cmrs_spmv_check on that workspace then reports CMRS_ERR_TIMEOUT
 * and clears the bit.  workspace == NULL names the status word of the fixed
 * array of cmrs_spmv_noalloc on the current device, which
 * cmrs_spmv_noalloc_check then reports.  No copy is issued, so none is left
 * in flight.  CMRS_ERR_ARG for a misaligned workspace or a bad `tries`.
 * Asynchronous on `stream`. */
int cmrs_wait_probe(void *workspace, uint32_t tries, int arrive, void *stream);

/* Diagnostic, not in the paper: the floor of a product whose x reads are
 * gathers (Section 6.3 reads a low eta_+ as x fetched many times over).
 * Streams col[nnz] (device int32, a CRS column array) and val[nnz] (device
 * float, or NULL for ones) once, in order, gathers x[col[k]] (device float
 * [cols]) and adds val[k] * x[col[k]] into *out (device float, overwritten;
 * the summation order is not fixed).  No row structure: the time of a call on
 * a matrix's own columns is what any SpMV kernel pays for that matrix's
 * gathers and streams alone.  A column outside [0, cols) reads x[cols - 1].
 * CMRS_ERR_ARG for negative sizes or missing pointers.  Asynchronous. */
int cmrs_gather_probe(int nnz, int cols, const int32_t *col, const float *val, const float *x, float *out,
                      void *stream);

/* ---- strip sharding over several GPUs --------------------------------------
 * Strips are independent (Section 4: a strip's warp reads only its own
 * entries and writes only its own rows of y), so a product can be split into
 * contiguous ranges of whole strips, one per device; every device multiplies
 * its range once it holds all of x, and y needs no reduction.
 * cmrs_shard_rows: bounds[p] .. bounds[p+1] are the rows of part p, for
 * p < parts (bounds: host int32 [parts + 1], bounds[0] = 0, bounds[parts] =
 * rows).  Each inner bound is a strip start (a multiple of height, or rows),
 * chosen as the first strip start at which the weight before it -- entries
 * plus rows -- reaches ceil(p * total / parts); parts may be empty when
 * there are fewer strips than parts.  row_ptr: host int32 [rows + 1], a CRS
 * row pointer (RowPtr[0] = 0, non-decreasing; only RowPtr[0] is checked).
 * Host only, pure.  CMRS_ERR_ARG for bad sizes or pointers, CMRS_ERR_HEIGHT
 * for a height outside 1..32, CMRS_ERR_CSR_INVALID if RowPtr[0] != 0. */
int cmrs_shard_rows(int rows, const int32_t *row_ptr, int height, int parts, int32_t *bounds);

/* ---- multi right-hand-side SpMM, single and batched ----------------------
 * Y = A X for CMRS_F32 matrices with unsorted strips; X device [cols][k] and
 * Y device [rows][k], row-major FP32, FP32 accumulation.  Not in the paper:
 * the strip layout of Section 3 applied to k right-hand sides at once.
 * cmrs_spmm: one matrix, one launch, asynchronous. */
int cmrs_spmm(const cmrs_matrix *A, int k, const float *X, float *Y, void *stream);

/* Batched form: many uneven matrices in one persistent launch.  A plan holds
 * the schedule -- work units (matrix, row range) of about `work_target`
 * entry-columns each, heaviest first, fetched by warps from a device queue --
 * and, with use_graph != 0, a CUDA graph of {queue reset, persistent kernel}.
 * A[b] (host array of pointers to host structs), k[b], X[b], Y[b] (host
 * arrays of device pointers) for b < batch.  The plan's device part lives in
 * `workspace` (>= cmrs_spmm_plan_workspace() bytes, 256-byte aligned), which
 * must outlive the plan; creation copies the schedule and synchronises
 * `stream` once.  cmrs_spmm_batched replays the plan on `stream`
 * (asynchronous).  The plan is a host object released by
 * cmrs_spmm_plan_destroy. */
typedef struct cmrs_spmm_plan cmrs_spmm_plan;
int cmrs_spmm_plan_workspace(int batch, const cmrs_matrix *const *A, const int32_t *k, int work_target,
                             size_t *bytes);
int cmrs_spmm_plan_create(int batch, const cmrs_matrix *const *A, const int32_t *k, const float *const *X,
                          float *const *Y, int work_target, int use_graph, void *workspace,
                          size_t workspace_bytes, void *stream, cmrs_spmm_plan **plan);
int cmrs_spmm_batched(cmrs_spmm_plan *plan, void *stream);
int cmrs_spmm_plan_info(const cmrs_spmm_plan *plan, int *nunits, int *grid, int *work_target);
int cmrs_spmm_plan_destroy(cmrs_spmm_plan *plan);

/* Autotuner of the batch schedule: times `reps` replays of a graph plan for
 * each candidate work_target and returns the fastest (best_ms: mean per
 * replay).  Synchronises `stream`.  workspace as for the largest plan. */
int cmrs_spmm_autotune(int batch, const cmrs_matrix *const *A, const int32_t *k, const float *const *X,
                       float *const *Y, const int *candidates, int ncand, int reps, void *workspace,
                       size_t workspace_bytes, void *stream, int *best_target, float *best_ms);

/* ---- strip selector -------------------------------------------------------
 * Not in the paper: Section 6.2 chooses the strip height by brute force and
 * Section 6.7 measures what per-matrix tuning gains.  The selector predicts
 * (height, variant) from CMRS_NFEAT features of the CRS matrix with a small
 * MLP (CMRS_NFEAT -> nh -> nh -> CMRS_SEL_CHOICES, ReLU), trained on this
 * library's own timings by the kernels below.  Choice c < 18 means plain
 * CMRS with height {1,2,4,8,16,32}[c / 3] and variant c % 3; choices 18, 19
 * and 20 mean the modified CMRS of Section 6.6 (variant CMRS_VARIANT_PADDED)
 * at (height, slots) = (32, 1), (32, 2) and (16, 8).  The network outputs a
 * predicted cost per choice and the smallest wins. */
#define CMRS_NFEAT 32
#define CMRS_SEL_CHOICES 21

/* Features (device double[CMRS_NFEAT]) of a CRS matrix (device row_ptr,
 * col_ind), from exact integer sums: log2 rows, log2 nnz, log2(1+mu), row
 * length CV, log2(1+max row), empty-row fraction, 8 row-length bins,
 * |col-row| statistics, equal-length neighbour fraction, per-strip column
 * spread for h = 1..32 (features 0..23); log2(items / nnz) of the modified
 * CMRS of Section 6.6 at (height, slots) = (32, 1), (32, 2), (16, 8), a strip
 * of n_s entries with longest row m_s taking max(ceil(n_s/32),
 * ceil(m_s/slots)) passes of 32 items (24..26); the fraction of entries in
 * rows of at least 32, 512 and 8192 entries (27..29); the spread (std / mean)
 * and log2(1 + max / mean) of the entry counts of 32-row strips (30, 31).
 * All but the first three describe the matrix's shape, not its size.
 * Asynchronous. */
int cmrs_features_workspace(int rows, size_t *bytes);
int cmrs_features(int rows, int nnz, const int32_t *row_ptr, const int32_t *col_ind, double *feat,
                  void *workspace, size_t workspace_bytes, void *stream);

/* Network parameters: one device float array, W1[nh][nin], b1[nh],
 * W2[nh][nh], b2[nh], W3[nout][nh], b3[nout].  acts (device): Z1, H1, Z2, H2
 * ([B][nh] each) then O ([B][nout]).  Loss = sum (O - T)^2 / (2 B nout);
 * grads has the parameter layout; scratch: B * (nout + 2 nh) floats; loss:
 * device float or NULL.  Adam: the textbook update with bias correction at
 * 1-based `step`.  All asynchronous. */
int64_t cmrs_mlp_param_count(int nin, int nh, int nout);
int cmrs_mlp_forward(int B, int nin, int nh, int nout, const float *X, const float *params, float *acts,
                     void *stream);
int cmrs_mlp_backward(int B, int nin, int nh, int nout, const float *X, const float *T, const float *params,
                      const float *acts, float *grads, float *scratch, float *loss, void *stream);
int cmrs_mlp_adam(int n, float *params, const float *grads, float *m, float *v, int step, float lr,
                  float beta1, float beta2, float eps, void *stream);

/* Training data of the network, on the device.  cmrs_feature_norm: per
 * feature j of F (device double [B][nin], row-major) its mean and population
 * standard deviation over the B rows (FP64 sums in row order), written as
 * mean[j] and scale[j] = 1 / std (0 for a feature that does not vary; both
 * device float [nin]); with X != NULL also X = (F - mean) * scale (device
 * float [B][nin]).  cmrs_feature_apply: X only, from a given mean and scale.
 * cmrs_cost_targets: T[n][c] = min(log2(times[n][c] / min_c times[n][c]), cap)
 * (times: device double [B][nout], positive; T: device float [B][nout]).
 * CMRS_ERR_ARG for bad sizes, pointers or cap <= 0.  Asynchronous. */
int cmrs_feature_norm(int B, int nin, const double *F, float *mean, float *scale, float *X, void *stream);
int cmrs_feature_apply(int B, int nin, const double *F, const float *mean, const float *scale, float *X,
                       void *stream);
int cmrs_cost_targets(int B, int nout, const double *times, float cap, float *T, void *stream);

/* A trained selector (device pointers): input x = (feature - feat_mean) *
 * feat_scale, nin = CMRS_NFEAT, nout = CMRS_SEL_CHOICES, nh <= 64. */
typedef struct cmrs_selector {
  int32_t nin, nh, nout;
  const float *params;
  const float *feat_mean;
  const float *feat_scale;
} cmrs_selector;

/* Picks (height, variant, slots) for a CRS matrix: *slots_out is 0 for
 * plain CMRS, else the slots of the padded form (variant
 * CMRS_VARIANT_PADDED).  model != NULL: features + network + argmin on the
 * device.  model == NULL: exhaustive autotune, converting with every height
 * and timing every variant and the three padded forms (5 timed calls each)
 * on FP32 copies held in the workspace; a padded form with more than
 * 2 * nnz + 32 * (rows / 16 + 2) items is not timed.  Synchronises
 * `stream`. */
int cmrs_select_strip_workspace(int rows, int cols, int nnz, int exhaustive, size_t *bytes);
int cmrs_select_strip(int rows, int cols, int nnz, const int32_t *row_ptr, const int32_t *col_ind,
                      const cmrs_selector *model, int *height_out, int *variant_out, int *slots_out,
                      void *workspace, size_t workspace_bytes, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* CMRS_H */
