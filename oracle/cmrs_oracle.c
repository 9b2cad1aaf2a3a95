/*
 * CMRS oracle -- TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.
 *
 * A plain, slow, single-threaded CPU restatement, in FP64, of what the
 * Compressed Multi-Row Storage (CMRS) method computes (Koza, Matyka, Szkoda,
 * Miroslaw, "Compressed Multi-Row Storage Format for Sparse Matrices on
 * Graphics Processing Units", arXiv:1203.2946).  Only the test suite,
 * __graft_entry__.smoke() and bench.py's cpu_baseline / reference legs may
 * load this library.  It shares no source, header, table or constant with the
 * CUDA library under paper_1203_2946_gb300/csrc; the two are checked against
 * each other only through their outputs.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off (see build_oracle.py).  With
 * contraction off every product and every sum below is a separately rounded
 * IEEE-754 double operation, taken in the order the loops state.
 *
 * Pins (tests/test_oracle_*.py) tie every function here to something other
 * than itself: the worked 5x5 example of Sections 2.3, 3 and 4, dense
 * matrix-vector products, closed-form stencil row sums, bit-exact round trips,
 * the closed forms of Section 5 and its appendix, brute force on tiny inputs,
 * central finite differences for the selector network.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Error codes of this oracle (independent of the product's codes). */
#define ORC_OK 0
#define ORC_BAD_HEIGHT 1
#define ORC_BAD_CSR 2
#define ORC_COL_OVERFLOW 3
#define ORC_BAD_ARG 4

/* ------------------------------------------------------------------------ */
/* Section 4: the column index and RowInStrip share one 32-bit word; the low
 * CMRS_BITS bits hold RowInStrip (Algorithm 1 recovers r = c mod M and
 * c = floor(c / M) with M = 2^CMRS_BITS).  The paper fixes CMRS_BITS = 4 for
 * heights up to 16.  Heights 17..32 need a fifth bit; the reading used here
 * is bits = max(4, ceil(log2(height))). */
int orc_bits_for_height(int height) {
  if (height < 1 || height > 32) return -1;
  int bits = 0;
  while ((1 << bits) < height) ++bits;
  return bits < 4 ? 4 : bits;
}

/* ------------------------------------------------------------------------ */
/* Section 2.1 / 2.3: y = A x with A in CRS.  Row i owns entries
 * RowPtr[i] .. RowPtr[i+1]-1.  y_i starts from +0.0 and adds Val*x in CRS
 * order.  absy_i = sum |Val| * |x| is the scale the FP64 tolerance is stated
 * against ((|A||x|)_i).  Either output may be NULL. */
void orc_csr_spmv(int rows, const int32_t *row_ptr, const int32_t *col_ind,
                  const double *val, const double *x, double *y, double *absy) {
  for (int i = 0; i < rows; ++i) {
    double s = 0.0, a = 0.0;
    for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
      double p = val[k] * x[col_ind[k]];
      s = s + p;
      a = a + fabs(val[k]) * fabs(x[col_ind[k]]);
    }
    if (y) y[i] = s;
    if (absy) absy[i] = a;
  }
}

/* Dense row-major matrix-vector product, the textbook definition. */
void orc_dense_matvec(int rows, int cols, const double *a, const double *x,
                      double *y) {
  for (int i = 0; i < rows; ++i) {
    double s = 0.0;
    for (int j = 0; j < cols; ++j) s = s + a[(size_t)i * cols + j] * x[j];
    y[i] = s;
  }
}

/* CRS validity as Section 2.3 defines it: RowPtr has rows+1 entries,
 * RowPtr[0] = 0, consecutive differences are row lengths (so non-negative),
 * RowPtr[rows] = nnz, and every column lies in [0, cols). */
static int csr_check(int rows, int cols, int nnz, const int32_t *row_ptr,
                     const int32_t *col_ind) {
  if (rows < 0 || cols < 0 || nnz < 0) return ORC_BAD_ARG;
  if (row_ptr[0] != 0 || row_ptr[rows] != nnz) return ORC_BAD_CSR;
  for (int i = 0; i < rows; ++i)
    if (row_ptr[i + 1] < row_ptr[i]) return ORC_BAD_CSR;
  for (int k = 0; k < nnz; ++k)
    if (col_ind[k] < 0 || col_ind[k] >= cols) return ORC_BAD_CSR;
  return ORC_OK;
}

/* Key used by the in-strip sort: column first, then the entry's position in
 * the strip before sorting, which makes the order total and the sort stable. */
typedef struct {
  uint32_t col;
  int32_t pos;
} orc_sort_key;

static int key_cmp(const void *pa, const void *pb) {
  const orc_sort_key *a = (const orc_sort_key *)pa, *b = (const orc_sort_key *)pb;
  if (a->col != b->col) return a->col < b->col ? -1 : 1;
  return (a->pos > b->pos) - (a->pos < b->pos);
}

/* Section 3: CRS -> CMRS.
 *   strips = ceil(rows / height)
 *   StripPtr[j] = RowPtr[j * height] for j < strips, StripPtr[strips] = nnz
 *   RowInStrip[k] = (row of entry k) mod height
 * Val and ColInd keep the CRS order.  Section 4 packs RowInStrip into the low
 * `bits` bits of the column word: packed = (col << bits) | RowInStrip.
 * With `sorted` set, Section 4's fourth optimisation reorders each strip's
 * entries by column; ties keep their CRS order (the worked example of
 * Section 4 fixes that reading).
 * Outputs: strip_ptr[strips+1], packed[nnz], row_in_strip[nnz] (may be NULL),
 * val_out[nnz] (may be NULL), src[nnz] = CRS index each output entry came
 * from (may be NULL).  Columns must fit in 32 - bits bits. */
int orc_csr_to_cmrs(int rows, int cols, int nnz, const int32_t *row_ptr,
                    const int32_t *col_ind, const double *val, int height,
                    int sorted, int32_t *strip_ptr, uint32_t *packed,
                    int32_t *row_in_strip, double *val_out, int32_t *src) {
  int bits = orc_bits_for_height(height);
  if (bits < 0) return ORC_BAD_HEIGHT;
  int rc = csr_check(rows, cols, nnz, row_ptr, col_ind);
  if (rc) return rc;
  if ((uint64_t)cols > ((uint64_t)1 << (32 - bits))) return ORC_COL_OVERFLOW;
  int strips = (rows + height - 1) / height;
  for (int j = 0; j < strips; ++j) strip_ptr[j] = row_ptr[j * height];
  strip_ptr[strips] = nnz;

  int32_t *from = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
  for (int k = 0; k < nnz; ++k) from[k] = k;
  if (sorted) {
    orc_sort_key *keys = (orc_sort_key *)malloc(sizeof(orc_sort_key) * (size_t)(nnz > 0 ? nnz : 1));
    for (int j = 0; j < strips; ++j) {
      int a = strip_ptr[j], b = strip_ptr[j + 1];
      for (int k = a; k < b; ++k) {
        keys[k].col = (uint32_t)col_ind[k];
        keys[k].pos = k - a;
      }
      qsort(keys + a, (size_t)(b - a), sizeof(orc_sort_key), key_cmp);
      for (int k = a; k < b; ++k) from[k] = a + keys[k].pos;
    }
    free(keys);
  }
  /* row of each CRS entry, from RowPtr */
  int32_t *row_of = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
  for (int i = 0; i < rows; ++i)
    for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) row_of[k] = i;
  for (int k = 0; k < nnz; ++k) {
    int32_t f = from[k];
    uint32_t ris = (uint32_t)(row_of[f] % height);
    packed[k] = ((uint32_t)col_ind[f] << bits) | ris;
    if (row_in_strip) row_in_strip[k] = (int32_t)ris;
    if (val_out) val_out[k] = val[f];
    if (src) src[k] = f;
  }
  free(row_of);
  free(from);
  return ORC_OK;
}

/* CMRS -> CRS, the inverse conversion Section 3 calls trivial ("to and from"
 * in the abstract and Section 7).  Row s*height + r owns the entries of strip
 * s whose RowInStrip is r; its count gives RowPtr by a running sum that starts
 * at StripPtr[s].  Within a row, entries keep their order in the strip (a
 * stable counting sort by RowInStrip), so for an unsorted CMRS matrix this is
 * the exact inverse, and for a strip-sorted one each row comes out in column
 * order.  Entries whose RowInStrip names a row >= rows make it fail. */
int orc_cmrs_to_csr(int rows, int nnz, int height, const int32_t *strip_ptr,
                    const uint32_t *packed, const double *val,
                    int32_t *row_ptr, int32_t *col_ind, double *val_out,
                    int32_t *src) {
  int bits = orc_bits_for_height(height);
  if (bits < 0) return ORC_BAD_HEIGHT;
  int strips = (rows + height - 1) / height;
  if (strip_ptr[0] != 0 || strip_ptr[strips] != nnz) return ORC_BAD_CSR;
  uint32_t mask = ((uint32_t)1 << bits) - 1;
  int32_t *cnt = (int32_t *)calloc((size_t)rows + 1, sizeof(int32_t));
  for (int s = 0; s < strips; ++s) {
    if (strip_ptr[s + 1] < strip_ptr[s]) { free(cnt); return ORC_BAD_CSR; }
    for (int32_t k = strip_ptr[s]; k < strip_ptr[s + 1]; ++k) {
      int64_t row = (int64_t)s * height + (packed[k] & mask);
      if ((packed[k] & mask) >= (uint32_t)height || row >= rows) { free(cnt); return ORC_BAD_CSR; }
      cnt[row] += 1;
    }
  }
  for (int s = 0; s < strips; ++s) {
    int32_t p = strip_ptr[s];
    for (int r = 0; r < height && s * height + r < rows; ++r) {
      row_ptr[s * height + r] = p;
      p += cnt[s * height + r];
    }
  }
  row_ptr[rows] = nnz;
  int32_t *fill = (int32_t *)calloc((size_t)rows + 1, sizeof(int32_t));
  for (int s = 0; s < strips; ++s) {
    for (int32_t k = strip_ptr[s]; k < strip_ptr[s + 1]; ++k) {
      int row = s * height + (int)(packed[k] & mask);
      int32_t d = row_ptr[row] + fill[row]++;
      col_ind[d] = (int32_t)(packed[k] >> bits);
      if (val_out) val_out[d] = val[k];
      if (src) src[d] = k;
    }
  }
  free(fill);
  free(cnt);
  return ORC_OK;
}

/* Algorithm 1 (Section 4), stated sequentially: every row sum starts at +0.0;
 * each strip's entries are visited in storage order, RowInStrip and the
 * column are unpacked from the packed word, and Val * x[col] is added to
 * row strip*height + RowInStrip.  Rows with no entries stay 0.  This reaches
 * y = A x (Section 2.1); the per-lane partial buffers and the lane reduction
 * of Algorithm 1 only reorder the same sums. */
void orc_cmrs_spmv(int rows, int height, const int32_t *strip_ptr,
                   const uint32_t *packed, const double *val, const double *x,
                   double *y) {
  int bits = orc_bits_for_height(height);
  uint32_t m = (uint32_t)1 << bits;
  int strips = (rows + height - 1) / height;
  for (int i = 0; i < rows; ++i) y[i] = 0.0;
  for (int s = 0; s < strips; ++s) {
    for (int32_t j = strip_ptr[s]; j < strip_ptr[s + 1]; ++j) {
      uint32_t c = packed[j];
      uint32_t r = c % m;
      c = c / m;
      y[s * height + (int)r] = y[s * height + (int)r] + val[j] * x[c];
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Value storage forms.  The paper stores Val as float or double (Section
 * 6.2).  The reduced forms below are this library's own definitions, written
 * with integer operations so that the stored bits are unambiguous:
 *   F32   : (float)v, IEEE round to nearest even.
 *   BF16  : the upper 16 bits of the FP32 pattern of (float)v, rounded to
 *           nearest even: (u + 0x7FFF + ((u >> 16) & 1)) >> 16.
 *   BF16X2: hi = BF16(v), lo = BF16(v - (double)hi); v ~ hi + lo.
 * Inputs carry no NaN or infinity. */
uint16_t orc_bf16_from_f32(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  uint32_t lsb = (u >> 16) & 1u;
  return (uint16_t)((u + 0x7FFFu + lsb) >> 16);
}

float orc_f32_from_bf16(uint16_t h) {
  uint32_t u = (uint32_t)h << 16;
  float f;
  memcpy(&f, &u, 4);
  return f;
}

/* dtype: 0 = F64 copy, 1 = F32, 2 = BF16, 3 = BF16X2 (hi[n] then lo[n]). */
int orc_encode_f64(int n, const double *v, int dtype, void *out) {
  if (dtype == 0) {
    memcpy(out, v, sizeof(double) * (size_t)n);
  } else if (dtype == 1) {
    float *o = (float *)out;
    for (int k = 0; k < n; ++k) o[k] = (float)v[k];
  } else if (dtype == 2) {
    uint16_t *o = (uint16_t *)out;
    for (int k = 0; k < n; ++k) o[k] = orc_bf16_from_f32((float)v[k]);
  } else if (dtype == 3) {
    uint16_t *hi = (uint16_t *)out, *lo = hi + n;
    for (int k = 0; k < n; ++k) {
      hi[k] = orc_bf16_from_f32((float)v[k]);
      double rest = v[k] - (double)orc_f32_from_bf16(hi[k]);
      lo[k] = orc_bf16_from_f32((float)rest);
    }
  } else {
    return ORC_BAD_ARG;
  }
  return ORC_OK;
}

/* Same forms from FP32 input values (the F64 form widens exactly). */
int orc_encode_f32(int n, const float *v, int dtype, void *out) {
  if (dtype == 0) {
    double *o = (double *)out;
    for (int k = 0; k < n; ++k) o[k] = (double)v[k];
  } else if (dtype == 1) {
    memcpy(out, v, sizeof(float) * (size_t)n);
  } else if (dtype == 2) {
    uint16_t *o = (uint16_t *)out;
    for (int k = 0; k < n; ++k) o[k] = orc_bf16_from_f32(v[k]);
  } else if (dtype == 3) {
    uint16_t *hi = (uint16_t *)out, *lo = hi + n;
    for (int k = 0; k < n; ++k) {
      hi[k] = orc_bf16_from_f32(v[k]);
      double rest = (double)v[k] - (double)orc_f32_from_bf16(hi[k]);
      lo[k] = orc_bf16_from_f32((float)rest);
    }
  } else {
    return ORC_BAD_ARG;
  }
  return ORC_OK;
}

/* The value each stored form represents, widened to FP64 (hi + lo for the
 * split form, summed in double).  Used by the quantised-input oracle, which
 * separates storage error from accumulation error. */
int orc_decode_to_f64(int n, const void *stored, int dtype, double *out) {
  if (dtype == 0) {
    memcpy(out, stored, sizeof(double) * (size_t)n);
  } else if (dtype == 1) {
    const float *s = (const float *)stored;
    for (int k = 0; k < n; ++k) out[k] = (double)s[k];
  } else if (dtype == 2) {
    const uint16_t *s = (const uint16_t *)stored;
    for (int k = 0; k < n; ++k) out[k] = (double)orc_f32_from_bf16(s[k]);
  } else if (dtype == 3) {
    const uint16_t *hi = (const uint16_t *)stored, *lo = hi + n;
    for (int k = 0; k < n; ++k)
      out[k] = (double)orc_f32_from_bf16(hi[k]) + (double)orc_f32_from_bf16(lo[k]);
  } else {
    return ORC_BAD_ARG;
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Section 5 and its appendix: the transfer-waste model.
 * A chunk of n bytes made of b-byte items, starting at a random b-aligned
 * offset, touches on average S = 1 + (n - b) / lambda segments of lambda
 * bytes; the bytes moved over the bytes asked for are lambda*S/n =
 * 1 + (lambda - b)/n.  With n = h*mu*b this is Eq. (5.1), f(h, mu); Eq. (5.2)
 * is a(h, mu) = f(1, mu) / f(h, mu). */
double orc_model_segments(double n, double lambda, double b) {
  return 1.0 + (n - b) / lambda;
}

double orc_model_f(double h, double mu, double lambda, double b) {
  return 1.0 + (lambda - b) / (h * mu * b);
}

double orc_model_a(double h, double mu, double lambda, double b) {
  return orc_model_f(1.0, mu, lambda, b) / orc_model_f(h, mu, lambda, b);
}

/* Segments touched by a chunk of n bytes starting at byte offset `start`
 * (counting every lambda-aligned segment that holds at least one byte). */
double orc_segments_at(long n, long lambda, long start) {
  if (n <= 0) return 0.0;
  long first = start / lambda, last = (start + n - 1) / lambda;
  return (double)(last - first + 1);
}

/* Eq. (6.1): minimum bytes moved, x not cached (beta_minus) and x fully
 * cached (beta_plus); s_v value size, s_i = 4 index size. */
void orc_beta(double nnz, double rows, double strips, double s_v, double s_i,
              double *beta_minus, double *beta_plus) {
  *beta_minus = (2.0 * s_v + s_i) * nnz + s_i * strips + s_v * rows;
  *beta_plus = (s_v + s_i) * nnz + s_i * strips + 2.0 * s_v * rows;
}

/* ------------------------------------------------------------------------ */
/* Strip selector (not in the paper; Section 6.2 tunes height by brute force
 * and Section 6.7 measures what per-matrix tuning gains).  The selector reads
 * 32 features of a CRS matrix, computed here with plain loops and exact
 * integer sums:
 *   f0  log2(rows)                 f1  log2(max(nnz, 1))
 *   f2  log2(1 + mu), mu = nnz/rows
 *   f3  sigma_L / max(mu, 1)       (sigma_L: population std of row lengths)
 *   f4  log2(1 + max row length)   f5  fraction of empty rows
 *   f6..f13 fraction of rows with length in [1,1], [2,3], [4,7], [8,15],
 *           [16,31], [32,63], [64,127], [128, inf)
 *   f14 log2(1 + mean |col - row|) over entries
 *   f15 log2(1 + max |col - row|)
 *   f16 fraction of entries with |col - row| <= 64
 *   f17 fraction of rows i >= 1 with the same length as row i-1
 *   f18..f23 for h = 1, 2, 4, 8, 16, 32: log2(1 + mean over non-empty strips
 *           of (max col - min col) within the strip)
 *   f24..f26 log2(items / nnz) of the modified CMRS (Section 6.6) at
 *           (height, M) = (32, 1), (32, 2), (16, 8): a strip of n_s entries
 *           whose longest row has m_s becomes max(ceil(n_s/32), ceil(m_s/M))
 *           passes of 32 items (the fewest possible); 0 when nnz = 0
 *   f27..f29 fraction of the entries that lie in rows of at least 32, 512
 *           and 8192 entries
 *   f30 sigma(n_32) / max(mean n_32, 1), n_32 the entries of a strip of 32
 *       rows, over the ceil(rows/32) strips (population std)
 *   f31 log2(1 + max n_32 / max(mean n_32, 1)) */
#define ORC_NFEAT 32
void orc_features(int rows, int nnz, const int32_t *row_ptr,
                  const int32_t *col_ind, double *f) {
  uint64_t sum_l2 = 0, max_l = 0, empty = 0, same = 0, near = 0;
  uint64_t bins[8] = {0};
  uint64_t sum_d = 0, max_d = 0;
  for (int i = 0; i < rows; ++i) {
    uint64_t l = (uint64_t)(row_ptr[i + 1] - row_ptr[i]);
    sum_l2 += l * l;
    if (l > max_l) max_l = l;
    if (l == 0) empty++;
    if (i > 0 && l == (uint64_t)(row_ptr[i] - row_ptr[i - 1])) same++;
    if (l >= 1) {
      int b = 0;
      while (b < 7 && l >= ((uint64_t)2 << b)) ++b;
      bins[b]++;
    }
    for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
      int64_t d = (int64_t)col_ind[k] - i;
      uint64_t ad = (uint64_t)(d < 0 ? -d : d);
      sum_d += ad;
      if (ad > max_d) max_d = ad;
      if (ad <= 64) near++;
    }
  }
  double n = (double)rows, z = (double)nnz;
  double mu = z / n;
  double var = (double)sum_l2 / n - mu * mu;
  if (var < 0.0) var = 0.0;
  f[0] = log2(n);
  f[1] = log2(z > 1.0 ? z : 1.0);
  f[2] = log2(1.0 + mu);
  f[3] = sqrt(var) / (mu > 1.0 ? mu : 1.0);
  f[4] = log2(1.0 + (double)max_l);
  f[5] = (double)empty / n;
  for (int b = 0; b < 8; ++b) f[6 + b] = (double)bins[b] / n;
  f[14] = log2(1.0 + (nnz > 0 ? (double)sum_d / z : 0.0));
  f[15] = log2(1.0 + (double)max_d);
  f[16] = nnz > 0 ? (double)near / z : 0.0;
  f[17] = rows > 1 ? (double)same / (double)(rows - 1) : 0.0;
  for (int e = 0; e < 6; ++e) {
    int h = 1 << e;
    uint64_t spread = 0, nonempty = 0;
    for (int s = 0; s * h < rows; ++s) {
      int r1 = (s + 1) * h < rows ? (s + 1) * h : rows;
      int32_t lo = INT32_MAX, hi = -1;
      for (int i = s * h; i < r1; ++i)
        for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
          if (col_ind[k] < lo) lo = col_ind[k];
          if (col_ind[k] > hi) hi = col_ind[k];
        }
      if (hi >= 0) {
        spread += (uint64_t)(hi - lo);
        nonempty++;
      }
    }
    f[18 + e] = log2(1.0 + (nonempty > 0 ? (double)spread / (double)nonempty : 0.0));
  }
  /* the modified CMRS item counts (f24..f26) and the 32-row strip sizes */
  static const int pad_h[3] = {32, 32, 16}, pad_m[3] = {1, 2, 8};
  for (int q = 0; q < 3; ++q) {
    uint64_t items = 0;
    for (int s = 0; s * pad_h[q] < rows; ++s) {
      int r1 = (s + 1) * pad_h[q] < rows ? (s + 1) * pad_h[q] : rows;
      uint64_t ns = 0, ms = 0;
      for (int i = s * pad_h[q]; i < r1; ++i) {
        uint64_t l = (uint64_t)(row_ptr[i + 1] - row_ptr[i]);
        ns += l;
        if (l > ms) ms = l;
      }
      uint64_t by_items = (ns + 31) / 32, by_row = (ms + (uint64_t)pad_m[q] - 1) / (uint64_t)pad_m[q];
      items += 32 * (by_items > by_row ? by_items : by_row);
    }
    f[24 + q] = nnz > 0 ? log2((double)items / z) : 0.0;
  }
  uint64_t e32 = 0, e512 = 0, e8192 = 0;
  for (int i = 0; i < rows; ++i) {
    uint64_t l = (uint64_t)(row_ptr[i + 1] - row_ptr[i]);
    if (l >= 32) e32 += l;
    if (l >= 512) e512 += l;
    if (l >= 8192) e8192 += l;
  }
  f[27] = nnz > 0 ? (double)e32 / z : 0.0;
  f[28] = nnz > 0 ? (double)e512 / z : 0.0;
  f[29] = nnz > 0 ? (double)e8192 / z : 0.0;
  uint64_t sq = 0, smax = 0;
  int strips32 = (rows + 31) / 32;
  for (int s = 0; s < strips32; ++s) {
    int r1 = (s + 1) * 32 < rows ? (s + 1) * 32 : rows;
    uint64_t ns = (uint64_t)(row_ptr[r1] - row_ptr[s * 32]);
    sq += ns * ns;
    if (ns > smax) smax = ns;
  }
  double sm = z / (double)strips32;
  double svar = (double)sq / (double)strips32 - sm * sm;
  if (svar < 0.0) svar = 0.0;
  double sden = sm > 1.0 ? sm : 1.0;
  f[30] = sqrt(svar) / sden;
  f[31] = log2(1.0 + (double)smax / sden);
}

/* Selector network: nin -> nh (ReLU) -> nh (ReLU) -> nout, weights row-major
 * [out][in].  Z1/H1/Z2/H2/O are [B][*] buffers the caller provides. */
void orc_mlp_forward(int B, int nin, int nh, int nout, const double *X,
                     const double *W1, const double *b1, const double *W2,
                     const double *b2, const double *W3, const double *b3,
                     double *Z1, double *H1, double *Z2, double *H2, double *O) {
  for (int n = 0; n < B; ++n) {
    for (int j = 0; j < nh; ++j) {
      double s = b1[j];
      for (int i = 0; i < nin; ++i) s = s + W1[j * nin + i] * X[n * nin + i];
      Z1[n * nh + j] = s;
      H1[n * nh + j] = s > 0.0 ? s : 0.0;
    }
    for (int j = 0; j < nh; ++j) {
      double s = b2[j];
      for (int i = 0; i < nh; ++i) s = s + W2[j * nh + i] * H1[n * nh + i];
      Z2[n * nh + j] = s;
      H2[n * nh + j] = s > 0.0 ? s : 0.0;
    }
    for (int j = 0; j < nout; ++j) {
      double s = b3[j];
      for (int i = 0; i < nh; ++i) s = s + W3[j * nh + i] * H2[n * nh + i];
      O[n * nout + j] = s;
    }
  }
}

/* Loss L = 1/(2*B*nout) * sum (O - T)^2 and its gradient by the chain rule
 * (ReLU derivative taken as 1 for z > 0, else 0).  Returns L. */
double orc_mlp_backward(int B, int nin, int nh, int nout, const double *X,
                        const double *W2, const double *W3, const double *Z1,
                        const double *H1, const double *Z2, const double *H2,
                        const double *O, const double *T, double *dW1,
                        double *db1, double *dW2, double *db2, double *dW3,
                        double *db3) {
  double scale = 1.0 / ((double)B * (double)nout);
  double loss = 0.0;
  memset(dW1, 0, sizeof(double) * (size_t)nh * nin);
  memset(db1, 0, sizeof(double) * (size_t)nh);
  memset(dW2, 0, sizeof(double) * (size_t)nh * nh);
  memset(db2, 0, sizeof(double) * (size_t)nh);
  memset(dW3, 0, sizeof(double) * (size_t)nout * nh);
  memset(db3, 0, sizeof(double) * (size_t)nout);
  double *gO = (double *)malloc(sizeof(double) * (size_t)nout);
  double *g2 = (double *)malloc(sizeof(double) * (size_t)nh);
  double *g1 = (double *)malloc(sizeof(double) * (size_t)nh);
  for (int n = 0; n < B; ++n) {
    for (int j = 0; j < nout; ++j) {
      double e = O[n * nout + j] - T[n * nout + j];
      loss = loss + e * e;
      gO[j] = e * scale;
    }
    for (int j = 0; j < nout; ++j) {
      db3[j] = db3[j] + gO[j];
      for (int i = 0; i < nh; ++i) dW3[j * nh + i] = dW3[j * nh + i] + gO[j] * H2[n * nh + i];
    }
    for (int i = 0; i < nh; ++i) {
      double s = 0.0;
      for (int j = 0; j < nout; ++j) s = s + W3[j * nh + i] * gO[j];
      g2[i] = Z2[n * nh + i] > 0.0 ? s : 0.0;
    }
    for (int j = 0; j < nh; ++j) {
      db2[j] = db2[j] + g2[j];
      for (int i = 0; i < nh; ++i) dW2[j * nh + i] = dW2[j * nh + i] + g2[j] * H1[n * nh + i];
    }
    for (int i = 0; i < nh; ++i) {
      double s = 0.0;
      for (int j = 0; j < nh; ++j) s = s + W2[j * nh + i] * g2[j];
      g1[i] = Z1[n * nh + i] > 0.0 ? s : 0.0;
    }
    for (int j = 0; j < nh; ++j) {
      db1[j] = db1[j] + g1[j];
      for (int i = 0; i < nin; ++i) dW1[j * nin + i] = dW1[j * nin + i] + g1[j] * X[n * nin + i];
    }
  }
  free(gO);
  free(g2);
  free(g1);
  return 0.5 * loss * scale;
}

/* Adam (Kingma and Ba, 2015), one step at 1-based step count t:
 *   m = b1 m + (1-b1) g ; v = b2 v + (1-b2) g^2
 *   p = p - lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps) */
void orc_adam_step(int n, double *p, const double *g, double *m, double *v,
                   int t, double lr, double b1, double b2, double eps) {
  double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
  for (int k = 0; k < n; ++k) {
    m[k] = b1 * m[k] + (1.0 - b1) * g[k];
    v[k] = b2 * v[k] + (1.0 - b2) * g[k] * g[k];
    double mh = m[k] / c1, vh = v[k] / c2;
    p[k] = p[k] - lr * mh / (sqrt(vh) + eps);
  }
}

/* ------------------------------------------------------------------------ */
/* Section 6.6, modified CMRS.  Algorithm 1's per-warp buffer shrinks from
 * 32 x HEIGHT to M x HEIGHT when the lane that takes an item adds into slot
 * (lane mod M) of the item's row; that is race-free when two items of one
 * row handled in the same 32-item warp pass sit at positions that differ
 * mod M.  The section obtains this by rearranging each strip -- at most M
 * items of a row per pass, stored contiguously -- with explicit zeroes where
 * needed, and pads every strip to a multiple of 32 items.  The arrangement
 * itself is left open; the reading used here:
 *   - a strip becomes a sequence of 32-item chunks (one warp pass each);
 *   - as few chunks as the strip allows: C = max(ceil(items / 32),
 *     ceil(longest row / M)) for the items still left;
 *   - per chunk, every row first takes what it must so that the rest fits in
 *     C - 1 chunks, max(0, left - M (C - 1)) items (these fit: they sum to
 *     at most 32); the room still free then goes to rows in order of most
 *     items left after that (ties: lower row first), each topped up to
 *     min(M, left) items, until the chunk holds 32 items; items are taken in
 *     CRS order;
 *   - room still left is filled with zero items, rows 0 upwards, each row
 *     topped up to M items in the chunk (height * M >= 32 leaves room);
 *   - inside a chunk the rows appear in ascending order, each as one run:
 *     its real items, then its zero items.
 * A zero item has column 0 and value +0.0.  Input: unsorted strips
 * (RowInStrip non-decreasing inside each strip).  Output: the new StripPtr
 * (multiples of 32), the packed words, and src[i] = source position of item
 * i, or -1 for a zero item.  packed_out and src_out may be NULL (sizes
 * only).  Returns ORC_BAD_ARG for height * slots < 32 or a count overflow. */
int orc_pad_arrange(int rows, int height, int slots, const int32_t *strip_ptr,
                    const uint32_t *packed, int32_t *strip_ptr_out,
                    uint32_t *packed_out, int64_t *src_out) {
  int bits = orc_bits_for_height(height);
  if (bits < 0 || slots < 1 || slots > 32 || height * slots < 32) return ORC_BAD_ARG;
  int strips = (rows + height - 1) / height;
  uint32_t mask = (1u << bits) - 1;
  int64_t out = 0;
  strip_ptr_out[0] = 0;
  for (int s = 0; s < strips; ++s) {
    int64_t next[32], left[32];
    for (int r = 0; r < 32; ++r) left[r] = 0;
    for (int32_t k = strip_ptr[s]; k < strip_ptr[s + 1]; ++k) {
      uint32_t r = packed[k] & mask;
      if ((int)r >= height) return ORC_BAD_ARG;
      left[r] += 1;
    }
    /* rows are contiguous runs in RowInStrip order inside an unsorted strip */
    int64_t at = strip_ptr[s];
    for (int r = 0; r < height; ++r) {
      next[r] = at;
      at += left[r];
    }
    for (;;) {
      int64_t total = 0;
      for (int r = 0; r < height; ++r) total += left[r];
      if (total == 0) break;
      int64_t longest = 0;
      for (int r = 0; r < height; ++r)
        if (left[r] > longest) longest = left[r];
      int64_t chunks = (total + 31) / 32;
      if ((longest + slots - 1) / slots > chunks) chunks = (longest + slots - 1) / slots;
      int take[32], pad[32], served[32];
      for (int r = 0; r < 32; ++r) take[r] = pad[r] = served[r] = 0;
      int room = 32;
      for (int r = 0; r < height; ++r) {
        int64_t must = left[r] - (int64_t)slots * (chunks - 1);
        if (must > 0) {
          take[r] = (int)must;
          room -= (int)must;
        }
      }
      if (room < 0) return ORC_BAD_ARG; /* cannot happen: the musts sum to at most 32 */
      while (room > 0) {
        int best = -1;
        for (int r = 0; r < height; ++r)
          if (!served[r] && left[r] - take[r] > 0 && take[r] < slots &&
              (best < 0 || left[r] - take[r] > left[best] - take[best]))
            best = r;
        if (best < 0) break;
        served[best] = 1;
        int64_t cap = left[best] < slots ? left[best] : slots;
        int64_t t = cap - take[best];
        if (t > room) t = room;
        take[best] += (int)t;
        room -= (int)t;
      }
      for (int r = 0; r < height && room > 0; ++r) {
        int e = slots - take[r];
        if (e > room) e = room;
        pad[r] = e;
        room -= e;
      }
      for (int r = 0; r < height; ++r) {
        for (int j = 0; j < take[r]; ++j) {
          if (packed_out) packed_out[out] = packed[next[r]];
          if (src_out) src_out[out] = next[r];
          next[r] += 1;
          out += 1;
        }
        left[r] -= take[r];
        for (int j = 0; j < pad[r]; ++j) {
          if (packed_out) packed_out[out] = (uint32_t)r;
          if (src_out) src_out[out] = -1;
          out += 1;
        }
      }
    }
    if (out > 2147483647) return ORC_BAD_ARG;
    strip_ptr_out[s + 1] = (int32_t)out;
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Row reordering, the off-line optimisation the paper recommends for CMRS
 * (Section 7; Section 6.3 reads a low eta_+ as a sign that it would pay):
 * rows of similar length placed in the same strip need fewer zero items in
 * the modified form of Section 6.6.  The order used here: windows of
 * `window` consecutive rows (the last one may be shorter); inside a window,
 * rows by length, longest first, equal lengths in their original order.
 * perm[i] = the original row placed at position i.  A plain selection of the
 * longest remaining row, window by window. */
int orc_row_order(int rows, const int32_t *row_ptr, int window, int32_t *perm) {
  if (rows < 0 || window < 1) return ORC_BAD_ARG;
  char *taken = (char *)malloc((size_t)window);
  if (!taken) return ORC_BAD_ARG;
  for (int w0 = 0; w0 < rows; w0 += window) {
    int w1 = w0 + window < rows ? w0 + window : rows;
    memset(taken, 0, (size_t)window);
    for (int pos = w0; pos < w1; ++pos) {
      int best = -1;
      int32_t best_len = -1;
      for (int r = w0; r < w1; ++r) {
        if (taken[r - w0]) continue;
        int32_t len = row_ptr[r + 1] - row_ptr[r];
        if (len > best_len) {
          best_len = len;
          best = r;
        }
      }
      taken[best - w0] = 1;
      perm[pos] = best;
    }
  }
  free(taken);
  return ORC_OK;
}

/* CRS of the row-permuted matrix P A: row i is the original row perm[i],
 * its entries in their original order.  row_ptr_out [rows + 1]. */
void orc_permute_csr(int rows, const int32_t *row_ptr, const int32_t *col_ind,
                     const double *val, const int32_t *perm, int32_t *row_ptr_out,
                     int32_t *col_ind_out, double *val_out) {
  int32_t at = 0;
  row_ptr_out[0] = 0;
  for (int i = 0; i < rows; ++i) {
    int r = perm[i];
    for (int32_t k = row_ptr[r]; k < row_ptr[r + 1]; ++k) {
      col_ind_out[at] = col_ind[k];
      val_out[at] = val[k];
      at += 1;
    }
    row_ptr_out[i + 1] = at;
  }
}
