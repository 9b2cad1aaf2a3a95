// Strip selector: per-matrix features on the device, a small MLP (forward,
// backward, Adam) in FP32, and cmrs_select_strip.  Not in the paper: Section
// 6.2 picks the strip height by brute force over all heights and Section 6.7
// measures how much per-matrix tuning gains; here a network trained on this
// library's own timings predicts the choice, with the brute-force sweep as
// fallback and as the yardstick of its regret.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace cmrs {
namespace {

constexpr int kNFeat = 32;
constexpr int kHeights[6] = {1, 2, 4, 8, 16, 32};
// choices 18, 19, 20: the modified CMRS of Section 6.6 at (height, slots)
constexpr int kPadChoice[3][2] = {{32, 1}, {32, 2}, {16, 8}};

struct FeatAcc {
  unsigned long long sum_l2, max_l, empty, same, near, sum_d, max_d;
  unsigned long long bins[8];
  unsigned long long spread[6], nonempty[6];
  // modified CMRS items at (32, 1), (32, 2), (16, 8); entries in rows of
  // >= 32, 512, 8192; sum of squares and max of 32-row strip entry counts
  unsigned long long pad[3], elong[3], s32_sq, s32_max;
};

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ unsigned long long warp_max(unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Row length statistics, |col - row| statistics and each row's min/max
// column (for the strip spreads).  A warp takes 32 consecutive rows at a
// time: lane r holds row r's bounds and length statistics; the rows' entries
// are one contiguous range, read in coalesced batches of 32 (kFeatU in
// flight per lane); an entry finds its row among the 32 row starts by a
// five-step shuffle search, adds its |col - row| to sums over all entries,
// and a segmented shuffle scan over the batch gives each row's min and max,
// which the row's lane carries over batches.  The strips of every height
// h = 2^e <= 32 are aligned groups of h lanes, so a shuffle tree over the
// rows' min and max gives each strip's column spread in the same pass, and
// one over the row lengths each 32- and 16-row strip's entry count and
// longest row (the modified CMRS pass counts).  A group with an invalid
// RowPtr range is skipped.
constexpr int kFeatU = 4;
__global__ void k_feat_rows(int rows, int nnz, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                            FeatAcc *acc) {
  __shared__ unsigned long long s[23], s_spread[6], s_ne[6];
  if (threadIdx.x < 23) s[threadIdx.x] = 0;
  if (threadIdx.x < 6) {
    s_spread[threadIdx.x] = 0;
    s_ne[threadIdx.x] = 0;
  }
  __syncthreads();
  const unsigned kAll = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long groups = ((long long)rows + 31) / 32;
  unsigned long long l2 = 0, mxl = 0, empty = 0, same = 0, near = 0, sd = 0, mxd = 0;
  unsigned long long bins[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  unsigned long long pad1 = 0, pad2 = 0, pad8 = 0, e32 = 0, e512 = 0, e8192 = 0, ssq = 0, smx = 0;
  for (long long g = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < groups; g += nw) {
    const long long r0 = g * 32, r = r0 + lane;
    const int nrows = (int)min(32LL, (long long)rows - r0);
    const int start = r < rows ? rp[r] : 0;
    const int last = rp[min(r0 + 32, (long long)rows)];
    int end = __shfl_down_sync(kAll, start, 1);
    if (lane == 31 || r + 1 >= rows) end = last;
    const bool ok = lane >= nrows || (start >= 0 && end >= start && end <= nnz);
    if (!__all_sync(kAll, ok)) continue;
    // row lengths (lane r)
    const int len = end - start;
    int lprev = __shfl_up_sync(kAll, len, 1);
    if (lane == 0) lprev = r0 > 0 ? start - rp[r0 - 1] : -1;
    if (lane < nrows) {
      const unsigned long long l = (unsigned long long)len;
      l2 += l * l;
      mxl = max(mxl, l);
      empty += l == 0;
      if (r > 0 && len == lprev) same++;
      if (l >= 1) {
        int bb = 0;
        while (bb < 7 && l >= (2ull << bb)) ++bb;
#pragma unroll
        for (int q = 0; q < 8; ++q) bins[q] += q == bb;  // registers, not a local array
      }
      e32 += l >= 32 ? l : 0ull;
      e512 += l >= 512 ? l : 0ull;
      e8192 += l >= 8192 ? l : 0ull;
    }
    // this group is strip g of height 32 and strips 2g, 2g+1 of height 16:
    // entries and longest row of each, by a shuffle tree over the lanes
    {
      unsigned long long ns = lane < nrows ? (unsigned long long)len : 0ull, ms = ns;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        if (o == 16 && (lane & 15) == 0) {  // the 16-row strips, before their halves meet
          const unsigned long long c = max((ns + 31) / 32, (ms + 7) / 8);
          pad8 += 32 * c;
        }
        ns += __shfl_xor_sync(kAll, ns, o);
        ms = max(ms, __shfl_xor_sync(kAll, ms, o));
      }
      if (lane == 0) {
        pad1 += 32 * ms;
        pad2 += 32 * max((ns + 31) / 32, (ms + 1) / 2);
        ssq += ns * ns;
        smx = max(smx, ns);
      }
    }
    // entries
    const int key = lane < nrows ? start : last;  // rows past the matrix sort last
    const int e0 = __shfl_sync(kAll, start, 0);
    int lo = INT32_MAX, hi = -1;  // row `lane`'s min and max column
    for (int k0 = e0; k0 < last; k0 += 32 * kFeatU) {
      int c[kFeatU];
#pragma unroll
      for (int u = 0; u < kFeatU; ++u) {
        const int k = k0 + 32 * u + lane;
        c[u] = k < last ? ci[k] : 0;
      }
#pragma unroll
      for (int u = 0; u < kFeatU; ++u) {
        const int kb = k0 + 32 * u;  // first entry of this batch
        if (kb >= last) break;       // warp-uniform
        const int k = kb + lane;
        const bool valid = k < last;
        int j = 0;  // row of entry k: the last of the group's rows starting at or before k
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
          const int sj = __shfl_sync(kAll, key, j + step);
          if (sj <= k) j += step;
        }
        if (valid) {
          const long long d = (long long)c[u] - (r0 + j);
          const unsigned long long ad = (unsigned long long)(d < 0 ? -d : d);
          sd += ad;
          mxd = max(mxd, ad);
          near += ad <= 64 ? 1ull : 0ull;
        }
        // min / max over the lanes of the same row in this batch
        const int seg = max(__shfl_sync(kAll, key, j), kb) - kb;  // first lane of row j in the batch
        int vmin = valid ? c[u] : INT32_MAX, vmax = valid ? c[u] : -1;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int tmin = __shfl_up_sync(kAll, vmin, o), tmax = __shfl_up_sync(kAll, vmax, o);
          if (lane - o >= seg) {
            vmin = min(vmin, tmin);
            vmax = max(vmax, tmax);
          }
        }
        // row `lane` takes the scan at its last entry in the batch
        const int my_e = min(end, kb + 32) - kb - 1;
        const bool mine = lane < nrows && max(start, kb) - kb <= my_e;
        const int m1 = __shfl_sync(kAll, vmin, mine ? my_e : 0), m2 = __shfl_sync(kAll, vmax, mine ? my_e : 0);
        if (mine) {
          lo = min(lo, m1);
          hi = max(hi, m2);
        }
      }
    }
    // strip spreads: after step e each lane holds the min and max of its
    // aligned group of 2^e rows (rows past the matrix, and empty rows, are
    // neutral); the group's first lane counts the strip if it has entries
    int slo = lane < nrows ? lo : INT32_MAX, shi = lane < nrows ? hi : -1;
#pragma unroll
    for (int e = 0; e < 6; ++e) {
      if (e > 0) {
        slo = min(slo, __shfl_xor_sync(kAll, slo, 1 << (e - 1)));
        shi = max(shi, __shfl_xor_sync(kAll, shi, 1 << (e - 1)));
      }
      const bool counted = (lane & ((1 << e) - 1)) == 0 && shi >= 0;
      const unsigned long long sp = warp_sum(counted ? (unsigned long long)(shi - slo) : 0ull);
      const unsigned long long ne = warp_sum(counted ? 1ull : 0ull);
      if (lane == 0 && ne) {
        atomicAdd(&s_spread[e], sp);
        atomicAdd(&s_ne[e], ne);
      }
    }
  }
  l2 = warp_sum(l2);
  mxl = warp_max(mxl);
  empty = warp_sum(empty);
  same = warp_sum(same);
  near = warp_sum(near);
  sd = warp_sum(sd);
  mxd = warp_max(mxd);
  for (int bb = 0; bb < 8; ++bb) bins[bb] = warp_sum(bins[bb]);
  pad1 = warp_sum(pad1);
  pad2 = warp_sum(pad2);
  pad8 = warp_sum(pad8);
  e32 = warp_sum(e32);
  e512 = warp_sum(e512);
  e8192 = warp_sum(e8192);
  ssq = warp_sum(ssq);
  smx = warp_max(smx);
  if (lane == 0) {
    atomicAdd(&s[0], l2);
    atomicMax(&s[1], mxl);
    atomicAdd(&s[2], empty);
    atomicAdd(&s[3], same);
    atomicAdd(&s[4], near);
    atomicAdd(&s[5], sd);
    atomicMax(&s[6], mxd);
    for (int bb = 0; bb < 8; ++bb) atomicAdd(&s[7 + bb], bins[bb]);
    atomicAdd(&s[15], pad1);
    atomicAdd(&s[16], pad2);
    atomicAdd(&s[17], pad8);
    atomicAdd(&s[18], e32);
    atomicAdd(&s[19], e512);
    atomicAdd(&s[20], e8192);
    atomicAdd(&s[21], ssq);
    atomicMax(&s[22], smx);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    atomicAdd(&acc->sum_l2, s[0]);
    atomicMax(&acc->max_l, s[1]);
    atomicAdd(&acc->empty, s[2]);
    atomicAdd(&acc->same, s[3]);
    atomicAdd(&acc->near, s[4]);
    atomicAdd(&acc->sum_d, s[5]);
    atomicMax(&acc->max_d, s[6]);
    for (int bb = 0; bb < 8; ++bb) atomicAdd(&acc->bins[bb], s[7 + bb]);
    for (int q = 0; q < 3; ++q) {
      atomicAdd(&acc->pad[q], s[15 + q]);
      atomicAdd(&acc->elong[q], s[18 + q]);
    }
    atomicAdd(&acc->s32_sq, s[21]);
    atomicMax(&acc->s32_max, s[22]);
  }
  if (threadIdx.x < 6) {
    atomicAdd(&acc->spread[threadIdx.x], s_spread[threadIdx.x]);
    atomicAdd(&acc->nonempty[threadIdx.x], s_ne[threadIdx.x]);
  }
}

// The 32 features from the integer sums, with the same operations, in the
// same order, as their definition (no contraction into FMAs); thread t
// computes feature t.
__global__ void k_feat_final(int rows, int nnz, const FeatAcc *acc, double *f) {
  const int t = threadIdx.x;
  if (blockIdx.x != 0 || t >= kNFeat) return;
  const double n = (double)rows, z = (double)nnz;
  const double mu = __ddiv_rn(z, n);
  double v;
  if (t == 0) {
    v = log2(n);
  } else if (t == 1) {
    v = log2(z > 1.0 ? z : 1.0);
  } else if (t == 2) {
    v = log2(__dadd_rn(1.0, mu));
  } else if (t == 3) {
    double var = __dsub_rn(__ddiv_rn((double)acc->sum_l2, n), __dmul_rn(mu, mu));
    if (var < 0.0) var = 0.0;
    v = __ddiv_rn(sqrt(var), mu > 1.0 ? mu : 1.0);
  } else if (t == 4) {
    v = log2(__dadd_rn(1.0, (double)acc->max_l));
  } else if (t == 5) {
    v = __ddiv_rn((double)acc->empty, n);
  } else if (t < 14) {
    v = __ddiv_rn((double)acc->bins[t - 6], n);
  } else if (t == 14) {
    v = log2(__dadd_rn(1.0, nnz > 0 ? __ddiv_rn((double)acc->sum_d, z) : 0.0));
  } else if (t == 15) {
    v = log2(__dadd_rn(1.0, (double)acc->max_d));
  } else if (t == 16) {
    v = nnz > 0 ? __ddiv_rn((double)acc->near, z) : 0.0;
  } else if (t == 17) {
    v = rows > 1 ? __ddiv_rn((double)acc->same, (double)(rows - 1)) : 0.0;
  } else if (t < 24) {
    const double ne = (double)acc->nonempty[t - 18];
    v = log2(__dadd_rn(1.0, ne > 0 ? __ddiv_rn((double)acc->spread[t - 18], ne) : 0.0));
  } else if (t < 27) {
    v = nnz > 0 ? log2(__ddiv_rn((double)acc->pad[t - 24], z)) : 0.0;
  } else if (t < 30) {
    v = nnz > 0 ? __ddiv_rn((double)acc->elong[t - 27], z) : 0.0;
  } else {
    const double ns = (double)((rows + 31) / 32);
    const double sm = __ddiv_rn(z, ns);
    const double sden = sm > 1.0 ? sm : 1.0;
    if (t == 30) {
      double var = __dsub_rn(__ddiv_rn((double)acc->s32_sq, ns), __dmul_rn(sm, sm));
      if (var < 0.0) var = 0.0;
      v = __ddiv_rn(sqrt(var), sden);
    } else {
      v = log2(__dadd_rn(1.0, __ddiv_rn((double)acc->s32_max, sden)));
    }
  }
  f[t] = v;
}

// ------------------------------------------------------------------ MLP (FP32)
// Z[n][j] = b[j] + sum_i W[j][i] X[n][i]; H = relu(Z) (or Z for the output).
__global__ void k_dense_fwd(int B, int nin, int nout, const float *__restrict__ X, const float *__restrict__ W,
                            const float *__restrict__ bias, float *__restrict__ Z, float *__restrict__ H, int relu) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * nout) return;
  const int n = t / nout, j = t - n * nout;
  float s = bias[j];
  for (int i = 0; i < nin; ++i) s = fmaf(W[j * nin + i], X[n * nin + i], s);
  if (Z) Z[t] = s;
  if (H) H[t] = relu ? fmaxf(s, 0.f) : s;
}

// gO = (O - T) / (B * nout); loss = sum (O - T)^2 / (2 B nout), one block.
__global__ void k_out_grad(int total, float scale, const float *__restrict__ O, const float *__restrict__ T,
                           float *__restrict__ G, float *loss) {
  __shared__ float part[256];
  float s = 0.f;
  for (int i = threadIdx.x; i < total; i += blockDim.x) {
    const float e = O[i] - T[i];
    G[i] = e * scale;
    s = fmaf(e, e, s);
  }
  part[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0 && loss) *loss = 0.5f * part[0] * scale;
}

// dW[j][i] = sum_n G[n][j] H[n][i]; db[j] = sum_n G[n][j] (thread per (j, i),
// i == nin for the bias); sums run over n in order.
__global__ void k_weight_grad(int B, int nin, int nout, const float *__restrict__ G, const float *__restrict__ H,
                              float *__restrict__ dW, float *__restrict__ db) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nout * (nin + 1)) return;
  const int j = t / (nin + 1), i = t - j * (nin + 1);
  float s = 0.f;
  if (i < nin) {
    for (int n = 0; n < B; ++n) s = fmaf(G[n * nout + j], H[n * nin + i], s);
    dW[j * nin + i] = s;
  } else {
    for (int n = 0; n < B; ++n) s += G[n * nout + j];
    db[j] = s;
  }
}

// Gin[n][i] = (Z[n][i] > 0) * sum_j W[j][i] G[n][j]
__global__ void k_back_hidden(int B, int nin, int nout, const float *__restrict__ G, const float *__restrict__ W,
                              const float *__restrict__ Z, float *__restrict__ Gin) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * nin) return;
  const int n = t / nin, i = t - n * nin;
  float s = 0.f;
  for (int j = 0; j < nout; ++j) s = fmaf(W[j * nin + i], G[n * nout + j], s);
  Gin[t] = Z[t] > 0.f ? s : 0.f;
}

// Adam (Kingma and Ba 2015); c1 = 1 - beta1^t, c2 = 1 - beta2^t.
__global__ void k_adam(int n, float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// x = (f - mean) * scale as FP32 network input; then the argmin of the
// network's predicted cost over the choices.
__global__ void k_normalize(int nf, const double *__restrict__ f, const float *__restrict__ mean,
                            const float *__restrict__ scale, float *__restrict__ x) {
  const int i = threadIdx.x;
  if (i < nf) x[i] = ((float)f[i] - mean[i]) * scale[i];
}

__global__ void k_argmin(int n, const float *__restrict__ o, int *__restrict__ out) {
  if (threadIdx.x != 0) return;
  int best = 0;
  for (int i = 1; i < n; ++i)
    if (o[i] < o[best]) best = i;
  *out = best;
}

inline int grid_for(long long n, int t) { return (int)std::max<long long>(1, (n + t - 1) / t); }

size_t param_count(int nin, int nh, int nout) {
  return (size_t)nh * nin + nh + (size_t)nh * nh + nh + (size_t)nout * nh + nout;
}

size_t features_ws(int rows) {
  (void)rows;
  return align256(sizeof(FeatAcc));
}

}  // namespace
}  // namespace cmrs

using namespace cmrs;

extern "C" int cmrs_features_workspace(int rows, size_t *bytes) {
  if (rows < 0 || !bytes) return CMRS_ERR_ARG;
  *bytes = features_ws(rows);
  return CMRS_OK;
}

extern "C" int cmrs_features(int rows, int nnz, const int32_t *row_ptr, const int32_t *col_ind, double *feat,
                             void *workspace, size_t workspace_bytes, void *stream) {
  CMRS_TRACE();
  if (rows < 1 || nnz < 0 || !row_ptr || !feat || (nnz > 0 && !col_ind)) return CMRS_ERR_ARG;
  if (!workspace || workspace_bytes < features_ws(rows) || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return CMRS_ERR_WORKSPACE;
  cudaStream_t st = as_stream(stream);
  char *ws = reinterpret_cast<char *>(workspace);
  FeatAcc *acc = reinterpret_cast<FeatAcc *>(ws);
  CMRS_CUDA_TRY(cudaMemsetAsync(acc, 0, sizeof(FeatAcc), st));
  const int sms = sm_count();
  const int g = (int)std::min<long long>(ceil_div((long long)rows, 256), (long long)sms * 8);  // 8 warps x 32 rows
  k_feat_rows<<<g, 256, 0, st>>>(rows, nnz, row_ptr, col_ind, acc);
  CMRS_LAUNCH_CHECK();
  k_feat_final<<<1, 32, 0, st>>>(rows, nnz, acc, feat);
  CMRS_LAUNCH_CHECK();
  return CMRS_OK;
}

extern "C" int64_t cmrs_mlp_param_count(int nin, int nh, int nout) {
  if (nin < 1 || nh < 1 || nout < 1) return -1;
  return (int64_t)param_count(nin, nh, nout);
}

// acts layout: Z1[B][nh], H1[B][nh], Z2[B][nh], H2[B][nh], O[B][nout]
extern "C" int cmrs_mlp_forward(int B, int nin, int nh, int nout, const float *X, const float *params, float *acts,
                                void *stream) {
  CMRS_TRACE();
  if (B < 1 || nin < 1 || nh < 1 || nout < 1 || !X || !params || !acts) return CMRS_ERR_ARG;
  cudaStream_t st = as_stream(stream);
  const float *W1 = params, *b1 = W1 + (size_t)nh * nin, *W2 = b1 + nh, *b2 = W2 + (size_t)nh * nh, *W3 = b2 + nh,
              *b3 = W3 + (size_t)nout * nh;
  float *Z1 = acts, *H1 = Z1 + (size_t)B * nh, *Z2 = H1 + (size_t)B * nh, *H2 = Z2 + (size_t)B * nh,
        *O = H2 + (size_t)B * nh;
  k_dense_fwd<<<grid_for((long long)B * nh, 128), 128, 0, st>>>(B, nin, nh, X, W1, b1, Z1, H1, 1);
  k_dense_fwd<<<grid_for((long long)B * nh, 128), 128, 0, st>>>(B, nh, nh, H1, W2, b2, Z2, H2, 1);
  k_dense_fwd<<<grid_for((long long)B * nout, 128), 128, 0, st>>>(B, nh, nout, H2, W3, b3, nullptr, O, 0);
  CMRS_LAUNCH_CHECK();
  return CMRS_OK;
}

// Loss 1/(2 B nout) sum (O - T)^2 and its gradient (same layout as params).
// scratch: B * (nout + 2 nh) floats.  loss: device float (may be NULL).
extern "C" int cmrs_mlp_backward(int B, int nin, int nh, int nout, const float *X, const float *T,
                                 const float *params, const float *acts, float *grads, float *scratch, float *loss,
                                 void *stream) {
  CMRS_TRACE();
  if (B < 1 || nin < 1 || nh < 1 || nout < 1 || !X || !T || !params || !acts || !grads || !scratch)
    return CMRS_ERR_ARG;
  cudaStream_t st = as_stream(stream);
  const float *W2 = params + (size_t)nh * nin + nh, *W3 = W2 + (size_t)nh * nh + nh;
  const float *Z1 = acts, *H1 = Z1 + (size_t)B * nh, *Z2 = H1 + (size_t)B * nh, *H2 = Z2 + (size_t)B * nh,
              *O = H2 + (size_t)B * nh;
  float *dW1 = grads, *db1 = dW1 + (size_t)nh * nin, *dW2 = db1 + nh, *db2 = dW2 + (size_t)nh * nh,
        *dW3 = db2 + nh, *db3 = dW3 + (size_t)nout * nh;
  float *gO = scratch, *g2 = gO + (size_t)B * nout, *g1 = g2 + (size_t)B * nh;
  const float scale = 1.0f / ((float)B * (float)nout);
  k_out_grad<<<1, 256, 0, st>>>(B * nout, scale, O, T, gO, loss);
  k_weight_grad<<<grid_for((long long)nout * (nh + 1), 128), 128, 0, st>>>(B, nh, nout, gO, H2, dW3, db3);
  k_back_hidden<<<grid_for((long long)B * nh, 128), 128, 0, st>>>(B, nh, nout, gO, W3, Z2, g2);
  k_weight_grad<<<grid_for((long long)nh * (nh + 1), 128), 128, 0, st>>>(B, nh, nh, g2, H1, dW2, db2);
  k_back_hidden<<<grid_for((long long)B * nh, 128), 128, 0, st>>>(B, nh, nh, g2, W2, Z1, g1);
  k_weight_grad<<<grid_for((long long)nh * (nin + 1), 128), 128, 0, st>>>(B, nin, nh, g1, X, dW1, db1);
  CMRS_LAUNCH_CHECK();
  return CMRS_OK;
}

extern "C" int cmrs_mlp_adam(int n, float *params, const float *grads, float *m, float *v, int step, float lr,
                             float beta1, float beta2, float eps, void *stream) {
  CMRS_TRACE();
  if (n < 1 || !params || !grads || !m || !v || step < 1) return CMRS_ERR_ARG;
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  k_adam<<<grid_for(n, 256), 256, 0, as_stream(stream)>>>(n, params, grads, m, v, lr, beta1, beta2, eps, c1, c2);
  CMRS_LAUNCH_CHECK();
  return CMRS_OK;
}

// ------------------------------------------------------------------ selection
// Padded forms the exhaustive sweep times must fit this many items; a form
// padded beyond it (more than twice the entries) is not a candidate.
static size_t pad_cap(int rows, int nnz) { return 2 * (size_t)nnz + 32 * ((size_t)rows / 16 + 2); }

static size_t select_ws(int rows, int cols, int nnz, int exhaustive) {
  size_t b = features_ws(rows) + align256(kNFeat * 8) + align256(1024 * 4) + align256(64);
  if (exhaustive) {
    const size_t strips = (size_t)rows + 1;
    b += align256(strips * 4) + align256((size_t)std::max(nnz, 1) * 4) * 3 + align256((size_t)std::max(cols, 1) * 4) +
         align256((size_t)std::max(rows, 1) * 4);
    size_t s = 0;
    cmrs_from_csr_workspace(rows, nnz, 1, 0, CMRS_F32, &s);
    b += align256(s);
    // padded forms: StripPtr, items (packed + FP32 values) and the layout pass's workspace
    b += align256(((size_t)rows / 16 + 2) * 4) + 2 * align256(pad_cap(rows, nnz) * 4) + align256(256) +
         align256(((size_t)rows / 16 + 2) * 4) + align256(((size_t)rows / 16 + 2) * 8) + align256(((size_t)rows / 16 / 1024 + 2) * 8);
    b += align256(merge_workspace_bytes(nnz, CMRS_F32) + 4096);
  }
  return b;
}

// ------------------------------------------------------------------ training data
namespace cmrs {
namespace {
// Feature j's mean and population standard deviation over the B rows, summed
// in row order in FP64 (one thread per feature); scale = 1 / std, or 0 for a
// feature that does not vary (it then leaves the network's input).
__global__ void k_feat_stats(int B, int nin, const double *__restrict__ F, float *__restrict__ mean,
                             float *__restrict__ scale) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nin) return;
  double s = 0.0;
  for (int n = 0; n < B; ++n) s = __dadd_rn(s, F[(size_t)n * nin + j]);
  const double m = __ddiv_rn(s, (double)B);
  double q = 0.0;
  for (int n = 0; n < B; ++n) {
    const double d = __dsub_rn(F[(size_t)n * nin + j], m);
    q = __dadd_rn(q, __dmul_rn(d, d));
  }
  const double sd = sqrt(__ddiv_rn(q, (double)B));
  mean[j] = (float)m;
  scale[j] = sd > 1e-12 ? (float)__ddiv_rn(1.0, sd) : 0.f;
}

// X = (F - mean) * scale in FP32, row-major [B][nin].
__global__ void k_feat_apply(int total, int nin, const double *__restrict__ F, const float *__restrict__ mean,
                             const float *__restrict__ scale, float *__restrict__ X) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  const int j = t % nin;
  X[t] = ((float)F[t] - mean[j]) * scale[j];
}

// T[n][c] = min(log2(t[n][c] / min_c t[n][c]), cap): each choice's cost
// relative to the row's best, one thread per row.
__global__ void k_cost_targets(int B, int nout, const double *__restrict__ times, float cap, float *__restrict__ T) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= B) return;
  const double *t = times + (size_t)n * nout;
  double best = t[0];
  for (int c = 1; c < nout; ++c) best = t[c] < best ? t[c] : best;
  for (int c = 0; c < nout; ++c) {
    const double r = log2(__ddiv_rn(t[c], best));
    T[(size_t)n * nout + c] = (float)(r < (double)cap ? r : (double)cap);
  }
}
}  // namespace
}  // namespace cmrs

extern "C" int cmrs_feature_norm(int B, int nin, const double *F, float *mean, float *scale, float *X, void *stream) {
  CMRS_TRACE();
  if (B < 1 || nin < 1 || !F || !mean || !scale) return CMRS_ERR_ARG;
  cudaStream_t st = as_stream(stream);
  k_feat_stats<<<(nin + 63) / 64, 64, 0, st>>>(B, nin, F, mean, scale);
  CMRS_LAUNCH_CHECK();
  if (X) {
    const long long total = (long long)B * nin;
    if (total >= (1LL << 31)) return CMRS_ERR_ARG;
    k_feat_apply<<<(int)ceil_div(total, 256), 256, 0, st>>>((int)total, nin, F, mean, scale, X);
    CMRS_LAUNCH_CHECK();
  }
  return CMRS_OK;
}

extern "C" int cmrs_feature_apply(int B, int nin, const double *F, const float *mean, const float *scale, float *X,
                                  void *stream) {
  CMRS_TRACE();
  const long long total = (long long)B * nin;
  if (B < 1 || nin < 1 || !F || !mean || !scale || !X || total >= (1LL << 31)) return CMRS_ERR_ARG;
  k_feat_apply<<<(int)ceil_div(total, 256), 256, 0, as_stream(stream)>>>((int)total, nin, F, mean, scale, X);
  CMRS_LAUNCH_CHECK();
  return CMRS_OK;
}

extern "C" int cmrs_cost_targets(int B, int nout, const double *times, float cap, float *T, void *stream) {
  CMRS_TRACE();
  if (B < 1 || nout < 1 || !times || !T || !(cap > 0.f)) return CMRS_ERR_ARG;
  k_cost_targets<<<(B + 127) / 128, 128, 0, as_stream(stream)>>>(B, nout, times, cap, T);
  CMRS_LAUNCH_CHECK();
  return CMRS_OK;
}

extern "C" int cmrs_select_strip_workspace(int rows, int cols, int nnz, int exhaustive, size_t *bytes) {
  if (rows < 1 || cols < 1 || nnz < 0 || !bytes) return CMRS_ERR_ARG;
  *bytes = select_ws(rows, cols, nnz, exhaustive);
  return CMRS_OK;
}

__global__ void k_fill(float *p, long long n, float v) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = v;
}

extern "C" int cmrs_select_strip(int rows, int cols, int nnz, const int32_t *row_ptr, const int32_t *col_ind,
                                 const cmrs_selector *model, int *height_out, int *variant_out, int *slots_out,
                                 void *workspace, size_t workspace_bytes, void *stream) {
  CMRS_TRACE();
  if (rows < 1 || cols < 1 || nnz < 0 || !row_ptr || !height_out || !variant_out || !slots_out) return CMRS_ERR_ARG;
  const int exhaustive = model == nullptr;
  const size_t need = select_ws(rows, cols, nnz, exhaustive);
  if (!workspace || workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255)) return CMRS_ERR_WORKSPACE;
  cudaStream_t st = as_stream(stream);
  char *ws = reinterpret_cast<char *>(workspace);
  size_t off = features_ws(rows);
  double *feat = reinterpret_cast<double *>(ws + off);
  off += align256(kNFeat * 8);
  float *buf = reinterpret_cast<float *>(ws + off);
  off += align256(1024 * 4);
  int *choice = reinterpret_cast<int *>(ws + off);
  off += align256(64);
  if (!exhaustive) {
    if (model->nin != kNFeat || model->nout != CMRS_SEL_CHOICES || model->nh < 1 || model->nh > 64 || !model->params ||
        !model->feat_mean || !model->feat_scale)
      return CMRS_ERR_ARG;
    int rc = cmrs_features(rows, nnz, row_ptr, col_ind, feat, workspace, features_ws(rows), stream);
    if (rc) return rc;
    const int nh = model->nh, nout = model->nout;
    float *x = buf, *acts = buf + 32;  // 4*nh + nout <= 4*64 + 21 floats fit in the 992 left
    k_normalize<<<1, 32, 0, st>>>(kNFeat, feat, model->feat_mean, model->feat_scale, x);
    rc = cmrs_mlp_forward(1, kNFeat, nh, nout, x, model->params, acts, stream);
    if (rc) return rc;
    k_argmin<<<1, 32, 0, st>>>(nout, acts + 4 * nh, choice);
    CMRS_LAUNCH_CHECK();
    int c = 0;
    CMRS_CUDA_TRY(cudaMemcpyAsync(&c, choice, sizeof(int), cudaMemcpyDeviceToHost, st));
    CMRS_CUDA_TRY(cudaStreamSynchronize(st));
    if (c < 18) {
      *height_out = kHeights[c / 3];
      *variant_out = c % 3;
      *slots_out = 0;
    } else {
      *height_out = kPadChoice[c - 18][0];
      *variant_out = CMRS_VARIANT_PADDED;
      *slots_out = kPadChoice[c - 18][1];
    }
    return CMRS_OK;
  }
  // Exhaustive autotune (Section 6.2's brute force): convert with every
  // height and time every variant; the values are ones (timing does not
  // depend on them).
  int32_t *sp = reinterpret_cast<int32_t *>(ws + off);
  off += align256(((size_t)rows + 1) * 4);
  uint32_t *pk = reinterpret_cast<uint32_t *>(ws + off);
  off += align256((size_t)std::max(nnz, 1) * 4);
  float *val = reinterpret_cast<float *>(ws + off);
  off += align256((size_t)std::max(nnz, 1) * 4);
  float *ones = reinterpret_cast<float *>(ws + off);
  off += align256((size_t)std::max(nnz, 1) * 4);
  float *x = reinterpret_cast<float *>(ws + off);
  off += align256((size_t)cols * 4);
  float *y = reinterpret_cast<float *>(ws + off);
  off += align256((size_t)rows * 4);
  size_t cws = 0;
  cmrs_from_csr_workspace(rows, nnz, 1, 0, CMRS_F32, &cws);
  char *conv_ws = ws + off;
  off += align256(cws);
  const size_t cap = pad_cap(rows, nnz);
  int32_t *psp = reinterpret_cast<int32_t *>(ws + off);
  off += align256(((size_t)rows / 16 + 2) * 4);
  uint32_t *ppk = reinterpret_cast<uint32_t *>(ws + off);
  off += align256(cap * 4);
  float *pval = reinterpret_cast<float *>(ws + off);
  off += align256(cap * 4);
  char *pad_ws = ws + off;
  const size_t pad_ws_bytes = align256(256) + align256(((size_t)rows / 16 + 2) * 4) +
                              align256(((size_t)rows / 16 + 2) * 8) + align256(((size_t)rows / 16 / 1024 + 2) * 8);
  off += pad_ws_bytes;
  char *spmv_ws = ws + off;
  const size_t spmv_bytes = workspace_bytes - off;
  k_fill<<<grid_for(std::max(nnz, 1), 256), 256, 0, st>>>(ones, std::max(nnz, 1), 1.f);
  k_fill<<<grid_for(cols, 256), 256, 0, st>>>(x, cols, 1.f);
  CMRS_LAUNCH_CHECK();
  CMRS_CUDA_TRY(cudaMemsetAsync(spmv_ws, 0, 256, st));
  cudaEvent_t e0, e1;
  CMRS_CUDA_TRY(cudaEventCreate(&e0));
  CMRS_CUDA_TRY(cudaEventCreate(&e1));
  float best = 1e30f;
  int bh = 4, bv = 0, bm = 0, rc = CMRS_OK;
  auto time_one = [&](const cmrs_matrix *M, int v, int h, int m) {
    for (int w = 0; w < 2 && rc == CMRS_OK; ++w) rc = cmrs_spmv(M, x, y, v, spmv_ws, spmv_bytes, stream);
    cudaEventRecord(e0, st);
    for (int r = 0; r < 5 && rc == CMRS_OK; ++r) rc = cmrs_spmv(M, x, y, v, spmv_ws, spmv_bytes, stream);
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess && rc == CMRS_OK) rc = set_cuda_error(e);
    if (rc == CMRS_OK && ms < best) {
      best = ms;
      bh = h;
      bv = v;
      bm = m;
    }
  };
  for (int hi = 0; hi < 6 && rc == CMRS_OK; ++hi) {
    cmrs_matrix A;
    rc = cmrs_from_csr(rows, cols, nnz, row_ptr, col_ind, ones, CMRS_F32, kHeights[hi], 0, CMRS_F32, sp, pk, val,
                       conv_ws, cws, stream, &A);
    for (int v = 0; v < 3 && rc == CMRS_OK; ++v) time_one(&A, v, kHeights[hi], 0);
    // the padded forms built from this height's CMRS
    for (int j = 0; j < 3 && rc == CMRS_OK; ++j) {
      if (kPadChoice[j][0] != kHeights[hi]) continue;
      int32_t npad = 0;
      rc = cmrs_pad_layout(&A, kPadChoice[j][1], psp, &npad, pad_ws, pad_ws_bytes, stream);
      if (rc == CMRS_OK && (size_t)npad <= cap) {
        cmrs_matrix P;
        rc = cmrs_pad_fill(&A, kPadChoice[j][1], psp, npad, ppk, pval, stream, &P);
        if (rc == CMRS_OK) time_one(&P, CMRS_VARIANT_PADDED, kHeights[hi], kPadChoice[j][1]);
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  *height_out = bh;
  *variant_out = bv;
  *slots_out = bm;
  return CMRS_OK;
}
