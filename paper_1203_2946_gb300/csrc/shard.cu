// Row ranges for strip sharding over several GPUs.  Strips are independent
// (Section 4: each is processed by its own warp and touches only its own
// rows of y), so a matrix splits into contiguous ranges of whole strips, one
// per GPU, each multiplied on its own device once every device holds all of
// x.  This file only chooses the ranges; host code, no device work.
#include "common.cuh"

extern "C" int cmrs_shard_rows(int rows, const int32_t *row_ptr, int height, int parts, int32_t *bounds) {
  if (rows < 0 || parts < 1 || !bounds || (rows > 0 && !row_ptr)) return CMRS_ERR_ARG;
  if (height < 1 || height > 32) return CMRS_ERR_HEIGHT;
  if (rows > 0 && (row_ptr[0] != 0 || row_ptr[rows] < 0)) return CMRS_ERR_CSR_INVALID;
  const long long strips = (rows + (long long)height - 1) / height;
  // weight of the rows before strip s: its entries plus its rows (a row costs
  // its y write and its share of the strip bookkeeping even when empty)
  auto weight = [&](long long s) -> long long {
    const long long r = s * height < rows ? s * height : rows;
    return (long long)row_ptr[r] + r;
  };
  const long long total = weight(strips);
  bounds[0] = 0;
  long long lo_s = 0;
  for (int p = 1; p < parts; ++p) {
    // the first strip whose start carries at least p / parts of the weight
    const long long target = (total * p + parts - 1) / parts;
    long long lo = lo_s, hi = strips;
    while (lo < hi) {
      const long long mid = (lo + hi) >> 1;
      if (weight(mid) >= target) hi = mid;
      else lo = mid + 1;
    }
    lo_s = lo;
    const long long r = lo * height < rows ? lo * height : rows;
    bounds[p] = (int32_t)r;
  }
  bounds[parts] = rows;
  return CMRS_OK;
}
