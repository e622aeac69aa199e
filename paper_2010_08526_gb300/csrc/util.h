// Host-callable wrappers of the helper kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace spg {

int64_t scan_partials_len(int64_t n);
// out[i] = sum_{j<i} in[j], i in [0, n) (and out[n] = total when write_total).
cudaError_t exclusive_scan_i64(const int64_t *in, int64_t n, int64_t *out, int64_t *partials,
                               int write_total, cudaStream_t st);
cudaError_t rebase_colptr(const int64_t *src, int64_t n, void *dst, int dst_is_i64,
                          cudaStream_t st);
cudaError_t validate_csc(const void *colptr, const void *rowidx, int idx64, int64_t ncols,
                         int64_t nrows, int64_t nnz, int *d_bad, cudaStream_t st);
cudaError_t column_bytes(const int64_t *cnt, const int64_t *extra, int64_t n, int64_t r,
                         int64_t ptr_bytes, int64_t *w, cudaStream_t st);
cudaError_t add_i64(int64_t *dst, const int64_t *src, int64_t n, cudaStream_t st);

__global__ void k_numeric_tier(const int64_t *cnt, const int64_t *dense_sel, int64_t c_lo,
                               int64_t c_hi, int hash_cap_max, uint8_t *tier_out,
                               int32_t *tier_hist);
__global__ void k_bin_scatter(const uint8_t *tier, int64_t c_lo, int64_t c_hi,
                              const int32_t *tier_hist, int32_t *cursor, int32_t *list,
                              int32_t *list_off, int32_t *heavy_ord);

}  // namespace spg
