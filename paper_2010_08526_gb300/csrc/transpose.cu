// spgemm_transpose: the CSC of A^T (equivalently the CSR of A) on the device.
// A^T serves A A^T (Sec. V's BELLA workload) and the row-by-row batching the
// paper mentions for square inputs (Sec. IV-B): the row batches of C = A B
// are the column batches of C^T = B^T A^T.
//
//   1. count[i] = entries in row i of A      (one atomic per entry)
//   2. colptr of A^T = exclusive scan of count
//   3. every entry (i, j, v) of A goes to a slot of column i of A^T, taken
//      with an atomic cursor: row index j, value v.
// Values are moved as raw 4- or 8-byte words. Rows inside an output column
// come in an unspecified order (as every output of the library).
#include <algorithm>
#include <string>

#include "../../include/spgemm.h"
#include "plan.h"
#include "util.h"

namespace spg {

// rows outside [0, m) are skipped and flagged (corrupt input)
template <class I>
__global__ void k_t_count(const I *rowidx, int64_t nnz, int64_t m, unsigned long long *count, int *err) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nnz; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = (int64_t)rowidx[q];
        if (i < 0 || i >= m) { atomicOr(err, 1); continue; }
        atomicAdd(&count[i], 1ull);
    }
}

// one warp per input column
template <class P, class I, class W>
__global__ void k_t_scatter(const P *colptr, const I *rowidx, const W *vals, int64_t ncols, int64_t m,
                            unsigned long long *cursor, I *out_rows, W *out_vals) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t base = (int64_t)colptr[0];
    for (int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < ncols; j += nw) {
        const int64_t a = (int64_t)colptr[j] - base, b = (int64_t)colptr[j + 1] - base;
        for (int64_t q = a + lane; q < b; q += 32) {
            const int64_t i = (int64_t)rowidx[q];
            if (i < 0 || i >= m) continue;
            const unsigned long long pos = atomicAdd(&cursor[i], 1ull);
            out_rows[pos] = (I)j;
            out_vals[pos] = vals[q];
        }
    }
}

template <class T>
__global__ void k_t_colptr(const int64_t *src, int64_t n, T *dst) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (T)src[i];
}

template <class P, class I, class W>
static spgemm_status transpose_typed(const spgemm_csc *in, spgemm_csc *out, cudaStream_t st) {
    const int64_t m = in->nrows, n = in->ncols, nnz = in->nnz;
    DevBuf count, scan, part, err;
    cudaError_t e;
    if ((e = count.ensure(sizeof(int64_t) * (size_t)(m + 1))) != cudaSuccess ||
        (e = scan.ensure(sizeof(int64_t) * (size_t)(m + 1))) != cudaSuccess ||
        (e = part.ensure(sizeof(int64_t) * (size_t)scan_partials_len(m + 1))) != cudaSuccess ||
        (e = err.ensure(sizeof(int) * 4)) != cudaSuccess) {
        if (e == cudaErrorMemoryAllocation) {
            set_error("transpose: workspace allocation failed");
            return SPGEMM_ERR_OOM;
        }
        return cuda_fail(e, "transpose workspace");
    }
    if ((e = cudaMemsetAsync(count.p, 0, sizeof(int64_t) * (size_t)(m + 1), st)) != cudaSuccess ||
        (e = cudaMemsetAsync(err.p, 0, sizeof(int), st)) != cudaSuccess)
        return cuda_fail(e, "cudaMemsetAsync");
    const unsigned eb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((nnz + 255) / 256, 1 << 20));
    const unsigned cb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 7) / 8, 1 << 20));
    const unsigned mb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((m + 256) / 256, 1 << 20));
    // entry q of the input is rowidx[q - colptr[0]] (the pointers address
    // the first entry), as everywhere in the library
    if (nnz > 0)
        k_t_count<I><<<eb, 256, 0, st>>>((const I *)in->rowidx, nnz, m, count.as<unsigned long long>(), err.as<int>());
    if ((e = exclusive_scan_i64(count.as<int64_t>(), m, scan.as<int64_t>(), part.as<int64_t>(), 1, st)) != cudaSuccess)
        return cuda_fail(e, "scan");
    if (out->ptr_type == SPGEMM_I64) k_t_colptr<int64_t><<<mb, 256, 0, st>>>(scan.as<int64_t>(), m + 1, (int64_t *)out->colptr);
    else k_t_colptr<int32_t><<<mb, 256, 0, st>>>(scan.as<int64_t>(), m + 1, (int32_t *)out->colptr);
    if (nnz > 0)
        k_t_scatter<P, I, W><<<cb, 256, 0, st>>>((const P *)in->colptr, (const I *)in->rowidx, (const W *)in->vals, n,
                                                 m, scan.as<unsigned long long>(), (I *)out->rowidx, (W *)out->vals);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "transpose kernels");
    // the workspace is freed on return: wait for the kernels that use it
    int herr = 0;
    if ((e = cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_fail(e, "cudaStreamSynchronize");
    if (herr) { set_error("transpose: a row index lies outside [0, nrows)"); return SPGEMM_ERR_INVALID; }
    return SPGEMM_OK;
}

}  // namespace spg

using namespace spg;

extern "C" spgemm_status spgemm_transpose(const spgemm_csc *in, spgemm_csc *out, cudaStream_t stream) {
    if (!in || !out) { set_error("NULL argument"); return SPGEMM_ERR_INVALID; }
    if (in->nrows < 0 || in->ncols < 0 || in->nnz < 0 || in->nrows >= 0x7fffffffLL || in->ncols >= 0x7fffffffLL) {
        set_error("transpose: bad shape (dimensions must be < 2^31-1)"); return SPGEMM_ERR_INVALID;
    }
    if (!in->colptr || (in->nnz > 0 && (!in->rowidx || !in->vals))) {
        set_error("transpose: NULL input array"); return SPGEMM_ERR_INVALID;
    }
    if (out->nrows != in->ncols || out->ncols != in->nrows || out->nnz != in->nnz ||
        out->idx_type != in->idx_type || out->val_type != in->val_type || !out->colptr ||
        (in->nnz > 0 && (!out->rowidx || !out->vals)) ||
        (out->ptr_type != SPGEMM_I32 && out->ptr_type != SPGEMM_I64) ||
        (in->ptr_type != SPGEMM_I32 && in->ptr_type != SPGEMM_I64)) {
        set_error("transpose: out must be ncols x nrows with the input's nnz, index and value types");
        return SPGEMM_ERR_INVALID;
    }
    if (out->ptr_type == SPGEMM_I32 && in->nnz >= 0x7fffffffLL) {
        set_error("transpose: nnz does not fit a 32-bit colptr"); return SPGEMM_ERR_INDEX_OVERFLOW;
    }
    const bool p64 = in->ptr_type == SPGEMM_I64, i64 = in->idx_type == SPGEMM_I64;
    const bool w8 = in->val_type != SPGEMM_F32;
#define TR(P, I, W) return transpose_typed<P, I, W>(in, out, stream)
    if (p64) {
        if (i64) { if (w8) TR(int64_t, int64_t, uint64_t); else TR(int64_t, int64_t, uint32_t); }
        else { if (w8) TR(int64_t, int32_t, uint64_t); else TR(int64_t, int32_t, uint32_t); }
    } else {
        if (i64) { if (w8) TR(int32_t, int64_t, uint64_t); else TR(int32_t, int64_t, uint32_t); }
        else { if (w8) TR(int32_t, int32_t, uint64_t); else TR(int32_t, int32_t, uint32_t); }
    }
#undef TR
}
