// The C ABI (include/spgemm.h): argument checks, plan lifetime, dispatch to
// the typed engines.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "../../include/spgemm.h"
#include "plan.h"
#include "util.h"

namespace spg {

static thread_local std::string g_err = "no error";

void set_error(const std::string &msg) { g_err = msg; }

spgemm_status cuda_fail(cudaError_t e, const char *where) {
    if (e == cudaErrorMemoryAllocation) {
        g_err = std::string("allocation failed in ") + where;
        return SPGEMM_ERR_OOM;
    }
    g_err = std::string("CUDA error in ") + where + ": " + cudaGetErrorString(e);
    return SPGEMM_ERR_CUDA;
}

thread_local AllocFns tl_alloc;

void *alloc_mem(const AllocFns &a, size_t bytes, int kind, cudaError_t &e) {
    void *p = nullptr;
    if (a.alloc) {
        p = a.alloc(a.ctx, bytes, kind);
        if (!p) { e = cudaErrorMemoryAllocation; return nullptr; }
        if (reinterpret_cast<uintptr_t>(p) % 256) {   // the callbacks promise 256-byte alignment
            a.free(a.ctx, p, bytes, kind);
            e = cudaErrorInvalidValue;
            return nullptr;
        }
        e = cudaSuccess;
        return p;
    }
    e = kind == SPGEMM_MEM_DEVICE ? cudaMalloc(&p, bytes) : cudaHostAlloc(&p, bytes, cudaHostAllocDefault);
    if (e != cudaSuccess) {
        cudaGetLastError();   // a failed allocation must not look like a failed launch later
        p = nullptr;
    }
    return p;
}

void free_mem(const AllocFns &a, void *p, size_t bytes, int kind) {
    if (a.alloc) {
        // the caller's allocator may hand the block out again at once: every
        // use of it on the device must have finished (as cudaFree ensures)
        cudaDeviceSynchronize();
        a.free(a.ctx, p, bytes, kind);
        return;
    }
    if (kind == SPGEMM_MEM_DEVICE) cudaFree(p); else cudaFreeHost(p);
}

size_t PlanState::workspace_bytes() const {
    const DevBuf *bufs[] = {&probs, &f, &cnt, &colptr, &tier, &list_sym, &list_num, &hist, &cursor,
                            &off_sym, &off_num, &heavy_ord, &pcnt, &err, &scan_part, &wbytes,
                            &valid_flag, &ap_end, &ap_row, &ap_val, &apc_off, &apc_row, &apc_val, &stage_cnt, &stage_colptr,
                            &stage_pcnt, &merge_tmp, &drows, &dvals, &parts_tab, &items, &item_cnt,
                            &item_off, &item_order, &pref_cnt, &pref_colptr, &pref_pcnt};
    size_t s = 0;
    for (auto *b : bufs) s += b->bytes;
    return s;
}

void PlanState::release_all() {
    DevBuf *bufs[] = {&probs, &f, &cnt, &colptr, &tier, &list_sym, &list_num, &hist, &cursor,
                      &off_sym, &off_num, &heavy_ord, &pcnt, &err, &scan_part, &wbytes,
                      &valid_flag, &ap_end, &ap_row, &ap_val, &apc_off, &apc_row, &apc_val, &stage_cnt, &stage_colptr,
                      &stage_pcnt, &merge_tmp, &drows, &dvals, &parts_tab, &items, &item_cnt,
                      &item_off, &item_order, &pref_cnt, &pref_colptr, &pref_pcnt};
    for (auto *b : bufs) b->release();
    h_colptr.release();
    h_pref_colptr.release();
    h_small.release();
    h_stage_colptr.release();
    h_parts.release();
    for (auto &b : ring_pcol) b.release();
    for (auto &b : ring_prow) b.release();
    for (auto &b : ring_pval) b.release();
    for (auto &b : ring_hpc) b.release();
    for (auto &w : ring_pws) w.release();
    for (auto &b : ring_col) b.release();
    for (auto &b : ring_row) b.release();
    for (auto &b : ring_val) b.release();
    for (auto &h : host_slots) h.release();
    ring_col.clear(); ring_row.clear(); ring_val.clear(); host_slots.clear();
    timer.release();
}

static int value_bytes(spgemm_value_t v) { return v == SPGEMM_F32 ? 4 : 8; }

static spgemm_status check_csc(const spgemm_csc *M, const char *name, bool input) {
    if (!M) { set_error(std::string(name) + " is NULL"); return SPGEMM_ERR_INVALID; }
    if (M->nrows < 0 || M->ncols < 0 || M->nnz < 0) {
        set_error(std::string(name) + ": negative size"); return SPGEMM_ERR_INVALID;
    }
    if (M->ptr_type != SPGEMM_I32 && M->ptr_type != SPGEMM_I64) {
        set_error(std::string(name) + ": bad ptr_type"); return SPGEMM_ERR_INVALID;
    }
    if (M->idx_type != SPGEMM_I32 && M->idx_type != SPGEMM_I64) {
        set_error(std::string(name) + ": bad idx_type"); return SPGEMM_ERR_INVALID;
    }
    if (M->val_type != SPGEMM_F64 && M->val_type != SPGEMM_F32 && M->val_type != SPGEMM_INT64) {
        set_error(std::string(name) + ": bad val_type"); return SPGEMM_ERR_INVALID;
    }
    if (input && M->ptr_type != M->idx_type) {
        set_error(std::string(name) + ": input ptr_type must equal idx_type"); return SPGEMM_ERR_INVALID;
    }
    if (M->nrows > 0x7fffffffLL) {   // row indices <= 2^31 - 2: 0xffffffff stays the empty hash key
        set_error(std::string(name) + ": nrows must be <= 2^31-1"); return SPGEMM_ERR_INVALID;
    }
    if (M->idx_type == SPGEMM_I32 && (M->nnz > 0x7fffffffLL || M->ncols >= 0x7fffffffLL)) {
        set_error(std::string(name) + ": nnz or ncols exceeds int32 index range"); return SPGEMM_ERR_INDEX_OVERFLOW;
    }
    if (!M->colptr || (M->nnz > 0 && (!M->rowidx || !M->vals))) {
        set_error(std::string(name) + ": NULL array"); return SPGEMM_ERR_INVALID;
    }
    return SPGEMM_OK;
}

}  // namespace spg

using namespace spg;

extern "C" {

const char *spgemm_last_error(void) { return g_err.c_str(); }

const char *spgemm_version(void) { return "gb300-spgemm 0.1 (sm_103a)"; }

spgemm_status spgemm_plan_create(const spgemm_csc *A, const spgemm_csc *B, const spgemm_opts *opts,
                                 int validate, cudaStream_t stream, spgemm_plan **out) {
    if (!out) { set_error("out is NULL"); return SPGEMM_ERR_INVALID; }
    *out = nullptr;
    spgemm_status s;
    if ((s = check_csc(A, "A", true)) != SPGEMM_OK) return s;
    if ((s = check_csc(B, "B", true)) != SPGEMM_OK) return s;
    if (A->ncols != B->nrows) {
        set_error("A.ncols != B.nrows"); return SPGEMM_ERR_INVALID;
    }
    if (A->idx_type != B->idx_type || A->val_type != B->val_type) {
        set_error("A and B must share index and value types"); return SPGEMM_ERR_INVALID;
    }
    if (B->ncols >= 0x7fffffffLL) { set_error("B.ncols must be < 2^31-1"); return SPGEMM_ERR_INVALID; }
    const int kst = opts && opts->kstages > 0 ? opts->kstages : 1;
    if (kst > 64) { set_error("kstages must be in [1, 64]"); return SPGEMM_ERR_INVALID; }
    if (opts && opts->prune && std::isnan(opts->prune_threshold)) {
        set_error("prune_threshold is NaN"); return SPGEMM_ERR_INVALID;
    }
    if (opts && opts->merge_mode != SPGEMM_MERGE_AT_END && opts->merge_mode != SPGEMM_MERGE_INCREMENTAL) {
        set_error("unknown merge_mode"); return SPGEMM_ERR_INVALID;
    }
    if (opts && opts->semiring != SPGEMM_PLUS_TIMES && opts->semiring != SPGEMM_OR_AND) {
        if (opts->semiring != SPGEMM_MIN_PLUS) { set_error("unknown semiring"); return SPGEMM_ERR_INVALID; }
        if (A->val_type == SPGEMM_INT64) {
            set_error("the min-plus semiring needs floating-point values"); return SPGEMM_ERR_INVALID;
        }
    }
    if (opts && opts->allocator && (!opts->allocator->alloc || !opts->allocator->free)) {
        set_error("an allocator needs both its alloc and free callbacks"); return SPGEMM_ERR_INVALID;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceProperties");
    if (prop.major < 10) {
        set_error("this library is built for sm_103a (Blackwell) devices");
        return SPGEMM_ERR_CUDA;
    }
    auto *plan = new (std::nothrow) spgemm_plan_s();
    if (!plan) { set_error("host allocation failed"); return SPGEMM_ERR_OOM; }
    PlanState &ps = plan->ps;
    ps.A = *A; ps.B = *B;
    if (opts) ps.opts = *opts;
    ps.opts.allocator = nullptr;   // copied below; the caller's struct need not outlive the call
    if (opts && opts->allocator) {
        ps.alloc.alloc = opts->allocator->alloc;
        ps.alloc.free = opts->allocator->free;
        ps.alloc.ctx = opts->allocator->ctx;
    }
    AllocScope scope(ps.alloc);
    ps.s = kst;
    ps.idx64 = A->idx_type == SPGEMM_I64;
    ps.vtype = A->val_type;
    ps.m = A->nrows; ps.k = A->ncols; ps.n = B->ncols;
    ps.dev = dev; ps.nsm = prop.multiProcessorCount;
    // tuning
    const spgemm_tuning *tu = opts ? opts->tuning : nullptr;
    ps.tun.log2R = value_bytes((spgemm_value_t)ps.vtype) == 4 ? 14 : 13;
    if (tu) {
        if (tu->hash_max_cap) ps.tun.hash_cap_max = tu->hash_max_cap;
        if (tu->panel_rows) {
            int l = 0;
            while ((1 << l) < tu->panel_rows) ++l;
            ps.tun.log2R = l;
        }
        if (tu->short_seg) ps.tun.short_seg = tu->short_seg;
        if (tu->huge_seg) ps.tun.huge_seg = tu->huge_seg;
        if (tu->block_tier_threads) ps.tun.block_threads = tu->block_tier_threads;
        ps.tun.hybrid_sort = tu->hybrid_sort ? 1 : 0;
    }
    {
        bool ok = false;
        for (int c = 256; c <= 8192; c <<= 1) ok |= ps.tun.hash_cap_max == c;
        const int R = 1 << ps.tun.log2R;
        const int dense_smem = R * value_bytes((spgemm_value_t)ps.vtype) + R;
        if (!ok || ps.tun.log2R < 10 || ps.tun.log2R > 16 || dense_smem > 200 * 1024 ||
            ps.tun.short_seg < 1 || ps.tun.short_seg > 64 || ps.tun.huge_seg < 64 ||
            (ps.tun.block_threads && (ps.tun.block_threads % 32 || ps.tun.block_threads < 128 ||
                                      ps.tun.block_threads > 1024))) {
            set_error("invalid tuning parameters");
            delete plan;
            return SPGEMM_ERR_INVALID;
        }
    }
    // panels
    const int64_t R = 1LL << ps.tun.log2R;
    ps.P = (int)((ps.m + R - 1) / R);
    if (ps.P < 1) ps.P = 1;
    const int64_t maxbm = (int64_t)(160 * 1024) * 8;   // bitmap rows per CTA
    const int64_t mpad = ((ps.m + R - 1) / R) * R;
    ps.Rs = mpad <= maxbm ? (mpad > 0 ? mpad : R) : (maxbm / R) * R;
    ps.Q = (int)((ps.m + ps.Rs - 1) / ps.Rs);
    if (ps.Q < 1) ps.Q = 1;
    // budget
    size_t freeb = 0, totb = 0;
    e = cudaMemGetInfo(&freeb, &totb);
    if (e != cudaSuccess) { delete plan; return cuda_fail(e, "cudaMemGetInfo"); }
    ps.budget = (opts && opts->budget_bytes) ? opts->budget_bytes : (size_t)(0.8 * (double)freeb);
    ps.eng = make_engine(ps.idx64, ps.vtype, opts ? opts->semiring : SPGEMM_PLUS_TIMES);
    if (!ps.eng) { set_error("unsupported type combination"); delete plan; return SPGEMM_ERR_INVALID; }
    // structural checks
    auto read_last = [&](const spgemm_csc *M, int64_t *v) -> cudaError_t {
        if (M->ptr_type == SPGEMM_I64)
            return cudaMemcpy(v, (const int64_t *)M->colptr + M->ncols, 8, cudaMemcpyDeviceToHost);
        int32_t x = 0;
        cudaError_t ee = cudaMemcpy(&x, (const int32_t *)M->colptr + M->ncols, 4, cudaMemcpyDeviceToHost);
        *v = x;
        return ee;
    };
    int64_t la = 0, lb = 0;
    if ((e = read_last(A, &la)) != cudaSuccess || (e = read_last(B, &lb)) != cudaSuccess) {
        delete ps.eng; delete plan; return cuda_fail(e, "reading colptr");
    }
    if (la != A->nnz || lb != B->nnz) {
        set_error("nnz does not match colptr[ncols]");
        delete ps.eng; delete plan;
        return SPGEMM_ERR_INVALID;
    }
    s = ps.eng->setup(ps, stream);
    if (s != SPGEMM_OK) { ps.release_all(); delete ps.eng; delete plan; return s; }
    if (validate) {
        if ((e = ps.valid_flag.ensure(16)) != cudaSuccess ||
            (e = cudaMemsetAsync(ps.valid_flag.p, 0, 4, stream)) != cudaSuccess ||
            (e = validate_csc(A->colptr, A->rowidx, ps.idx64, A->ncols, A->nrows, A->nnz,
                              ps.valid_flag.as<int>(), stream)) != cudaSuccess ||
            (e = validate_csc(B->colptr, B->rowidx, ps.idx64, B->ncols, B->nrows, B->nnz,
                              ps.valid_flag.as<int>(), stream)) != cudaSuccess) {
            ps.release_all(); delete ps.eng; delete plan;
            return cuda_fail(e, "validate");
        }
        int bad = 0;
        e = cudaMemcpyAsync(&bad, ps.valid_flag.p, 4, cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) { ps.release_all(); delete ps.eng; delete plan; return cuda_fail(e, "validate"); }
        if (bad) {
            set_error(bad & 1 ? "corrupt CSC: colptr not monotone from 0 to nnz"
                              : "corrupt CSC: row index out of range");
            ps.release_all(); delete ps.eng; delete plan;
            return SPGEMM_ERR_INVALID;
        }
    }
    *out = plan;
    return SPGEMM_OK;
}

spgemm_status spgemm_plan_destroy(spgemm_plan *plan) {
    if (!plan) return SPGEMM_OK;
    plan->ps.release_all();
    delete plan->ps.eng;
    delete plan;
    return SPGEMM_OK;
}

spgemm_status spgemm_symbolic(spgemm_plan *plan, cudaStream_t stream) {
    if (!plan) { set_error("plan is NULL"); return SPGEMM_ERR_INVALID; }
    AllocScope scope(plan->ps.alloc);
    return plan->ps.eng->symbolic(plan->ps, stream);
}

spgemm_status spgemm_plan_query(const spgemm_plan *plan, spgemm_plan_info *info) {
    if (!plan || !info) { set_error("NULL argument"); return SPGEMM_ERR_INVALID; }
    const PlanState &ps = plan->ps;
    if (!ps.have_symbolic) { set_error("call spgemm_symbolic first"); return SPGEMM_ERR_STATE; }
    std::memset(info, 0, sizeof(*info));
    info->flops = ps.flops;
    info->nnz_c = ps.nnz_c;
    info->unmerged_nnz = ps.unmerged;
    info->stage_buffer_nnz = ps.stage_buffer_nnz;
    info->nbatches = (int64_t)ps.batches.size();
    for (auto &b : ps.batches) {
        if (b.nnz > info->max_batch_nnz) info->max_batch_nnz = b.nnz;
        if (b.c1 - b.c0 > info->max_batch_cols) info->max_batch_cols = b.c1 - b.c0;
    }
    info->bytes_per_nnz = ps.bytes_per_nnz;
    info->batch_cap_bytes = ps.batch_cap;
    int64_t h = 0;
    for (auto &b : ps.batches) h += b.heavy;
    info->heavy_columns = h;
    return SPGEMM_OK;
}

spgemm_status spgemm_plan_batch(const spgemm_plan *plan, int64_t t, int64_t *col_begin,
                                int64_t *col_end, int64_t *nnz) {
    if (!plan) { set_error("plan is NULL"); return SPGEMM_ERR_INVALID; }
    const PlanState &ps = plan->ps;
    if (!ps.have_symbolic) { set_error("call spgemm_symbolic first"); return SPGEMM_ERR_STATE; }
    if (t < 0 || t >= (int64_t)ps.batches.size()) { set_error("batch out of range"); return SPGEMM_ERR_INVALID; }
    const Batch &b = ps.batches[(size_t)t];
    if (col_begin) *col_begin = b.c0;
    if (col_end) *col_end = b.c1;
    if (nnz) *nnz = b.nnz;
    return SPGEMM_OK;
}

spgemm_status spgemm_plan_column_counts(const spgemm_plan *plan, int64_t *counts_out,
                                        cudaStream_t stream) {
    if (!plan || !counts_out) { set_error("NULL argument"); return SPGEMM_ERR_INVALID; }
    const PlanState &ps = plan->ps;
    if (!ps.have_symbolic) { set_error("call spgemm_symbolic first"); return SPGEMM_ERR_STATE; }
    cudaError_t e = cudaMemcpyAsync(counts_out, ps.cnt.p, sizeof(int64_t) * ps.n,
                                    cudaMemcpyDeviceToDevice, stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
    return SPGEMM_OK;
}

spgemm_status spgemm_numeric(spgemm_plan *plan, int64_t t, spgemm_csc *C, cudaStream_t stream) {
    if (!plan || !C) { set_error("NULL argument"); return SPGEMM_ERR_INVALID; }
    PlanState &ps = plan->ps;
    AllocScope scope(ps.alloc);
    if (!ps.have_symbolic) { set_error("call spgemm_symbolic first"); return SPGEMM_ERR_STATE; }
    if (t < 0 || t >= (int64_t)ps.batches.size()) { set_error("batch out of range"); return SPGEMM_ERR_INVALID; }
    const Batch &b = ps.batches[(size_t)t];
    if (C->nrows != ps.m || C->ncols != b.c1 - b.c0 || C->nnz != b.nnz) {
        set_error("C_out shape/nnz does not match the batch"); return SPGEMM_ERR_INVALID;
    }
    if (C->idx_type != (ps.idx64 ? SPGEMM_I64 : SPGEMM_I32) || C->val_type != ps.vtype ||
        (C->ptr_type != SPGEMM_I32 && C->ptr_type != SPGEMM_I64)) {
        set_error("C_out types do not match the plan"); return SPGEMM_ERR_INVALID;
    }
    if (C->ptr_type == SPGEMM_I32 && b.nnz > 0x7fffffffLL) {
        set_error("batch nnz does not fit a 32-bit colptr"); return SPGEMM_ERR_INDEX_OVERFLOW;
    }
    if (!C->colptr || (b.nnz > 0 && (!C->rowidx || !C->vals))) {
        set_error("C_out has NULL arrays"); return SPGEMM_ERR_INVALID;
    }
    return ps.eng->numeric(ps, t, C, stream);
}

spgemm_status spgemm_backward(spgemm_plan *plan, const spgemm_csc *G, void *dA_vals, void *dB_vals,
                              cudaStream_t stream) {
    if (!plan || !G) { set_error("NULL argument"); return SPGEMM_ERR_INVALID; }
    const PlanState &ps = plan->ps;
    AllocScope scope(ps.alloc);
    spgemm_status s = check_csc(G, "G", false);
    if (s != SPGEMM_OK) return s;
    if (G->nrows != ps.m || G->ncols != ps.n) { set_error("G must have C's shape"); return SPGEMM_ERR_INVALID; }
    if (G->idx_type != (ps.idx64 ? SPGEMM_I64 : SPGEMM_I32) || G->val_type != ps.vtype) {
        set_error("G must share the plan's index and value types"); return SPGEMM_ERR_INVALID;
    }
    if ((ps.A.nnz && !dA_vals) || (ps.B.nnz && !dB_vals)) { set_error("NULL gradient buffer"); return SPGEMM_ERR_INVALID; }
    if (ps.s != 1) { set_error("backward works on plans with one stage"); return SPGEMM_ERR_INVALID; }
    return plan->ps.eng->backward(plan->ps, G, dA_vals, dB_vals, stream);
}

}  // extern "C"

namespace spg {
void MultiState::release_all() {
    DevBuf *bufs[] = {&probs, &f, &cnt, &colptr, &tier, &list, &off, &hist, &cursor, &err,
                      &scan_part, &rows, &vals, &counter, &gsize, &gtab_off, &gkeys, &gvals};
    for (auto *b : bufs) b->release();
    h_small.release();
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (own) cudaStreamDestroy(own);
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    exec = nullptr; graph = nullptr; own = nullptr; ev_in = ev_out = nullptr;
}
}  // namespace spg

extern "C" {

spgemm_status spgemm_plan_colptr(const spgemm_plan *plan, void *colptr_out, spgemm_index_t ptr_type,
                                 cudaStream_t stream) {
    if (!plan || !colptr_out) { set_error("NULL argument"); return SPGEMM_ERR_INVALID; }
    const PlanState &ps = plan->ps;
    if (!ps.have_symbolic) { set_error("call spgemm_symbolic first"); return SPGEMM_ERR_STATE; }
    if (ptr_type == SPGEMM_I32 && ps.nnz_c > 0x7fffffffLL) {
        set_error("nnz(C) does not fit a 32-bit colptr"); return SPGEMM_ERR_INDEX_OVERFLOW;
    }
    cudaError_t e = rebase_colptr(ps.colptr.as<int64_t>(), ps.n, colptr_out, ptr_type == SPGEMM_I64, stream);
    return e == cudaSuccess ? SPGEMM_OK : cuda_fail(e, "rebase_colptr");
}

spgemm_status spgemm_plan_set_timing(spgemm_plan *plan, int enable) {
    if (!plan) { set_error("plan is NULL"); return SPGEMM_ERR_INVALID; }
    plan->ps.timer.enabled = enable != 0;
    return SPGEMM_OK;
}

spgemm_status spgemm_plan_stats(spgemm_plan *plan, int reset, spgemm_stats *out) {
    if (!plan || !out) { set_error("NULL argument"); return SPGEMM_ERR_INVALID; }
    PhaseTimer &tm = plan->ps.timer;
    tm.collect();
    out->launches = tm.launches;
    for (int i = 0; i < SPGEMM_NUM_PHASES; ++i) { out->ms[i] = tm.ms[i]; out->count[i] = tm.count[i]; }
    if (reset) tm.reset();
    return SPGEMM_OK;
}

spgemm_status spgemm_plan_check(const spgemm_plan *plan, cudaStream_t stream) {
    if (!plan) { set_error("plan is NULL"); return SPGEMM_ERR_INVALID; }
    const PlanState &ps = plan->ps;
    int flags = 0;
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e == cudaSuccess) e = cudaMemcpy(&flags, ps.err.p, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "spgemm_plan_check");
    if (flags) {
        set_error("device error flags " + std::to_string(flags) +
                  ((flags & 2) ? " (a column's nnz differed from its symbolic count)" : "") +
                  ((flags & 1) ? " (hash probe bound exceeded)" : ""));
        return SPGEMM_ERR_OVERFLOW;
    }
    return SPGEMM_OK;
}

spgemm_status spgemm_prune(const spgemm_csc *in, double threshold, int64_t topk, spgemm_csc *out,
                           cudaStream_t stream) {
    if (!in || !out) { set_error("NULL argument"); return SPGEMM_ERR_INVALID; }
    spgemm_status s = check_csc(in, "in", false);
    if (s != SPGEMM_OK) return s;
    if (std::isnan(threshold)) { set_error("threshold is NaN"); return SPGEMM_ERR_INVALID; }
    if (!out->colptr || out->nrows != in->nrows || out->ncols != in->ncols || out->idx_type != in->idx_type ||
        out->val_type != in->val_type || out->ptr_type != SPGEMM_I64) {
        set_error("out does not match in (int64 colptr required)"); return SPGEMM_ERR_INVALID;
    }
    if (out->rowidx && out->nnz > 0 && !out->vals) { set_error("out->vals is NULL"); return SPGEMM_ERR_INVALID; }
    return prune_dispatch(in, threshold, topk, out, stream);
}

spgemm_status spgemm_merge(const spgemm_csc *parts, int nparts, spgemm_csc *out, cudaStream_t stream) {
    spgemm_status s = check_merge_args(parts, nparts, out);
    if (s != SPGEMM_OK) return s;
    return merge_dispatch(parts, nparts, out, stream);
}

}  // extern "C"

spgemm_status spg::check_merge_args(const spgemm_csc *parts, int nparts, const spgemm_csc *out) {
    if (!parts || nparts < 1 || !out) { set_error("bad arguments"); return SPGEMM_ERR_INVALID; }
    spgemm_status s;
    for (int i = 0; i < nparts; ++i) {
        if ((s = check_csc(&parts[i], "part", false)) != SPGEMM_OK) return s;
        if (parts[i].nrows != parts[0].nrows || parts[i].ncols != parts[0].ncols ||
            parts[i].idx_type != parts[0].idx_type || parts[i].val_type != parts[0].val_type) {
            set_error("parts differ in shape or type"); return SPGEMM_ERR_INVALID;
        }
    }
    if (!out->colptr || out->nrows != parts[0].nrows || out->ncols != parts[0].ncols ||
        out->idx_type != parts[0].idx_type || out->val_type != parts[0].val_type ||
        (out->ptr_type != SPGEMM_I32 && out->ptr_type != SPGEMM_I64)) {
        set_error("out does not match the parts"); return SPGEMM_ERR_INVALID;
    }
    if (out->rowidx && out->nnz > 0 && !out->vals) { set_error("out->vals is NULL"); return SPGEMM_ERR_INVALID; }
    if (parts[0].ncols >= 0x7fffffffLL) { set_error("ncols must be < 2^31-1"); return SPGEMM_ERR_INVALID; }
    return SPGEMM_OK;
}

extern "C" {

spgemm_status spgemm_multi_create(int nprob, const spgemm_csc *As, const spgemm_csc *Bs,
                                  const spgemm_opts *opts, cudaStream_t stream, spgemm_multi **out) {
    if (!out || !As || !Bs || nprob < 1) { set_error("bad arguments"); return SPGEMM_ERR_INVALID; }
    *out = nullptr;
    spgemm_status s;
    int64_t total = 0;
    for (int i = 0; i < nprob; ++i) {
        if ((s = check_csc(&As[i], "A_i", true)) != SPGEMM_OK) return s;
        if ((s = check_csc(&Bs[i], "B_i", true)) != SPGEMM_OK) return s;
        if (As[i].ncols != Bs[i].nrows) { set_error("A_i.ncols != B_i.nrows"); return SPGEMM_ERR_INVALID; }
        if (As[i].idx_type != As[0].idx_type || Bs[i].idx_type != As[0].idx_type ||
            As[i].val_type != As[0].val_type || Bs[i].val_type != As[0].val_type) {
            set_error("all problems must share index and value types"); return SPGEMM_ERR_INVALID;
        }
        total += Bs[i].ncols;
    }
    if (total >= 0x7fffffffLL) { set_error("total columns must be < 2^31-1"); return SPGEMM_ERR_INVALID; }
    if (opts && opts->kstages > 1) { set_error("batched problems take no k-split"); return SPGEMM_ERR_INVALID; }
    if (opts && (opts->semiring != SPGEMM_PLUS_TIMES || opts->sort_output || opts->prune)) {
        set_error("batched problems run the plus-times product, unsorted and unpruned "
                  "(semiring, sort_output and prune are plan options)");
        return SPGEMM_ERR_INVALID;
    }
    if (opts && opts->allocator && (!opts->allocator->alloc || !opts->allocator->free)) {
        set_error("an allocator needs both its alloc and free callbacks"); return SPGEMM_ERR_INVALID;
    }
    int dev = 0;
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaGetDeviceProperties(&prop, dev);
    if (e != cudaSuccess) return cuda_fail(e, "device query");
    auto *mh = new (std::nothrow) spgemm_multi_s();
    if (!mh) { set_error("host allocation failed"); return SPGEMM_ERR_OOM; }
    MultiState &ms = mh->ms;
    if (opts && opts->allocator) {
        ms.alloc.alloc = opts->allocator->alloc;
        ms.alloc.free = opts->allocator->free;
        ms.alloc.ctx = opts->allocator->ctx;
    }
    AllocScope scope(ms.alloc);
    ms.nprob = nprob;
    ms.idx64 = As[0].idx_type == SPGEMM_I64;
    ms.vtype = As[0].val_type;
    ms.nsm = prop.multiProcessorCount;
    // defaults of the persistent passes: small shared tables and 128-thread
    // CTAs keep many CTAs resident per SM (batched problems are mostly small)
    ms.tun.hash_cap_max = 1024;
    ms.warp_tiers = 3;   // warp tables up to 256 rows
    if (opts && opts->tuning) {
        const spgemm_tuning *tu = opts->tuning;
        if (tu->hash_max_cap) ms.tun.hash_cap_max = tu->hash_max_cap;
        if (tu->short_seg) ms.tun.short_seg = tu->short_seg;
        if (tu->huge_seg) ms.tun.huge_seg = tu->huge_seg;
        if (tu->block_tier_threads) ms.tun.block_threads = tu->block_tier_threads;
        if (tu->warp_max_cap) {
            static const int kWarpCaps[5] = {0, 32, 128, 256, 512};   // warp tiers 1..4
            int wt = 0;
            for (int t = 1; t <= 4; ++t) if (kWarpCaps[t] == tu->warp_max_cap) wt = t;
            if (!wt) {
                set_error("warp_max_cap must be 32, 128, 256 or 512");
                delete mh;
                return SPGEMM_ERR_INVALID;
            }
            ms.warp_tiers = wt;
        }
    }
    {
        bool ok = false;
        for (int c = 256; c <= 8192; c <<= 1) ok |= ms.tun.hash_cap_max == c;
        static const int kWarpCaps[5] = {0, 32, 128, 256, 512};
        if (!ok || ms.tun.hash_cap_max < kWarpCaps[ms.warp_tiers]) {
            set_error("hash_max_cap must be a power of two from 256 to 8192, at least warp_max_cap");
            delete mh;
            return SPGEMM_ERR_INVALID;
        }
    }
    ms.threads = ms.tun.block_threads == 0 ? 128 : ms.tun.block_threads >= 512 ? 512
                 : ms.tun.block_threads >= 256 ? 256 : 128;
    s = multi_create_typed(ms, As, Bs, stream);
    if (s != SPGEMM_OK) { ms.release_all(); delete mh; return s; }
    *out = mh;
    return SPGEMM_OK;
}

spgemm_status spgemm_multi_destroy(spgemm_multi *m) {
    if (!m) return SPGEMM_OK;
    m->ms.release_all();
    delete m;
    return SPGEMM_OK;
}

spgemm_status spgemm_multi_run(spgemm_multi *m, int use_graph, cudaStream_t stream) {
    if (!m) { set_error("NULL argument"); return SPGEMM_ERR_INVALID; }
    MultiState &ms = m->ms;
    AllocScope scope(ms.alloc);
    cudaError_t e;
    if (!use_graph) return ms.enqueue(ms, stream);
    // graphs are captured on a private stream (the legacy default stream cannot
    // be captured); the caller's stream is ordered around the launch with events
    if (!ms.own) {
        if ((e = cudaStreamCreateWithFlags(&ms.own, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(e, "cudaStreamCreate");
        if ((e = cudaEventCreateWithFlags(&ms.ev_in, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&ms.ev_out, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(e, "cudaEventCreate");
    }
    if (!ms.exec) {
        if ((e = cudaStreamBeginCapture(ms.own, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            return cuda_fail(e, "cudaStreamBeginCapture");
        spgemm_status s = ms.enqueue(ms, ms.own);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(ms.own, &g);
        if (s != SPGEMM_OK) { if (g) cudaGraphDestroy(g); return s; }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        ms.graph = g;
        if ((e = cudaGraphInstantiate(&ms.exec, ms.graph, 0)) != cudaSuccess)
            return cuda_fail(e, "cudaGraphInstantiate");
    }
    if ((e = cudaEventRecord(ms.ev_in, stream)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(ms.own, ms.ev_in, 0)) != cudaSuccess ||
        (e = cudaGraphLaunch(ms.exec, ms.own)) != cudaSuccess ||
        (e = cudaEventRecord(ms.ev_out, ms.own)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(stream, ms.ev_out, 0)) != cudaSuccess)
        return cuda_fail(e, "graph launch");
    return SPGEMM_OK;
}

spgemm_status spgemm_multi_output(const spgemm_multi *m, int64_t **colptr, void **rowidx, void **vals,
                                  int64_t *total_cols, int64_t *capacity) {
    if (!m) { set_error("NULL argument"); return SPGEMM_ERR_INVALID; }
    const MultiState &ms = m->ms;
    if (colptr) *colptr = ms.colptr.as<int64_t>();
    if (rowidx) *rowidx = ms.rows.p;
    if (vals) *vals = ms.vals.p;
    if (total_cols) *total_cols = ms.total_cols;
    if (capacity) *capacity = ms.capacity;
    return SPGEMM_OK;
}

}  // extern "C"
