// Plan state shared by the C ABI and the typed engines.
#pragma once

#include <cstdint>
#include <array>
#include <string>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/spgemm.h"

namespace spg {

// The allocator a buffer takes its memory from: the callbacks of
// spgemm_allocator, or (alloc == nullptr) cudaMalloc / cudaHostAlloc.
struct AllocFns {
    spgemm_alloc_fn alloc = nullptr;
    spgemm_free_fn free = nullptr;
    void *ctx = nullptr;
};

// The allocator of the plan whose call is running on this thread (a plan is
// used by one host thread at a time); set for the length of a call by
// AllocScope. Buffers remember the allocator that produced them and give
// their memory back to it.
extern thread_local AllocFns tl_alloc;
struct AllocScope {
    AllocFns saved;
    explicit AllocScope(const AllocFns &a) : saved(tl_alloc) { tl_alloc = a; }
    ~AllocScope() { tl_alloc = saved; }
};

// Memory of `kind` from the current allocator; cudaErrorMemoryAllocation when
// it fails (no CUDA error state is left behind).
void *alloc_mem(const AllocFns &a, size_t bytes, int kind, cudaError_t &e);
void free_mem(const AllocFns &a, void *p, size_t bytes, int kind);

// A grow-only buffer of device (KIND = SPGEMM_MEM_DEVICE) or pinned host
// memory; it owns its block (moved, never copied) and frees it when destroyed.
template <int KIND> struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
    AllocFns how;
    Buf() = default;
    Buf(const Buf &) = delete;
    Buf &operator=(const Buf &) = delete;
    Buf(Buf &&o) noexcept : p(o.p), bytes(o.bytes), how(o.how) { o.p = nullptr; o.bytes = 0; }
    Buf &operator=(Buf &&o) noexcept {
        if (this != &o) {
            release();
            p = o.p; bytes = o.bytes; how = o.how;
            o.p = nullptr; o.bytes = 0;
        }
        return *this;
    }
    ~Buf() { release(); }
    cudaError_t ensure(size_t want) {
        if (want <= bytes && p) return cudaSuccess;
        release();
        if (want == 0) want = 16;
        cudaError_t e = cudaSuccess;
        how = tl_alloc;
        p = alloc_mem(how, want, KIND, e);
        if (e == cudaSuccess) bytes = want; else p = nullptr;
        return e;
    }
    void release() {
        if (p) free_mem(how, p, bytes, KIND);
        p = nullptr;
        bytes = 0;
    }
    template <class T> T *as() const { return static_cast<T *>(p); }
};
using DevBuf = Buf<SPGEMM_MEM_DEVICE>;
using HostBuf = Buf<SPGEMM_MEM_PINNED_HOST>;

int64_t scan_partials_len(int64_t n);

// Workspace of the column prune (per column: kept count, mode, selection
// list, selected key and tie quota; scan partials).
struct PruneWs {
    DevBuf keep, mode, sel, nsel, key, quota, part, row;
    cudaError_t ensure(int64_t ncols) {
        cudaError_t e;
        if ((e = keep.ensure(sizeof(int64_t) * (size_t)(ncols + 1))) != cudaSuccess) return e;
        if ((e = mode.ensure((size_t)ncols + 16)) != cudaSuccess) return e;
        if ((e = sel.ensure(sizeof(int64_t) * (size_t)(ncols + 1))) != cudaSuccess) return e;
        if ((e = nsel.ensure(sizeof(unsigned long long) * 2)) != cudaSuccess) return e;
        if ((e = key.ensure(sizeof(uint64_t) * (size_t)(ncols + 1))) != cudaSuccess) return e;
        if ((e = quota.ensure(sizeof(int64_t) * (size_t)(ncols + 1))) != cudaSuccess) return e;
        if ((e = row.ensure(sizeof(uint32_t) * (size_t)(ncols + 1))) != cudaSuccess) return e;
        return part.ensure(sizeof(int64_t) * (size_t)scan_partials_len(ncols + 1));
    }
    size_t bytes() const {
        return keep.bytes + mode.bytes + sel.bytes + nsel.bytes + key.bytes + quota.bytes + part.bytes + row.bytes;
    }
    void release() {
        keep.release(); mode.release(); sel.release(); nsel.release(); key.release(); quota.release();
        part.release(); row.release();
    }
};

struct Tuning {
    int hash_cap_max = 8192;
    int log2R = 15;          // dense panel rows (set per value type at plan time)
    int short_seg = 1;
    int huge_seg = 4096;
    int block_threads = 0;   // 0: per-tier default
    int hybrid_sort = 0;     // CTA tiers: sort-accumulate columns whose products fit the table
};

struct Batch {
    int64_t c0 = 0, c1 = 0;  // column range
    int64_t nnz = 0;         // nnz(C) of the batch
    int64_t pnnz = 0;        // bound on the pruned batch (opts.prune)
    int64_t unmerged = 0;    // sum over stages of nnz(D_t) of the batch (s > 1)
    // incremental merge (s > 1): entries of the largest stage partial D_t
    // (t >= 1) and of the largest running sum M_u (u <= s - 2) of the batch
    int64_t dsz = 0, msz = 0;
    // numeric hash-tier populations: [0] the product (s = 1) or the merge,
    // [1 + t] stage t (s > 1); host copies computed from the counts
    std::vector<std::array<int, 16>> tc;
    int64_t heavy = 0;       // columns above the largest hash table
    std::vector<int64_t> doff;  // offset of stage t's partials in the partial buffer
};

// Per-phase device time (CUDA events on the launching stream) and kernel
// launch counts of a plan.
enum Phase : int {
    kPhFlopsBin = 0, kPhSymHash = 1, kPhSymHeavy = 2, kPhScan = 3, kPhPanels = 4,
    kPhNumHash = 5, kPhNumDense = 6, kPhMerge = 7, kPhBackward = 8, kNumPhases = 9
};

struct PhaseTimer {
    bool enabled = false;
    struct Rec { int phase; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    double ms[kNumPhases] = {0};
    int64_t count[kNumPhases] = {0};
    int64_t launches = 0;
    cudaEvent_t get() {
        if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    int begin(int phase, cudaStream_t st) {
        if (!enabled) return -1;
        Rec r{phase, get(), get()};
        cudaEventRecord(r.a, st);
        recs.push_back(r);
        return (int)recs.size() - 1;
    }
    void end(int idx, cudaStream_t st) {
        if (idx < 0) return;
        cudaEventRecord(recs[(size_t)idx].b, st);
    }
    void collect() {
        for (auto &r : recs) {
            float t = 0.f;
            cudaEventSynchronize(r.b);
            if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
                ms[r.phase] += t;
                count[r.phase] += 1;
            }
            pool.push_back(r.a);
            pool.push_back(r.b);
        }
        recs.clear();
    }
    void reset() {
        collect();
        for (int i = 0; i < kNumPhases; ++i) { ms[i] = 0; count[i] = 0; }
        launches = 0;
    }
    void release() {
        collect();
        for (auto e : pool) cudaEventDestroy(e);
        pool.clear();
    }
};

struct EngineBase;

struct PlanState {
    spgemm_csc A{}, B{};
    spgemm_opts opts{};
    AllocFns alloc;          // workspace allocator (opts->allocator, copied)
    Tuning tun;
    int idx64 = 0, vtype = 0;
    int64_t m = 0, k = 0, n = 0;
    int s = 1;
    size_t budget = 0;
    int dev = 0, nsm = 148;
    EngineBase *eng = nullptr;

    // device workspace
    DevBuf probs, f, cnt, colptr, tier, list_sym, list_num, hist, cursor, off_sym, off_num;
    DevBuf heavy_ord, pcnt, err, scan_part, wbytes, valid_flag;
    DevBuf ap_end, ap_row, ap_val;
    DevBuf apc_off, apc_row, apc_val;   // A grouped by panel within each column
    DevBuf stage_cnt, stage_colptr, stage_pcnt, drows, dvals, parts_tab;  // k-split
    DevBuf pref_cnt, pref_colptr, pref_pcnt;   // incremental merge: nnz(M_u), u = 1..s-2
    DevBuf merge_tmp;
    DevBuf items, item_cnt, item_off, item_order;  // heavy work items (dense panels / hash ranges)
    int64_t n_items = 0;
    std::vector<int64_t> batch_item_off;   // batch t's items: item_order[off[t], off[t+1])
    HostBuf h_colptr, h_small, h_stage_colptr, h_parts, h_pref_colptr;
    std::vector<DevBuf> ring_col, ring_row, ring_val;   // spgemm_run_batched device ring
    std::vector<DevBuf> ring_pcol, ring_prow, ring_pval;  // pruned copies (opts.prune)
    std::vector<HostBuf> ring_hpc;                        // their colptrs on the host
    std::vector<PruneWs> ring_pws;
    std::vector<int64_t> prune_prefix;                    // sum of min(nnz_j, topk) over columns < j
    std::vector<HostBuf> host_slots;                     // spgemm_run_batched pinned slots

    PhaseTimer timer;

    // symbolic results
    bool have_symbolic = false;
    int64_t flops = 0, nnz_c = 0, unmerged = 0;
    int64_t stage_buffer_nnz = 0;   // entries of the largest batch's stage buffers (s > 1)
    int sym_hist[16] = {0};
    int nheavy = 0;          // symbolic heavy columns (dense path candidates)
    int P = 0, Q = 0;        // numeric panels, symbolic panels
    int64_t Rs = 0;          // symbolic bitmap rows
    bool panels_built = false;
    bool defer_sort = false;   // spgemm_run_batched sorts after its prune instead
    std::vector<Batch> batches;
    int64_t batch_cap = 0;
    int64_t bytes_per_nnz = 0;

    size_t workspace_bytes() const;
    void release_all();
};

// Typed engine: one per (index, value) type pair.
struct EngineBase {
    virtual ~EngineBase() {}
    virtual spgemm_status setup(PlanState &ps, cudaStream_t st) = 0;
    virtual spgemm_status symbolic(PlanState &ps, cudaStream_t st) = 0;
    virtual spgemm_status numeric(PlanState &ps, int64_t t, spgemm_csc *C, cudaStream_t st) = 0;
    virtual spgemm_status backward(PlanState &ps, const spgemm_csc *G, void *dA, void *dB,
                                   cudaStream_t st) = 0;
    // the plan's prune (opts.prune) of one batch output: colptr relative
    // (ncols + 1, int64), into ocolptr / orows / ovals
    virtual spgemm_status prune_batch(PlanState &ps, int64_t ncols, const int64_t *colptr, const void *rows,
                                      const void *vals, int64_t *ocolptr, void *orows, void *ovals,
                                      PruneWs &ws, cudaStream_t st) = 0;
};

// Type-erased standalone merge (spgemm_merge).
spgemm_status merge_dispatch(const spgemm_csc *parts, int nparts, spgemm_csc *out,
                             cudaStream_t st);

// Type-erased column prune (spgemm_prune).
spgemm_status prune_dispatch(const spgemm_csc *in, double threshold, int64_t topk, spgemm_csc *out,
                             cudaStream_t st);

// The merge with caller-free scratch (spgemm_merge_noalloc).
spgemm_status merge_noalloc_dispatch(const spgemm_csc *parts, int nparts, spgemm_csc *out,
                                     cudaStream_t st, unsigned char *scratch, size_t cap,
                                     int32_t *stage, int nsm);

// Argument checks shared by the merge entry points.
spgemm_status check_merge_args(const spgemm_csc *parts, int nparts, const spgemm_csc *out);

EngineBase *make_engine(int idx64, int vtype, int semiring);

// thread-local error message
void set_error(const std::string &msg);
spgemm_status cuda_fail(cudaError_t e, const char *where);

}  // namespace spg

struct spgemm_plan_s {
    spg::PlanState ps;
};

namespace spg {

// State of a multi-problem run (spgemm_multi).
struct MultiState {
    int nprob = 0, idx64 = 0, vtype = 0, nsm = 148;
    AllocFns alloc;          // workspace allocator (opts->allocator, copied)
    Tuning tun;
    DevBuf probs, f, cnt, colptr, tier, list, off, hist, cursor, err, scan_part;
    DevBuf rows, vals;
    DevBuf counter;                // work counters of the two persistent passes (2 each)
    DevBuf gsize, gtab_off, gkeys, gvals;   // global tables of the heavy columns
    HostBuf h_small;
    int64_t total_cols = 0, capacity = 0, total_flops = 0, heavy_cols = 0;
    int warp_tiers = 4;            // tiers 1..warp_tiers run one warp per column
    int threads = 512;             // CTA width of the persistent passes
    int grid = 0;                  // resident CTAs of the persistent passes
    size_t smem = 0;               // their dynamic shared memory
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t own = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    spgemm_status (*enqueue)(MultiState &, cudaStream_t) = nullptr;
    void release_all();
};

spgemm_status multi_create_typed(MultiState &ms, const spgemm_csc *As, const spgemm_csc *Bs,
                                 cudaStream_t st);

}  // namespace spg

struct spgemm_multi_s {
    spg::MultiState ms;
};
