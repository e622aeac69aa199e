/*
 * spgemm.h -- C ABI of the GB300 (sm_103a) memory-constrained SpGEMM library.
 *
 * The library computes C = A * B for sparse matrices in compressed sparse
 * column (CSC) form over the plus-times semiring, with int32 or int64 indices
 * and float64, float32 or int64 values. It restates, for one GPU, the local
 * hot path of Hussain, Selvitopi, Buluc and Azad, "Communication-Avoiding and
 * Memory-Constrained Sparse Matrix-Matrix Multiplication at Extreme Scale":
 *
 *   - the symbolic step that counts nonzeros per output column and chooses the
 *     number of column batches b for a memory budget (Algorithm 3, Eq. (2));
 *   - the sort-free hash-accumulator Gustavson multiply (Sec. II-C formula,
 *     Sec. IV-D "sort-free local SpGEMM");
 *   - the sort-free hash merge of partial products when the inner dimension is
 *     split into stages (Algorithm 1's stages and merge, Sec. IV-D);
 *   - the batch loop that hands each finished column batch of C to the host
 *     (Algorithm 4).
 *
 * Conventions for every call:
 *   - Every function returns an spgemm_status; no exception or abort crosses
 *     the ABI. spgemm_last_error() returns a message for the calling thread's
 *     last failure.
 *   - Matrix pointers inside spgemm_csc are DEVICE pointers unless a call says
 *     otherwise. The caller owns them; the library never frees them.
 *   - Rows inside an input column may be stored in any order. An input (row,
 *     col) pair that appears twice behaves as if its values were summed.
 *   - Output columns are NOT sorted by row unless a call says so (the paper
 *     keeps intermediate results unsorted, Sec. IV-D).
 *   - Structural nonzeros of C are all (i, j) reached by at least one product
 *     A(i,k) B(k,j); sums that cancel to zero are still stored.
 *   - float32 products are accumulated in float32, float64 in float64, int64
 *     with two's-complement wrap-around. Floating-point summation order is
 *     unspecified (hash-table atomics), so results may differ in the last bits
 *     between runs.
 *   - Calls enqueue work on the given stream and return without waiting,
 *     except where a call documents a host synchronisation.
 *   - A plan is not thread-safe; use one plan per host thread.
 *   - There is no CPU fallback: without a usable sm_103a device every compute
 *     call returns SPGEMM_ERR_CUDA.
 */
#ifndef SPGEMM_GB300_H
#define SPGEMM_GB300_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SPGEMM_OK = 0,
    SPGEMM_ERR_INVALID = 1,        /* bad argument, shape or type mismatch, corrupt CSC */
    SPGEMM_ERR_OOM = 2,            /* device or pinned-host allocation failed */
    SPGEMM_ERR_BUDGET = 3,         /* budget below A + B + workspace, or one column alone exceeds a batch */
    SPGEMM_ERR_OVERFLOW = 4,       /* a hash table probe exceeded its bound (internal error guard) */
    SPGEMM_ERR_INDEX_OVERFLOW = 5, /* an output offset does not fit the requested index type */
    SPGEMM_ERR_CUDA = 6,           /* a CUDA runtime call failed (message has the CUDA error) */
    SPGEMM_ERR_TIMEOUT = 7,        /* reserved: a bounded device-side wait gave up (no call waits on the device) */
    SPGEMM_ERR_SINK = 8,           /* the batch sink callback returned non-zero */
    SPGEMM_ERR_STATE = 9           /* call out of order (e.g. numeric before symbolic) */
} spgemm_status;

typedef enum { SPGEMM_I32 = 0, SPGEMM_I64 = 1 } spgemm_index_t;
typedef enum { SPGEMM_F64 = 0, SPGEMM_F32 = 1, SPGEMM_INT64 = 2 } spgemm_value_t;

/*
 * The semiring of the product (the paper's algorithms hold over any semiring,
 * Sec. II). PLUS_TIMES: C(i,j) = sum_k A(i,k) B(k,j). MIN_PLUS (float64 and
 * float32 values): C(i,j) = min_k A(i,k) + B(k,j), NaN sums ignored (a column
 * entry whose every candidate is NaN holds +infinity). OR_AND (any value
 * type, Boolean): a value is true when nonzero (-0.0 false, NaN true);
 * C(i,j) = 1 if A(i,k) and B(k,j) are both true for some k, else 0, in the
 * value type. The structure of C is the same in all three.
 */
typedef enum { SPGEMM_PLUS_TIMES = 0, SPGEMM_MIN_PLUS = 1, SPGEMM_OR_AND = 2 } spgemm_semiring_t;

/* How the k-split (kstages = s > 1) sums a batch's stage partials D_0..D_{s-1}.
 * AT_END: all s partials are kept and hash-merged once (the paper's choice,
 * Sec. IV-D); a batch holds sum_t nnz(D_t) partial entries.
 * INCREMENTAL: each stage is merged into the running sum as soon as it is
 * produced, M_t = M_{t-1} + D_t (M_0 = D_0, M_{s-1} = C); a batch holds one
 * stage partial and two running sums, max_t nnz(D_t) + 2 max_t nnz(M_t)
 * entries (one running sum when s = 2), at the price of re-reading M_{t-1}
 * in every merge and of s - 2 more symbolic passes that count nnz(M_t). */
typedef enum { SPGEMM_MERGE_AT_END = 0, SPGEMM_MERGE_INCREMENTAL = 1 } spgemm_merge_t;

/*
 * A CSC matrix: colptr[ncols+1] (type ptr_type), rowidx[nnz] and vals[nnz]
 * (types idx_type and val_type). For inputs ptr_type must equal idx_type.
 * For outputs ptr_type may be SPGEMM_I64 while idx_type is SPGEMM_I32.
 * Row indices must be < 2^31 - 1 (the hash tables hold 32-bit keys).
 */
typedef struct {
    int64_t nrows;
    int64_t ncols;
    int64_t nnz;
    void *colptr;
    void *rowidx;
    void *vals;
    spgemm_index_t ptr_type;
    spgemm_index_t idx_type;
    spgemm_value_t val_type;
} spgemm_csc;

/*
 * Tuning knobs. Zero in any field means "library default". The autotuner in
 * the Python package fills these from timed trials.
 *   hash_max_cap   largest column (distinct rows) kept in a shared-memory hash
 *                  table; larger columns use the dense row-panel accumulator.
 *                  Powers of two from 256 to 8192.
 *   panel_rows     rows per dense row panel (2^13, 2^14 or 2^15).
 *   short_seg      A-column segments up to this length are walked by one thread;
 *                  longer ones by a whole warp (1..64).
 *   huge_seg       segments longer than this are walked by the whole CTA.
 *   block_tier_threads  threads per CTA of the hash tiers (128..1024).
 *   hybrid_sort    1: a column of the CTA hash tiers whose products fit its
 *                  table (at most 2x its distinct rows, i.e. a low compression
 *                  factor) is accumulated by sorting its products by row and
 *                  summing equal rows instead of hashing them (a hybrid
 *                  accumulator chosen per column); 0: hash only.
 *   warp_max_cap   batched products (spgemm_multi_*): largest column bound
 *                  handled by one warp with a private table (32, 128, 256 or
 *                  512; default 256); larger columns take a whole CTA.
 * For spgemm_multi_*, hash_max_cap is the largest shared-memory table (larger
 * columns use a global-memory table; default 1024) and block_tier_threads the
 * CTA width of its persistent passes (128, 256 or 512; default 128).
 */
typedef struct {
    int hash_max_cap;
    int panel_rows;
    int short_seg;
    int huge_seg;
    int block_tier_threads;
    int hybrid_sort;
    int warp_max_cap;
    int reserved[1];
} spgemm_tuning;

/*
 * Caller-supplied memory for a plan's workspace. The paper's processes hold
 * the batch buffers of Algorithm 4 inside a fixed memory budget (Sec. IV-A);
 * here the application that owns the device memory (for example PyTorch's
 * caching allocator) hands it to the library through these callbacks.
 *   alloc(ctx, bytes, kind) returns `bytes` of memory of `kind`, aligned to
 *     256 bytes, or NULL when it cannot (the call then fails with
 *     SPGEMM_ERR_OOM and frees what it had allocated for the failed step);
 *   free(ctx, p, bytes, kind) returns a block that alloc gave. The library
 *     calls it only after the device has finished every use of the block
 *     (it synchronises the device first), when a buffer grows or when the
 *     plan is destroyed.
 * Both run on the calling host thread with the plan's device current, from
 * inside the library call that needs the memory; they must not call back
 * into the library. kind: SPGEMM_MEM_DEVICE for device memory,
 * SPGEMM_MEM_PINNED_HOST for page-locked host memory (the host ring of
 * spgemm_run_batched and small staging reads).
 */
typedef enum { SPGEMM_MEM_DEVICE = 0, SPGEMM_MEM_PINNED_HOST = 1 } spgemm_mem_kind;
typedef void *(*spgemm_alloc_fn)(void *ctx, size_t bytes, int kind);
typedef void (*spgemm_free_fn)(void *ctx, void *p, size_t bytes, int kind);
typedef struct {
    spgemm_alloc_fn alloc;   /* both non-NULL */
    spgemm_free_fn free;
    void *ctx;               /* passed back unchanged */
} spgemm_allocator;

typedef struct {
    size_t budget_bytes;     /* device memory for A, B, workspace and batch outputs;
                                0 = 80% of the free device memory at plan time */
    int kstages;             /* s >= 1: split the inner dimension into s contiguous stages
                                (A by columns, B by rows) and hash-merge the partials */
    int ring_depth;          /* device output buffers kept in flight by spgemm_run_batched (>= 1; 0 = 2) */
    size_t host_slot_bytes;  /* pinned host slot size for spgemm_run_batched (0 = 256 MiB) */
    int host_slots;          /* pinned host slots (>= 2; 0 = 3) */
    int sort_output;         /* 1: sort rows inside each output column (the paper keeps the final
                                C sorted within columns, Sec. IV-D); 0: unsorted */
    const spgemm_tuning *tuning; /* NULL = defaults */
    int prune;               /* 1: spgemm_run_batched prunes every batch on the device before its
                                copy to the host, with spgemm_prune's rule and the two fields
                                below (the batch consumer of Sec. III / V-F); 0: off */
    double prune_threshold;  /* keep values >= this (-INFINITY: no threshold) */
    int64_t prune_topk;      /* then at most this many per column (<= 0: no limit) */
    int semiring;            /* spgemm_semiring_t (0 = plus-times); min-plus and or-and apply
                                to the product, the k-stage merge and spgemm_run_batched,
                                and spgemm_backward refuses them */
    int merge_mode;          /* spgemm_merge_t (0 = merge at the end); used when kstages > 1 */
    const spgemm_allocator *allocator; /* workspace memory of the plan (copied at plan
                                creation); NULL: cudaMalloc and cudaHostAlloc */
} spgemm_opts;

typedef struct spgemm_plan_s spgemm_plan;

/* Summary filled by spgemm_plan_query after spgemm_symbolic. */
typedef struct {
    int64_t flops;            /* sum_j f_j: multiplications (Sec. II-A) */
    int64_t nnz_c;            /* nnz(C) */
    int64_t unmerged_nnz;     /* sum_t nnz(D_t) over the s stages (= nnz_c when s = 1) */
    int64_t nbatches;         /* b */
    int64_t max_batch_nnz;    /* largest nnz(C) of one batch */
    int64_t max_batch_cols;
    int64_t bytes_per_nnz;    /* r = index bytes + value bytes */
    int64_t batch_cap_bytes;  /* bytes one batch may occupy on the device */
    int64_t heavy_columns;    /* columns handled by the dense row-panel accumulator */
    int64_t stage_buffer_nnz; /* k-split: entries the largest batch's stage buffers hold
                                 (sum_t nnz(D_t) merging at the end; max_t nnz(D_t) plus
                                 the running sums merging incrementally); 0 when s = 1 */
} spgemm_plan_info;

/*
 * Per-phase statistics of a plan (kernel launches always; device time only
 * while timing is enabled). Phases: 0 flop count + binning, 1 symbolic hash
 * tiers, 2 symbolic bitmap (heavy columns), 3 scans, 4 row-panel copy of A,
 * 5 numeric hash tiers, 6 numeric heavy columns (dense row panels and hash
 * row ranges), 7 stage merge, 8 backward. Times come from CUDA events
 * recorded on the stream each phase was launched on.
 */
#define SPGEMM_NUM_PHASES 9
typedef struct {
    int64_t launches;                  /* kernel launches since the last reset */
    double ms[SPGEMM_NUM_PHASES];      /* summed device time per phase */
    int64_t count[SPGEMM_NUM_PHASES];  /* timed instances per phase */
} spgemm_stats;

/* Thread-local message of the last failing call (never NULL). */
const char *spgemm_last_error(void);

/* Library version string. */
const char *spgemm_version(void);

/*
 * spgemm_plan_create -- validate A and B and set up a plan for C = A * B.
 * Checks A.ncols == B.nrows, equal index and value types, nnz == colptr[ncols]
 * (one device read) and, when validate != 0, monotone colptr and rows in range
 * (a device check, one synchronisation). The plan is the state of one product
 * C = A * B (the problem of Sec. II-B) through Algorithm 3's symbolic step and
 * Algorithm 4's batches. Plan workspace, and the pinned host ring of
 * spgemm_run_batched, come from opts->allocator when it is set, else from
 * cudaMalloc / cudaHostAlloc; every later call on the plan uses the same
 * allocator. A and B must stay valid and unchanged for the plan's lifetime.
 * Errors: SPGEMM_ERR_INVALID (also an allocator with a NULL callback),
 * SPGEMM_ERR_OOM (an allocation failed; nothing the failed call allocated is
 * kept), SPGEMM_ERR_CUDA.
 */
spgemm_status spgemm_plan_create(const spgemm_csc *A, const spgemm_csc *B,
                                 const spgemm_opts *opts, int validate,
                                 cudaStream_t stream, spgemm_plan **out);

/* Release a plan and all workspace it owns. NULL is accepted. */
spgemm_status spgemm_plan_destroy(spgemm_plan *plan);

/*
 * spgemm_symbolic -- the symbolic step (Algorithm 3 on one device):
 * flops per column (Sec. II-A), exact nnz per output column by hash /
 * bitmap insertion (LocalSymbolic), with s > 1 also the per-stage counts
 * nnz(D_t(:, j)) whose sum is the unmerged memory of Eq. (1), and the batch
 * plan: the smallest number of contiguous column ranges whose outputs fit the
 * budget (Eq. (2), Sec. V-C). Synchronises the stream once (to read totals).
 *
 * The batch plan. With r = index bytes + value bytes, a batch over columns
 * [c0, c1) needs these bytes (sums over the batch's columns j):
 *   sum_j (r nnz(C(:,j)) + 8)                      the output and an int64 colptr
 *   + r sum_j sum_t nnz(D_t(:,j))                  kstages = s > 1, merge at the end:
 *                                                  every stage partial of the batch
 *   + r (max_{t>=1} sum_j nnz(D_t(:,j))            s > 1, incremental merge: one stage
 *        + m max_{u<=s-2} sum_j nnz(M_u(:,j)))     partial and m running sums (m = 2,
 *                                                  1 when s = 2; M_u = the product over
 *                                                  stages 0..u, M_0 = D_0)
 *   + sum_j (r min(nnz(C(:,j)), topk) + 8 + 40)    opts.prune: the pruned copy, its
 *                                                  colptr and 40 B of prune workspace
 *                                                  per column (topk <= 0: nnz(C(:,j)))
 * The cap of one batch (spgemm_plan_info.batch_cap_bytes) is (budget -
 * r (nnz(A) + nnz(B)) - index bytes (ncols(A) + ncols(B) + 2) - plan
 * workspace) / ring_depth. Starting at column 0, each range is extended while
 * the next column still fits under the cap; b is the number of ranges.
 * Errors: SPGEMM_ERR_BUDGET (inputs alone exceed the budget, or one column's
 * output exceeds a batch), SPGEMM_ERR_CUDA, SPGEMM_ERR_OOM.
 */
spgemm_status spgemm_symbolic(spgemm_plan *plan, cudaStream_t stream);

/* Plan summary (host struct). Errors: SPGEMM_ERR_STATE before symbolic. */
spgemm_status spgemm_plan_query(const spgemm_plan *plan, spgemm_plan_info *info);

/* Column range [col_begin, col_end) and nnz of batch t (host values). */
spgemm_status spgemm_plan_batch(const spgemm_plan *plan, int64_t t, int64_t *col_begin,
                                int64_t *col_end, int64_t *nnz);

/*
 * Copy the per-column output counts nnz(C(:, j)) (int64, B.ncols entries) to
 * the device buffer counts_out, enqueued on stream.
 */
spgemm_status spgemm_plan_column_counts(const spgemm_plan *plan, int64_t *counts_out,
                                        cudaStream_t stream);

/*
 * Write the colptr of the whole product C (ncols+1 entries of type ptr_type,
 * device buffer) on stream. Errors: SPGEMM_ERR_STATE, SPGEMM_ERR_INDEX_OVERFLOW
 * (nnz(C) does not fit a 32-bit colptr).
 */
spgemm_status spgemm_plan_colptr(const spgemm_plan *plan, void *colptr_out,
                                 spgemm_index_t ptr_type, cudaStream_t stream);

/*
 * Synchronise the stream and report the plan's device error flags: returns
 * SPGEMM_ERR_OVERFLOW if a kernel found a hash probe sequence longer than its
 * table or a column whose numeric nnz differed from its symbolic count
 * (internal consistency guards; neither happens on valid input).
 */
spgemm_status spgemm_plan_check(const spgemm_plan *plan, cudaStream_t stream);

/*
 * Enable (1) or disable (0) per-phase event timing on the plan. Timing adds
 * two event records per phase; results are read with spgemm_plan_stats.
 */
spgemm_status spgemm_plan_set_timing(spgemm_plan *plan, int enable);

/*
 * Read the plan's statistics (waits for the timed events to complete), then
 * clear them when reset != 0.
 */
spgemm_status spgemm_plan_stats(spgemm_plan *plan, int reset, spgemm_stats *out);

/*
 * spgemm_numeric -- compute batch t of C (columns [col_begin, col_end) of the
 * plan) into caller-allocated device buffers: C_out->colptr (ncols+1 entries,
 * offsets relative to the batch), rowidx and vals (nnz entries each), with
 * nrows = A.nrows, ncols and nnz as spgemm_plan_batch reports. Columns are
 * unsorted unless opts.sort_output. With s > 1 stages the stage products
 * D_t are formed in plan workspace and hash-merged (Algorithm 1's merge).
 * Errors: SPGEMM_ERR_STATE, SPGEMM_ERR_INVALID (shape/type of C_out),
 * SPGEMM_ERR_INDEX_OVERFLOW (nnz does not fit a 32-bit colptr), SPGEMM_ERR_CUDA,
 * SPGEMM_ERR_OVERFLOW (internal hash-probe guard tripped).
 */
spgemm_status spgemm_numeric(spgemm_plan *plan, int64_t t, spgemm_csc *C_out,
                             cudaStream_t stream);

/*
 * spgemm_merge -- sort-free hash merge (Sec. IV-D): out(:, j) = sum over parts
 * of parts[i](:, j), adding values of equal rows. All parts share shape and
 * types. Two calls: with out->rowidx == NULL the call fills out->colptr
 * (device, ncols+1, type out->ptr_type) and sets out->nnz, synchronising the
 * stream once; the second call (rowidx and vals allocated with out->nnz
 * entries, colptr unchanged) fills them. Unsorted output.
 * Errors: SPGEMM_ERR_INVALID, SPGEMM_ERR_CUDA, SPGEMM_ERR_OOM, SPGEMM_ERR_INDEX_OVERFLOW.
 */
spgemm_status spgemm_merge(const spgemm_csc *parts, int nparts, spgemm_csc *out,
                           cudaStream_t stream);

/*
 * spgemm_prune -- column-wise prune of a result batch (Markov clustering keeps
 * the largest entries of every column of each batch, Sec. III; HipMCL prunes
 * each batch, Sec. V-F). For each column of `in`, in storage order:
 *   1. candidates are the entries with value >= threshold (compared in the
 *      value type against the smallest representable value >= threshold;
 *      NaN is never a candidate; -INFINITY keeps every non-NaN entry);
 *   2. if topk > 0 and more than topk candidates remain, the topk largest are
 *      kept; among equal values the earlier stored entry wins (for sorted
 *      columns: the smaller row);
 *   3. the kept entries are written in their input order (sorted input gives
 *      sorted output).
 * `in`: device CSC as produced by spgemm_numeric (ptr I32 or I64, idx and
 * value types as the product). `out`: same nrows, ncols, idx_type and
 * val_type; out->ptr_type SPGEMM_I64. Two calls, as spgemm_merge: with
 * out->rowidx == NULL the call fills out->colptr (device, ncols+1 int64) and
 * sets out->nnz, synchronising the stream once; the second call (rowidx and
 * vals allocated with out->nnz entries, colptr unchanged) fills them.
 * Errors: SPGEMM_ERR_INVALID, SPGEMM_ERR_OOM, SPGEMM_ERR_CUDA.
 */
spgemm_status spgemm_prune(const spgemm_csc *in, double threshold, int64_t topk, spgemm_csc *out,
                           cudaStream_t stream);

/*
 * spgemm_transpose -- out = in^T on the device (the CSC of the transpose, i.e.
 * the CSR of `in`). A^T serves the A A^T products of Sec. V (BELLA's shared
 * k-mers) and the row-by-row batching Sec. IV-B mentions for square inputs:
 * the row batches of C = A B are the column batches of C^T = B^T A^T.
 * `out`: nrows = in.ncols, ncols = in.nrows, nnz = in.nnz, the same index and
 * value types, colptr (in.nrows + 1 entries, I32 or I64), rowidx and vals all
 * caller-allocated. Rows inside an output column come in unspecified order.
 * Synchronises the stream once (the work buffers are freed on return).
 * Errors: SPGEMM_ERR_INVALID (shapes, types, a row index outside [0, nrows)),
 * SPGEMM_ERR_INDEX_OVERFLOW, SPGEMM_ERR_OOM, SPGEMM_ERR_CUDA.
 */
spgemm_status spgemm_transpose(const spgemm_csc *in, spgemm_csc *out, cudaStream_t stream);

/*
 * spgemm_merge_noalloc -- the same merge as spgemm_merge (same arguments, same
 * two-call protocol, unsorted output) for callers that may not allocate device
 * memory, e.g. code running under another framework's fixed device-memory pool
 * or in a loop where cudaMalloc's implicit synchronisation is not acceptable.
 * The paper has no counterpart; this is a calling convention of the library.
 * It calls no cudaMalloc, cudaFree or other allocating routine: its work
 * buffers live in one 32 MiB device array that every GPU loading the library
 * keeps until exit, so it accepts at most about 1.1 million columns
 * (29 bytes per column plus a few KiB) and at most 64 parts, and for every
 * column the number of entries summed over the parts, capped at nrows, must
 * be at most 8192 (the tier is chosen from that bound before the rows are
 * counted, and the largest shared-memory hash table holds 8192 rows; parts
 * that share rows count each copy); larger inputs return SPGEMM_ERR_INVALID
 * with the limit in the message. The first call on each device looks up the
 * array's address on that device. Every call synchronises the stream once (to
 * read the merged size). All calls on
 * one device share that device's array (it keeps the last call's contents):
 * calls that overlap on one GPU race, so serialise them.
 * Errors: as spgemm_merge, plus SPGEMM_ERR_INVALID for sizes beyond the array.
 */
spgemm_status spgemm_merge_noalloc(const spgemm_csc *parts, int nparts, spgemm_csc *out,
                                   cudaStream_t stream);

/*
 * Sink for spgemm_run_batched. Called on the calling host thread once per
 * finished piece of C: columns [col_begin, col_end) of C, a CSC whose arrays
 * are PINNED HOST memory owned by the library and valid only during the call
 * (colptr is int64 and relative to the piece). A batch arrives as one or more
 * pieces, in column order. Return 0 to continue, non-zero to stop (the run
 * then drains in-flight copies and returns SPGEMM_ERR_SINK).
 */
typedef int (*spgemm_sink_fn)(void *ctx, int64_t batch, int64_t col_begin, int64_t col_end,
                              const spgemm_csc *piece);

/*
 * spgemm_run_batched -- the memory-constrained batch loop (Algorithm 4): for
 * every batch t = 0..b-1, compute C[t] on `compute` into one of ring_depth
 * device buffers, then copy it on `copy` into pinned host slots and hand it to
 * the sink, overlapping the copy of batch t with the multiply of batch t+1.
 * With opts.sort_output the columns arrive sorted by row; with opts.prune each
 * batch is pruned on the device (spgemm_prune's rule) before the copy, so only
 * the kept entries cross to the host (the plan's batches then also hold the
 * pruned copy: at most min(nnz(C(:,j)), topk) entries per column). With both,
 * the result is that of sorting first and pruning after (equal values go to
 * the smaller rows); for 0 < topk <= 8192 the batch is pruned unsorted and
 * only the kept entries are sorted.
 * Requires spgemm_symbolic first. Returns after the last sink call.
 * Errors: SPGEMM_ERR_SINK, SPGEMM_ERR_OOM, SPGEMM_ERR_CUDA, SPGEMM_ERR_STATE.
 */
spgemm_status spgemm_run_batched(spgemm_plan *plan, spgemm_sink_fn sink, void *ctx,
                                 cudaStream_t compute, cudaStream_t copy);

/*
 * spgemm_backward -- gradients of loss = sum over pattern(C) of C(i,j) G(i,j)
 * with respect to the stored values of A and B (not in the paper; follows
 * from the Sec. II-C product): dA(i,k) = sum_j G(i,j) B(k,j) on pattern(A),
 * dB(k,j) = sum_i A(i,k) G(i,j) on pattern(B). G is a device CSC with C's
 * shape and pattern (any row order inside columns), same value type as A.
 * dA_vals / dB_vals are device arrays of nnz(A) / nnz(B) values in A's / B's
 * storage order, overwritten. Floating-point values only. Works on plans with
 * s = 1; needs no symbolic step (G carries the pattern).
 * Errors: SPGEMM_ERR_INVALID, SPGEMM_ERR_CUDA, SPGEMM_ERR_OVERFLOW.
 */
spgemm_status spgemm_backward(spgemm_plan *plan, const spgemm_csc *G, void *dA_vals,
                              void *dB_vals, cudaStream_t stream);

/* ---------------------------------------------------------------------------
 * Many independent products C_i = A_i * B_i of uneven sizes in one pass.
 * ------------------------------------------------------------------------- */
typedef struct spgemm_multi_s spgemm_multi;

/*
 * spgemm_multi_create -- plan nprob products (all with the same index and
 * value types). The host arrays As and Bs (nprob entries each) are copied;
 * their device buffers must stay valid. The output is one arena: the
 * concatenation of the C_i column by column (C_i's columns follow C_{i-1}'s;
 * rows stay local to each problem), with an int64 colptr over all
 * sum_i B_i.ncols columns. The arena is sized from the flop count
 * (nnz(C_i) <= flops_i), so the whole pipeline needs no host synchronisation
 * and can be captured in a CUDA graph. Of opts only the tuning applies:
 * kstages > 1, a semiring other than plus-times, sort_output and prune are
 * refused with SPGEMM_ERR_INVALID. Errors: SPGEMM_ERR_INVALID,
 * SPGEMM_ERR_OOM, SPGEMM_ERR_CUDA.
 */
spgemm_status spgemm_multi_create(int nprob, const spgemm_csc *As, const spgemm_csc *Bs,
                                  const spgemm_opts *opts, cudaStream_t stream,
                                  spgemm_multi **out);

spgemm_status spgemm_multi_destroy(spgemm_multi *m);

/*
 * spgemm_multi_run -- flops, symbolic, scan and numeric for all problems,
 * enqueued on stream without host synchronisation. With use_graph != 0 the
 * sequence is captured once into a CUDA graph and replayed on later calls.
 */
spgemm_status spgemm_multi_run(spgemm_multi *m, int use_graph, cudaStream_t stream);

/*
 * Device pointers of the output arena (valid until destroy): colptr (int64,
 * total_cols+1 entries, global offsets), rowidx (index type of the inputs),
 * vals; plus total_cols and the arena capacity in entries. The product's nnz
 * is colptr[total_cols] (read it after the stream completes).
 */
spgemm_status spgemm_multi_output(const spgemm_multi *m, int64_t **colptr, void **rowidx,
                                  void **vals, int64_t *total_cols, int64_t *capacity);

#ifdef __cplusplus
}
#endif
#endif /* SPGEMM_GB300_H */
