/*
 * CPU oracle for the memory-constrained SpGEMM hot path.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow, obviously correct
 * definition that the CUDA path is checked against. Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg may load it; the library itself
 * never calls it and shares no code, header or table with it.
 *
 * Conventions (all functions):
 *   - CSC with int64 colptr / rowidx (the Python wrapper widens int32 input).
 *   - Values: vtype 0 = float64 (float32 inputs are upcast exactly by the
 *     wrapper and accumulated in float64), vtype 2 = int64 accumulated with
 *     two's-complement wrap-around (done in uint64_t), vtype 3 = float64 over
 *     the min-plus semiring (the paper's algorithms hold over any semiring,
 *     Sec. II): a (x) b = a + b, (+) = min, NaN products ignored (fmin);
 *     vtype 4 (float64 storage) and vtype 5 (int64 storage) = the Boolean
 *     or-and semiring: a value is true when it is nonzero (-0.0 is false, NaN
 *     true), a (x) b = a AND b, (+) = OR, and an entry of C holds 1 when one
 *     of its products is true, else 0.
 *   - Rows inside an input column may be in any order; (row, col) is unique.
 *   - Output columns are sorted ascending by row; numerically-zero sums are
 *     kept as structural nonzeros (a nonzero of C is any (i, j) reached by at
 *     least one product).
 *   - The k-range [k0, k1) restricts the product to A(:, k0:k1) * B(k0:k1, :),
 *     i.e. one stage of a split inner dimension (Algorithm 1's stages).
 *
 * Parallelism: OpenMP over output columns with one dense accumulator per
 * thread; the arithmetic per column is the sequential definition.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int64_t nrows, ncols;
    const int64_t *colptr;
    const int64_t *rowidx;
    const void *vals; /* double* (vtype 0) or int64_t* (vtype 2) */
} ocsc;

static int cmp_i64(const void *a, const void *b) {
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/*
 * flops per output column (Sec. II-A: flops = number of multiplications).
 * f[j] = sum over B(k, j) != 0 with k0 <= k < k1 of nnz(A(:, k)).
 */
void oracle_flops(const ocsc *A, const ocsc *B, int64_t k0, int64_t k1, int64_t *f) {
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t j = 0; j < B->ncols; ++j) {
        int64_t s = 0;
        for (int64_t p = B->colptr[j]; p < B->colptr[j + 1]; ++p) {
            int64_t k = B->rowidx[p];
            if (k < k0 || k >= k1) continue;
            s += A->colptr[k + 1] - A->colptr[k];
        }
        f[j] = s;
    }
}

/*
 * Number of structural nonzeros of C(:, j) for j in [c0, c1) (the quantity
 * LocalSymbolic produces in Algorithm 3): the number of distinct rows in the
 * union of A(:, k) over B(k, j) != 0, k in [k0, k1). Dense marker array.
 */
void oracle_symbolic(const ocsc *A, const ocsc *B, int64_t k0, int64_t k1,
                     int64_t c0, int64_t c1, int64_t *cnt) {
#pragma omp parallel
    {
        int64_t *mark = (int64_t *)malloc(sizeof(int64_t) * (size_t)(A->nrows > 0 ? A->nrows : 1));
        for (int64_t i = 0; i < A->nrows; ++i) mark[i] = -1;
#pragma omp for schedule(dynamic, 64)
        for (int64_t j = c0; j < c1; ++j) {
            int64_t c = 0;
            for (int64_t p = B->colptr[j]; p < B->colptr[j + 1]; ++p) {
                int64_t k = B->rowidx[p];
                if (k < k0 || k >= k1) continue;
                for (int64_t q = A->colptr[k]; q < A->colptr[k + 1]; ++q) {
                    int64_t i = A->rowidx[q];
                    if (mark[i] != j) { mark[i] = j; ++c; }
                }
            }
            cnt[j - c0] = c;
        }
        free(mark);
    }
}

/*
 * Column-Gustavson product (Sec. II-C): C(:, j) = sum_{k : B(k,j) != 0}
 * A(:, k) B(k, j), for j in [c0, c1), with a dense sparse accumulator.
 * The caller supplies colptr_out (c1-c0+1 entries, from oracle_symbolic's
 * counts) and arrays of that many entries. absterm_out (may be NULL; float
 * only) receives sum |A(i,k) B(k,j)| per output entry, the scale of the
 * rounding error any reordering of the sum may have. nterm_out (may be NULL)
 * receives, per output entry, the number of products A(i,k) B(k,j) that reach
 * it: the n of the summation error bound of that entry alone.
 */
void oracle_spgemm(const ocsc *A, const ocsc *B, int vtype, int64_t k0, int64_t k1,
                   int64_t c0, int64_t c1, const int64_t *colptr_out,
                   int64_t *rowidx_out, void *vals_out, double *absterm_out,
                   int64_t *nterm_out) {
#pragma omp parallel
    {
        int64_t m = A->nrows > 0 ? A->nrows : 1;
        int64_t *mark = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
        double *spa = (double *)malloc(sizeof(double) * (size_t)m);
        double *spa_abs = (double *)malloc(sizeof(double) * (size_t)m);
        uint64_t *spa_i = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)m);
        int64_t *spa_n = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
        for (int64_t i = 0; i < A->nrows; ++i) mark[i] = -1;
#pragma omp for schedule(dynamic, 64)
        for (int64_t j = c0; j < c1; ++j) {
            int64_t base = colptr_out[j - c0];
            int64_t len = 0;
            for (int64_t p = B->colptr[j]; p < B->colptr[j + 1]; ++p) {
                int64_t k = B->rowidx[p];
                if (k < k0 || k >= k1) continue;
                for (int64_t q = A->colptr[k]; q < A->colptr[k + 1]; ++q) {
                    int64_t i = A->rowidx[q];
                    if (mark[i] != j) {
                        mark[i] = j;
                        rowidx_out[base + len++] = i;
                        spa[i] = vtype == 3 ? INFINITY : 0.0;   /* the (+) identity */
                        spa_abs[i] = 0.0; spa_i[i] = 0; spa_n[i] = 0;
                    }
                    ++spa_n[i];
                    if (vtype == 2) {
                        uint64_t a = (uint64_t)((const int64_t *)A->vals)[q];
                        uint64_t b = (uint64_t)((const int64_t *)B->vals)[p];
                        spa_i[i] += a * b;
                    } else if (vtype == 3) {
                        const double a = ((const double *)A->vals)[q], b = ((const double *)B->vals)[p];
                        spa[i] = fmin(spa[i], a + b);
                        const double s = fabs(a) + fabs(b);
                        if (s > spa_abs[i]) spa_abs[i] = s;
                    } else if (vtype == 4 || vtype == 5) {
                        const int a = vtype == 4 ? ((const double *)A->vals)[q] != 0.0
                                                 : ((const int64_t *)A->vals)[q] != 0;
                        const int b = vtype == 4 ? ((const double *)B->vals)[p] != 0.0
                                                 : ((const int64_t *)B->vals)[p] != 0;
                        if (a && b) spa_i[i] = 1;
                    } else {
                        double t = ((const double *)A->vals)[q] * ((const double *)B->vals)[p];
                        spa[i] += t;
                        spa_abs[i] += t < 0 ? -t : t;
                    }
                }
            }
            qsort(rowidx_out + base, (size_t)len, sizeof(int64_t), cmp_i64);
            for (int64_t t = 0; t < len; ++t) {
                int64_t i = rowidx_out[base + t];
                if (vtype == 2 || vtype == 5) ((int64_t *)vals_out)[base + t] = (int64_t)spa_i[i];
                else if (vtype == 4) ((double *)vals_out)[base + t] = (double)spa_i[i];
                else {
                    ((double *)vals_out)[base + t] = spa[i];
                    if (absterm_out) absterm_out[base + t] = spa_abs[i];
                }
                if (nterm_out) nterm_out[base + t] = spa_n[i];
            }
        }
        free(mark); free(spa); free(spa_abs); free(spa_i); free(spa_n);
    }
}

/*
 * Merge of partial results (Sec. III-A, the step after all SUMMA stages):
 * entries of the nparts inputs with the same (row, col) are added. Column j of
 * the output is formed from column j of every part (the hash-merge's
 * contract, Sec. IV-D); output sorted by row. cnt_only != 0: only fill
 * colptr_out[1..] with per-column counts (colptr_out[0] = 0, then prefix).
 */
void oracle_merge(const ocsc *parts, int nparts, int vtype, int cnt_only,
                  int64_t *colptr_out, int64_t *rowidx_out, void *vals_out) {
    int64_t m = parts[0].nrows, n = parts[0].ncols;
    if (cnt_only) {
        int64_t *mark = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
        for (int64_t i = 0; i < m; ++i) mark[i] = -1;
        colptr_out[0] = 0;
        for (int64_t j = 0; j < n; ++j) {
            int64_t c = 0;
            for (int t = 0; t < nparts; ++t)
                for (int64_t q = parts[t].colptr[j]; q < parts[t].colptr[j + 1]; ++q) {
                    int64_t i = parts[t].rowidx[q];
                    if (mark[i] != j) { mark[i] = j; ++c; }
                }
            colptr_out[j + 1] = colptr_out[j] + c;
        }
        free(mark);
        return;
    }
#pragma omp parallel
    {
        int64_t *mark = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
        double *spa = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
        uint64_t *spa_i = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(m > 0 ? m : 1));
        for (int64_t i = 0; i < m; ++i) mark[i] = -1;
#pragma omp for schedule(dynamic, 64)
        for (int64_t j = 0; j < n; ++j) {
            int64_t base = colptr_out[j], len = 0;
            for (int t = 0; t < nparts; ++t)
                for (int64_t q = parts[t].colptr[j]; q < parts[t].colptr[j + 1]; ++q) {
                    int64_t i = parts[t].rowidx[q];
                    if (mark[i] != j) {
                        mark[i] = j; rowidx_out[base + len++] = i;
                        spa[i] = vtype == 3 ? INFINITY : 0.0; spa_i[i] = 0;
                    }
                    if (vtype == 2) spa_i[i] += (uint64_t)((const int64_t *)parts[t].vals)[q];
                    else if (vtype == 3) spa[i] = fmin(spa[i], ((const double *)parts[t].vals)[q]);
                    else if (vtype == 4) { if (((const double *)parts[t].vals)[q] != 0.0) spa_i[i] = 1; }
                    else if (vtype == 5) { if (((const int64_t *)parts[t].vals)[q] != 0) spa_i[i] = 1; }
                    else spa[i] += ((const double *)parts[t].vals)[q];
                }
            qsort(rowidx_out + base, (size_t)len, sizeof(int64_t), cmp_i64);
            for (int64_t t = 0; t < len; ++t) {
                int64_t i = rowidx_out[base + t];
                if (vtype == 2 || vtype == 5) ((int64_t *)vals_out)[base + t] = (int64_t)spa_i[i];
                else if (vtype == 4) ((double *)vals_out)[base + t] = (double)spa_i[i];
                else ((double *)vals_out)[base + t] = spa[i];
            }
        }
        free(mark); free(spa); free(spa_i);
    }
}

/*
 * Gradients of loss = sum_{(i,j) in pattern(C)} C(i,j) G(i,j) with respect to
 * the stored values of A and B. Every product A(i,k) B(k,j) of the forward
 * Gustavson loop contributes G(i,j) B(k,j) to dA(i,k) and A(i,k) G(i,j) to
 * dB(k,j):  dA = (G B^T) masked to pattern(A),  dB = (A^T G) masked to
 * pattern(B). G is given as a CSC on pattern(C) (any row order).
 * Float64 only. Sequential (the dA updates of different columns collide).
 */
void oracle_backward(const ocsc *A, const ocsc *B, const ocsc *G,
                     double *dA, double *dB) {
    int64_t m = A->nrows > 0 ? A->nrows : 1;
    double *gcol = (double *)malloc(sizeof(double) * (size_t)m);
    int64_t *mark = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
    for (int64_t i = 0; i < A->nrows; ++i) mark[i] = -1;
    memset(dA, 0, sizeof(double) * (size_t)A->colptr[A->ncols]);
    memset(dB, 0, sizeof(double) * (size_t)B->colptr[B->ncols]);
    const double *av = (const double *)A->vals, *bv = (const double *)B->vals;
    const double *gv = (const double *)G->vals;
    for (int64_t j = 0; j < B->ncols; ++j) {
        for (int64_t q = G->colptr[j]; q < G->colptr[j + 1]; ++q) {
            mark[G->rowidx[q]] = j;
            gcol[G->rowidx[q]] = gv[q];
        }
        for (int64_t p = B->colptr[j]; p < B->colptr[j + 1]; ++p) {
            int64_t k = B->rowidx[p];
            for (int64_t q = A->colptr[k]; q < A->colptr[k + 1]; ++q) {
                int64_t i = A->rowidx[q];
                double g = (mark[i] == j) ? gcol[i] : 0.0;
                dA[q] += g * bv[p];
                dB[p] += av[q] * g;
            }
        }
    }
    free(gcol); free(mark);
}

/*
 * Batch plan (Algorithm 3's b and Algorithm 4's ColSplit, single device).
 * w[j] = bytes column j of the batch output needs (r * nnz, plus whatever the
 * caller folds in). Columns are cut into contiguous ranges; a new range starts
 * whenever adding the next column would push the running total above cap.
 * Writes range starts to begin[0..b] (begin[b] = n) and returns b, or -1 if a
 * single column alone exceeds cap. begin must hold n+1 entries.
 */
int64_t oracle_plan_batches(const int64_t *w, int64_t n, int64_t cap, int64_t *begin) {
    int64_t b = 0, acc = 0;
    begin[0] = 0;
    if (n == 0) { begin[1] = 0; return 1; }
    for (int64_t j = 0; j < n; ++j) {
        if (w[j] > cap) return -1;
        if (acc + w[j] > cap) { begin[++b] = j; acc = 0; }
        acc += w[j];
    }
    begin[++b] = n;
    return b;
}

/*
 * Column-wise prune of a result batch (the consumer Sec. III's batching is
 * shaped for: Markov clustering keeps the largest entries of every column of
 * each batch, Sec. V-F). Per column, in storage order:
 *   1. the candidates are the entries with value >= threshold (vtype 0:
 *      compared in float64; vtype 2: int64 compared against the smallest
 *      int64 >= threshold);
 *   2. if topk > 0 and more than topk candidates remain, keep the topk with
 *      the largest values; among equal values the earlier stored entry wins;
 *   3. the kept entries are written in their input order.
 * cnt_only != 0: only fill colptr_out (colptr_out[0] = 0, then the prefix of
 * kept counts). Otherwise colptr_out must already hold those offsets.
 */
typedef struct {
    int64_t pos;
    double v;
    int64_t vi;
} pcand;

static int g_prune_int;  /* comparator mode, set before each qsort (serial) */

static int cmp_cand_desc(const void *a, const void *b) {
    const pcand *x = (const pcand *)a, *y = (const pcand *)b;
    if (g_prune_int) {
        if (x->vi != y->vi) return x->vi > y->vi ? -1 : 1;
    } else {
        if (x->v != y->v) return x->v > y->v ? -1 : 1;
    }
    return (x->pos > y->pos) - (x->pos < y->pos);
}

static int cmp_cand_pos(const void *a, const void *b) {
    const pcand *x = (const pcand *)a, *y = (const pcand *)b;
    return (x->pos > y->pos) - (x->pos < y->pos);
}

void oracle_prune(const ocsc *C, int vtype, double threshold, int64_t topk, int cnt_only,
                  int64_t *colptr_out, int64_t *rowidx_out, void *vals_out) {
    const double *dv = (const double *)C->vals;
    const int64_t *iv = (const int64_t *)C->vals;
    int64_t ithr = INT64_MIN;
    if (vtype == 2 && threshold > -1e300) {
        if (threshold > 9.2e18) ithr = INT64_MAX;
        else {
            ithr = (int64_t)threshold;               /* truncation toward zero */
            if ((double)ithr < threshold) ++ithr;     /* smallest int64 >= threshold */
        }
    }
    int64_t maxlen = 1;
    for (int64_t j = 0; j < C->ncols; ++j)
        if (C->colptr[j + 1] - C->colptr[j] > maxlen) maxlen = C->colptr[j + 1] - C->colptr[j];
    pcand *cand = (pcand *)malloc(sizeof(pcand) * (size_t)maxlen);
    g_prune_int = vtype == 2;
    if (cnt_only) colptr_out[0] = 0;
    for (int64_t j = 0; j < C->ncols; ++j) {
        int64_t nc = 0;
        for (int64_t q = C->colptr[j]; q < C->colptr[j + 1]; ++q) {
            const int keep = vtype == 2 ? (iv[q] >= ithr) : (dv[q] >= threshold);
            if (keep) {
                cand[nc].pos = q;
                cand[nc].v = vtype == 2 ? 0.0 : dv[q];
                cand[nc].vi = vtype == 2 ? iv[q] : 0;
                ++nc;
            }
        }
        if (topk > 0 && nc > topk) {
            qsort(cand, (size_t)nc, sizeof(pcand), cmp_cand_desc);
            nc = topk;
            qsort(cand, (size_t)nc, sizeof(pcand), cmp_cand_pos);
        }
        if (cnt_only) {
            colptr_out[j + 1] = colptr_out[j] + nc;
            continue;
        }
        const int64_t base = colptr_out[j];
        for (int64_t t = 0; t < nc; ++t) {
            const int64_t q = cand[t].pos;
            rowidx_out[base + t] = C->rowidx[q];
            if (vtype == 2) ((int64_t *)vals_out)[base + t] = iv[q];
            else ((double *)vals_out)[base + t] = dv[q];
        }
    }
    free(cand);
}
