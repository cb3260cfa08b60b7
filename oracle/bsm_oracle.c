/*
 * bsm_oracle.c -- plain, slow, obviously correct CPU oracle for the local
 * block-sparse matrix product of the DBCSR method (Bethune et al. 2017, §2).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this library.  It shares
 * no code, header, table or helper with the CUDA path in
 * paper_1708_03604_gb300/csrc; the two meet only through the seeded input
 * generator, which holds none of the method's arithmetic.
 *
 * Everything is FP64, single-threaded, and follows the method's definition
 * in the order the paper states it:
 *   - matrices are block-CSR: row pointers, column-block indices, small dense
 *     blocks of m x k (A) and k x n (B) elements (§2, first paragraph);
 *   - the local product is C = C + A.B computed as pairwise products of
 *     small dense blocks (§2, second paragraph), here generalised to
 *     C = alpha*A.B + beta*C;
 *   - the traversal loops over A's row-blocks and, for each, over the B
 *     blocks reachable from that row (Gustavson's row-by-row SpGEMM, §1.1);
 *   - a block product is skipped unless the two block norms multiplied
 *     together are above the filter threshold (on-the-fly filtering, §2).
 *
 * Readings taken where the paper is silent:
 *   - block norm = Frobenius norm, accumulated as an fma chain x*x + n over
 *     the block's elements in row-major order starting from +0.0, then an
 *     IEEE square root; FP32 data is widened to FP64 first;
 *   - keep a product iff eps <= 0 or nA*nB > eps (strict);
 *   - elements inside a block are row-major; blocks lie at blk_off;
 *   - beta == 0 never reads old C and drops its pattern; beta != 0 merges
 *     the old pattern (union) and scales its values;
 *   - a C block whose products are all filtered does not exist (unless it
 *     is carried by beta != 0);
 *   - the add Z = a*X + b*Y is over the union of patterns; with eps > 0 a
 *     result block is kept iff its norm > eps.
 *
 * Build: gcc -std=c11 -O2 -ffp-contract=off -fPIC -shared -o liboracle.so
 *        bsm_oracle.c -lm
 * (-ffp-contract=off keeps every a*b+c as a separate multiply and add,
 *  except where fma() is written out.)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t nbr, nbc;          /* block rows, block columns                 */
    const int32_t *row_bs;     /* [nbr] rows of each block row              */
    const int32_t *col_bs;     /* [nbc] columns of each block column        */
    const int64_t *row_ptr;    /* [nbr+1]                                    */
    const int32_t *col_idx;    /* [nnzb], ascending within a row             */
    const int64_t *blk_off;    /* [nnzb], element offset of each block       */
    const double *data;        /* element storage, row-major inside a block  */
} or_bcsr;

typedef struct {
    int64_t nnzb;              /* blocks in the result                       */
    int64_t *row_ptr;          /* [nbr+1]                                    */
    int32_t *col_idx;          /* [nnzb]                                     */
    int64_t *blk_off;          /* [nnzb], contiguous in CSR order            */
    double *data;              /* [data_len] (NULL when values not wanted)   */
    int64_t data_len;
    int64_t nprod;             /* kept block products                        */
    int32_t *prod_a;           /* [nprod] A block index of each product      */
    int32_t *prod_b;           /* [nprod] B block index                      */
    int32_t *prod_c;           /* [nprod] C block index                      */
    int64_t nfiltered;         /* candidate products dropped by the filter   */
    double useful_flop;        /* sum of 2*m*n*k over kept products          */
} or_result;

/* ------------------------------------------------------------------ */
/* small growable arrays                                               */
/* ------------------------------------------------------------------ */
typedef struct { void *p; int64_t n, cap; size_t esz; } vec;
static int vec_push(vec *v, const void *e) {
    if (v->n == v->cap) {
        int64_t nc = v->cap ? 2 * v->cap : 1024;
        void *np = realloc(v->p, (size_t)nc * v->esz);
        if (!np) return -1;
        v->p = np; v->cap = nc;
    }
    memcpy((char *)v->p + (size_t)v->n * v->esz, e, v->esz);
    v->n++;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Block norm (filtering criterion of §2): Frobenius norm, fma chain in */
/* row-major order from +0.0, then IEEE sqrt.                           */
/* ------------------------------------------------------------------ */
static double block_norm(const double *x, int64_t len) {
    double s = 0.0;
    for (int64_t e = 0; e < len; ++e) s = fma(x[e], x[e], s);
    return sqrt(s);
}

void or_block_norms(const or_bcsr *X, double *out) {
    for (int32_t i = 0; i < X->nbr; ++i)
        for (int64_t b = X->row_ptr[i]; b < X->row_ptr[i + 1]; ++b) {
            int64_t len = (int64_t)X->row_bs[i] * X->col_bs[X->col_idx[b]];
            out[b] = block_norm(X->data + X->blk_off[b], len);
        }
}

/* ------------------------------------------------------------------ */
/* The local multiply: Gustavson over blocks with on-the-fly filtering. */
/* ------------------------------------------------------------------ */
typedef struct { int32_t a, b, j; } prod_rec;   /* one kept block product */

static int cmp_prod(const void *x, const void *y) {
    const prod_rec *p = (const prod_rec *)x, *q = (const prod_rec *)y;
    if (p->j != q->j) return p->j < q->j ? -1 : 1;     /* C column first  */
    if (p->a != q->a) return p->a < q->a ? -1 : 1;     /* then A block (k) */
    return 0;
}
static int cmp_i32(const void *x, const void *y) {
    int32_t a = *(const int32_t *)x, b = *(const int32_t *)y;
    return (a > b) - (a < b);
}

/*
 * C = alpha * A.B + beta * C_old  (C_old may be NULL when beta == 0).
 *
 *  eps        filter threshold; products with !(nA*nB > eps) are skipped
 *             when eps > 0.
 *  rows       if non-NULL, only these block rows (ascending) are produced;
 *             every other row of the result is empty.
 *  want_values  0: pattern and product list only (no block arithmetic).
 *
 * Products are returned in canonical order: C block row i ascending, then
 * C block column j ascending, then A block (i.e. k) ascending.
 * Returns 0 on success, -1 on allocation failure, -2 on blocking mismatch.
 */
int or_multiply(double alpha, const or_bcsr *A, const or_bcsr *B, double beta,
                const or_bcsr *Cold, double eps, const int32_t *rows, int32_t nrows,
                int want_values, or_result *out) {
    memset(out, 0, sizeof(*out));
    if (A->nbc != B->nbr) return -2;
    for (int32_t k = 0; k < A->nbc; ++k)
        if (A->col_bs[k] != B->row_bs[k]) return -2;
    if (beta != 0.0 && Cold) {
        if (Cold->nbr != A->nbr || Cold->nbc != B->nbc) return -2;
    }
    const int use_old = (beta != 0.0 && Cold != NULL);
    const int32_t nbr = A->nbr, nbc = B->nbc;
    int64_t nnzA = A->row_ptr[nbr], nnzB = B->row_ptr[B->nbr];

    double *nA = malloc(sizeof(double) * (size_t)(nnzA ? nnzA : 1));
    double *nB = malloc(sizeof(double) * (size_t)(nnzB ? nnzB : 1));
    int32_t *mark = malloc(sizeof(int32_t) * (size_t)(nbc ? nbc : 1));
    int32_t *pos = malloc(sizeof(int32_t) * (size_t)(nbc ? nbc : 1));
    double **acc = calloc((size_t)(nbc ? nbc : 1), sizeof(double *));
    int32_t *rowcols = malloc(sizeof(int32_t) * (size_t)(nbc ? nbc : 1));
    out->row_ptr = calloc((size_t)nbr + 1, sizeof(int64_t));
    if (!nA || !nB || !mark || !pos || !acc || !rowcols || !out->row_ptr) goto oom;
    if (eps > 0.0) { or_block_norms(A, nA); or_block_norms(B, nB); }
    for (int32_t j = 0; j < nbc; ++j) mark[j] = -1;

    vec vcol = {0, 0, 0, sizeof(int32_t)}, voff = {0, 0, 0, sizeof(int64_t)};
    vec vdat = {0, 0, 0, sizeof(double)};
    vec vpa = {0, 0, 0, sizeof(int32_t)}, vpb = {0, 0, 0, sizeof(int32_t)},
        vpc = {0, 0, 0, sizeof(int32_t)};
    vec vrow = {0, 0, 0, sizeof(prod_rec)};
    int64_t data_len = 0;
    int32_t next_row = 0;

    for (int32_t i = 0; i < nbr; ++i) {
        int active = 1;
        if (rows) {
            if (next_row < nrows && rows[next_row] == i) next_row++;
            else active = 0;
        }
        out->row_ptr[i] = vcol.n;
        if (!active) continue;
        const int32_t m = A->row_bs[i];
        int32_t ncols = 0;
        vrow.n = 0;
        /* loop over A's blocks of row i (k ascending), then B's row k */
        for (int64_t a = A->row_ptr[i]; a < A->row_ptr[i + 1]; ++a) {
            const int32_t k = A->col_idx[a];
            const int32_t kk = A->col_bs[k];
            for (int64_t b = B->row_ptr[k]; b < B->row_ptr[k + 1]; ++b) {
                const int32_t j = B->col_idx[b];
                if (eps > 0.0 && !(nA[a] * nB[b] > eps)) { out->nfiltered++; continue; }
                const int32_t n = B->col_bs[j];
                if (mark[j] != i) {
                    mark[j] = i;
                    rowcols[ncols++] = j;
                    if (want_values) {
                        acc[j] = calloc((size_t)m * n, sizeof(double));
                        if (!acc[j]) goto oom;
                    }
                }
                prod_rec pr = {(int32_t)a, (int32_t)b, j};
                if (vec_push(&vrow, &pr)) goto oom;
                out->useful_flop += 2.0 * m * n * kk;
                if (want_values) {
                    /* naive block product, FP64: acc += A_ik . B_kj */
                    const double *Ab = A->data + A->blk_off[a];
                    const double *Bb = B->data + B->blk_off[b];
                    double *Cb = acc[j];
                    for (int32_t r = 0; r < m; ++r)
                        for (int32_t c = 0; c < n; ++c) {
                            double s = Cb[(int64_t)r * n + c];
                            for (int32_t t = 0; t < kk; ++t)
                                s = s + Ab[(int64_t)r * kk + t] * Bb[(int64_t)t * n + c];
                            Cb[(int64_t)r * n + c] = s;
                        }
                }
            }
        }
        /* beta != 0: the old row's blocks join the pattern */
        if (use_old) {
            for (int64_t c = Cold->row_ptr[i]; c < Cold->row_ptr[i + 1]; ++c) {
                const int32_t j = Cold->col_idx[c];
                if (mark[j] != i) {
                    mark[j] = i;
                    rowcols[ncols++] = j;
                    if (want_values) {
                        acc[j] = calloc((size_t)m * B->col_bs[j], sizeof(double));
                        if (!acc[j]) goto oom;
                    }
                }
            }
        }
        qsort(rowcols, (size_t)ncols, sizeof(int32_t), cmp_i32);
        for (int32_t q = 0; q < ncols; ++q) {
            const int32_t j = rowcols[q];
            const int32_t n = B->col_bs[j];
            pos[j] = (int32_t)(vcol.n);
            int64_t off = data_len;
            if (vec_push(&vcol, &j) || vec_push(&voff, &off)) goto oom;
            data_len += (int64_t)m * n;
            if (want_values) {
                /* old value of C_ij, if present: locate it in the old row */
                const double *old = NULL;
                if (use_old) {
                    for (int64_t c = Cold->row_ptr[i]; c < Cold->row_ptr[i + 1]; ++c)
                        if (Cold->col_idx[c] == j) { old = Cold->data + Cold->blk_off[c]; break; }
                }
                for (int64_t e = 0; e < (int64_t)m * n; ++e) {
                    double v = alpha * acc[j][e];
                    if (old) v = v + beta * old[e];
                    if (vec_push(&vdat, &v)) goto oom;
                }
                free(acc[j]);
                acc[j] = NULL;
            }
        }
        /* canonical product order inside the row: (j, k) ascending */
        qsort(vrow.p, (size_t)vrow.n, sizeof(prod_rec), cmp_prod);
        for (int64_t p = 0; p < vrow.n; ++p) {
            const prod_rec *pr = (const prod_rec *)vrow.p + p;
            int32_t c = pos[pr->j];
            if (vec_push(&vpa, &pr->a) || vec_push(&vpb, &pr->b) || vec_push(&vpc, &c)) goto oom;
        }
    }
    out->row_ptr[nbr] = vcol.n;
    out->nnzb = vcol.n;
    out->col_idx = vcol.p;
    out->blk_off = voff.p;
    out->data = want_values ? (double *)vdat.p : NULL;
    if (!want_values) free(vdat.p);
    out->data_len = data_len;
    out->nprod = vpa.n;
    out->prod_a = vpa.p;
    out->prod_b = vpb.p;
    out->prod_c = vpc.p;
    free(vrow.p);
    free(nA); free(nB); free(mark); free(pos); free(acc); free(rowcols);
    return 0;
oom:
    free(nA); free(nB); free(mark); free(pos); free(rowcols);
    if (acc) { for (int32_t j = 0; j < nbc; ++j) free(acc[j]); free(acc); }
    return -1;
}

void or_result_free(or_result *r) {
    free(r->row_ptr); free(r->col_idx); free(r->blk_off); free(r->data);
    free(r->prod_a); free(r->prod_b); free(r->prod_c);
    memset(r, 0, sizeof(*r));
}

/* ------------------------------------------------------------------ */
/* Adjoint of C = alpha*A.B at fixed keep-decisions.                    */
/*   dA_ik += alpha * dC_ij . B_kj^T   for every kept product (i,k,j)   */
/*   dB_kj += alpha * A_ik^T . dC_ij                                     */
/* dA has A's layout, dB has B's layout; both are overwritten.          */
/* Either may be NULL.  dC is laid out with C's blk_off.                 */
/* ------------------------------------------------------------------ */
int or_multiply_backward(double alpha, const or_bcsr *A, const or_bcsr *B,
                          const int64_t *c_blk_off, const double *dC,
                          int64_t nprod, const int32_t *prod_a, const int32_t *prod_b,
                          const int32_t *prod_c,
                          double *dA, int64_t dA_len, double *dB, int64_t dB_len) {
    if (dA) memset(dA, 0, sizeof(double) * (size_t)dA_len);
    if (dB) memset(dB, 0, sizeof(double) * (size_t)dB_len);
    /* block row of every A block, for its row count m */
    int64_t nnzA = A->row_ptr[A->nbr];
    int32_t *arow = malloc(sizeof(int32_t) * (size_t)(nnzA ? nnzA : 1));
    if (!arow) return -1;
    for (int32_t i = 0; i < A->nbr; ++i)
        for (int64_t a = A->row_ptr[i]; a < A->row_ptr[i + 1]; ++a) arow[a] = i;
    for (int64_t p = 0; p < nprod; ++p) {
        const int32_t a = prod_a[p], b = prod_b[p], c = prod_c[p], i = arow[a];
        const int32_t k = A->col_idx[a];
        const int32_t j = B->col_idx[b];
        const int32_t m = A->row_bs[i], kk = A->col_bs[k], n = B->col_bs[j];
        const double *Ab = A->data + A->blk_off[a];
        const double *Bb = B->data + B->blk_off[b];
        const double *G = dC + c_blk_off[c];
        if (dA) {
            double *gA = dA + A->blk_off[a];
            for (int32_t r = 0; r < m; ++r)
                for (int32_t t = 0; t < kk; ++t) {
                    double s = 0.0;
                    for (int32_t q = 0; q < n; ++q)
                        s = s + G[(int64_t)r * n + q] * Bb[(int64_t)t * n + q];
                    gA[(int64_t)r * kk + t] = gA[(int64_t)r * kk + t] + alpha * s;
                }
        }
        if (dB) {
            double *gB = dB + B->blk_off[b];
            for (int32_t t = 0; t < kk; ++t)
                for (int32_t q = 0; q < n; ++q) {
                    double s = 0.0;
                    for (int32_t r = 0; r < m; ++r)
                        s = s + Ab[(int64_t)r * kk + t] * G[(int64_t)r * n + q];
                    gB[(int64_t)t * n + q] = gB[(int64_t)t * n + q] + alpha * s;
                }
        }
    }
    free(arow);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Z = a*X + b*Y over the union of the two patterns; with eps > 0 a      */
/* result block survives iff its Frobenius norm > eps.                  */
/* ------------------------------------------------------------------ */
int or_add(double a, const or_bcsr *X, double b, const or_bcsr *Y, double eps, or_result *out) {
    memset(out, 0, sizeof(*out));
    if (X->nbr != Y->nbr || X->nbc != Y->nbc) return -2;
    for (int32_t i = 0; i < X->nbr; ++i) if (X->row_bs[i] != Y->row_bs[i]) return -2;
    for (int32_t j = 0; j < X->nbc; ++j) if (X->col_bs[j] != Y->col_bs[j]) return -2;
    const int32_t nbr = X->nbr;
    out->row_ptr = calloc((size_t)nbr + 1, sizeof(int64_t));
    if (!out->row_ptr) return -1;
    vec vcol = {0, 0, 0, sizeof(int32_t)}, voff = {0, 0, 0, sizeof(int64_t)};
    vec vdat = {0, 0, 0, sizeof(double)};
    double *tmp = NULL;
    int64_t data_len = 0;
    for (int32_t i = 0; i < nbr; ++i) {
        out->row_ptr[i] = vcol.n;
        int64_t px = X->row_ptr[i], py = Y->row_ptr[i];
        const int64_t ex = X->row_ptr[i + 1], ey = Y->row_ptr[i + 1];
        while (px < ex || py < ey) {
            int32_t jx = px < ex ? X->col_idx[px] : INT32_MAX;
            int32_t jy = py < ey ? Y->col_idx[py] : INT32_MAX;
            int32_t j = jx < jy ? jx : jy;
            const int64_t len = (int64_t)X->row_bs[i] * X->col_bs[j];
            double *t2 = realloc(tmp, sizeof(double) * (size_t)len);
            if (!t2) { free(tmp); return -1; }
            tmp = t2;
            const double *xv = (jx == j) ? X->data + X->blk_off[px] : NULL;
            const double *yv = (jy == j) ? Y->data + Y->blk_off[py] : NULL;
            for (int64_t e = 0; e < len; ++e) {
                double v = 0.0;
                if (xv) v = a * xv[e];
                if (yv) v = xv ? v + b * yv[e] : b * yv[e];
                tmp[e] = v;
            }
            if (jx == j) px++;
            if (jy == j) py++;
            if (eps > 0.0 && !(block_norm(tmp, len) > eps)) continue;
            int64_t off = data_len;
            if (vec_push(&vcol, &j) || vec_push(&voff, &off)) { free(tmp); return -1; }
            for (int64_t e = 0; e < len; ++e)
                if (vec_push(&vdat, &tmp[e])) { free(tmp); return -1; }
            data_len += len;
        }
    }
    free(tmp);
    out->row_ptr[nbr] = vcol.n;
    out->nnzb = vcol.n;
    out->col_idx = vcol.p;
    out->blk_off = voff.p;
    out->data = vdat.p;
    out->data_len = data_len;
    return 0;
}
