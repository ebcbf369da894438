/*
 * oracle.c -- plain, slow, obviously correct CPU reference for C = A*B.
 *
 * TEST INFRASTRUCTURE ONLY.  The test suite, the package smoke check and the
 * benchmark's CPU-baseline leg are the only users of this library.  The GPU
 * product path never calls into it, includes none of its declarations and
 * shares no source with it.
 *
 * Every routine writes out a quantity from its plain definition in
 * Deveci, Trott, Rajamanickam, "Multi-threaded Sparse Matrix-Matrix
 * Multiplication for Many-Core and GPU Architectures":
 *
 *   oracle_row_flops ............ f_m, the multiplication count of Gustavson's
 *                                 algorithm (Section 2, after Algorithm 1), and
 *                                 maxrf, the largest per-row count (Section 3.1.2,
 *                                 memory pool paragraph)
 *   oracle_compress_* ........... column-set compression of B: CSI = col >> 5,
 *                                 CS = OR of (1 << (col & 31)) (Section 3.2)
 *   oracle_symbolic_plain ....... |C(i,:)| by its definition, the number of
 *                                 distinct l with A(i,j) != 0 and B(j,l) != 0
 *                                 (Algorithm 2, symbolic phase)
 *   oracle_symbolic_compressed .. |C(i,:)| the way the symbolic phase computes it
 *                                 on the compressed B: OR-union of column sets,
 *                                 then the number of set bits (Section 3.2,
 *                                 Algorithm 3)
 *   oracle_numeric .............. C(i,:) = sum_j A(i,j) * B(j,:) (Algorithm 1),
 *                                 as a gather of all products of the row, a
 *                                 stable sort by column, and an in-order sum
 *   oracle_transpose ............ counting transpose with its value permutation
 *   oracle_masked_count ......... row sums of (X*Y) on a pattern S over the
 *                                 counting semiring (symbolic-only graph use,
 *                                 Section 2): triangle counts when X = Y = S = L
 *   oracle_masked_dA / _dB ...... gradients of a loss sum(W o (A*B)) on fixed
 *                                 patterns, by their definition:
 *                                 dA(i,j) = sum_l G(i,l) B(j,l) on A's pattern,
 *                                 dB(j,l) = sum_i A(i,j) G(i,l) on B's pattern
 *
 * Conventions: rowptr int64[nrows+1], colidx int32[nnz] (any order within a
 * row unless stated), values double.  Output rows of C are sorted by column.
 * Parallelism: OpenMP over rows; every row's arithmetic runs in the order
 * stated above and does not depend on the thread count.
 * Return value: 0 on success, -1 when a scratch allocation fails,
 * -2 for an invalid argument.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#ifdef _OPENMP
#include <omp.h>
#endif

static int oracle_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static int oracle_tid(void) {
#ifdef _OPENMP
    return omp_get_thread_num();
#else
    return 0;
#endif
}

int oracle_num_threads(void) { return oracle_threads(); }

/* ------------------------------------------------------------------------ */
/* f_m: number of multiplications; rf[i] = sum_{j in A(i,:)} |B(j,:)|.        */
/* ------------------------------------------------------------------------ */
int oracle_row_flops(int64_t m, const int64_t *Ap, const int32_t *Aj,
                     const int64_t *Bp, int64_t *rf, int64_t *f_m, int64_t *maxrf) {
    int64_t total = 0, mx = 0;
    #pragma omp parallel for schedule(dynamic, 1024) reduction(+:total) reduction(max:mx)
    for (int64_t i = 0; i < m; ++i) {
        int64_t s = 0;
        for (int64_t p = Ap[i]; p < Ap[i + 1]; ++p) {
            int64_t j = Aj[p];
            s += Bp[j + 1] - Bp[j];
        }
        if (rf) rf[i] = s;
        total += s;
        if (s > mx) mx = s;
    }
    *f_m = total;
    *maxrf = mx;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Compression (Section 3.2).  Row j of B becomes the set of distinct column  */
/* set indices CSI = col >> 5, each with CS = OR over its columns of          */
/* 1 << (col & 31).  Rows are emitted with CSI ascending.                     */
/* ------------------------------------------------------------------------ */
static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

int oracle_compress_count(int64_t n, const int64_t *Bp, const int32_t *Bj, int64_t *cnt) {
    int64_t maxlen = 0;
    for (int64_t j = 0; j < n; ++j) {
        int64_t l = Bp[j + 1] - Bp[j];
        if (l > maxlen) maxlen = l;
    }
    int nt = oracle_threads();
    int32_t *buf = (int32_t *)malloc((size_t)(maxlen > 0 ? maxlen : 1) * sizeof(int32_t) * nt);
    if (!buf) return -1;
    #pragma omp parallel for schedule(dynamic, 256)
    for (int64_t j = 0; j < n; ++j) {
        int32_t *b = buf + (size_t)oracle_tid() * (size_t)(maxlen > 0 ? maxlen : 1);
        int64_t len = Bp[j + 1] - Bp[j];
        for (int64_t q = 0; q < len; ++q) b[q] = Bj[Bp[j] + q] >> 5;
        qsort(b, (size_t)len, sizeof(int32_t), cmp_i32);
        int64_t c = 0;
        for (int64_t q = 0; q < len; ++q)
            if (q == 0 || b[q] != b[q - 1]) ++c;
        cnt[j] = c;
    }
    free(buf);
    return 0;
}

int oracle_compress_fill(int64_t n, const int64_t *Bp, const int32_t *Bj,
                         const int64_t *Bcp, int32_t *csi, uint32_t *cs) {
    int64_t maxlen = 0;
    for (int64_t j = 0; j < n; ++j) {
        int64_t l = Bp[j + 1] - Bp[j];
        if (l > maxlen) maxlen = l;
    }
    int nt = oracle_threads();
    size_t stride = (size_t)(maxlen > 0 ? maxlen : 1);
    int32_t *buf = (int32_t *)malloc(stride * sizeof(int32_t) * nt);
    if (!buf) return -1;
    #pragma omp parallel for schedule(dynamic, 256)
    for (int64_t j = 0; j < n; ++j) {
        int32_t *b = buf + (size_t)oracle_tid() * stride;
        int64_t len = Bp[j + 1] - Bp[j];
        for (int64_t q = 0; q < len; ++q) b[q] = Bj[Bp[j] + q];
        qsort(b, (size_t)len, sizeof(int32_t), cmp_i32);
        int64_t o = Bcp[j] - 1;
        for (int64_t q = 0; q < len; ++q) {
            int32_t set = b[q] >> 5;
            uint32_t bit = 1u << (b[q] & 31);
            if (q == 0 || set != (b[q - 1] >> 5)) {
                ++o;
                csi[o] = set;
                cs[o] = 0u;
            }
            cs[o] |= bit;
        }
    }
    free(buf);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Symbolic, plain definition: rowsize[i] = |{ l : exists j, A(i,j), B(j,l) }| */
/* ------------------------------------------------------------------------ */
int oracle_symbolic_plain(int64_t m, int64_t k, const int64_t *Ap, const int32_t *Aj,
                          const int64_t *Bp, const int32_t *Bj, int64_t *rowsize) {
    int nt = oracle_threads();
    int64_t *mark = (int64_t *)malloc((size_t)(k > 0 ? k : 1) * sizeof(int64_t) * nt);
    if (!mark) return -1;
    for (size_t q = 0; q < (size_t)(k > 0 ? k : 1) * nt; ++q) mark[q] = -1;
    #pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < m; ++i) {
        int64_t *mk = mark + (size_t)oracle_tid() * (size_t)(k > 0 ? k : 1);
        int64_t c = 0;
        for (int64_t p = Ap[i]; p < Ap[i + 1]; ++p) {
            int64_t j = Aj[p];
            for (int64_t q = Bp[j]; q < Bp[j + 1]; ++q) {
                int64_t l = Bj[q];
                if (mk[l] != i) { mk[l] = i; ++c; }
            }
        }
        rowsize[i] = c;
    }
    free(mark);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Symbolic on the compressed B: OR the column sets of every B_c(j,:) with    */
/* j in A(i,:) per CSI, then count the set bits of the union.                */
/* ------------------------------------------------------------------------ */
static int popcount32(uint32_t x) {
    int c = 0;
    while (x) { x &= x - 1u; ++c; }
    return c;
}

int oracle_symbolic_compressed(int64_t m, int64_t kc, const int64_t *Ap, const int32_t *Aj,
                               const int64_t *Bcp, const int32_t *csi, const uint32_t *cs,
                               int64_t *rowsize, int64_t *rowflops_c) {
    int nt = oracle_threads();
    size_t stride = (size_t)(kc > 0 ? kc : 1);
    uint32_t *acc = (uint32_t *)calloc(stride * nt, sizeof(uint32_t));
    int64_t *touched = (int64_t *)malloc(stride * sizeof(int64_t) * nt);
    if (!acc || !touched) { free(acc); free(touched); return -1; }
    #pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < m; ++i) {
        uint32_t *a = acc + (size_t)oracle_tid() * stride;
        int64_t *t = touched + (size_t)oracle_tid() * stride;
        int64_t nt_ = 0, flops = 0;
        for (int64_t p = Ap[i]; p < Ap[i + 1]; ++p) {
            int64_t j = Aj[p];
            flops += Bcp[j + 1] - Bcp[j];
            for (int64_t q = Bcp[j]; q < Bcp[j + 1]; ++q) {
                int64_t s = csi[q];
                if (a[s] == 0u) t[nt_++] = s;
                a[s] |= cs[q];
            }
        }
        int64_t c = 0;
        for (int64_t q = 0; q < nt_; ++q) { c += popcount32(a[t[q]]); a[t[q]] = 0u; }
        rowsize[i] = c;
        if (rowflops_c) rowflops_c[i] = flops;
    }
    free(acc);
    free(touched);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Numeric (Algorithm 1): gather every product of row i in A's row order and  */
/* B's row order, stable-sort by column, then sum equal columns in gather     */
/* order.  S[q] = sum |A(i,j)|*|B(j,l)| for the same entry (error scale).      */
/* Cp must already hold the row pointers of C (from the symbolic routines).   */
/* ------------------------------------------------------------------------ */
typedef struct { int32_t col; int64_t seq; double v; double a; } prod_t;

static int cmp_prod(const void *x, const void *y) {
    const prod_t *p = (const prod_t *)x, *q = (const prod_t *)y;
    if (p->col != q->col) return (p->col > q->col) - (p->col < q->col);
    return (p->seq > q->seq) - (p->seq < q->seq);
}

int oracle_numeric(int64_t m, const int64_t *Ap, const int32_t *Aj, const double *Ax,
                   const int64_t *Bp, const int32_t *Bj, const double *Bx,
                   const int64_t *Cp, int32_t *Cj, double *Cx, double *S) {
    int64_t f_m = 0, maxrf = 0;
    oracle_row_flops(m, Ap, Aj, Bp, NULL, &f_m, &maxrf);
    int nt = oracle_threads();
    size_t stride = (size_t)(maxrf > 0 ? maxrf : 1);
    prod_t *buf = (prod_t *)malloc(stride * sizeof(prod_t) * nt);
    if (!buf) return -1;
    int bad = 0;
    #pragma omp parallel for schedule(dynamic, 64) reduction(|:bad)
    for (int64_t i = 0; i < m; ++i) {
        prod_t *b = buf + (size_t)oracle_tid() * stride;
        int64_t n = 0;
        for (int64_t p = Ap[i]; p < Ap[i + 1]; ++p) {
            int64_t j = Aj[p];
            double a = Ax ? Ax[p] : 1.0;
            for (int64_t q = Bp[j]; q < Bp[j + 1]; ++q) {
                double bv = Bx ? Bx[q] : 1.0;
                b[n].col = Bj[q];
                b[n].seq = n;
                b[n].v = a * bv;
                b[n].a = fabs(a) * fabs(bv);
                ++n;
            }
        }
        qsort(b, (size_t)n, sizeof(prod_t), cmp_prod);
        int64_t o = Cp[i] - 1;
        for (int64_t q = 0; q < n; ++q) {
            if (q == 0 || b[q].col != b[q - 1].col) {
                ++o;
                if (o >= Cp[i + 1]) { bad = 1; break; }
                Cj[o] = b[q].col;
                Cx[o] = 0.0;
                if (S) S[o] = 0.0;
            }
            Cx[o] += b[q].v;
            if (S) S[o] += b[q].a;
        }
        if (o != Cp[i + 1] - 1) bad = 1;
    }
    free(buf);
    return bad ? -2 : 0;
}

/* ------------------------------------------------------------------------ */
/* Counting transpose.  Row c of At lists the rows i with A(i,c) != 0 in      */
/* ascending i; perm[q] is the position in A of entry q of At.               */
/* ------------------------------------------------------------------------ */
int oracle_transpose(int64_t m, int64_t n, const int64_t *Ap, const int32_t *Aj,
                     const double *Ax, int64_t *Atp, int32_t *Atj, double *Atx, int64_t *perm) {
    int64_t nnz = Ap[m];
    int64_t *cur = (int64_t *)calloc((size_t)(n + 1), sizeof(int64_t));
    if (!cur) return -1;
    for (int64_t q = 0; q <= n; ++q) Atp[q] = 0;
    for (int64_t q = 0; q < nnz; ++q) Atp[Aj[q] + 1] += 1;
    for (int64_t c = 0; c < n; ++c) Atp[c + 1] += Atp[c];
    for (int64_t c = 0; c < n; ++c) cur[c] = Atp[c];
    for (int64_t i = 0; i < m; ++i)
        for (int64_t p = Ap[i]; p < Ap[i + 1]; ++p) {
            int64_t c = Aj[p];
            int64_t o = cur[c]++;
            Atj[o] = (int32_t)i;
            if (Atx) Atx[o] = Ax[p];
            if (perm) perm[o] = p;
        }
    free(cur);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* dA(i,j) = sum_l G(i,l) * B(j,l) over l in both G(i,:) and B(j,:), for     */
/* every stored (i,j) of A.  S = the same sum of absolute products.           */
/* ------------------------------------------------------------------------ */
int oracle_masked_dA(int64_t m, int64_t k, const int64_t *Ap, const int32_t *Aj,
                     const int64_t *Gp, const int32_t *Gj, const double *Gx,
                     const int64_t *Bp, const int32_t *Bj, const double *Bx,
                     double *dA, double *S) {
    int nt = oracle_threads();
    size_t stride = (size_t)(k > 0 ? k : 1);
    double *g = (double *)calloc(stride * nt, sizeof(double));
    int64_t *mk = (int64_t *)malloc(stride * sizeof(int64_t) * nt);
    if (!g || !mk) { free(g); free(mk); return -1; }
    for (size_t q = 0; q < stride * nt; ++q) mk[q] = -1;
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < m; ++i) {
        double *gg = g + (size_t)oracle_tid() * stride;
        int64_t *mm = mk + (size_t)oracle_tid() * stride;
        for (int64_t q = Gp[i]; q < Gp[i + 1]; ++q) { gg[Gj[q]] = Gx[q]; mm[Gj[q]] = i; }
        for (int64_t p = Ap[i]; p < Ap[i + 1]; ++p) {
            int64_t j = Aj[p];
            double s = 0.0, sa = 0.0;
            for (int64_t q = Bp[j]; q < Bp[j + 1]; ++q) {
                int64_t l = Bj[q];
                if (mm[l] == i) { s += gg[l] * Bx[q]; sa += fabs(gg[l]) * fabs(Bx[q]); }
            }
            dA[p] = s;
            if (S) S[p] = sa;
        }
    }
    free(g);
    free(mk);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* dB(j,l) = sum_i A(i,j) * G(i,l) over i with A(i,j) and G(i,l) stored, for  */
/* every stored (j,l) of B.  Runs over the columns of A via its transpose.    */
/* ------------------------------------------------------------------------ */
int oracle_masked_dB(int64_t m, int64_t n, int64_t k, const int64_t *Ap, const int32_t *Aj,
                     const double *Ax, const int64_t *Gp, const int32_t *Gj, const double *Gx,
                     const int64_t *Bp, const int32_t *Bj, double *dB, double *S) {
    int64_t nnzA = Ap[m];
    int64_t *Atp = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
    int32_t *Atj = (int32_t *)malloc((size_t)(nnzA > 0 ? nnzA : 1) * sizeof(int32_t));
    double *Atx = (double *)malloc((size_t)(nnzA > 0 ? nnzA : 1) * sizeof(double));
    int nt = oracle_threads();
    size_t stride = (size_t)(k > 0 ? k : 1);
    double *acc = (double *)calloc(stride * nt, sizeof(double));
    double *acca = (double *)calloc(stride * nt, sizeof(double));
    if (!Atp || !Atj || !Atx || !acc || !acca) {
        free(Atp); free(Atj); free(Atx); free(acc); free(acca);
        return -1;
    }
    oracle_transpose(m, n, Ap, Aj, Ax, Atp, Atj, Atx, NULL);
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t j = 0; j < n; ++j) {
        double *ac = acc + (size_t)oracle_tid() * stride;
        double *aa = acca + (size_t)oracle_tid() * stride;
        for (int64_t p = Atp[j]; p < Atp[j + 1]; ++p) {
            int64_t i = Atj[p];
            double a = Atx[p];
            for (int64_t q = Gp[i]; q < Gp[i + 1]; ++q) {
                ac[Gj[q]] += a * Gx[q];
                aa[Gj[q]] += fabs(a) * fabs(Gx[q]);
            }
        }
        for (int64_t q = Bp[j]; q < Bp[j + 1]; ++q) {
            dB[q] = ac[Bj[q]];
            if (S) S[q] = aa[Bj[q]];
        }
        for (int64_t p = Atp[j]; p < Atp[j + 1]; ++p) {
            int64_t i = Atj[p];
            for (int64_t q = Gp[i]; q < Gp[i + 1]; ++q) { ac[Gj[q]] = 0.0; aa[Gj[q]] = 0.0; }
        }
    }
    free(Atp); free(Atj); free(Atx); free(acc); free(acca);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* counts[i] = sum over l in S(i,:) of |{ j : (i,j) in X and (j,l) in Y }|:  */
/* the row sums of (X*Y) sampled on S over the counting semiring (the        */
/* symbolic-only product of graph analytics, Section 2), by definition: mark  */
/* S(i,:), then walk every product of row i and count those that land on a   */
/* mark.  Values are not read.                                               */
/* ------------------------------------------------------------------------ */
int oracle_masked_count(int64_t m, int64_t k, const int64_t *Xp, const int32_t *Xj, const int64_t *Yp,
                        const int32_t *Yj, const int64_t *Sp, const int32_t *Sj, int64_t *counts) {
    int nt = oracle_threads();
    size_t stride = (size_t)(k > 0 ? k : 1);
    int64_t *mark = (int64_t *)malloc(stride * nt * sizeof(int64_t));
    if (!mark) return -1;
    for (size_t x = 0; x < stride * nt; ++x) mark[x] = -1;
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < m; ++i) {
        int64_t *mk = mark + (size_t)oracle_tid() * stride;
        for (int64_t p = Sp[i]; p < Sp[i + 1]; ++p) mk[Sj[p]] = i;
        int64_t c = 0;
        for (int64_t p = Xp[i]; p < Xp[i + 1]; ++p) {
            int64_t j = Xj[p];
            for (int64_t q = Yp[j]; q < Yp[j + 1]; ++q)
                if (mk[Yj[q]] == i) ++c;
        }
        counts[i] = c;
    }
    free(mark);
    return 0;
}
