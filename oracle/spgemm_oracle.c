/*
 * CPU oracle for sparse matrix-matrix multiplication C = A*B on CSR.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the library's product path links, loads
 * or calls this file; only the test suite, the package's smoke check and the
 * benchmark's CPU-baseline leg do. It shares no code, header or table with the
 * CUDA implementation.
 *
 * What it computes is the plain definition of the product:
 *   c_ij = sum_k a_ik * b_kj                       (Eq. inner_product)
 * evaluated row by row as
 *   C[i,:] = sum_{k in A_i} A[i,k] * B[k,:]         (Eq. row_wise)
 * with a dense sparse accumulator (SPA): one accumulator slot per column of B,
 * a stamp that says whether column j was touched by the current row, and the
 * list of touched columns, which is sorted ascending when the row is emitted.
 *
 * The structure of C is the set of (i, j) reached by at least one product; a
 * value that cancels to zero stays a stored entry. Duplicate column indices in
 * A or B are separate terms of the sum.
 *
 * Floating point: every product a*b is formed exactly as a double-double
 * (p, e) with e = fma(a, b, -p), and the row sums are accumulated in
 * double-double (Knuth's TwoSum). The emitted value hi+lo is the exact sum to
 * within about 2^-100 * s_ij, where s_ij = sum_k |a_ik||b_kj| is emitted beside
 * it as the scale for tolerance checks. float32 inputs are widened to double
 * (exactly) by the caller. An int64 variant accumulates integer-valued inputs
 * exactly.
 *
 * The row flop count (number of products of row i, Gustavson's first pass,
 * "Window Distribution Phase") is here too:
 *   flop_i = sum_{k in A_i} |B_k|.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

void oracle_row_flops(int64_t m, const int64_t *a_rp, const int32_t *a_ci, const int64_t *b_rp,
                      int64_t *flop) {
    for (int64_t i = 0; i < m; ++i) {
        int64_t f = 0;
        for (int64_t e = a_rp[i]; e < a_rp[i + 1]; ++e) {
            int64_t k = a_ci[e];
            f += b_rp[k + 1] - b_rp[k];
        }
        flop[i] = f;
    }
}

static int cmp_i32(const void *x, const void *y) {
    int32_t a = *(const int32_t *)x, b = *(const int32_t *)y;
    return (a > b) - (a < b);
}

/* Selected rows: sel == NULL means rows 0..nsel-1. */
static inline int64_t row_of(const int64_t *sel, int64_t r) { return sel ? sel[r] : r; }

/*
 * Pass 1: number of distinct columns of each selected row of C.
 * Returns the total, or -1 if memory could not be obtained.
 */
int64_t oracle_count(int64_t nsel, const int64_t *sel, int64_t ncols_b, const int64_t *a_rp,
                     const int32_t *a_ci, const int64_t *b_rp, const int32_t *b_ci,
                     int64_t *out_nnz) {
    int64_t *stamp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ncols_b > 0 ? ncols_b : 1));
    if (!stamp) return -1;
    for (int64_t j = 0; j < ncols_b; ++j) stamp[j] = -1;
    int64_t total = 0;
    for (int64_t r = 0; r < nsel; ++r) {
        int64_t i = row_of(sel, r);
        int64_t cnt = 0;
        for (int64_t e = a_rp[i]; e < a_rp[i + 1]; ++e) {
            int64_t k = a_ci[e];
            for (int64_t f = b_rp[k]; f < b_rp[k + 1]; ++f) {
                int32_t j = b_ci[f];
                if (stamp[j] != r) {
                    stamp[j] = r;
                    ++cnt;
                }
            }
        }
        out_nnz[r] = cnt;
        total += cnt;
    }
    free(stamp);
    return total;
}

/* Knuth TwoSum: s + err == a + b exactly. */
static inline void two_sum(double a, double b, double *s, double *err) {
    double t = a + b;
    double bb = t - a;
    *err = (a - (t - bb)) + (b - bb);
    *s = t;
}

/*
 * Pass 2 (floating point): fills the selected rows of C given out_rp, the
 * prefix sum of pass 1's counts over the selected rows (out_rp[0] = 0).
 * out_val = exact sum rounded to double; out_abs = sum of |a||b|.
 * Returns 0, or -1 if memory could not be obtained.
 */
int oracle_fill_f64(int64_t nsel, const int64_t *sel, int64_t ncols_b, const int64_t *a_rp,
                    const int32_t *a_ci, const double *a_val, const int64_t *b_rp,
                    const int32_t *b_ci, const double *b_val, const int64_t *out_rp,
                    int32_t *out_ci, double *out_val, double *out_abs) {
    size_t nc = (size_t)(ncols_b > 0 ? ncols_b : 1);
    int64_t *stamp = (int64_t *)malloc(sizeof(int64_t) * nc);
    double *hi = (double *)malloc(sizeof(double) * nc);
    double *lo = (double *)malloc(sizeof(double) * nc);
    double *ab = (double *)malloc(sizeof(double) * nc);
    if (!stamp || !hi || !lo || !ab) {
        free(stamp); free(hi); free(lo); free(ab);
        return -1;
    }
    for (size_t j = 0; j < nc; ++j) stamp[j] = -1;
    for (int64_t r = 0; r < nsel; ++r) {
        int64_t i = row_of(sel, r);
        int32_t *touched = out_ci + out_rp[r];
        int64_t cnt = 0;
        for (int64_t e = a_rp[i]; e < a_rp[i + 1]; ++e) {
            int64_t k = a_ci[e];
            double a = a_val[e];
            for (int64_t f = b_rp[k]; f < b_rp[k + 1]; ++f) {
                int32_t j = b_ci[f];
                double b = b_val[f];
                double p = a * b;
                double pe = fma(a, b, -p);
                if (stamp[j] != r) {
                    stamp[j] = r;
                    touched[cnt++] = j;
                    hi[j] = 0.0;
                    lo[j] = 0.0;
                    ab[j] = 0.0;
                }
                double s, err;
                two_sum(hi[j], p, &s, &err);
                hi[j] = s;
                lo[j] += err + pe;
                ab[j] += fabs(a) * fabs(b);
            }
        }
        qsort(touched, (size_t)cnt, sizeof(int32_t), cmp_i32);
        for (int64_t t = 0; t < cnt; ++t) {
            int32_t j = touched[t];
            out_val[out_rp[r] + t] = hi[j] + lo[j];
            out_abs[out_rp[r] + t] = ab[j];
        }
    }
    free(stamp); free(hi); free(lo); free(ab);
    return 0;
}

/* Pass 2 (integers): exact int64 products and sums. */
int oracle_fill_i64(int64_t nsel, const int64_t *sel, int64_t ncols_b, const int64_t *a_rp,
                    const int32_t *a_ci, const int64_t *a_val, const int64_t *b_rp,
                    const int32_t *b_ci, const int64_t *b_val, const int64_t *out_rp,
                    int32_t *out_ci, int64_t *out_val) {
    size_t nc = (size_t)(ncols_b > 0 ? ncols_b : 1);
    int64_t *stamp = (int64_t *)malloc(sizeof(int64_t) * nc);
    int64_t *acc = (int64_t *)malloc(sizeof(int64_t) * nc);
    if (!stamp || !acc) {
        free(stamp); free(acc);
        return -1;
    }
    for (size_t j = 0; j < nc; ++j) stamp[j] = -1;
    for (int64_t r = 0; r < nsel; ++r) {
        int64_t i = row_of(sel, r);
        int32_t *touched = out_ci + out_rp[r];
        int64_t cnt = 0;
        for (int64_t e = a_rp[i]; e < a_rp[i + 1]; ++e) {
            int64_t k = a_ci[e];
            for (int64_t f = b_rp[k]; f < b_rp[k + 1]; ++f) {
                int32_t j = b_ci[f];
                if (stamp[j] != r) {
                    stamp[j] = r;
                    touched[cnt++] = j;
                    acc[j] = 0;
                }
                acc[j] += a_val[e] * b_val[f];
            }
        }
        qsort(touched, (size_t)cnt, sizeof(int32_t), cmp_i32);
        for (int64_t t = 0; t < cnt; ++t) out_val[out_rp[r] + t] = acc[touched[t]];
    }
    free(stamp); free(acc);
    return 0;
}
