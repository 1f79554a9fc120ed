/*
 * A-CholQR2 restated on the CPU, for the benchmark's timed CPU baseline of
 * the method itself (not the oracle of the result: that is CHOL-EQR,
 * orc_oblique_qr in oqr_oracle.c).
 *
 * TEST AND BASELINE INFRASTRUCTURE ONLY, like the rest of this directory: the
 * CUDA library never loads it.  It shares no code with the CUDA library.
 *
 * Each pass is Algorithm 1 (CHOLQR, Sec. 2) as written, with loops ordered so
 * that a multicore CPU streams A once per pass:
 *   W = A X      rows of W split into blocks of RB rows, one block per thread
 *                at a time; for every KB columns of A the block's RB x KB
 *                entries of A update the block's RB x n slice of W (kept in
 *                cache);
 *   C = X^T W    one thread per column of C;
 *   R_p = chol(C)             (orc_chol_upper, the oracle's definition)
 *   Q = X / R_p               (orc_trsm_right_upper, row by row)
 * and A-CholQR2 is two passes with R = R_2 R_1 (orc_upper_times_upper).
 * A is read in full (both triangles, symmetric); X = Z in the first pass and
 * Q_1 in the second.  Column-major storage as everywhere in this directory.
 */
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define AT(X, i, j, ld) (X)[(size_t)(i) + (size_t)(j) * (size_t)(ld)]
#define RB 64
#define KB 8

int orc_chol_upper(int n, const double *A, long lda, double *C, long ldc);
void orc_trsm_right_upper(int m, int n, const double *Z, long ldz,
                          const double *R, long ldr, double *Q, long ldq);
void orc_upper_times_upper(int n, const double *U, long ldu, const double *S,
                           long lds, double *R, long ldr);

/* W = A X (A m x m symmetric, read in full; X m x n; W m x n with ld m).
 * Columns of A are taken KB at a time, so that each pass over the block's
 * slice of W adds KB products (fewer trips through the cache for W). */
static void cpu_symm_rowblock(int m, int n, const double *A, long lda,
                              const double *X, long ldx, double *W)
{
    const long nblk = (m + RB - 1) / RB;
#pragma omp parallel for schedule(dynamic, 1)
    for (long b = 0; b < nblk; ++b) {
        const long i0 = b * RB, rows = (i0 + RB <= m) ? RB : m - i0;
        for (long c = 0; c < n; ++c)
            memset(&AT(W, i0, c, m), 0, sizeof(double) * (size_t)rows);
        long k = 0;
        for (; k + KB <= m; k += KB) {
            const double *a = &AT(A, i0, k, lda);
            for (long c = 0; c < n; ++c) {
                const double *x = &AT(X, k, c, ldx);
                double *w = &AT(W, i0, c, m);
                for (long i = 0; i < rows; ++i) {
                    double t = 0.0;
                    for (long kk = 0; kk < KB; ++kk)
                        t += a[i + kk * lda] * x[kk];
                    w[i] += t;
                }
            }
        }
        for (; k < m; ++k) {
            const double *a = &AT(A, i0, k, lda);
            for (long c = 0; c < n; ++c) {
                const double x = AT(X, k, c, ldx);
                double *w = &AT(W, i0, c, m);
                for (long i = 0; i < rows; ++i)
                    w[i] += a[i] * x;
            }
        }
    }
}

/* C = X^T W (n x n, ld n). */
static void cpu_cross(int m, int n, const double *X, long ldx, const double *W,
                      double *C)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (long c = 0; c < n; ++c)
        for (long r = 0; r < n; ++r) {
            double s = 0.0;
            for (long i = 0; i < m; ++i)
                s += AT(X, i, r, ldx) * AT(W, i, c, m);
            AT(C, r, c, n) = s;
        }
}

/* One CHOLQR pass: Q = X / chol(X^T A X); R_p written to Rp (ld n).  Returns
 * 0 or the 1-based Cholesky breakdown column. */
static int cpu_pass(int m, int n, const double *A, long lda, const double *X,
                    long ldx, double *Q, long ldq, double *Rp, double *W,
                    double *C)
{
    cpu_symm_rowblock(m, n, A, lda, X, ldx, W);
    cpu_cross(m, n, X, ldx, W, C);
    const int info = orc_chol_upper(n, C, n, Rp, n);
    if (info)
        return info;
    orc_trsm_right_upper(m, n, X, ldx, Rp, n, Q, ldq);
    return 0;
}

/* A-CholQR2 on the CPU: Q (m x n, may alias Z exactly) and R = R_2 R_1.
 * Returns 0, the 1-based breakdown column, or -1 when memory runs out. */
int orc_cpu_cholqr2(int m, int n, const double *A, long lda, const double *Z,
                    long ldz, double *Q, long ldq, double *R, long ldr)
{
    double *W = (double *)malloc(sizeof(double) * (size_t)m * (size_t)n);
    double *C = (double *)malloc(sizeof(double) * (size_t)n * (size_t)n);
    double *R1 = (double *)malloc(sizeof(double) * (size_t)n * (size_t)n);
    double *R2 = (double *)malloc(sizeof(double) * (size_t)n * (size_t)n);
    int info = -1;
    if (W && C && R1 && R2) {
        info = cpu_pass(m, n, A, lda, Z, ldz, Q, ldq, R1, W, C);
        if (info == 0)
            info = cpu_pass(m, n, A, lda, Q, ldq, Q, ldq, R2, W, C);
        if (info == 0)
            orc_upper_times_upper(n, R2, n, R1, n, R, ldr);
    }
    free(W);
    free(C);
    free(R1);
    free(R2);
    return info;
}

/* Threads an OpenMP parallel region of this library uses. */
int orc_cpu_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
