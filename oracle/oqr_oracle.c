/*
 * CPU FP64 oracle for QR factorization in an oblique inner product
 * (Lowery & Langou, "Stability Analysis of QR factorization in an Oblique
 * Inner Product", arXiv:1401.5171).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Only the test suite, the smoke check and the
 * timed CPU baseline of the benchmark may load it.  It shares no code, header,
 * table or helper with the CUDA library, and the CUDA library never calls it.
 *
 * Problem (Sec. 1): given A (m x m, symmetric positive definite) and a
 * full-rank Z (m x n, m >= n), find Q (m x n) with Q^T A Q = I and R (n x n)
 * upper triangular with Z = Q R.  With a positive diagonal on R the pair is
 * unique, because Z^T A Z = R^T R (Sec. 2) fixes R as the Cholesky factor.
 *
 * The top-level oracle, orc_oblique_qr, follows Algorithm 3 (CHOL-EQR,
 * Sec. 4): Cholesky of A, then a Euclidean Householder QR of C Z, then
 * Q = C^{-1} Y.  This route does not share the rounding behaviour of the
 * normal-equation path it checks (its orthogonality does not grow with
 * kappa(Z)^2, Thm 4.1).  The remaining functions are the plain definitions of
 * each step of Algorithm 1 (CHOLQR), used to check single kernels.
 *
 * Conventions: column-major storage, element (i,j) of X at X[i + j*ldx];
 * only the lower triangle of every symmetric input is read; every sum runs in
 * index order; no blocking, no reassociation.  Compile without -ffast-math
 * and with -ffp-contract=off so that results do not depend on the host's
 * fused multiply-add.
 *
 * Parity status of each function (what pins it) is listed in the test file
 * tests/test_oracle_pins.py; every function here is pinned there.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define AT(X, i, j, ld) (X)[(size_t)(i) + (size_t)(j) * (size_t)(ld)]

/* a(i,j) of a symmetric matrix stored by its lower triangle. */
static double sym_lower(const double *A, long lda, long i, long j)
{
    return i >= j ? AT(A, i, j, lda) : AT(A, j, i, lda);
}

/*
 * Cholesky factor of a symmetric positive definite matrix, upper form:
 * A = C^T C with C upper triangular and positive diagonal.  This is the
 * "chol" of Algorithm 1 (line 3, Sec. 2) and Algorithm 3 (line 1, Sec. 4),
 * MATLAB convention.  Dot-product (row-by-row of C) form:
 *   c_jj = sqrt(a_jj - sum_{k<j} c_kj^2),
 *   c_ji = (a_ij - sum_{k<j} c_ki c_kj) / c_jj   for i > j.
 * The strict lower triangle of C is set to zero.  Returns 0, or the 1-based
 * column j at which the pivot a_jj - sum c_kj^2 is not positive (the matrix
 * is not numerically positive definite); C is then only partly written.
 */
int orc_chol_upper(int n, const double *A, long lda, double *C, long ldc)
{
    for (long j = 0; j < n; ++j)
        for (long i = j + 1; i < n; ++i)
            AT(C, i, j, ldc) = 0.0;
    for (long j = 0; j < n; ++j) {
        double s = AT(A, j, j, lda);
        for (long k = 0; k < j; ++k)
            s -= AT(C, k, j, ldc) * AT(C, k, j, ldc);
        if (!(s > 0.0))
            return (int)(j + 1);
        const double cjj = sqrt(s);
        AT(C, j, j, ldc) = cjj;
#pragma omp parallel for schedule(static)
        for (long i = j + 1; i < n; ++i) {
            double t = AT(A, i, j, lda);
            for (long k = 0; k < j; ++k)
                t -= AT(C, k, i, ldc) * AT(C, k, j, ldc);
            AT(C, j, i, ldc) = t / cjj;
        }
    }
    return 0;
}

/*
 * B = A Z with A symmetric (lower triangle read): line 1 of Algorithm 1.
 * b_ic = sum_k a_ik z_kc.
 */
void orc_symm_times(int m, int n, const double *A, long lda,
                    const double *Z, long ldz, double *B, long ldb)
{
#pragma omp parallel for schedule(static)
    for (long i = 0; i < m; ++i)
        for (long c = 0; c < n; ++c) {
            double s = 0.0;
            for (long k = 0; k < m; ++k)
                s += sym_lower(A, lda, i, k) * AT(Z, k, c, ldz);
            AT(B, i, c, ldb) = s;
        }
}

/*
 * Gram (normal-equation) matrix C = Z^T A Z: lines 1-2 of Algorithm 1
 * (B = A Z, then C = Z^T B).  g_rc = sum_i z_ir b_ic.  All n*n entries are
 * formed as written; the result is symmetric only up to rounding.
 */
void orc_gram(int m, int n, const double *A, long lda, const double *Z,
              long ldz, double *G, long ldg)
{
    double *B = (double *)malloc(sizeof(double) * (size_t)m * (size_t)n);
    orc_symm_times(m, n, A, lda, Z, ldz, B, m);
    for (long r = 0; r < n; ++r)
        for (long c = 0; c < n; ++c) {
            double s = 0.0;
            for (long i = 0; i < m; ++i)
                s += AT(Z, i, r, ldz) * AT(B, i, c, m);
            AT(G, r, c, ldg) = s;
        }
    free(B);
}

/*
 * Q = Z / R (MATLAB right division) with R upper triangular: line 4 of
 * Algorithm 1.  Solved row by row, as in the backward-error model of Sec. 2
 * (each row of Q solves q_i (R + dR^i) = z_i):
 *   q_ij = (z_ij - sum_{k<j} q_ik r_kj) / r_jj.
 * Q may alias Z exactly.
 */
void orc_trsm_right_upper(int m, int n, const double *Z, long ldz,
                          const double *R, long ldr, double *Q, long ldq)
{
#pragma omp parallel for schedule(static)
    for (long i = 0; i < m; ++i)
        for (long j = 0; j < n; ++j) {
            double t = AT(Z, i, j, ldz);
            for (long k = 0; k < j; ++k)
                t -= AT(Q, i, k, ldq) * AT(R, k, j, ldr);
            AT(Q, i, j, ldq) = t / AT(R, j, j, ldr);
        }
}

/*
 * Product of two upper triangular matrices, R = U S (the "R = US" of
 * Algorithm 2, line 3): r_ij = sum_{i<=k<=j} u_ik s_kj, zero below the
 * diagonal.  R must not alias U or S.
 */
void orc_upper_times_upper(int n, const double *U, long ldu, const double *S,
                           long lds, double *R, long ldr)
{
    for (long j = 0; j < n; ++j)
        for (long i = 0; i < n; ++i) {
            double s = 0.0;
            if (i <= j)
                for (long k = i; k <= j; ++k)
                    s += AT(U, i, k, ldu) * AT(S, k, j, lds);
            AT(R, i, j, ldr) = s;
        }
}

/*
 * CHOLQR, Algorithm 1, all four lines as written: B = A Z; C = Z^T B;
 * R = chol(C); Q = Z / R.  Returns 0 or the 1-based Cholesky breakdown column.
 * This restates the method itself on the CPU (it is not the oracle of the
 * result; orc_oblique_qr is).
 */
int orc_cholqr(int m, int n, const double *A, long lda, const double *Z,
               long ldz, double *Q, long ldq, double *R, long ldr)
{
    double *C = (double *)malloc(sizeof(double) * (size_t)n * (size_t)n);
    orc_gram(m, n, A, lda, Z, ldz, C, n);
    int info = orc_chol_upper(n, C, n, R, ldr);
    if (info == 0)
        orc_trsm_right_upper(m, n, Z, ldz, R, ldr, Q, ldq);
    free(C);
    return info;
}

/*
 * Euclidean Householder QR of W (m x n, m >= n): W = Y R_h with Y having
 * orthonormal columns (formed explicitly, thin) and R_h upper triangular.
 * Line 3 of Algorithm 3.  Reflector k: x = W(k:m, k), alpha = -sign(x_1)||x||
 * (sign(0) = +1), v = x - alpha e_1, H_k = I - 2 v v^T / (v^T v); H_k is
 * applied to the trailing columns, and Y = H_1 H_2 ... H_n [I_n; 0] is built
 * by applying the reflectors in reverse order to the thin identity.
 * W is overwritten.
 */
void orc_householder_qr(int m, int n, double *W, long ldw, double *Y, long ldy,
                        double *Rh, long ldr)
{
    double *V = (double *)calloc((size_t)m * (size_t)n, sizeof(double));
    double *vtv = (double *)calloc((size_t)n, sizeof(double));
    for (long k = 0; k < n; ++k) {
        double nrm2 = 0.0;
        for (long i = k; i < m; ++i)
            nrm2 += AT(W, i, k, ldw) * AT(W, i, k, ldw);
        const double nrm = sqrt(nrm2);
        const double x1 = AT(W, k, k, ldw);
        const double alpha = (x1 >= 0.0) ? -nrm : nrm;
        for (long i = k; i < m; ++i)
            AT(V, i, k, m) = AT(W, i, k, ldw);
        AT(V, k, k, m) -= alpha;
        double s = 0.0;
        for (long i = k; i < m; ++i)
            s += AT(V, i, k, m) * AT(V, i, k, m);
        vtv[k] = s;
        if (s == 0.0)
            continue; /* the column is already zero below the diagonal */
#pragma omp parallel for schedule(static)
        for (long j = k; j < n; ++j) {
            double d = 0.0;
            for (long i = k; i < m; ++i)
                d += AT(V, i, k, m) * AT(W, i, j, ldw);
            const double f = 2.0 * d / s;
            for (long i = k; i < m; ++i)
                AT(W, i, j, ldw) -= f * AT(V, i, k, m);
        }
    }
    for (long j = 0; j < n; ++j)
        for (long i = 0; i < n; ++i)
            AT(Rh, i, j, ldr) = (i <= j) ? AT(W, i, j, ldw) : 0.0;
    for (long j = 0; j < n; ++j)
        for (long i = 0; i < m; ++i)
            AT(Y, i, j, ldy) = (i == j) ? 1.0 : 0.0;
    for (long k = n - 1; k >= 0; --k) {
        if (vtv[k] == 0.0)
            continue;
#pragma omp parallel for schedule(static)
        for (long j = 0; j < n; ++j) {
            double d = 0.0;
            for (long i = k; i < m; ++i)
                d += AT(V, i, k, m) * AT(Y, i, j, ldy);
            const double f = 2.0 * d / vtv[k];
            for (long i = k; i < m; ++i)
                AT(Y, i, j, ldy) -= f * AT(V, i, k, m);
        }
    }
    free(vtv);
    free(V);
}

/*
 * The oracle: oblique QR by CHOL-EQR (Algorithm 3, Sec. 4).
 *   1. C = chol(A), A = C^T C, C upper.
 *   2. W = C Z.
 *   3. [Y, R_h] = qr(W), Householder, thin Y explicit.
 *   4. Sign normalisation: D = diag(sign(r_h,ii)), sign(0) = +1;
 *      R = D R_h, Y <- Y D, so that R has a positive diagonal and (Q, R) is
 *      the unique factorization (MATLAB's qr leaves the signs free).
 *   5. Q = C^{-1} Y, back substitution column by column.  The algorithm's
 *      last line is printed as "Q = C \ Z"; the text of Sec. 4 says Q is
 *      obtained from C^{-1} Y, which is what is computed here.
 * Q (m x n), R (n x n, zero below the diagonal) are outputs.  Returns 0, or
 * the 1-based column at which the Cholesky factorization of A breaks down.
 */
int orc_oblique_qr(int m, int n, const double *A, long lda, const double *Z,
                   long ldz, double *Q, long ldq, double *R, long ldr)
{
    double *C = (double *)malloc(sizeof(double) * (size_t)m * (size_t)m);
    double *W = (double *)malloc(sizeof(double) * (size_t)m * (size_t)n);
    int info = orc_chol_upper(m, A, lda, C, m);
    if (info != 0) {
        free(W);
        free(C);
        return info;
    }
    /* W = C Z, C upper: w_ic = sum_{k>=i} c_ik z_kc */
#pragma omp parallel for schedule(static)
    for (long c = 0; c < n; ++c)
        for (long i = 0; i < m; ++i) {
            double s = 0.0;
            for (long k = i; k < m; ++k)
                s += AT(C, i, k, m) * AT(Z, k, c, ldz);
            AT(W, i, c, m) = s;
        }
    orc_householder_qr(m, n, W, m, Q, ldq, R, ldr);
    for (long j = 0; j < n; ++j) {
        if (AT(R, j, j, ldr) < 0.0) {
            for (long c = j; c < n; ++c)
                AT(R, j, c, ldr) = -AT(R, j, c, ldr);
            for (long i = 0; i < m; ++i)
                AT(Q, i, j, ldq) = -AT(Q, i, j, ldq);
        }
    }
    /* Q <- C^{-1} Q in place: for k = m-1 .. 0, q_k /= c_kk, then
     * q_i -= c_ik q_k for i < k (column-oriented back substitution). */
#pragma omp parallel for schedule(static)
    for (long c = 0; c < n; ++c)
        for (long k = m - 1; k >= 0; --k) {
            const double qk = AT(Q, k, c, ldq) / AT(C, k, k, m);
            AT(Q, k, c, ldq) = qk;
            for (long i = 0; i < k; ++i)
                AT(Q, i, c, ldq) -= AT(C, i, k, m) * qk;
        }
    free(W);
    free(C);
    return 0;
}

/*
 * Loss of orthogonality as a matrix: E = Q^T A Q - I (the quantity whose
 * 2-norm Sec. 7 plots), every entry summed in long double, A symmetric by its
 * lower triangle.  e_rc = sum_i sum_k q_ir a_ik q_kc - delta_rc.
 */
void orc_orth_defect(int m, int n, const double *A, long lda, const double *Q,
                     long ldq, double *E, long lde)
{
    long double *AQ = (long double *)malloc(sizeof(long double) * (size_t)m * (size_t)n);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < m; ++i)
        for (long c = 0; c < n; ++c) {
            long double s = 0.0L;
            for (long k = 0; k < m; ++k)
                s += (long double)sym_lower(A, lda, i, k) * (long double)AT(Q, k, c, ldq);
            AQ[(size_t)i + (size_t)c * (size_t)m] = s;
        }
    for (long r = 0; r < n; ++r)
        for (long c = 0; c < n; ++c) {
            long double s = 0.0L;
            for (long i = 0; i < m; ++i)
                s += (long double)AT(Q, i, r, ldq) * AQ[(size_t)i + (size_t)c * (size_t)m];
            AT(E, r, c, lde) = (double)(s - (r == c ? 1.0L : 0.0L));
        }
    free(AQ);
}

/*
 * Representativity residual D = Z - Q R (Sec. 7 plots ||Z - QR|| / ||Z||),
 * each entry summed in long double over the upper triangle of R.
 */
void orc_repres_residual(int m, int n, const double *Z, long ldz,
                         const double *Q, long ldq, const double *R, long ldr,
                         double *D, long ldd)
{
#pragma omp parallel for schedule(static)
    for (long i = 0; i < m; ++i)
        for (long j = 0; j < n; ++j) {
            long double s = 0.0L;
            for (long k = 0; k <= j; ++k)
                s += (long double)AT(Q, i, k, ldq) * (long double)AT(R, k, j, ldr);
            AT(D, i, j, ldd) = (double)((long double)AT(Z, i, j, ldz) - s);
        }
}

/*
 * The oracle for a tridiagonal A (Sec. 8's second workload, where the paper
 * notes that factoring A is cheap, so CHOL-EQR is viable): Algorithm 3 with
 * A = T, T(i, i) = d_i, T(i + 1, i) = T(i, i + 1) = e_i.
 *   1. T = C^T C with C upper bidiagonal (the Cholesky recurrence of
 *      orc_chol_upper restricted to T's nonzeros):
 *        c_00 = sqrt(d_0),  c_{i-1,i} = e_{i-1} / c_{i-1,i-1},
 *        c_ii = sqrt(d_i - c_{i-1,i}^2).
 *   2. W = C Z: w_ic = c_ii z_ic + c_{i,i+1} z_{i+1,c}.
 *   3. Householder QR of W (orc_householder_qr), 4. sign normalisation,
 *   5. Q = C^{-1} Y by bidiagonal back substitution,
 *        q_{m-1} = y_{m-1} / c_{m-1,m-1},  q_i = (y_i - c_{i,i+1} q_{i+1}) / c_ii.
 * Returns 0, or the 1-based row at which a pivot of T is not positive.
 */
int orc_oblique_qr_tridiag(int m, int n, const double *d, const double *e,
                           const double *Z, long ldz, double *Q, long ldq,
                           double *R, long ldr)
{
    double *cd = (double *)malloc(sizeof(double) * (size_t)m);
    double *cu = (double *)malloc(sizeof(double) * (size_t)m); /* cu[i] = c_{i,i+1} */
    double *W = (double *)malloc(sizeof(double) * (size_t)m * (size_t)n);
    for (long i = 0; i < m; ++i) {
        double p = d[i];
        if (i > 0)
            p -= cu[i - 1] * cu[i - 1];
        if (!(p > 0.0)) {
            free(W);
            free(cu);
            free(cd);
            return (int)(i + 1);
        }
        cd[i] = sqrt(p);
        cu[i] = (i + 1 < m) ? e[i] / cd[i] : 0.0;
    }
#pragma omp parallel for schedule(static)
    for (long c = 0; c < n; ++c)
        for (long i = 0; i < m; ++i)
            AT(W, i, c, m) = cd[i] * AT(Z, i, c, ldz) +
                             ((i + 1 < m) ? cu[i] * AT(Z, i + 1, c, ldz) : 0.0);
    orc_householder_qr(m, n, W, m, Q, ldq, R, ldr);
    for (long j = 0; j < n; ++j) {
        if (AT(R, j, j, ldr) < 0.0) {
            for (long c = j; c < n; ++c)
                AT(R, j, c, ldr) = -AT(R, j, c, ldr);
            for (long i = 0; i < m; ++i)
                AT(Q, i, j, ldq) = -AT(Q, i, j, ldq);
        }
    }
#pragma omp parallel for schedule(static)
    for (long c = 0; c < n; ++c)
        for (long i = m - 1; i >= 0; --i) {
            double t = AT(Q, i, c, ldq);
            if (i + 1 < m)
                t -= cu[i] * AT(Q, i + 1, c, ldq);
            AT(Q, i, c, ldq) = t / cd[i];
        }
    free(W);
    free(cu);
    free(cd);
    return 0;
}

/*
 * E = Q^T T Q - I for tridiagonal T, every entry summed in long double:
 * (T Q)_ic = e_{i-1} q_{i-1,c} + d_i q_ic + e_i q_{i+1,c}.
 */
void orc_orth_defect_tridiag(int m, int n, const double *d, const double *e,
                             const double *Q, long ldq, double *E, long lde)
{
    long double *TQ = (long double *)malloc(sizeof(long double) * (size_t)m * (size_t)n);
#pragma omp parallel for schedule(static)
    for (long c = 0; c < n; ++c)
        for (long i = 0; i < m; ++i) {
            long double s = (long double)d[i] * (long double)AT(Q, i, c, ldq);
            if (i > 0)
                s += (long double)e[i - 1] * (long double)AT(Q, i - 1, c, ldq);
            if (i + 1 < m)
                s += (long double)e[i] * (long double)AT(Q, i + 1, c, ldq);
            TQ[(size_t)i + (size_t)c * (size_t)m] = s;
        }
#pragma omp parallel for schedule(static)
    for (long c = 0; c < n; ++c)
        for (long r = 0; r < n; ++r) {
            long double s = 0.0L;
            for (long i = 0; i < m; ++i)
                s += (long double)AT(Q, i, r, ldq) * TQ[(size_t)i + (size_t)c * (size_t)m];
            AT(E, r, c, lde) = (double)(s - (r == c ? 1.0L : 0.0L));
        }
    free(TQ);
}
