/*
 * liboqr: QR factorization in an oblique inner product on one GB300 GPU.
 *
 * Problem (Lowery & Langou, arXiv:1401.5171, Sec. 1): given A (m x m,
 * symmetric positive definite) and Z (m x n, full rank, m >= n >= 1), find
 * Q (m x n) with Q^T A Q = I and R (n x n, upper triangular) with Z = Q R.
 * R has a positive diagonal, which makes (Q, R) unique: R is the Cholesky
 * factor of the normal-equation matrix Z^T A Z (Sec. 2).
 *
 * Conventions for every entry point below:
 *   - Matrices are FP64, column-major: element (i, j) of X is X[i + j*ldx],
 *     ldx >= number of rows.  All matrix pointers are DEVICE pointers owned by
 *     the caller.
 *   - A is read from its lower triangle only; the strict upper triangle is
 *     never read and may hold anything.
 *   - R is written in full: positive diagonal, zeros below it.
 *   - Q may alias Z exactly (in-place factorization).  Any other overlap of an
 *     output with an input is not allowed and is not detected.
 *   - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *     stream) and runs asynchronously.  If `info` is non-NULL the call
 *     synchronizes the stream and reports device-side outcomes (Cholesky
 *     breakdown, timeouts) in the return value and in *info.  If `info` is
 *     NULL the call returns after enqueueing; device-side outcomes are then
 *     read with oqr_get_status.
 *   - The context's device must be the current device of the calling thread.
 *   - Scratch memory comes from the context's workspace: a buffer that the
 *     context allocates on first need and keeps (grown when a larger problem
 *     arrives), or one the caller hands over with oqr_set_workspace.
 *   - Errors never abort, trap or hang: every device-side wait has a time
 *     limit (oqr_opts.spin_limit) after which the kernel records
 *     OQR_ERR_TIMEOUT and returns.
 */
#ifndef OQR_H
#define OQR_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    OQR_OK = 0,
    OQR_ERR_INVALID_ARG = 1,   /* bad size, leading dimension, pointer or option */
    OQR_ERR_NOT_SPD = 2,       /* Cholesky breakdown; info = 1-based column */
    OQR_ERR_CHECK_FAILED = 3,  /* the requested orthogonality check exceeded its tolerance */
    OQR_ERR_CUDA = 4,          /* a CUDA runtime call failed */
    OQR_ERR_NO_MEMORY = 5,     /* workspace could not be allocated or is too small */
    OQR_ERR_TIMEOUT = 6,       /* a device-side wait ran past spin_limit */
    OQR_ERR_UNSUPPORTED = 7    /* size or option outside what the library supports */
} oqr_status;

typedef enum {
    OQR_FP64 = 0,     /* every product in FP64 (DFMA) */
    OQR_BF16X3 = 1,   /* hi/lo BF16 split, 3 products, FP32 accumulation (tensor cores) */
    OQR_FP8 = 2,      /* E4M3 with a power-of-two scale per (row or column, 128-long chunk of the
                         contraction), one product, drained and scaled every chunk (tensor cores) */
    OQR_FP64_TC = 3,  /* FP64-accurate products from 7 exact BF16 slices per operand, exact FP32
                         accumulation per 256-long chunk, double-float sum (tensor cores) */
    OQR_TC2 = 4       /* the 2 leading slices of the OQR_FP64_TC split (16 bits of each element
                         relative to its 256-chunk's largest magnitude), 3 products per chunk in FP32,
                         scaled every chunk (tensor cores).  Within one factorization, passes in
                         OQR_TC2 and OQR_FP64_TC (and an opts->check = 2) split A once and share it. */
} oqr_precision;

typedef enum { OQR_ALGO_CHOLQR = 0, OQR_ALGO_CHOLQR2 = 1, OQR_ALGO_SCHOLQR3 = 2, OQR_ALGO_CGS2 = 3 } oqr_algo;

/* Options; a NULL pointer means all defaults (the values in brackets). */
typedef struct {
    int passes;       /* oqr_cholqr2: passes of the normal-equation method [2]; 3 when shifted */
    int shifted;      /* oqr_cholqr2: 1 = shifted A-CholQR3, a shifted first pass then two plain ones [0] */
    int prec;         /* oqr_precision of the preconditioning passes [OQR_FP64] */
    double shift_c;   /* constant c of the shift s = c u (m n + n (n+1)) ||A||_F ||Z||_F^2 [11] */
    int block;        /* oqr_cgs2: column block size b [64] */
    int check;        /* measure ||Q^T A Q - I||_2 after the factorization into info->orth_err [0]:
                         1 = with an FP64 Gram, 2 = with the FP64-accurate tensor-core Gram */
    long spin_limit;  /* time limit of any device-side wait, in nanoseconds [4e9] */
    int final_prec;   /* oqr_cholqr2: oqr_precision of the last pass [OQR_FP64]; the last pass sets the
                         final orthogonality, so FP64-level results need OQR_FP64 or OQR_FP64_TC */
    int prec_mid;     /* passes between the first and the last: oqr_precision, or -1 = same as prec [-1] */
    int reuse_w;      /* oqr_cholqr2 (FP64, two passes, dense A): 1 = form W = A Z once and take the second
                         pass's A Q_1 as W R_1^{-1} instead of a second product with A [0] */
    /* oqr_batched only: */
    const int* batch_splits;      /* OQR_BATCHED_FP64: the work plan, the number of k-ranges each instance's Gram
                                     is cut into (host, count ints in 1..64, as an autotuner chose them); NULL =
                                     the built-in heuristic [NULL] */
    const float* selector_params; /* OQR_BATCHED_SELECTOR: the trained network (device, oqr_mlp_param_count()
                                     FP32 values, the layout of oqr_mlp_forward) [NULL] */
    double selector_tol;          /* OQR_BATCHED_SELECTOR: the largest ||Q^T A Q - I||_F a one-pass (or
                                     checked) result may keep [1e-12] */
    int selector_check;           /* OQR_BATCHED_SELECTOR: 0 = check the one-pass results only (their check is
                                     the Gram the second pass would factor), 1 = also every other tensor-core
                                     result, with one more Gram [0] */
    double* batch_orth;           /* optional device output (count doubles): the checks.  OQR_BATCHED_TC*:
                                     ||Q_b^T A_b Q_b - I||_2 estimates (power iteration on one more FP64-accurate
                                     Gram of Q_b; +inf after a breakdown); OQR_BATCHED_SELECTOR: ||Q_b^T A_b Q_b -
                                     I||_F of the checked Gram (an upper bound of the 2-norm); NaN where the mode
                                     did not check the instance [NULL] */
    int* batch_choice;            /* OQR_BATCHED_SELECTOR: optional device output (count ints), the option whose
                                     result each instance holds: 0 one pass, 1 two passes, 2 shifted three passes
                                     (all FP64-accurate on the tensor cores), 3 FP64 A-CholQR2 [NULL] */
} oqr_opts;

/* Optional per-call report (filled only when passed non-NULL). */
typedef struct {
    int info;          /* 1-based breakdown column for OQR_ERR_NOT_SPD, else 0 */
    int passes_run;    /* normal-equation passes (or CGS2 sweeps per block) executed */
    double orth_err;   /* ||Q^T A Q - I||_2 estimate when opts->check, else -1 */
    double shift;      /* shift s used by the first pass of shifted A-CholQR3, else 0 */
} oqr_info;

typedef struct oqr_ctx oqr_ctx;

/* Fills *opts with the defaults. */
void oqr_default_opts(oqr_opts* opts);

/* Human-readable name of a status code (static string). */
const char* oqr_status_string(oqr_status s);

/* Creates a context bound to CUDA device `device` (made current by the call).
 * No workspace is allocated yet. */
oqr_status oqr_create(oqr_ctx** ctx, int device);

/* Releases the context and the workspace it allocated (not one handed over
 * with oqr_set_workspace).  NULL is accepted. */
oqr_status oqr_destroy(oqr_ctx* ctx);

/* Bytes of workspace that `algo` (oqr_algo) needs for an m x n problem. */
oqr_status oqr_workspace_size(oqr_ctx* ctx, int algo, int m, int n, const oqr_opts* opts, size_t* bytes);

/* Hands the context a caller-owned device buffer of `bytes` bytes (256-byte
 * aligned) to use as workspace; the context then never allocates.  A call
 * that needs more returns OQR_ERR_NO_MEMORY.  ptr = NULL returns to
 * context-owned workspace. */
oqr_status oqr_set_workspace(oqr_ctx* ctx, void* ptr, size_t bytes);

/* Device-side outcome of the last call on this context: synchronizes
 * `stream`, returns the status code and writes the breakdown column to
 * *info (may be NULL). */
oqr_status oqr_get_status(oqr_ctx* ctx, void* stream, int* info);

/*
 * A-CholQR: one pass of Algorithm 1 (CHOLQR, Sec. 2):
 *   B = A Z;  C = Z^T B;  R = chol(C);  Q = Z / R.
 * B is never stored: C is formed by one fused kernel as P + P^T with
 * P = Z^T (M Z), M = tril(A, -1) + diag(A)/2, reading A's lower triangle
 * once.  Q = Z / R is the row-wise triangular solve of Sec. 2.
 * Accuracy (Thm 2.1): ||Q^T A Q - I|| grows like u kappa(A^{1/2} Z)^2.
 */
oqr_status oqr_cholqr(oqr_ctx* ctx, int m, int n, const double* A, long lda, const double* Z, long ldz,
                      double* Q, long ldq, double* R, long ldr, const oqr_opts* opts, oqr_info* info,
                      void* stream);

/*
 * A-CholQR2 (default) and shifted A-CholQR3 (opts->shifted = 1): Algorithm 1
 * repeated on its own output, Q_1 = Z R_1^{-1}, Q = Q_1 R_2^{-1},
 * R = R_2 R_1 (the product form of "R = U S", Algorithm 2).  The shifted form
 * adds s I to the first pass's normal-equation matrix so that its Cholesky
 * completes for ill-conditioned Z, then runs two plain passes,
 * R = R_3 R_2 R_1.  Neither repetition is in the paper; they follow the
 * Euclidean CholeskyQR2 and shifted CholeskyQR3 with Z^T Z replaced by
 * Z^T A Z.  Every pass but the last forms its normal-equation matrix in
 * opts->prec and the last in opts->final_prec; the Cholesky factorizations,
 * the shift, the triangular solves and R = R_2 R_1 are always FP64.  The
 * mixed form (prec = OQR_BF16X3, final_prec = OQR_FP64_TC) runs all products
 * on the tensor cores; its accuracy comes from the last pass, whose
 * normal-equation matrix is FP64-accurate.  The shift of a shifted first pass
 * is c u (m n + n (n+1)) ||A||_F ||Z||_F^2 (u = 2^-53) when that pass is FP64
 * or FP64_TC, and c u trace(G) (u = 2^-16, G the pass's BF16X3 matrix) when
 * it is BF16X3, whose rounding error scales with G rather than with the
 * worst-case bound.
 * With opts->reuse_w = 1 (FP64 only, two passes, not shifted; anything else
 * returns OQR_ERR_UNSUPPORTED) the first pass keeps W = A Z (one FP64 product
 * over A's lower triangle, m x n of workspace) and the second pass takes
 * A Q_1 = W R_1^{-1} (a triangular solve, O(m n^2)) instead of a second
 * product with A: Q_1 = Z R_1^{-1}, G_2 = Q_1^T (W R_1^{-1}), R_2 = chol(G_2),
 * Q = Q_1 R_2^{-1}, R = R_2 R_1.  The paper has no such variant; it trades
 * accuracy (A Q_1's rounding is no longer that of a fresh product, so the
 * loss of orthogonality keeps one factor of kappa(A^{1/2} Z)) for the second
 * product with A.
 */
oqr_status oqr_cholqr2(oqr_ctx* ctx, int m, int n, const double* A, long lda, const double* Z, long ldz,
                       double* Q, long ldq, double* R, long ldr, const oqr_opts* opts, oqr_info* info,
                       void* stream);

/*
 * A-CGS2: classical Gram-Schmidt with reorthogonalisation in the A inner
 * product (Sec. 6, Thm 6.4), in block form with column blocks of
 * opts->block columns.  For each block Z_j: twice
 * { r = (A Q)^T Z_j; Z_j -= Q r; R(<j, j) += r }; then S_j = A Z_j of the
 * projected block and A-CholQR2 of the block against S_j, whose solves give
 * the block's A Q; A Q is kept so that each block costs one product with A.
 * Needs an extra m x n of workspace for A Q.
 */
/*
 * oqr_cholqr2_host: oqr_cholqr2 with A, Z, Q and R in HOST memory (column-major,
 * the same meaning, layouts and options).  Only A's lower triangle is copied to
 * the device, in panels of 256 columns (rows j0..m-1 of each), on an internal
 * copy stream; when the first pass runs in OQR_TC2 or OQR_FP64_TC, each panel's
 * slices are made on `stream` as soon as the panel has arrived, under the
 * copies of the later panels.  Z is copied in one piece; Q and R are copied
 * back on `stream` at the end.  For the copies to run asynchronously the host
 * buffers must be pinned (cudaHostAlloc or cudaHostRegister); with pageable
 * memory the call still gives the same results.  The device copies of A, Z, Q
 * and R are held by the context and reused; the call must not overlap another
 * call on the same context.  Returns when the work is enqueued, unless info is
 * non-NULL (then it synchronizes and reports as oqr_cholqr2 does).  The paper
 * has no counterpart: it is the host-to-result form of the same factorization.
 */
oqr_status oqr_cholqr2_host(oqr_ctx* ctx, int m, int n, const double* A, long lda, const double* Z, long ldz,
                            double* Q, long ldq, double* R, long ldr, const oqr_opts* opts, oqr_info* info,
                            void* stream);

oqr_status oqr_cgs2(oqr_ctx* ctx, int m, int n, const double* A, long lda, const double* Z, long ldz,
                    double* Q, long ldq, double* R, long ldr, const oqr_opts* opts, oqr_info* info,
                    void* stream);

/*
 * Step kernels of Algorithm 1, exposed for testing and composition.
 *
 * oqr_gram: G = Z^T A Z (lines 1-2 of Algorithm 1), n x n, written in full
 *   and exactly symmetric.  prec selects the arithmetic of the products:
 *   OQR_FP64 (DFMA), or OQR_BF16X3, OQR_FP8, OQR_FP64_TC, OQR_TC2 (tensor cores).
 * oqr_potrf: R = chol(G + shift I) (line 3), G read from its lower triangle,
 *   R upper with positive diagonal, zeros below.  Breakdown is reported as
 *   OQR_ERR_NOT_SPD with the 1-based column (synchronizes the stream when
 *   info != NULL).
 * oqr_trsm: Q = Z / R (line 4), row-wise substitution; Q may alias Z.
 * oqr_trsm_tc: the same solve in 64-column blocks: for each block, the
 *   product of the already solved columns with R's block column is formed
 *   FP64-accurately on the tensor cores (the OQR_FP64_TC slices), and the
 *   64 x 64 diagonal block is solved by FP64 row-wise substitution.  The
 *   factorizations use it in every pass whose Gram runs on the tensor cores,
 *   except the last pass of a multi-pass one (oqr_trsm_last).
 *   Uses the context's workspace; Q may alias Z.
 * oqr_trsm_last: the solve of a multi-pass factorization's last tensor-core
 *   pass, Q = Z / R, given the symmetric G = R^T R the factor came from (read
 *   from its lower triangle).  When ||G - I||_F <= 0.5 (every eigenvalue of G
 *   in [0.5, 1.5], so cond(R)^2 <= 3), R^{-1} is formed by FP64 back
 *   substitution and Q = Z R^{-1} is one FP64-accurate tensor-core product;
 *   otherwise it is oqr_trsm (FP64 row-wise substitution).  The choice is
 *   taken on the device (no synchronization).  n <= 8192 (else
 *   OQR_ERR_UNSUPPORTED; the factorizations then solve their last pass with
 *   oqr_trsm_tc's method).
 *   Uses the context's workspace; Q may alias Z.
 * oqr_rprod: R = U S for upper triangular U, S (R must not alias U or S).
 * oqr_check: E = Q^T A Q - I (n x n, written in full when E != NULL), and
 *   the estimate of ||E||_2 (Sec. 7's orthogonality measure) in *orth2 and
 *   ||E||_F in *orthF (host pointers, may be NULL; non-NULL synchronizes).
 */
oqr_status oqr_gram(oqr_ctx* ctx, int m, int n, const double* A, long lda, const double* Z, long ldz,
                    double* G, long ldg, int prec, void* stream);
oqr_status oqr_potrf(oqr_ctx* ctx, int n, const double* G, long ldg, double shift, double* R, long ldr,
                     int* info, void* stream);
oqr_status oqr_trsm_tc(oqr_ctx* ctx, int m, int n, const double* Z, long ldz, const double* R, long ldr,
                       double* Q, long ldq, void* stream);
oqr_status oqr_trsm(oqr_ctx* ctx, int m, int n, const double* Z, long ldz, const double* R, long ldr,
                    double* Q, long ldq, void* stream);
oqr_status oqr_trsm_last(oqr_ctx* ctx, int m, int n, const double* G, long ldg, const double* Z, long ldz,
                         const double* R, long ldr, double* Q, long ldq, void* stream);
oqr_status oqr_rprod(oqr_ctx* ctx, int n, const double* U, long ldu, const double* S, long lds, double* R,
                     long ldr, void* stream);
oqr_status oqr_check(oqr_ctx* ctx, int m, int n, const double* A, long lda, const double* Q, long ldq,
                     double* E, long lde, double* orth2, double* orthF, void* stream);

/*
 * Diagnostic of the failure path: one device-side wait that nothing
 * completes, limited to limit_ns (1 ns .. 10 s), after which the kernel records
 * OQR_ERR_TIMEOUT in the context's status (read it with oqr_get_status), as
 * every time-limited wait of the library does.  Nothing asynchronous is in
 * flight when it gives up, so the context stays usable; the next call resets
 * the status.  Asynchronous.
 */
oqr_status oqr_diag_timeout(oqr_ctx* ctx, long limit_ns, void* stream);

/*
 * oqr_repres: Sec. 7's representativity measure of a factorization,
 * ||Z - Q R||_2 / ||Z||_2, in *res2 (the two 2-norms estimated by power
 * iteration on D^T D and Z^T Z, D = Z - Q R formed in FP64; lower bounds that
 * converge to them), and ||Z - Q R||_F / ||Z||_F in *resF (host pointers, may
 * be NULL).  Z, Q (m x n) and R (n x n, read in full) are column-major device
 * memory; 1 <= n <= min(m, 1024) (n above 1024 returns OQR_ERR_UNSUPPORTED).
 * Uses the context's workspace (m n + 2 n^2 doubles and split-K partials) and
 * synchronizes the stream.
 */
oqr_status oqr_repres(oqr_ctx* ctx, int m, int n, const double* Z, long ldz, const double* Q, long ldq,
                      const double* R, long ldr, double* res2, double* resF, void* stream);

/*
 * PRE-CHOLQR (Algorithm 2, Sec. 3): [Y, S] = qr(Z) (Euclidean), then
 * [Q, U] = CHOLQR(A, Y), R = U S.  The Euclidean QR is Householder QR
 * (oqr_tsqr, FP64), so Y is orthonormal to working precision and the loss of
 * orthogonality of Q no longer depends on kappa(Z) (Thm 3.1:
 * ||Q^T A Q - I||_2 <= c m n^2 u ||Q||_2^2 ||A||_2).  The CHOLQR pass runs in
 * opts->final_prec (OQR_FP64 or OQR_FP64_TC; opts->check as for
 * oqr_cholqr2); R has a positive diagonal.  Q may alias Z.  Workspace: the
 * Householder QR's (about 3 m n doubles for n > 32) and the pass's.
 * oqr_precholqr_tridiag: the same for a tridiagonal A (d, e as for
 *   oqr_cholqr2_tridiag).
 * oqr_tsqr: the Euclidean step alone, Z = Y S with Y (m x n, device) having
 *   orthonormal columns and S (n x n, device) upper triangular with a
 *   positive diagonal (zeros below).  Y must not overlap Z.  For n <= 32 it is
 *   Householder QR on a reduction tree (TSQR: leaves of max(n, 256) rows,
 *   stacked pairs of R factors, Y formed top-down).  Above, it is blocked
 *   Householder QR: panels of 32 columns, each factored column by column
 *   (LAPACK's reflectors) in one cooperative launch over all SMs with
 *   time-limited grid-wide waits, blocked as I - V T V^T, the trailing
 *   columns updated as C - V T^T V^T C and Y formed by applying the
 *   reflectors to [I; 0], both by FP64 GEMMs.  oqr_tsqr synchronizes the
 *   stream and returns the context status (OQR_ERR_TIMEOUT if a grid-wide
 *   wait of the panel factorization ran out).
 */
oqr_status oqr_precholqr(oqr_ctx* ctx, int m, int n, const double* A, long lda, const double* Z, long ldz, double* Q,
                         long ldq, double* R, long ldr, const oqr_opts* opts, oqr_info* info, void* stream);
oqr_status oqr_precholqr_tridiag(oqr_ctx* ctx, int m, int n, const double* d, const double* e, const double* Z,
                                 long ldz, double* Q, long ldq, double* R, long ldr, const oqr_opts* opts,
                                 oqr_info* info, void* stream);
oqr_status oqr_tsqr(oqr_ctx* ctx, int m, int n, const double* Z, long ldz, double* Y, long ldy, double* S, long lds,
                    void* stream);

/*
 * Tridiagonal A (Sec. 8's second workload): A = T with diagonal d (m
 * doubles) and off-diagonal e (m - 1 doubles; may be NULL when m = 1),
 * T(i, i) = d[i], T(i + 1, i) = T(i, i + 1) = e[i]; d and e are device
 * memory.  Products with T cost O(m n), so each pass is O(m n^2), the
 * paper's normalised count 2 m n^2 per CHOLQR.
 *
 * oqr_cholqr2_tridiag: the normal-equation method of oqr_cholqr2 (and
 *   oqr_cholqr with opts->passes = 1, shifted A-CholQR3 with opts->shifted)
 *   for A = T, with the same options, outputs, aliasing and reporting.  Each
 *   pass forms U = M X (M = tril(T, -1) + diag(T) / 2, written once, m x n),
 *   then C = X^T U in the pass's precision (FP64 GEMM, or the tensor cores
 *   for OQR_FP64_TC, OQR_TC2, OQR_BF16X3, OQR_FP8) and G = C + C^T; the
 *   Cholesky factorization, Q = X / R and R = R_2 R_1 are as in oqr_cholqr2.
 *   The shift of a shifted FP64 or FP64_TC first pass uses ||T||_F.
 * oqr_gram_tridiag: that pass's G = Z^T T Z (n x n, exactly symmetric) alone.
 */
oqr_status oqr_cholqr2_tridiag(oqr_ctx* ctx, int m, int n, const double* d, const double* e, const double* Z, long ldz,
                               double* Q, long ldq, double* R, long ldr, const oqr_opts* opts, oqr_info* info,
                               void* stream);
oqr_status oqr_gram_tridiag(oqr_ctx* ctx, int m, int n, const double* d, const double* e, const double* Z, long ldz,
                            double* G, long ldg, int prec, void* stream);

/*
 * oqr_glls: the generalized least-squares application of Sec. 1,
 *   x = argmin ||Z x - b||_A = R^{-1} Q^T A b,
 *   for k right-hand sides B (m x k, column-major device memory) given the
 *   oblique QR (Q, R) of Z (from any factorization above; Q m x n, R n x n
 *   upper triangular, read in full).  X (n x k, device) receives the
 *   solutions.  A is read from its lower triangle, once per group of 8
 *   right-hand sides (the step that HBM bandwidth bounds); Q^T (A B) and the
 *   back substitution with R are FP64.  Uses the context's workspace (per
 *   64 x 64 tile of A's lower triangle, 1 KB per right-hand side up to 8, and
 *   m k + n k doubles).  Asynchronous; argument errors are returned.
 * oqr_symm: C = A B (m x k) for the symmetric A of this library's
 *   convention (lower triangle read), the first step of oqr_glls: 64 x 64
 *   tiles of A's lower triangle, each read once, every row of C summed in a
 *   fixed order (deterministic).  C must not overlap A or B.
 */
oqr_status oqr_glls(oqr_ctx* ctx, int m, int n, int k, const double* A, long lda, const double* Q, long ldq,
                    const double* R, long ldr, const double* B, long ldb, double* X, long ldx, void* stream);
oqr_status oqr_symm(oqr_ctx* ctx, int m, int k, const double* A, long lda, const double* B, long ldb, double* C,
                    long ldc, void* stream);

/*
 * Batched oblique QR: `count` independent instances, instance b with A_b
 * (m[b] x m[b], lower triangle read), Z_b (m[b] x n[b]) -> Q_b, R_b, all
 * column-major FP64 device memory, 1 <= n[b] <= min(m[b], 64), m[b] <= 4096.
 * m, n, the pointer arrays and the leading-dimension arrays are HOST arrays
 * (the pointers in them are device pointers).  status is a DEVICE array of
 * count ints: 0 for success, else the 1-based column at which instance b's
 * Cholesky broke down (its Q_b, R_b are then undefined; the other instances
 * are unaffected), or -1 for every instance when a tensor-core wait timed out.
 * mode (oqr_batched_mode):
 *   OQR_BATCHED_FP64: A-CholQR2, Algorithm 1 twice (CHOLQR, Sec. 2;
 *     R = R_2 R_1), every Gram in FP64 FMA; opts->batch_splits is the work
 *     plan.  The batch-wide kernel sequence (about 13 launches) is captured into
 *     one CUDA graph that the context caches and replays while the batch's
 *     shape signature is unchanged; on the legacy default stream it runs directly.
 *   OQR_BATCHED_TC, OQR_BATCHED_TC2_FIRST, OQR_BATCHED_SHIFTED_TC: the
 *     tensor-core form (oqr_batched_mixed) with every instance's program
 *     OQR_BATCH_CHOLQR2_TC, OQR_BATCH_CHOLQR2_TC2 or OQR_BATCH_SCHOLQR3_TC;
 *     opts->batch_orth, when given, receives each instance's check.
 *   OQR_BATCHED_SELECTOR: the learned selector (no counterpart in the paper).
 *     Every instance first runs one FP64-accurate pass on the tensor cores
 *     (its Gram G_0 = Z^T A Z and Cholesky factor R_1); 16 features of G_0 and
 *     R_1 (Gram diagonal spread, coherence and pivots of the diagonally scaled
 *     G_0, breakdown, a sketched estimate of kappa(R_1) from an n x 2n Gaussian
 *     sketch, sizes) go through the MLP 16 -> 64 -> 64 -> 4 (opts->
 *     selector_params, BF16 inference), whose argmax says how the instance
 *     finishes: unshifted (options 0 and 1), 2 with a shifted first pass
 *     refactored from the same G_0 and two more passes (shifted A-CholQR3),
 *     3 with FP64 A-CholQR2.  Options 0 and 1 share the Gram of pass 1,
 *     G_1 = Q_1^T A Q_1 with Q_1 = Z R_1^{-1}, which decides on the device:
 *     ||G_1 - I||_F <= opts->selector_tol keeps Q_1 (one pass, checked);
 *     <= 0.5 factors G_1 once more (A-CholQR2: within 0.5 of I the last pass
 *     leaves the orthogonality at rounding level); larger, or a breakdown,
 *     redoes the instance as shifted A-CholQR3 from the saved G_0 in the same
 *     wave.  Every wave is one fixed sequence of launches over its packed
 *     instances (each takes part in the Gram passes its route needs), reading
 *     the wave's one split of A; no host round trip sits between the passes.
 *     A breakdown, or the network's choice 3, ends with FP64 A-CholQR2 after
 *     the waves (accepted once it completes).  opts->batch_orth and
 *     opts->batch_choice, when given, receive the checks and the option each
 *     result comes from (2 for a shifted refactor).  This mode synchronizes
 *     the stream once, after the waves.
 * Argument errors are returned; otherwise every mode but the selector returns
 * after enqueueing.
 */
typedef enum {
    OQR_BATCHED_FP64 = 0,
    OQR_BATCHED_TC = 1,
    OQR_BATCHED_TC2_FIRST = 2,
    OQR_BATCHED_SHIFTED_TC = 3,
    OQR_BATCHED_SELECTOR = 4
} oqr_batched_mode;

oqr_status oqr_batched(oqr_ctx* ctx, int count, const int* m, const int* n, const double* const* A, const long* lda,
                       const double* const* Z, const long* ldz, double* const* Q, const long* ldq, double* const* R,
                       const long* ldr, int mode, const oqr_opts* opts, int* status, void* stream);

/*
 * oqr_batched_features: the selector's 16 features of each instance (device,
 * count x 16 floats, row-major, in the callers' instance order) after the
 * first FP64-accurate pass that OQR_BATCHED_SELECTOR runs, without the rest:
 * the training inputs of the selector's network.  Same instance limits as
 * oqr_batched.  Synchronizes the stream.
 */
oqr_status oqr_batched_features(oqr_ctx* ctx, int count, const int* m, const int* n, const double* const* A,
                                const long* lda, const double* const* Z, const long* ldz, float* feat, void* stream);

/* Per-instance programs of the batched tensor-core path. */
typedef enum {
    OQR_BATCH_CHOLQR_TC = 0,    /* Algorithm 1 once (CHOLQR), FP64_TC Gram */
    OQR_BATCH_CHOLQR2_TC2 = 1,  /* A-CholQR2: TC2 pass, then FP64_TC pass */
    OQR_BATCH_CHOLQR2_TC = 2,   /* A-CholQR2: two FP64_TC passes */
    OQR_BATCH_SCHOLQR3_TC = 3   /* shifted A-CholQR3: FP64_TC pass on G + sI, then two FP64_TC passes;
                                   s = 11 u (m n + n (n + 1)) ||A||_F ||Z||_F^2, u = 2^-53 */
} oqr_batch_program;

/*
 * Batched oblique QR on the tensor cores: the same instances, arguments and
 * status words as oqr_batched, each instance running its own program
 * (program[b], host array; NULL = all OQR_BATCH_CHOLQR2_TC): Algorithm 1
 * repeated 1 to 3 times (Sec. 2), every Gram G = Z^T A Z formed on the BF16
 * tensor cores (OQR_TC2 or OQR_FP64_TC), and the Cholesky factors,
 * Q = Z R^{-1} and R = R_p ... R_1 in FP64.  An instance's results do not
 * depend on the other instances of the batch.  Instances run in waves
 * (largest m first) whose BF16 slice planes (14 bytes per element of A, Z
 * and Z^T A) fit 16 GiB of workspace (oqr_set_batch_budget); A is split once
 * per wave and read by every pass.  orth (device, count doubles, may be NULL): when given, each
 * instance's result is checked, orth[b] = an estimate of ||Q_b^T A_b Q_b - I||_2
 * (Sec. 7's orthogonality measure; power iteration, a lower bound) from one
 * more FP64_TC Gram of the final Q, or +inf after a breakdown.
 * status[b] = -1 for every instance when a tensor-core wait timed out (the
 * context's status then reports OQR_ERR_TIMEOUT).  Q may alias Z (each row is
 * solved in place).  The sequence is captured into one CUDA graph, cached
 * while every instance's (m, n, program), the status and orth addresses and
 * the wave budget are unchanged (on the legacy default stream it runs
 * directly).  Asynchronous: returns after enqueueing (argument errors,
 * including a program outside the enum, are returned).
 */
oqr_status oqr_batched_mixed(oqr_ctx* ctx, int count, const int* m, const int* n, const double* const* A,
                             const long* lda, const double* const* Z, const long* ldz, double* const* Q,
                             const long* ldq, double* const* R, const long* ldr, const int* program, int* status,
                             double* orth, void* stream);

/* The slice-plane bytes per wave of the tensor-core batches (oqr_batched_mixed;
 * 0 restores the default of 16 GiB).  A wave always holds at least one
 * instance, so a small budget gives one instance per wave.  Results do not
 * depend on it; memory and the number of launches do. */
oqr_status oqr_set_batch_budget(oqr_ctx* ctx, size_t bytes);

/* The built-in work plan of oqr_batched for one instance (splits of its Gram). */
int oqr_batched_default_splits(int m, int n);

/*
 * Selector (no counterpart in the paper: it chooses, per instance, the passes
 * and precisions of the normal-equation method).
 *
 * oqr_features: 16 floats (device, feat) describing one instance, read from its
 *   BF16X3 normal-equation matrix and the norms of A and Z (Gram diagonal
 *   spread, coherence, pivots of the diagonally scaled Cholesky and its
 *   breakdown column, sizes).  n <= 1024.
 * oqr_mlp_forward: logits (device, B x 4, may be NULL) and argmax choice
 *   (device, B ints, may be NULL) of the MLP 16 -> 64 -> 64 -> 4 (ReLU) for
 *   B feature rows X (device, B x 16, row-major); params (device) is the flat
 *   FP32 array of oqr_mlp_param_count() floats: W1[64][16], b1[64],
 *   W2[64][64], b2[64], W3[4][64], b3[4].  bf16 = 1 rounds weights and
 *   activations to BF16 (FP32 accumulation).
 * oqr_mlp_grad: the gradient (device, param_count floats) of the mean softmax
 *   cross-entropy over the B rows with integer labels y (device) and, if loss
 *   is non-NULL, the loss (device, 1 float).  Deterministic (fixed summation
 *   order).  Scratch comes from the context's workspace.
 * oqr_mlp_adam: one Adam step on params with moments m, v (device), step t >= 1.
 */
oqr_status oqr_features(oqr_ctx* ctx, int m, int n, const double* A, long lda, const double* Z, long ldz, float* feat,
                        void* stream);
int oqr_mlp_param_count(void);
oqr_status oqr_mlp_forward(oqr_ctx* ctx, int B, const float* X, const float* params, int bf16, float* logits,
                           int* choice, void* stream);
oqr_status oqr_mlp_grad(oqr_ctx* ctx, int B, const float* X, const int* y, const float* params, float* grad,
                        float* loss, void* stream);
oqr_status oqr_mlp_adam(oqr_ctx* ctx, float* params, const float* grad, float* m, float* v, float lr, float beta1,
                        float beta2, float eps, int t, void* stream);

/*
 * Measurement helper (no counterpart in the paper): runs oqr_gram's pipeline
 * for prec and returns the CUDA-event duration of each phase on `stream`, in
 * milliseconds, in phase_ms[0..*nphase).  OQR_FP64: {Gram kernel, reduction}.
 * OQR_BF16X3 / OQR_FP64_TC: {split of A and Z, U = M Z product, its reduction
 * and the split of U, C = Z^T U product, its reduction and G = C + C^T}.
 * phase_ms holds at least 6 floats.  Synchronizes the stream.
 */
oqr_status oqr_gram_phases(oqr_ctx* ctx, int m, int n, const double* A, long lda, const double* Z, long ldz,
                           double* G, long ldg, int prec, float* phase_ms, int* nphase, void* stream);

/*
 * oqr_gram_noalloc: the same G = Z^T A Z as oqr_gram (FP64), for callers that
 *   cannot allocate device memory (a plug-in under another framework's caching
 *   allocator that owns the memory; real-time or embedded hosts that fix their
 *   memory at start-up).  The paper has no counterpart: this is a
 *   deployment variant of the step kernel.  It takes no context and allocates
 *   nothing: its scratch (split-K partials and a status word) is one
 *   file-scope device array of 8 MiB + 256 B that every GPU loading the
 *   library holds until the process exits.  A, Z, G are caller-owned device
 *   memory on the current device; A is read from its lower triangle.
 *   Limits: n <= 1024 (n above that returns OQR_ERR_UNSUPPORTED); the
 *   partial count is capped at floor(8 MiB / (8 n^2)), so large n runs on
 *   fewer CTAs than oqr_gram: for n > 724 one partial, i.e. ceil(n / 64)
 *   CTAs (16 at n = 1024).  The first call on a device looks up the array's
 *   device address and should come before any stream capture on that
 *   device; cudaDeviceReset after it is not supported.  All calls share the
 *   array: calls that overlap on the GPU race.  There is no context to hold
 *   a device-side outcome, so when a time-limited wait of the kernel gives up
 *   every element of G is set to NaN.
 */
oqr_status oqr_gram_noalloc(int m, int n, const double* A, long lda, const double* Z, long ldz, double* G,
                            long ldg, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* OQR_H */
