// Internal declarations of the oblique-QR CUDA library (sm_103a).
// Shared by the kernel translation units and the C-ABI layer; never exported.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/oqr.h"

namespace oqr {

// ------------------------------------------------------------------ status --
// Device status block, one per context (in its workspace):
//   code  : first error raised by a kernel (oqr_status), 0 = none
//   info  : 1-based Cholesky breakdown column, or a kernel-specific detail
//   where : which kernel timed out or broke down (small integer tag)
struct DevStatus {
    int code;
    int info;
    int where;
    int pad;
    double shift;       // shift applied by the last shifted pass
    double normA_fro;   // ||A||_F of the last shifted pass
    double normZ_fro2;  // ||Z||_F^2 of the last shifted pass
    double orth2;       // ||Q^T A Q - I||_2 estimate from the last check
    double orthF;       // ||Q^T A Q - I||_F from the last check
    double pad2[5];
};
static_assert(sizeof(DevStatus) == 96, "status layout");

enum KernelTag { TAG_GRAM = 1, TAG_POTRF = 2, TAG_TRSM = 3, TAG_GEMM = 4, TAG_CHECK = 5, TAG_MIXED = 6,
                 TAG_BATCH = 7, TAG_DIAG = 8 };

// A device-side branch between two enqueued alternatives: a gated launch does nothing (every block returns
// at once) unless *gate == want; a NULL gate always runs.
__device__ __forceinline__ bool gated_off(const int* gate, int want)
{
    return gate != nullptr && *(volatile const int*)gate != want;
}

__device__ inline void raise_status(DevStatus* st, int code, int info, int where)
{
    if (atomicCAS(&st->code, 0, code) == 0) {
        st->info = info;
        st->where = where;
    }
}

__device__ inline uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Barrier over the whole (cooperative) grid: count arrivals, the last one resets the count and advances the
// generation; the others wait for the generation to change, giving up when the status word is set (every
// block then returns) or after limit_ns (OQR_ERR_TIMEOUT with the given tag).  Returns false if the grid
// must stop.  Data written before the barrier by other blocks is read after it through L2 (__ldcg).
__device__ inline bool grid_barrier(unsigned* count, unsigned* gen, uint64_t limit_ns, DevStatus* st, int* ok_s,
                                    int tag)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* vg = gen;
        const unsigned g = *vg;
        __threadfence();
        bool ok = *(volatile int*)&st->code == 0;
        if (atomicAdd(count, 1u) == gridDim.x - 1) {
            *(volatile unsigned*)count = 0;
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            const uint64_t t0 = global_ns();
            while (ok && *vg == g) {
                if (*(volatile int*)&st->code != 0) ok = false;
                else if (global_ns() - t0 > limit_ns) {
                    raise_status(st, OQR_ERR_TIMEOUT, 0, tag);
                    ok = false;
                }
            }
        }
        __threadfence();
        *ok_s = ok ? 1 : 0;
    }
    __syncthreads();
    return *ok_s != 0;
}

__device__ inline uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---------------------------------------------------------------- mbarrier --
__device__ inline void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ inline void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ inline void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ inline bool mbar_test(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the phase with the given parity to complete, for at most
// limit_ns nanoseconds of wall time.  Returns false on timeout.
__device__ inline bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns)
{
    if (mbar_test(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_test(bar, parity)) {
        if (global_ns() - t0 > limit_ns) return false;
    }
    return true;
}

// Bound of the waits on a kernel's exit path, for bulk copies or MMAs that may
// still be in flight after an abort.  Their shared or tensor memory must not be
// released (by the CTA's exit, or by tcgen05.dealloc) while the hardware can
// still write or read it, so these waits never give up sooner than
// EXIT_DRAIN_NS, however small the caller's spin_limit: a copy or MMA that was
// issued completes in microseconds unless the GPU itself has stopped.
constexpr uint64_t EXIT_DRAIN_NS = 2000000000ull;
__host__ __device__ inline uint64_t exit_drain_ns(uint64_t limit_ns)
{
    return limit_ns > EXIT_DRAIN_NS ? limit_ns : EXIT_DRAIN_NS;
}

__device__ inline void fence_barrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ inline void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// -------------------------------------------------------------------- TMA --
// 2-D tiled bulk tensor load into shared memory, completion signalled on bar.
__device__ inline void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cta.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ inline void tma_prefetch_desc(const CUtensorMap* map)
{
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// ---------------------------------------------------------- host helpers --
// Builds a 2-D tensor map over a column-major matrix (rows contiguous).
// Returns false when the driver refuses it (alignment, stride) or is absent.
bool make_tensor_map_2d(CUtensorMap* map, CUtensorMapDataType dtype, int elem_bytes, const void* base,
                        long rows, long cols, long ld, int box_rows, int box_cols);

// True when a column-major matrix can be read by TMA: 16-byte aligned base and
// a leading dimension whose byte stride is a multiple of 16.
inline bool tma_ok(const void* p, long ld, int elem_bytes)
{
    return (reinterpret_cast<uintptr_t>(p) % 16 == 0) && ((ld * elem_bytes) % 16 == 0);
}

// ---------------------------------------------------- kernel entry points --
// Fused symmetric Gram, FP64: P_s = Z^T (M Z) restricted to split s, with
// M = tril(A,-1) + diag(A)/2; see k_gram_f64.cu.
struct GramPlan {
    int m, n;
    int bn;        // column chunk width
    int chunks;    // ceil(n / bn)
    int splits;    // work splits of the lower triangle
    long steps;    // total k-steps over the lower triangle (per chunk)
};
GramPlan gram_plan(int m, int n, int sm_count);
size_t gram_partials_bytes(const GramPlan& p);
cudaError_t launch_gram_f64(const GramPlan& p, const double* A, long lda, const double* Z, long ldz,
                            double* partials, DevStatus* st, uint64_t limit_ns, cudaStream_t s);
// G = sum_s (P_s + P_s^T) (+ shift*I if shift_ptr), G dense n x n with ldg.
cudaError_t launch_gram_reduce(const GramPlan& p, const double* partials, double* G, long ldg,
                               const double* shift_ptr, DevStatus* st, cudaStream_t s);

// Dense small kernels (k_dense.cu).
cudaError_t launch_potrf(int n, const double* G, long ldg, double* R, long ldr, const double* shift_ptr,
                         DevStatus* st, cudaStream_t s);
cudaError_t launch_trsm(int m, int n, const double* Z, long ldz, const double* R, long ldr, double* Q, long ldq,
                        DevStatus* st, cudaStream_t s, const int* gate = nullptr, int want = 0);
// One 64-column block of the blocked TRSM: Q(:, jb:jb+bw) = (Z(:, jb:jb+bw) - U) R_bb^{-1}.
cudaError_t launch_trsm_block(int m, int jb, int bw, const double* Z, long ldz, const double* U, long ldu,
                              const double* R, long ldr, double* Q, long ldq, DevStatus* st, cudaStream_t s,
                              const int* gate = nullptr, int want = 0);
cudaError_t launch_rprod(int n, const double* U, long ldu, const double* S, long lds, double* R, long ldr,
                         cudaStream_t s);
cudaError_t launch_copy_upper(int n, const double* S, long lds, double* D, long ldd, cudaStream_t s);
// D (cols x rows) = S^T (S rows x cols).
cudaError_t launch_transpose(int rows, int cols, const double* S, long lds, double* D, long ldd, cudaStream_t s);
// X = R^{-1} (upper triangular, n x n, n <= TRINV_MAX_N), FP64 column-oriented back substitution.
constexpr int TRINV_MAX_N = 8192;
cudaError_t launch_trinv(int n, const double* R, long ldr, double* X, long ldx, const DevStatus* st, cudaStream_t s);
// out[0] = ||G - I||_F (out holds GRAM_DEFECT_DOUBLES doubles: the result, then the blocks' partial sums);
// gate[0] = 1 if ||G - I||_F <= gate_tol, else 0 (also for a NaN).
constexpr int GRAM_DEFECT_DOUBLES = 1 + 64;
cudaError_t launch_gram_defect(int n, const double* G, long ldg, double* out, int* gate, double gate_tol,
                               cudaStream_t s);
// Shift for the shifted pass: s = c * u * (m n + n (n+1)) * ||A||_F * ||Z||_F^2.
cudaError_t launch_norms_and_shift(int m, int n, const double* A, long lda, const double* Z, long ldz,
                                   double c, double u, double* scratch, int scratch_len, DevStatus* st,
                                   cudaStream_t s);
// Orthogonality check: E = G - I given G (n x n); writes E (if non-NULL),
// orth2 (power-iteration estimate of ||E||_2) and orthF into st.  work holds
// n*n + 2n doubles.
// A device-side wait that nothing completes, limited to limit_ns; records
// OQR_ERR_TIMEOUT (the timeout path, with nothing asynchronous in flight).
cudaError_t launch_timeout_probe(DevStatus* st, uint64_t limit_ns, cudaStream_t s);
// out[0] = lambda_max(S) estimate (power iteration), out[1] = trace(S), for
// symmetric positive semidefinite S (n x n); work: 2 n doubles.
cudaError_t launch_lambda_max(int n, const double* S, long lds, double* work, double* out, cudaStream_t s);
cudaError_t launch_check_finish(int n, const double* G, long ldg, double* E, long lde, double* work,
                                DevStatus* st, cudaStream_t s);

// Generic FP64 GEMM used by CGS2: C = beta*C + alpha * op(A) * B with
// op(A) = A (m x k), A^T (A stored k x m), or the symmetric matrix stored in
// the lower triangle of A (m x m).
enum GemmOp { GEMM_N = 0, GEMM_T = 1, GEMM_SYML = 2 };
size_t gemm_splitk_bytes(int M, int N, int splits);
cudaError_t launch_gemm_f64(GemmOp op, int M, int N, int K, double alpha, const double* A, long lda,
                            const double* B, long ldb, double beta, double* C, long ldc, double* splitk_ws,
                            int splits, cudaStream_t s);

// Tensor-core normal-equation matrix (k_tc.cu): G = Z^T A Z from BF16 (or
// E4M3) slices of the FP64 operands.
struct TcPlan {
    int m, n;
    int mode;       // 0 BF16X3, 1 FP64-accurate emulation, 2 FP8 E4M3, 3 TC2 (two leading emulation slices)
    int es;         // bytes per plane element
    int S;          // slices per operand used by the products
    int SA;         // slices of A made and kept in the workspace (>= S; 7 when shared with mode 1)
    int N;          // UMMA N (column chunk)
    long ldp;       // leading dimension of the slice planes
    int kch;        // exponent chunks of the contraction (256 long; 128 for FP8)
    int nitems_max; // work items of the larger of the two products
    int noA;        // 1: no planes of A (only C = X^T U; launch_tc_cross)
};
TcPlan tc_plan(int m, int n, int mode, int sa = 0, bool no_a = false);
size_t tc_plan_bytes(const TcPlan& p);
size_t tc_workspace_bytes(const TcPlan& p);
// The split of A made chunk by chunk (host-buffer path: each 256-column chunk as it arrives).
cudaError_t tc_split_a_begin(const TcPlan& p, void* ws, cudaStream_t s);
cudaError_t tc_split_a_chunk(const TcPlan& p, const double* A, long lda, int kc, void* ws, cudaStream_t s);
cudaError_t launch_tc_gram(const TcPlan& p, const double* A, long lda, const double* Z, long ldz, double* G, long ldg,
                           const double* shift_ptr, void* ws, DevStatus* st, uint64_t limit_ns, int sms,
                           cudaStream_t s, cudaEvent_t* ev = nullptr, bool a_ready = false);

// G = C + C^T (+ shift) with C = X^T U on the tensor cores, U = M X formed by
// the caller (FP64, m x n); p from tc_plan(m, n, mode, 0, true).
cudaError_t launch_tc_cross(const TcPlan& p, const double* X, long ldx, const double* U, long ldu, double* G, long ldg,
                            const double* shift_ptr, void* ws, DevStatus* st, uint64_t limit_ns, int sms,
                            cudaStream_t s);

// C = X^T Y (n1 x n2, leading dimension ldc) for X (K x n1) and Y (K x n2), FP64-accurate on the tensor
// cores (the EMU64 slices); ws holds tc_xty_bytes(K, n1, n2) bytes.
size_t tc_xty_bytes(int K, int n1, int n2);
// gate/want: see gated_off (every launch of the product is gated).
cudaError_t launch_tc_xty(int K, int n1, int n2, const double* X, long ldx, const double* Y, long ldy, double* C,
                          long ldc, void* ws, DevStatus* st, uint64_t limit_ns, int sms, cudaStream_t s,
                          const int* gate = nullptr, int want = 0);

// Euclidean Householder QR of a tall-skinny Z on a reduction tree (k_tsqr.cu):
// Z = Y S with Y (m x n) orthonormal and S upper triangular with a positive
// diagonal; the workspace holds tsqr_plan(m, n).doubles doubles.
struct TsqrPlan {
    int m, n;
    int b0;               // rows per leaf (the last leaf takes the rest: b0 <= rows < 2 b0)
    int leaves, levels;
    int level_count[32];  // nodes per tree level (each node stacks 2 children's R, or 3 for the last of an odd count)
    size_t doubles;       // workspace
};
TsqrPlan tsqr_plan(int m, int n);
cudaError_t launch_tsqr(const TsqrPlan& p, const double* Z, long ldz, double* Y, long ldy, double* S, long lds,
                        double* ws, cudaStream_t s);

// Blocked Householder QR of a tall-skinny Z (k_bhqr.cu), the same contract as launch_tsqr: Z = Y S, Y
// orthonormal, S upper triangular with a positive diagonal.  Panels of BH_B columns are factored column
// by column over all SMs, blocked as I - V T V^T, the trailing columns and Y updated with the
// products V^T X and V (T^T W) FP64-accurate on the tensor cores; the workspace holds
// bhqr_plan(m, n, sms).doubles doubles.
constexpr int BH_B = 32;
struct BhqrPlan {
    int m, n, panels, sms, blocks_max;
    int smem_rows;  // rows per block that the shared-memory panel kernel can hold
    size_t oX, oV, oT, oD, oW, oW2, oG, oBeta, oTau, oPart, oDpart, oBar, oXj, oXT, oVt, oPt;  // offsets (doubles)
    size_t doubles;
};
BhqrPlan bhqr_plan(int m, int n, int sms);
// The panel kernel's grid barriers wait at most limit_ns; past it the status st is raised (OQR_ERR_TIMEOUT)
// and the factorization's results are not to be used.
cudaError_t launch_bhqr(const BhqrPlan& p, const double* Z, long ldz, double* Y, long ldy, double* S, long lds,
                        double* ws, DevStatus* st, uint64_t limit_ns, cudaStream_t s);

// Tridiagonal A (k_tridiag.cu): d (m), e (m - 1); U = M X with M = tril(T, -1) + diag(T) / 2.
cudaError_t launch_tridiag_u(int m, int n, const double* d, const double* e, const double* X, long ldx, double* U,
                             long ldu, cudaStream_t s);
cudaError_t launch_tridiag_norms_and_shift(int m, int n, const double* d, const double* e, const double* X, long ldx,
                                           double c, double u, double* scratch, int scratch_len, DevStatus* st,
                                           cudaStream_t s);
// G = C + C^T (+ shift I), n x n (FP64).
cudaError_t launch_sym_plus_transpose(int n, const double* C, long ldc, double* G, long ldg, const double* shift_ptr,
                                      const DevStatus* st, cudaStream_t s);

// Blocked TRSM Q = Z / R with FP64-accurate tensor-core products for the
// off-diagonal blocks and FP64 substitution for the 64 x 64 diagonal blocks
// (k_tc.cu).  ws holds trsm_tc_workspace_bytes(m, n).
size_t trsm_tc_workspace_bytes(int m, int n);
cudaError_t launch_trsm_tc(int m, int n, const double* Z, long ldz, const double* R, long ldr, double* Q, long ldq,
                           void* ws, DevStatus* st, uint64_t limit_ns, int sms, cudaStream_t s,
                           const int* gate = nullptr, int want = 0);

// Batched A-CholQR2 (k_batched.cu): one descriptor per instance, n <= 64, m <= 4096.
constexpr int BATCH_MAX_N = 64;
constexpr int BATCH_MAX_M = 4096;
struct BatchDesc {
    const double* A;
    const double* Z;
    double* Q;
    double* R;
    long lda, ldz, ldq, ldr;
    int m, n;
    int splits;     // Gram work splits (the plan)
    int npass;      // normal-equation passes of this instance (the FP64 path: 2)
    double* partials;  // splits x n x n
    double* G;         // n x n
    double* R1;        // n x n
    double* R2;        // n x n
    double* G0;        // n x n: the first pass's Gram, kept by the selector for a later shifted refactor
};
cudaError_t launch_batched_cholqr2(const BatchDesc* d, int count, const int* const* cls_idx, const int* cls_count,
                                   const int* cls_max_splits, int max_n, int* status, cudaStream_t s);
// Pieces of the batched sequence over a sub-range of BatchDesc (k_batched.cu);
// instances whose npass <= pass sit the pass out:
//   factor: G_b = P_b + P_b^T from one partial (splits = 1), + shifts[b] I in
//           pass 0 (shifts may be NULL), R = chol(G_b) (R1 for pass 0, R2
//           later), Q_b = X_b / R (X = Z in pass 0, Q in place later), and for
//           pass > 0 R1 <- R2 R1;
//   rfinal: the caller's R_b = R1;
//   shifts: shifts[b] = c u (m n + n (n + 1)) ||A_b||_F ||Z_b||_F^2 where
//           mask[b], else 0, with ||A_b||_F^2 = anorm2[b], ||Z_b||_F^2 = znorm2[b] (from the splits);
//   scatter: status[perm[i]] = st_sorted[i], or -1 for every instance when a
//           tensor-core wait of the context timed out.
cudaError_t launch_batched_factor(const BatchDesc* d, int count, int* status, int pass, const double* shifts,
                                  cudaStream_t s);
cudaError_t launch_batched_rfinal(const BatchDesc* d, int count, int* status, cudaStream_t s);
// R1 = chol(G) for the instances with chol_mask[b] != 0, then Q = Z / R1 for those with solve_mask[b] != 0
// (a first pass from a new G; NULL masks: every instance).
cudaError_t launch_batched_chol_solve(const BatchDesc* d, int count, int* status, const int* chol_mask,
                                      const int* solve_mask, cudaStream_t s);
cudaError_t launch_batched_shifts(const BatchDesc* d, int count, const int* mask, const double* anorm2,
                                  const double* znorm2, double c, double u, double* shifts, cudaStream_t s);
cudaError_t launch_batch_status_scatter(const int* st_sorted, const int* perm, int count, const DevStatus* st,
                                        int* status, cudaStream_t s);
// The check of the instances whose factor passes end at pass (npass == pass):
// E = P + P^T - I from the partial of Q^T A Q, orth[b] = an estimate of
// ||E||_2 (power iteration, a lower bound); orth[b] = inf after a breakdown.
cudaError_t launch_batched_check(const BatchDesc* d, int count, const int* status, int pass, double* orth,
                                 cudaStream_t s);
// Pass 0's G = P + P^T and R1 = chol(G) only (no solve; the selector's features of a batch).
cudaError_t launch_batched_gram_chol(const BatchDesc* d, int count, int* status, cudaStream_t s);
// Rows of width floats: out[perm[i]] = in[i].
cudaError_t launch_batch_scatter_rows_f32(const float* in, const int* perm, int count, int width, float* out,
                                          cudaStream_t s);
// The selector's 16 features of each instance of a batch after its first FP64-accurate pass (k_features.cu).
// wtab: the sketches W_n of every n <= BATCH_MAX_N (launch_sketch_table, SKETCH_TABLE_DOUBLES doubles).
cudaError_t launch_features_batched(const BatchDesc* d, int count, const int* status, const double* wtab, float* feat,
                                    cudaStream_t s);
constexpr long SKETCH_TABLE_DOUBLES = (long)BATCH_MAX_N * (BATCH_MAX_N + 1) * (2 * BATCH_MAX_N + 1) / 3;
cudaError_t launch_sketch_table(double* tab, cudaStream_t s);
// defect[b] = ||Q^T A Q - I||_2 estimate of the Gram that instance b's last factor pass factors (the
// instances with 2 or more passes whose last factor pass is pass), read from that Gram's partial before the
// factor; a free check of the result: the last pass leaves orthogonality at rounding level when it is small.
cudaError_t launch_batched_last_defect(const BatchDesc* d, int count, const int* status, int pass, double* defect,
                                       cudaStream_t s);
// out[perm[i]] = in[i] (count doubles).
cudaError_t launch_batch_scatter_f64(const double* in, const int* perm, int count, double* out, cudaStream_t s);

// The learned selector's decisions on the device (k_select.cu), over a wave of count instances.
// Routes: SEL_R_PLAIN (unshifted passes), SEL_R_SHIFT (shifted A-CholQR3 from the probe's Gram), SEL_R_FP64
// (FP64 A-CholQR2 after the waves), SEL_R_LATE (an unshifted result that failed: shifted A-CholQR3 redone
// from the saved probe Gram G0).  Options reported: SEL_ONE, SEL_TWO, SEL_SHIFTED, SEL_FP64.
// gpass[b]: the Gram passes instance b takes part in (the tensor-core launches skip the others);
// BatchDesc.npass: its factor passes.  Status -3 (transient): the instance skips this pass's factor for
// its late refactor.
constexpr int SEL_R_PLAIN = 0, SEL_R_SHIFT = 1, SEL_R_FP64 = 2, SEL_R_LATE = 3;
constexpr int SEL_ONE = 0, SEL_TWO = 1, SEL_SHIFTED = 2, SEL_FP64 = 3;
constexpr int SEL_ST_LATE = -3;
struct SelWave {
    BatchDesc* d;   // count descriptors (npass updated on the device)
    int* status;
    int* route;
    int* opt;       // the option used
    int* gpass;
    int* mask;      // scratch: shifted first pass or late refactor
    double* anorm2; // ||A_b||_F^2 (from the splits)
    double* znorm2; // ||Z_b||_F^2
    double* shifts;
    double* orth;   // ||E||_F of the checked Gram, NaN where not checked
    double* defect; // ||E||_F of the Gram that the last factor pass factored
    int count;
    int extra;      // 1: every result is checked with one more Gram
    double tol;
};
// After the probe's Gram, its Cholesky, the features and the network: routes, pass counts, G0, the mask
// of shifted first passes.
cudaError_t launch_sel_route(const SelWave& w, const int* choice, cudaStream_t s);
// After the Gram of pass p (p >= 1): ONE / TWO / LATE for plain instances at p = 1, the defect of the
// Gram that a shifted route's last factor pass factors (reported), the extra check's value.
cudaError_t launch_sel_decide(const SelWave& w, int pass, cudaStream_t s);
// After the factor of pass p: an instance whose factor failed takes part in no later Gram.
cudaError_t launch_sel_after_factor(const SelWave& w, int pass, cudaStream_t s);
// The late refactor: mask = late instances, status 0, G = G0 + shift I (shifts from launch_batched_shifts
// over the mask), then launch_batched_chol_solve over the mask.
cudaError_t launch_sel_late_mask(const SelWave& w, cudaStream_t s);
cudaError_t launch_sel_late_prep(const SelWave& w, cudaStream_t s);
// G += shift I for the instances of the mask (the shifted route's first factor, G holding G0).
cudaError_t launch_sel_shift_g(const SelWave& w, cudaStream_t s);

// Packed tensor-core batches (k_tc.cu).  Instances (sorted by m, largest
// first) are cut into waves whose slice planes fit a byte budget; a wave's A
// planes are stacked by rows and its Z and U planes by columns, so that one
// tensor map per operand and one persistent launch per product cover every
// instance of the wave.  A is split once per wave and read by both passes.
struct TcBatchShape {
    int m, n;
    int mode0;  // tensor-core mode of pass 0 (1: EMU64, 3: TC2); later passes are EMU64
    int npass;  // Gram passes: 1..3 normal-equation passes, + 1 when the result is checked (Q^T A Q)
};
constexpr int TC_BATCH_MAX_PASS = 5;
struct TcBatchIn {
    const double* A;
    long lda;
    const double* Z;
    long ldz;
    double* Q;
    long ldq;
    double* C;  // n x n product Z^T A Z's half (the BatchDesc partial), column-major
};
struct TcBatchLaunch {
    int mode;              // 1 EMU64, 3 TC2
    int ninst, nitems;
    int piece_k;           // k per work item
    int nrblk;             // blocks of the reduction
    size_t inst, item0, cum, rblk;  // byte offsets of the launch's tables
};
struct TcBatchWave {
    int first, count;     // instances [first, first + count) of the sorted order
    long rows, cols, ldp;  // packed rows (sum of m), packed columns (sum of n), plane row pitch
    int K, kch, tilesA, max_items, max_rblk;
    size_t splitA, splitZ, splitQ, splitU;  // SplitInst tables (byte offsets)
    size_t tileTab, colTab;                 // the A split's tiles, the packed columns' instances
    TcBatchLaunch u[TC_BATCH_MAX_PASS][2], c[TC_BATCH_MAX_PASS][2];  // [pass][launch]: pass 0 one per mode present
    int nl[TC_BATCH_MAX_PASS];
    int maxpass;
    long upool;  // U pool doubles
};
struct TcBatchPlan {
    std::vector<TcBatchWave> waves;
    size_t table_bytes = 0;    // device tables
    size_t scratch_bytes = 0;  // the largest wave's planes, exponents and slots
    long upool_doubles = 0;    // the largest wave's U pool
};
TcBatchPlan tc_batch_plan(const std::vector<TcBatchShape>& sh, size_t budget);
// Host image of the tables for the given device addresses (table, U pool).
void tc_batch_tables(const TcBatchPlan& p, const std::vector<TcBatchShape>& sh, const std::vector<TcBatchIn>& in,
                     const void* table_dev, double* upool, std::vector<char>& image);
// Wave w: the split of A (once), then the Gram of pass p into the C of each
// instance with npass > p (X = Z in pass 0, Q later).
// The split of A leaves each tile's share of ||A||_F^2 in the scratch, and pass 0's split of Z each
// chunk's and column's sum of squares; tc_batch_norms (after pass 0's Gram) sums them per instance in a
// fixed order: anorm2[i] = ||A_i||_F^2, znorm2[i] = ||Z_i||_F^2 for the wave's instance i.
cudaError_t tc_batch_split_a(const TcBatchPlan& p, int w, const void* table_dev, void* scratch, cudaStream_t s);
cudaError_t tc_batch_norms(const TcBatchPlan& p, int w, const void* table_dev, void* scratch, double* anorm2,
                           double* znorm2, cudaStream_t s);
// live (the wave's per-instance Gram pass counts on the device, or NULL): instances with live[i] <= pass
// sit the pass out, their tiles skipped, so that one set of tables serves passes chosen on the device.
cudaError_t tc_batch_gram(const TcBatchPlan& p, int w, int pass, const void* table_dev, void* scratch,
                          DevStatus* st, uint64_t limit_ns, int sms, cudaStream_t s, const int* live = nullptr);


// Selector (k_mlp.cu, k_features.cu).
constexpr int MLP_IN = 16, MLP_HIDDEN = 64, MLP_OUT = 4;
constexpr int MLP_PARAMS = MLP_HIDDEN * MLP_IN + MLP_HIDDEN + MLP_HIDDEN * MLP_HIDDEN + MLP_HIDDEN +
                           MLP_OUT * MLP_HIDDEN + MLP_OUT;
size_t mlp_scratch_bytes(int B);
cudaError_t launch_mlp_forward(int B, const float* X, const float* P, int bf16, float* logits, int* choice,
                               cudaStream_t s);
cudaError_t launch_mlp_grad(int B, const float* X, const int* y, const float* P, float* grad, float* loss, float* scr,
                            cudaStream_t s);
cudaError_t launch_adam(int n, float* P, const float* g, float* m, float* v, float lr, float b1, float b2, float eps,
                        int t, cudaStream_t s);
cudaError_t launch_features(int m, int n, const double* G, long ldg, double* work, const DevStatus* st, float* feat,
                            cudaStream_t s);
cudaError_t launch_trace_shift(int n, double* G, long ldg, double c, double u, DevStatus* st, cudaStream_t s);

// C = A B (m x k) for symmetric A read from its lower triangle (k_glls.cu): 64 x 64 tiles of the
// lower triangle, per-tile partials (symm_workspace_doubles(m, k) doubles), fixed-order sum.
size_t symm_workspace_doubles(int m, int k);
cudaError_t launch_symm(int m, int k, const double* A, long lda, const double* B, long ldb, double* C, long ldc,
                        double* part, int sms, cudaStream_t s);
// X = R^{-1} Y for upper triangular R (n x n) and k right-hand sides; X may alias Y.
cudaError_t launch_upper_solve(int n, int k, const double* R, long ldr, const double* Y, long ldy, double* X,
                               long ldx, cudaStream_t s);

// Y = alpha X + beta Y (M x N, column-major).
cudaError_t launch_axpby(int M, int N, double alpha, const double* X, long ldx, double beta, double* Y, long ldy,
                         cudaStream_t s);

}  // namespace oqr
