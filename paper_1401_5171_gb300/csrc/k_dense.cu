// Small dense FP64 kernels of the normal-equation path (Algorithm 1, lines
// 3-4, and the pass composition), the norms behind the shift, the
// orthogonality check, and the generic FP64 GEMM used by block A-CGS2.
// FP64 on GB300 issues about 2 FMAs per clock per SM; these kernels are
// sized so that their cost stays O(m n^2 + n^3) next to the m^2 n Gram.
#include <math.h>

#include "oqr_internal.cuh"

namespace oqr {
namespace {

// ------------------------------------------------------------- Cholesky ----
// R = chol(G + shift I), upper, G read from its lower triangle
// (Algorithm 1, line 3).  Right-looking, 32-column panels, one SM's FP64 rate
// being far too low for n^3/3 flops on a single CTA: per panel
//   potrf_diag  (1 CTA)   factor the 32 x 32 diagonal block in shared memory;
//   potrf_row   (a warp per column) solve the panel row R(p, c) <- D^{-T} R(p, c);
//   potrf_trail (tiles)   R(r, c) -= sum_k R(p_k, r) R(p_k, c) on the trailing
//                         upper triangle, 16 x 16 tiles.
// A pivot that is not positive (or NaN) stops the factorization: the status
// word records OQR_ERR_NOT_SPD with the 1-based column and every later launch
// returns at once.
constexpr int PNB = 32;

__global__ void potrf_init_kernel(int n, const double* __restrict__ G, long ldg, double* R, long ldr,
                                  const double* shift_ptr, const DevStatus* st)
{
    if (*(volatile const int*)&st->code != 0) return;
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long)n * n) return;
    const long i = e % n, j = e / n;
    double v = 0.0;
    if (i <= j) {
        v = G[j + i * ldg];
        if (i == j && shift_ptr) v += *shift_ptr;
    }
    R[i + j * ldr] = v;
}

// GB300's FP64 pipe holds a sub-partition for about 64 clocks per 32-lane FP64
// instruction, so the factorization's dependent pivot chain is costed in FP64
// warp-instructions: the kernels below keep them few and densely packed.
//
// Diagonal block of panel jb.  The pairs (r, c), 0 < r <= c < 32, are listed
// by decreasing r; at pivot step j the pairs still updated (r > j) are a
// prefix of that list, (31 - j)(32 - j)/2 long, so the update runs on densely
// packed threads.  The thread that owns (j+1, j+1) computes the next pivot's
// reciprocal right after updating it, so the division overlaps the rest of the
// update.  R's rows are written at the end (row r scaled by 1/sqrt(pivot r)).
constexpr int PAIRS = PNB * (PNB - 1) / 2;  // 496
__global__ void __launch_bounds__(512) potrf_diag_kernel(int n, int jb, double* R, long ldr, DevStatus* st)
{
    __shared__ double D[PNB][PNB + 1];
    __shared__ double pinv[2];
    __shared__ int bad;
    if (*(volatile int*)&st->code != 0) return;
    const int nb = min(PNB, n - jb);
    for (int e = threadIdx.x; e < PNB * PNB; e += blockDim.x) {
        const int i = e % PNB, j = e / PNB;
        D[i][j] = (i <= j && j < nb) ? R[(jb + i) + (long)(jb + j) * ldr] : (i == j ? 1.0 : 0.0);
    }
    // this thread's pair: index t in the list ordered by decreasing r, then increasing c
    const int t = threadIdx.x;
    int pr = 0, pc = 0;
    if (t < PAIRS) {
        int rem = t, r = PNB - 1;
        while (rem >= PNB - r) {
            rem -= PNB - r;
            --r;
        }
        pr = r;
        pc = r + rem;
    }
    if (t == 0) bad = 0;
    __syncthreads();
    if (t == 0) {
        const double p0 = D[0][0];
        if (!(p0 > 0.0)) bad = jb + 1;
        pinv[0] = 1.0 / p0;
    }
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        if (bad) {  // the same value in every thread: a uniform exit
            if (t == 0) raise_status(st, OQR_ERR_NOT_SPD, bad, TAG_POTRF);
            return;
        }
        const int active = (PNB - 1 - j) * (PNB - j) / 2;
        if (t < active) {  // pr > j
            const double v = D[pr][pc] - (D[j][pr] * pinv[j & 1]) * D[j][pc];
            D[pr][pc] = v;
            if (pr == j + 1 && pc == j + 1 && j + 1 < nb) {  // look-ahead: the next pivot is final now
                if (!(v > 0.0)) bad = jb + j + 2;
                pinv[(j + 1) & 1] = 1.0 / v;
            }
        }
        __syncthreads();
    }
    // R(block) rows: R[r][r] = sqrt(d_r), R[r][c] = D[r][c] / sqrt(d_r)
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        const int i = e % nb, c = e / nb;
        if (i > c) continue;
        const double sd = sqrt(D[i][i]);
        R[(jb + i) + (long)(jb + c) * ldr] = i == c ? sd : D[i][c] / sd;
    }
}

// Panel row: R(p, c) <- R(p, p)^{-T} R(p, c) for the trailing columns c.  One
// warp per column, lane i = row i: column-oriented substitution, x_i = b_i /
// d_i broadcast by a shuffle, then b_k -= R(i, k) x_i on lanes k > i (two FP64
// instructions per step); PROW_WARPS columns per CTA.
constexpr int PROW_WARPS = 4;
__global__ void __launch_bounds__(32 * PROW_WARPS) potrf_row_kernel(int n, int jb, double* R, long ldr,
                                                                    const DevStatus* st)
{
    __shared__ double D[PNB][PNB + 1];
    __shared__ double dinv[PNB];
    if (*(volatile const int*)&st->code != 0) return;
    const int nb = min(PNB, n - jb);
    for (int e = threadIdx.x; e < PNB * PNB; e += blockDim.x) {
        const int i = e % PNB, j = e / PNB;
        D[i][j] = (i <= j && i < nb && j < nb) ? R[(jb + i) + (long)(jb + j) * ldr] : 0.0;
    }
    __syncthreads();
    if (threadIdx.x < nb) dinv[threadIdx.x] = 1.0 / D[threadIdx.x][threadIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int c = jb + nb + blockIdx.x * PROW_WARPS + w;
    if (c >= n) return;  // a whole warp leaves together
    double* col = R + jb + (long)c * ldr;
    double b = lane < nb ? col[lane] : 0.0;
    for (int i = 0; i < nb; ++i) {
        const double x = __shfl_sync(0xffffffffu, b, i) * dinv[i];
        if (lane == i) b = x;
        else if (lane > i) b -= D[i][lane] * x;
    }
    if (lane < nb) col[lane] = b;
}

// Trailing update on TT x TT tiles (tr <= tc) of the upper triangle right of
// the panel: R(r, c) -= sum_k R(p_k, r) R(p_k, c); one thread per element.
constexpr int TT = 16;
__global__ void __launch_bounds__(TT * TT) potrf_trail_kernel(int n, int jb, double* R, long ldr,
                                                              const DevStatus* st)
{
    __shared__ double Pr[PNB][TT + 1];  // panel rows, tile's row columns
    __shared__ double Pc[PNB][TT + 1];  // panel rows, tile's columns
    if (*(volatile const int*)&st->code != 0) return;
    const int nb = min(PNB, n - jb);
    const int t0 = jb + nb;
    const int nt = (n - t0 + TT - 1) / TT;
    // blockIdx.x enumerates the upper-triangular tile pairs (tr <= tc)
    int tr = 0, rem = blockIdx.x;
    while (rem >= nt - tr) {
        rem -= nt - tr;
        ++tr;
    }
    const int tc = tr + rem;
    const int r0 = t0 + tr * TT, c0 = t0 + tc * TT;
    for (int e = threadIdx.x; e < PNB * TT; e += TT * TT) {
        const int k = e % PNB, j = e / PNB;
        Pr[k][j] = (k < nb && r0 + j < n) ? R[(jb + k) + (long)(r0 + j) * ldr] : 0.0;
        Pc[k][j] = (k < nb && c0 + j < n) ? R[(jb + k) + (long)(c0 + j) * ldr] : 0.0;
    }
    __syncthreads();
    const int i = threadIdx.x % TT, j = threadIdx.x / TT;
    const int r = r0 + i, c = c0 + j;
    if (r >= n || c >= n || r > c) return;
    double s0 = R[r + (long)c * ldr], s1 = 0.0;
    for (int k = 0; k + 1 < nb; k += 2) {
        s0 -= Pr[k][i] * Pc[k][j];
        s1 -= Pr[k + 1][i] * Pc[k + 1][j];
    }
    if (nb & 1) s0 -= Pr[nb - 1][i] * Pc[nb - 1][j];
    R[r + (long)c * ldr] = s0 + s1;
}

// ----------------------------------------------------------------- TRSM ----
// Q = Z / R (Algorithm 1, line 4): every row of Q solves q (R) = z.  A CTA
// holds ROWS rows of Z in shared memory and walks 32-column blocks: a GEMM
// update from the already solved columns, then substitution within the block
// against R's diagonal block.  In place when Q aliases Z.
constexpr int TRSM_THREADS = 256;
constexpr int TNB = 32;

__global__ void __launch_bounds__(TRSM_THREADS) trsm_kernel(int m, int n, int rows, const double* Z, long ldz,
                                                            const double* __restrict__ R, long ldr, double* Q,
                                                            long ldq, const DevStatus* st, const int* gate,
                                                            int want)
{
    extern __shared__ double ts[];
    if (*(volatile const int*)&st->code != 0 || gated_off(gate, want)) return;
    const int ldsm = n + 1;                         // padded row stride
    double* Zs = ts;                                // [rows][n+1]
    double* Rd = ts + (size_t)rows * ldsm;          // [TNB][TNB+1] diagonal block
    double* Rt = Rd + TNB * (TNB + 1);              // [TNB][TNB+1] off-diagonal tile
    const int tid = threadIdx.x;
    const long row0 = (long)blockIdx.x * rows;
    for (long e = tid; e < (long)rows * n; e += TRSM_THREADS) {
        const int r = (int)(e % rows), c = (int)(e / rows);
        const long gr = row0 + r;
        Zs[r * ldsm + c] = gr < m ? Z[gr + c * ldz] : 0.0;
    }
    const int j = tid & 31, rg = tid >> 5;  // update phase: column j of the block, rows rg + 8 t
    constexpr int RPT = 8;                  // rows per thread per pass (rows <= 64)
    for (int jb = 0; jb < n; jb += TNB) {
        const int nb = min(TNB, n - jb);
        double acc[RPT];
#pragma unroll
        for (int t = 0; t < RPT; ++t) acc[t] = 0.0;
        for (int k0 = 0; k0 < jb; k0 += TNB) {   // S(:, block) -= Q(:, k0:k0+32) R(k0:k0+32, block)
            __syncthreads();
            for (int e = tid; e < TNB * TNB; e += TRSM_THREADS) {
                const int k = e % TNB, c = e / TNB;
                Rt[k * (TNB + 1) + c] = (c < nb) ? R[(k0 + k) + (long)(jb + c) * ldr] : 0.0;
            }
            __syncthreads();
#pragma unroll
            for (int t = 0; t < RPT; ++t) {
                const int r = rg + 8 * t;
                if (r < rows) {
                    double s = 0.0;
                    const double* zr = Zs + r * ldsm + k0;
#pragma unroll 8
                    for (int k = 0; k < TNB; ++k) s = fma(zr[k], Rt[k * (TNB + 1) + j], s);
                    acc[t] += s;
                }
            }
        }
        __syncthreads();
        for (int e = tid; e < TNB * TNB; e += TRSM_THREADS) {
            const int i = e % TNB, c = e / TNB;
            Rd[i * (TNB + 1) + c] = (i < nb && c < nb) ? R[(jb + i) + (long)(jb + c) * ldr] : 0.0;
        }
        if (j < nb) {
#pragma unroll
            for (int t = 0; t < RPT; ++t) {
                const int r = rg + 8 * t;
                if (r < rows) Zs[r * ldsm + jb + j] -= acc[t];
            }
        }
        __syncthreads();
        for (int r = tid; r < rows; r += TRSM_THREADS) {
            double* zr = Zs + r * ldsm + jb;
            for (int c = 0; c < nb; ++c) {
                double t = zr[c];
                for (int k = 0; k < c; ++k) t -= zr[k] * Rd[k * (TNB + 1) + c];
                zr[c] = t / Rd[c * (TNB + 1) + c];
            }
        }
    }
    __syncthreads();
    for (long e = tid; e < (long)rows * n; e += TRSM_THREADS) {
        const int r = (int)(e % rows), c = (int)(e / rows);
        const long gr = row0 + r;
        if (gr < m) Q[gr + c * ldq] = Zs[r * ldsm + c];
    }
}

// ------------------------------------------------- TRSM, one column block ----
// Q(:, jb:jb+bw) = (Z(:, jb:jb+bw) - U) R(jb:jb+bw, jb:jb+bw)^{-1}, bw <= 64:
// row-wise substitution, one thread per row (column-oriented order with the
// reciprocals of the diagonal), the row's 64 values in registers.  U (m x bw,
// column-major) is the product of the already solved columns with
// R(0:jb, jb:jb+bw), formed elsewhere (NULL for the first block).  In place
// when Q aliases Z.
constexpr int TBW = 64;
constexpr int TB_THREADS = 32;  // one warp of rows per CTA: ~1000 CTAs spread the FP64 work evenly over the SMs
constexpr int TB_PACKED = TBW * (TBW + 1) / 2;
// The upper triangle of the diagonal block, packed row by row: (c, k), k >= c, at c TBW - c (c - 1) / 2 + k - c.
__host__ __device__ constexpr int tb_idx(int c, int k) { return c * TBW - c * (c - 1) / 2 + (k - c); }
__global__ void __launch_bounds__(TB_THREADS) trsm_block_kernel(int m, int jb, int bw, const double* Z, long ldz,
                                                                const double* __restrict__ U, long ldu,
                                                                const double* __restrict__ R, long ldr, double* Q,
                                                                long ldq, const DevStatus* st, const int* gate,
                                                                int want)
{
    __shared__ double D[TB_PACKED];
    __shared__ double dinv[TBW];
    if (*(volatile const int*)&st->code != 0 || gated_off(gate, want)) return;
    for (int c = 0; c < TBW; ++c)
        for (int k = c + threadIdx.x; k < TBW; k += TB_THREADS)
            D[tb_idx(c, k)] = k < bw ? R[(jb + c) + (long)(jb + k) * ldr] : 0.0;
    for (int c = threadIdx.x; c < TBW; c += TB_THREADS) dinv[c] = c < bw ? 1.0 / R[(jb + c) + (long)(jb + c) * ldr] : 0.0;
    __syncthreads();
    const long i = (long)blockIdx.x * TB_THREADS + threadIdx.x;
    if (i >= m) return;
    double b[TBW];
#pragma unroll
    for (int c = 0; c < TBW; ++c) {
        b[c] = 0.0;
        if (c < bw) b[c] = Z[i + (long)(jb + c) * ldz] - (U ? U[i + (long)c * ldu] : 0.0);
    }
#pragma unroll
    for (int c = 0; c < TBW; ++c) {
        if (c < bw) {
            asm volatile("" ::: "memory");  // keeps only row c of D live: no hoisted loads, no spills
            b[c] *= dinv[c];
#pragma unroll
            for (int k = c + 1; k < TBW; ++k) b[k] -= D[tb_idx(c, k)] * b[c];
        }
    }
#pragma unroll
    for (int c = 0; c < TBW; ++c)
        if (c < bw) Q[i + (long)(jb + c) * ldq] = b[c];
}

// ------------------------------------------------------------ R = U S ------
__global__ void rprod_kernel(int n, const double* __restrict__ U, long ldu, const double* __restrict__ S, long lds,
                             double* R, long ldr)
{
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long)n * n) return;
    const int i = (int)(e % n), j = (int)(e / n);
    double s = 0.0;
    if (i <= j)
        for (int k = i; k <= j; ++k) s += U[i + (long)k * ldu] * S[k + (long)j * lds];
    R[i + (long)j * ldr] = s;
}

// D (cols x rows, leading dimension ldd) = S^T for S (rows x cols, leading dimension lds): 32 x 32 tiles.
__global__ void transpose_kernel(int rows, int cols, const double* __restrict__ S, long lds, double* D, long ldd)
{
    __shared__ double t[32][33];
    const long r0 = (long)blockIdx.x * 32, c0 = (long)blockIdx.y * 32;
    {
        const long r = r0 + threadIdx.x, c = c0 + threadIdx.y;  // coalesced along S's rows
        t[threadIdx.y][threadIdx.x] = (r < rows && c < cols) ? S[r + c * lds] : 0.0;
    }
    __syncthreads();
    const long c = c0 + threadIdx.x, r = r0 + threadIdx.y;  // coalesced along D's rows (S's columns)
    if (r < rows && c < cols) D[c + r * ldd] = t[threadIdx.x][threadIdx.y];
}

// ||G - I||_F for a symmetric G (n x n) read from its lower triangle (an off-diagonal element counts twice),
// in two launches with a fixed summation order: block b sums the columns j = b (mod GD_BLOCKS) into
// part[b] (FP64 being about 2 FMAs per clock per SM, one block would take tens of microseconds), then one
// warp sums the parts, writes out[0] and gate[0] = (out[0] <= tol).
constexpr int GD_BLOCKS = 64, GD_THREADS = 256;
__global__ void __launch_bounds__(GD_THREADS) gram_defect_part_kernel(int n, const double* __restrict__ G, long ldg,
                                                                      double* part)
{
    __shared__ double red[GD_THREADS / 32];
    double a = 0.0;
    for (int j = blockIdx.x; j < n; j += GD_BLOCKS)
        for (int i = j + threadIdx.x; i < n; i += GD_THREADS) {
            const double v = G[i + (long)j * ldg] - (i == j ? 1.0 : 0.0);
            a = fma(i == j ? v : 2.0 * v, v, a);
        }
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < GD_THREADS / 32; ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

__global__ void gram_defect_sum_kernel(const double* __restrict__ part, double* out, int* gate, double tol)
{
    double v = part[threadIdx.x] + part[threadIdx.x + 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) {
        const double f = sqrt(v);
        out[0] = f;
        gate[0] = f <= tol ? 1 : 0;
    }
}

// X = R^{-1} for upper triangular R (n x n), one block per column j: x = R^{-1} e_j by column-oriented back
// substitution, x_i = x_i / r_ii (as a product with the reciprocal), then x_t -= x_i r_ti for t < i; column
// j costs j^2 / 2 FMAs and j block barriers, and the n columns run side by side.  Each thread keeps rows
// t + TI_THREADS k (k < RPT) and loads their elements of R's columns TI_AHEAD steps before use, so a step
// waits on a barrier, not on a load.  X's strict lower triangle is written with zeros.
constexpr int TI_THREADS = 256, TI_AHEAD = 8;
template <int RPT>
__global__ void __launch_bounds__(TI_THREADS) trinv_upper_kernel(int n, const double* __restrict__ R, long ldr,
                                                                 double* X, long ldx, const DevStatus* st)
{
    extern __shared__ double ti_sh[];  // x (n), then the diagonal's reciprocals (n)
    if (*(volatile const int*)&st->code != 0) return;
    const int j = blockIdx.x;
    double* x = ti_sh;
    double* dinv = ti_sh + n;
    for (int t = threadIdx.x; t <= j; t += TI_THREADS) {
        x[t] = t == j ? 1.0 : 0.0;
        dinv[t] = 1.0 / R[t + (long)t * ldr];
    }
    // ring[u][k]: R(row_k, i0 - u) for the TI_AHEAD steps from i0 down
    double ring[TI_AHEAD][RPT], next[TI_AHEAD][RPT];
    auto load = [&](double (&b)[TI_AHEAD][RPT], int i0) {
#pragma unroll
        for (int u = 0; u < TI_AHEAD; ++u)
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                const int row = threadIdx.x + k * TI_THREADS, col = i0 - u;
                b[u][k] = (col >= 0 && row < col) ? R[row + (long)col * ldr] : 0.0;
            }
    };
    load(ring, j);
    __syncthreads();
    for (int i0 = j; i0 >= 0; i0 -= TI_AHEAD) {
        load(next, i0 - TI_AHEAD);
#pragma unroll
        for (int u = 0; u < TI_AHEAD; ++u) {
            const int i = i0 - u;
            if (i < 0) break;  // uniform over the block
            if (threadIdx.x < i) {  // only the threads with rows above i spend FP64 work
                const double q = x[i] * dinv[i];
#pragma unroll
                for (int k = 0; k < RPT; ++k) {
                    const int row = threadIdx.x + k * TI_THREADS;
                    if (row < i) x[row] = fma(-q, ring[u][k], x[row]);
                }
            }
            __syncthreads();                               // every read of x[i] is done; x[0..i-1] updated
            if (threadIdx.x == 0) x[i] = x[i] * dinv[i];  // x[i] is read by no later step
        }
#pragma unroll
        for (int u = 0; u < TI_AHEAD; ++u)
#pragma unroll
            for (int k = 0; k < RPT; ++k) ring[u][k] = next[u][k];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < n; t += TI_THREADS) X[t + (long)j * ldx] = t <= j ? x[t] : 0.0;
}

__global__ void copy_upper_kernel(int n, const double* __restrict__ S, long lds, double* D, long ldd)
{
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long)n * n) return;
    const int i = (int)(e % n), j = (int)(e / n);
    D[i + (long)j * ldd] = i <= j ? S[i + (long)j * lds] : 0.0;
}

// ------------------------------------------------------ timeout probe ------
// One thread waits on an mbarrier that no thread arrives at, for limit_ns, then
// records OQR_ERR_TIMEOUT: the path every time-limited wait of the library takes,
// here with no copy or MMA in flight, so the context stays usable.
__global__ void timeout_probe_kernel(DevStatus* st, uint64_t limit_ns)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    fence_barrier_init();
    if (!mbar_wait(&bar, 0, limit_ns)) raise_status(st, OQR_ERR_TIMEOUT, 0, TAG_DIAG);
}

// --------------------------------------------------- 2-norm of a Gram -----
// For symmetric positive semidefinite S (n x n, column-major): out[0] = an
// estimate of lambda_max(S) (power iteration, a lower bound that converges to
// it), out[1] = trace(S).  One CTA; x and y in shared memory.
constexpr int LMAX_THREADS = 256;
constexpr int LMAX_ITERS = 60;
__global__ void __launch_bounds__(LMAX_THREADS) lambda_max_kernel(int n, const double* __restrict__ S, long lds,
                                                                  double* x, double* y, double* out)
{
    __shared__ double red[LMAX_THREADS / 32];
    __shared__ double bc[2];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    auto bsum = [&](double v) {
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        __syncthreads();
        if (lane == 0) red[w] = v;
        __syncthreads();
        double r = 0.0;
        for (int k = 0; k < LMAX_THREADS / 32; ++k) r += red[k];
        return r;
    };
    double tr = 0.0;
    for (int i = t; i < n; i += LMAX_THREADS) {
        tr += S[i + (long)i * lds];
        x[i] = 1.0 + 1e-3 * (i % 7);  // not orthogonal to the dominant eigenvector of a nonnegative S
    }
    tr = bsum(tr);
    double best = 0.0;
    for (int it = 0; it < LMAX_ITERS; ++it) {
        __syncthreads();
        double ny = 0.0, nx = 0.0;
        for (int i = t; i < n; i += LMAX_THREADS) {
            double v = 0.0;
            for (int j = 0; j < n; ++j) v = fma(S[j + (long)i * lds], x[j], v);  // S symmetric: row i = column i
            y[i] = v;
            ny += v * v;
            nx += x[i] * x[i];
        }
        ny = bsum(ny);
        nx = bsum(nx);
        if (t == 0) {
            bc[0] = nx > 0.0 ? sqrt(ny / nx) : 0.0;
            bc[1] = ny > 0.0 ? 1.0 / sqrt(ny) : 0.0;
        }
        __syncthreads();
        best = fmax(best, bc[0]);
        if (bc[1] == 0.0) break;
        for (int i = t; i < n; i += LMAX_THREADS) x[i] = y[i] * bc[1];
    }
    if (t == 0) {
        out[0] = best;
        out[1] = tr;
    }
}

// ------------------------------------------------------- norms and shift ---
// Partial sums of ||A||_F^2 over the lower triangle (off-diagonal twice) and
// of ||Z||_F^2; block b handles columns b, b + gridDim.x, ...
constexpr int NORM_THREADS = 256;

__device__ inline double block_sum(double v, double* red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    return s;
}

__global__ void norms_partial_kernel(int m, int n, const double* __restrict__ A, long lda,
                                     const double* __restrict__ Z, long ldz, double* scratch)
{
    __shared__ double red[32];
    double sa = 0.0, sz = 0.0;
    for (long j = blockIdx.x; j < m; j += gridDim.x) {
        for (long i = j + threadIdx.x; i < m; i += NORM_THREADS) {
            const double v = A[i + j * lda];
            sa += (i == j ? 1.0 : 2.0) * v * v;
        }
        if (j < n)
            for (long i = threadIdx.x; i < m; i += NORM_THREADS) {
                const double v = Z[i + j * ldz];
                sz += v * v;
            }
    }
    const double ta = block_sum(sa, red);
    const double tz = block_sum(sz, red);
    if (threadIdx.x == 0) {
        scratch[2 * blockIdx.x] = ta;
        scratch[2 * blockIdx.x + 1] = tz;
    }
}

__global__ void shift_finish_kernel(int m, int n, int parts, const double* scratch, double c, double u,
                                    DevStatus* st)
{
    if (threadIdx.x != 0) return;
    double sa = 0.0, sz = 0.0;
    for (int p = 0; p < parts; ++p) {
        sa += scratch[2 * p];
        sz += scratch[2 * p + 1];
    }
    const double nA = sqrt(sa);
    st->normA_fro = nA;
    st->normZ_fro2 = sz;
    st->shift = c * u * ((double)m * n + (double)n * (n + 1)) * nA * sz;
}

// ------------------------------------------------------ orthogonality ------
// E = G - I, ||E||_F, and a power-iteration estimate of ||E||_2 (E is
// symmetric; the estimate max ||E x|| / ||x|| is a lower bound that
// converges to ||E||_2).
constexpr int CHECK_THREADS = 512;

__global__ void __launch_bounds__(CHECK_THREADS) check_finish_kernel(int n, const double* __restrict__ G, long ldg,
                                                                      double* E, long lde, double* work,
                                                                      DevStatus* st)
{
    __shared__ double red[32];
    __shared__ double bc;
    double sf = 0.0;
    for (long e = threadIdx.x; e < (long)n * n; e += CHECK_THREADS) {
        const long i = e % n, j = e / n;
        const double v = G[i + j * ldg] - (i == j ? 1.0 : 0.0);
        if (E) E[i + j * lde] = v;
        work[e] = v;
        sf += v * v;
    }
    const double tf = block_sum(sf, red);
    if (threadIdx.x == 0) st->orthF = sqrt(tf);
    double* x = work + (size_t)n * n;
    double* y = x + n;
    for (int i = threadIdx.x; i < n; i += CHECK_THREADS) x[i] = 1.0 + 0.25 * sin(1.0 + i);
    __syncthreads();
    double best = 0.0;
    for (int it = 0; it < 32; ++it) {
        double sx = 0.0;
        for (int i = threadIdx.x; i < n; i += CHECK_THREADS) sx += x[i] * x[i];
        const double nx = block_sum(sx, red);
        if (threadIdx.x == 0) bc = sqrt(nx);
        __syncthreads();
        const double nrm = bc;
        if (!(nrm > 0.0)) break;
        for (int i = threadIdx.x; i < n; i += CHECK_THREADS) {
            double s = 0.0;
            for (int k = 0; k < n; ++k) s += work[i + (size_t)k * n] * x[k];
            y[i] = s / nrm;
        }
        __syncthreads();
        double sy = 0.0;
        for (int i = threadIdx.x; i < n; i += CHECK_THREADS) sy += y[i] * y[i];
        const double ny = block_sum(sy, red);
        if (threadIdx.x == 0) bc = sqrt(ny);
        __syncthreads();
        best = fmax(best, bc);
        for (int i = threadIdx.x; i < n; i += CHECK_THREADS) x[i] = y[i];
        __syncthreads();
    }
    if (threadIdx.x == 0) st->orth2 = best;
}

// ---------------------------------------------------------- FP64 GEMM ------
// C = beta C + alpha op(A) B, 64 x 64 tiles, 16-deep k-steps, 4 x 4 per
// thread; gridDim.z > 1 splits K and writes partials that a second kernel
// sums in a fixed order.
constexpr int GT = 64, GK = 16, GTHREADS = 256;

__device__ inline double opa(GemmOp op, const double* A, long lda, long i, long k)
{
    if (op == GEMM_N) return A[i + k * lda];
    if (op == GEMM_T) return A[k + i * lda];
    return i >= k ? A[i + k * lda] : A[k + i * lda];
}

__global__ void __launch_bounds__(GTHREADS) gemm_f64_kernel(GemmOp op, int M, int N, int K, double alpha,
                                                            const double* __restrict__ A, long lda,
                                                            const double* __restrict__ B, long ldb, double beta,
                                                            double* C, long ldc, double* ws)
{
    __shared__ double As[GK][GT + 1];
    __shared__ double Bs[GK][GT + 1];
    const int tid = threadIdx.x, ty = tid & 15, tx = tid >> 4;
    const long i0 = (long)blockIdx.x * GT, j0 = (long)blockIdx.y * GT;
    const int splits = gridDim.z;
    const long kper = ((K + splits - 1) / splits + GK - 1) / GK * GK;
    const long k0 = (long)blockIdx.z * kper, k1 = min((long)K, k0 + kper);
    double acc[4][4] = {};
    for (long kk = k0; kk < k1; kk += GK) {
        for (int e = tid; e < GT * GK; e += GTHREADS) {
            int r, k;
            if (op == GEMM_T) { k = e % GK; r = e / GK; } else { r = e % GT; k = e / GT; }
            const long gi = i0 + r, gk = kk + k;
            As[k][r] = (gi < M && gk < k1) ? opa(op, A, lda, gi, gk) : 0.0;
        }
        for (int e = tid; e < GT * GK; e += GTHREADS) {
            const int k = e % GK, c = e / GK;
            const long gk = kk + k, gj = j0 + c;
            Bs[k][c] = (gk < k1 && gj < N) ? B[gk + gj * ldb] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < GK; ++k) {
            double av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = As[k][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Bs[k][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const long gi = i0 + ty + 16 * i, gj = j0 + tx + 16 * j;
            if (gi >= M || gj >= N) continue;
            if (splits == 1) {
                const double c0 = beta == 0.0 ? 0.0 : beta * C[gi + gj * ldc];
                C[gi + gj * ldc] = c0 + alpha * acc[i][j];
            } else {
                ws[(size_t)blockIdx.z * M * N + gi + gj * (size_t)M] = acc[i][j];
            }
        }
}

// C = beta C + alpha A^T B for M <= 32 (A stored K x M): 32 x 128 tiles, so a narrow A^T fills the tile;
// the same 16-deep k-steps, 4 x 4 per thread, and split-K partials as gemm_f64_kernel.
constexpr int GTN_M = 32, GTN_N = 128;
__global__ void __launch_bounds__(GTHREADS) gemm_f64_tn32_kernel(int M, int N, int K, double alpha,
                                                                 const double* __restrict__ A, long lda,
                                                                 const double* __restrict__ B, long ldb, double beta,
                                                                 double* C, long ldc, double* ws)
{
    __shared__ double As[GK][GTN_M + 1];
    __shared__ double Bs[GK][GTN_N + 1];
    const int tid = threadIdx.x, ty = tid & 7, tx = tid >> 3;
    const long j0 = (long)blockIdx.y * GTN_N;
    const int splits = gridDim.z;
    const long kper = ((K + splits - 1) / splits + GK - 1) / GK * GK;
    const long k0 = (long)blockIdx.z * kper, k1 = min((long)K, k0 + kper);
    double acc[4][4] = {};
    for (long kk = k0; kk < k1; kk += GK) {
        for (int e = tid; e < GTN_M * GK; e += GTHREADS) {
            const int k = e % GK, r = e / GK;
            const long gk = kk + k;
            As[k][r] = (r < M && gk < k1) ? A[gk + r * lda] : 0.0;
        }
        for (int e = tid; e < GK * GTN_N; e += GTHREADS) {
            const int k = e % GK, c = e / GK;
            const long gk = kk + k, gj = j0 + c;
            Bs[k][c] = (gk < k1 && gj < N) ? B[gk + gj * ldb] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < GK; ++k) {
            double av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = As[k][ty + 8 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Bs[k][tx + 32 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const long gi = ty + 8 * i, gj = j0 + tx + 32 * j;
            if (gi >= M || gj >= N) continue;
            if (splits == 1) {
                const double c0 = beta == 0.0 ? 0.0 : beta * C[gi + gj * ldc];
                C[gi + gj * ldc] = c0 + alpha * acc[i][j];
            } else {
                ws[(size_t)blockIdx.z * M * N + gi + gj * (size_t)M] = acc[i][j];
            }
        }
}

// One warp per output element: lane l sums partials l, l + 32, ..., then a fixed shuffle tree.
__global__ void gemm_splitk_reduce_kernel(int M, int N, int splits, double alpha, const double* ws, double beta,
                                          double* C, long ldc)
{
    const long e = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (e >= (long)M * N) return;
    const long i = e % M, j = e / M;
    double s = 0.0;
    for (int z = lane; z < splits; z += 32) s += ws[(size_t)z * M * N + e];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane != 0) return;
    const double c0 = beta == 0.0 ? 0.0 : beta * C[i + j * ldc];
    C[i + j * ldc] = c0 + alpha * s;
}

__global__ void axpby_kernel(int M, int N, double alpha, const double* X, long ldx, double beta, double* Y, long ldy)
{
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long)M * N) return;
    const long i = e % M, j = e / M;
    const double y0 = beta == 0.0 ? 0.0 : beta * Y[i + j * ldy];
    Y[i + j * ldy] = y0 + alpha * X[i + j * ldx];
}

}  // namespace

cudaError_t launch_axpby(int M, int N, double alpha, const double* X, long ldx, double beta, double* Y, long ldy,
                         cudaStream_t s)
{
    const long total = (long)M * N;
    if (total <= 0) return cudaSuccess;
    axpby_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(M, N, alpha, X, ldx, beta, Y, ldy);
    return cudaGetLastError();
}

cudaError_t launch_potrf(int n, const double* G, long ldg, double* R, long ldr, const double* shift_ptr,
                         DevStatus* st, cudaStream_t s)
{
    const long total = (long)n * n;
    potrf_init_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(n, G, ldg, R, ldr, shift_ptr, st);
    for (int jb = 0; jb < n; jb += PNB) {
        potrf_diag_kernel<<<1, 512, 0, s>>>(n, jb, R, ldr, st);
        const int rest = n - jb - PNB;
        if (rest <= 0) break;
        potrf_row_kernel<<<(rest + PROW_WARPS - 1) / PROW_WARPS, 32 * PROW_WARPS, 0, s>>>(n, jb, R, ldr, st);
        const int nt = (rest + TT - 1) / TT;
        potrf_trail_kernel<<<nt * (nt + 1) / 2, TT * TT, 0, s>>>(n, jb, R, ldr, st);
    }
    return cudaGetLastError();
}

cudaError_t launch_trsm_block(int m, int jb, int bw, const double* Z, long ldz, const double* U, long ldu,
                              const double* R, long ldr, double* Q, long ldq, DevStatus* st, cudaStream_t s,
                              const int* gate, int want)
{
    if (m <= 0 || bw <= 0) return cudaSuccess;
    if (bw > TBW) return cudaErrorInvalidValue;
    trsm_block_kernel<<<(unsigned)((m + TB_THREADS - 1) / TB_THREADS), TB_THREADS, 0, s>>>(m, jb, bw, Z, ldz, U, ldu, R,
                                                                                          ldr, Q, ldq, st, gate, want);
    return cudaGetLastError();
}

cudaError_t launch_trsm(int m, int n, const double* Z, long ldz, const double* R, long ldr, double* Q, long ldq,
                        DevStatus* st, cudaStream_t s, const int* gate, int want)
{
    int rows = 64;
    while (rows > 8 && (size_t)rows * (n + 1) * sizeof(double) > 160 * 1024) rows /= 2;
    const size_t smem = ((size_t)rows * (n + 1) + 2 * TNB * (TNB + 1)) * sizeof(double);
    if (smem > 220 * 1024) return cudaErrorInvalidValue;
    cudaFuncSetAttribute(trsm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const unsigned blocks = (unsigned)((m + rows - 1) / rows);
    trsm_kernel<<<blocks, TRSM_THREADS, smem, s>>>(m, n, rows, Z, ldz, R, ldr, Q, ldq, st, gate, want);
    return cudaGetLastError();
}

cudaError_t launch_rprod(int n, const double* U, long ldu, const double* S, long lds, double* R, long ldr,
                         cudaStream_t s)
{
    const long total = (long)n * n;
    rprod_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(n, U, ldu, S, lds, R, ldr);
    return cudaGetLastError();
}

cudaError_t launch_transpose(int rows, int cols, const double* S, long lds, double* D, long ldd, cudaStream_t s)
{
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    transpose_kernel<<<dim3((unsigned)((rows + 31) / 32), (unsigned)((cols + 31) / 32)), dim3(32, 32), 0, s>>>(
        rows, cols, S, lds, D, ldd);
    return cudaGetLastError();
}

cudaError_t launch_gram_defect(int n, const double* G, long ldg, double* out, int* gate, double gate_tol,
                               cudaStream_t s)
{
    static_assert(GD_BLOCKS == 64, "the sum kernel reads two parts per lane");
    gram_defect_part_kernel<<<GD_BLOCKS, GD_THREADS, 0, s>>>(n, G, ldg, out + 1);
    gram_defect_sum_kernel<<<1, 32, 0, s>>>(out + 1, out, gate, gate_tol);
    return cudaGetLastError();
}

cudaError_t launch_trinv(int n, const double* R, long ldr, double* X, long ldx, const DevStatus* st, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const size_t smem = (size_t)2 * n * sizeof(double);
    if (n > TRINV_MAX_N) return cudaErrorInvalidValue;
    auto run = [&](auto kernel) {
        if (smem > 48 * 1024) {
            const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        kernel<<<(unsigned)n, TI_THREADS, smem, s>>>(n, R, ldr, X, ldx, st);
        return cudaGetLastError();
    };
    const int rpt = (n + TI_THREADS - 1) / TI_THREADS;
    if (rpt <= 1) return run(trinv_upper_kernel<1>);
    if (rpt <= 2) return run(trinv_upper_kernel<2>);
    if (rpt <= 4) return run(trinv_upper_kernel<4>);
    if (rpt <= 8) return run(trinv_upper_kernel<8>);
    if (rpt <= 16) return run(trinv_upper_kernel<16>);
    return run(trinv_upper_kernel<32>);
}

cudaError_t launch_copy_upper(int n, const double* S, long lds, double* D, long ldd, cudaStream_t s)
{
    const long total = (long)n * n;
    copy_upper_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(n, S, lds, D, ldd);
    return cudaGetLastError();
}

cudaError_t launch_norms_and_shift(int m, int n, const double* A, long lda, const double* Z, long ldz, double c,
                                   double u, double* scratch, int scratch_len, DevStatus* st, cudaStream_t s)
{
    int parts = scratch_len / 2;
    if (parts > m) parts = m;
    if (parts < 1) return cudaErrorInvalidValue;
    norms_partial_kernel<<<parts, NORM_THREADS, 0, s>>>(m, n, A, lda, Z, ldz, scratch);
    shift_finish_kernel<<<1, 32, 0, s>>>(m, n, parts, scratch, c, u, st);
    return cudaGetLastError();
}

cudaError_t launch_check_finish(int n, const double* G, long ldg, double* E, long lde, double* work,
                                DevStatus* st, cudaStream_t s)
{
    check_finish_kernel<<<1, CHECK_THREADS, 0, s>>>(n, G, ldg, E, lde, work, st);
    return cudaGetLastError();
}

size_t gemm_splitk_bytes(int M, int N, int splits)
{
    return splits > 1 ? (size_t)splits * M * N * sizeof(double) : 0;
}

cudaError_t launch_gemm_f64(GemmOp op, int M, int N, int K, double alpha, const double* A, long lda,
                            const double* B, long ldb, double beta, double* C, long ldc, double* splitk_ws,
                            int splits, cudaStream_t s)
{
    if (M <= 0 || N <= 0) return cudaSuccess;
    if (splits < 1) splits = 1;
    if (op == GEMM_T && M <= GTN_M) {
        dim3 grid(1, (N + GTN_N - 1) / GTN_N, splits);
        gemm_f64_tn32_kernel<<<grid, GTHREADS, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, splitk_ws);
    } else {
        dim3 grid((M + GT - 1) / GT, (N + GT - 1) / GT, splits);
        gemm_f64_kernel<<<grid, GTHREADS, 0, s>>>(op, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, splitk_ws);
    }
    if (splits > 1) {
        const long total = (long)M * N * 32;  // a warp per element
        gemm_splitk_reduce_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(M, N, splits, alpha, splitk_ws,
                                                                                 beta, C, ldc);
    }
    return cudaGetLastError();
}

cudaError_t launch_lambda_max(int n, const double* S, long lds, double* work, double* out, cudaStream_t s)
{
    lambda_max_kernel<<<1, LMAX_THREADS, 0, s>>>(n, S, lds, work, work + n, out);
    return cudaGetLastError();
}

cudaError_t launch_timeout_probe(DevStatus* st, uint64_t limit_ns, cudaStream_t s)
{
    timeout_probe_kernel<<<1, 32, 0, s>>>(st, limit_ns);
    return cudaGetLastError();
}

}  // namespace oqr
