// Batched oblique QR: thousands of independent (A_b, Z_b), n_b <= 64, in a
// handful of launches (Algorithm 1 repeated as A-CholQR2, per instance).
//
// Each instance is described by one BatchDesc in device memory.  The launches
// of one normal-equation pass cover the whole batch:
//   gram_batched   grid (split, instance): the symmetric Gram of Sec. 2 with
//                  A = M + M^T, M = tril(A,-1) + diag(A)/2, over 64-row blocks
//                  and k-steps of 16 of A's lower triangle, in FP64 FMA;
//                  column tiles of NP = 16, 32 or 64 (the plan's choice for
//                  n_b); every split owns its partial P_s (deterministic).
//   reduce         G_b = sum_s P_s + P_s^T (fixed order, exactly symmetric).
//   potrf_batched  one CTA per instance, G_b (<= 64 x 64) in shared memory.
//   trsm_batched   grid (row block, instance): Q_b = Z_b / R_b row by row.
//   rprod_batched  R_b = R_2 R_1.
// The tensor-core batches (packed waves, k_tc.cu) form the Grams' halves C_b
// on the tensor cores and use the same descriptors for the FP64 steps, with
// 1 to 3 passes per instance (BatchDesc.npass; instances whose passes are done
// sit later passes out): reduce (+ s_b I on a shifted first pass), potrf,
// trsm, racc_batched (R1 <- R2 R1 after every later pass), rfinal_batched
// (the caller's R = R1), shift_batched (the first pass's shift, ||A||_F from the split) and
// check_batched (||Q^T A Q - I||_2 from one more Gram of Q).
// A Cholesky breakdown is recorded in the instance's own status word and that
// instance's later kernels skip it; other instances are unaffected.
#include <math.h>

#include "oqr_internal.cuh"

namespace oqr {
namespace {

constexpr int BBM = 64;   // rows per row block
constexpr int BBK = 16;   // k-step
constexpr int BTHREADS = 256;
static_assert(BATCH_MAX_N == 64, "the per-instance kernels hold n x n <= 64 x 64 in shared memory");

__device__ __host__ inline long bk_steps_of(long I, long m)
{
    long hi = (I + 1) * BBM;
    if (hi > m) hi = m;
    return (hi + BBK - 1) / BBK;
}
__device__ __host__ inline long bk_cum(long I) { return 2 * I * (I + 1); }  // 4 k-steps per full block
static_assert(BBM / BBK == 4, "bk_cum assumes 4 k-steps per full row block");

__device__ inline long bk_block_of(long u, long nblocks)
{
    long I = (long)((sqrt(1.0 + 2.0 * (double)u) - 1.0) * 0.5);
    if (I < 0) I = 0;
    if (I > nblocks - 1) I = nblocks - 1;
    while (I > 0 && bk_cum(I) > u) --I;
    while (I + 1 < nblocks && bk_cum(I + 1) <= u) ++I;
    return I;
}

// G_b partials: P_s (n x n, row-major) for s < splits_b, at partials + s n^2.
template <int NP>
__global__ void __launch_bounds__(BTHREADS) gram_batched_kernel(const BatchDesc* __restrict__ d, const int* idx,
                                                                int* status, const int pass_in_place)
{
    __shared__ double As[BBK][BBM + 1];
    __shared__ double Zs[BBK][NP + 1];
    __shared__ double Ts[BBM][NP + 1];
    const int b = idx[blockIdx.y];
    const BatchDesc D = d[b];
    const int split = blockIdx.x;
    if (split >= D.splits || status[b] != 0) return;
    const int m = D.m, n = D.n;
    const double* X = pass_in_place ? D.Q : D.Z;  // pass 1 reads Z, later passes read Q
    const long ldx = pass_in_place ? D.ldq : D.ldz;
    const long nblocks = (m + BBM - 1) / BBM;
    const long steps = bk_cum(nblocks - 1) + bk_steps_of(nblocks - 1, m);
    const long u0 = steps * split / D.splits, u1 = steps * (split + 1) / D.splits;
    double* P = D.partials + (size_t)split * n * n;
    const int tid = threadIdx.x;
    // thread tile: rows ty + 16 i (i < 4), columns tx + (NP/4)... : 16 x 16 threads
    constexpr int CJ = NP / 16;  // columns per thread
    const int ty = tid & 15, tx = tid >> 4;
    bool first = true;
    long u = u0;
    while (u < u1) {
        const long I = bk_block_of(u, nblocks);
        const long kb0 = u - bk_cum(I);
        long nk = bk_steps_of(I, m) - kb0;
        if (nk > u1 - u) nk = u1 - u;
        double acc[4][CJ];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < CJ; ++j) acc[i][j] = 0.0;
        for (long it = 0; it < nk; ++it) {
            const long kb = kb0 + it;
            const long row0 = I * BBM, col0 = kb * BBK;
            __syncthreads();
            for (int e = tid; e < BBM * BBK; e += BTHREADS) {
                const int r = e % BBM, k = e / BBM;
                const long gr = row0 + r, gc = col0 + k;
                double v = 0.0;
                if (gr < m && gc < m && gc <= gr) {
                    v = D.A[gr + gc * D.lda];
                    if (gc == gr) v *= 0.5;
                }
                As[k][r] = v;
            }
            for (int e = tid; e < BBK * NP; e += BTHREADS) {
                const int k = e % BBK, c = e / BBK;
                const long gr = col0 + k;
                Zs[k][c] = (gr < m && c < n) ? X[gr + (long)c * ldx] : 0.0;
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < BBK; ++k) {
                double av[4], zv[CJ];
#pragma unroll
                for (int i = 0; i < 4; ++i) av[i] = As[k][ty + 16 * i];
#pragma unroll
                for (int j = 0; j < CJ; ++j) zv[j] = Zs[k][tx + 16 * j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < CJ; ++j) acc[i][j] = fma(av[i], zv[j], acc[i][j]);
            }
        }
        // epilogue: P(:, c) (+)= X(I rows, :)^T T
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < CJ; ++j) Ts[ty + 16 * i][tx + 16 * j] = acc[i][j];
        __syncthreads();
        const long row0 = I * BBM;
        for (int e = tid; e < n * n; e += BTHREADS) {
            const int r = e / n, c = e % n;
            double s = 0.0;
            for (int i = 0; i < BBM; ++i) {
                const long gr = row0 + i;
                if (gr >= m) break;
                s = fma(X[gr + (long)r * ldx], Ts[i][c], s);
            }
            P[(size_t)r * n + c] = first ? s : P[(size_t)r * n + c] + s;
        }
        first = false;
        u += nk;
    }
    if (first)
        for (int e = tid; e < n * n; e += BTHREADS) P[e] = 0.0;
}

__global__ void reduce_batched_kernel(const BatchDesc* __restrict__ d, const int* status, const double* shifts,
                                      int pass)
{
    const int b = blockIdx.y;
    const BatchDesc D = d[b];
    if (status[b] != 0 || pass >= D.npass) return;
    const int n = D.n;
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long)n * n) return;
    const int r = (int)(e % n), c = (int)(e / n);
    double s = 0.0;
    const size_t nn = (size_t)n * n;
    for (int p = 0; p < D.splits; ++p) {
        const double* P = D.partials + p * nn;
        s += P[(size_t)r * n + c] + P[(size_t)c * n + r];
    }
    if (shifts && r == c) s += shifts[b];  // G + s I (the shifted first pass)
    D.G[r + (size_t)c * n] = s;
}

// One CTA per instance: R = chol(G), G n x n (n <= 64) in shared memory,
// right-looking, column by column.  Writes R (upper, zeros below) into Rout.
// mask (or NULL for all): the instances to factor.  Per column j: the row
// R(j, j+1:n) = S(j, j+1:n) / R(j, j) into srow, then the trailing update of
// the upper triangle over its pairs (r, c), j < r <= c, read from a table
// built once per block.  Thread 0 owns the first pair, (j+1, j+1), so it
// takes the next pivot (1 / sqrt by FP64 rsqrt, the diagonal as pivot times
// that) while the other threads finish the update: two block barriers per
// column.
constexpr int POTRF_PAIRS = 63 * 64 / 2;
__global__ void __launch_bounds__(256) potrf_batched_kernel(const BatchDesc* __restrict__ d, int* status, int which,
                                                            int pass, const int* mask = nullptr)
{
    __shared__ double S[64][65];
    __shared__ double srow[64];
    __shared__ unsigned short pair[POTRF_PAIRS];  // (r' << 8) | c', r' <= c': the trailing triangle column by column
    __shared__ double rinv_s;
    __shared__ int broke;
    const int b = blockIdx.x;
    const BatchDesc D = d[b];
    if (status[b] != 0 || pass >= D.npass || (mask && !mask[b])) return;
    const int n = D.n;
    double* Rout = which == 0 ? D.R1 : D.R2;
    const int tid = threadIdx.x;
    for (int e = tid; e < n * n; e += 256) {
        const int i = e % n, j = e / n;
        S[i][j] = (i <= j) ? D.G[j + (size_t)i * n] : 0.0;  // lower triangle of G -> upper of S
    }
    for (int e = tid; e < POTRF_PAIRS; e += 256) {
        int c = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
        while (c * (c + 1) / 2 > e) --c;
        while ((c + 1) * (c + 2) / 2 <= e) ++c;
        pair[e] = (unsigned short)(((e - c * (c + 1) / 2) << 8) | c);
    }
    auto pivot = [&](int j) {  // thread 0
        const double piv = S[j][j];
        if (!(piv > 0.0)) {
            broke = j + 1;
        } else {
            const double r = rsqrt(piv);
            S[j][j] = piv * r;
            rinv_s = r;
        }
    };
    __syncthreads();
    if (tid == 0) {
        broke = 0;
        pivot(0);
    }
    __syncthreads();
    for (int j = 0; j < n; ++j) {
        if (broke) break;
        const double rj = rinv_s;
        for (int c = j + 1 + tid; c < n; c += 256) {
            const double v = S[j][c] * rj;
            srow[c] = v;
            S[j][c] = v;
        }
        __syncthreads();
        const int w = n - j - 1;
        for (int e = tid; e < w * (w + 1) / 2; e += 256) {
            const int p = pair[e];
            const int r = j + 1 + (p >> 8), c = j + 1 + (p & 255);
            S[r][c] = fma(-srow[r], srow[c], S[r][c]);
            if (e == 0) pivot(j + 1);  // thread 0, pair (j+1, j+1)
        }
        __syncthreads();
    }
    if (broke) {
        if (tid == 0) status[b] = broke;
        return;
    }
    for (int e = tid; e < n * n; e += 256) {
        const int i = e % n, j = e / n;
        Rout[i + (size_t)j * n] = (i <= j) ? S[i][j] : 0.0;
    }
}

// Q = X / R row by row, TRSM_ROWS rows per CTA (one per thread; FP64 is scarce, so an instance's rows
// are spread over many SMs), R (<= 64 x 64) in shared memory.
// mask (or NULL for all): the instances to solve.
constexpr int TRSM_ROWS = 64;
__global__ void __launch_bounds__(TRSM_ROWS) trsm_batched_kernel(const BatchDesc* __restrict__ d, const int* status,
                                                           int pass_in_place, int which, int pass,
                                                           const int* mask = nullptr)
{
    __shared__ double Rs[64][65];
    __shared__ double dinv[64];
    const int b = blockIdx.y;
    const BatchDesc D = d[b];
    if (status[b] != 0 || pass >= D.npass || (mask && !mask[b])) return;
    const int m = D.m, n = D.n;
    const long row0 = (long)blockIdx.x * TRSM_ROWS;
    if (row0 >= m) return;  // the grid covers the largest m of the batch
    const double* Rin = which == 0 ? D.R1 : D.R2;
    for (int e = threadIdx.x; e < n * n; e += TRSM_ROWS) {
        const int i = e % n, j = e / n;
        Rs[i][j] = Rin[i + (size_t)j * n];
    }
    if (threadIdx.x < n) dinv[threadIdx.x] = 1.0 / Rin[threadIdx.x + (size_t)threadIdx.x * n];
    __syncthreads();
    const long r = row0 + threadIdx.x;
    if (r >= m) return;
    const double* X = pass_in_place ? D.Q : D.Z;
    const long ldx = pass_in_place ? D.ldq : D.ldz;
    double q[64];
#pragma unroll
    for (int j = 0; j < 64; ++j) {
        if (j < n) {
            double t = X[r + (long)j * ldx];
            for (int k = 0; k < j; ++k) t -= q[k] * Rs[k][j];
            q[j] = t * dinv[j];  // one division per column and CTA, not per element
        }
    }
#pragma unroll
    for (int j = 0; j < 64; ++j)
        if (j < n) D.Q[r + (long)j * D.ldq] = q[j];
}

// R_out = R2 R1 (upper), written into the caller's R.
__global__ void rprod_batched_kernel(const BatchDesc* __restrict__ d, const int* status)
{
    const int b = blockIdx.y;
    const BatchDesc D = d[b];
    if (status[b] != 0) return;
    const int n = D.n;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * n) return;
    const int i = e % n, j = e / n;
    double s = 0.0;
    if (i <= j)
        for (int k = i; k <= j; ++k) s += D.R2[i + (size_t)k * n] * D.R1[k + (size_t)j * n];
    D.R[i + (long)j * D.ldr] = s;
}

// R1 <- R2 R1 (upper x upper) after a later pass: one CTA per instance, the
// product held in shared memory until every thread has read R1.
__global__ void __launch_bounds__(256) racc_batched_kernel(const BatchDesc* __restrict__ d, const int* status,
                                                           int pass)
{
    __shared__ double T[64][65];
    const int b = blockIdx.x;
    const BatchDesc D = d[b];
    if (status[b] != 0 || pass >= D.npass) return;
    const int n = D.n;
    for (int e = threadIdx.x; e < n * n; e += 256) {
        const int i = e % n, j = e / n;
        double s = 0.0;
        for (int k = i; k <= j; ++k) s += D.R2[i + (size_t)k * n] * D.R1[k + (size_t)j * n];
        T[i][j] = s;  // 0 below the diagonal
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * n; e += 256) {
        const int i = e % n, j = e / n;
        D.R1[i + (size_t)j * n] = T[i][j];
    }
}

// The caller's R = R1 (upper, zeros below the diagonal).
__global__ void rfinal_batched_kernel(const BatchDesc* __restrict__ d, const int* status)
{
    const int b = blockIdx.y;
    const BatchDesc D = d[b];
    if (status[b] != 0) return;
    const int n = D.n;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * n) return;
    const int i = e % n, j = e / n;
    D.R[i + (long)j * D.ldr] = i <= j ? D.R1[i + (size_t)j * n] : 0.0;
}

// s_b = c u (m n + n (n + 1)) ||A_b||_F ||Z_b||_F^2 for a shifted instance (mask[b] != 0), else 0, from the
// squared norms the splits summed (anorm2, znorm2).
__global__ void shift_batched_kernel(const BatchDesc* __restrict__ d, int count, const int* __restrict__ mask,
                                     const double* anorm2, const double* znorm2, double c, double u, double* shifts)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= count) return;
    const BatchDesc D = d[b];
    shifts[b] = mask[b] ? c * u * ((double)D.m * D.n + (double)D.n * (D.n + 1)) * sqrt(anorm2[b]) * znorm2[b] : 0.0;
}

// ||E||_2 estimate of E = G - I for the instances checked at this pass (one CTA each).
constexpr int BCHECK_ITERS = 40;
// last = false: the check of the instances whose factor passes end at pass (D.npass == pass), from one
// more Gram of Q.  last = true: the defect of the Gram that an instance's last factor pass factors
// (D.npass >= 2, pass == D.npass - 1): ||Q_prev^T A Q_prev - I||_2 of the previous pass's Q.
template <bool LAST>
__global__ void __launch_bounds__(256) check_batched_kernel(const BatchDesc* __restrict__ d, const int* status,
                                                            int pass, double* orth)
{
    __shared__ double E[64][65];
    __shared__ double x[64], y[64];
    __shared__ double red[8];
    const int b = blockIdx.x;
    const BatchDesc D = d[b];
    if (LAST ? (D.npass < 2 || pass != D.npass - 1) : (D.npass != pass)) return;
    if (status[b] != 0) {
        if (threadIdx.x == 0) orth[b] = INFINITY;
        return;
    }
    const int n = D.n;
    const double* P = D.partials;
    for (int e = threadIdx.x; e < n * n; e += 256) {
        const int i = e % n, j = e / n;
        E[i][j] = P[(size_t)i * n + j] + P[(size_t)j * n + i] - (i == j ? 1.0 : 0.0);
    }
    if (threadIdx.x < n) x[threadIdx.x] = 1.0 + 0.01 * threadIdx.x;  // not orthogonal to a dominant vector
    __syncthreads();
    double best = 0.0;
    for (int it = 0; it < BCHECK_ITERS; ++it) {
        // y = E x (one warp per 8 rows), then ||y|| / ||x|| and x = y / ||y||
        const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int i = w; i < n; i += 8) {
            double t = 0.0;
            for (int k = lane; k < n; k += 32) t += E[i][k] * x[k];
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) y[i] = t;
        }
        __syncthreads();
        if (w == 0) {
            double ny = 0.0, nx = 0.0;
            for (int k = lane; k < n; k += 32) {
                ny += y[k] * y[k];
                nx += x[k] * x[k];
            }
            for (int o = 16; o > 0; o >>= 1) {
                ny += __shfl_xor_sync(0xffffffffu, ny, o);
                nx += __shfl_xor_sync(0xffffffffu, nx, o);
            }
            if (lane == 0) {
                red[0] = sqrt(ny / nx);
                red[1] = ny > 0.0 ? 1.0 / sqrt(ny) : 0.0;
            }
        }
        __syncthreads();
        best = fmax(best, red[0]);
        if (red[1] == 0.0) break;  // E x = 0
        if (threadIdx.x < n) x[threadIdx.x] = y[threadIdx.x] * red[1];
        __syncthreads();
    }
    if (threadIdx.x == 0) orth[b] = best;
}

__global__ void scatter_rows_f32_kernel(const float* in, const int* perm, int count, int width, float* out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    for (int k = 0; k < width; ++k) out[(long)perm[i] * width + k] = in[(long)i * width + k];
}

__global__ void scatter_f64_kernel(const double* in, const int* perm, int count, double* out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) out[perm[i]] = in[i];
}

// status[perm[i]] = st_sorted[i]; -1 for all when a kernel of the context timed out.
__global__ void status_scatter_kernel(const int* st_sorted, const int* perm, int count, const DevStatus* st,
                                      int* status)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    status[perm[i]] = st->code != 0 ? -1 : st_sorted[i];
}

}  // namespace

// Gram kernels take the instances of one tile class through an index list.
cudaError_t launch_batched_cholqr2(const BatchDesc* d, int count, const int* const* cls_idx, const int* cls_count,
                                   const int* cls_max_splits, int max_n, int* status, cudaStream_t s)
{
    for (int pass = 0; pass < 2; ++pass) {
        for (int c = 0; c < 3; ++c) {
            if (cls_count[c] == 0) continue;
            dim3 g(cls_max_splits[c], cls_count[c]);
            if (c == 0) gram_batched_kernel<16><<<g, BTHREADS, 0, s>>>(d, cls_idx[c], status, pass);
            else if (c == 1) gram_batched_kernel<32><<<g, BTHREADS, 0, s>>>(d, cls_idx[c], status, pass);
            else gram_batched_kernel<64><<<g, BTHREADS, 0, s>>>(d, cls_idx[c], status, pass);
        }
        dim3 gr((max_n * max_n + 255) / 256, count);
        reduce_batched_kernel<<<gr, 256, 0, s>>>(d, status, nullptr, pass);
        potrf_batched_kernel<<<count, 256, 0, s>>>(d, status, pass, pass);
        dim3 gt(BATCH_MAX_M / TRSM_ROWS, count);
        trsm_batched_kernel<<<gt, TRSM_ROWS, 0, s>>>(d, status, pass, pass, pass);
    }
    dim3 gp((64 * 64 + 255) / 256, count);
    rprod_batched_kernel<<<gp, 256, 0, s>>>(d, status);
    return cudaGetLastError();
}

cudaError_t launch_batched_factor(const BatchDesc* d, int count, int* status, int pass, const double* shifts,
                                  cudaStream_t s)
{
    const int which = pass == 0 ? 0 : 1;
    dim3 gr((BATCH_MAX_N * BATCH_MAX_N + 255) / 256, count);
    reduce_batched_kernel<<<gr, 256, 0, s>>>(d, status, pass == 0 ? shifts : nullptr, pass);
    potrf_batched_kernel<<<count, 256, 0, s>>>(d, status, which, pass);
    dim3 gt(BATCH_MAX_M / TRSM_ROWS, count);
    trsm_batched_kernel<<<gt, TRSM_ROWS, 0, s>>>(d, status, pass > 0, which, pass);
    if (pass > 0) racc_batched_kernel<<<count, 256, 0, s>>>(d, status, pass);
    return cudaGetLastError();
}

cudaError_t launch_batched_gram_chol(const BatchDesc* d, int count, int* status, cudaStream_t s)
{
    dim3 gr((BATCH_MAX_N * BATCH_MAX_N + 255) / 256, count);
    reduce_batched_kernel<<<gr, 256, 0, s>>>(d, status, nullptr, 0);
    potrf_batched_kernel<<<count, 256, 0, s>>>(d, status, 0, 0);
    return cudaGetLastError();
}

cudaError_t launch_batched_chol_solve(const BatchDesc* d, int count, int* status, const int* chol_mask,
                                      const int* solve_mask, cudaStream_t s)
{
    potrf_batched_kernel<<<count, 256, 0, s>>>(d, status, 0, 0, chol_mask);
    dim3 gt(BATCH_MAX_M / TRSM_ROWS, count);
    trsm_batched_kernel<<<gt, TRSM_ROWS, 0, s>>>(d, status, 0, 0, 0, solve_mask);
    return cudaGetLastError();
}

cudaError_t launch_batched_rfinal(const BatchDesc* d, int count, int* status, cudaStream_t s)
{
    dim3 gp((BATCH_MAX_N * BATCH_MAX_N + 255) / 256, count);
    rfinal_batched_kernel<<<gp, 256, 0, s>>>(d, status);
    return cudaGetLastError();
}

cudaError_t launch_batched_shifts(const BatchDesc* d, int count, const int* mask, const double* anorm2,
                                  const double* znorm2, double c, double u, double* shifts, cudaStream_t s)
{
    if (count > 0) shift_batched_kernel<<<(count + 127) / 128, 128, 0, s>>>(d, count, mask, anorm2, znorm2, c, u, shifts);
    return cudaGetLastError();
}

cudaError_t launch_batch_status_scatter(const int* st_sorted, const int* perm, int count, const DevStatus* st,
                                        int* status, cudaStream_t s)
{
    status_scatter_kernel<<<(count + 255) / 256, 256, 0, s>>>(st_sorted, perm, count, st, status);
    return cudaGetLastError();
}

cudaError_t launch_batched_check(const BatchDesc* d, int count, const int* status, int pass, double* orth,
                                 cudaStream_t s)
{
    check_batched_kernel<false><<<count, 256, 0, s>>>(d, status, pass, orth);
    return cudaGetLastError();
}

cudaError_t launch_batched_last_defect(const BatchDesc* d, int count, const int* status, int pass, double* defect,
                                       cudaStream_t s)
{
    check_batched_kernel<true><<<count, 256, 0, s>>>(d, status, pass, defect);
    return cudaGetLastError();
}

cudaError_t launch_batch_scatter_rows_f32(const float* in, const int* perm, int count, int width, float* out,
                                          cudaStream_t s)
{
    scatter_rows_f32_kernel<<<(count + 255) / 256, 256, 0, s>>>(in, perm, count, width, out);
    return cudaGetLastError();
}

cudaError_t launch_batch_scatter_f64(const double* in, const int* perm, int count, double* out, cudaStream_t s)
{
    scatter_f64_kernel<<<(count + 255) / 256, 256, 0, s>>>(in, perm, count, out);
    return cudaGetLastError();
}

}  // namespace oqr
