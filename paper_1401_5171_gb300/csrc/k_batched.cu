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

__global__ void reduce_batched_kernel(const BatchDesc* __restrict__ d, const int* status, double* shift_or_null)
{
    const int b = blockIdx.y;
    const BatchDesc D = d[b];
    if (status[b] != 0) return;
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
    D.G[r + (size_t)c * n] = s;
}

// One CTA per instance: R = chol(G), G n x n (n <= 64) in shared memory,
// right-looking, column by column.  Writes R (upper, zeros below) into Rout.
__global__ void __launch_bounds__(256) potrf_batched_kernel(const BatchDesc* __restrict__ d, int* status, int which)
{
    __shared__ double S[64][65];
    __shared__ int broke;
    const int b = blockIdx.x;
    const BatchDesc D = d[b];
    if (status[b] != 0) return;
    const int n = D.n;
    double* Rout = which == 0 ? D.R1 : D.R2;
    const int tid = threadIdx.x;
    for (int e = tid; e < n * n; e += 256) {
        const int i = e % n, j = e / n;
        S[i][j] = (i <= j) ? D.G[j + (size_t)i * n] : 0.0;  // lower triangle of G -> upper of S
    }
    if (tid == 0) broke = 0;
    __syncthreads();
    for (int j = 0; j < n; ++j) {
        const double piv = S[j][j];
        if (!(piv > 0.0)) {
            if (tid == 0) broke = j + 1;
        }
        __syncthreads();
        if (broke) break;
        const double dj = sqrt(piv);
        __syncthreads();
        if (tid == 0) S[j][j] = dj;
        for (int c = j + 1 + tid; c < n; c += 256) S[j][c] /= dj;
        __syncthreads();
        // trailing update of the upper triangle
        for (int e = tid; e < (n - j - 1) * (n - j - 1); e += 256) {
            const int r = j + 1 + e % (n - j - 1), c = j + 1 + e / (n - j - 1);
            if (r <= c) S[r][c] -= S[j][r] * S[j][c];
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

// Q = X / R row by row, 128 rows per CTA, R (<= 64 x 64) in shared memory.
__global__ void __launch_bounds__(128) trsm_batched_kernel(const BatchDesc* __restrict__ d, const int* status,
                                                           int pass_in_place, int which)
{
    __shared__ double Rs[64][65];
    __shared__ double dinv[64];
    const int b = blockIdx.y;
    const BatchDesc D = d[b];
    if (status[b] != 0) return;
    const int m = D.m, n = D.n;
    const long row0 = (long)blockIdx.x * 128;
    if (row0 >= m) return;  // the grid covers the largest m of the batch
    const double* Rin = which == 0 ? D.R1 : D.R2;
    for (int e = threadIdx.x; e < n * n; e += 128) {
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
        reduce_batched_kernel<<<gr, 256, 0, s>>>(d, status, nullptr);
        potrf_batched_kernel<<<count, 256, 0, s>>>(d, status, pass);
        dim3 gt(BATCH_MAX_M / 128, count);
        trsm_batched_kernel<<<gt, 128, 0, s>>>(d, status, pass, pass);
    }
    dim3 gp((64 * 64 + 255) / 256, count);
    rprod_batched_kernel<<<gp, 256, 0, s>>>(d, status);
    return cudaGetLastError();
}

cudaError_t launch_batched_factor(const BatchDesc* d, int count, int* status, int pass, cudaStream_t s)
{
    dim3 gr((BATCH_MAX_N * BATCH_MAX_N + 255) / 256, count);
    reduce_batched_kernel<<<gr, 256, 0, s>>>(d, status, nullptr);
    potrf_batched_kernel<<<count, 256, 0, s>>>(d, status, pass);
    dim3 gt(BATCH_MAX_M / 128, count);
    trsm_batched_kernel<<<gt, 128, 0, s>>>(d, status, pass, pass);
    return cudaGetLastError();
}

cudaError_t launch_batched_rprod(const BatchDesc* d, int count, int* status, cudaStream_t s)
{
    dim3 gp((BATCH_MAX_N * BATCH_MAX_N + 255) / 256, count);
    rprod_batched_kernel<<<gp, 256, 0, s>>>(d, status);
    return cudaGetLastError();
}

cudaError_t launch_batch_status_scatter(const int* st_sorted, const int* perm, int count, const DevStatus* st,
                                        int* status, cudaStream_t s)
{
    status_scatter_kernel<<<(count + 255) / 256, 256, 0, s>>>(st_sorted, perm, count, st, status);
    return cudaGetLastError();
}

}  // namespace oqr
