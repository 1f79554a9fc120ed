// The generalized least-squares solve of Sec. 1, x = R^{-1} Q^T A b, and its
// product with A: C = A B for a symmetric A read from its lower triangle.
//
// C = A B reads A's lower triangle (m^2/2 doubles) once per group of right-hand
// sides, with two FP64 FMAs per stored element and right-hand side; on GB300
// (about 0.19 flop per byte of HBM bandwidth at FP64) those FMAs, not HBM, bound
// it even for one right-hand side.  A's lower
// triangle is cut into 64 x 64 tiles (I, J), I >= J, each read from memory
// exactly once.  With M = tril(A, -1) + diag(A)/2, A = M + M^T, and tile (I, J)
// of M contributes M_IJ B_J to block row I of C and M_IJ^T B_I to block row J.
// A CTA stages its tile in shared memory and forms both products from there;
// each product is written as a per-tile partial, and a second kernel sums, for
// every row, the partials of its block row and block column in a fixed order,
// so the result is deterministic and no atomics are used.  The right-hand
// sides are processed SY_KMAX at a time (a larger k re-reads A per group).
#include "oqr_internal.cuh"

namespace oqr {
namespace {

constexpr int SY_T = 64;        // tile edge
constexpr int SY_LD = SY_T + 1;  // shared-memory column pitch (doubles): column reads hit distinct banks
constexpr int SY_THREADS = 256;
constexpr int SY_KMAX = 8;       // right-hand sides per pass over A

// Tile t of the lower triangle in row order: I (I + 1) / 2 <= t < (I + 1) (I + 2) / 2.
__device__ inline void tile_of(long t, int* I, int* J)
{
    long i = (long)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while (i * (i + 1) / 2 > t) --i;
    while ((i + 1) * (i + 2) / 2 <= t) ++i;
    *I = (int)i;
    *J = (int)(t - i * (i + 1) / 2);
}

__device__ inline long tile_index(int I, int J) { return (long)I * (I + 1) / 2 + J; }

// part: per tile, a row partial (M_IJ B_J, 64 x KC) then a column partial (M_IJ^T B_I, 64 x KC),
// each element (r, kk) at r * KC + kk.  KC is the exact number of right-hand sides of the launch: on
// GB300 the FP64 FMAs (two per stored element and right-hand side), not HBM, bound this kernel.
template <int KC>
__global__ void __launch_bounds__(SY_THREADS) symm_tiles_kernel(int m, const double* __restrict__ A, long lda,
                                                                 const double* __restrict__ B, long ldb,
                                                                 double* __restrict__ part, long ntiles)
{
    __shared__ double tile[SY_T * SY_LD];
    __shared__ double bI[SY_T * KC], bJ[SY_T * KC];
    __shared__ double red[4][SY_T * KC];
    __shared__ int tij[2];
    const int tid = threadIdx.x;
    for (long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        if (tid == 0) tile_of(t, &tij[0], &tij[1]);
        __syncthreads();
        const int I = tij[0], J = tij[1];
        const long r0 = (long)I * SY_T, c0 = (long)J * SY_T;
        // the tile of M: below the diagonal as stored, the diagonal halved, zero above it and past m
        double v[SY_T * SY_T / SY_THREADS];
#pragma unroll
        for (int q = 0; q < SY_T * SY_T / SY_THREADS; ++q) {
            const int e = tid + q * SY_THREADS, r = e % SY_T, c = e / SY_T;
            const long gr = r0 + r, gc = c0 + c;
            v[q] = (gr < m && gc < m && gr >= gc) ? __ldg(A + gr + gc * lda) : 0.0;
        }
#pragma unroll
        for (int q = 0; q < SY_T * SY_T / SY_THREADS; ++q) {
            const int e = tid + q * SY_THREADS, r = e % SY_T, c = e / SY_T;
            tile[r + c * SY_LD] = (r0 + r == c0 + c) ? 0.5 * v[q] : v[q];
        }
        for (int e = tid; e < SY_T * KC; e += SY_THREADS) {
            const int r = e % SY_T, kk = e / SY_T;
            bI[r * KC + kk] = r0 + r < m ? B[r0 + r + kk * ldb] : 0.0;
            bJ[r * KC + kk] = c0 + r < m ? B[c0 + r + kk * ldb] : 0.0;
        }
        __syncthreads();
        const int x = tid % SY_T, q = tid / SY_T;  // a row (or column) of the tile, a quarter of the other axis
        double acc[KC], acc2[KC];
#pragma unroll
        for (int kk = 0; kk < KC; ++kk) acc[kk] = acc2[kk] = 0.0;
        // row partial: sum over the quarter's columns of M(x, c) B_J(c); column partial: over its rows of
        // M(r, x) B_I(r)
#pragma unroll 4
        for (int c = q * 16; c < q * 16 + 16; ++c) {
            const double a = tile[x + c * SY_LD], at = tile[c + x * SY_LD];
#pragma unroll
            for (int kk = 0; kk < KC; ++kk) {
                acc[kk] = fma(a, bJ[c * KC + kk], acc[kk]);
                acc2[kk] = fma(at, bI[c * KC + kk], acc2[kk]);
            }
        }
#pragma unroll
        for (int kk = 0; kk < KC; ++kk) red[q][x * KC + kk] = acc[kk];
        __syncthreads();
        double* prow = part + (size_t)(2 * t) * SY_T * KC;
        for (int e = tid; e < SY_T * KC; e += SY_THREADS)
            prow[e] = ((red[0][e] + red[1][e]) + red[2][e]) + red[3][e];
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < KC; ++kk) red[q][x * KC + kk] = acc2[kk];
        __syncthreads();
        double* pcol = prow + SY_T * KC;
        for (int e = tid; e < SY_T * KC; e += SY_THREADS)
            pcol[e] = ((red[0][e] + red[1][e]) + red[2][e]) + red[3][e];
        __syncthreads();  // the tile, bI, bJ and red are rewritten by the next tile
    }
}

// C(i, kk) = sum_{J <= I} rowpart(I, J)(r, kk) + sum_{I' >= I} colpart(I', I)(r, kk), i = 64 I + r.
__global__ void symm_reduce_kernel(int m, int kc, int nb, const double* __restrict__ part, double* C, long ldc)
{
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long)m * kc) return;
    const long i = e % m;
    const int kk = (int)(e / m);
    const int I = (int)(i / SY_T), r = (int)(i % SY_T);
    const size_t tsz = (size_t)SY_T * kc;
    double s = 0.0;
    for (int J = 0; J <= I; ++J) s += part[2 * tile_index(I, J) * tsz + (size_t)r * kc + kk];
    for (int I2 = I; I2 < nb; ++I2) s += part[(2 * tile_index(I2, I) + 1) * tsz + (size_t)r * kc + kk];
    C[i + (long)kk * ldc] = s;
}

// X(:, j) = R^{-1} Y(:, j): back substitution, one warp per right-hand side,
// x_i = (y_i - sum_{l > i} r_il x_l) / r_ii with the sum over l in a fixed
// lane order (each lane sums its strided share, then a fixed shuffle tree).
__global__ void upper_solve_kernel(int n, int k, const double* __restrict__ R, long ldr, const double* Y, long ldy,
                                   double* X, long ldx)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= k) return;
    const double* y = Y + (long)warp * ldy;
    double* x = X + (long)warp * ldx;
    for (int i = n - 1; i >= 0; --i) {
        double s = 0.0;
        for (int l = i + 1 + lane; l < n; l += 32) s = fma(R[i + (long)l * ldr], x[l], s);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) x[i] = (y[i] - s) / R[i + (long)i * ldr];
        __syncwarp();
    }
}

}  // namespace

size_t symm_workspace_doubles(int m, int k)
{
    const long nb = (m + SY_T - 1) / SY_T;
    const long ntiles = nb * (nb + 1) / 2;
    const int kc = k < SY_KMAX ? k : SY_KMAX;
    return (size_t)ntiles * 2 * SY_T * kc;
}

cudaError_t launch_symm(int m, int k, const double* A, long lda, const double* B, long ldb, double* C, long ldc,
                        double* part, int sms, cudaStream_t s)
{
    if (m <= 0 || k <= 0) return cudaSuccess;
    const int nb = (m + SY_T - 1) / SY_T;
    const long ntiles = (long)nb * (nb + 1) / 2;
    const long grid = ntiles < 4L * sms ? ntiles : 4L * sms;
    for (int k0 = 0; k0 < k; k0 += SY_KMAX) {
        const int kc = k - k0 < SY_KMAX ? k - k0 : SY_KMAX;
        const double* Bk = B + (long)k0 * ldb;
        switch (kc) {
            case 1: symm_tiles_kernel<1><<<(unsigned)grid, SY_THREADS, 0, s>>>(m, A, lda, Bk, ldb, part, ntiles); break;
            case 2: symm_tiles_kernel<2><<<(unsigned)grid, SY_THREADS, 0, s>>>(m, A, lda, Bk, ldb, part, ntiles); break;
            case 3: symm_tiles_kernel<3><<<(unsigned)grid, SY_THREADS, 0, s>>>(m, A, lda, Bk, ldb, part, ntiles); break;
            case 4: symm_tiles_kernel<4><<<(unsigned)grid, SY_THREADS, 0, s>>>(m, A, lda, Bk, ldb, part, ntiles); break;
            case 5: symm_tiles_kernel<5><<<(unsigned)grid, SY_THREADS, 0, s>>>(m, A, lda, Bk, ldb, part, ntiles); break;
            case 6: symm_tiles_kernel<6><<<(unsigned)grid, SY_THREADS, 0, s>>>(m, A, lda, Bk, ldb, part, ntiles); break;
            case 7: symm_tiles_kernel<7><<<(unsigned)grid, SY_THREADS, 0, s>>>(m, A, lda, Bk, ldb, part, ntiles); break;
            default: symm_tiles_kernel<8><<<(unsigned)grid, SY_THREADS, 0, s>>>(m, A, lda, Bk, ldb, part, ntiles); break;
        }
        const long tot = (long)m * kc;
        symm_reduce_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(m, kc, nb, part, C + (long)k0 * ldc, ldc);
    }
    return cudaGetLastError();
}

cudaError_t launch_upper_solve(int n, int k, const double* R, long ldr, const double* Y, long ldy, double* X,
                               long ldx, cudaStream_t s)
{
    if (n <= 0 || k <= 0) return cudaSuccess;
    const int warps_per_block = 4;
    upper_solve_kernel<<<(k + warps_per_block - 1) / warps_per_block, 32 * warps_per_block, 0, s>>>(n, k, R, ldr, Y,
                                                                                                  ldy, X, ldx);
    return cudaGetLastError();
}

}  // namespace oqr
