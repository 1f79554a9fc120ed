// Tridiagonal A (Sec. 8's second workload): A = T with diagonal d (m) and
// off-diagonal e (m - 1), T(i, i) = d_i, T(i + 1, i) = T(i, i + 1) = e_i.
//
// The normal-equation matrix G = X^T T X is formed as G = C + C^T with
// C = X^T U and U = M X, M = tril(T, -1) + diag(T) / 2, the same split the
// dense path uses (so G is exactly symmetric).  U costs 3 m n flops and is
// written once (m x n, HBM-bound); C = X^T U then runs on the FP64 GEMM or on
// the tensor cores (k_tc.cu, launch_tc_cross), O(m n^2) like the TRSM: the
// paper's normalised count for this case is 2 m n^2 per pass.
#include "oqr_internal.cuh"

namespace oqr {
namespace {

constexpr int TRI_THREADS = 256;

// U(i, c) = d_i / 2 X(i, c) + e_{i-1} X(i - 1, c)   (e_{-1} X(-1, c) = 0)
__global__ void tridiag_u_kernel(int m, int n, const double* __restrict__ d, const double* __restrict__ e,
                                 const double* __restrict__ X, long ldx, double* __restrict__ U, long ldu)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const double hd = 0.5 * d[i];
    const double lo = i > 0 ? e[i - 1] : 0.0;
    for (int c = blockIdx.y; c < n; c += gridDim.y) {
        const double* x = X + (long)c * ldx;
        const double prev = i > 0 ? x[i - 1] : 0.0;
        U[i + (long)c * ldu] = fma(lo, prev, hd * x[i]);
    }
}

__device__ inline double tri_block_sum(double v, double* red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    return t;  // valid in thread 0
}

// Per block: sum of d_i^2 + 2 e_i^2 over its rows (||T||_F^2) and of X(i, c)^2 (||X||_F^2).
__global__ void tridiag_norms_kernel(int m, int n, const double* __restrict__ d, const double* __restrict__ e,
                                     const double* __restrict__ X, long ldx, double* scratch)
{
    __shared__ double red[32];
    double sa = 0.0, sz = 0.0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (long)gridDim.x * blockDim.x) {
        sa += d[i] * d[i];
        if (i + 1 < m) sa += 2.0 * e[i] * e[i];
        for (int c = 0; c < n; ++c) {
            const double v = X[i + (long)c * ldx];
            sz += v * v;
        }
    }
    const double ta = tri_block_sum(sa, red);
    const double tz = tri_block_sum(sz, red);
    if (threadIdx.x == 0) {
        scratch[2 * blockIdx.x] = ta;
        scratch[2 * blockIdx.x + 1] = tz;
    }
}

// s = c u (m n + n (n + 1)) ||T||_F ||X||_F^2, the dense path's shift with ||A||_F = ||T||_F.
__global__ void tridiag_shift_kernel(int m, int n, int parts, const double* scratch, double c, double u,
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

// G = C + C^T (+ shift I), n x n.
__global__ void sym_plus_transpose_kernel(int n, const double* __restrict__ C, long ldc, double* G, long ldg,
                                          const double* shift_ptr, const DevStatus* st)
{
    if (*(volatile const int*)&st->code != 0) return;
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long)n * n) return;
    const long r = e % n, c = e / n;
    double v = C[r + c * ldc] + C[c + r * ldc];
    if (r == c && shift_ptr) v += *shift_ptr;
    G[r + c * ldg] = v;
}

}  // namespace

cudaError_t launch_tridiag_u(int m, int n, const double* d, const double* e, const double* X, long ldx, double* U,
                             long ldu, cudaStream_t s)
{
    if (m <= 0 || n <= 0) return cudaSuccess;
    const dim3 grid((unsigned)((m + TRI_THREADS - 1) / TRI_THREADS), (unsigned)(n < 64 ? n : 64));
    tridiag_u_kernel<<<grid, TRI_THREADS, 0, s>>>(m, n, d, e, X, ldx, U, ldu);
    return cudaGetLastError();
}

cudaError_t launch_tridiag_norms_and_shift(int m, int n, const double* d, const double* e, const double* X, long ldx,
                                           double c, double u, double* scratch, int scratch_len, DevStatus* st,
                                           cudaStream_t s)
{
    int parts = scratch_len / 2;
    const int need = (m + TRI_THREADS - 1) / TRI_THREADS;
    if (parts > need) parts = need;
    if (parts < 1) return cudaErrorInvalidValue;
    tridiag_norms_kernel<<<parts, TRI_THREADS, 0, s>>>(m, n, d, e, X, ldx, scratch);
    tridiag_shift_kernel<<<1, 32, 0, s>>>(m, n, parts, scratch, c, u, st);
    return cudaGetLastError();
}

cudaError_t launch_sym_plus_transpose(int n, const double* C, long ldc, double* G, long ldg, const double* shift_ptr,
                                      const DevStatus* st, cudaStream_t s)
{
    const long tot = (long)n * n;
    sym_plus_transpose_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(n, C, ldc, G, ldg, shift_ptr, st);
    return cudaGetLastError();
}

}  // namespace oqr
