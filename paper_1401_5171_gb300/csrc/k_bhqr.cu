// Blocked Householder QR of a tall-skinny Z (the Euclidean QR of PRE-CHOLQR,
// Algorithm 2): Z = Y S, Y (m x n) with orthonormal columns, S upper
// triangular with a positive diagonal.
//
// Panels of BH_B columns.  Panel p (columns k..k+w-1 of the working copy X,
// rows k..m-1) is factored by the Householder TSQR (k_tsqr.cu) into an
// explicit Qp (orthonormal, m-k x w) and Rp.  Its Householder vectors V and
// triangular factor T, with (I - V T V^T)[I; 0] = Qp D, are recovered from Qp
// by an LU factorization without pivoting of Qp - [D; 0] (Ballard, Demmel,
// Grigori, Jacquelin, Nguyen and Solomonik, "Reconstructing Householder
// vectors from tall-skinny QR", 2015): V = L, T = -U D L1^{-T}, the signs D
// chosen as the elimination goes (d_j = -sign of the current pivot, so every
// pivot has magnitude at least 1).  The panel's Householder R is D Rp; the
// trailing columns C = X(k:m, k+w:n) become (I - V T V^T)^T C =
// C - V (T^T (V^T C)), and their top w rows are R's next rows.  Y is formed
// from the right: [I_n; 0], then (I - V T V^T) applied to it for the panels
// in reverse order.  Y D and D R_h give S's positive diagonal.
#include "oqr_internal.cuh"

namespace oqr {
namespace {

constexpr int HR_THREADS = 256;

// The top w x w block of Qp (w <= BH_B): LU without pivoting of Qp1 - D with the
// signs chosen on the fly; writes V's top block (L1: unit diagonal, zeros above), U,
// T = -U D L1^{-T} (upper) and d.
__global__ void __launch_bounds__(HR_THREADS) hr_top_kernel(int w, const double* __restrict__ Qp, long ldq,
                                                            double* V, long ldv, double* U, double* T, long ldt,
                                                            double* dsign)
{
    __shared__ double Y[BH_B][BH_B + 1];
    __shared__ double Mi[BH_B][BH_B + 1];  // L1^{-1}
    __shared__ double d[BH_B];
    const int tid = threadIdx.x;
    for (int e = tid; e < w * w; e += HR_THREADS) Y[e % w][e / w] = Qp[e % w + (long)(e / w) * ldq];
    __syncthreads();
    for (int j = 0; j < w; ++j) {
        if (tid == 0) {
            const double sj = Y[j][j] >= 0.0 ? -1.0 : 1.0;
            d[j] = sj;
            Y[j][j] -= sj;  // |pivot| >= 1
        }
        __syncthreads();
        const double piv = Y[j][j];
        for (int i = j + 1 + tid; i < w; i += HR_THREADS) Y[i][j] /= piv;
        __syncthreads();
        for (int e = tid; e < (w - j - 1) * (w - j - 1); e += HR_THREADS) {
            const int i = j + 1 + e % (w - j - 1), c = j + 1 + e / (w - j - 1);
            Y[i][c] = fma(-Y[i][j], Y[j][c], Y[i][c]);
        }
        __syncthreads();
    }
    // Mi = L1^{-1} (unit lower), column by column
    for (int c = tid; c < w; c += HR_THREADS) {
        for (int i = 0; i < w; ++i) Mi[i][c] = i == c ? 1.0 : 0.0;
        for (int i = c + 1; i < w; ++i) {
            double t = 0.0;
            for (int l = c; l < i; ++l) t = fma(Y[i][l], Mi[l][c], t);
            Mi[i][c] = -t;
        }
    }
    __syncthreads();
    for (int e = tid; e < w * w; e += HR_THREADS) {
        const int i = e % w, j = e / w;
        V[i + (long)j * ldv] = i > j ? Y[i][j] : (i == j ? 1.0 : 0.0);
        U[i + j * BH_B] = i <= j ? Y[i][j] : 0.0;
        // T(i, j) = -sum_k U(i, k) d_k L1^{-T}(k, j) = -sum_{k = i..j} U(i, k) d_k Mi(j, k)
        double t = 0.0;
        for (int k = i; k <= j; ++k) t = fma(Y[i][k] * d[k], Mi[j][k], t);
        T[i + (long)j * ldt] = i <= j ? -t : 0.0;
    }
    if (tid < w) dsign[tid] = d[tid];
}

// Rows w..rows-1 of V: V(i, :) = Qp(i, :) U^{-1}, one row per thread.
__global__ void __launch_bounds__(128) hr_rows_kernel(int rows, int w, const double* __restrict__ Qp, long ldq,
                                                      const double* __restrict__ U, double* V, long ldv)
{
    __shared__ double Us[BH_B][BH_B + 1];
    __shared__ double dinv[BH_B];
    for (int e = threadIdx.x; e < w * w; e += 128) Us[e % w][e / w] = U[e % w + (e / w) * BH_B];
    if (threadIdx.x < w) dinv[threadIdx.x] = 1.0 / U[threadIdx.x * (BH_B + 1)];
    __syncthreads();
    const long i = (long)w + (long)blockIdx.x * 128 + threadIdx.x;
    if (i >= rows) return;
    double x[BH_B];
#pragma unroll
    for (int j = 0; j < BH_B; ++j) {
        if (j < w) {
            double t = Qp[i + (long)j * ldq];
            for (int l = 0; l < j; ++l) t = fma(-x[l], Us[l][j], t);
            x[j] = t * dinv[j];
        }
    }
#pragma unroll
    for (int j = 0; j < BH_B; ++j)
        if (j < w) V[i + (long)j * ldv] = x[j];
}

// S(k:k+w, k:k+w) = D (D Rp) = Rp (the panel's Householder R, rows scaled by D), and
// S(k:k+w, k+w:n) = D C(0:w, :) (the panel rows of the updated trailing columns).
__global__ void panel_r_kernel(int w, int nrest, const double* __restrict__ Rp, const double* __restrict__ C, long ldc,
                               const double* __restrict__ dsign, double* S, long lds)
{
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long ncol = (long)w + nrest;
    if (e >= (long)w * ncol) return;
    const int i = (int)(e % w);
    const long j = e / w;
    double v;
    if (j < w) v = i <= j ? Rp[i + j * (long)w] : 0.0;  // D (D Rp): Rp itself
    else v = dsign[i] * C[i + (j - w) * ldc];
    S[i + j * lds] = v;
}

// Y = [I_n; 0]
__global__ void identity_kernel(int m, int n, double* Y, long ldy)
{
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long)m * n) return;
    const long i = e % m, j = e / m;
    Y[i + j * ldy] = i == j ? 1.0 : 0.0;
}

// Y(:, j) *= d_j
__global__ void scale_columns_kernel(int m, int n, double* Y, long ldy, const double* __restrict__ dsign)
{
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long)m * n) return;
    const long i = e % m, j = e / m;
    Y[i + j * ldy] *= dsign[j];
}

}  // namespace

BhqrPlan bhqr_plan(int m, int n, int sms)
{
    BhqrPlan p{};
    p.m = m;
    p.n = n;
    p.panels = (n + BH_B - 1) / BH_B;
    p.sms = sms;
    size_t ts = 0;  // the panels' TSQR workspace, the largest over the panels
    for (int pi = 0; pi < p.panels; ++pi) {
        const int k = pi * BH_B, w = n - k < BH_B ? n - k : BH_B;
        const size_t d = tsqr_plan(m - k, w).doubles;
        if (d > ts) ts = d;
    }
    p.splits_max = 2 * sms;
    size_t o = 0;
    auto take = [&](size_t doubles) {
        const size_t r = o;
        o += (doubles + 31) & ~size_t(31);
        return r;
    };
    p.oX = take((size_t)m * n);
    p.oV = take((size_t)m * n);
    p.oQp = take((size_t)m * BH_B);
    p.oRp = take((size_t)BH_B * BH_B);
    p.oU = take((size_t)BH_B * BH_B);
    p.oT = take((size_t)p.panels * BH_B * BH_B);
    p.oD = take((size_t)p.panels * BH_B);
    p.oW = take((size_t)BH_B * n);
    p.oW2 = take((size_t)BH_B * n);
    p.oSK = take(gemm_splitk_bytes(BH_B, n, p.splits_max) / sizeof(double) + 1);
    p.oTS = take(ts);
    p.doubles = o;
    return p;
}

cudaError_t launch_bhqr(const BhqrPlan& p, const double* Z, long ldz, double* Y, long ldy, double* S, long lds,
                        double* ws, cudaStream_t s)
{
    const int m = p.m, n = p.n;
    double *X = ws + p.oX, *V = ws + p.oV, *Qp = ws + p.oQp, *Rp = ws + p.oRp, *U = ws + p.oU;
    double *W = ws + p.oW, *W2 = ws + p.oW2, *SK = ws + p.oSK, *TS = ws + p.oTS;
    cudaError_t e;
    if ((e = cudaMemcpy2DAsync(X, (size_t)m * sizeof(double), Z, ldz * sizeof(double), (size_t)m * sizeof(double), n,
                               cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(V, 0, (size_t)m * n * sizeof(double), s)) != cudaSuccess) return e;
    if ((e = cudaMemset2DAsync(S, lds * sizeof(double), 0, (size_t)n * sizeof(double), n, s)) != cudaSuccess) return e;
    auto splits_for = [&](int M, int N) {
        const int tiles = ((M + 63) / 64) * ((N + 63) / 64);
        const int sp = 2 * p.sms / tiles;
        return sp < 1 ? 1 : sp > p.splits_max ? p.splits_max : sp;
    };
    for (int pi = 0; pi < p.panels; ++pi) {
        const int k = pi * BH_B, w = n - k < BH_B ? n - k : BH_B, mk = m - k, nrest = n - k - w;
        double* T = ws + p.oT + (size_t)pi * BH_B * BH_B;
        double* D = ws + p.oD + (size_t)pi * BH_B;
        double* Vp = V + k + (size_t)k * m;  // rows k.., columns k..k+w-1 of V
        double* C = X + k + (size_t)(k + w) * m;
        const TsqrPlan tp = tsqr_plan(mk, w);
        if ((e = launch_tsqr(tp, X + k + (size_t)k * m, m, Qp, mk, Rp, w, TS, s)) != cudaSuccess) return e;
        hr_top_kernel<<<1, HR_THREADS, 0, s>>>(w, Qp, mk, Vp, m, U, T, BH_B, D);
        if (mk > w) hr_rows_kernel<<<(unsigned)((mk - w + 127) / 128), 128, 0, s>>>(mk, w, Qp, mk, U, Vp, m);
        if (nrest > 0) {
            // C = C - V (T^T (V^T C))
            const int sp = splits_for(w, nrest);
            if ((e = launch_gemm_f64(GEMM_T, w, nrest, mk, 1.0, Vp, m, C, m, 0.0, W, BH_B, SK, sp, s)) != cudaSuccess)
                return e;
            if ((e = launch_gemm_f64(GEMM_T, w, nrest, w, 1.0, T, BH_B, W, BH_B, 0.0, W2, BH_B, nullptr, 1, s)) !=
                cudaSuccess)
                return e;
            if ((e = launch_gemm_f64(GEMM_N, mk, nrest, w, -1.0, Vp, m, W2, BH_B, 1.0, C, m, nullptr, 1, s)) !=
                cudaSuccess)
                return e;
        }
        const long tot = (long)w * (w + nrest);
        panel_r_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(w, nrest, Rp, C, m, D, S + k + (size_t)k * lds,
                                                                     lds);
    }
    // Y = H_0 ... H_{P-1} [I_n; 0], then Y D
    identity_kernel<<<(unsigned)(((long)m * n + 255) / 256), 256, 0, s>>>(m, n, Y, ldy);
    for (int pi = p.panels - 1; pi >= 0; --pi) {
        const int k = pi * BH_B, w = n - k < BH_B ? n - k : BH_B, mk = m - k, nc = n - k;
        const double* T = ws + p.oT + (size_t)pi * BH_B * BH_B;
        const double* Vp = V + k + (size_t)k * m;
        double* B = Y + k + (size_t)k * ldy;
        const int sp = splits_for(w, nc);
        if ((e = launch_gemm_f64(GEMM_T, w, nc, mk, 1.0, Vp, m, B, ldy, 0.0, W, BH_B, SK, sp, s)) != cudaSuccess)
            return e;
        if ((e = launch_gemm_f64(GEMM_N, w, nc, w, 1.0, T, BH_B, W, BH_B, 0.0, W2, BH_B, nullptr, 1, s)) != cudaSuccess)
            return e;
        if ((e = launch_gemm_f64(GEMM_N, mk, nc, w, -1.0, Vp, m, W2, BH_B, 1.0, B, ldy, nullptr, 1, s)) != cudaSuccess)
            return e;
    }
    scale_columns_kernel<<<(unsigned)(((long)m * n + 255) / 256), 256, 0, s>>>(m, n, Y, ldy, ws + p.oD);
    return cudaGetLastError();
}

}  // namespace oqr
