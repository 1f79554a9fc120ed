// Blocked Householder QR of a tall-skinny Z (the Euclidean QR of PRE-CHOLQR,
// Algorithm 2): Z = Y S, Y (m x n) with orthonormal columns, S upper
// triangular with a positive diagonal.
//
// Panels of BH_B columns.  Panel p (columns k..k+w-1 of the working copy X,
// rows k..m-1) is factored column by column by Householder reflections
// H_j = I - tau_j v_j v_j^T (LAPACK's construction: beta = -sign(x0) ||x||,
// v = x / (x0 - beta) below its leading 1, tau = (beta - x0) / beta), every
// step spread over all SMs: one kernel forms the reflector from the column's
// norm and the partial dot products with the panel's later columns, the next
// applies it and sums the next column's norm; the block partials are reduced
// in a fixed order.  The panel's reflectors are then blocked as
// I - V T V^T with T upper triangular (T_jj = tau_j, T(0:j, j) =
// -tau_j T(0:j, 0:j) V(:, 0:j)^T v_j), and the trailing columns
// C = X(k:m, k+w:n) become C - V (T^T (V^T C)): V^T C (contraction over the
// m - k rows) and V W (contraction over the w columns, formed transposed as
// W^T V^T and subtracted transposed) FP64-accurate on the tensor cores
// (launch_tc_xty), T^T (V^T C) in FP64.  Y is formed from the right:
// [I_n; 0], then I - V T V^T applied for the panels in reverse order, the
// same way.  With D = sign(diag(R)), Y D and D R give S's positive
// diagonal.
#include "oqr_internal.cuh"

namespace oqr {
namespace {

constexpr int HH_THREADS = 256;

// The rows [r0, r1) of the panel (mk rows) that block b takes.
__device__ inline void hh_rows(int mk, int* r0, int* r1)
{
    const int per = (mk + gridDim.x - 1) / gridDim.x;
    *r0 = blockIdx.x * per;
    *r1 = min(mk, *r0 + per);
}

// Fixed-order sum of v[0..len) by one warp (every block computes the same value); the values come from
// other blocks, so they are read past L1.
__device__ inline double warp_sum_fixed(const double* v, int len, int lane)
{
    double s = 0.0;
    for (int i = lane; i < len; i += 32) s += __ldcg(v + i);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// Block sum in a fixed tree; red holds HH_THREADS / 32 doubles.
__device__ inline double block_sum(double v, double* red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < HH_THREADS / 32; ++w) t += red[w];
    return t;
}

// The grid-wide barrier of the cooperative launches below is grid_barrier (oqr_internal.cuh): count and gen
// in global memory, zero before the launch; past limit_ns the status is raised and every block returns
// false at this or its next barrier, so the kernel ends.
// The panel (mk x w, leading dimension ldp) factored by w Householder reflections, one cooperative launch:
// per column, the reflector from the column's norm (partials summed in a fixed order by every block), the
// partial dot products with the later columns; a grid barrier; their sums, the update of the later columns
// and the next column's norm partials; a grid barrier.  v below the diagonal goes into P; beta, tau out.
__global__ void __launch_bounds__(HH_THREADS) hh_panel_kernel(int mk, int w, double* P, long ldp, double* part,
                                                              double* dpart, double* beta, double* tau,
                                                              unsigned* bar, DevStatus* st, uint64_t limit_ns)
{
    __shared__ double red[HH_THREADS / 32];
    __shared__ double wred[HH_THREADS / 32][BH_B];
    __shared__ double wv[BH_B];
    __shared__ double sc_s, tau_s;
    __shared__ int ok_s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int r0, r1;
    hh_rows(mk, &r0, &r1);
    // column 0's norm below its first row
    {
        double a = 0.0;
        for (int i = max(r0, 1) + threadIdx.x; i < r1; i += HH_THREADS) {
            const double x = P[i];
            a = fma(x, x, a);
        }
        a = block_sum(a, red);
        if (threadIdx.x == 0) part[blockIdx.x] = a;
    }
    if (!grid_barrier(bar, bar + 1, limit_ns, st, &ok_s, TAG_DIAG)) return;
    for (int j = 0; j < w; ++j) {
        // the reflector
        if (threadIdx.x < 32) {
            const double s2 = warp_sum_fixed(part, gridDim.x, lane);
            if (lane == 0) {
                const double x0 = __ldcg(P + j + (long)j * ldp);  // updated by the block holding row j
                double b = x0, t = 0.0, sc = 0.0;
                if (s2 > 0.0) {
                    b = -copysign(sqrt(fma(x0, x0, s2)), x0);
                    t = (b - x0) / b;
                    sc = 1.0 / (x0 - b);
                }
                sc_s = sc;
                tau_s = t;
                if (blockIdx.x == 0) {
                    beta[j] = b;
                    tau[j] = t;
                }
            }
        }
        __syncthreads();
        const double sc = sc_s, t = tau_s;
        double d[BH_B];
#pragma unroll
        for (int c = 0; c < BH_B; ++c) d[c] = 0.0;
        for (int i = max(r0, j) + threadIdx.x; i < r1; i += HH_THREADS) {
            double v = 1.0;
            if (i > j) {
                v = P[i + (long)j * ldp] * sc;
                P[i + (long)j * ldp] = v;
            }
#pragma unroll
            for (int c = 0; c < BH_B; ++c)
                if (c > j && c < w) d[c] = fma(v, P[i + (long)c * ldp], d[c]);
        }
#pragma unroll
        for (int c = 0; c < BH_B; ++c) {
            if (c > j && c < w) {
                double x = d[c];
                for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                if (lane == 0) wred[warp][c] = x;
            }
        }
        __syncthreads();
        if (threadIdx.x > j && threadIdx.x < w) {
            double x = 0.0;
            for (int q = 0; q < HH_THREADS / 32; ++q) x += wred[q][threadIdx.x];
            dpart[(long)threadIdx.x * gridDim.x + blockIdx.x] = x;
        }
        if (j + 1 == w) break;  // nothing after the last column (the same for every block)
        if (!grid_barrier(bar, bar + 1, limit_ns, st, &ok_s, TAG_DIAG)) return;
        // the update of the later columns, and the next column's norm
        for (int c = j + 1 + warp; c < w; c += HH_THREADS / 32) {
            const double x = warp_sum_fixed(dpart + (long)c * gridDim.x, gridDim.x, lane);
            if (lane == 0) wv[c] = t * x;
        }
        __syncthreads();
        double a = 0.0;
        for (int i = max(r0, j) + threadIdx.x; i < r1; i += HH_THREADS) {
            const double v = i > j ? P[i + (long)j * ldp] : 1.0;
            for (int c = j + 1; c < w; ++c) {
                const double x = fma(-wv[c], v, P[i + (long)c * ldp]);
                P[i + (long)c * ldp] = x;
                if (c == j + 1 && i > j + 1) a = fma(x, x, a);
            }
        }
        a = block_sum(a, red);
        if (threadIdx.x == 0) part[blockIdx.x] = a;
        if (!grid_barrier(bar, bar + 1, limit_ns, st, &ok_s, TAG_DIAG)) return;
    }
}

// The same factorization with each block's rows of the panel held in shared memory for the whole panel
// (rows r0..r1-1 at tile[(i - r0) * TS_LD + c]): only the partial sums, and each pivot P(j, j) (published
// by the block holding row j into xj[j]), go through global memory.  Dynamic shared memory:
// rows per block x TS_LD doubles.
constexpr int TS_LD = BH_B + 1;
__global__ void __launch_bounds__(HH_THREADS) hh_panel_smem_kernel(int mk, int w, double* P, long ldp, double* part,
                                                                   double* dpart, double* beta, double* tau,
                                                                   double* xj, int rpb, unsigned* bar,
                                                                   DevStatus* st, uint64_t limit_ns)
{
    extern __shared__ double tile[];
    __shared__ double red[HH_THREADS / 32];
    __shared__ double wred[HH_THREADS / 32][BH_B];
    __shared__ double wv[BH_B];
    __shared__ double sc_s, tau_s;
    __shared__ int ok_s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r0 = blockIdx.x * rpb, r1 = min(mk, r0 + rpb), nr = max(0, r1 - r0);
    for (int e = threadIdx.x; e < nr * w; e += HH_THREADS) {
        const int i = e % nr, c = e / nr;
        tile[i * TS_LD + c] = P[r0 + i + (long)c * ldp];
    }
    __syncthreads();
    {
        double a = 0.0;
        for (int i = max(r0, 1) + threadIdx.x; i < r1; i += HH_THREADS) {
            const double x = tile[(i - r0) * TS_LD];
            a = fma(x, x, a);
        }
        a = block_sum(a, red);
        if (threadIdx.x == 0) {
            part[blockIdx.x] = a;
            if (r0 == 0 && nr > 0) xj[0] = tile[0];
        }
    }
    if (!grid_barrier(bar, bar + 1, limit_ns, st, &ok_s, TAG_DIAG)) return;
    for (int j = 0; j < w; ++j) {
        if (threadIdx.x < 32) {
            const double x0 = __ldcg(xj + j);  // in flight with the partials below
            const double s2 = warp_sum_fixed(part, gridDim.x, lane);
            if (lane == 0) {
                double b = x0, t = 0.0, sc = 0.0;
                if (s2 > 0.0) {
                    b = -copysign(sqrt(fma(x0, x0, s2)), x0);
                    t = (b - x0) / b;
                    sc = 1.0 / (x0 - b);
                }
                sc_s = sc;
                tau_s = t;
                if (blockIdx.x == 0) {
                    beta[j] = b;
                    tau[j] = t;
                }
            }
        }
        __syncthreads();
        const double sc = sc_s, t = tau_s;
        double d[BH_B];
#pragma unroll
        for (int c = 0; c < BH_B; ++c) d[c] = 0.0;
        for (int i = max(r0, j) + threadIdx.x; i < r1; i += HH_THREADS) {
            double* row = tile + (i - r0) * TS_LD;
            double v = 1.0;
            if (i > j) {
                v = row[j] * sc;
                row[j] = v;
            }
#pragma unroll
            for (int c = 0; c < BH_B; ++c)
                if (c > j && c < w) d[c] = fma(v, row[c], d[c]);
        }
#pragma unroll
        for (int c = 0; c < BH_B; ++c) {
            if (c > j && c < w) {
                double x = d[c];
                for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                if (lane == 0) wred[warp][c] = x;
            }
        }
        __syncthreads();
        if (threadIdx.x > j && threadIdx.x < w) {
            double x = 0.0;
            for (int q = 0; q < HH_THREADS / 32; ++q) x += wred[q][threadIdx.x];
            dpart[(long)threadIdx.x * gridDim.x + blockIdx.x] = x;
        }
        if (j + 1 == w) break;  // the same for every block
        if (!grid_barrier(bar, bar + 1, limit_ns, st, &ok_s, TAG_DIAG)) return;
        {
            // this warp's columns c = j+1+warp, +8, ... (at most BH_B / 8): every partial load in flight
            // before the fixed-order sums
            constexpr int CPW = BH_B / (HH_THREADS / 32);
            double x[CPW];
#pragma unroll
            for (int q = 0; q < CPW; ++q) {
                const int c = j + 1 + warp + q * (HH_THREADS / 32);
                double a = 0.0;
                if (c < w)
                    for (int b = lane; b < (int)gridDim.x; b += 32) a += __ldcg(dpart + (long)c * gridDim.x + b);
                x[q] = a;
            }
#pragma unroll
            for (int q = 0; q < CPW; ++q) {
                for (int o = 16; o > 0; o >>= 1) x[q] += __shfl_xor_sync(0xffffffffu, x[q], o);
                const int c = j + 1 + warp + q * (HH_THREADS / 32);
                if (lane == 0 && c < w) wv[c] = t * x[q];
            }
        }
        __syncthreads();
        double a = 0.0;
        for (int i = max(r0, j) + threadIdx.x; i < r1; i += HH_THREADS) {
            double* row = tile + (i - r0) * TS_LD;
            const double v = i > j ? row[j] : 1.0;
            for (int c = j + 1; c < w; ++c) {
                const double x = fma(-wv[c], v, row[c]);
                row[c] = x;
                if (c == j + 1 && i > j + 1) a = fma(x, x, a);
            }
            if (i == j + 1) xj[j + 1] = row[j + 1];  // the next pivot, for every block
        }
        a = block_sum(a, red);
        if (threadIdx.x == 0) part[blockIdx.x] = a;
        if (!grid_barrier(bar, bar + 1, limit_ns, st, &ok_s, TAG_DIAG)) return;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nr * w; e += HH_THREADS) {
        const int i = e % nr, c = e / nr;
        P[r0 + i + (long)c * ldp] = tile[i * TS_LD + c];
    }
}

// The panel's V (unit lower trapezoidal, explicit) from P's strict lower part.
__global__ void hh_copy_v_kernel(int mk, int w, const double* __restrict__ P, long ldp, double* V, long ldv)
{
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long)mk * w) return;
    const long i = e % mk;
    const int j = (int)(e / mk);
    V[i + j * ldv] = i > j ? P[i + j * ldp] : (i == j ? 1.0 : 0.0);
}

// T (w x w, upper) from tau and G = V^T V: T_jj = tau_j, T(0:j, j) = -tau_j T(0:j, 0:j) G(0:j, j).  One block.
__global__ void hh_t_kernel(int w, const double* __restrict__ G, const double* __restrict__ tau, double* T, long ldt)
{
    __shared__ double Ts[BH_B][BH_B + 1];
    __shared__ double g[BH_B];
    const int t = threadIdx.x;
    for (int e = t; e < BH_B * BH_B; e += blockDim.x) Ts[e % BH_B][e / BH_B] = 0.0;
    __syncthreads();
    for (int j = 0; j < w; ++j) {
        if (t < j) g[t] = G[t + j * BH_B];
        __syncthreads();
        if (t < j) {
            double s = 0.0;
            for (int l = t; l < j; ++l) s = fma(Ts[t][l], g[l], s);
            Ts[t][j] = -tau[j] * s;
        }
        if (t == 0) Ts[j][j] = tau[j];
        __syncthreads();
    }
    for (int e = t; e < w * w; e += blockDim.x) T[e % w + (long)(e / w) * ldt] = Ts[e % w][e / w];
}

// S(k:k+w, k:n) = D R: the panel's R (beta on the diagonal, P's upper part above it) and the updated
// trailing rows C(0:w, :), rows scaled by d = sign(beta); dsign = d.
__global__ void panel_r_kernel(int w, int nrest, const double* __restrict__ P, long ldp, const double* __restrict__ C,
                               long ldc, const double* __restrict__ beta, double* dsign, double* S, long lds)
{
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long ncol = (long)w + nrest;
    if (e >= (long)w * ncol) return;
    const int i = (int)(e % w);
    const long j = e / w;
    const double d = beta[i] < 0.0 ? -1.0 : 1.0;
    double v;
    if (j < w) v = j < i ? 0.0 : (j == i ? beta[i] : P[i + j * ldp]);
    else v = C[i + (j - w) * ldc];
    S[i + j * lds] = d * v;
    if (j == 0) dsign[i] = d;
}

// Vt (w x rows, leading dimension ldt) = V^T for V (rows x w, leading dimension ldv).
__global__ void transpose_kernel(int rows, int w, const double* __restrict__ V, long ldv, double* Vt, long ldt)
{
    __shared__ double t[32][33];
    const int r0 = blockIdx.x * 32, c = threadIdx.y;
    {
        const int r = r0 + threadIdx.x;  // coalesced read of V along its rows
        t[threadIdx.x][c] = (r < rows && c < w) ? V[r + (long)c * ldv] : 0.0;
    }
    __syncthreads();
    const int r = r0 + threadIdx.y;
    if (threadIdx.x < w && r < rows) Vt[threadIdx.x + (long)r * ldt] = t[threadIdx.y][threadIdx.x];
}

// B(i, j) -= P(j, i) for B rows x cols (leading dimension ldb) and P cols x rows (leading dimension ldp).
__global__ void sub_transposed_kernel(int rows, int cols, const double* __restrict__ P, long ldp, double* B, long ldb)
{
    __shared__ double t[32][33];
    const int j0 = blockIdx.y * 32, i0 = blockIdx.x * 32;
    {
        const int j = j0 + threadIdx.x, i = i0 + threadIdx.y;  // coalesced read of P along j
        t[threadIdx.y][threadIdx.x] = (j < cols && i < rows) ? P[j + (long)i * ldp] : 0.0;
    }
    __syncthreads();
    const int i = i0 + threadIdx.x, j = j0 + threadIdx.y;  // coalesced update of B along i
    if (i < rows && j < cols) B[i + (long)j * ldb] -= t[threadIdx.x][threadIdx.y];
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
    // the panel kernel's blocks must all be resident (cooperative launch)
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hh_panel_kernel, HH_THREADS, 0) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    p.blocks_max = per_sm >= 2 ? 2 * sms : sms;
    // the shared-memory panel kernel: its tile and static arrays in one SM's shared memory
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, 0) != cudaSuccess) {
        cudaGetLastError();
        optin = 0;
    }
    const int static_bytes = 8 * 1024;  // red, wred, wv and scalars, rounded up
    p.smem_rows = optin > static_bytes ? (optin - static_bytes) / (TS_LD * (int)sizeof(double)) : 0;
    if (p.smem_rows > 0 &&
        cudaFuncSetAttribute(hh_panel_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             p.smem_rows * TS_LD * (int)sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        p.smem_rows = 0;
    }
    size_t o = 0;
    auto take = [&](size_t doubles) {
        const size_t r = o;
        o += (doubles + 31) & ~size_t(31);
        return r;
    };
    p.oX = take((size_t)m * n);
    p.oV = take((size_t)m * n);
    p.oT = take((size_t)p.panels * BH_B * BH_B);
    p.oD = take((size_t)p.panels * BH_B);
    p.oW = take((size_t)BH_B * n);
    p.oW2 = take((size_t)BH_B * n);
    p.oG = take((size_t)BH_B * BH_B);
    p.oBeta = take(BH_B);
    p.oTau = take(BH_B);
    p.oPart = take((size_t)p.blocks_max);
    p.oDpart = take((size_t)BH_B * p.blocks_max);
    p.oBar = take(1);
    p.oXj = take(BH_B);
    const size_t xt1 = tc_xty_bytes(m, BH_B, n), xt2 = tc_xty_bytes(BH_B, n, m);
    p.oXT = take((xt1 > xt2 ? xt1 : xt2) / sizeof(double) + 1);
    p.oVt = take((size_t)BH_B * m);
    p.oPt = take((size_t)n * m);
    p.doubles = o;
    return p;
}

cudaError_t launch_bhqr(const BhqrPlan& p, const double* Z, long ldz, double* Y, long ldy, double* S, long lds,
                        double* ws, DevStatus* st, uint64_t limit_ns, cudaStream_t s)
{
    const int m = p.m, n = p.n;
    double *X = ws + p.oX, *V = ws + p.oV, *W = ws + p.oW, *W2 = ws + p.oW2, *G = ws + p.oG;
    double *beta = ws + p.oBeta, *tau = ws + p.oTau, *part = ws + p.oPart, *dpart = ws + p.oDpart;
    unsigned* bar = reinterpret_cast<unsigned*>(ws + p.oBar);
    double *Vt = ws + p.oVt, *Pt = ws + p.oPt;
    double* xj = ws + p.oXj;
    cudaError_t e;
    if ((e = cudaMemcpy2DAsync(X, (size_t)m * sizeof(double), Z, ldz * sizeof(double), (size_t)m * sizeof(double), n,
                               cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(V, 0, (size_t)m * n * sizeof(double), s)) != cudaSuccess) return e;
    if ((e = cudaMemset2DAsync(S, lds * sizeof(double), 0, (size_t)n * sizeof(double), n, s)) != cudaSuccess) return e;
    for (int pi = 0; pi < p.panels; ++pi) {
        const int k = pi * BH_B, w = n - k < BH_B ? n - k : BH_B, mk = m - k, nrest = n - k - w;
        double* T = ws + p.oT + (size_t)pi * BH_B * BH_B;
        double* D = ws + p.oD + (size_t)pi * BH_B;
        double* P = X + k + (size_t)k * m;   // the panel, rows k.., leading dimension m
        double* Vp = V + k + (size_t)k * m;
        double* C = X + k + (size_t)(k + w) * m;
        // the panel's reflectors, column by column (one cooperative launch); each block's rows in shared
        // memory when the panel fits (one block per SM), else in global memory
        if ((e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s)) != cudaSuccess) return e;
        int mk_ = mk, w_ = w;
        long ldp_ = m;
        uint64_t lim = limit_ns;
        int rpb = (mk + p.sms - 1) / p.sms;
        if (rpb < 512) rpb = 512;
        if (rpb <= p.smem_rows) {
            int nb = (mk + rpb - 1) / rpb;
            void* args[] = {&mk_, &w_, &P, &ldp_, &part, &dpart, &beta, &tau, &xj, &rpb, &bar, &st, &lim};
            if ((e = cudaLaunchCooperativeKernel((const void*)hh_panel_smem_kernel, dim3(nb), dim3(HH_THREADS), args,
                                                 (size_t)rpb * TS_LD * sizeof(double), s)) != cudaSuccess)
                return e;
        } else {
            int nb = (mk + 511) / 512;
            nb = nb < 1 ? 1 : nb > p.blocks_max ? p.blocks_max : nb;
            void* args[] = {&mk_, &w_, &P, &ldp_, &part, &dpart, &beta, &tau, &bar, &st, &lim};
            if ((e = cudaLaunchCooperativeKernel((const void*)hh_panel_kernel, dim3(nb), dim3(HH_THREADS), args, 0,
                                                 s)) != cudaSuccess)
                return e;
        }
        // V explicit, then T from V^T V
        hh_copy_v_kernel<<<(unsigned)(((long)mk * w + 255) / 256), 256, 0, s>>>(mk, w, P, m, Vp, m);
        if ((e = launch_tc_xty(mk, w, w, Vp, m, Vp, m, G, BH_B, ws + p.oXT, st, limit_ns, p.sms, s)) != cudaSuccess)
            return e;
        transpose_kernel<<<dim3((mk + 31) / 32), dim3(32, 32), 0, s>>>(mk, w, Vp, m, Vt, BH_B);
        hh_t_kernel<<<1, 64, 0, s>>>(w, G, tau, T, BH_B);
        if (nrest > 0) {
            // C = C - V (T^T (V^T C))
            if ((e = launch_tc_xty(mk, w, nrest, Vp, m, C, m, W, BH_B, ws + p.oXT, st, limit_ns, p.sms, s)) !=
                cudaSuccess)
                return e;
            if ((e = launch_gemm_f64(GEMM_T, w, nrest, w, 1.0, T, BH_B, W, BH_B, 0.0, W2, BH_B, nullptr, 1, s)) !=
                cudaSuccess)
                return e;
            // C -= V W2, formed transposed on the tensor cores: Pt = W2^T V^T (nrest x mk), contraction w
            if ((e = launch_tc_xty(w, nrest, mk, W2, BH_B, Vt, BH_B, Pt, nrest, ws + p.oXT, st, limit_ns, p.sms,
                                   s)) != cudaSuccess)
                return e;
            sub_transposed_kernel<<<dim3((mk + 31) / 32, (nrest + 31) / 32), dim3(32, 32), 0, s>>>(mk, nrest, Pt,
                                                                                                  nrest, C, m);
        }
        const long tot = (long)w * (w + nrest);
        panel_r_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(w, nrest, P, m, C, m, beta, D,
                                                                     S + k + (size_t)k * lds, lds);
    }
    // Y = H_0 ... H_{P-1} [I_n; 0], then Y D
    identity_kernel<<<(unsigned)(((long)m * n + 255) / 256), 256, 0, s>>>(m, n, Y, ldy);
    for (int pi = p.panels - 1; pi >= 0; --pi) {
        const int k = pi * BH_B, w = n - k < BH_B ? n - k : BH_B, mk = m - k, nc = n - k;
        const double* T = ws + p.oT + (size_t)pi * BH_B * BH_B;
        const double* Vp = V + k + (size_t)k * m;
        double* B = Y + k + (size_t)k * ldy;
        if ((e = launch_tc_xty(mk, w, nc, Vp, m, B, ldy, W, BH_B, ws + p.oXT, st, limit_ns, p.sms, s)) != cudaSuccess)
            return e;
        if ((e = launch_gemm_f64(GEMM_N, w, nc, w, 1.0, T, BH_B, W, BH_B, 0.0, W2, BH_B, nullptr, 1, s)) != cudaSuccess)
            return e;
        transpose_kernel<<<dim3((mk + 31) / 32), dim3(32, 32), 0, s>>>(mk, w, Vp, m, Vt, BH_B);
        if ((e = launch_tc_xty(w, nc, mk, W2, BH_B, Vt, BH_B, Pt, nc, ws + p.oXT, st, limit_ns, p.sms, s)) !=
            cudaSuccess)
            return e;
        sub_transposed_kernel<<<dim3((mk + 31) / 32, (nc + 31) / 32), dim3(32, 32), 0, s>>>(mk, nc, Pt, nc, B, ldy);
    }
    scale_columns_kernel<<<(unsigned)(((long)m * n + 255) / 256), 256, 0, s>>>(m, n, Y, ldy, ws + p.oD);
    return cudaGetLastError();
}

}  // namespace oqr
