// Euclidean QR of a tall-skinny Z by Householder reflections on a reduction
// tree (TSQR): the "[Y, S] = qr(Z)" of PRE-CHOLQR (Algorithm 2, Sec. 3), whose
// analysis needs Y orthonormal to working precision and Z = Y S + dZ with a
// small dZ, which Householder QR gives.
//
// Leaves: Z's rows in blocks of b0 = max(n, 256) rows (the last block takes
// the remainder, b0 <= rows < 2 b0); one CTA factors each block in place
// (reflectors below the diagonal, R on and above it, tau per column).  Tree:
// the leaves' R factors are stacked two at a time (three for the last node of
// an odd count) and factored again, level by level, until one R remains.  A
// stacked node's reflector j touches only row j of its first triangle and rows
// 0..j of the others, so those are the only rows a node visits.  The root's R
// gets a positive diagonal (S = D R, D = diag(sign r_jj)), and Y = Q_E is
// formed top-down: the root applies its reflectors to [D; 0], each node's
// result is cut into its children's n x n blocks, and each leaf applies its
// reflectors to [X; 0] into its rows of Y.  Every reflector is
// H = I - tau v v^T with v_j = 1 (LAPACK's convention): beta = -sign(alpha)
// sqrt(alpha^2 + sigma^2), tau = (beta - alpha) / beta, v = x / (alpha - beta),
// and tau = 0 (no reflection) when the column is already zero below the
// diagonal.  One CTA per block works in global memory (a leaf block of
// 256 x 256 doubles is 512 KB and stays in L2).
#include "oqr_internal.cuh"

namespace oqr {
namespace {

constexpr int TS_THREADS = 256;
constexpr int TS_WARPS = TS_THREADS / 32;

__device__ inline double ts_block_sum(double v, double* red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < TS_WARPS; ++k) t += red[k];  // the same order in every thread
    __syncthreads();
    return t;
}

// The rows of a block below row j that column j's reflector touches, in a
// fixed enumeration k = 0, 1, ...: dense blocks all rows j+1 .. rows-1;
// stacked triangles (kids > 1 children of n rows each) rows c n + r for
// c = 1 .. kids-1, r = 0 .. j.
// A stacked node has at most three children, so row k of the enumeration is
// n + k for the second child and 2 n + (k - j - 1) for the third.
struct Active {
    bool tri;
    int rows, n, j, kids;
    __device__ int count() const { return tri ? (kids - 1) * (j + 1) : rows - j - 1; }
    __device__ int row(int k) const { return tri ? (k <= j ? n + k : 2 * n + (k - j - 1)) : j + 1 + k; }
};

// Block geometry of node t at a level: leaves (tri = false) of b0 rows (the
// last takes the rest of m), or stacked nodes of 2 (3 for the last of an odd
// child count) triangles of n rows.
struct Geo {
    long off;
    int rows, kids;
};
__device__ inline Geo leaf_geo(int t, int count, int m, int b0)
{
    Geo g;
    g.off = (long)t * b0;
    g.rows = t == count - 1 ? m - t * b0 : b0;
    g.kids = 1;
    return g;
}
__device__ inline Geo node_geo(int t, int count_below, int n)
{
    Geo g;
    g.kids = (t == count_below / 2 - 1 && (count_below & 1)) ? 3 : 2;
    g.off = (long)2 * t * n;
    g.rows = g.kids * n;
    return g;
}

// Columns c0 .. n-1 of X (ld) -= tau (x_jc + v^T x_c) v for the reflector of
// column j (v_j = 1 at row j, the active rows below it in v, a column of the
// factored block).  Each warp takes its columns CG at a time, so that CG
// columns' loads are in flight together (the block is in L2, and one column
// at a time leaves the warp waiting on two round trips per column).
constexpr int CG = 4;
__device__ inline void apply_reflector(double* X, long ld, const double* v, const Active& act, double tj, int c0,
                                       int n, int warp, int lane)
{
    const int na = act.count(), j = act.j;
    for (int cb = c0 + warp * CG; cb < n; cb += TS_WARPS * CG) {
        double w[CG];
#pragma unroll
        for (int u = 0; u < CG; ++u) w[u] = 0.0;
        for (int k = lane; k < na; k += 32) {
            const int r = act.row(k);
            const double vr = v[r];
#pragma unroll
            for (int u = 0; u < CG; ++u)
                if (cb + u < n) w[u] = fma(vr, X[r + (long)(cb + u) * ld], w[u]);
        }
#pragma unroll
        for (int u = 0; u < CG; ++u) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) w[u] += __shfl_xor_sync(0xffffffffu, w[u], o);
            if (cb + u < n) w[u] = tj * (w[u] + X[j + (long)(cb + u) * ld]);
        }
        for (int k = lane; k < na; k += 32) {
            const int r = act.row(k);
            const double vr = v[r];
#pragma unroll
            for (int u = 0; u < CG; ++u)
                if (cb + u < n) X[r + (long)(cb + u) * ld] = fma(-w[u], vr, X[r + (long)(cb + u) * ld]);
        }
        if (lane == 0) {
#pragma unroll
            for (int u = 0; u < CG; ++u)
                if (cb + u < n) X[j + (long)(cb + u) * ld] -= w[u];
        }
    }
}

// Householder QR of each block of a level, in place.
__global__ void __launch_bounds__(TS_THREADS) tsqr_factor_kernel(double* V, long ld, int n, int count, int m, int b0,
                                                                 int tri, int count_below, double* tau)
{
    __shared__ double red[TS_WARPS];
    const int t = blockIdx.x;
    if (t >= count) return;
    const Geo g = tri ? node_geo(t, count_below, n) : leaf_geo(t, count, m, b0);
    double* X = V + g.off;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int j = 0; j < n; ++j) {
        const Active act{tri != 0, g.rows, n, j, g.kids};
        const int na = act.count();
        double s = 0.0;
        for (int k = tid; k < na; k += TS_THREADS) {
            const double x = X[act.row(k) + (long)j * ld];
            s = fma(x, x, s);
        }
        const double sigma2 = ts_block_sum(s, red);
        const double alpha = X[j + (long)j * ld];
        double beta = alpha, tj = 0.0, scale = 0.0;
        if (sigma2 > 0.0) {
            const double nrm = sqrt(fma(alpha, alpha, sigma2));
            beta = alpha >= 0.0 ? -nrm : nrm;
            tj = (beta - alpha) / beta;
            scale = 1.0 / (alpha - beta);
        }
        if (sigma2 > 0.0)
            for (int k = tid; k < na; k += TS_THREADS) X[act.row(k) + (long)j * ld] *= scale;  // v below row j
        __syncthreads();
        if (sigma2 > 0.0)  // trailing columns: x_c -= tau (x_jc + v^T x_c) v, with v_j = 1
            apply_reflector(X, ld, X + (long)j * ld, act, tj, j + 1, n, warp, lane);
        if (tid == 0) {
            X[j + (long)j * ld] = beta;
            tau[(long)t * n + j] = tj;
        }
        __syncthreads();
    }
}

// S_next rows [t n, (t + 1) n) = the upper triangle of node t's top n rows (zeros below).
__global__ void tsqr_gather_r_kernel(const double* V, long ld, int n, int count, int m, int b0, int tri,
                                     int count_below, double* S, long lds)
{
    const int t = blockIdx.y;
    const Geo g = tri ? node_geo(t, count_below, n) : leaf_geo(t, count, m, b0);
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < (long)n * n; e += (long)gridDim.x * blockDim.x) {
        const int r = (int)(e % n), c = (int)(e / n);
        S[(long)t * n + r + (long)c * lds] = r <= c ? V[g.off + r + (long)c * ld] : 0.0;
    }
}

// The root: S = D R with D = diag(sign r_jj) (sign(0) = +1), and the root's
// block X = D.
__global__ void tsqr_root_kernel(const double* Rt, long ldr, int n, double* S, long lds, double* X, long ldx)
{
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < (long)n * n; e += (long)gridDim.x * blockDim.x) {
        const int r = (int)(e % n), c = (int)(e / n);
        const double dr = Rt[r + (long)r * ldr] < 0.0 ? -1.0 : 1.0;
        S[r + (long)c * lds] = r <= c ? dr * Rt[r + (long)c * ldr] : 0.0;
        X[r + (long)c * ldx] = r == c ? dr : 0.0;
    }
}

// Y_t = H_t [X_t; 0] for every block t of a level: X_t is rows [t n, (t + 1) n)
// of Xin; Y_t goes to rows [off_t, off_t + rows_t) of Y (ld ldy).  The
// reflectors are applied last to first.
__global__ void __launch_bounds__(TS_THREADS) tsqr_apply_kernel(const double* V, long ld, int n, int count, int m,
                                                                int b0, int tri, int count_below, const double* tau,
                                                                const double* Xin, long ldxin, double* Y, long ldy)
{
    const int t = blockIdx.x;
    if (t >= count) return;
    const Geo g = tri ? node_geo(t, count_below, n) : leaf_geo(t, count, m, b0);
    const double* Vt = V + g.off;
    double* Yt = Y + g.off;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (long e = tid; e < (long)g.rows * n; e += TS_THREADS) {
        const long r = e % g.rows, c = e / g.rows;
        Yt[r + c * ldy] = r < n ? Xin[(long)t * n + r + c * ldxin] : 0.0;
    }
    __syncthreads();
    for (int j = n - 1; j >= 0; --j) {
        const double tj = tau[(long)t * n + j];
        if (tj != 0.0) {
            const Active act{tri != 0, g.rows, n, j, g.kids};
            apply_reflector(Yt, ldy, Vt + (long)j * ld, act, tj, 0, n, warp, lane);
        }
        __syncthreads();
    }
}

}  // namespace

TsqrPlan tsqr_plan(int m, int n)
{
    TsqrPlan p{};
    p.m = m;
    p.n = n;
    p.b0 = n > 256 ? n : 256;
    p.leaves = m / p.b0 < 1 ? 1 : m / p.b0;
    int count = p.leaves;
    p.levels = 0;
    while (count > 1) {
        count /= 2;
        p.level_count[p.levels++] = count;
    }
    size_t doubles = (size_t)m * n + (size_t)p.leaves * n;  // leaves' blocks and taus
    size_t below = p.leaves;
    for (int l = 0; l < p.levels; ++l) {
        doubles += below * n * n;                       // stacked R's of the children (factored in place)
        doubles += (size_t)p.level_count[l] * n;        // taus
        doubles += below * n * n;                       // the children's X blocks
        below = p.level_count[l];
    }
    doubles += (size_t)n * n;  // the root's X
    p.doubles = doubles;
    return p;
}

cudaError_t launch_tsqr(const TsqrPlan& p, const double* Z, long ldz, double* Y, long ldy, double* S, long lds,
                        double* ws, cudaStream_t s)
{
    const int m = p.m, n = p.n;
    double* V0 = ws;
    double* tau0 = V0 + (size_t)m * n;
    double* cur = tau0 + (size_t)p.leaves * n;
    double* Sl[32];
    double* taul[32];
    double* Xl[32];  // Xl[l]: the X blocks of level l's children (count_below blocks)
    size_t below = p.leaves;
    for (int l = 0; l < p.levels; ++l) {
        Sl[l] = cur;
        cur += below * n * n;
        taul[l] = cur;
        cur += (size_t)p.level_count[l] * n;
        Xl[l] = cur;
        cur += below * n * n;
        below = p.level_count[l];
    }
    double* Xroot = cur;
    cudaError_t e = cudaMemcpy2DAsync(V0, (size_t)m * 8, Z, (size_t)ldz * 8, (size_t)m * 8, n,
                                      cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    // leaves
    tsqr_factor_kernel<<<p.leaves, TS_THREADS, 0, s>>>(V0, m, n, p.leaves, m, p.b0, 0, 0, tau0);
    // tree
    int count_below = p.leaves;
    const double* Vprev = V0;
    long ldprev = m;
    int tri_prev = 0, cb_prev = 0;
    for (int l = 0; l < p.levels; ++l) {
        const long lds_l = (long)count_below * n;
        tsqr_gather_r_kernel<<<dim3(8, count_below), 256, 0, s>>>(Vprev, ldprev, n, count_below, m, p.b0, tri_prev,
                                                                   cb_prev, Sl[l], lds_l);
        tsqr_factor_kernel<<<p.level_count[l], TS_THREADS, 0, s>>>(Sl[l], lds_l, n, p.level_count[l], m, p.b0, 1,
                                                                   count_below, taul[l]);
        Vprev = Sl[l];
        ldprev = lds_l;
        tri_prev = 1;
        cb_prev = count_below;
        count_below = p.level_count[l];
    }
    // root: S = D R, X = D
    tsqr_root_kernel<<<8, 256, 0, s>>>(Vprev, ldprev, n, S, lds, Xroot, n);
    // Y top-down: level l's nodes write their children's X blocks, the leaves write Y
    const double* Xin = Xroot;
    long ldxin = n;
    for (int l = p.levels - 1; l >= 0; --l) {
        const int cb = l == 0 ? p.leaves : p.level_count[l - 1];
        const long lds_l = (long)cb * n;
        tsqr_apply_kernel<<<p.level_count[l], TS_THREADS, 0, s>>>(Sl[l], lds_l, n, p.level_count[l], m, p.b0, 1, cb,
                                                                  taul[l], Xin, ldxin, Xl[l], lds_l);
        Xin = Xl[l];
        ldxin = lds_l;
    }
    tsqr_apply_kernel<<<p.leaves, TS_THREADS, 0, s>>>(V0, m, n, p.leaves, m, p.b0, 0, 0, tau0, Xin, ldxin, Y, ldy);
    return cudaGetLastError();
}

}  // namespace oqr
