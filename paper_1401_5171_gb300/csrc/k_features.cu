// Per-instance features for the selector (no counterpart in the paper): read
// from the instance's BF16X3 normal-equation matrix G = Z^T A Z, which costs a
// small fraction of one FP64-accurate pass.  One CTA; G is n x n.
//   f0 log10(m)/4          f1 log10(n)/2          f2 n/m
//   f3 log10(max G_ii / min G_ii)/6              (Gram diagonal spread)
//   f4 max_{i!=j} |G_ij| / sqrt(G_ii G_jj)       (coherence)
//   f5 1 if the Cholesky of C = D^{-1/2} G D^{-1/2} breaks down, else 0
//   f6 breakdown column / n (0 if none)
//   f7 -log10(min pivot of C)/6, f8 log10(max pivot of C)/6  (a conditioning estimate)
//   f9 log10(||A||_F)/6    f10 log10(||Z||_F^2)/6  f11 log10(trace G / max G_ii)/3
//   f12..f15 0 (reserved)
#include <math.h>

#include "oqr_internal.cuh"

namespace oqr {
namespace {

__device__ inline double bmax(double v, double* red)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = red[0];
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) r = fmax(r, red[i]);
    return r;
}

__device__ inline double bsum(double v, double* red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += red[i];
    return r;
}

__global__ void __launch_bounds__(256) features_kernel(int m, int n, const double* __restrict__ G, long ldg,
                                                       double* C, const DevStatus* st, float* feat)
{
    __shared__ double red[8];
    __shared__ int broke;
    const int tid = threadIdx.x;
    double dmax = 0.0, dmin = INFINITY, dsum = 0.0;
    for (int i = tid; i < n; i += 256) {
        const double d = G[i + (long)i * ldg];
        dmax = fmax(dmax, d);
        dmin = fmin(dmin, d);
        dsum += d;
    }
    dmax = bmax(dmax, red);
    dmin = -bmax(-dmin, red);
    dsum = bsum(dsum, red);
    // scaled matrix (upper triangle from G's lower triangle) and coherence
    double coh = 0.0;
    for (long e = tid; e < (long)n * n; e += 256) {
        const int i = (int)(e % n), j = (int)(e / n);
        if (i > j) continue;
        const double di = G[i + (long)i * ldg], dj = G[j + (long)j * ldg];
        const double sc = (di > 0.0 && dj > 0.0) ? 1.0 / sqrt(di * dj) : 0.0;
        const double v = G[j + (long)i * ldg] * sc;
        C[i + (long)j * n] = v;
        if (i != j) coh = fmax(coh, fabs(v));
    }
    coh = bmax(coh, red);
    if (tid == 0) broke = 0;
    __syncthreads();
    double pmin = INFINITY, pmax = 0.0;
    for (int j = 0; j < n; ++j) {
        const double piv = C[j + (long)j * n];
        if (!(piv > 0.0)) {
            if (tid == 0) broke = j + 1;
        }
        __syncthreads();
        if (broke) break;
        pmin = fmin(pmin, piv);
        pmax = fmax(pmax, piv);
        const double d = sqrt(piv);
        __syncthreads();
        for (int c = j + 1 + tid; c < n; c += 256) C[j + (long)c * n] /= d;
        __syncthreads();
        for (long e = tid; e < (long)(n - j - 1) * (n - j - 1); e += 256) {
            const int r = j + 1 + (int)(e % (n - j - 1)), c = j + 1 + (int)(e / (n - j - 1));
            if (r <= c) C[r + (long)c * n] -= C[j + (long)r * n] * C[j + (long)c * n];
        }
        __syncthreads();
    }
    if (tid == 0) {
        float f[MLP_IN];
        for (int i = 0; i < MLP_IN; ++i) f[i] = 0.f;
        f[0] = (float)(log10((double)m) / 4.0);
        f[1] = (float)(log10((double)n) / 2.0);
        f[2] = (float)((double)n / m);
        f[3] = (dmin > 0.0) ? (float)(log10(dmax / dmin) / 6.0) : 4.f;
        f[4] = (float)coh;
        f[5] = broke ? 1.f : 0.f;
        f[6] = broke ? (float)broke / n : 0.f;
        f[7] = (pmin > 0.0 && pmin < INFINITY) ? (float)(-log10(pmin) / 6.0) : 0.f;
        f[8] = (pmax > 0.0) ? (float)(log10(pmax) / 6.0) : 0.f;
        f[9] = st->normA_fro > 0.0 ? (float)(log10(st->normA_fro) / 6.0) : 0.f;
        f[10] = st->normZ_fro2 > 0.0 ? (float)(log10(st->normZ_fro2) / 6.0) : 0.f;
        f[11] = (dmax > 0.0) ? (float)(log10(dsum / dmax) / 3.0) : 0.f;
        for (int i = 0; i < MLP_IN; ++i) feat[i] = f[i];
    }
}

// s = c u trace(G), added to G's diagonal (the shift of a low-precision first pass).
__global__ void trace_shift_kernel(int n, double* G, long ldg, double c, double u, DevStatus* st)
{
    __shared__ double red[8];
    if (*(volatile int*)&st->code != 0) return;
    double t = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) t += G[i + (long)i * ldg];
    t = bsum(t, red);
    const double s = c * u * t;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += 256) G[i + (long)i * ldg] += s;
    if (threadIdx.x == 0) st->shift = s;
}

// ---- features of a batch (the selector behind oqr_batched) -----------------
// Read after the first FP64-accurate normal-equation pass of each instance:
// G0 = Z^T A Z (exact to rounding, in the descriptor's G), the pass's Cholesky
// status and, when it completed, its factor R1 (descriptor's R1).  Scale-free:
//   f0 log10(m)/4       f1 log10(n)/2       f2 n/m
//   f3 log10(max G_ii / min G_ii)/6                      (Gram diagonal spread)
//   f4 max_{i!=j} |C_ij|, C = D^{-1/2} G0 D^{-1/2}       (coherence)
//   f5 1 if the Cholesky of C breaks down, f6 its column / n
//   f7 -log10(min pivot of C)/6, f8 log10(max pivot of C)/6
//   f9 log10(trace G0 / max G_ii)/3
//   f10 1 if the pass's Cholesky of G0 broke down, f11 its column / n
//   f12 log10(kappa_sketch)/8, kappa_sketch = ||R1||_F ||R1^{-1} W||_F / ||W||_F
//       with W an n x 2n Gaussian sketch (0 after a breakdown)
//   f13..f15 0
// W(i, j) comes from a counter-based generator both the library and its
// tests implement from the published definitions: SplitMix64 (Steele, Lea and
// Flood, 2014) on counters 2c and 2c + 1, c = j n + i, seed SKETCH_SEED,
// turned into two uniforms (the top 53 bits; the first shifted to (0, 1]) and
// one normal deviate by the Box-Muller transform sqrt(-2 ln u1) cos(2 pi u2).
constexpr unsigned long long SKETCH_SEED = 0x0123456789ABCDEFull;

__device__ inline unsigned long long splitmix64_at(unsigned long long counter)
{
    unsigned long long z = SKETCH_SEED + (counter + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ inline double sketch_gauss(int i, int j, int n)
{
    const unsigned long long c = (unsigned long long)j * n + i;
    const double u1 = (double)((splitmix64_at(2 * c) >> 11) + 1ull) * 0x1.0p-53;
    const double u2 = (double)(splitmix64_at(2 * c + 1) >> 11) * 0x1.0p-53;
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

// W_n (n x 2n, column-major) for every n <= 64, one after another: W_n starts at sketch_offset(n).
__host__ __device__ inline long sketch_offset(int n) { return (long)(n - 1) * n * (2 * n - 1) / 3; }

__global__ void sketch_table_kernel(double* tab, long total)
{
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int n = 1;
    while (sketch_offset(n + 1) <= t) ++n;
    const long loc = t - sketch_offset(n);
    tab[t] = sketch_gauss((int)(loc % n), (int)(loc / n), n);
}

constexpr int FEAT_PAIRS = 63 * 64 / 2;
// One CTA per instance.  The scaled Cholesky runs column by column with its trailing pairs from a table
// and thread 0 taking the next pivot while the update finishes (two block barriers per column); the
// sketch solve R1 X = W runs one column of W per thread, held in registers, column-oriented.
__global__ void __launch_bounds__(256) features_batched_kernel(const BatchDesc* __restrict__ d, const int* status,
                                                               const double* __restrict__ wtab, float* feat)
{
    __shared__ double C[64][65];
    __shared__ double srow[64];
    __shared__ double dinv[64];
    __shared__ unsigned short pair[FEAT_PAIRS];
    __shared__ double red[8];
    __shared__ double rinv_s;
    __shared__ int broke;
    const int b = blockIdx.x, tid = threadIdx.x;
    const BatchDesc D = d[b];
    const int n = D.n, m = D.m;
    const double* G = D.G;
    const int probe = status[b];
    double dmax = 0.0, dmin = INFINITY, dsum = 0.0;
    for (int i = tid; i < n; i += 256) {
        const double v = G[i + (long)i * n];
        dmax = fmax(dmax, v);
        dmin = fmin(dmin, v);
        dsum += v;
    }
    dmax = bmax(dmax, red);
    dmin = -bmax(-dmin, red);
    dsum = bsum(dsum, red);
    double coh = 0.0;
    for (int e = tid; e < n * n; e += 256) {
        const int i = e % n, j = e / n;
        if (i > j) continue;
        const double di = G[i + (long)i * n], dj = G[j + (long)j * n];
        const double sc = (di > 0.0 && dj > 0.0) ? 1.0 / sqrt(di * dj) : 0.0;
        const double v = G[j + (long)i * n] * sc;  // G's lower triangle
        C[i][j] = v;
        if (i != j) coh = fmax(coh, fabs(v));
    }
    for (int e = tid; e < FEAT_PAIRS; e += 256) {
        int c = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
        while (c * (c + 1) / 2 > e) --c;
        while ((c + 1) * (c + 2) / 2 <= e) ++c;
        pair[e] = (unsigned short)(((e - c * (c + 1) / 2) << 8) | c);
    }
    coh = bmax(coh, red);  // (its barriers also publish C and the pair table)
    double pmin = INFINITY, pmax = 0.0;  // thread 0's
    auto pivot = [&](int j) {
        const double piv = C[j][j];
        if (!(piv > 0.0)) {
            broke = j + 1;
        } else {
            pmin = fmin(pmin, piv);
            pmax = fmax(pmax, piv);
            const double r = rsqrt(piv);
            C[j][j] = piv * r;
            rinv_s = r;
        }
    };
    if (tid == 0) {
        broke = 0;
        pivot(0);
    }
    __syncthreads();
    for (int j = 0; j < n; ++j) {
        if (broke) break;
        const double rj = rinv_s;
        for (int c = j + 1 + tid; c < n; c += 256) {
            const double v = C[j][c] * rj;
            srow[c] = v;
            C[j][c] = v;
        }
        __syncthreads();
        const int w = n - j - 1;
        for (int e = tid; e < w * (w + 1) / 2; e += 256) {
            const int p = pair[e];
            const int r = j + 1 + (p >> 8), c = j + 1 + (p & 255);
            C[r][c] = fma(-srow[r], srow[c], C[r][c]);
            if (e == 0) pivot(j + 1);  // thread 0, pair (j+1, j+1)
        }
        __syncthreads();
    }
    // sketched kappa(R1): ||R1||_F ||R1^{-1} W||_F / ||W||_F
    double ksk = 0.0;
    if (probe == 0) {
        __syncthreads();
        for (int e = tid; e < n * n; e += 256) {
            const int i = e % n, j = e / n;
            C[i][j] = i <= j ? D.R1[i + (long)j * n] : 0.0;
        }
        __syncthreads();
        if (tid < n) dinv[tid] = 1.0 / C[tid][tid];
        double rf = 0.0, xf = 0.0, wf = 0.0;
        for (int e = tid; e < n * n; e += 256) rf += C[e % n][e / n] * C[e % n][e / n];
        __syncthreads();
        if (tid < 2 * n) {
            const double* wc = wtab + sketch_offset(n) + (long)tid * n;
            double x[64];  // this column of W, becoming R1^{-1} W from the bottom up
#pragma unroll
            for (int i = 0; i < 64; ++i) {
                x[i] = i < n ? wc[i] : 0.0;
                wf = fma(x[i], x[i], wf);
            }
#pragma unroll
            for (int i = 63; i >= 0; --i) {
                if (i < n) {
                    x[i] *= dinv[i];
                    xf = fma(x[i], x[i], xf);
#pragma unroll
                    for (int l = 0; l < i; ++l) x[l] = fma(-C[l][i], x[i], x[l]);
                }
            }
        }
        rf = bsum(rf, red);
        xf = bsum(xf, red);
        wf = bsum(wf, red);
        ksk = sqrt(rf) * sqrt(xf / wf);
    }
    if (tid == 0) {
        float f[MLP_IN];
        for (int i = 0; i < MLP_IN; ++i) f[i] = 0.f;
        f[0] = (float)(log10((double)m) / 4.0);
        f[1] = (float)(log10((double)n) / 2.0);
        f[2] = (float)((double)n / m);
        f[3] = (dmin > 0.0) ? (float)(log10(dmax / dmin) / 6.0) : 4.f;
        f[4] = (float)coh;
        f[5] = broke ? 1.f : 0.f;
        f[6] = broke ? (float)broke / n : 0.f;
        f[7] = (pmin > 0.0 && pmin < INFINITY) ? (float)(-log10(pmin) / 6.0) : 0.f;
        f[8] = (pmax > 0.0) ? (float)(log10(pmax) / 6.0) : 0.f;
        f[9] = (dmax > 0.0 && dsum > 0.0) ? (float)(log10(dsum / dmax) / 3.0) : 0.f;
        f[10] = probe ? 1.f : 0.f;
        f[11] = probe > 0 ? (float)probe / n : 0.f;
        f[12] = ksk > 0.0 ? (float)(log10(ksk) / 8.0) : 0.f;
        for (int i = 0; i < MLP_IN; ++i) feat[(long)b * MLP_IN + i] = f[i];
    }
}

}  // namespace

cudaError_t launch_sketch_table(double* tab, cudaStream_t s)
{
    const long total = sketch_offset(BATCH_MAX_N + 1);
    sketch_table_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(tab, total);
    return cudaGetLastError();
}

cudaError_t launch_features_batched(const BatchDesc* d, int count, const int* status, const double* wtab, float* feat,
                                    cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    features_batched_kernel<<<count, 256, 0, s>>>(d, status, wtab, feat);
    return cudaGetLastError();
}

cudaError_t launch_features(int m, int n, const double* G, long ldg, double* work, const DevStatus* st, float* feat,
                            cudaStream_t s)
{
    features_kernel<<<1, 256, 0, s>>>(m, n, G, ldg, work, st, feat);
    return cudaGetLastError();
}

cudaError_t launch_trace_shift(int n, double* G, long ldg, double c, double u, DevStatus* st, cudaStream_t s)
{
    trace_shift_kernel<<<1, 256, 0, s>>>(n, G, ldg, c, u, st);
    return cudaGetLastError();
}

}  // namespace oqr
