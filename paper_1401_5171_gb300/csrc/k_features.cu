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

}  // namespace

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
