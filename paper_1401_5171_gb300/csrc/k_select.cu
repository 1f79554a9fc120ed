// The learned selector's decisions, taken on the device between the passes of
// a packed tensor-core wave (oqr_batched, OQR_BATCHED_SELECTOR).
//
// Every option starts with the same FP64-accurate Gram G0 = Z^T A Z (the
// probe).  The network reads the probe's features and picks a route per
// instance; the passes after it are the same launches for the whole wave, and
// each instance takes part in the Gram passes its route needs (gpass; the
// tensor-core launches skip the tiles of the others):
//   plain:  Q1 = Z R1^{-1} (R1 = chol(G0)); the Gram of pass 1, G1 = Q1^T A Q1,
//           then decides: ||G1 - I||_F <= tol: Q1 is the result (one pass,
//           checked: the Frobenius norm bounds the 2-norm); <= 0.5: one more
//           factor pass (A-CholQR2; a Gram within 0.5 of I leaves
//           kappa(Q1)^2 <= 3 in the A inner product, so the pass ends at
//           rounding level, Thm 2.1); larger, or a breakdown: late, below.
//   shift:  shifted A-CholQR3 (Sec. 4) from the same G0: R1 = chol(G0 + s I),
//           then two unshifted passes.  Its last pass may start from a Gram
//           farther than 0.5 from I (kappa(Z) near 1/u leaves the first two
//           passes a Q of modest condition) and still end at rounding level,
//           so the route is accepted once it completes, as shifted A-CholQR3
//           is (the defect of that Gram is reported).
//   late:   the shifted route redone from the saved G0 after pass 1 (two more
//           Grams, passes 2 and 3).
//   fp64:   FP64 A-CholQR2, run by the host after the waves.
// ||E||_F of E = P + P^T - I is summed in a fixed order (deterministic).
#include <math.h>

#include "oqr_internal.cuh"

namespace oqr {
namespace {

constexpr int ST = 256;  // threads per instance block

// ||P + P^T - I||_F of an instance's Gram partial (n x n, row-major), one block.
__device__ double defect_frobenius(const double* P, int n, double* red)
{
    double s = 0.0;
    for (int e = threadIdx.x; e < n * n; e += ST) {
        const int i = e / n, j = e % n;
        const double v = P[(size_t)i * n + j] + P[(size_t)j * n + i] - (i == j ? 1.0 : 0.0);
        s = fma(v, v, s);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < ST / 32; ++w) t += red[w];
    __syncthreads();
    return sqrt(t);
}

__global__ void __launch_bounds__(ST) sel_route_kernel(SelWave w, const int* choice)
{
    const int b = blockIdx.x;
    BatchDesc& D = w.d[b];
    const int c = choice[b];
    const int r = c == SEL_FP64 ? SEL_R_FP64 : (c == SEL_ONE || c == SEL_TWO) && w.status[b] == 0 ? SEL_R_PLAIN
                                                                                                  : SEL_R_SHIFT;
    if (r == SEL_R_PLAIN) {  // kept for a late shifted refactor
        const int nn = D.n * D.n;
        for (int e = threadIdx.x; e < nn; e += ST) D.G0[e] = D.G[e];
    }
    if (threadIdx.x == 0) {
        w.route[b] = r;
        w.mask[b] = r == SEL_R_SHIFT;
        w.status[b] = 0;
        w.orth[b] = nan("");
        w.defect[b] = nan("");
        // plain: two passes until pass 1 decides; shift: three factor passes
        D.npass = r == SEL_R_PLAIN ? 2 : r == SEL_R_SHIFT ? 3 : 0;
        w.gpass[b] = r == SEL_R_PLAIN ? 2 : r == SEL_R_SHIFT ? 3 + w.extra : 0;
        w.opt[b] = r == SEL_R_PLAIN ? SEL_TWO : r == SEL_R_SHIFT ? SEL_SHIFTED : SEL_FP64;
    }
}

__global__ void __launch_bounds__(ST) sel_decide_kernel(SelWave w, int pass)
{
    __shared__ double red[ST / 32];
    const int b = blockIdx.x;
    if (w.gpass[b] <= pass || w.status[b] != 0) return;
    BatchDesc& D = w.d[b];
    const double f = defect_frobenius(D.partials, D.n, red);
    if (threadIdx.x != 0) return;
    const int np = D.npass;
    if (w.route[b] == SEL_R_PLAIN && pass == 1) {
        if (f <= w.tol) {  // one pass, checked
            D.npass = 1;
            w.gpass[b] = 2;
            w.orth[b] = f;
            w.opt[b] = SEL_ONE;
        } else if (f <= 0.5) {  // A-CholQR2: this Gram is the last factor pass's
            w.gpass[b] = 2 + w.extra;
            w.defect[b] = f;
            w.opt[b] = SEL_TWO;
        } else {  // late: shifted A-CholQR3 from G0 (also for a NaN)
            D.npass = 4;
            w.gpass[b] = 4 + w.extra;
            w.route[b] = SEL_R_LATE;
            w.opt[b] = SEL_SHIFTED;
            w.status[b] = SEL_ST_LATE;  // skips this pass's factor
        }
        return;
    }
    if (pass == np) w.orth[b] = f;  // the extra check of the final Q
    else if (pass == np - 1) w.defect[b] = f;
}

__global__ void sel_after_factor_kernel(SelWave w, int pass)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= w.count) return;
    const int st = w.status[b];
    if (st != 0 && st != SEL_ST_LATE && w.gpass[b] > pass + 1) w.gpass[b] = pass + 1;
}

__global__ void sel_late_mask_kernel(SelWave w)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= w.count) return;
    w.mask[b] = w.status[b] == SEL_ST_LATE;
}

// G = G0 + shift I for a late instance; its status back to 0.
__global__ void __launch_bounds__(ST) sel_late_prep_kernel(SelWave w)
{
    const int b = blockIdx.x;
    if (!w.mask[b]) return;
    BatchDesc& D = w.d[b];
    const int n = D.n;
    const double sh = w.shifts[b];
    for (int e = threadIdx.x; e < n * n; e += ST) D.G[e] = D.G0[e] + (e % n == e / n ? sh : 0.0);
    if (threadIdx.x == 0) w.status[b] = 0;
}

// G += shift I on the diagonal for an instance of the mask.
__global__ void sel_shift_g_kernel(SelWave w)
{
    const int b = blockIdx.x;
    if (!w.mask[b]) return;
    BatchDesc& D = w.d[b];
    if (threadIdx.x < D.n) D.G[threadIdx.x * (D.n + 1)] += w.shifts[b];
}

}  // namespace

cudaError_t launch_sel_shift_g(const SelWave& w, cudaStream_t s)
{
    if (w.count > 0) sel_shift_g_kernel<<<w.count, 64, 0, s>>>(w);
    return cudaGetLastError();
}

cudaError_t launch_sel_route(const SelWave& w, const int* choice, cudaStream_t s)
{
    if (w.count > 0) sel_route_kernel<<<w.count, ST, 0, s>>>(w, choice);
    return cudaGetLastError();
}

cudaError_t launch_sel_decide(const SelWave& w, int pass, cudaStream_t s)
{
    if (w.count > 0) sel_decide_kernel<<<w.count, ST, 0, s>>>(w, pass);
    return cudaGetLastError();
}

cudaError_t launch_sel_after_factor(const SelWave& w, int pass, cudaStream_t s)
{
    if (w.count > 0) sel_after_factor_kernel<<<(w.count + 255) / 256, 256, 0, s>>>(w, pass);
    return cudaGetLastError();
}

cudaError_t launch_sel_late_mask(const SelWave& w, cudaStream_t s)
{
    if (w.count > 0) sel_late_mask_kernel<<<(w.count + 255) / 256, 256, 0, s>>>(w);
    return cudaGetLastError();
}

cudaError_t launch_sel_late_prep(const SelWave& w, cudaStream_t s)
{
    if (w.count > 0) sel_late_prep_kernel<<<w.count, ST, 0, s>>>(w);
    return cudaGetLastError();
}

}  // namespace oqr
