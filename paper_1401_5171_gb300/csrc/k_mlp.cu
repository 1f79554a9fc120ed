// Selector network: features (16 floats per instance) -> MLP 16 -> 64 -> 64 -> 4
// (ReLU) -> logits over the factorization options.  The paper has no such
// component; it chooses, per instance, how many normal-equation passes and
// which precision to run.
//
// Parameters are one flat FP32 array (MLP_PARAMS floats):
//   W1[64][16], b1[64], W2[64][64], b2[64], W3[4][64], b3[4]   (row-major).
// Forward: FP32, or BF16 inference (weights and activations rounded to BF16,
// products accumulated in FP32).  Training: softmax cross-entropy, mean over
// the minibatch; the gradient is formed in two deterministic phases (per
// sample, then per parameter summing samples in index order) and Adam updates
// the parameters in place.
#include <cuda_bf16.h>
#include <math.h>

#include "oqr_internal.cuh"

namespace oqr {
namespace {

constexpr int F = MLP_IN, H = MLP_HIDDEN, O = MLP_OUT;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + H * F, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H,
              OFF_W3 = OFF_B2 + H, OFF_B3 = OFF_W3 + O * H;
static_assert(OFF_B3 + O == MLP_PARAMS, "parameter layout");

__device__ inline float bf(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

template <bool BF16>
__global__ void __launch_bounds__(128) mlp_forward_kernel(int B, const float* __restrict__ X,
                                                          const float* __restrict__ P, float* logits, int* choice)
{
    __shared__ float w[MLP_PARAMS];
    for (int i = threadIdx.x; i < MLP_PARAMS; i += blockDim.x) w[i] = BF16 ? bf(P[i]) : P[i];
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= B) return;
    float x[F], h1[H], h2[H];
#pragma unroll
    for (int j = 0; j < F; ++j) x[j] = BF16 ? bf(X[(size_t)s * F + j]) : X[(size_t)s * F + j];
    for (int i = 0; i < H; ++i) {
        float a = w[OFF_B1 + i];
#pragma unroll
        for (int j = 0; j < F; ++j) a = fmaf(w[OFF_W1 + i * F + j], x[j], a);
        a = a > 0.f ? a : 0.f;
        h1[i] = BF16 ? bf(a) : a;
    }
    for (int i = 0; i < H; ++i) {
        float a = w[OFF_B2 + i];
        for (int j = 0; j < H; ++j) a = fmaf(w[OFF_W2 + i * H + j], h1[j], a);
        a = a > 0.f ? a : 0.f;
        h2[i] = BF16 ? bf(a) : a;
    }
    int best = 0;
    float bv = -INFINITY;
    for (int i = 0; i < O; ++i) {
        float a = w[OFF_B3 + i];
        for (int j = 0; j < H; ++j) a = fmaf(w[OFF_W3 + i * H + j], h2[j], a);
        if (logits) logits[(size_t)s * O + i] = a;
        if (a > bv) {
            bv = a;
            best = i;
        }
    }
    if (choice) choice[s] = best;
}

// Phase 1, one thread per sample: forward in FP32, the sample's loss, and the
// back-propagated signals d_logits (O), d_h2 (H), d_h1 (H) together with the
// activations h1, h2 (H each), stored per sample in scratch.
constexpr int SCR = 4 * H + O + 1;  // floats per sample: h1, h2, dh2, dh1, dlogit, loss

__global__ void __launch_bounds__(128) mlp_backprop_kernel(int B, const float* __restrict__ X, const int* __restrict__ y,
                                                           const float* __restrict__ P, float* scr)
{
    __shared__ float w[MLP_PARAMS];
    for (int i = threadIdx.x; i < MLP_PARAMS; i += blockDim.x) w[i] = P[i];
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= B) return;
    float* out = scr + (size_t)s * SCR;
    float* h1 = out;
    float* h2 = out + H;
    float* dh2 = out + 2 * H;
    float* dh1 = out + 3 * H;
    float* dl = out + 4 * H;
    const float* x = X + (size_t)s * F;
    for (int i = 0; i < H; ++i) {
        float a = w[OFF_B1 + i];
        for (int j = 0; j < F; ++j) a = fmaf(w[OFF_W1 + i * F + j], x[j], a);
        h1[i] = a > 0.f ? a : 0.f;
    }
    for (int i = 0; i < H; ++i) {
        float a = w[OFF_B2 + i];
        for (int j = 0; j < H; ++j) a = fmaf(w[OFF_W2 + i * H + j], h1[j], a);
        h2[i] = a > 0.f ? a : 0.f;
    }
    float z[O], zmax = -INFINITY;
    for (int i = 0; i < O; ++i) {
        float a = w[OFF_B3 + i];
        for (int j = 0; j < H; ++j) a = fmaf(w[OFF_W3 + i * H + j], h2[j], a);
        z[i] = a;
        zmax = fmaxf(zmax, a);
    }
    float se = 0.f;
    for (int i = 0; i < O; ++i) se += expf(z[i] - zmax);
    const int lab = y[s];
    out[4 * H + O] = logf(se) + zmax - z[lab];  // -log softmax(z)[lab]
    const float invB = 1.0f / (float)B;
    for (int i = 0; i < O; ++i) dl[i] = (expf(z[i] - zmax) / se - (i == lab ? 1.f : 0.f)) * invB;
    for (int j = 0; j < H; ++j) {
        float a = 0.f;
        for (int i = 0; i < O; ++i) a = fmaf(w[OFF_W3 + i * H + j], dl[i], a);
        dh2[j] = h2[j] > 0.f ? a : 0.f;
    }
    for (int j = 0; j < H; ++j) {
        float a = 0.f;
        for (int i = 0; i < H; ++i) a = fmaf(w[OFF_W2 + i * H + j], dh2[i], a);
        dh1[j] = h1[j] > 0.f ? a : 0.f;
    }
}

// Phase 2, one thread per parameter: sums the per-sample products in sample order.
__global__ void mlp_param_grad_kernel(int B, const float* __restrict__ X, const float* __restrict__ scr, float* grad,
                                      float* loss)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p == MLP_PARAMS && loss) {
        float l = 0.f;
        for (int s = 0; s < B; ++s) l += scr[(size_t)s * SCR + 4 * H + O];
        *loss = l / (float)B;
        return;
    }
    if (p >= MLP_PARAMS) return;
    float g = 0.f;
    for (int s = 0; s < B; ++s) {
        const float* r = scr + (size_t)s * SCR;
        const float* h1 = r;
        const float* h2 = r + H;
        const float* dh2 = r + 2 * H;
        const float* dh1 = r + 3 * H;
        const float* dl = r + 4 * H;
        float t;
        if (p < OFF_B1) t = dh1[(p - OFF_W1) / F] * X[(size_t)s * F + (p - OFF_W1) % F];
        else if (p < OFF_W2) t = dh1[p - OFF_B1];
        else if (p < OFF_B2) t = dh2[(p - OFF_W2) / H] * h1[(p - OFF_W2) % H];
        else if (p < OFF_W3) t = dh2[p - OFF_B2];
        else if (p < OFF_B3) t = dl[(p - OFF_W3) / H] * h2[(p - OFF_W3) % H];
        else t = dl[p - OFF_B3];
        g += t;
    }
    grad[p] = g;
}

__global__ void adam_kernel(int n, float* P, const float* __restrict__ g, float* m, float* v, float lr, float b1,
                            float b2, float eps, int t)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float mi = b1 * m[i] + (1.f - b1) * g[i];
    const float vi = b2 * v[i] + (1.f - b2) * g[i] * g[i];
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / (1.f - powf(b1, (float)t));
    const float vh = vi / (1.f - powf(b2, (float)t));
    P[i] -= lr * mh / (sqrtf(vh) + eps);
}

}  // namespace

size_t mlp_scratch_bytes(int B) { return (size_t)B * SCR * sizeof(float); }

cudaError_t launch_mlp_forward(int B, const float* X, const float* P, int bf16, float* logits, int* choice,
                               cudaStream_t s)
{
    if (B <= 0) return cudaSuccess;
    const int blocks = (B + 127) / 128;
    if (bf16) mlp_forward_kernel<true><<<blocks, 128, 0, s>>>(B, X, P, logits, choice);
    else mlp_forward_kernel<false><<<blocks, 128, 0, s>>>(B, X, P, logits, choice);
    return cudaGetLastError();
}

cudaError_t launch_mlp_grad(int B, const float* X, const int* y, const float* P, float* grad, float* loss, float* scr,
                            cudaStream_t s)
{
    if (B <= 0) return cudaErrorInvalidValue;
    mlp_backprop_kernel<<<(B + 127) / 128, 128, 0, s>>>(B, X, y, P, scr);
    mlp_param_grad_kernel<<<(MLP_PARAMS + 1 + 127) / 128, 128, 0, s>>>(B, X, scr, grad, loss);
    return cudaGetLastError();
}

cudaError_t launch_adam(int n, float* P, const float* g, float* m, float* v, float lr, float b1, float b2, float eps,
                        int t, cudaStream_t s)
{
    adam_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, P, g, m, v, lr, b1, b2, eps, t);
    return cudaGetLastError();
}

}  // namespace oqr
