// Fused normal-equation (Gram) kernel, FP64: lines 1-2 of Algorithm 1
// (B = A Z, C = Z^T B) without ever storing B.
//
// A is symmetric and read from its lower triangle only.  Write
// A = M + M^T with M = tril(A, -1) + diag(A)/2; then
//   Z^T A Z = P + P^T,   P = Z^T (M Z),
// so the product with A costs m^2 n multiply-adds instead of 2 m^2 n and A's
// upper triangle is never touched.  The lower triangle is cut into row blocks
// I of BM rows; row block I needs the k-steps kb (BK columns each) with
// kb*BK < min((I+1)*BM, m).  All k-steps of all row blocks are laid out in one
// sequence and cut into `splits` equal contiguous ranges.  CTA (s, c) walks
// range s for column chunk c of Z (BN columns): for every row-block segment
// of its range it accumulates T = M(I, range) Z(range, chunk) in registers
// (FP64 FMA), then adds Z(I, :)^T T into its private partial P_s(:, chunk).
// A second kernel sums the partials in a fixed order, G = sum_s P_s + P_s^T,
// which is exactly symmetric and bit-reproducible run to run.
//
// GB300 runs FP64 at about 2 FMA per clock per SM (DFMA; the FP64 mma.sync
// path is slower), so this kernel is bound by the FP64 pipe, not by memory:
// a 128 x 64 x 16 k-step is 131072 FMAs against 24 KB of tiles.  Tiles are
// staged by TMA (cp.async.bulk.tensor) into a 4-deep ring with mbarrier
// completion; every wait is time-limited.  Matrices whose base or leading
// dimension TMA cannot address use the same kernel with plain loads.
#include <math.h>
#include <stdio.h>

#include "oqr_internal.cuh"

namespace oqr {
namespace {

constexpr int BM = 128;       // rows of A per row block
constexpr int BN = 64;        // columns of Z per chunk
constexpr int BK = 16;        // k-step
constexpr int STAGES = 4;     // TMA ring depth
constexpr int THREADS = 256;  // 16 x 16 threads, 8 x 4 FP64 accumulators each
constexpr int A_TILE = BM * BK;   // doubles, stored [BK][BM]
constexpr int Z_TILE = BK * BN;   // doubles, stored [BN][BK]
constexpr int STAGE_DOUBLES = A_TILE + Z_TILE;
constexpr int EPI_ZC = 32;        // Z columns staged per epilogue round
constexpr int SMEM_DOUBLES = STAGES * STAGE_DOUBLES;  // 12288 = 96 KB
constexpr size_t SMEM_BYTES = SMEM_DOUBLES * sizeof(double) + STAGES * sizeof(uint64_t);
static_assert(BM * BN + BM * EPI_ZC <= SMEM_DOUBLES, "epilogue must fit in the ring");
constexpr uint32_t STAGE_TX_BYTES = STAGE_DOUBLES * sizeof(double);

// k-steps of row block I.
__device__ __host__ inline long ksteps_of(long I, long m)
{
    long hi = (I + 1) * BM;
    if (hi > m) hi = m;
    return (hi + BK - 1) / BK;
}

// First global k-step index of row block I (all earlier blocks are full).
__device__ __host__ inline long cum_of(long I) { return 4 * I * (I + 1); }
static_assert(BM / BK == 8, "cum_of assumes 8 k-steps per full row block");

__device__ inline long block_of_step(long u, long nblocks)
{
    long I = (long)((sqrt(1.0 + (double)u) - 1.0) * 0.5);
    if (I < 0) I = 0;
    if (I > nblocks - 1) I = nblocks - 1;
    while (I > 0 && cum_of(I) > u) --I;
    while (I + 1 < nblocks && cum_of(I + 1) <= u) ++I;
    return I;
}

struct Args {
    const double* A;
    long lda;
    const double* Z;
    long ldz;
    double* partials;  // splits x (n x n), row-major per split
    DevStatus* st;
    long steps;
    int m, n, splits;
    uint64_t limit_ns;
};

// Zero (diag: halve) the part of an A tile on or above the diagonal.
__device__ inline void mask_diag_tile(double* As, long row0, long col0)
{
    for (int e = threadIdx.x; e < A_TILE; e += THREADS) {
        const int r = e % BM, k = e / BM;
        const long gr = row0 + r, gc = col0 + k;
        if (gc > gr) As[e] = 0.0;
        else if (gc == gr) As[e] *= 0.5;
    }
}

__device__ inline void load_tiles_plain(const Args& a, double* As, double* Zs, long I, long kb, int chunk)
{
    const long row0 = I * BM, col0 = kb * BK;
    for (int e = threadIdx.x; e < A_TILE; e += THREADS) {
        const int r = e % BM, k = e / BM;
        const long gr = row0 + r, gc = col0 + k;
        As[e] = (gr < a.m && gc < a.m) ? a.A[gr + gc * a.lda] : 0.0;
    }
    for (int e = threadIdx.x; e < Z_TILE; e += THREADS) {
        const int k = e % BK, c = e / BK;
        const long gr = col0 + k, gc = (long)chunk * BN + c;
        Zs[e] = (gr < a.m && gc < a.n) ? a.Z[gr + gc * a.ldz] : 0.0;
    }
}

// Epilogue of one row-block segment: P_s(:, chunk) (+)= Z(I rows, :)^T T.
__device__ void epilogue(const Args& a, double* smem, double (&acc)[8][4], long I, int chunk, int split,
                         bool first)
{
    const int tid = threadIdx.x, ty = tid & 15, tx = tid >> 4;
    double* Ts = smem;                 // [BM][BN], row-major (c fastest)
    double* Zc = smem + BM * BN;       // [BM][EPI_ZC]
    __syncthreads();                   // ring no longer read
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) Ts[(ty + 16 * i) * BN + tx + 16 * j] = acc[i][j];
    const int c = tid & (BN - 1);
    const int rg = tid >> 6;  // 0..3
    const long row0 = I * BM;
    const long gcol = (long)chunk * BN + c;
    double* P = a.partials + (size_t)split * a.n * a.n;
    for (int r0 = 0; r0 < a.n; r0 += EPI_ZC) {
        __syncthreads();
        for (int e = tid; e < BM * EPI_ZC; e += THREADS) {
            const int i = e / EPI_ZC, rr = e % EPI_ZC;
            const long gr = row0 + i, gc = r0 + rr;
            Zc[e] = (gr < a.m && gc < a.n) ? a.Z[gr + gc * a.ldz] : 0.0;
        }
        __syncthreads();
        double out[EPI_ZC / 4];
#pragma unroll
        for (int t = 0; t < EPI_ZC / 4; ++t) out[t] = 0.0;
        for (int i = 0; i < BM; ++i) {
            const double tv = Ts[i * BN + c];
#pragma unroll
            for (int t = 0; t < EPI_ZC / 4; ++t) out[t] = fma(Zc[i * EPI_ZC + rg + 4 * t], tv, out[t]);
        }
        if (gcol < a.n) {
#pragma unroll
            for (int t = 0; t < EPI_ZC / 4; ++t) {
                const int r = r0 + rg + 4 * t;
                if (r < a.n) {
                    double* p = P + (size_t)r * a.n + gcol;
                    *p = first ? out[t] : *p + out[t];
                }
            }
        }
    }
    fence_proxy_async_smem();  // generic writes to the ring precede the next TMA writes
    __syncthreads();
}

template <bool USE_TMA>
__global__ void __launch_bounds__(THREADS, 2)
    gram_f64_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapZ, Args a)
{
    extern __shared__ __align__(128) double smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + SMEM_DOUBLES);  // after the ring
    const int tid = threadIdx.x, ty = tid & 15, tx = tid >> 4;
    const int split = blockIdx.x, chunk = blockIdx.y;
    if (*(volatile int*)&a.st->code != 0) return;
    if (USE_TMA && (smem_u32(smem) & 127u) != 0) {  // TMA destinations need 128-byte alignment here
        if (tid == 0) raise_status(a.st, OQR_ERR_UNSUPPORTED, 0, TAG_GRAM);
        return;
    }

    const long nblocks = (a.m + BM - 1) / BM;
    const long u0 = a.steps * split / a.splits, u1 = a.steps * (split + 1) / a.splits;
    if (USE_TMA && tid == 0) {
        tma_prefetch_desc(&mapA);
        tma_prefetch_desc(&mapZ);
        for (int s = 0; s < STAGES; ++s) mbar_init(&full[s], 1);
        fence_barrier_init();
    }
    __syncthreads();

    bool first = true;
    long g = 0;  // running k-step counter of this CTA (slot/parity bookkeeping)
    long u = u0;
    while (u < u1) {
        const long I = block_of_step(u, nblocks);
        const long kb0 = u - cum_of(I);
        long nk = ksteps_of(I, a.m) - kb0;
        if (nk > u1 - u) nk = u1 - u;
        const long diag_kb = (I * BM) / BK;  // first k-step that touches the diagonal block

        double acc[8][4];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

        if (USE_TMA && tid == 0) {
            fence_proxy_async_smem();
            for (long p = 0; p < nk && p < STAGES; ++p) {
                const int slot = (int)((g + p) % STAGES);
                double* As = smem + slot * STAGE_DOUBLES;
                mbar_expect_tx(&full[slot], STAGE_TX_BYTES);
                tma_load_2d(As, &mapA, &full[slot], (int)(I * BM), (int)((kb0 + p) * BK));
                tma_load_2d(As + A_TILE, &mapZ, &full[slot], (int)((kb0 + p) * BK), chunk * BN);
            }
        }
        for (long it = 0; it < nk; ++it) {
            const long kb = kb0 + it;
            const int slot = (int)((g + it) % STAGES);
            double* As = smem + slot * STAGE_DOUBLES;
            double* Zs = As + A_TILE;
            if (USE_TMA) {
                const uint32_t parity = (uint32_t)(((g + it) / STAGES) & 1);
                const bool ok = mbar_wait(&full[slot], parity, a.limit_ns);
                if (__syncthreads_or(!ok)) {
                    if (tid == 0) {
                        raise_status(a.st, OQR_ERR_TIMEOUT, (int)kb, TAG_GRAM);
                        // drain what is still in flight before the CTA exits
                        for (long q = it; q < nk && q < it + STAGES; ++q) {
                            const int sl = (int)((g + q) % STAGES);
                            mbar_wait(&full[sl], (uint32_t)(((g + q) / STAGES) & 1), exit_drain_ns(a.limit_ns));
                        }
                    }
                    return;
                }
                // every thread finished k-step it-1: refill its slot
                if (tid == 0 && it >= 1 && it - 1 + STAGES < nk) {
                    const long q = it - 1 + STAGES;
                    const int sl = (int)((g + q) % STAGES);
                    double* Ar = smem + sl * STAGE_DOUBLES;
                    mbar_expect_tx(&full[sl], STAGE_TX_BYTES);
                    tma_load_2d(Ar, &mapA, &full[sl], (int)(I * BM), (int)((kb0 + q) * BK));
                    tma_load_2d(Ar + A_TILE, &mapZ, &full[sl], (int)((kb0 + q) * BK), chunk * BN);
                }
            } else {
                __syncthreads();
                load_tiles_plain(a, As, Zs, I, kb, chunk);
                __syncthreads();
            }
            if (kb >= diag_kb) {  // tile meets the diagonal block: apply M's mask
                mask_diag_tile(As, I * BM, kb * BK);
                if (USE_TMA) fence_proxy_async_smem();
                __syncthreads();
            }
#pragma unroll
            for (int k = 0; k < BK; ++k) {
                double av[8], zv[4];
#pragma unroll
                for (int i = 0; i < 8; ++i) av[i] = As[k * BM + ty + 16 * i];
#pragma unroll
                for (int j = 0; j < 4; ++j) zv[j] = Zs[(tx + 16 * j) * BK + k];
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], zv[j], acc[i][j]);
            }
        }
        g += nk;
        epilogue(a, smem, acc, I, chunk, split, first);
        first = false;
        u += nk;
    }
    if (first) {  // empty range: the partial still has to be defined
        double* P = a.partials + (size_t)split * a.n * a.n;
        for (long e = tid; e < (long)a.n * BN; e += THREADS) {
            const long r = e / BN, c = (long)chunk * BN + e % BN;
            if (c < a.n) P[r * a.n + c] = 0.0;
        }
    }
}

__global__ void gram_reduce_kernel(const double* __restrict__ partials, int n, int splits, double* G, long ldg,
                                   const double* shift_ptr, const DevStatus* st)
{
    if (*(volatile const int*)&st->code != 0) return;
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long)n * n) return;
    const long r = e % n, c = e / n;
    const size_t nn = (size_t)n * n;
    double s = 0.0;
    for (int p = 0; p < splits; ++p) {
        const double* P = partials + p * nn;
        s += P[r * n + c] + P[c * n + r];  // the same two terms, in either orientation
    }
    if (r == c && shift_ptr) s += *shift_ptr;
    G[r + c * ldg] = s;
}

}  // namespace

GramPlan gram_plan(int m, int n, int sm_count)
{
    GramPlan p;
    p.m = m;
    p.n = n;
    p.bn = BN;
    p.chunks = (n + BN - 1) / BN;
    const long nblocks = (m + BM - 1) / BM;
    p.steps = cum_of(nblocks - 1) + ksteps_of(nblocks - 1, m);
    long target = 2L * sm_count / p.chunks;  // two resident CTAs per SM
    if (target < 1) target = 1;
    if (target > p.steps) target = p.steps;
    p.splits = (int)target;
    return p;
}

size_t gram_partials_bytes(const GramPlan& p) { return (size_t)p.splits * p.n * p.n * sizeof(double); }

cudaError_t launch_gram_f64(const GramPlan& p, const double* A, long lda, const double* Z, long ldz,
                            double* partials, DevStatus* st, uint64_t limit_ns, cudaStream_t s)
{
    Args a{A, lda, Z, ldz, partials, st, p.steps, p.m, p.n, p.splits, limit_ns};
    CUtensorMap mA{}, mZ{};
    bool tma = p.m >= 2 && tma_ok(A, lda, 8) && tma_ok(Z, ldz, 8);
    if (tma) {
        tma = make_tensor_map_2d(&mA, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 8, A, p.m, p.m, lda, BM, BK) &&
              make_tensor_map_2d(&mZ, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 8, Z, p.m, p.n, ldz, BK, BN);
    }
    const size_t smem = SMEM_BYTES;
    dim3 grid(p.splits, p.chunks);
    if (tma) {
        cudaFuncSetAttribute(gram_f64_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        gram_f64_kernel<true><<<grid, THREADS, smem, s>>>(mA, mZ, a);
    } else {
        cudaFuncSetAttribute(gram_f64_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        gram_f64_kernel<false><<<grid, THREADS, smem, s>>>(mA, mZ, a);
    }
    return cudaGetLastError();
}

cudaError_t launch_gram_reduce(const GramPlan& p, const double* partials, double* G, long ldg,
                               const double* shift_ptr, DevStatus* st, cudaStream_t s)
{
    const long total = (long)p.n * p.n;
    const int threads = 256;
    gram_reduce_kernel<<<(unsigned)((total + threads - 1) / threads), threads, 0, s>>>(partials, p.n, p.splits, G,
                                                                                      ldg, shift_ptr, st);
    return cudaGetLastError();
}

}  // namespace oqr
