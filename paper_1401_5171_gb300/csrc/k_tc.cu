// Tensor-core (tcgen05, BF16 -> FP32 in TMEM) products for the
// normal-equation matrix of Algorithm 1 (lines 1-2: B = A Z, C = Z^T B).
//
// The paper forms both products in FP64 (MKL).  On GB300 FP64 runs at about
// 1/1600 of the BF16 tensor rate, so this file computes them from BF16 slices
// of the FP64 operands on the 5th-generation tensor cores, in one of three modes:
//
//  * BF16X3 (preconditioning passes): x = hi + lo with hi = bf16(x),
//    lo = bf16(x - hi); the product sums hi*hi + hi*lo + lo*hi in one FP32
//    TMEM accumulator.  Relative accuracy about 2^-16 per product plus FP32
//    accumulation.
//
//  * EMU64 (FP64-accurate final pass; error-free slicing in the manner of
//    Ozaki, Ogita, Oishi and Rump 2012): for every row of the left operand and
//    every 256-long chunk of the contraction index k, a power-of-two exponent e
//    is taken from the chunk's largest magnitude, and x 2^(7-e) is written as
//    sum_s d_s 2^(-8s), s = 0..6, with integers d_s in [-128, 128], rounded to
//    nearest at 2^-48; slice s is stored as d_s 2^(-8s) (exact in BF16).  The
//    right operand is sliced the same way per column.  The slice products
//    (s, t) of one level L = s + t + 2 are integers of magnitude at most 2^14
//    in the units of that level; the at most 4 products of a level L <= 5
//    summed over one 256-long chunk stay within 2^24 and are exact in their
//    FP32 accumulator; L6 (5 products) is exact unless its sum passes 2^24,
//    and then rounds by at most 2^0.32 units, below 2^-53 of the chunk's
//    largest possible value.  Levels 7 and 8 share one accumulator (their
//    rounding is below 2^-58 of it).  After every chunk the drain warps scale the
//    accumulators by the chunk's row and column powers of two and add them
//    into a double-float (hi, lo) register sum; with 7 slices the truncation
//    error is about 2^-55 relative to the chunk's largest term.
//
//  * FP8 E4M3 with per-(row, 128-chunk) power-of-two scales, one product,
//    drained every chunk.
//
// Kernel structure (one CTA per SM, persistent over work items): warp 0 is
// the TMA producer (all slice tiles of A and B per k-step), warp 1 allocates
// TMEM and holds the single MMA-issuing thread, and the remaining warps drain
// the accumulators with tcgen05.ld (TMEM lane = row), several warps per TMEM
// lane quarter.  tc_kernel serves BF16X3 and FP8 (one accumulator);
// emu_kernel serves EMU64 with its drain overlapping the next chunk's MMAs.
// An item is (128-row tile I of the left operand, a piece of its k range,
// an N-column chunk of the right operand); its result goes to its own
// slot, and a reduce kernel sums the slots of each tile in a fixed order.
// In triangular mode the left operand is M = tril(A,-1) + diag(A)/2 (rows i,
// columns k <= i), so row tile I stops at k = 128 (I + 1).
//
// Every mbarrier wait is bounded by %globaltimer; on timeout the CTA records
// OQR_ERR_TIMEOUT, stops issuing, drains in-flight copies with a bounded wait,
// frees its TMEM and returns.
#include <cuda_bf16.h>
#include <math.h>

#include "oqr_internal.cuh"

namespace oqr {
namespace {

constexpr int TM = 128;            // UMMA M (rows of the left operand per tile)
constexpr int KCH_EMU = 256;       // exponent chunk of the EMU64 family (FP64_TC, TC2): exact level sums
constexpr int KCH_FP8 = 128;       // exponent chunk of FP8 (128-long scale blocks)
// exponent chunk (and split tile width) of a mode: 256 for the EMU64 family (1, 3), 128 for FP8 (2) and for
// the BF16X3 split (0, which records no exponents)
__host__ __device__ constexpr int kch_of(int mode) { return (mode == 1 || mode == 3) ? KCH_EMU : KCH_FP8; }
constexpr int EXP_NONE = -100000;  // exponent of an all-zero chunk
constexpr int TC_THREADS = 320;   // producer warp, MMA warp, 8 drain warps

// ------------------------------------------------------------ splitting ----
// GB300 issues about two FP64 instructions per clock per SM, so an FP64
// operation per element of A costs about a millisecond at m = 32768.  The
// splits therefore work on the FP64 bit pattern with integer instructions:
// x = (-1)^s M 2^E with M the 53-bit integer significand.

struct Bits {
    unsigned long long M;  // integer significand (implicit bit included for normal numbers)
    int Eb;                // biased exponent, 1 for zero and subnormals
    bool neg;
};

__device__ inline Bits bits_of(double x)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const int b = (int)((u >> 52) & 0x7FF);
    const unsigned long long f = u & 0xFFFFFFFFFFFFFull;
    Bits r;
    r.M = b ? (f | (1ull << 52)) : f;
    r.Eb = b ? b : 1;
    r.neg = (u >> 63) != 0;
    return r;
}

// Round-to-nearest-even right shift of a non-negative integer.
__device__ inline unsigned long long rne_shift(unsigned long long v, int sh)
{
    if (sh <= 0) return v;
    if (sh >= 64) return 0;
    const unsigned long long q = v >> sh, rem = v & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    return q + ((rem > half || (rem == half && (q & 1))) ? 1 : 0);
}

// EMU64 slices of x for chunk exponent e (|x| < 2^e): with y = x 2^(7-e),
// Y = RNE(y 2^48) is an integer below 2^55, written in balanced base 256,
// Y = sum_s d_s 2^(8(6-s)), d_s integers in [-128, 128].  The slices are
// stored with their weight, out[s] = d_s 2^(-8s) (exact in BF16), so that
// y = sum_s out[s] up to the rounding at 2^-48 and every slice product
// carries the weight of its level.
__device__ inline void emu_slices7(double x, int e, float* out)
{
    const Bits b = bits_of(x);
    const int k = b.Eb - e - 1020;  // y 2^48 = M 2^k, k <= 2 because |x| < 2^e
    long long Y = 0;
    if (b.M != 0) {
        // k < 0: round M 2^k to the nearest integer, ties to even, as (M + 2^(-k-1) - 1 + lsb) >> -k with
        // lsb the kept part's last bit (no overflow: M < 2^53); M 2^k < 1/2 for -k >= 54
        unsigned long long mag;
        if (k >= 0) {
            mag = b.M << k;
        } else {
            const int sh = -k;
            mag = sh >= 54 ? 0ull : (b.M + ((1ull << (sh - 1)) - 1ull) + ((b.M >> sh) & 1ull)) >> sh;
        }
        Y = b.neg ? -(long long)mag : (long long)mag;
    }
    // Balanced digits: with W = Y + sum_{t<7} 128 256^t, byte t of W is d + 128 for the digit of weight
    // 256^t (the digits d + 128 lie in [0, 255], so the representation of W has no carries), and
    // d_0 = W / 2^48 - 128 in [-128, 128].  One 64-bit add replaces a carry chain.  d 2^(-8s) is then
    // formed exactly from the byte by a magic-number float: 2^(23-8s) + (d + 128) 2^(-8s) (the byte
    // placed in the low mantissa bits), minus 2^(23-8s) + 128 2^(-8s).
    const unsigned long long W = (unsigned long long)Y + 0x0080808080808080ull;
    const unsigned lo = (unsigned)W;
    const unsigned hi = (unsigned)(W >> 32);
#pragma unroll
    for (int t = 0; t < 6; ++t) {  // byte t of W -> digit s = 6 - t
        const int sd = 6 - t;
        const unsigned base = 0x4B000000u - ((8u * sd) << 23);
        const unsigned bits = __byte_perm(t < 4 ? lo : hi, base, 0x7650u | (unsigned)(t & 3));
        out[sd] = __uint_as_float(bits) - __uint_as_float(base + 128u);
    }
    const int top = (int)((long long)W >> 48) - 128;  // d_0
    out[0] = __int_as_float(0x4B000000 + top + 128) - __int_as_float(0x4B000000 + 128);
}

// FP8 E4M3 code of x 2^(8-e) (|x| < 2^e, so the value is below 256 <= 448),
// round-to-nearest-even: 4 significant bits for normal values (exponent bias
// 7), q 2^-9 (q = 0..7) below 2^-6.  Bit 7 is the sign.
__device__ inline unsigned char e4m3_code(double x, int e)
{
    const Bits b = bits_of(x);
    if (b.M == 0) return 0;
    const int msb = 63 - __clzll((long long)b.M);
    const int E = b.Eb - 1075;
    int p = msb + E + 8 - e;  // unbiased exponent of the scaled value
    unsigned int code;
    if (p >= -6) {
        unsigned long long q = rne_shift(b.M, msb - 3);  // 8..16
        if (q == 16) {
            q = 8;
            ++p;
        }
        if (p > 8) {  // saturate (not reached for |x| < 2^e)
            p = 8;
            q = 14;
        }
        code = ((unsigned)(p + 7) << 3) | (unsigned)(q - 8);
    } else {
        const unsigned long long q = rne_shift(b.M, e - E - 17);  // RNE(value 2^9), 0..8
        code = q >= 8 ? (1u << 3) : (unsigned)q;
    }
    return (unsigned char)(code | (b.neg ? 0x80u : 0u));
}

// hi = bf16(x), lo = bf16(x - hi), both round-to-nearest-even (8 significant bits).
// Valid for |x| within the normal FP32 range, as BF16 itself.
__device__ inline void bf16x2_split(double x, __nv_bfloat16& hi, __nv_bfloat16& lo)
{
    const Bits b = bits_of(x);
    if (b.M == 0) {
        hi = lo = __float2bfloat16_rn(0.0f);
        return;
    }
    const int E = b.Eb - 1075;  // x = +-M 2^E
    const int msb = 63 - __clzll((long long)b.M);
    const int sh = msb - 7;
    float hf, lf = 0.0f;
    if (sh <= 0) {
        hf = ldexpf((float)b.M, E);
    } else {
        const unsigned long long q = rne_shift(b.M, sh);  // <= 256
        hf = ldexpf((float)q, E + sh);
        const long long r = (long long)b.M - (long long)(q << sh);
        if (r != 0) {
            const unsigned long long ar = (unsigned long long)(r < 0 ? -r : r);
            const int msb2 = 63 - __clzll((long long)ar);
            const int sh2 = msb2 - 7 > 0 ? msb2 - 7 : 0;
            const unsigned long long q2 = rne_shift(ar, sh2);
            lf = ldexpf((float)q2, E + sh2);
            if (r < 0) lf = -lf;
        }
    }
    if (b.neg) {
        hf = -hf;
        lf = -lf;
    }
    hi = __float2bfloat16_rn(hf);  // exact: at most 8 significant bits
    lo = __float2bfloat16_rn(lf);
}

// Slices of one element for chunk exponent e (MODE 1: S exact BF16 slices,
// pre-scaled; MODE 0: BF16 hi/lo).
template <int MODE>
__device__ inline void slice_element(double x, int e, int S, float* sl)
{
    (void)S;
    if constexpr (MODE == 0) {
        __nv_bfloat16 hi, lo;
        bf16x2_split(x, hi, lo);
        sl[0] = __bfloat162float(hi);
        sl[1] = __bfloat162float(lo);
    } else {
        if (e == EXP_NONE) {
#pragma unroll
            for (int t = 0; t < 7; ++t) sl[t] = 0.f;
        } else {
            emu_slices7(x, e, sl);
        }
    }
}

// Chunk exponent of the magnitudes held by a warp (VPL values per lane): the
// exponent field's maximum over the high words (32-bit warp reductions), and
// EXP_NONE when every value is zero.
template <int VPL>
__device__ inline int warp_chunk_exponent(const double* v)
{
    unsigned hk = 0, nz = 0;
#pragma unroll
    for (int j = 0; j < VPL; ++j) {
        const unsigned long long u = (unsigned long long)__double_as_longlong(v[j]);
        const unsigned h = (unsigned)(u >> 32) & 0x7FFFFFFFu;
        hk = h > hk ? h : hk;
        nz |= h | (unsigned)u;
    }
    hk = __reduce_max_sync(0xffffffffu, hk);
    nz = __reduce_or_sync(0xffffffffu, nz);
    if (nz == 0) return EXP_NONE;
    const int b = (int)(hk >> 20);
    return b ? b - 1022 : -1021;
}

// Writes VPL consecutive plane elements (k .. k+VPL-1) of every slice: one
// vector store per plane (2 B per element for BF16 planes, 1 B for E4M3).
template <int MODE, int VPL>
__device__ inline void store_run(__nv_bfloat16* planes, size_t plane, size_t off, int S, const double* v, int e)
{
    if constexpr (MODE == 2) {
        unsigned w[VPL / 4];
#pragma unroll
        for (int q = 0; q < VPL / 4; ++q) {
            unsigned word = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                word |= (unsigned)(e == EXP_NONE ? 0 : e4m3_code(v[4 * q + j], e)) << (8 * j);
            w[q] = word;
        }
        unsigned char* dst = reinterpret_cast<unsigned char*>(planes) + off;
        if constexpr (VPL == 4) *reinterpret_cast<unsigned*>(dst) = w[0];
        else *reinterpret_cast<uint2*>(dst) = make_uint2(w[0], w[1]);
    } else if (MODE == 1 && VPL == 8) {
        // element pairs packed as BF16x2 words as they are sliced (28 live words), then one 16-byte
        // store per plane: the warp writes 512 contiguous bytes of each plane
        unsigned wd[7][4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float a[7], c[7];
            slice_element<1>(v[2 * q], e, S, a);
            slice_element<1>(v[2 * q + 1], e, S, c);
#pragma unroll
            for (int t = 0; t < 7; ++t)  // at most 8 significant bits: BF16 is the float's upper half
                wd[t][q] = __byte_perm(__float_as_uint(a[t]), __float_as_uint(c[t]), 0x7632u);
        }
#pragma unroll
        for (int t = 0; t < 7; ++t)
            if (t < S)
                *reinterpret_cast<uint4*>(planes + t * plane + off) = make_uint4(wd[t][0], wd[t][1], wd[t][2], wd[t][3]);
    } else {
        // runs of four elements: 28 live slice values, one 8-byte store per plane and run
        const int np = MODE == 0 ? 2 : S;
#pragma unroll
        for (int h = 0; h < VPL / 4; ++h) {
            float sl[4][7];
#pragma unroll
            for (int j = 0; j < 4; ++j) slice_element<MODE>(v[4 * h + j], e, S, sl[j]);
#pragma unroll
            for (int t = 0; t < 7; ++t) {
                if (t < np) {
                    // the values have at most 8 significant bits, so BF16 is the float's upper half
                    const unsigned lo2 = __byte_perm(__float_as_uint(sl[0][t]), __float_as_uint(sl[1][t]), 0x7632u);
                    const unsigned hi2 = __byte_perm(__float_as_uint(sl[2][t]), __float_as_uint(sl[3][t]), 0x7632u);
                    *reinterpret_cast<uint2*>(planes + t * plane + off + 4 * h) = make_uint2(lo2, hi2);
                }
            }
        }
    }
}

// TRI: A (m x m, column-major, lower triangle) -> slices of
// M = tril(A,-1) + diag(A)/2; otherwise a general column-major m x K matrix.
// Written row-major (row i, k contiguous): planes + s*plane + i*ldp + k, ldp a
// multiple of CW (the row is written up to its chunk's end).
// One CTA: 4096 / CW rows x one CW-column chunk (CW = 128 or 256); 8 warps.
// The tile is transposed through shared memory stored as
// T[row][(k % VPL) * 33 + k / VPL], VPL = CW / 32, so that lane l reads
// k = VPL l .. VPL l + VPL-1 of a row without bank conflicts and writes them
// with one vector store per plane.
// MODE 0: BF16 hi/lo planes; 1: S exact BF16 slices (S <= 7); 2: one FP8 E4M3
// plane (bytes).  Modes 1 and 2 record the chunk exponent of every row.
// One tile of the row split: rows [row0, row0 + ROWS) of A (m x K, column-major)
// and the CW-chunk kc; the output rows are offset by roff (a packed batch) and
// the exponents are strided by erows (the packed row count).
template <int MODE, bool TRI, int CW>
// sq (or NULL): the tile's share of ||A||_F^2 (lower-triangle elements, off-diagonal ones twice, to a
// relative 2^-20 or so: a scale for a shift), summed in a fixed order and written to *sq.
__device__ __forceinline__ void split_lower_tile(int m, int K, const double* __restrict__ A, long lda, int S,
                                                 __nv_bfloat16* planes, long ldp, size_t plane, int* eA, int* emax,
                                                 int kc, int ib, long roff, long erows, double* sq = nullptr)
{
    constexpr bool SCALED = MODE != 0;  // exponents are recorded
    constexpr int VPL = CW / 32;        // values per lane
    constexpr int ROWS = 4096 / CW;     // rows per tile
    constexpr int CG = 256 / ROWS;      // column groups in the load phase
    __shared__ double T[ROWS][VPL * 33 + 1];
    __shared__ double red[8];
    const long row0 = (long)ib * ROWS, col0 = (long)kc * CW;
    if (row0 >= m || (TRI && col0 > row0 + ROWS - 1)) {
        if (sq && threadIdx.x == 0) *sq = 0.0;
        return;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int lr = threadIdx.x % ROWS, lg = threadIdx.x / ROWS;  // load phase: row, column group
    double ld[16];  // all of this thread's loads in flight before the first store
    if (row0 + ROWS <= m && col0 + CW <= K && (!TRI || col0 + CW <= row0 + 1)) {
        // a tile inside the matrix (and below the diagonal): no per-element bounds
        const double* p = A + (row0 + lr) + (col0 + lg) * lda;
#pragma unroll
        for (int t = 0; t < 16; ++t) ld[t] = p[(long)CG * t * lda];
    } else {
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            const int k = lg + CG * t;
            const long i = row0 + lr, kk = col0 + k;
            double v = 0.0;
            if (i < m && kk < K && (!TRI || kk <= i)) v = A[i + kk * lda];
            ld[t] = v;
        }
    }
#pragma unroll
    for (int t = 0; t < 16; ++t) {
        const int k = lg + CG * t;
        T[lr][(k % VPL) * 33 + k / VPL] = ld[t];
    }
    if (sq) {
        // Elements outside A's lower triangle were loaded as zeros.  FP64 arithmetic is scarce, so the
        // squares are summed in FP32: |v| = 1.f 2^(E - 1023) becomes 1.f' 2^(E - emax) with f' the top 20
        // bits of f (relative error below 2^-20; zeros and subnormals add nothing), emax the largest
        // exponent of the thread's values, then of its warp; one FP64 scaling per warp.
        int ex[16], emx = 0;
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            ex[t] = (__double2hiint(ld[t]) >> 20) & 0x7FF;
            emx = max(emx, ex[t]);
        }
        float acc = 0.0f;
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            const int d = ex[t] - emx;
            if (ex[t] != 0 && d > -60) {
                const float f = __int_as_float(((127 + d) << 23) | ((__double2hiint(ld[t]) & 0xFFFFF) << 3));
                const float wf = (col0 + lg + CG * t == row0 + lr) ? f : 2.0f * f;  // off-diagonal: twice
                acc = fmaf(wf, f, acc);
            }
        }
        int ew = emx;
        for (int o = 16; o > 0; o >>= 1) ew = max(ew, __shfl_xor_sync(0xffffffffu, ew, o));
        const int dd = 2 * (emx - ew);
        float a = (emx != 0 && dd > -120) ? acc * __int_as_float((127 + dd) << 23) : 0.0f;
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if ((threadIdx.x & 31) == 0) {
            const double sc = ew == 0 ? 0.0 : __hiloint2double(ew << 20, 0);  // 2^(ew - 1023)
            red[threadIdx.x >> 5] = ((double)a * sc) * sc;
        }
    }
    __syncthreads();
    if (sq && threadIdx.x == 0) *sq = ((red[0] + red[1]) + (red[2] + red[3])) + ((red[4] + red[5]) + (red[6] + red[7]));
    if constexpr (TRI) {
        // M's diagonal is A's halved: one FP64 multiply per diagonal element, only in the tiles that
        // hold the diagonal (FP64 instructions are scarce, so none sits in the load loop)
        if (col0 < row0 + ROWS && row0 < col0 + CW) {  // the same for the whole block
            if (threadIdx.x < ROWS) {
                const long kk = row0 + threadIdx.x - col0;
                if (kk >= 0 && kk < CW && row0 + threadIdx.x < m)
                    T[threadIdx.x][(kk % VPL) * 33 + kk / VPL] *= 0.5;
            }
            __syncthreads();
        }
    }
    constexpr int RPW = ROWS / 8;  // rows per warp
    for (int r = w * RPW; r < w * RPW + RPW; ++r) {
        const long i = row0 + r;
        if (i >= m) break;
        double v[VPL];
#pragma unroll
        for (int j = 0; j < VPL; ++j) v[j] = T[r][j * 33 + lane];  // k = VPL lane + j
        const int e = SCALED ? warp_chunk_exponent<VPL>(v) : 0;
        if (SCALED && lane == 0) {
            eA[(size_t)kc * erows + roff + i] = e;
            if (e != EXP_NONE) atomicMax(&emax[roff + i], e);
        }
        store_run<MODE, VPL>(planes, plane, (size_t)(roff + i) * ldp + col0 + VPL * lane, S, v, e);
    }
}

template <int MODE, bool TRI, int CW>
__global__ void __launch_bounds__(256, 4) split_lower_kernel(int m, int K, const double* __restrict__ A, long lda, int S,
                                                          __nv_bfloat16* planes, long ldp, size_t plane,
                                                          int* eA, int* emax, int kc0 = 0,
                                                          const int* gate = nullptr, int want = 0)
{
    if (gated_off(gate, want)) return;
    split_lower_tile<MODE, TRI, CW>(m, K, A, lda, S, planes, ldp, plane, eA, emax, kc0 + blockIdx.x, blockIdx.y, 0,
                                    m);
}

// One instance of a batched split: its matrix X (rows x K, column-major, ldx)
// goes to packed rows (or columns) [off, off + rows or cols), in kch chunks.
struct SplitInst {
    const double* X;
    long ldx;
    int rows, K, cols;
    long off;
    int kch;
    int tile0, ntiles;  // the A split: the instance's tiles in the wave's tile list
};
static_assert(BATCH_MAX_M <= 4096, "tile codes hold 4 chunk bits, 8 row-block bits; reduce codes 10 block bits");

// The triangular row split of a packed batch of A's: block j takes the tile
// tiles[j] = (instance << 12) | (chunk << 8) | 16-row block, listed for the
// lower-triangle tiles only, and writes the tile's share of ||A||_F^2 to sq[j].
__global__ void __launch_bounds__(256, 4) split_lower_batch_kernel(const SplitInst* __restrict__ inst,
                                                                const int* __restrict__ tiles, int S,
                                                                __nv_bfloat16* planes, long ldp, size_t plane, int* eA,
                                                                int* emax, long erows, double* sq)
{
    const int code = tiles[blockIdx.x];
    const SplitInst I = inst[code >> 12];
    split_lower_tile<1, true, KCH_EMU>(I.rows, I.rows, I.X, I.ldx, S, planes, ldp, plane, eA, emax, (code >> 8) & 15,
                                       code & 255, I.off, erows, sq + blockIdx.x);
}

// ||A_i||_F^2 and ||Z_i||_F^2 of the wave's instances from the splits' shares (A: per tile, Z: per chunk
// and column): one block per instance, each thread a strided share, then a fixed tree.
__global__ void __launch_bounds__(128) norms_batch_kernel(const SplitInst* __restrict__ instA,
                                                          const SplitInst* __restrict__ instZ,
                                                          const double* __restrict__ asq,
                                                          const double* __restrict__ zsq, long ecols, double* anorm2,
                                                          double* znorm2)
{
    __shared__ double red[2][4];
    const SplitInst IA = instA[blockIdx.x], IZ = instZ[blockIdx.x];
    double a = 0.0, z = 0.0;
    for (int t = threadIdx.x; t < IA.ntiles; t += 128) a += asq[IA.tile0 + t];
    for (int t = threadIdx.x; t < IZ.kch * IZ.cols; t += 128)
        z += zsq[(size_t)(t / IZ.cols) * ecols + IZ.off + t % IZ.cols];
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        z += __shfl_xor_sync(0xffffffffu, z, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = a;
        red[1][threadIdx.x >> 5] = z;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        anorm2[blockIdx.x] = (red[0][0] + red[0][1]) + (red[0][2] + red[0][3]);
        znorm2[blockIdx.x] = (red[1][0] + red[1][1]) + (red[1][2] + red[1][3]);
    }
}

// X (K x C, column-major) -> slices written column-major (column c, k
// contiguous, ldp a multiple of CW): planes + s*plane + c*ldp + k.  One warp
// per (CW-chunk, column); lane l handles k = VPL l .. VPL l + VPL-1.  The
// output column is offset by coff and the exponents are strided by ecols (a
// packed batch).
template <int MODE, int CW>
// sq (or NULL): the chunk's sum of squares of the column, written to sq[kc * ecols + coff + c].
__device__ __forceinline__ void split_tall_column(int K, const double* __restrict__ X, long ldx, long c, int S,
                                                  __nv_bfloat16* planes, long ldp, size_t plane, int* eX, int* xmax,
                                                  int kc, long coff, long ecols, double* sq = nullptr)
{
    constexpr bool SCALED = MODE != 0;  // exponents are recorded
    constexpr int VPL = CW / 32;
    const int lane = threadIdx.x & 31;
    const long k0 = (long)kc * CW + VPL * lane;
    double v[VPL];
#pragma unroll
    for (int j = 0; j < VPL; ++j) {
        const long k = k0 + j;
        v[j] = k < K ? X[k + c * ldx] : 0.0;
    }
    const int e = SCALED ? warp_chunk_exponent<VPL>(v) : 0;
    if (SCALED && lane == 0) {
        eX[(size_t)kc * ecols + coff + c] = e;
        if (e != EXP_NONE) atomicMax(&xmax[coff + c], e);
    }
    if (sq) {
        double a = 0.0;
#pragma unroll
        for (int j = 0; j < VPL; ++j) a = fma(v[j], v[j], a);
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) sq[(size_t)kc * ecols + coff + c] = a;
    }
    store_run<MODE, VPL>(planes, plane, (size_t)(coff + c) * ldp + k0, S, v, e);
}

template <int MODE, int CW>
__global__ void __launch_bounds__(256) split_tall_kernel(int K, int C, const double* __restrict__ X, long ldx, int S,
                                                         __nv_bfloat16* planes, long ldp, size_t plane, int* eX,
                                                         int* xmax, const int* gate = nullptr, int want = 0)
{
    if (gated_off(gate, want)) return;
    const long c = (long)blockIdx.y * 8 + (threadIdx.x >> 5);
    if (c >= C) return;
    split_tall_column<MODE, CW>(K, X, ldx, c, S, planes, ldp, plane, eX, xmax, blockIdx.x, 0, C);
}

// The column split of a packed batch: warp w of block y takes packed column
// 8y + w, of instance colinst[8y + w] (skipped when live[instance] <= pass).
__global__ void __launch_bounds__(256) split_tall_batch_kernel(const SplitInst* __restrict__ inst,
                                                               const int* __restrict__ colinst, int S,
                                                               __nv_bfloat16* planes, long ldp, size_t plane, int* eX,
                                                               int* xmax, long ecols, const int* live, int pass,
                                                               double* sq)
{
    const long gc = (long)blockIdx.y * 8 + (threadIdx.x >> 5);
    if (gc >= ecols) return;
    if (live && live[colinst[gc]] <= pass) return;  // the instance sits this pass out
    const SplitInst I = inst[colinst[gc]];
    const int kc = blockIdx.x;
    if (kc >= I.kch) return;
    split_tall_column<1, KCH_EMU>(I.K, I.X, I.ldx, gc - I.off, S, planes, ldp, plane, eX, xmax, kc, I.off, ecols, sq);
}

__global__ void fill_int_kernel(int* p, long n, int v)
{
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

// ---------------------------------------------------------- work items ----
// One instance of a packed batch: its left operand occupies rows
// [roff, roff + rows) of the packed left planes, its right operand columns
// [coff, coff + cols) of the packed right planes; K is its contraction length.
// Its items are [item0, item0 + items); cum + cum0 holds its per-row-tile
// item prefix (rt + 1 entries).  Its output (rows x cols, column-major, ldo)
// starts at out.  wi is its index within the wave (the index of its pass count in TcArgs.live).
struct TcInst {
    int rows, cols, K, tri;
    int roff, coff;
    int rt, cc;
    int item0, cum0;
    double* out;
    long ldo;
    int wi;
};

struct TcArgs {
    int rowsA, colsB, K;  // one instance: its sizes; a packed batch: total rows, total columns, largest K
    int tri;              // 1: row tile I stops at k = 128 (I + 1)
    int ks;               // k-step (elements)
    int piece;            // k-steps per item
    int cc;               // column chunks (one instance)
    int rt;               // row tiles (one instance)
    int nitems;
    const int* cum;       // one instance: rt + 1 item offsets; a batch: the instances' prefixes
    double* slots;        // nitems x 128 x N, column-major per slot: (r, c) at c * 128 + r (FP32 slots use the
                          // first half); a warp's 32 rows of one column are one coalesced store or load
    const int* eA;        // [chunks][rowsA]
    const int* eB;        // [chunks][colsB]
    const int* emaxA;     // [rowsA]
    const int* emaxB;     // [colsB]
    DevStatus* st;
    uint64_t limit_ns;
    int ninst;            // 0: one instance; > 0: a packed batch of ninst instances
    const TcInst* inst;   // [ninst]
    const int* inst_item0;  // [ninst + 1]: first item of each instance, then the total
    const int* rblk;      // a batch: the reduction's blocks (instance << 10 | block)
    int nrblk;            // a batch: their count
    const int* live;      // a batch, or NULL: the wave's Gram pass counts; instances with live[wi] <= pass sit
    int pass;             // this launch out (their items are not in list, their outputs are not written)
    const int* list;      // NULL: items 0..nitems-1; else list[0] items, list[1..]: their indices
    const int* gate;      // NULL, or the launch does nothing unless *gate == gate_want
    int gate_want;
};

__device__ inline int item_total(const TcArgs& a) { return a.list ? a.list[0] : a.nitems; }
__device__ inline int item_index(const TcArgs& a, int jj) { return a.list ? a.list[1 + jj] : jj; }

// The items of a packed launch whose instance takes part in this pass (live[wi] > pass), in item order:
// list[0] = their count, list[1..] = their indices; with blocks (rlist), the same for the reduction's
// blocks (rlist[1..]: codes (member << 10) | block).  One block; instances in chunks of its threads.
constexpr int ALIST_THREADS = 1024;
__device__ inline int reduce_blocks(const TcInst& I) { return (int)(((long)I.rows * I.cols + 255) / 256); }
template <bool BLOCKS>
__global__ void __launch_bounds__(ALIST_THREADS) active_items_kernel(const TcInst* __restrict__ inst,
                                                                     const int* __restrict__ item0, int ninst,
                                                                     const int* __restrict__ live, int pass, int* list)
{
    __shared__ int wsum[ALIST_THREADS / 32];
    __shared__ int base;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    if (t == 0) base = 0;
    __syncthreads();
    for (int k0 = 0; k0 < ninst; k0 += ALIST_THREADS) {
        const int k = k0 + t;
        const bool on = k < ninst && live[inst[k].wi] > pass;
        const int c = !on ? 0 : BLOCKS ? reduce_blocks(inst[k]) : item0[k + 1] - item0[k];
        int incl = c;  // inclusive scan within the warp, then over the warps
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) wsum[w] = incl;
        __syncthreads();
        if (w == 0) {
            int x = wsum[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += v;
            }
            wsum[lane] = x;  // inclusive over warps
        }
        __syncthreads();
        const int excl = base + (w > 0 ? wsum[w - 1] : 0) + incl - c;
        for (int q = 0; q < c; ++q) list[1 + excl + q] = BLOCKS ? ((k << 10) | q) : item0[k] + q;
        const int total = base + wsum[ALIST_THREADS / 32 - 1];
        __syncthreads();  // every thread has read base and wsum
        if (t == 0) base = total;
        __syncthreads();
    }
    if (t == 0) list[0] = base;
}

__device__ __host__ inline int kend_of(int K, int tri, int I)
{
    if (!tri) return K;
    const long e = (long)(I + 1) * TM;
    return e < K ? (int)e : K;
}
__device__ __host__ inline int nks_of(int K, int tri, int ks, int I) { return (kend_of(K, tri, I) + ks - 1) / ks; }
__device__ __host__ inline int pieces_of(int K, int tri, int ks, int piece, int I)
{
    return (nks_of(K, tri, ks, I) + piece - 1) / piece;
}
__device__ __host__ inline int pieces_of(const TcArgs& a, int I) { return pieces_of(a.K, a.tri, a.ks, a.piece, I); }

// cum[I] = items of row tiles 0..I-1 (I = 0..rt).  One block of 256 threads:
// each thread sums a contiguous run of tiles, the runs' sums are scanned by
// warp shuffles, and each thread then writes its run's prefixes.
constexpr int PREFIX_THREADS = 256;
__global__ void __launch_bounds__(PREFIX_THREADS) item_prefix_kernel(TcArgs a, int* cum)
{
    if (gated_off(a.gate, a.gate_want)) return;
    __shared__ int wsum[PREFIX_THREADS / 32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int run = (a.rt + PREFIX_THREADS - 1) / PREFIX_THREADS;
    const int I0 = t * run, I1 = min(a.rt, I0 + run);
    int mine = 0;
    for (int I = I0; I < I1; ++I) mine += pieces_of(a, I) * a.cc;
    int incl = mine;  // inclusive scan within the warp
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    int base = 0;
    for (int k = 0; k < w; ++k) base += wsum[k];
    int s = base + incl - mine;  // exclusive prefix of this thread's run
    for (int I = I0; I < I1; ++I) {
        cum[I] = s;
        s += pieces_of(a, I) * a.cc;
    }
    if (t == PREFIX_THREADS - 1) cum[a.rt] = s;  // the last run ends at rt (its run may be empty)
}

// A work item: row tile I, k-steps [ks0, ks1), column chunk c, of the
// instance whose operands start at row roff / column coff and have rows x cols
// valid entries.
struct Item {
    int I, ks0, ks1, c;
    int roff, coff, rows, cols;
};

__device__ inline int last_le(const int* v, int lo, int hi, int j)  // last index i in [lo, hi] with v[i] <= j
{
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (v[mid] <= j) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ inline Item item_of(const TcArgs& a, int j)
{
    Item it;
    int K = a.K, tri = a.tri, cc = a.cc, rt = a.rt, jl = j;
    const int* cum = a.cum;
    it.roff = 0;
    it.coff = 0;
    it.rows = a.rowsA;
    it.cols = a.colsB;
    if (a.ninst > 0) {
        const int b = last_le(a.inst_item0, 0, a.ninst - 1, j);
        const TcInst& I = a.inst[b];
        K = I.K;
        tri = I.tri;
        cc = I.cc;
        rt = I.rt;
        jl = j - I.item0;
        cum = a.cum + I.cum0;
        it.roff = I.roff;
        it.coff = I.coff;
        it.rows = I.rows;
        it.cols = I.cols;
    }
    it.I = last_le(cum, 0, rt - 1, jl);
    const int rem = jl - cum[it.I];
    const int p = rem / cc;
    it.c = rem % cc;
    it.ks0 = p * a.piece;
    it.ks1 = min(nks_of(K, tri, a.ks, it.I), it.ks0 + a.piece);
    return it;
}

// ------------------------------------------------------ tcgen05 helpers ----
__device__ inline uint64_t smem_desc(uint32_t addr, int swizzle_bytes)
{
    const uint64_t sbo = (uint64_t)(8 * swizzle_bytes) >> 4;  // 8 rows x swizzle width
    const uint64_t layout = swizzle_bytes == 128 ? 2ull : swizzle_bytes == 64 ? 4ull : 6ull;  // 128B, 64B, 32B
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | (1ull << 16) | (sbo << 32) | (1ull << 46) | (layout << 61);
}

// kind::f16 instruction descriptor: D = F32, A = B = BF16, both K-major, M = 128.
__host__ __device__ constexpr uint32_t idesc_bf16(int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

__device__ inline void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

// kind::f8f6f4 instruction descriptor: D = F32, A = B = E4M3 (format 0), both K-major, M = 128.
__host__ __device__ constexpr uint32_t idesc_e4m3(int N)
{
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

__device__ inline void umma_e4m3(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ inline void umma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ inline void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ inline void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ inline void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cta.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// 32 consecutive accumulator columns of this thread's TMEM lane; load and wait
// in one asm statement, so no use of the values can precede the wait.
__device__ inline void tmem_ld32(uint32_t taddr, float* v)
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ inline float pow2f(int d)
{
    if (d < -126) return 0.0f;  // below 2^-126 of the row/column scale: negligible
    if (d > 127) d = 127;
    return __int_as_float((d + 127) << 23);
}

// ---------------------------------------------------------- the kernel ----
// BF16X3 (MODE 0), FP8 E4M3 with chunk scales (MODE 2) and TC2 (MODE 3: the
// two leading pre-scaled EMU64 slices, three products, chunk scales); the
// FP64-accurate emulation has its own kernel below (emu_kernel).
template <int KS, int N, int S, int MODE>
struct TcCfg {
    static constexpr int ES = MODE == 2 ? 1 : 2;      // element bytes
    static constexpr int SW = KS * ES;                 // swizzle width = one K-major row of KS elements
    static constexpr int A_TILE = TM * KS * ES;        // bytes
    static constexpr int B_TILE = N * KS * ES;
    static constexpr int STAGE = S * A_TILE + S * B_TILE;
    // as many stages as ~192 KB holds (2..6): a short k-step needs more bytes in flight
    static constexpr int STAGES = 196608 / STAGE < 2 ? 2 : 196608 / STAGE > 6 ? 6 : 196608 / STAGE;
    static constexpr int TMEM_COLS = 2 * N <= 128 ? 128 : 2 * N <= 256 ? 256 : 512;  // two accumulator buffers
    static constexpr int KPI = MODE == 2 ? 32 : 16;    // K per MMA instruction (32 bytes of K)
    static constexpr int KCH = kch_of(MODE);           // exponent chunk of this mode
    static constexpr int CH_STEPS = MODE == 0 ? 1 << 30 : KCH / KS;  // k-steps per drained chunk
    static constexpr int MAXCH = 2048 / KCH;           // chunks per item (items are 2048 long)
    // align slack + barriers and drain flags + (chunked modes) an item's row and column chunk scales
    static constexpr size_t SMEM =
        1024 + STAGES * (size_t)STAGE + 2048 + (MODE != 0 ? (size_t)MAXCH * (TM + N) * sizeof(float) : 0);
    static_assert(MODE == 0 || MODE == 2 || MODE == 3, "mode");
    static_assert(SW == 64 || SW == 128, "swizzle");
    static_assert(N % 64 == 0 && N >= 64 && N <= 256, "N");
    static_assert(A_TILE % 1024 == 0 && B_TILE % 1024 == 0, "tile alignment");
};

template <int KS, int N, int S, int MODE>
__global__ void __launch_bounds__(TC_THREADS, 1)
    tc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, TcArgs a)
{
    using C = TcCfg<KS, N, S, MODE>;
    constexpr bool CHUNKED = MODE != 0;  // drained every 128 of the contraction, with the chunk scales
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    unsigned char* smem =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::STAGES * C::STAGE);
    uint64_t* empty = full + C::STAGES;
    uint64_t* accf = empty + C::STAGES;  // [2]: accumulator buffer b complete (by chunk parity)
    uint64_t* acce = accf + 2;           // [2]: accumulator buffer b read by the drain
    uint64_t* done = acce + 2;           // every MMA of this CTA complete
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);  // the drain's flag at +32 ints

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nit = item_total(a);  // the launch's items (a packed batch: only the active instances')
    if (*(volatile int*)&a.st->code != 0) return;
    if (threadIdx.x == 0) {
        for (int s = 0; s < C::STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], 1);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        fence_barrier_init();
        tma_prefetch_desc(&mapA);
        tma_prefetch_desc(&mapB);
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                     "r"(C::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;

    auto fail = [&](int where_info) {
        if (*abort_flag == 0) {
            *abort_flag = 1;
            raise_status(a.st, OQR_ERR_TIMEOUT, where_info, TAG_MIXED);
        }
    };

    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            long it = 0;
            for (int jj = blockIdx.x; jj < nit && !*abort_flag; jj += gridDim.x) {
                const int j = item_index(a, jj);
                const Item item = item_of(a, j);
                for (int ks = item.ks0; ks < item.ks1 && !*abort_flag; ++ks, ++it) {
                    const int stg = (int)(it % C::STAGES);
                    const uint32_t ph = (uint32_t)((it / C::STAGES) & 1);
                    if (!mbar_wait(&empty[stg], ph ^ 1u, a.limit_ns)) {
                        fail(1);
                        break;
                    }
                    unsigned char* base = smem + stg * C::STAGE;
                    mbar_expect_tx(&full[stg], C::STAGE);
                    for (int s = 0; s < S; ++s)
                        tma_load_3d(base + s * C::A_TILE, &mapA, &full[stg], ks * KS, item.roff + item.I * TM, s);
                    for (int t = 0; t < S; ++t)
                        tma_load_3d(base + S * C::A_TILE + t * C::B_TILE, &mapB, &full[stg], ks * KS,
                                    item.coff + item.c * N, t);
                }
            }
            // copies still in flight must land before the CTA may exit
            const long issued = it;
            for (long q = issued - C::STAGES; q < issued; ++q)
                if (q >= 0)
                    mbar_wait(&full[q % C::STAGES], (uint32_t)((q / C::STAGES) & 1), exit_drain_ns(a.limit_ns));
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = MODE == 2 ? idesc_e4m3(N) : idesc_bf16(N);
            long it = 0, chunk = 0;
            for (int jj = blockIdx.x; jj < nit && !*abort_flag; jj += gridDim.x) {
                const int j = item_index(a, jj);
                const Item item = item_of(a, j);
                for (int ks = item.ks0; ks < item.ks1 && !*abort_flag; ++ks, ++it) {
                    const bool chunk_start = CHUNKED ? ((ks - item.ks0) % C::CH_STEPS == 0) : (ks == item.ks0);
                    const bool chunk_end = CHUNKED ? ((ks - item.ks0 + 1) % C::CH_STEPS == 0 || ks + 1 == item.ks1)
                                                   : (ks + 1 == item.ks1);
                    const int b = (int)(chunk & 1);  // accumulator buffer of this chunk
                    const uint32_t d = tmem + (uint32_t)(b * N);
                    if (chunk_start && chunk >= 2) {  // the drain must have emptied this buffer (two chunks ago)
                        if (!mbar_wait(&acce[b], (uint32_t)(((chunk - 2) >> 1) & 1), a.limit_ns)) {
                            fail(2);
                            break;
                        }
                        tc_fence_after();
                    }
                    const int stg = (int)(it % C::STAGES);
                    if (!mbar_wait(&full[stg], (uint32_t)((it / C::STAGES) & 1), a.limit_ns)) {
                        fail(3);
                        break;
                    }
                    tc_fence_after();
                    const uint32_t base = smem_u32(smem + stg * C::STAGE);
                    if (MODE == 2) {
                        // one E4M3 product per k-step, K = 32 per instruction
#pragma unroll
                        for (int kk = 0; kk < KS / C::KPI; ++kk) {
                            const uint64_t ad = smem_desc(base + kk * 32, C::SW);
                            const uint64_t bd = smem_desc(base + C::A_TILE + kk * 32, C::SW);
                            umma_e4m3(d, ad, bd, idesc, (chunk_start && kk == 0) ? 0u : 1u);
                        }
                    } else {
                        // hi*hi, hi*lo, lo*hi into one accumulator
                        const int sa[3] = {0, 0, 1}, tb[3] = {0, 1, 0};
#pragma unroll
                        for (int p = 0; p < 3; ++p)
#pragma unroll
                            for (int kk = 0; kk < KS / 16; ++kk) {
                                const uint64_t ad = smem_desc(base + sa[p] * C::A_TILE + kk * 32, C::SW);
                                const uint64_t bd =
                                    smem_desc(base + S * C::A_TILE + tb[p] * C::B_TILE + kk * 32, C::SW);
                                umma_bf16(d, ad, bd, idesc, (chunk_start && p == 0 && kk == 0) ? 0u : 1u);
                            }
                    }
                    umma_commit(&empty[stg]);
                    if (chunk_end) {
                        umma_commit(&accf[b]);
                        ++chunk;
                    }
                }
            }
            // every MMA issued by this thread must be complete before TMEM is released
            umma_commit(done);
            mbar_wait(done, 0, exit_drain_ns(a.limit_ns));
        }
    } else {
        // ------------------------------------------------ drain (warps 2..9)
        // One drain thread waits on the accumulator barrier (time-limited) and
        // publishes the outcome; the 256 drain threads then pass a named
        // barrier together, so every exit below is taken by all of them.
        constexpr int NH = N / 2;             // columns owned by this thread
        const int dt = threadIdx.x - 64;      // 0..255 within the drain group
        const int q = warp & 3;               // TMEM lane quarter this warp may access
        const int half = (warp - 2) >> 2;     // which half of the N columns
        const int r = q * 32 + lane;          // row within the tile = TMEM lane
        const uint32_t lane_addr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(half * NH);
        volatile int* go = const_cast<int*>(abort_flag) + 32;  // outcome of the wait, published by dt == 0
        // chunked modes: the item's row scales [chunk][row] and column scales [chunk][column]
        float* rowsc = reinterpret_cast<float*>(smem + C::STAGES * C::STAGE + 2048);
        float* colsc = rowsc + C::MAXCH * TM;
        long chunk = 0;
        bool stop = false;
        for (int jj = blockIdx.x; jj < nit && !stop; jj += gridDim.x) {
            const int j = item_index(a, jj);
            const Item item = item_of(a, j);
            double* slot = a.slots + (size_t)j * TM * N + (size_t)(half * NH) * TM + r;  // MODE 0: FP64 slots
            float H[CHUNKED ? NH : 1];
#pragma unroll
            for (int c = 0; c < (CHUNKED ? NH : 1); ++c) H[c] = 0.f;
            const int nsteps = item.ks1 - item.ks0;
            const int nch = CHUNKED ? (nsteps + C::CH_STEPS - 1) / C::CH_STEPS : 1;
            if constexpr (CHUNKED) {
                // FP8: products of x 2^(8-e_r) and y 2^(8-e_c), scaled back by 2^(e_r + e_c - 16); TC2:
                // products of slices of x 2^(7-e_r) and y 2^(7-e_c), scaled back by 2^(e_r + e_c - 14);
                // both relative to the row and column maxima.  All of the item's scales are loaded
                // once, so no global load sits between a chunk's accumulators and their drain.
                const int kc0 = (item.ks0 * KS) / C::KCH;
                for (int e = dt; e < nch * TM; e += 256) {
                    const int ch = e / TM, rr = e % TM;
                    const int g = item.I * TM + rr;  // row within the instance
                    float v = 0.0f;
                    if (g < item.rows) {
                        const long gr = item.roff + g;
                        const int er = a.eA[(size_t)(kc0 + ch) * a.rowsA + gr];
                        if (er != EXP_NONE) v = pow2f(er - a.emaxA[gr] - (MODE == 2 ? 16 : 14));
                    }
                    rowsc[ch * TM + rr] = v;
                }
                for (int e = dt; e < nch * N; e += 256) {
                    const int ch = e / N, cc = e % N;
                    const int col = item.c * N + cc;  // column within the instance
                    float v = 0.0f;
                    if (col < item.cols) {
                        const long gc = item.coff + col;
                        const int eb = a.eB[(size_t)(kc0 + ch) * a.colsB + gc];
                        if (eb != EXP_NONE) v = pow2f(eb - a.emaxB[gc]);
                    }
                    colsc[ch * N + cc] = v;
                }
                asm volatile("bar.sync 1, 256;" ::: "memory");
            }
            for (int ch = 0; ch < nch; ++ch, ++chunk) {
                const int b = (int)(chunk & 1);
                const uint32_t buf = lane_addr + (uint32_t)(b * N);
                if (dt == 0) {
                    const bool ok = mbar_wait(&accf[b], (uint32_t)((chunk >> 1) & 1), a.limit_ns);
                    if (!ok) fail(4);
                    *go = (ok && !*abort_flag) ? 1 : 0;
                }
                asm volatile("bar.sync 1, 256;" ::: "memory");
                if (*go == 0) {
                    stop = true;
                    break;
                }
                tc_fence_after();
                if constexpr (CHUNKED) {  // FP32 accumulation suits these precisions
                    const float* colscale = colsc + ch * N + half * NH;
                    const float rs = rowsc[ch * TM + r];
#pragma unroll
                    for (int h = 0; h < NH / 32; ++h) {
                        float v[32];
                        tmem_ld32(buf + (uint32_t)(h * 32), v);
#pragma unroll
                        for (int c = 0; c < 32; c += 2) {  // two columns per FP32x2 instruction
                            const float2 p = __fmul2_rn(make_float2(v[c], v[c + 1]), make_float2(rs, rs));
                            const float2 hh = __ffma2_rn(p, make_float2(colscale[h * 32 + c], colscale[h * 32 + c + 1]),
                                                         make_float2(H[h * 32 + c], H[h * 32 + c + 1]));
                            H[h * 32 + c] = hh.x;
                            H[h * 32 + c + 1] = hh.y;
                        }
                    }
                } else {
#pragma unroll 1
                    for (int h = 0; h < NH / 32; ++h) {
                        float v[32];
                        tmem_ld32(buf + (uint32_t)(h * 32), v);
#pragma unroll
                        for (int c = 0; c < 32; ++c) slot[(size_t)(h * 32 + c) * TM] = (double)v[c];
                    }
                }
                tc_fence_before();
                asm volatile("bar.sync 1, 256;" ::: "memory");  // TMEM and the scales fully read
                if (dt == 0) mbar_arrive(&acce[b]);
            }
            if (stop) break;
            if constexpr (CHUNKED) {
                // FP32 slots relative to 2^(emax_row + emax_col): the reduce sums the pieces and scales
                // once per output element (no FP64 work here)
                float* fslot = reinterpret_cast<float*>(a.slots) + (size_t)j * TM * N + (size_t)(half * NH) * TM + r;
#pragma unroll
                for (int c = 0; c < NH; ++c) fslot[(size_t)c * TM] = H[c];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TMEM_COLS)
                     : "memory");
    }
}

// x 2^k as a double, exact: for a normal x with the result in the normal range
// the double is assembled from x's sign, exponent and significand with integer
// operations (no FP64 instruction); otherwise by conversion and ldexp.
__device__ inline double f32_scaled_to_f64(float x, int k)
{
    const unsigned u = __float_as_uint(x);
    const int ex = (int)((u >> 23) & 0xFF);
    const int e64 = ex - 127 + k + 1023;
    if (ex != 0 && ex != 0xFF && e64 >= 1 && e64 <= 2046) {
        const unsigned long long b = ((unsigned long long)(u >> 31) << 63) | ((unsigned long long)e64 << 52) |
                                     ((unsigned long long)(u & 0x7FFFFF) << 29);
        return __longlong_as_double((long long)b);
    }
    return x == 0.0f ? 0.0 : ldexp((double)x, k);
}

// out (rowsA x colsB, column-major, ldo) = sum over the pieces of each tile.
template <int N>
__global__ void slot_reduce_kernel(TcArgs a, double* out, long ldo, const DevStatus* st)
{
    if (*(volatile const int*)&st->code != 0 || gated_off(a.gate, a.gate_want)) return;
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long)a.rowsA * a.colsB) return;
    const int col = (int)(e / a.rowsA), row = (int)(e % a.rowsA);
    const int I = row / TM, c = col / N;
    const int np = pieces_of(a, I);
    double s = 0.0;
    for (int p = 0; p < np; ++p) {
        const int j = a.cum[I] + p * a.cc + c;
        s += a.slots[(size_t)j * TM * N + (size_t)(col % N) * TM + (row % TM)];
    }
    out[row + (long)col * ldo] = s;
}

// Chunked modes (FP8, TC2): out = (sum over the pieces of the FP32 slots, in
// piece order) 2^(emax_row + emax_col).
template <int N>
__global__ void slot_reduce_f32_kernel(TcArgs a, double* out, long ldo, const DevStatus* st)
{
    if (*(volatile const int*)&st->code != 0) return;
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long)a.rowsA * a.colsB) return;
    const int col = (int)(e / a.rowsA), row = (int)(e % a.rowsA);
    const int I = row / TM, c = col / N;
    const int np = pieces_of(a, I);
    const float* slots = reinterpret_cast<const float*>(a.slots);
    float s = 0.0f;
    for (int p = 0; p < np; ++p) {
        const int j = a.cum[I] + p * a.cc + c;
        s += slots[(size_t)j * TM * N + (size_t)(col % N) * TM + (row % TM)];
    }
    const int er = a.emaxA[row], ec = a.emaxB[col];
    out[row + (long)col * ldo] = (er == EXP_NONE || ec == EXP_NONE) ? 0.0 : f32_scaled_to_f64(s, er + ec);
}

// One reduction block: the 256 elements [256 b, 256 b + 256) of member k's output, code = (k << 10) | b.
template <int N, bool F32>
__device__ inline void slot_reduce_block(const TcArgs& a, int code)
{
    const TcInst I = a.inst[code >> 10];
    const long el = (long)(code & 1023) * 256 + threadIdx.x;
    if (el >= (long)I.rows * I.cols) return;
    const int col = (int)(el / I.rows), row = (int)(el % I.rows);
    const int T = row / TM, c = col / N;
    const int np = pieces_of(I.K, I.tri, a.ks, a.piece, T);
    const int* cum = a.cum + I.cum0;
    double r;
    if constexpr (F32) {
        const float* slots = reinterpret_cast<const float*>(a.slots);
        float s = 0.0f;
        for (int p = 0; p < np; ++p) {
            const int j = I.item0 + cum[T] + p * I.cc + c;
            s += slots[(size_t)j * TM * N + (size_t)(col % N) * TM + (row % TM)];
        }
        const int er = a.emaxA[I.roff + row], ec = a.emaxB[I.coff + col];
        r = (er == EXP_NONE || ec == EXP_NONE) ? 0.0 : f32_scaled_to_f64(s, er + ec);
    } else {
        double s = 0.0;
        for (int p = 0; p < np; ++p) {
            const int j = I.item0 + cum[T] + p * I.cc + c;
            s += a.slots[(size_t)j * TM * N + (size_t)(col % N) * TM + (row % TM)];
        }
        r = s;
    }
    I.out[row + (long)col * I.ldo] = r;
}

// A packed batch: every instance's output (rows x cols, column-major, ldo) is
// the sum over the pieces of each tile of its slots, in piece order; F32: FP32
// slots scaled by 2^(emax_row + emax_col) (TC2), else FP64 slots (EMU64).
// The blocks are the launch's rblk codes, or (rlist) those of the instances
// taking part in the pass; grid-stride over them.
template <int N, bool F32>
__global__ void slot_reduce_batch_kernel(TcArgs a, const int* rlist)
{
    if (*(volatile const int*)&a.st->code != 0) return;
    const int nb = rlist ? rlist[0] : a.nrblk;
    for (int q = blockIdx.x; q < nb; q += gridDim.x) slot_reduce_block<N, F32>(a, rlist ? rlist[1 + q] : a.rblk[q]);
}

// G = C + C^T (+ shift I), exactly symmetric.
__global__ void symmetrize_kernel(int n, const double* __restrict__ Cm, long ldc, double* G, long ldg,
                                  const double* shift_ptr, const DevStatus* st)
{
    if (*(volatile const int*)&st->code != 0) return;
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long)n * n) return;
    const long r = e % n, c = e / n;
    double v = Cm[r + c * ldc] + Cm[c + r * ldc];
    if (r == c && shift_ptr) v += *shift_ptr;
    G[r + c * ldg] = v;
}

// ------------------------------------------- FP64-accurate (EMU64) kernel ----
// Levels L = s + t + 2 of the slice products (s, t) with s + t <= 6.  Each of
// L2..L6 owns a TMEM accumulator.  Over one 256-long chunk L2..L5 are exact
// (at most 4 products of magnitude at most 2^14 in the units of their level,
// 256 terms: within 2^24); L6 (5 products) can pass 2^24 by at most 2^0.32,
// so its FP32 rounding stays below 2^-53 of the chunk's largest possible
// value.  L7 and L8 (13 products) share one accumulator; their sum is below
// 2^-37 of that value, so FP32 rounding there costs below 2^-58 of it.
//
// TMEM: 8 slots of 64 columns.  L2..L5 use slots 0..3 in every chunk; L6 and
// L7+8 alternate between slots 4, 5 (even chunks) and 6, 7 (odd chunks).  The
// first k-step of a chunk issues the L6..L8 products first (their slots were
// drained two chunks ago) and only then waits for the drain to have read the
// previous chunk's L2..L5: the drain of a chunk overlaps the next chunk's
// MMAs.
//
// Warps: 0 TMA producer, 1 TMEM allocation + MMA issuer, 2..17 drain (four
// warps per TMEM lane quarter, 16 columns each).
//
// Staging: k-steps of 32 (one 64-byte swizzled row of BF16 per tile row, two
// MMAs per product), two stages.  The MMA issue bounds the kernel (measured:
// the drain's work removed leaves the U product's time unchanged; the MMAs
// removed halve it), and part of it is a cost per k-step: 16-long k-steps in
// four stages of the same bytes took 8.32 ms against 7.22.
constexpr int EMU_KS = 32;                          // k-step: one 64-byte swizzled row of BF16
constexpr int EMU_N = 64;                           // UMMA N
constexpr int EMU_S = 7;                            // slices per operand
constexpr int EMU_A_TILE = TM * EMU_KS * 2;         // 8 KB
constexpr int EMU_B_TILE = EMU_N * EMU_KS * 2;      // 4 KB
constexpr int EMU_STAGE = EMU_S * (EMU_A_TILE + EMU_B_TILE);
constexpr int EMU_STAGES = 2;
constexpr int EMU_CH = KCH_EMU / EMU_KS;            // k-steps per chunk
constexpr int EMU_DRAIN = 512;                      // drain threads
constexpr int EMU_THREADS = 64 + EMU_DRAIN;
constexpr int EMU_CPT = EMU_N / 4;                  // columns per drain thread
constexpr int EMU_MAXCH = 2048 / KCH_EMU;           // chunks per item (items are 2048 long)
// align slack + stages + barriers and flags + an item's row and column chunk scales
constexpr size_t EMU_SMEM = 1024 + (size_t)EMU_STAGES * EMU_STAGE + 1024 + (size_t)EMU_MAXCH * (TM + EMU_N) * 4;
static_assert(EMU_STAGE % 1024 == 0, "stage alignment");

// 8 consecutive accumulator columns of this thread's TMEM lane; the load and
// its wait are one asm statement, so no use of r can precede the wait.
__device__ inline void tmem_ld8(uint32_t taddr, uint32_t* r)
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
        : "r"(taddr)
        : "memory");
}

// 8 consecutive columns at taddr and at taddr2, under one wait.
__device__ inline void tmem_ld8x2(uint32_t taddr, uint32_t taddr2, uint32_t* r, uint32_t* u)
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%16];\n"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8,%9,%10,%11,%12,%13,%14,%15}, [%17];\n"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7])
        : "r"(taddr), "r"(taddr2)
        : "memory");
}

// (H, L) += t by TwoSum, two columns per FP32x2 instruction.  The roundings are
// those of the scalar form: fma(x, -1, y) is y - x rounded once.
__device__ __forceinline__ void two_sum2(float2& H, float2& L, float2 t)
{
    const float2 m1 = make_float2(-1.0f, -1.0f);
    const float2 sm = __fadd2_rn(H, t);
    const float2 bp = __ffma2_rn(H, m1, sm);  // sm - H
    const float2 q = __ffma2_rn(bp, m1, sm);  // sm - bp
    const float2 e1 = __ffma2_rn(q, m1, H);   // H - (sm - bp)
    const float2 e2 = __ffma2_rn(bp, m1, t);  // t - bp
    H = sm;
    L = __fadd2_rn(L, __fadd2_rn(e1, e2));
}

// The products (s, L - 2 - s) of level L: two MMAs (K = 16 each) per product.
// desc0A / desc0B: descriptors of plane 0 of the stage; plane offsets are
// added to the 16-byte address field (no carry: shared memory is below 256 KB).
template <int L>
__device__ __forceinline__ void emu_issue_level(uint32_t d, uint64_t desc0A, uint64_t desc0B, uint32_t idesc,
                                                bool first)
{
#pragma unroll
    for (int s = 0; s <= L - 2; ++s) {
        const int t = L - 2 - s;
#pragma unroll
        for (int kk = 0; kk < EMU_KS / 16; ++kk) {  // one MMA (K = 16) per 32 bytes of the row
            const uint64_t ad = desc0A + (uint64_t)((s * EMU_A_TILE + kk * 32) >> 4);
            const uint64_t bd = desc0B + (uint64_t)((t * EMU_B_TILE + kk * 32) >> 4);
            umma_bf16(d, ad, bd, idesc, (first && s == 0 && kk == 0) ? 0u : 1u);
        }
    }
}

__global__ void __launch_bounds__(EMU_THREADS, 1)
    emu_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, TcArgs a)
{
    if (gated_off(a.gate, a.gate_want)) return;  // uniform over the grid, before any barrier or TMEM
    extern __shared__ __align__(1024) unsigned char emu_smem_raw[];
    unsigned char* smem =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(emu_smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + EMU_STAGES * EMU_STAGE);
    uint64_t* empty = full + EMU_STAGES;
    uint64_t* accf = empty + EMU_STAGES;  // chunk's MMAs complete
    uint64_t* lo_empty = accf + 1;        // chunk's L2..L5 read
    uint64_t* hi_empty = lo_empty + 1;    // [2]: chunk's L6, L7+8 read, by chunk parity
    uint64_t* done = hi_empty + 2;        // every MMA of this CTA complete
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
    volatile int* go = abort_flag + 1;                                 // outcome of the drain's wait
    // the item's row scales [chunk][row] and column scales [chunk][column]
    float* rowsc = reinterpret_cast<float*>(smem + EMU_STAGES * EMU_STAGE + 1024);
    float* colsc = rowsc + EMU_MAXCH * TM;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nit = item_total(a);  // the launch's items (a packed batch: only the active instances')
    if (*(volatile int*)&a.st->code != 0) return;
    if (threadIdx.x == 0) {
        for (int s = 0; s < EMU_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(accf, 1);
        mbar_init(lo_empty, 1);
        mbar_init(&hi_empty[0], 1);
        mbar_init(&hi_empty[1], 1);
        mbar_init(done, 1);
        *abort_flag = 0;
        fence_barrier_init();
        tma_prefetch_desc(&mapA);
        tma_prefetch_desc(&mapB);
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;

    auto fail = [&](int where_info) {
        if (*abort_flag == 0) {
            *abort_flag = 1;
            raise_status(a.st, OQR_ERR_TIMEOUT, where_info, TAG_MIXED);
        }
    };

    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            long it = 0;
            for (int jj = blockIdx.x; jj < nit && !*abort_flag; jj += gridDim.x) {
                const int j = item_index(a, jj);
                const Item item = item_of(a, j);
                for (int ks = item.ks0; ks < item.ks1 && !*abort_flag; ++ks, ++it) {
                    const int stg = (int)(it % EMU_STAGES);
                    const uint32_t ph = (uint32_t)((it / EMU_STAGES) & 1);
                    if (!mbar_wait(&empty[stg], ph ^ 1u, a.limit_ns)) {
                        fail(11);
                        break;
                    }
                    unsigned char* base = smem + stg * EMU_STAGE;
                    mbar_expect_tx(&full[stg], EMU_STAGE);
                    for (int s = 0; s < EMU_S; ++s)
                        tma_load_3d(base + s * EMU_A_TILE, &mapA, &full[stg], ks * EMU_KS, item.roff + item.I * TM,
                                    s);
                    for (int t = 0; t < EMU_S; ++t)
                        tma_load_3d(base + EMU_S * EMU_A_TILE + t * EMU_B_TILE, &mapB, &full[stg], ks * EMU_KS,
                                    item.coff + item.c * EMU_N, t);
                }
            }
            const long issued = it;  // copies still in flight must land before the CTA may exit
            for (long q = issued - EMU_STAGES; q < issued; ++q)
                if (q >= 0)
                    mbar_wait(&full[q % EMU_STAGES], (uint32_t)((q / EMU_STAGES) & 1), exit_drain_ns(a.limit_ns));
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16(EMU_N);
            long it = 0, chunk = 0;
            bool ok = true;
            for (int jj = blockIdx.x; jj < nit && ok && !*abort_flag; jj += gridDim.x) {
                const int j = item_index(a, jj);
                const Item item = item_of(a, j);
                for (int ks = item.ks0; ks < item.ks1 && !*abort_flag; ++ks, ++it) {
                    const int kin = ks - item.ks0;
                    const bool cstart = kin % EMU_CH == 0;
                    const bool cend = (kin + 1) % EMU_CH == 0 || ks + 1 == item.ks1;
                    const int stg = (int)(it % EMU_STAGES);
                    if (!mbar_wait(&full[stg], (uint32_t)((it / EMU_STAGES) & 1), a.limit_ns)) {
                        fail(13);
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t base = smem_u32(smem + stg * EMU_STAGE);
                    const uint64_t dA = smem_desc(base, EMU_KS * 2), dB = smem_desc(base + EMU_S * EMU_A_TILE, EMU_KS * 2);
                    const uint32_t hi = tmem + 256u + (uint32_t)((chunk & 1) * 128);
                    if (cstart && chunk >= 2) {  // this parity's L6, L7+8 slots: read two chunks ago
                        if (!mbar_wait(&hi_empty[chunk & 1], (uint32_t)(((chunk - 2) >> 1) & 1), a.limit_ns)) {
                            fail(14);
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                    }
                    emu_issue_level<6>(hi, dA, dB, idesc, cstart);
                    emu_issue_level<7>(hi + 64u, dA, dB, idesc, cstart);
                    emu_issue_level<8>(hi + 64u, dA, dB, idesc, false);
                    if (cstart && chunk >= 1) {  // L2..L5 slots: the previous chunk's must have been read
                        if (!mbar_wait(lo_empty, (uint32_t)((chunk - 1) & 1), a.limit_ns)) {
                            fail(15);
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                    }
                    emu_issue_level<5>(tmem + 192u, dA, dB, idesc, cstart);
                    emu_issue_level<4>(tmem + 128u, dA, dB, idesc, cstart);
                    emu_issue_level<3>(tmem + 64u, dA, dB, idesc, cstart);
                    emu_issue_level<2>(tmem, dA, dB, idesc, cstart);
                    umma_commit(&empty[stg]);
                    if (cend) {
                        umma_commit(accf);
                        ++chunk;
                    }
                }
            }
            // every MMA issued by this thread must be complete before TMEM is released
            umma_commit(done);
            mbar_wait(done, 0, exit_drain_ns(a.limit_ns));
        }
    } else {
        // ------------------------------------------------ drain (warps 2..17)
        // One drain thread waits on the accumulator barrier (time-limited) and
        // publishes the outcome; the drain threads then pass a named barrier
        // together, so every exit below is taken by all of them.
        const int dt = threadIdx.x - 64;      // 0..511 within the drain group
        const int q = warp & 3;               // TMEM lane quarter this warp may access
        const int g = (warp - 2) >> 2;        // column group (EMU_CPT columns)
        const int r = q * 32 + lane;          // row within the tile = TMEM lane
        const uint32_t lane_addr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(g * EMU_CPT);
        long chunk = 0;
        bool stop = false;
        for (int jj = blockIdx.x; jj < nit && !stop; jj += gridDim.x) {
            const int j = item_index(a, jj);
            const Item item = item_of(a, j);
            const int gi = item.I * TM + r;  // row within the instance
            const bool row_ok = gi < item.rows;
            float2 H[EMU_CPT / 2], L[EMU_CPT / 2];  // column pairs
#pragma unroll
            for (int c = 0; c < EMU_CPT / 2; ++c) H[c] = L[c] = make_float2(0.f, 0.f);
            const int nsteps = item.ks1 - item.ks0;
            const int emax_r = row_ok ? a.emaxA[item.roff + gi] : 0;
            const int nch = (nsteps + EMU_CH - 1) / EMU_CH;
            {
                // all of the item's scales, loaded once: row scale 2^(e_row - emax_row - 14) (x y =
                // 2^(e_r + e_c - 14) times the sum of the slice products) and column scale
                // 2^(e_col - emax_col), 0 for an all-zero chunk; no global load then sits between a
                // chunk's accumulators and their drain
                const int kc0 = (item.ks0 * EMU_KS) / KCH_EMU;
                for (int e = dt; e < nch * TM; e += EMU_DRAIN) {
                    const int ch = e / TM, rr = e % TM;
                    const int g = item.I * TM + rr;  // row within the instance
                    float v = 0.0f;
                    if (g < item.rows) {
                        const long gr = item.roff + g;
                        const int er = a.eA[(size_t)(kc0 + ch) * a.rowsA + gr];
                        if (er != EXP_NONE) v = pow2f(er - a.emaxA[gr] - 14);
                    }
                    rowsc[ch * TM + rr] = v;
                }
                for (int e = dt; e < nch * EMU_N; e += EMU_DRAIN) {
                    const int ch = e / EMU_N, cc = e % EMU_N;
                    const int col = item.c * EMU_N + cc;  // column within the instance
                    float v = 0.0f;
                    if (col < item.cols) {
                        const long gc = item.coff + col;
                        const int eb = a.eB[(size_t)(kc0 + ch) * a.colsB + gc];
                        if (eb != EXP_NONE) v = pow2f(eb - a.emaxB[gc]);
                    }
                    colsc[ch * EMU_N + cc] = v;
                }
            }
            for (int ch = 0; ch < nch; ++ch, ++chunk) {
                if (dt == 0) {
                    const bool okw = mbar_wait(accf, (uint32_t)(chunk & 1), a.limit_ns);
                    if (!okw) fail(16);
                    *go = (okw && !*abort_flag) ? 1 : 0;
                }
                asm volatile("bar.sync 1, 512;" ::: "memory");  // also publishes the item's scales
                if (*go == 0) {
                    stop = true;
                    break;
                }
                tc_fence_after();
                const float rs = rowsc[ch * TM + r];
                float2 sc[EMU_CPT / 2];
#pragma unroll
                for (int c = 0; c < EMU_CPT / 2; ++c)  // exact
                    sc[c] = __fmul2_rn(make_float2(rs, rs), make_float2(colsc[ch * EMU_N + g * EMU_CPT + 2 * c],
                                                                      colsc[ch * EMU_N + g * EMU_CPT + 2 * c + 1]));
                // L5, L4, L3, L2: exact level sums, added into (H, L) by TwoSum
#pragma unroll
                for (int lv = 0; lv < 4; ++lv)
#pragma unroll
                    for (int half = 0; half < 2; ++half) {  // 8 columns at a time: fewer live registers
                        uint32_t v[EMU_CPT / 2];
                        tmem_ld8(lane_addr + (uint32_t)((3 - lv) * 64 + 8 * half), v);
#pragma unroll
                        for (int cc = 0; cc < EMU_CPT / 4; ++cc) {
                            const int c = half * (EMU_CPT / 4) + cc;
                            two_sum2(H[c], L[c],
                                     __fmul2_rn(make_float2(__uint_as_float(v[2 * cc]), __uint_as_float(v[2 * cc + 1])),
                                                sc[c]));
                        }
                    }
                tc_fence_before();
                asm volatile("bar.sync 1, 512;" ::: "memory");  // L2..L5 fully read
                if (dt == 0) mbar_arrive(lo_empty);
                // L6 and L7+8: below 2^-29 of the chunk's scale, added into the low part
                const uint32_t hi = lane_addr + 256u + (uint32_t)((chunk & 1) * 128);
#pragma unroll
                for (int half = 0; half < 2; ++half) {  // 8 columns at a time: fewer live registers
                    uint32_t v6[EMU_CPT / 2], v78[EMU_CPT / 2];
                    tmem_ld8x2(hi + (uint32_t)(8 * half), hi + 64u + (uint32_t)(8 * half), v6, v78);
#pragma unroll
                    for (int cc = 0; cc < EMU_CPT / 4; ++cc) {
                        const int c = half * (EMU_CPT / 4) + cc;
                        const float2 m1 = make_float2(-1.0f, -1.0f);
                        const float2 h =
                            __fadd2_rn(make_float2(__uint_as_float(v6[2 * cc]), __uint_as_float(v6[2 * cc + 1])),
                                       make_float2(__uint_as_float(v78[2 * cc]), __uint_as_float(v78[2 * cc + 1])));
                        L[c] = __ffma2_rn(h, sc[c], L[c]);
                        const float2 sm = __fadd2_rn(H[c], L[c]);              // renormalise (Fast2Sum)
                        L[c] = __ffma2_rn(__ffma2_rn(H[c], m1, sm), m1, L[c]);  // L - (sm - H)
                        H[c] = sm;
                    }
                }
                tc_fence_before();
                asm volatile("bar.sync 1, 512;" ::: "memory");  // L6, L7+8 and the scales fully read
                if (dt == 0) mbar_arrive(&hi_empty[chunk & 1]);
            }
            if (stop) break;
            // (H + L) 2^(emax_row + emax_col) into this item's FP64 slot: H and L become scaled doubles
            // by integer operations, and one FP64 add (exact: H and L do not overlap) joins them
            double* slot = a.slots + (size_t)j * TM * EMU_N + (size_t)(g * EMU_CPT) * TM + r;
#pragma unroll
            for (int c = 0; c < EMU_CPT; ++c) {
                const int col = item.c * EMU_N + g * EMU_CPT + c;  // column within the instance
                const int ec = col < item.cols ? __ldg(a.emaxB + item.coff + col) : EXP_NONE;
                double out = 0.0;
                if (row_ok && emax_r != EXP_NONE && ec != EXP_NONE) {
                    const int k = emax_r + ec;
                    const float hc = (c & 1) ? H[c / 2].y : H[c / 2].x, lc = (c & 1) ? L[c / 2].y : L[c / 2].x;
                    out = f32_scaled_to_f64(hc, k) + f32_scaled_to_f64(lc, k);
                }
                slot[(size_t)c * TM] = out;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
    }
}

// ------------------------------------------------------------ host side ----
bool make_map_3d(CUtensorMap* map, const void* base, long kext, long rows, long ldp, size_t plane_bytes, int S,
                 int box_k, int box_rows, int elem_bytes);

template <int KS, int N, int S, int MODE>
cudaError_t launch_tc(const TcArgs& a0, const void* planesA, long ldpA, size_t planeA, const void* planesB, long ldpB,
                      size_t planeB, int sms, cudaStream_t s)
{
    using C = TcCfg<KS, N, S, MODE>;
    TcArgs a = a0;
    CUtensorMap mA{}, mB{};
    if (!make_map_3d(&mA, planesA, a.K, a.rowsA, ldpA, planeA * C::ES, S, KS, TM, C::ES)) return cudaErrorInvalidValue;
    if (!make_map_3d(&mB, planesB, a.K, a.colsB, ldpB, planeB * C::ES, S, KS, N, C::ES)) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(tc_kernel<KS, N, S, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)C::SMEM);
    if (e != cudaSuccess) return e;
    const int grid = a.nitems < sms ? a.nitems : sms;
    if (grid > 0) tc_kernel<KS, N, S, MODE><<<grid, TC_THREADS, C::SMEM, s>>>(mA, mB, a);
    return cudaGetLastError();
}


cudaError_t launch_emu(const TcArgs& a0, const void* planesA, long ldpA, size_t planeA, const void* planesB, long ldpB,
                       size_t planeB, int sms, cudaStream_t s)
{
    TcArgs a = a0;
    CUtensorMap mA{}, mB{};
    if (!make_map_3d(&mA, planesA, a.K, a.rowsA, ldpA, planeA * 2, EMU_S, EMU_KS, TM, 2)) return cudaErrorInvalidValue;
    if (!make_map_3d(&mB, planesB, a.K, a.colsB, ldpB, planeB * 2, EMU_S, EMU_KS, EMU_N, 2))
        return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(emu_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)EMU_SMEM);
    if (e != cudaSuccess) return e;
    const int grid = a.nitems < sms ? a.nitems : sms;
    if (grid > 0) emu_kernel<<<grid, EMU_THREADS, EMU_SMEM, s>>>(mA, mB, a);
    return cudaGetLastError();
}
}  // namespace

// -------------------------------------------------------- public (internal) API
size_t tc_plan_bytes(const TcPlan& p)
{
    return (size_t)p.nitems_max * TM * p.N * sizeof(double);
}

static TcArgs make_args(const TcPlan& p, int rowsA, int colsB, int K, int tri, int N)
{
    TcArgs a{};
    a.rowsA = rowsA;
    a.colsB = colsB;
    a.K = K;
    a.tri = tri;
    a.ks = p.mode == 1 ? EMU_KS : p.mode == 2 ? 128 : 64;
    a.piece = 2048 / a.ks;  // k-steps per item (a multiple of the exponent chunk)
    a.cc = (colsB + N - 1) / N;
    a.rt = (rowsA + TM - 1) / TM;
    int s = 0;
    for (int I = 0; I < a.rt; ++I) s += pieces_of(a, I) * a.cc;
    a.nitems = s;
    return a;
}

TcPlan tc_plan(int m, int n, int mode, int sa, bool no_a)
{
    TcPlan p{};
    p.m = m;
    p.n = n;
    p.mode = mode;
    p.noA = no_a ? 1 : 0;
    p.S = mode == 1 ? EMU_S : mode == 2 ? 1 : 2;
    p.SA = sa > p.S ? sa : p.S;
    p.es = mode == 2 ? 1 : 2;
    // FP8 and TC2 keep N <= 128: their drain holds N/2 FP32 sums per thread
    p.N = mode == 1 ? EMU_N : (n <= 64 ? 64 : (n <= 128 || mode >= 2) ? 128 : 256);
    p.ldp = ((long)m + 255) / 256 * 256;  // the splits write to the end of their chunk
    p.kch = (m + kch_of(mode) - 1) / kch_of(mode);
    const TcArgs c = make_args(p, n, n, m, 0, p.N);
    if (p.noA) {  // only the product C = X^T U
        p.nitems_max = c.nitems;
        return p;
    }
    const TcArgs u = make_args(p, m, n, m, 1, p.N);
    p.nitems_max = u.nitems > c.nitems ? u.nitems : c.nitems;
    return p;
}

namespace {
// Workspace of a plan.  The split of A (its SA planes, chunk exponents and row
// maxima) comes first, so that plans of the same m, ldp and SA share it.
struct TcLayout {
    __nv_bfloat16 *Ap, *Zp, *Up;
    int *eA, *mA, *eZ, *eU, *mZ, *mU, *cum1, *cum2;
    double *slots, *U, *Cm;
    size_t bytes;
};
TcLayout tc_layout(const TcPlan& p, void* ws)
{
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    char* base = static_cast<char*>(ws);
    size_t o = 0;
    auto take = [&](size_t bytes) {
        char* q = base ? base + o : nullptr;
        o += al(bytes);
        return q;
    };
    const size_t planeA = p.noA ? 0 : (size_t)p.m * p.ldp, planeZ = (size_t)p.n * p.ldp;  // elements
    const size_t rowsA = p.noA ? 0 : (size_t)p.m;
    TcLayout L;
    L.Ap = reinterpret_cast<__nv_bfloat16*>(take((size_t)p.SA * planeA * p.es));
    L.eA = reinterpret_cast<int*>(take((size_t)p.kch * rowsA * 4));
    L.mA = reinterpret_cast<int*>(take(rowsA * 4));
    L.Zp = reinterpret_cast<__nv_bfloat16*>(take((size_t)p.S * planeZ * p.es));
    L.Up = reinterpret_cast<__nv_bfloat16*>(take((size_t)p.S * planeZ * p.es));
    L.eZ = reinterpret_cast<int*>(take((size_t)p.kch * p.n * 4));
    L.eU = reinterpret_cast<int*>(take((size_t)p.kch * p.n * 4));
    L.mZ = reinterpret_cast<int*>(take((size_t)p.n * 4));
    L.mU = reinterpret_cast<int*>(take((size_t)p.n * 4));
    L.cum1 = reinterpret_cast<int*>(take((size_t)((p.m + TM - 1) / TM + 2) * 4));
    L.cum2 = reinterpret_cast<int*>(take((size_t)((p.m + TM - 1) / TM + 2) * 4));
    L.slots = reinterpret_cast<double*>(take(tc_plan_bytes(p)));
    L.U = reinterpret_cast<double*>(take(p.noA ? 0 : (size_t)p.m * p.n * 8));
    L.Cm = reinterpret_cast<double*>(take((size_t)p.n * p.n * 8));
    L.bytes = o;
    return L;
}
}  // namespace

size_t tc_workspace_bytes(const TcPlan& p) { return tc_layout(p, nullptr).bytes; }

// The EMU64-family split of A made one 256-column chunk at a time (as the
// chunks' columns arrive): tc_split_a_begin once, then tc_split_a_chunk for
// chunks kc = 0, 1, ... in any order; the result equals the split made inside
// launch_tc_gram for the same plan (mode 1 or 3, same SA).
cudaError_t tc_split_a_begin(const TcPlan& p, void* ws, cudaStream_t s)
{
    const TcLayout L = tc_layout(p, ws);
    fill_int_kernel<<<(p.m + 255) / 256, 256, 0, s>>>(L.mA, p.m, EXP_NONE);
    return cudaGetLastError();
}
cudaError_t tc_split_a_chunk(const TcPlan& p, const double* A, long lda, int kc, void* ws, cudaStream_t s)
{
    if (p.mode != 1 && p.mode != 3) return cudaErrorInvalidValue;
    const TcLayout L = tc_layout(p, ws);
    const int row0 = kc * KCH_EMU;  // rows above the chunk's first column hold only upper-triangle tiles
    const int rows = p.m - row0;
    if (rows <= 0) return cudaSuccess;
    const size_t plane = (size_t)p.m * p.ldp;
    split_lower_kernel<1, true, KCH_EMU><<<dim3(1, (p.m + 15) / 16), 256, 0, s>>>(p.m, p.m, A, lda, p.SA, L.Ap, p.ldp,
                                                                                plane, L.eA, L.mA, kc);
    return cudaGetLastError();
}

namespace {
// The split kernels of a plan's mode: TC2 (mode 3) takes the leading slices of the EMU64 split;
// the EMU64 family uses 256-long exponent chunks (16-row tiles), FP8 and BF16X3 128-long ones.
void split_lower_mode(const TcPlan& p, cudaStream_t s, const double* A, long lda, __nv_bfloat16* P, int* e, int* mx)
{
    const size_t plane = (size_t)p.m * p.ldp;
    if (p.mode == 1 || p.mode == 3)
        split_lower_kernel<1, true, KCH_EMU><<<dim3(p.kch, (p.m + 15) / 16), 256, 0, s>>>(p.m, p.m, A, lda, p.SA, P,
                                                                                        p.ldp, plane, e, mx);
    else if (p.mode == 2)
        split_lower_kernel<2, true, KCH_FP8><<<dim3(p.kch, (p.m + 31) / 32), 256, 0, s>>>(p.m, p.m, A, lda, p.SA, P,
                                                                                        p.ldp, plane, e, mx);
    else
        split_lower_kernel<0, true, KCH_FP8><<<dim3(p.kch, (p.m + 31) / 32), 256, 0, s>>>(p.m, p.m, A, lda, p.SA, P,
                                                                                        p.ldp, plane, e, mx);
}
void split_tall_mode(const TcPlan& p, cudaStream_t s, const double* X, long ldx, __nv_bfloat16* P, int* e, int* mx)
{
    const size_t plane = (size_t)p.n * p.ldp;
    const dim3 g(p.kch, (p.n + 7) / 8);
    if (p.mode == 1 || p.mode == 3)
        split_tall_kernel<1, KCH_EMU><<<g, 256, 0, s>>>(p.m, p.n, X, ldx, p.S, P, p.ldp, plane, e, mx);
    else if (p.mode == 2)
        split_tall_kernel<2, KCH_FP8><<<g, 256, 0, s>>>(p.m, p.n, X, ldx, p.S, P, p.ldp, plane, e, mx);
    else
        split_tall_kernel<0, KCH_FP8><<<g, 256, 0, s>>>(p.m, p.n, X, ldx, p.S, P, p.ldp, plane, e, mx);
}
cudaError_t launch_tc_mode(const TcPlan& p, const TcArgs& a, const void* PA, size_t planeA, const void* PB,
                           size_t planeB, int sms, cudaStream_t s)
{
    if (p.mode == 1) return launch_emu(a, PA, p.ldp, planeA, PB, p.ldp, planeB, sms, s);
    if (p.mode == 2) {
        if (p.N == 64) return launch_tc<128, 64, 1, 2>(a, PA, p.ldp, planeA, PB, p.ldp, planeB, sms, s);
        return launch_tc<128, 128, 1, 2>(a, PA, p.ldp, planeA, PB, p.ldp, planeB, sms, s);
    }
    if (p.mode == 3) {
        if (p.N == 64) return launch_tc<64, 64, 2, 3>(a, PA, p.ldp, planeA, PB, p.ldp, planeB, sms, s);
        return launch_tc<64, 128, 2, 3>(a, PA, p.ldp, planeA, PB, p.ldp, planeB, sms, s);
    }
    if (p.N == 64) return launch_tc<64, 64, 2, 0>(a, PA, p.ldp, planeA, PB, p.ldp, planeB, sms, s);
    if (p.N == 128) return launch_tc<64, 128, 2, 0>(a, PA, p.ldp, planeA, PB, p.ldp, planeB, sms, s);
    return launch_tc<64, 256, 2, 0>(a, PA, p.ldp, planeA, PB, p.ldp, planeB, sms, s);
}
void launch_slot_reduce(const TcPlan& p, const TcArgs& a, double* out, long ldo, const DevStatus* st, cudaStream_t s)
{
    const long tot = (long)a.rowsA * a.colsB;
    const unsigned g = (unsigned)((tot + 255) / 256);
    if (p.mode == 2 || p.mode == 3) {
        if (p.N == 64) slot_reduce_f32_kernel<64><<<g, 256, 0, s>>>(a, out, ldo, st);
        else slot_reduce_f32_kernel<128><<<g, 256, 0, s>>>(a, out, ldo, st);
        return;
    }
    if (p.N == 64) slot_reduce_kernel<64><<<g, 256, 0, s>>>(a, out, ldo, st);
    else if (p.N == 128) slot_reduce_kernel<128><<<g, 256, 0, s>>>(a, out, ldo, st);
    else slot_reduce_kernel<256><<<g, 256, 0, s>>>(a, out, ldo, st);
}
}  // namespace

namespace {
// The second product of the normal-equation matrix: C = X^T U on the tensor
// cores (X's planes already made), then G = C + C^T (+ shift).  U is FP64,
// m x n with leading dimension ldu.
cudaError_t tc_cross_phase(const TcPlan& p, const TcLayout& L, const double* U, long ldu, double* G, long ldg,
                           const double* shift_ptr, DevStatus* st, uint64_t limit_ns, int sms, cudaStream_t s,
                           cudaEvent_t* ev)
{
    const size_t planeZ = (size_t)p.n * p.ldp;
    const int mm = p.m, nn = p.n;
    split_tall_mode(p, s, U, ldu, L.Up, L.eU, L.mU);
    TcArgs a2 = make_args(p, nn, nn, mm, 0, p.N);
    a2.cum = L.cum2;
    a2.slots = L.slots;
    a2.eA = L.eZ;
    a2.eB = L.eU;
    a2.emaxA = L.mZ;
    a2.emaxB = L.mU;
    a2.st = st;
    a2.limit_ns = limit_ns;
    item_prefix_kernel<<<1, PREFIX_THREADS, 0, s>>>(a2, L.cum2);
    if (ev) cudaEventRecord(ev[3], s);
    cudaError_t e;
    if ((e = launch_tc_mode(p, a2, L.Zp, planeZ, L.Up, planeZ, sms, s)) != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[4], s);
    launch_slot_reduce(p, a2, L.Cm, nn, st, s);
    {
        const long tot = (long)nn * nn;
        symmetrize_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(nn, L.Cm, nn, G, ldg, shift_ptr, st);
    }
    if (ev) cudaEventRecord(ev[5], s);
    return cudaGetLastError();
}
}  // namespace

// G = X^T (M + M^T) X = C + C^T with C = X^T U, U = M X given (FP64, m x n):
// the normal-equation matrix of an A whose product M X the caller formed
// (tridiagonal A).  The plan has no planes of A (tc_plan(..., no_a = true)).
cudaError_t launch_tc_cross(const TcPlan& p, const double* X, long ldx, const double* U, long ldu, double* G, long ldg,
                            const double* shift_ptr, void* ws, DevStatus* st, uint64_t limit_ns, int sms,
                            cudaStream_t s)
{
    const TcLayout L = tc_layout(p, ws);
    const int nn = p.n;
    if (p.mode != 0) {
        fill_int_kernel<<<(nn + 255) / 256, 256, 0, s>>>(L.mZ, nn, EXP_NONE);
        fill_int_kernel<<<(nn + 255) / 256, 256, 0, s>>>(L.mU, nn, EXP_NONE);
    }
    split_tall_mode(p, s, X, ldx, L.Zp, L.eZ, L.mZ);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return tc_cross_phase(p, L, U, ldu, G, ldg, shift_ptr, st, limit_ns, sms, s, nullptr);
}

// C = X^T Y, FP64-accurate on the tensor cores, for X (K x n1) and Y (K x n2) of any widths (each up to
// the plane capacity given to tc_xty_bytes): the two column splits, the EMU64 product with items of
// XTY_PIECE k-steps (short, so that a narrow output still spreads over the SMs), the reduction of each
// element's pieces in order.  C is n1 x n2 with leading dimension ldc.
namespace {
constexpr int XTY_PIECE = 2 * EMU_CH;  // k-steps per item: two exponent chunks
struct XtyLayout {
    __nv_bfloat16 *Xp, *Yp;
    int *eX, *eY, *mX, *mY, *cum;
    double* slots;
    size_t bytes;
};
XtyLayout xty_layout(int K, int n1, int n2, void* ws)
{
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    char* base = static_cast<char*>(ws);
    size_t o = 0;
    auto take = [&](size_t bytes) {
        char* q = base ? base + o : nullptr;
        o += al(bytes);
        return q;
    };
    const long ldp = ((long)K + KCH_EMU - 1) / KCH_EMU * KCH_EMU;
    const int kch = (int)(ldp / KCH_EMU);
    const long items = (long)((n1 + TM - 1) / TM) * ((n2 + EMU_N - 1) / EMU_N) *
                       ((ldp / EMU_KS + XTY_PIECE - 1) / XTY_PIECE);
    XtyLayout L;
    L.Xp = reinterpret_cast<__nv_bfloat16*>(take((size_t)EMU_S * n1 * ldp * 2));
    L.Yp = reinterpret_cast<__nv_bfloat16*>(take((size_t)EMU_S * n2 * ldp * 2));
    L.eX = reinterpret_cast<int*>(take((size_t)kch * n1 * 4));
    L.eY = reinterpret_cast<int*>(take((size_t)kch * n2 * 4));
    L.mX = reinterpret_cast<int*>(take((size_t)n1 * 4));
    L.mY = reinterpret_cast<int*>(take((size_t)n2 * 4));
    L.cum = reinterpret_cast<int*>(take((size_t)((n1 + TM - 1) / TM + 2) * 4));
    L.slots = reinterpret_cast<double*>(take((size_t)items * TM * EMU_N * 8));
    L.bytes = o;
    return L;
}
}  // namespace

size_t tc_xty_bytes(int K, int n1, int n2) { return xty_layout(K, n1, n2, nullptr).bytes; }

cudaError_t launch_tc_xty(int K, int n1, int n2, const double* X, long ldx, const double* Y, long ldy, double* C,
                          long ldc, void* ws, DevStatus* st, uint64_t limit_ns, int sms, cudaStream_t s,
                          const int* gate, int want)
{
    if (K <= 0 || n1 <= 0 || n2 <= 0) return cudaSuccess;
    const XtyLayout L = xty_layout(K, n1, n2, ws);
    const long ldp = ((long)K + KCH_EMU - 1) / KCH_EMU * KCH_EMU;
    const int kch = (int)(ldp / KCH_EMU);
    const size_t planeX = (size_t)n1 * ldp, planeY = (size_t)n2 * ldp;
    fill_int_kernel<<<(n1 + 255) / 256, 256, 0, s>>>(L.mX, n1, EXP_NONE);
    fill_int_kernel<<<(n2 + 255) / 256, 256, 0, s>>>(L.mY, n2, EXP_NONE);
    split_tall_kernel<1, KCH_EMU><<<dim3(kch, (n1 + 7) / 8), 256, 0, s>>>(K, n1, X, ldx, EMU_S, L.Xp, ldp, planeX,
                                                                          L.eX, L.mX, gate, want);
    split_tall_kernel<1, KCH_EMU><<<dim3(kch, (n2 + 7) / 8), 256, 0, s>>>(K, n2, Y, ldy, EMU_S, L.Yp, ldp, planeY,
                                                                          L.eY, L.mY, gate, want);
    TcArgs a{};
    a.gate = gate;
    a.gate_want = want;
    a.rowsA = n1;
    a.colsB = n2;
    a.K = K;
    a.tri = 0;
    a.ks = EMU_KS;
    a.piece = XTY_PIECE;
    a.cc = (n2 + EMU_N - 1) / EMU_N;
    a.rt = (n1 + TM - 1) / TM;
    int items = 0;
    for (int I = 0; I < a.rt; ++I) items += pieces_of(a, I) * a.cc;
    a.nitems = items;
    a.cum = L.cum;
    a.slots = L.slots;
    a.eA = L.eX;
    a.eB = L.eY;
    a.emaxA = L.mX;
    a.emaxB = L.mY;
    a.st = st;
    a.limit_ns = limit_ns;
    item_prefix_kernel<<<1, PREFIX_THREADS, 0, s>>>(a, L.cum);
    cudaError_t e = launch_emu(a, L.Xp, ldp, planeX, L.Yp, ldp, planeY, sms, s);
    if (e != cudaSuccess) return e;
    const long tot = (long)n1 * n2;
    slot_reduce_kernel<EMU_N><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(a, C, ldc, st);
    return cudaGetLastError();
}

// G = Z^T A Z (+ shift) from A's lower triangle on the tensor cores; see the
// file comment.  ws holds tc_workspace_bytes(p).  a_ready: the workspace
// already holds the split of this A (planes, exponents, row maxima) made by a
// plan with the same m and SA, and it is not made again.
cudaError_t launch_tc_gram(const TcPlan& p, const double* A, long lda, const double* Z, long ldz, double* G, long ldg,
                           const double* shift_ptr, void* ws, DevStatus* st, uint64_t limit_ns, int sms,
                           cudaStream_t s, cudaEvent_t* ev, bool a_ready)
{
    auto mark = [&](int i) {
        if (ev) cudaEventRecord(ev[i], s);
    };
    mark(0);
    const TcLayout L = tc_layout(p, ws);
    const size_t planeA = (size_t)p.m * p.ldp, planeZ = (size_t)p.n * p.ldp;  // elements
    const int mm = p.m, nn = p.n;
    cudaError_t e;
    if (p.mode != 0) {
        if (!a_ready) fill_int_kernel<<<(mm + 255) / 256, 256, 0, s>>>(L.mA, mm, EXP_NONE);
        fill_int_kernel<<<(nn + 255) / 256, 256, 0, s>>>(L.mZ, nn, EXP_NONE);
        fill_int_kernel<<<(nn + 255) / 256, 256, 0, s>>>(L.mU, nn, EXP_NONE);
    }
    if (!a_ready) split_lower_mode(p, s, A, lda, L.Ap, L.eA, L.mA);
    split_tall_mode(p, s, Z, ldz, L.Zp, L.eZ, L.mZ);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // U = M Z (triangular)
    TcArgs a1 = make_args(p, mm, nn, mm, 1, p.N);
    a1.cum = L.cum1;
    a1.slots = L.slots;
    a1.eA = L.eA;
    a1.eB = L.eZ;
    a1.emaxA = L.mA;
    a1.emaxB = L.mZ;
    a1.st = st;
    a1.limit_ns = limit_ns;
    item_prefix_kernel<<<1, PREFIX_THREADS, 0, s>>>(a1, L.cum1);
    mark(1);
    if ((e = launch_tc_mode(p, a1, L.Ap, planeA, L.Zp, planeZ, sms, s)) != cudaSuccess) return e;
    mark(2);
    launch_slot_reduce(p, a1, L.U, mm, st, s);
    // C = Z^T U (left operand: Z's columns as rows, K-major), then G = C + C^T
    return tc_cross_phase(p, L, L.U, mm, G, ldg, shift_ptr, st, limit_ns, sms, s, ev);
}

// ------------------------------------------------------ blocked TRSM ----
// Q = Z / R (Algorithm 1, line 4) in 64-column blocks: for block J,
//   U = Q(:, 0:64J) R(0:64J, block)      FP64-accurate EMU64 product (tensor cores)
//   Q(:, block) = (Z(:, block) - U) R(block, block)^{-1}   FP64 row-wise substitution.
// The products carry the m n^2 / 2 - m n 32 FMAs of the off-diagonal part; the
// substitution keeps the diagonal blocks' m n 32 FMAs on the FP64 pipe.
namespace {
constexpr int TRSM_BW = 64;
struct TrsmLayout {
    __nv_bfloat16 *Xp, *Yp;
    int *eX, *mX, *eY, *mY, *cum;
    double *slots, *U;
    long ldp;
    int kch;
    size_t bytes;
};
TrsmLayout trsm_layout(int m, int n, void* ws)
{
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    char* base = static_cast<char*>(ws);
    size_t o = 0;
    auto take = [&](size_t bytes) {
        char* q = base ? base + o : nullptr;
        o += al(bytes);
        return q;
    };
    TrsmLayout L;
    const int kmax = n > TRSM_BW ? ((n - 1) / TRSM_BW) * TRSM_BW : 1;  // largest off-diagonal K
    L.ldp = ((long)kmax + KCH_EMU - 1) / KCH_EMU * KCH_EMU;
    L.kch = (kmax + KCH_EMU - 1) / KCH_EMU;
    const int rt = (m + TM - 1) / TM;
    const int pieces = (int)((L.ldp + 2047) / 2048);  // 2048-long items
    L.Xp = reinterpret_cast<__nv_bfloat16*>(take((size_t)EMU_S * m * L.ldp * 2));
    L.Yp = reinterpret_cast<__nv_bfloat16*>(take((size_t)EMU_S * TRSM_BW * L.ldp * 2));
    L.eX = reinterpret_cast<int*>(take((size_t)L.kch * m * 4));
    L.mX = reinterpret_cast<int*>(take((size_t)m * 4));
    L.eY = reinterpret_cast<int*>(take((size_t)L.kch * TRSM_BW * 4));
    L.mY = reinterpret_cast<int*>(take((size_t)TRSM_BW * 4));
    L.cum = reinterpret_cast<int*>(take((size_t)(rt + 2) * 4));
    L.slots = reinterpret_cast<double*>(take((size_t)rt * pieces * TM * EMU_N * 8));
    L.U = reinterpret_cast<double*>(take((size_t)m * TRSM_BW * 8));
    L.bytes = o;
    return L;
}
}  // namespace

size_t trsm_tc_workspace_bytes(int m, int n) { return trsm_layout(m, n, nullptr).bytes; }

cudaError_t launch_trsm_tc(int m, int n, const double* Z, long ldz, const double* R, long ldr, double* Q, long ldq,
                           void* ws, DevStatus* st, uint64_t limit_ns, int sms, cudaStream_t s, const int* gate,
                           int want)
{
    if (m <= 0 || n <= 0) return cudaSuccess;
    const TrsmLayout L = trsm_layout(m, n, ws);
    TcPlan p{};
    p.mode = 1;  // make_args: EMU64 k-step and piece
    cudaError_t e;
    for (int jb = 0; jb < n; jb += TRSM_BW) {
        const int bw = n - jb < TRSM_BW ? n - jb : TRSM_BW;
        const double* U = nullptr;
        if (jb > 0) {
            const int K = jb;
            const int kch = (K + KCH_EMU - 1) / KCH_EMU;
            fill_int_kernel<<<(m + 255) / 256, 256, 0, s>>>(L.mX, m, EXP_NONE);
            fill_int_kernel<<<1, TRSM_BW, 0, s>>>(L.mY, bw, EXP_NONE);
            const size_t planeX = (size_t)m * L.ldp, planeY = (size_t)TRSM_BW * L.ldp;
            split_lower_kernel<1, false, KCH_EMU><<<dim3(kch, (m + 15) / 16), 256, 0, s>>>(
                m, K, Q, ldq, EMU_S, L.Xp, L.ldp, planeX, L.eX, L.mX, 0, gate, want);
            split_tall_kernel<1, KCH_EMU><<<dim3(kch, (bw + 7) / 8), 256, 0, s>>>(K, bw, R + (long)jb * ldr, ldr, EMU_S,
                                                                                  L.Yp, L.ldp, planeY, L.eY, L.mY,
                                                                                  gate, want);
            TcArgs a = make_args(p, m, bw, K, 0, EMU_N);
            a.gate = gate;
            a.gate_want = want;
            a.cum = L.cum;
            a.slots = L.slots;
            a.eA = L.eX;
            a.eB = L.eY;
            a.emaxA = L.mX;
            a.emaxB = L.mY;
            a.st = st;
            a.limit_ns = limit_ns;
            item_prefix_kernel<<<1, PREFIX_THREADS, 0, s>>>(a, L.cum);
            if ((e = launch_emu(a, L.Xp, L.ldp, planeX, L.Yp, L.ldp, planeY, sms, s)) != cudaSuccess) return e;
            slot_reduce_kernel<EMU_N><<<(unsigned)(((long)m * bw + 255) / 256), 256, 0, s>>>(a, L.U, m, st);
            U = L.U;
        }
        if ((e = launch_trsm_block(m, jb, bw, Z, ldz, U, m, R, ldr, Q, ldq, st, s, gate, want)) != cudaSuccess)
            return e;
    }
    return cudaGetLastError();
}

// ------------------------------------------------------ packed batches ----
constexpr int BATCH_ITEMS_TARGET = 4 * 152;  // items of an n x n product: a few per SM
// Waves of instances (see oqr_internal.cuh): per wave the A planes hold the
// instances' rows one after another (instance b at packed row r_b) and the Z
// and U planes their columns (instance b at packed column c_b).  A work item
// of instance b reads its own rows and columns; rows and columns of a tile
// that pass the instance's end belong to the next instance (or are zero
// filled by the tensor map) and only touch outputs that the drain discards.
namespace {
struct WaveLayout {
    __nv_bfloat16 *Ap, *Zp, *Up;
    int *eA, *mA, *eZ, *mZ, *eU, *mU;
    double* slots;
    double* asq;  // the A split's per-tile shares of ||A||_F^2
    double* zsq;  // pass 0's Z split: per chunk and column, the sum of squares
    int* alist;   // a launch's active items (max_items + 1)
    int* rlist;   // a launch's active reduction blocks (max_rblk + 1)
    size_t bytes;
};
WaveLayout wave_layout(const TcBatchWave& w, void* ws)
{
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    char* base = static_cast<char*>(ws);
    size_t o = 0;
    auto take = [&](size_t bytes) {
        char* q = base ? base + o : nullptr;
        o += al(bytes);
        return q;
    };
    WaveLayout L;
    L.Ap = reinterpret_cast<__nv_bfloat16*>(take((size_t)EMU_S * w.rows * w.ldp * 2));
    L.eA = reinterpret_cast<int*>(take((size_t)w.kch * w.rows * 4));
    L.mA = reinterpret_cast<int*>(take((size_t)w.rows * 4));
    L.Zp = reinterpret_cast<__nv_bfloat16*>(take((size_t)EMU_S * w.cols * w.ldp * 2));
    L.Up = reinterpret_cast<__nv_bfloat16*>(take((size_t)EMU_S * w.cols * w.ldp * 2));
    L.eZ = reinterpret_cast<int*>(take((size_t)w.kch * w.cols * 4));
    L.eU = reinterpret_cast<int*>(take((size_t)w.kch * w.cols * 4));
    L.mZ = reinterpret_cast<int*>(take((size_t)w.cols * 4));
    L.mU = reinterpret_cast<int*>(take((size_t)w.cols * 4));
    L.slots = reinterpret_cast<double*>(take((size_t)w.max_items * TM * EMU_N * 8));
    L.asq = reinterpret_cast<double*>(take((size_t)w.tilesA * 8));
    L.zsq = reinterpret_cast<double*>(take((size_t)w.kch * w.cols * 8));
    L.alist = reinterpret_cast<int*>(take((size_t)(w.max_items + 1) * 4));
    L.rlist = reinterpret_cast<int*>(take((size_t)(w.max_rblk + 1) * 4));
    L.bytes = o;
    return L;
}
int batch_ks(int mode) { return mode == 1 ? EMU_KS : 64; }
// Items of one instance's product: U = M Z (tri, rows m) or C = Z^T U (rows n),
// in pieces of piece_k along k (a multiple of the 256-long exponent chunk).
int batch_items(int rows, int cols, int K, int tri, int mode, int piece_k)
{
    const int ks = batch_ks(mode), piece = piece_k / ks;
    const int rt = (rows + TM - 1) / TM, cc = (cols + EMU_N - 1) / EMU_N;
    int s = 0;
    for (int I = 0; I < rt; ++I) s += pieces_of(K, tri, ks, piece, I) * cc;
    return s;
}
// Members of a launch of pass p: the instances with more than p passes; pass 0 has one launch per
// first-pass mode present (TC2, then EMU64), later passes one EMU64 launch.
std::vector<int> launch_members(const std::vector<TcBatchShape>& sh, const TcBatchWave& w, int pass, int mode)
{
    std::vector<int> v;
    for (int b = w.first; b < w.first + w.count; ++b)
        if (sh[b].npass > pass && (pass > 0 || sh[b].mode0 == mode)) v.push_back(b);
    return v;
}
}  // namespace

TcBatchPlan tc_batch_plan(const std::vector<TcBatchShape>& sh, size_t budget)
{
    TcBatchPlan p;
    const int count = (int)sh.size();
    size_t tab = 0;
    auto tk = [&](size_t bytes) {
        const size_t o = tab;
        tab += (bytes + 255) & ~size_t(255);
        return o;
    };
    int b = 0;
    while (b < count) {
        TcBatchWave w{};
        w.first = b;
        w.K = sh[b].m;  // the largest m of the wave (sorted order)
        w.ldp = ((long)w.K + KCH_EMU - 1) / KCH_EMU * KCH_EMU;
        w.kch = (int)(w.ldp / KCH_EMU);
        long rows = 0, cols = 0;
        int e = b;
        while (e < count) {
            const long r2 = rows + sh[e].m, c2 = cols + sh[e].n;
            if (e > b && (size_t)EMU_S * 2 * w.ldp * (r2 + 2 * c2) > budget) break;
            rows = r2;
            cols = c2;
            ++e;
        }
        w.count = e - b;
        w.rows = rows;
        w.cols = cols;
        w.splitA = tk((size_t)w.count * sizeof(SplitInst));
        w.splitZ = tk((size_t)w.count * sizeof(SplitInst));
        w.splitQ = tk((size_t)w.count * sizeof(SplitInst));
        w.splitU = tk((size_t)w.count * sizeof(SplitInst));
        w.tilesA = 0;
        w.upool = 0;
        for (int i = b; i < e; ++i) {
            const int nrb = (sh[i].m + 15) / 16;
            for (int kc = 0; kc * KCH_EMU < sh[i].m; ++kc) w.tilesA += nrb - 16 * kc;  // lower-triangle tiles
            w.upool += (long)sh[i].m * sh[i].n;
        }
        w.tileTab = tk((size_t)w.tilesA * 4);
        w.colTab = tk((size_t)w.cols * 4);
        w.max_items = 1;
        w.max_rblk = 1;
        w.maxpass = 1;
        for (int i = b; i < e; ++i)
            if (sh[i].npass > w.maxpass) w.maxpass = sh[i].npass;
        for (int pass = 0; pass < TC_BATCH_MAX_PASS; ++pass) {
            w.nl[pass] = 0;
            const int modes[2] = {3, 1};
            for (int k = 0; k < 2 && pass < w.maxpass; ++k) {
                if (pass > 0 && k == 0) continue;
                const std::vector<int> mem = launch_members(sh, w, pass, modes[k]);
                if (mem.empty()) continue;
                const int li = w.nl[pass]++;
                for (int prod = 0; prod < 2; ++prod) {
                    TcBatchLaunch& L = prod == 0 ? w.u[pass][li] : w.c[pass][li];
                    L.mode = modes[k];
                    L.ninst = (int)mem.size();
                    // the n x n products have few tiles: shorter pieces until every SM has a few items
                    L.piece_k = 2048;
                    for (;;) {
                        L.nitems = 0;
                        for (int i : mem) {
                            const int rows_i = prod == 0 ? sh[i].m : sh[i].n;
                            L.nitems += batch_items(rows_i, sh[i].n, sh[i].m, prod == 0, L.mode, L.piece_k);
                        }
                        if (prod == 0 || L.piece_k == KCH_EMU || L.nitems >= BATCH_ITEMS_TARGET) break;
                        L.piece_k /= 2;
                    }
                    L.nrblk = 0;
                    long ncum = 0;
                    for (int i : mem) {
                        const int rows_i = prod == 0 ? sh[i].m : sh[i].n;
                        L.nrblk += (int)(((long)rows_i * sh[i].n + 255) / 256);
                        ncum += (rows_i + TM - 1) / TM + 1;
                    }
                    L.inst = tk((size_t)L.ninst * sizeof(TcInst));
                    L.item0 = tk((size_t)(L.ninst + 1) * 4);
                    L.cum = tk((size_t)ncum * 4);
                    L.rblk = tk((size_t)L.nrblk * 4);
                    if (L.nrblk > w.max_rblk) w.max_rblk = L.nrblk;
                    if (L.nitems > w.max_items) w.max_items = L.nitems;
                }
            }
        }
        const size_t sb = wave_layout(w, nullptr).bytes;
        if (sb > p.scratch_bytes) p.scratch_bytes = sb;
        if (w.upool > p.upool_doubles) p.upool_doubles = w.upool;
        p.waves.push_back(w);
        b = e;
    }
    p.table_bytes = tab;
    return p;
}

void tc_batch_tables(const TcBatchPlan& p, const std::vector<TcBatchShape>& sh, const std::vector<TcBatchIn>& in,
                     const void* table_dev, double* upool, std::vector<char>& image)
{
    (void)table_dev;
    image.assign(p.table_bytes, 0);
    char* img = image.data();
    for (const TcBatchWave& w : p.waves) {
        std::vector<long> roff(w.count), coff(w.count), uoff(w.count);
        long r = 0, c = 0, u = 0;
        for (int i = 0; i < w.count; ++i) {
            roff[i] = r;
            coff[i] = c;
            uoff[i] = u;
            r += sh[w.first + i].m;
            c += sh[w.first + i].n;
            u += (long)sh[w.first + i].m * sh[w.first + i].n;
        }
        SplitInst* sa = reinterpret_cast<SplitInst*>(img + w.splitA);
        SplitInst* sz = reinterpret_cast<SplitInst*>(img + w.splitZ);
        SplitInst* sq = reinterpret_cast<SplitInst*>(img + w.splitQ);
        SplitInst* su = reinterpret_cast<SplitInst*>(img + w.splitU);
        int* tiles = reinterpret_cast<int*>(img + w.tileTab);
        int* colinst = reinterpret_cast<int*>(img + w.colTab);
        int nt = 0;
        for (int i = 0; i < w.count; ++i) {
            const int b = w.first + i, m = sh[b].m, n = sh[b].n, kch = (m + KCH_EMU - 1) / KCH_EMU;
            sa[i] = SplitInst{in[b].A, in[b].lda, m, m, 0, roff[i], kch, nt, 0};
            sz[i] = SplitInst{in[b].Z, in[b].ldz, 0, m, n, coff[i], kch, 0, 0};
            sq[i] = SplitInst{in[b].Q, in[b].ldq, 0, m, n, coff[i], kch, 0, 0};
            su[i] = SplitInst{upool + uoff[i], (long)m, 0, m, n, coff[i], kch, 0, 0};
            const int nrb = (m + 15) / 16;
            for (int kc = 0; kc < kch; ++kc)
                for (int ib = 16 * kc; ib < nrb; ++ib) tiles[nt++] = (i << 12) | (kc << 8) | ib;
            sa[i].ntiles = nt - sa[i].tile0;
            for (int c = 0; c < n; ++c) colinst[coff[i] + c] = i;
        }
        for (int pass = 0; pass < w.maxpass; ++pass)
            for (int li = 0; li < w.nl[pass]; ++li)
                for (int prod = 0; prod < 2; ++prod) {
                    const TcBatchLaunch& L = prod == 0 ? w.u[pass][li] : w.c[pass][li];
                    const std::vector<int> mem = launch_members(sh, w, pass, L.mode);
                    TcInst* ti = reinterpret_cast<TcInst*>(img + L.inst);
                    int* item0 = reinterpret_cast<int*>(img + L.item0);
                    int* cum = reinterpret_cast<int*>(img + L.cum);
                    int* rblk = reinterpret_cast<int*>(img + L.rblk);
                    const int ks = batch_ks(L.mode), piece = L.piece_k / ks;
                    int it = 0, cm = 0, nb = 0;
                    for (size_t k = 0; k < mem.size(); ++k) {
                        const int b = mem[k], i = b - w.first, m = sh[b].m, n = sh[b].n;
                        TcInst t{};
                        t.rows = prod == 0 ? m : n;
                        t.cols = n;
                        t.K = m;
                        t.tri = prod == 0;
                        t.roff = (int)(prod == 0 ? roff[i] : coff[i]);
                        t.coff = (int)coff[i];
                        t.rt = (t.rows + TM - 1) / TM;
                        t.cc = (t.cols + EMU_N - 1) / EMU_N;
                        t.item0 = it;
                        t.cum0 = cm;
                        t.out = prod == 0 ? upool + uoff[i] : in[b].C;
                        t.ldo = t.rows;
                        t.wi = i;
                        int s = 0;
                        for (int I = 0; I < t.rt; ++I) {
                            cum[cm + I] = s;
                            s += pieces_of(t.K, t.tri, ks, piece, I) * t.cc;
                        }
                        cum[cm + t.rt] = s;
                        ti[k] = t;
                        item0[k] = it;
                        it += s;
                        cm += t.rt + 1;
                        const int blocks = (int)(((long)t.rows * t.cols + 255) / 256);
                        for (int q = 0; q < blocks; ++q) rblk[nb++] = ((int)k << 10) | q;
                    }
                    item0[mem.size()] = it;
                }
    }
}

cudaError_t tc_batch_split_a(const TcBatchPlan& p, int w, const void* table_dev, void* scratch, cudaStream_t s)
{
    const TcBatchWave& W = p.waves[w];
    const WaveLayout L = wave_layout(W, scratch);
    const char* tab = static_cast<const char*>(table_dev);
    fill_int_kernel<<<(unsigned)((W.rows + 255) / 256), 256, 0, s>>>(L.mA, W.rows, EXP_NONE);
    split_lower_batch_kernel<<<W.tilesA, 256, 0, s>>>(reinterpret_cast<const SplitInst*>(tab + W.splitA),
                                                      reinterpret_cast<const int*>(tab + W.tileTab), EMU_S, L.Ap,
                                                      W.ldp, (size_t)W.rows * W.ldp, L.eA, L.mA, W.rows, L.asq);
    return cudaGetLastError();
}

cudaError_t tc_batch_norms(const TcBatchPlan& p, int w, const void* table_dev, void* scratch, double* anorm2,
                           double* znorm2, cudaStream_t s)
{
    const TcBatchWave& W = p.waves[w];
    const WaveLayout L = wave_layout(W, scratch);
    const char* tab = static_cast<const char*>(table_dev);
    if (W.count > 0)
        norms_batch_kernel<<<W.count, 128, 0, s>>>(reinterpret_cast<const SplitInst*>(tab + W.splitA),
                                                   reinterpret_cast<const SplitInst*>(tab + W.splitZ), L.asq, L.zsq,
                                                   W.cols, anorm2, znorm2);
    return cudaGetLastError();
}

cudaError_t tc_batch_gram(const TcBatchPlan& p, int w, int pass, const void* table_dev, void* scratch,
                          DevStatus* st, uint64_t limit_ns, int sms, cudaStream_t s, const int* live)
{
    const TcBatchWave& W = p.waves[w];
    const WaveLayout L = wave_layout(W, scratch);
    const char* tab = static_cast<const char*>(table_dev);
    const size_t planeA = (size_t)W.rows * W.ldp, planeZ = (size_t)W.cols * W.ldp;  // elements
    const dim3 gt(W.kch, (unsigned)((W.cols + 7) / 8));
    auto args = [&](const TcBatchLaunch& B, long rowsA, const int* eA, const int* eB, const int* mA,
                    const int* mB) {
        TcArgs a{};
        a.rowsA = (int)rowsA;
        a.colsB = (int)W.cols;
        a.K = W.K;
        a.ks = batch_ks(B.mode);
        a.piece = B.piece_k / a.ks;
        a.nitems = B.nitems;
        a.cum = reinterpret_cast<const int*>(tab + B.cum);
        a.slots = L.slots;
        a.eA = eA;
        a.eB = eB;
        a.emaxA = mA;
        a.emaxB = mB;
        a.st = st;
        a.limit_ns = limit_ns;
        a.ninst = B.ninst;
        a.inst = reinterpret_cast<const TcInst*>(tab + B.inst);
        a.inst_item0 = reinterpret_cast<const int*>(tab + B.item0);
        a.rblk = reinterpret_cast<const int*>(tab + B.rblk);
        a.nrblk = B.nrblk;
        a.live = live;
        a.pass = pass;
        a.list = live ? L.alist : nullptr;
        return a;
    };
    auto product = [&](const TcBatchLaunch& B, const TcArgs& a, const void* PA, size_t plA, const void* PB) {
        cudaError_t e;
        if (live) {  // the items and reduction blocks of the instances taking part in this pass
            active_items_kernel<false><<<1, ALIST_THREADS, 0, s>>>(a.inst, a.inst_item0, a.ninst, live, pass, L.alist);
            active_items_kernel<true><<<1, ALIST_THREADS, 0, s>>>(a.inst, a.inst_item0, a.ninst, live, pass, L.rlist);
        }
        if (B.mode == 1) e = launch_emu(a, PA, W.ldp, plA, PB, W.ldp, planeZ, sms, s);
        else e = launch_tc<64, 64, 2, 3>(a, PA, W.ldp, plA, PB, W.ldp, planeZ, sms, s);
        if (e != cudaSuccess) return e;
        const unsigned g = (unsigned)(B.nrblk < 16 * sms ? B.nrblk : 16 * sms);
        const int* rl = live ? L.rlist : nullptr;
        if (B.mode == 1) slot_reduce_batch_kernel<EMU_N, false><<<g, 256, 0, s>>>(a, rl);
        else slot_reduce_batch_kernel<EMU_N, true><<<g, 256, 0, s>>>(a, rl);
        return cudaGetLastError();
    };
    cudaError_t e;
    // the split of X (Z in pass 0, Q in pass 1), then U = M X for every launch of the pass
    fill_int_kernel<<<(unsigned)((W.cols + 255) / 256), 256, 0, s>>>(L.mZ, W.cols, EXP_NONE);
    const int* colinst = reinterpret_cast<const int*>(tab + W.colTab);
    split_tall_batch_kernel<<<gt, 256, 0, s>>>(reinterpret_cast<const SplitInst*>(tab + (pass ? W.splitQ : W.splitZ)),
                                               colinst, EMU_S, L.Zp, W.ldp, planeZ, L.eZ, L.mZ, W.cols, live, pass,
                                               pass == 0 ? L.zsq : nullptr);
    for (int li = 0; li < W.nl[pass]; ++li) {
        const TcBatchLaunch& B = W.u[pass][li];
        if ((e = product(B, args(B, W.rows, L.eA, L.eZ, L.mA, L.mZ), L.Ap, planeA, L.Zp)) != cudaSuccess) return e;
    }
    // the split of U, then C = X^T U
    fill_int_kernel<<<(unsigned)((W.cols + 255) / 256), 256, 0, s>>>(L.mU, W.cols, EXP_NONE);
    split_tall_batch_kernel<<<gt, 256, 0, s>>>(reinterpret_cast<const SplitInst*>(tab + W.splitU), colinst, EMU_S,
                                               L.Up, W.ldp, planeZ, L.eU, L.mU, W.cols, live, pass, nullptr);
    for (int li = 0; li < W.nl[pass]; ++li) {
        const TcBatchLaunch& B = W.c[pass][li];
        if ((e = product(B, args(B, W.cols, L.eZ, L.eU, L.mZ, L.mU), L.Zp, planeZ, L.Up)) != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

namespace {
typedef CUresult (*EncodeTiledFn3)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn3 encode3()
{
    static EncodeTiledFn3 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn3>(p);
        cudaGetLastError();
    }
    return fn;
}

// Slice planes: dims {K (contiguous), rows, S}; box {box_k, box_rows, 1};
// swizzle = box_k * 2 bytes (32, 64 or 128), matching the UMMA K-major layout.
bool make_map_3d(CUtensorMap* map, const void* base, long kext, long rows, long ldp, size_t plane_bytes, int S,
                 int box_k, int box_rows, int elem_bytes)
{
    EncodeTiledFn3 fn = encode3();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)kext, (cuuint64_t)rows, (cuuint64_t)S};
    cuuint64_t strides[2] = {(cuuint64_t)ldp * elem_bytes, (cuuint64_t)plane_bytes};
    cuuint32_t box[3] = {(cuuint32_t)box_k, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    const CUtensorMapSwizzle sw = box_k * elem_bytes == 128  ? CU_TENSOR_MAP_SWIZZLE_128B
                                  : box_k * elem_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                                             : CU_TENSOR_MAP_SWIZZLE_32B;
    const CUtensorMapDataType dt = elem_bytes == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    CUresult r = fn(map, dt, 3, const_cast<void*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}
}  // namespace

}  // namespace oqr
