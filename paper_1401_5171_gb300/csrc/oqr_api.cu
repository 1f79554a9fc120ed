// C-ABI layer of liboqr: argument checking, workspace, and the composition of
// the step kernels into A-CholQR, A-CholQR2, shifted A-CholQR3 and A-CGS2.
// Every arithmetic step runs in this library's CUDA kernels; the host only
// validates, carves workspace and enqueues.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "oqr_internal.cuh"

using namespace oqr;

struct oqr_ctx {
    int device = 0;
    int sm_count = 0;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    bool ws_owned = true;
    DevStatus* st = nullptr;  // device status block (owned, allocated at create)
    // cached CUDA graph of the batched sequence and the signature it was captured for
    cudaGraphExec_t batch_exec = nullptr;
    long batch_key[10] = {0};
    // the same for the batched tensor-core (mixed) sequence: its signature is every instance's shape
    cudaGraphExec_t mixed_exec = nullptr;
    std::vector<long> mixed_key;
    size_t batch_budget = 0;  // slice-plane bytes per wave of the tensor-core batches (0: the default)
    // host-buffer path: device staging (A, Z, Q, R), a copy stream and one event per panel of A
    void* stage = nullptr;
    size_t stage_bytes = 0;
    cudaStream_t copy_stream = nullptr;
    std::vector<cudaEvent_t> events;
    // the selector's fallback calls: their per-instance status and orth (device)
    void* sel_buf = nullptr;
    size_t sel_bytes = 0;
    // the selector's pinned host buffers (choices read back and tables uploaded while the GPU works on)
    void* pin = nullptr;
    size_t pin_bytes = 0;
    cudaEvent_t sel_ev[2] = {nullptr, nullptr};
};

namespace {

constexpr double U64 = 1.1102230246251565e-16;  // 2^-53

// An NVTX range over a scope (host side: the enqueue of a pass or a wave), for
// profilers' timelines and for filtering kernels by range.
struct NvtxRange {
    explicit NvtxRange(const char* fmt, int k)
    {
        char buf[64];
        snprintf(buf, sizeof(buf), fmt, k);
        nvtxRangePushA(buf);
    }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
constexpr int SHIFT_PARTS = 1024;
constexpr int CGS_MAX_SPLITS = 64;
constexpr int KCH_PANEL = 256;  // host-buffer path: columns per panel of A (the EMU64 exponent chunk)

void fill_defaults(oqr_opts* o)
{
    o->passes = 2;
    o->shifted = 0;
    o->prec = OQR_FP64;
    o->shift_c = 11.0;
    o->block = 64;
    o->check = 0;
    o->spin_limit = 4000000000L;
    o->final_prec = OQR_FP64;
    o->prec_mid = -1;
    o->reuse_w = 0;
    o->batch_splits = nullptr;
    o->selector_params = nullptr;
    o->selector_tol = 1e-12;
    o->selector_check = 0;
    o->batch_orth = nullptr;
    o->batch_choice = nullptr;
}

oqr_opts resolve(const oqr_opts* o)
{
    oqr_opts r;
    fill_defaults(&r);
    if (o) r = *o;
    if (r.passes <= 0) r.passes = 2;
    if (r.shift_c <= 0) r.shift_c = 11.0;
    if (r.block <= 0) r.block = 64;
    if (r.spin_limit <= 0) r.spin_limit = 4000000000L;
    return r;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Bump allocator over the workspace.
struct Carve {
    char* base;
    size_t off = 0;
    explicit Carve(void* b) : base(static_cast<char*>(b)) {}
    template <class T>
    T* take(size_t count)
    {
        T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
        off += align256(count * sizeof(T));
        return p;
    }
};

// The last pass's solve (see launch_last_solve): R^{-1} (n x n), ||G - I||_F, the gate, X^T (n x m) and
// the tensor-core product's workspace.
struct LastSolve {
    double *Rinv = nullptr, *defect = nullptr, *Xt = nullptr;
    int* gate = nullptr;
    void* xtyws = nullptr;
};
template <class C>
void carve_last(C& c, int m, int n, bool on, LastSolve* L)
{
    const size_t nn = (size_t)n * n, nm = (size_t)n * m;
    L->Rinv = c.template take<double>(on ? nn : 0);
    L->defect = c.template take<double>(on ? GRAM_DEFECT_DOUBLES : 0);
    L->Xt = c.template take<double>(on ? nm : 0);
    L->gate = c.template take<int>(on ? 1 : 0);
    L->xtyws = c.template take<char>(on ? tc_xty_bytes(n, m, n) : 0);
}

// The solve Q = X R^{-1} of a pass whose Gram G (= R^T R) is close to I, as the last pass of a multi-pass
// factorization is.  When ||G - I||_F <= 0.5 every eigenvalue of G lies in [0.5, 1.5], so kappa(R)^2 <= 3:
// then X times R^{-1} (FP64 back substitution) is one FP64-accurate tensor-core product, as accurate as
// the substitution (the explicit inverse's error grows with kappa(R)^2) and with the residual X - Q R
// within a few units of rounding.  Otherwise (a pass that starts far from orthogonality) FP64 row-wise
// substitution runs: one launch, so that the gated-off alternative costs one empty launch.  Both are
// enqueued; the gate written by the defect kernel makes the other's launches return at once, so the host
// never waits.  Q may alias X.
cudaError_t launch_last_solve(oqr_ctx* ctx, int m, int n, const double* G, long ldg, const double* X, long ldx,
                              const double* R, long ldr, double* Q, long ldq, const LastSolve& L, uint64_t limit,
                              cudaStream_t s)
{
    cudaError_t e;
    if ((e = launch_gram_defect(n, G, ldg, L.defect, L.gate, 0.5, s)) != cudaSuccess) return e;
    if ((e = launch_trinv(n, R, ldr, L.Rinv, n, ctx->st, s)) != cudaSuccess) return e;
    if ((e = launch_transpose(m, n, X, ldx, L.Xt, n, s)) != cudaSuccess) return e;  // X^T, n x m
    if ((e = launch_tc_xty(n, m, n, L.Xt, n, L.Rinv, n, Q, ldq, L.xtyws, ctx->st, limit, ctx->sm_count, s, L.gate,
                           1)) != cudaSuccess)
        return e;
    return launch_trsm(m, n, X, ldx, R, ldr, Q, ldq, ctx->st, s, L.gate, 0);
}

// Workspace of the normal-equation family: Gram partials, G (+ check work),
// three n x n triangles, shift scratch.
template <class C>
void layout_cholqr(C& c, const GramPlan& p, double** partials, double** G, double** work, double** R1,
                   double** R2, double** R3, double** scratch)
{
    const size_t n = p.n;
    *partials = c.template take<double>(gram_partials_bytes(p) / sizeof(double));
    *G = c.template take<double>(n * n);
    *work = c.template take<double>(n * n + 2 * n);
    *R1 = c.template take<double>(n * n);
    *R2 = c.template take<double>(n * n);
    *R3 = c.template take<double>(n * n);
    *scratch = c.template take<double>(2 * SHIFT_PARTS);
}

struct CgsLayout {
    GramPlan gp;
    int b, splits;
    double *AQ, *S, *r, *sk, *Gb, *R1, *R2, *Rt, *work, *Rj;
};

template <class C>
void layout_cgs2(C& c, CgsLayout& L, int m, int n)
{
    const int b = L.b;
    L.AQ = c.template take<double>((size_t)m * n);
    L.S = c.template take<double>((size_t)m * b);
    L.r = c.template take<double>((size_t)n * b);
    L.sk = c.template take<double>((size_t)L.splits * std::max(n, b) * b);
    L.Gb = c.template take<double>((size_t)b * b);
    L.R1 = c.template take<double>((size_t)b * b);
    L.R2 = c.template take<double>((size_t)b * b);
    L.Rt = c.template take<double>((size_t)b * b);
    L.Rj = c.template take<double>((size_t)b * b);
    L.work = c.template take<double>((size_t)b * b + 2 * b);
}

oqr_status cuda_status(cudaError_t e) { return e == cudaSuccess ? OQR_OK : OQR_ERR_CUDA; }

oqr_status ensure_ws(oqr_ctx* ctx, size_t need)
{
    if (need <= ctx->ws_bytes) return OQR_OK;
    if (!ctx->ws_owned) return OQR_ERR_NO_MEMORY;
    if (ctx->ws) {
        cudaDeviceSynchronize();
        cudaFree(ctx->ws);
        ctx->ws = nullptr;
        ctx->ws_bytes = 0;
    }
    size_t want = need + need / 8;
    if (cudaMalloc(&ctx->ws, want) != cudaSuccess) {
        cudaGetLastError();
        ctx->ws = nullptr;
        return OQR_ERR_NO_MEMORY;
    }
    ctx->ws_bytes = want;
    return OQR_OK;
}

bool bad_matrix(const void* p, long ld, long rows, long cols)
{
    if (rows > 0 && cols > 0 && p == nullptr) return true;
    return ld < std::max(1L, rows);
}

oqr_status check_common(oqr_ctx* ctx, int m, int n, const double* A, long lda, const double* Z, long ldz,
                        const double* Q, long ldq, const double* R, long ldr)
{
    if (!ctx) return OQR_ERR_INVALID_ARG;
    if (m < 1 || n < 1 || n > m) return OQR_ERR_INVALID_ARG;
    if (bad_matrix(A, lda, m, m) || bad_matrix(Z, ldz, m, n) || bad_matrix(Q, ldq, m, n) ||
        bad_matrix(R, ldr, n, n))
        return OQR_ERR_INVALID_ARG;
    if (n > 1024) return OQR_ERR_UNSUPPORTED;
    // Q may alias Z exactly; any other overlap between Q and Z is refused.
    if (Q != Z) {
        const char* q0 = reinterpret_cast<const char*>(Q);
        const char* q1 = reinterpret_cast<const char*>(Q + (size_t)ldq * (n - 1) + m);
        const char* z0 = reinterpret_cast<const char*>(Z);
        const char* z1 = reinterpret_cast<const char*>(Z + (size_t)ldz * (n - 1) + m);
        if (q0 < z1 && z0 < q1) return OQR_ERR_INVALID_ARG;
    }
    return OQR_OK;
}

// Reads the device status block after the stream has drained.
oqr_status finish(oqr_ctx* ctx, cudaStream_t s, oqr_info* info, int passes_run, bool checked)
{
    if (!info) return cuda_status(cudaGetLastError());
    if (cudaStreamSynchronize(s) != cudaSuccess) return OQR_ERR_CUDA;
    DevStatus h;
    if (cudaMemcpy(&h, ctx->st, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return OQR_ERR_CUDA;
    info->info = h.code == OQR_ERR_NOT_SPD ? h.info : 0;
    info->passes_run = passes_run;
    info->orth_err = checked ? h.orth2 : -1.0;
    info->shift = h.shift;
    return static_cast<oqr_status>(h.code);
}

#define OQR_TRY(x)                                  \
    do {                                            \
        cudaError_t e_ = (x);                       \
        if (e_ != cudaSuccess) return OQR_ERR_CUDA; \
    } while (0)

oqr_status reset_status(oqr_ctx* ctx, cudaStream_t s)
{
    return cuda_status(cudaMemsetAsync(ctx->st, 0, sizeof(DevStatus), s));
}

oqr_status run_check(oqr_ctx* ctx, const GramPlan& gp, const double* A, long lda, const double* Q, long ldq,
                     double* partials, double* G, double* work, double* E, long lde, uint64_t limit, cudaStream_t s,
                     void* tcws = nullptr, bool a_ready = false)
{
    if (tcws) {  // FP64-accurate Gram on the tensor cores (reusing the split of A when a_ready)
        const TcPlan tp = tc_plan(gp.m, gp.n, 1);
        OQR_TRY(launch_tc_gram(tp, A, lda, Q, ldq, G, gp.n, nullptr, tcws, ctx->st, limit, ctx->sm_count, s, nullptr,
                               a_ready));
    } else {
        OQR_TRY(launch_gram_f64(gp, A, lda, Q, ldq, partials, ctx->st, limit, s));
        OQR_TRY(launch_gram_reduce(gp, partials, G, gp.n, nullptr, ctx->st, s));
    }
    OQR_TRY(launch_check_finish(gp.n, G, gp.n, E, lde, work, ctx->st, s));
    return OQR_OK;
}

bool prec_ok(int p)
{
    return p == OQR_FP64 || p == OQR_BF16X3 || p == OQR_FP64_TC || p == OQR_FP8 || p == OQR_TC2;
}

int tc_mode_of(int prec) { return prec == OQR_FP64_TC ? 1 : prec == OQR_FP8 ? 2 : prec == OQR_TC2 ? 3 : 0; }

// Modes 1 (FP64_TC) and 3 (TC2) take their operands from the same split of A.
bool emu_family(int prec) { return prec == OQR_FP64_TC || prec == OQR_TC2; }

// Tracks which split of A the tensor-core workspace holds within one call, so
// that passes (and the check) of the EMU64 family split A once.
struct ASplit {
    int sa = 0;         // planes of A kept by the EMU64-family plans of this call
    bool emu = false;   // the workspace holds this call's EMU64-family split of A
};

// The operator A of a factorization: a dense SPD matrix read from its lower
// triangle (A, lda), or a tridiagonal one (d: diagonal, m entries; e:
// off-diagonal, m - 1 entries), Sec. 8's two workloads.
struct AOp {
    const double* A = nullptr;
    long lda = 0;
    const double* d = nullptr;
    const double* e = nullptr;
    bool tri() const { return d != nullptr; }
};
AOp dense_op(const double* A, long lda)
{
    AOp o;
    o.A = A;
    o.lda = lda;
    return o;
}

// Splits of the FP64 GEMM X^T U of a tridiagonal pass (at most the dense plan's partial count, whose
// buffer it reuses).
int tri_splits(const GramPlan& gp, int sms)
{
    const int tiles = ((gp.n + 63) / 64) * ((gp.n + 63) / 64);
    return std::max(1, std::min(std::min(64, gp.splits), 2 * sms / tiles));
}

// G = X^T A X (+ shift) in the requested arithmetic.  Tridiagonal A: U = M X
// into Ubuf (m x n), C = X^T U (FP64 GEMM into Cbuf, n x n, or the tensor
// cores), G = C + C^T.
cudaError_t form_gram(oqr_ctx* ctx, int prec, const GramPlan& gp, const AOp& op, const double* X, long ldx,
                      double* partials, double* G, const double* shift_ptr, void* tcws, uint64_t limit,
                      cudaStream_t s, ASplit* as = nullptr, double* Ubuf = nullptr, double* Cbuf = nullptr)
{
    if (op.tri()) {
        cudaError_t e = launch_tridiag_u(gp.m, gp.n, op.d, op.e, X, ldx, Ubuf, gp.m, s);
        if (e != cudaSuccess) return e;
        if (prec == OQR_FP64) {
            e = launch_gemm_f64(GEMM_T, gp.n, gp.n, gp.m, 1.0, X, ldx, Ubuf, gp.m, 0.0, Cbuf, gp.n, partials,
                                tri_splits(gp, ctx->sm_count), s);
            if (e != cudaSuccess) return e;
            return launch_sym_plus_transpose(gp.n, Cbuf, gp.n, G, gp.n, shift_ptr, ctx->st, s);
        }
        const TcPlan tp = tc_plan(gp.m, gp.n, tc_mode_of(prec), 0, true);
        return launch_tc_cross(tp, X, ldx, Ubuf, gp.m, G, gp.n, shift_ptr, tcws, ctx->st, limit, ctx->sm_count, s);
    }
    if (prec == OQR_FP64) {
        cudaError_t e = launch_gram_f64(gp, op.A, op.lda, X, ldx, partials, ctx->st, limit, s);
        if (e != cudaSuccess) return e;
        return launch_gram_reduce(gp, partials, G, gp.n, shift_ptr, ctx->st, s);
    }
    const bool fam = emu_family(prec);
    const TcPlan tp = tc_plan(gp.m, gp.n, tc_mode_of(prec), (fam && as) ? as->sa : 0);
    const bool ready = fam && as && as->emu;
    cudaError_t e = launch_tc_gram(tp, op.A, op.lda, X, ldx, G, gp.n, shift_ptr, tcws, ctx->st, limit, ctx->sm_count,
                                   s, nullptr, ready);
    if (as) as->emu = fam;  // any other tensor-core mode overwrites the region
    return e;
}

size_t tc_bytes_for(int m, int n, int prec_a, int prec_b, int sa = 0, bool tri = false)
{
    size_t b = 0;
    for (int pr : {prec_a, prec_b})
        if (pr != OQR_FP64)
            b = std::max(b, tc_workspace_bytes(tc_plan(m, n, tc_mode_of(pr), (emu_family(pr) && !tri) ? sa : 0, tri)));
    return b;
}

// Workspace plan of one normal-equation call: the FP64 layout (layout_cholqr),
// then the tensor-core Gram region shared by the passes (A's split first),
// then the blocked-TRSM region.
struct NePlan {
    int passes = 0;
    bool shifted = false;
    bool tri = false;  // tridiagonal A: no split of A, U = M X buffer (m x n) and C (n x n)
    int prec_first = 0, prec_mid = 0, prec_final = 0;
    int sa = 0;        // planes of A kept for the EMU64-family passes (7 with any FP64_TC, else 0)
    size_t tcb = 0;    // tensor-core Gram region
    size_t trb = 0;    // blocked-TRSM region
    bool last = false;  // the last pass solves with launch_last_solve (a tensor-core pass after another pass)
    int prec_of(int p) const { return p == passes - 1 ? prec_final : (p == 0 ? prec_first : prec_mid); }
};

oqr_status ne_plan(const oqr_opts& o, int forced_passes, int m, int n, NePlan* P, bool tri = false)
{
    P->tri = tri;
    if (!prec_ok(o.prec) || !prec_ok(o.final_prec)) return OQR_ERR_INVALID_ARG;
    P->passes = forced_passes > 0 ? forced_passes : (o.shifted ? 3 : o.passes);
    if (P->passes < 1 || P->passes > 8) return OQR_ERR_INVALID_ARG;
    P->shifted = forced_passes == 0 && o.shifted;
    P->prec_mid = o.prec_mid >= 0 ? o.prec_mid : o.prec;
    if (!prec_ok(P->prec_mid)) return OQR_ERR_INVALID_ARG;
    P->prec_final = o.final_prec;
    P->prec_first = P->passes == 1 ? o.final_prec : o.prec;
    // one split of A for the EMU64-family passes and the tensor-core check: 7 planes when any of them is FP64_TC
    P->sa = (!tri && (P->prec_first == OQR_FP64_TC || P->prec_mid == OQR_FP64_TC || P->prec_final == OQR_FP64_TC ||
                      o.check == 2))
                ? 7
                : 0;
    P->tcb = tc_bytes_for(m, n, P->prec_first, P->prec_final, P->sa, tri);
    P->tcb = std::max(P->tcb, tc_bytes_for(m, n, P->prec_mid, P->prec_mid, P->sa, tri));
    if (o.check == 2) P->tcb = std::max(P->tcb, tc_bytes_for(m, n, OQR_FP64_TC, OQR_FP64_TC, P->sa, tri));
    // passes whose Gram runs on the tensor cores also solve Q = X / R with tensor-core products
    const bool any_tc = P->prec_first != OQR_FP64 || P->prec_mid != OQR_FP64 || P->prec_final != OQR_FP64;
    P->trb = any_tc ? trsm_tc_workspace_bytes(m, n) : 0;
    P->last = P->passes > 1 && P->prec_final != OQR_FP64 && n <= TRINV_MAX_N;
    return OQR_OK;
}

struct NeBuffers {
    double *partials, *G, *work, *R1, *R2, *R3, *scratch;
    void *tcws, *trws;
    double *U, *C;  // tridiagonal A: U = M X (m x n) and C = X^T U (n x n)
    LastSolve last;  // the last pass's solve (a tensor-core last pass after another pass)
};
// base == nullptr: offsets only; returns the bytes.
size_t ne_carve(void* base, const GramPlan& gp, const NePlan& P, NeBuffers* B)
{
    Carve c(base);
    layout_cholqr(c, gp, &B->partials, &B->G, &B->work, &B->R1, &B->R2, &B->R3, &B->scratch);
    B->tcws = c.take<char>(P.tcb);
    B->trws = c.take<char>(P.trb);
    B->U = c.take<double>(P.tri ? (size_t)gp.m * gp.n : 0);
    B->C = c.take<double>(P.tri ? (size_t)gp.n * gp.n : 0);
    carve_last(c, gp.m, gp.n, P.last, &B->last);
    return c.off;
}

// a_split_ready: the workspace's tensor-core region already holds the split of
// this A made for the first pass's plan (the host-buffer path makes it while A
// arrives), so the first EMU64-family pass does not make it again.
// ws_reserve: bytes at the start of the workspace that the caller keeps (the
// call carves its buffers after them; the caller has grown the workspace).
oqr_status normal_equation(oqr_ctx* ctx, int m, int n, const AOp& op, const double* Z, long ldz, double* Q, long ldq,
                           double* R, long ldr, const oqr_opts* opts_in, oqr_info* info, void* stream,
                           int forced_passes, bool a_split_ready = false, size_t ws_reserve = 0)
{
    oqr_status v;
    if (op.tri()) {
        if (!ctx || m < 1 || n < 1 || n > m || (m > 1 && !op.e) || bad_matrix(Z, ldz, m, n) ||
            bad_matrix(Q, ldq, m, n) || bad_matrix(R, ldr, n, n))
            return OQR_ERR_INVALID_ARG;
        if (n > 1024) return OQR_ERR_UNSUPPORTED;
        if (Q != Z) {
            const char *q0 = reinterpret_cast<const char*>(Q), *q1 = reinterpret_cast<const char*>(Q + (size_t)ldq * (n - 1) + m);
            const char *z0 = reinterpret_cast<const char*>(Z), *z1 = reinterpret_cast<const char*>(Z + (size_t)ldz * (n - 1) + m);
            if (q0 < z1 && z0 < q1) return OQR_ERR_INVALID_ARG;
        }
    } else if ((v = check_common(ctx, m, n, op.A, op.lda, Z, ldz, Q, ldq, R, ldr)) != OQR_OK) {
        return v;
    }
    const oqr_opts o = resolve(opts_in);
    NePlan P;
    if ((v = ne_plan(o, forced_passes, m, n, &P, op.tri())) != OQR_OK) return v;
    const int passes = P.passes;
    const bool shifted = P.shifted;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint64_t limit = (uint64_t)o.spin_limit;
    const GramPlan gp = gram_plan(m, n, ctx->sm_count);
    const int prec_first = P.prec_first;
    auto prec_of = [&](int p) { return P.prec_of(p); };
    NeBuffers B;
    if ((v = ensure_ws(ctx, ws_reserve + ne_carve(nullptr, gp, P, &B))) != OQR_OK) return v;
    ne_carve(static_cast<char*>(ctx->ws) + ws_reserve, gp, P, &B);
    double *partials = B.partials, *G = B.G, *work = B.work, *R1 = B.R1, *R2 = B.R2, *R3 = B.R3,
           *scratch = B.scratch;
    void* tcws = B.tcws;
    void* trws = B.trws;
    ASplit as;
    as.sa = P.sa;
    as.emu = a_split_ready && emu_family(prec_first);
    ASplit* asp = op.tri() ? nullptr : &as;  // a tridiagonal A has no split to share
    if ((v = reset_status(ctx, s)) != OQR_OK) return v;

    const double* shift_ptr = nullptr;
    const bool trace_shift = shifted && (prec_first == OQR_BF16X3 || prec_first == OQR_FP8 || prec_first == OQR_TC2);
    if (shifted && !trace_shift) {
        if (op.tri())
            OQR_TRY(launch_tridiag_norms_and_shift(m, n, op.d, op.e, Z, ldz, o.shift_c, U64, scratch, 2 * SHIFT_PARTS,
                                                   ctx->st, s));
        else
            OQR_TRY(launch_norms_and_shift(m, n, op.A, op.lda, Z, ldz, o.shift_c, U64, scratch, 2 * SHIFT_PARTS,
                                           ctx->st, s));
        shift_ptr = &ctx->st->shift;
    }
    // R accumulates as R_p ... R_1; Racc alternates between R2 and R3.
    const double* X = Z;
    long ldx = ldz;
    double* Racc = nullptr;
    for (int p = 0; p < passes; ++p) {
        const NvtxRange range("oqr: normal-equation pass %d", p + 1);
        double* Rp = (passes == 1) ? R : R1;
        const long ldrp = (passes == 1) ? ldr : n;
        const int prec = prec_of(p);
        OQR_TRY(form_gram(ctx, prec, gp, op, X, ldx, partials, G, p == 0 ? shift_ptr : nullptr, tcws, limit, s, asp,
                          B.U, B.C));
        if (p == 0 && trace_shift)  // u of the first pass's products: 2^-16 (BF16X3, TC2) or 2^-4 (E4M3)
            OQR_TRY(launch_trace_shift(n, G, n, o.shift_c, prec == OQR_FP8 ? 0.0625 : 1.52587890625e-05, ctx->st, s));
        OQR_TRY(launch_potrf(n, G, n, Rp, ldrp, nullptr, ctx->st, s));
        if (P.last && p == passes - 1) {
            OQR_TRY(launch_last_solve(ctx, m, n, G, n, X, ldx, Rp, ldrp, Q, ldq, B.last, limit, s));
        } else if (prec != OQR_FP64) {
            OQR_TRY(launch_trsm_tc(m, n, X, ldx, Rp, ldrp, Q, ldq, trws, ctx->st, limit, ctx->sm_count, s));
        } else {
            OQR_TRY(launch_trsm(m, n, X, ldx, Rp, ldrp, Q, ldq, ctx->st, s));
        }
        if (passes > 1) {
            if (p == 0) {
                OQR_TRY(launch_copy_upper(n, R1, n, R2, n, s));
                Racc = R2;
            } else if (p == passes - 1) {
                OQR_TRY(launch_rprod(n, R1, n, Racc, n, R, ldr, s));
            } else {
                double* Rn = (Racc == R2) ? R3 : R2;
                OQR_TRY(launch_rprod(n, R1, n, Racc, n, Rn, n, s));
                Racc = Rn;
            }
        }
        X = Q;
        ldx = ldq;
    }
    if (o.check) {
        if (op.tri()) {
            OQR_TRY(form_gram(ctx, o.check == 2 ? OQR_FP64_TC : OQR_FP64, gp, op, Q, ldq, partials, G, nullptr, tcws,
                              limit, s, nullptr, B.U, B.C));
            OQR_TRY(launch_check_finish(n, G, n, nullptr, 0, work, ctx->st, s));
        } else if ((v = run_check(ctx, gp, op.A, op.lda, Q, ldq, partials, G, work, nullptr, 0, limit, s,
                                  o.check == 2 ? tcws : nullptr, as.emu && as.sa == 7)) != OQR_OK) {
            return v;
        }
    }
    return finish(ctx, s, info, passes, o.check != 0);
}

// A-CholQR2 with the first pass's W = A Z kept: A Q_1 = W R_1^{-1} replaces the
// second product with A (FP64, dense A).
oqr_status cholqr2_reuse_w(oqr_ctx* ctx, int m, int n, const double* A, long lda, const double* Z, long ldz,
                           double* Q, long ldq, double* R, long ldr, const oqr_opts& o, oqr_info* info,
                           cudaStream_t s)
{
    oqr_status v = check_common(ctx, m, n, A, lda, Z, ldz, Q, ldq, R, ldr);
    if (v != OQR_OK) return v;
    if (o.shifted || o.passes != 2 || o.prec != OQR_FP64 || o.final_prec != OQR_FP64 ||
        (o.prec_mid != -1 && o.prec_mid != OQR_FP64) || o.check == 2)
        return OQR_ERR_UNSUPPORTED;
    const uint64_t limit = (uint64_t)o.spin_limit;
    const GramPlan gp = gram_plan(m, n, ctx->sm_count);
    const int tiles = ((n + 63) / 64) * ((n + 63) / 64);
    const int splits = std::max(1, std::min(64, 2 * ctx->sm_count / tiles));
    auto layout = [&](Carve& c, double** W, double** sk, double** G, double** R1, double** R2, double** partials,
                      double** work) {
        *W = c.take<double>((size_t)m * n);
        *sk = c.take<double>(gemm_splitk_bytes(n, n, splits) / sizeof(double) + 1);
        *G = c.take<double>((size_t)n * n);
        *R1 = c.take<double>((size_t)n * n);
        *R2 = c.take<double>((size_t)n * n);
        *partials = c.take<double>(o.check ? gram_partials_bytes(gp) / sizeof(double) : 0);
        *work = c.take<double>((size_t)n * n + 2 * n);
    };
    double *W, *sk, *G, *R1, *R2, *partials, *work;
    Carve probe(nullptr);
    layout(probe, &W, &sk, &G, &R1, &R2, &partials, &work);
    if ((v = ensure_ws(ctx, probe.off)) != OQR_OK) return v;
    Carve c(ctx->ws);
    layout(c, &W, &sk, &G, &R1, &R2, &partials, &work);
    if ((v = reset_status(ctx, s)) != OQR_OK) return v;
    // pass 1: W = A Z, G_1 = Z^T W, R_1 = chol(G_1), Q_1 = Z / R_1, then W <- W / R_1 (= A Q_1 up to rounding)
    OQR_TRY(launch_gemm_f64(GEMM_SYML, m, n, m, 1.0, A, lda, Z, ldz, 0.0, W, m, nullptr, 1, s));
    OQR_TRY(launch_gemm_f64(GEMM_T, n, n, m, 1.0, Z, ldz, W, m, 0.0, G, n, sk, splits, s));
    OQR_TRY(launch_potrf(n, G, n, R1, n, nullptr, ctx->st, s));
    OQR_TRY(launch_trsm(m, n, Z, ldz, R1, n, Q, ldq, ctx->st, s));
    OQR_TRY(launch_trsm(m, n, W, m, R1, n, W, m, ctx->st, s));
    // pass 2: G_2 = Q_1^T (W R_1^{-1}), R_2 = chol(G_2), Q = Q_1 / R_2, R = R_2 R_1
    OQR_TRY(launch_gemm_f64(GEMM_T, n, n, m, 1.0, Q, ldq, W, m, 0.0, G, n, sk, splits, s));
    OQR_TRY(launch_potrf(n, G, n, R2, n, nullptr, ctx->st, s));
    OQR_TRY(launch_trsm(m, n, Q, ldq, R2, n, Q, ldq, ctx->st, s));
    OQR_TRY(launch_rprod(n, R2, n, R1, n, R, ldr, s));
    if (o.check && (v = run_check(ctx, gp, A, lda, Q, ldq, partials, G, work, nullptr, 0, limit, s)) != OQR_OK)
        return v;
    return finish(ctx, s, info, 2, o.check != 0);
}

// PRE-CHOLQR (Algorithm 2, Sec. 3): [Y, S] = qr(Z) by Householder TSQR,
// [Q, U] = CHOLQR(A, Y) (one pass in opts->final_prec), R = U S.
// The Euclidean Householder QR Z = Y S (Y orthonormal, S with a positive diagonal): the TSQR for one
// panel's width or less, the blocked form (TSQR panels, trailing updates by FP64 GEMMs) above it.
size_t euclid_qr_bytes(int m, int n, int sms)
{
    return align256((n <= BH_B ? tsqr_plan(m, n).doubles : bhqr_plan(m, n, sms).doubles) * sizeof(double));
}
cudaError_t launch_euclid_qr(int m, int n, const double* Z, long ldz, double* Y, long ldy, double* S, long lds,
                             double* ws, int sms, DevStatus* st, uint64_t limit_ns, cudaStream_t s)
{
    if (n <= BH_B) return launch_tsqr(tsqr_plan(m, n), Z, ldz, Y, ldy, S, lds, ws, s);
    return launch_bhqr(bhqr_plan(m, n, sms), Z, ldz, Y, ldy, S, lds, ws, st, limit_ns, s);
}

oqr_status precholqr_impl(oqr_ctx* ctx, int m, int n, const AOp& op, const double* Z, long ldz, double* Q, long ldq,
                          double* R, long ldr, const oqr_opts* opts, oqr_info* info, cudaStream_t s)
{
    if (!ctx || m < 1 || n < 1 || n > m || bad_matrix(Z, ldz, m, n) || bad_matrix(Q, ldq, m, n) ||
        bad_matrix(R, ldr, n, n) || (!op.tri() && bad_matrix(op.A, op.lda, m, m)) || (op.tri() && m > 1 && !op.e))
        return OQR_ERR_INVALID_ARG;
    if (n > 1024) return OQR_ERR_UNSUPPORTED;
    if (Q != Z) {
        const char *q0 = reinterpret_cast<const char*>(Q), *q1 = reinterpret_cast<const char*>(Q + (size_t)ldq * (n - 1) + m);
        const char *z0 = reinterpret_cast<const char*>(Z), *z1 = reinterpret_cast<const char*>(Z + (size_t)ldz * (n - 1) + m);
        if (q0 < z1 && z0 < q1) return OQR_ERR_INVALID_ARG;
    }
    const oqr_opts o = resolve(opts);
    NePlan P;
    oqr_status v = ne_plan(o, 1, m, n, &P, op.tri());
    if (v != OQR_OK) return v;
    const GramPlan gp = gram_plan(m, n, ctx->sm_count);
    NeBuffers B;
    const size_t reserve = align256((size_t)2 * n * n * sizeof(double));  // S, U
    const size_t need = reserve + std::max(euclid_qr_bytes(m, n, ctx->sm_count), ne_carve(nullptr, gp, P, &B));
    if ((v = ensure_ws(ctx, need)) != OQR_OK) return v;
    double* S = static_cast<double*>(ctx->ws);
    double* Uf = S + (size_t)n * n;
    double* tws = reinterpret_cast<double*>(static_cast<char*>(ctx->ws) + reserve);
    {
        const NvtxRange range("oqr: Householder QR %d", n);
        if ((v = reset_status(ctx, s)) != OQR_OK) return v;
        OQR_TRY(launch_euclid_qr(m, n, Z, ldz, Q, ldq, S, n, tws, ctx->sm_count, ctx->st, (uint64_t)o.spin_limit,
                                 s));  // Y into Q
        if (n > BH_B) {  // the blocked QR's waits report through the status, which the pass below resets
            DevStatus h;
            if (cudaMemcpyAsync(&h, ctx->st, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                return OQR_ERR_CUDA;
            if (h.code != 0) return static_cast<oqr_status>(h.code);
        }
    }
    // CHOLQR on Y in place (Q aliases Y), its factor into U; no synchronization yet
    if ((v = normal_equation(ctx, m, n, op, Q, ldq, Q, ldq, Uf, n, &o, nullptr, s, 1, false, reserve)) != OQR_OK)
        return v;
    OQR_TRY(launch_rprod(n, Uf, n, S, n, R, ldr, s));
    return finish(ctx, s, info, 1, o.check != 0);
}

oqr_status cgs2_impl(oqr_ctx* ctx, int m, int n, const double* A, long lda, const double* Z, long ldz, double* Q,
                     long ldq, double* R, long ldr, const oqr_opts* opts_in, oqr_info* info, void* stream)
{
    oqr_status v = check_common(ctx, m, n, A, lda, Z, ldz, Q, ldq, R, ldr);
    if (v != OQR_OK) return v;
    const oqr_opts o = resolve(opts_in);
    if (o.prec != OQR_FP64) return OQR_ERR_UNSUPPORTED;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint64_t limit = (uint64_t)o.spin_limit;
    const GramPlan gp = gram_plan(m, n, ctx->sm_count);
    CgsLayout L;
    L.b = std::min(o.block, n);
    L.gp = gram_plan(m, L.b, ctx->sm_count);
    L.splits = CGS_MAX_SPLITS;
    double *partials, *G, *work, *R1, *R2, *R3, *scratch;
    Carve probe(nullptr);
    layout_cholqr(probe, gp, &partials, &G, &work, &R1, &R2, &R3, &scratch);
    layout_cgs2(probe, L, m, n);
    if ((v = ensure_ws(ctx, probe.off)) != OQR_OK) return v;
    Carve c(ctx->ws);
    layout_cholqr(c, gp, &partials, &G, &work, &R1, &R2, &R3, &scratch);
    layout_cgs2(c, L, m, n);
    if ((v = reset_status(ctx, s)) != OQR_OK) return v;
    OQR_TRY(cudaMemset2DAsync(R, ldr * sizeof(double), 0, n * sizeof(double), n, s));
    if (Q != Z)
        OQR_TRY(cudaMemcpy2DAsync(Q, ldq * sizeof(double), Z, ldz * sizeof(double), m * sizeof(double), n,
                                  cudaMemcpyDeviceToDevice, s));
    const int b = L.b;
    auto splits_for = [&](int M, int N) {
        const int tiles = ((M + 63) / 64) * ((N + 63) / 64);
        return std::max(1, std::min(CGS_MAX_SPLITS, 2 * ctx->sm_count / tiles));
    };
    for (int j0 = 0; j0 < n; j0 += b) {
        const int bj = std::min(b, n - j0);
        double* Zj = Q + (size_t)j0 * ldq;
        for (int sweep = 0; sweep < 2 && j0 > 0; ++sweep) {
            const int sp = splits_for(j0, bj);
            // r = (A Q)^T Z_j ; Z_j -= Q r ; R(:j0, block) += r
            OQR_TRY(launch_gemm_f64(GEMM_T, j0, bj, m, 1.0, L.AQ, m, Zj, ldq, 0.0, L.r, n, L.sk, sp, s));
            OQR_TRY(launch_gemm_f64(GEMM_N, m, bj, j0, -1.0, Q, ldq, L.r, n, 1.0, Zj, ldq, nullptr, 1, s));
            OQR_TRY(launch_axpby(j0, bj, 1.0, L.r, n, 1.0, R + (size_t)j0 * ldr, ldr, s));
        }
        // S = A Z_j of the projected block, formed afresh (symmetric A from its lower triangle): updating an
        // earlier A Z_j by the projections would cancel, with an error growing like kappa(Z), when the
        // projected block is much smaller than the original one
        OQR_TRY(launch_gemm_f64(GEMM_SYML, m, bj, m, 1.0, A, lda, Zj, ldq, 0.0, L.S, m, nullptr, 1, s));
        // A-CholQR2 of the block against S = A Z_j
        const int sp = splits_for(bj, bj);
        for (int pass = 0; pass < 2; ++pass) {
            double* Rp = pass == 0 ? L.R1 : L.R2;
            OQR_TRY(launch_gemm_f64(GEMM_T, bj, bj, m, 1.0, Zj, ldq, L.S, m, 0.0, L.Gb, b, L.sk, sp, s));
            OQR_TRY(launch_potrf(bj, L.Gb, b, Rp, b, nullptr, ctx->st, s));
            OQR_TRY(launch_trsm(m, bj, Zj, ldq, Rp, b, Zj, ldq, ctx->st, s));
            OQR_TRY(launch_trsm(m, bj, L.S, m, Rp, b, L.S, m, ctx->st, s));
        }
        OQR_TRY(launch_rprod(bj, L.R2, b, L.R1, b, R + (size_t)j0 + (size_t)j0 * ldr, ldr, s));
        OQR_TRY(cudaMemcpy2DAsync(L.AQ + (size_t)j0 * m, m * sizeof(double), L.S, m * sizeof(double),
                                  m * sizeof(double), bj, cudaMemcpyDeviceToDevice, s));
    }
    if (o.check) {
        if ((v = run_check(ctx, gp, A, lda, Q, ldq, partials, G, work, nullptr, 0, limit, s)) != OQR_OK) return v;
    }
    return finish(ctx, s, info, 2, o.check != 0);
}

}  // namespace

namespace {
// Slice planes of one wave of the batched tensor-core path (the packed A, Z and U planes).
constexpr size_t BATCH_WAVE_BYTES = size_t(16) << 30;

// Captures seq into the context's cached graph for key (or replays the cached
// one), then launches it on s; on the legacy default stream seq runs directly.
template <class F>
oqr_status run_cached_graph(oqr_ctx* ctx, const std::vector<long>& key, F seq, cudaStream_t s)
{
    if (s == nullptr) {
        OQR_TRY(seq());
        return OQR_OK;
    }
    if (!ctx->mixed_exec || key != ctx->mixed_key) {
        if (ctx->mixed_exec) {
            cudaStreamSynchronize(s);
            cudaGraphExecDestroy(ctx->mixed_exec);
            ctx->mixed_exec = nullptr;
            ctx->mixed_key.clear();
        }
        cudaGraph_t g = nullptr;
        OQR_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        const cudaError_t le = seq();
        const cudaError_t ce = cudaStreamEndCapture(s, &g);
        if (le != cudaSuccess || ce != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return OQR_ERR_CUDA;
        }
        const cudaError_t ie = cudaGraphInstantiate(&ctx->mixed_exec, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) {
            ctx->mixed_exec = nullptr;
            return OQR_ERR_CUDA;
        }
        ctx->mixed_key = key;
    }
    OQR_TRY(cudaGraphLaunch(ctx->mixed_exec, s));
    return OQR_OK;
}
}  // namespace

namespace {
// FP64 A-CholQR2 over a batch (oqr_batched mode 0).
oqr_status batched_fp64_impl(oqr_ctx* ctx, int count, const int* m, const int* n, const double* const* A,
                             const long* lda, const double* const* Z, const long* ldz, double* const* Q,
                             const long* ldq, double* const* R, const long* ldr, const int* splits, int* status,
                             cudaStream_t stream)
{
    std::vector<BatchDesc> desc((size_t)count);
    std::vector<int> idx[3];
    int cls_max_splits[3] = {1, 1, 1}, max_n = 1;
    size_t per_inst_doubles = 0;
    for (int b = 0; b < count; ++b) {
        const int mb = m[b], nb = n[b];
        if (mb < 1 || nb < 1 || nb > mb || nb > BATCH_MAX_N || mb > BATCH_MAX_M) return OQR_ERR_INVALID_ARG;
        if (bad_matrix(A[b], lda[b], mb, mb) || bad_matrix(Z[b], ldz[b], mb, nb) || bad_matrix(Q[b], ldq[b], mb, nb) ||
            bad_matrix(R[b], ldr[b], nb, nb))
            return OQR_ERR_INVALID_ARG;
        const int sp = splits ? splits[b] : oqr_batched_default_splits(mb, nb);
        if (sp < 1 || sp > 64) return OQR_ERR_INVALID_ARG;
        BatchDesc& d = desc[b];
        d.A = A[b];
        d.Z = Z[b];
        d.Q = Q[b];
        d.R = R[b];
        d.lda = lda[b];
        d.ldz = ldz[b];
        d.ldq = ldq[b];
        d.ldr = ldr[b];
        d.m = mb;
        d.n = nb;
        d.splits = sp;
        d.npass = 2;
        const int c = nb <= 16 ? 0 : nb <= 32 ? 1 : 2;
        idx[c].push_back(b);
        cls_max_splits[c] = std::max(cls_max_splits[c], sp);
        max_n = std::max(max_n, nb);
        per_inst_doubles += align256((size_t)(sp + 3) * nb * nb * sizeof(double)) / sizeof(double);
    }
    // workspace: descriptors, three index lists, per-instance partials + G + R1 + R2
    Carve probe(nullptr);
    probe.take<BatchDesc>((size_t)count);
    for (int c = 0; c < 3; ++c) probe.take<int>(std::max<size_t>(1, idx[c].size()));
    probe.take<double>(per_inst_doubles);
    oqr_status v = ensure_ws(ctx, probe.off);
    if (v != OQR_OK) return v;
    Carve cv(ctx->ws);
    BatchDesc* ddesc = cv.take<BatchDesc>((size_t)count);
    int* didx[3];
    for (int c = 0; c < 3; ++c) didx[c] = cv.take<int>(std::max<size_t>(1, idx[c].size()));
    double* pool = cv.take<double>(per_inst_doubles);
    for (int b = 0; b < count; ++b) {
        const size_t nn = (size_t)desc[b].n * desc[b].n;
        desc[b].partials = pool;
        desc[b].G = pool + desc[b].splits * nn;
        desc[b].R1 = desc[b].G + nn;
        desc[b].R2 = desc[b].R1 + nn;
        pool += align256((size_t)(desc[b].splits + 3) * nn * sizeof(double)) / sizeof(double);
    }
    cudaStream_t s = stream;
    OQR_TRY(cudaMemcpyAsync(ddesc, desc.data(), sizeof(BatchDesc) * count, cudaMemcpyHostToDevice, s));
    int cls_count[3];
    for (int c = 0; c < 3; ++c) {
        cls_count[c] = (int)idx[c].size();
        if (cls_count[c]) OQR_TRY(cudaMemcpyAsync(didx[c], idx[c].data(), sizeof(int) * cls_count[c],
                                                  cudaMemcpyHostToDevice, s));
    }
    OQR_TRY(cudaMemsetAsync(status, 0, sizeof(int) * count, s));
    if (s == nullptr) {  // the legacy default stream cannot be captured
        OQR_TRY(launch_batched_cholqr2(ddesc, count, didx, cls_count, cls_max_splits, max_n, status, s));
        return OQR_OK;
    }
    const long key[10] = {count, cls_count[0], cls_count[1], cls_count[2], cls_max_splits[0], cls_max_splits[1],
                          cls_max_splits[2], max_n, (long)reinterpret_cast<uintptr_t>(ctx->ws),
                          (long)reinterpret_cast<uintptr_t>(status)};
    if (!ctx->batch_exec || memcmp(key, ctx->batch_key, sizeof(key)) != 0) {
        if (ctx->batch_exec) {
            cudaStreamSynchronize(s);
            cudaGraphExecDestroy(ctx->batch_exec);
            ctx->batch_exec = nullptr;
        }
        cudaGraph_t g = nullptr;
        OQR_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        const cudaError_t le = launch_batched_cholqr2(ddesc, count, didx, cls_count, cls_max_splits, max_n, status, s);
        const cudaError_t ce = cudaStreamEndCapture(s, &g);
        if (le != cudaSuccess || ce != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return OQR_ERR_CUDA;
        }
        const cudaError_t ie = cudaGraphInstantiate(&ctx->batch_exec, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) {
            ctx->batch_exec = nullptr;
            return OQR_ERR_CUDA;
        }
        memcpy(ctx->batch_key, key, sizeof(key));
    }
    OQR_TRY(cudaGraphLaunch(ctx->batch_exec, s));
    return OQR_OK;
}

}  // namespace

// ---- the learned selector over a batch -------------------------------------
// (oqr_batched in OQR_BATCHED_SELECTOR mode, and oqr_batched_features.)
// Every option of the selector starts with the same first pass, an
// FP64-accurate Gram G0 = Z^T A Z on the tensor cores, so that pass runs
// first for the whole wave (the probe); its Gram and Cholesky factor give the
// features and the network picks a route per instance.  The rest of the wave
// is a fixed sequence of launches whose decisions are taken on the device
// (k_select.cu): each instance takes part in the Gram passes of its route, the
// tensor-core launches skipping the tiles of the others, so the host neither
// waits for the choices nor plans per choice.  Instances that end with a
// failed check, a breakdown or the network's FP64 choice are redone by FP64
// A-CholQR2 after the waves.
namespace {

struct SelInputs {
    int count;
    const int *m, *n;
    const double* const* A;
    const long* lda;
    const double* const* Z;
    const long* ldz;
    double* const* Q;  // nullptr: features only
    const long* ldq;
    double* const* R;
    const long* ldr;
};

// Host-side outcome per instance (caller order).
struct SelResult {
    std::vector<int> status, choice;
    std::vector<double> orth;  // NaN where not checked
};

// Instances sorted by m (largest first), their descriptors and tensor-core inputs, over a pool of
// per-instance n x n buffers (partials, G, R1, R2, G0).
struct SelSetup {
    std::vector<int> perm;
    std::vector<TcBatchShape> sh;
    std::vector<BatchDesc> desc;
    std::vector<TcBatchIn> in;
    size_t pool_doubles = 0;
};
constexpr int SEL_NN_BUFS = 5;

SelSetup sel_setup(const SelInputs& I, int npass)
{
    SelSetup S;
    const int count = I.count;
    S.perm.resize((size_t)count);
    for (int b = 0; b < count; ++b) S.perm[b] = b;
    std::stable_sort(S.perm.begin(), S.perm.end(), [&](int x, int y) { return I.m[x] > I.m[y]; });
    S.sh.resize((size_t)count);
    for (int i = 0; i < count; ++i) {
        const int b = S.perm[i];
        S.sh[i] = TcBatchShape{I.m[b], I.n[b], 1, npass};
        S.pool_doubles += align256((size_t)SEL_NN_BUFS * I.n[b] * I.n[b] * sizeof(double)) / sizeof(double);
    }
    return S;
}

void sel_fill(const SelInputs& I, SelSetup& S, double* pool)
{
    const bool features_only = I.Q == nullptr;
    const int count = I.count;
    S.desc.assign((size_t)count, BatchDesc{});
    S.in.resize((size_t)count);
    double* q = pool;
    for (int i = 0; i < count; ++i) {
        const int b = S.perm[i];
        const size_t nn = (size_t)I.n[b] * I.n[b];
        BatchDesc& d = S.desc[i];
        d.A = I.A[b];
        d.Z = I.Z[b];
        d.Q = features_only ? nullptr : I.Q[b];
        d.R = features_only ? nullptr : I.R[b];
        d.lda = I.lda[b];
        d.ldz = I.ldz[b];
        d.ldq = features_only ? I.m[b] : I.ldq[b];
        d.ldr = features_only ? I.n[b] : I.ldr[b];
        d.m = I.m[b];
        d.n = I.n[b];
        d.splits = 1;
        d.npass = 2;
        d.partials = q;
        d.G = q + nn;
        d.R1 = d.G + nn;
        d.R2 = d.R1 + nn;
        d.G0 = d.R2 + nn;
        q += align256(SEL_NN_BUFS * nn * sizeof(double)) / sizeof(double);
        S.in[i] = TcBatchIn{I.A[b], I.lda[b], I.Z[b], I.ldz[b], features_only ? const_cast<double*>(I.Z[b]) : I.Q[b],
                            features_only ? I.ldz[b] : I.ldq[b], d.partials};
    }
}

// Pinned host memory of the context, grown to bytes (the previous call's copies are complete: every
// selector call ends with a synchronization).
oqr_status sel_pinned(oqr_ctx* ctx, size_t bytes, cudaStream_t s)
{
    if (ctx->pin_bytes >= bytes) return OQR_OK;
    if (ctx->pin) {
        cudaStreamSynchronize(s);
        cudaFreeHost(ctx->pin);
        ctx->pin = nullptr;
        ctx->pin_bytes = 0;
    }
    if (cudaHostAlloc(&ctx->pin, bytes, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        return OQR_ERR_NO_MEMORY;
    }
    ctx->pin_bytes = bytes;
    return OQR_OK;
}

// The features of every instance after its first FP64-accurate pass (oqr_batched_features).
oqr_status features_waves(oqr_ctx* ctx, const SelInputs& I, float* feat_out, cudaStream_t s)
{
    const int count = I.count;
    SelSetup S = sel_setup(I, 1);
    const size_t budget = ctx->batch_budget ? ctx->batch_budget : BATCH_WAVE_BYTES;
    const TcBatchPlan plan = tc_batch_plan(S.sh, budget);
    double* wtab = nullptr;
    auto layout = [&](Carve& c, char** tab, BatchDesc** d, int** sts, float** feat, int** perm, double** pool,
                      double** upool, void** scr) {
        wtab = c.take<double>((size_t)SKETCH_TABLE_DOUBLES);
        *tab = c.take<char>(plan.table_bytes);
        *d = c.take<BatchDesc>((size_t)count);
        *sts = c.take<int>((size_t)count);
        *feat = c.take<float>((size_t)count * MLP_IN);
        *perm = c.take<int>((size_t)count);
        *pool = c.take<double>(S.pool_doubles);
        *upool = c.take<double>(plan.upool_doubles);
        *scr = c.take<char>(plan.scratch_bytes);
    };
    char* tab;
    BatchDesc* ddesc;
    int *sts, *dperm;
    float* feat;
    double *pool, *upool;
    void* scratch;
    Carve probe(nullptr);
    layout(probe, &tab, &ddesc, &sts, &feat, &dperm, &pool, &upool, &scratch);
    oqr_status v = ensure_ws(ctx, probe.off);
    if (v != OQR_OK) return v;
    Carve cv(ctx->ws);
    layout(cv, &tab, &ddesc, &sts, &feat, &dperm, &pool, &upool, &scratch);
    sel_fill(I, S, pool);
    std::vector<char> image;
    tc_batch_tables(plan, S.sh, S.in, tab, upool, image);
    OQR_TRY(cudaMemcpyAsync(tab, image.data(), image.size(), cudaMemcpyHostToDevice, s));
    OQR_TRY(cudaMemcpyAsync(ddesc, S.desc.data(), sizeof(BatchDesc) * count, cudaMemcpyHostToDevice, s));
    OQR_TRY(cudaMemcpyAsync(dperm, S.perm.data(), sizeof(int) * count, cudaMemcpyHostToDevice, s));
    OQR_TRY(cudaMemsetAsync(sts, 0, sizeof(int) * count, s));
    if ((v = reset_status(ctx, s)) != OQR_OK) return v;
    OQR_TRY(launch_sketch_table(wtab, s));
    const uint64_t limit = 4000000000ull;
    for (int w = 0; w < (int)plan.waves.size(); ++w) {
        const NvtxRange range("oqr: features wave %d", w);
        const TcBatchWave& W = plan.waves[w];
        BatchDesc* dw = ddesc + W.first;
        int* sw = sts + W.first;
        OQR_TRY(tc_batch_split_a(plan, w, tab, scratch, s));
        OQR_TRY(tc_batch_gram(plan, w, 0, tab, scratch, ctx->st, limit, ctx->sm_count, s));
        OQR_TRY(launch_batched_gram_chol(dw, W.count, sw, s));
        OQR_TRY(launch_features_batched(dw, W.count, sw, wtab, feat + (size_t)W.first * MLP_IN, s));
    }
    OQR_TRY(launch_batch_scatter_rows_f32(feat, dperm, count, MLP_IN, feat_out, s));
    // the pageable uploads above have left their host vectors once the stream is done
    if (cudaStreamSynchronize(s) != cudaSuccess) return OQR_ERR_CUDA;
    DevStatus hs;
    if (cudaMemcpy(&hs, ctx->st, sizeof(hs), cudaMemcpyDeviceToHost) != cudaSuccess) return OQR_ERR_CUDA;
    return hs.code != 0 ? OQR_ERR_TIMEOUT : OQR_OK;
}

// The selector over a batch: the probe, the network and every route's passes, wave by wave, with no
// host round trip until the end.
oqr_status selector_run(oqr_ctx* ctx, const SelInputs& I, const float* params, double tol, bool check_all,
                        SelResult* res, cudaStream_t s)
{
    const int count = I.count;
    const int extra = check_all ? 1 : 0;
    SelSetup S = sel_setup(I, TC_BATCH_MAX_PASS);
    const size_t budget = ctx->batch_budget ? ctx->batch_budget : BATCH_WAVE_BYTES;
    const TcBatchPlan plan = tc_batch_plan(S.sh, budget);
    struct Dev {
        char* tab;
        BatchDesc* d;
        int *sts, *route, *opt, *gpass, *mask, *choice;
        double *anorm2, *znorm2, *shifts, *orth, *defect, *pool, *upool, *wtab;
        float* feat;
        void* scratch;
    } D{};
    auto layout = [&](Carve& c, Dev& x) {
        x.wtab = c.take<double>((size_t)SKETCH_TABLE_DOUBLES);
        x.tab = c.take<char>(plan.table_bytes);
        x.d = c.take<BatchDesc>((size_t)count);
        x.sts = c.take<int>((size_t)count);
        x.route = c.take<int>((size_t)count);
        x.opt = c.take<int>((size_t)count);
        x.gpass = c.take<int>((size_t)count);
        x.mask = c.take<int>((size_t)count);
        x.choice = c.take<int>((size_t)count);
        x.anorm2 = c.take<double>((size_t)count);
        x.znorm2 = c.take<double>((size_t)count);
        x.shifts = c.take<double>((size_t)count);
        x.orth = c.take<double>((size_t)count);
        x.defect = c.take<double>((size_t)count);
        x.feat = c.take<float>((size_t)count * MLP_IN);
        x.pool = c.take<double>(S.pool_doubles);
        x.upool = c.take<double>(plan.upool_doubles);
        x.scratch = c.take<char>(plan.scratch_bytes);
    };
    Carve probe(nullptr);
    layout(probe, D);
    oqr_status v = ensure_ws(ctx, probe.off);
    if (v != OQR_OK) return v;
    Carve cv(ctx->ws);
    layout(cv, D);
    sel_fill(I, S, D.pool);
    // pinned: the table image and the descriptors going up, the statuses, options and checks coming back
    struct Pin {
        char* img;
        BatchDesc* desc;
        int *sts, *opt;
        double* orth;
        DevStatus* st;
    } P{};
    auto pin_layout = [&](Carve& c, Pin& x) {
        x.img = c.take<char>(plan.table_bytes);
        x.desc = c.take<BatchDesc>((size_t)count);
        x.sts = c.take<int>((size_t)count);
        x.opt = c.take<int>((size_t)count);
        x.orth = c.take<double>((size_t)count);
        x.st = c.take<DevStatus>(1);
    };
    Carve pprobe(nullptr);
    pin_layout(pprobe, P);
    if ((v = sel_pinned(ctx, pprobe.off, s)) != OQR_OK) return v;
    Carve pc(ctx->pin);
    pin_layout(pc, P);
    std::vector<char> image;
    tc_batch_tables(plan, S.sh, S.in, D.tab, D.upool, image);
    memcpy(P.img, image.data(), image.size());
    memcpy(P.desc, S.desc.data(), sizeof(BatchDesc) * count);
    OQR_TRY(cudaMemcpyAsync(D.tab, P.img, image.size(), cudaMemcpyHostToDevice, s));
    OQR_TRY(cudaMemcpyAsync(D.d, P.desc, sizeof(BatchDesc) * count, cudaMemcpyHostToDevice, s));
    OQR_TRY(cudaMemsetAsync(D.sts, 0, sizeof(int) * count, s));
    if ((v = reset_status(ctx, s)) != OQR_OK) return v;
    OQR_TRY(launch_sketch_table(D.wtab, s));
    const uint64_t limit = 4000000000ull;
    for (int w = 0; w < (int)plan.waves.size(); ++w) {
        const NvtxRange range("oqr: selector wave %d", w);
        const TcBatchWave& W = plan.waves[w];
        const int f = W.first, cnt = W.count;
        BatchDesc* dw = D.d + f;
        int* sw = D.sts + f;
        const SelWave sel{dw,           sw,           D.route + f, D.opt + f, D.gpass + f, D.mask + f, D.anorm2 + f,
                          D.znorm2 + f, D.shifts + f, D.orth + f,  D.defect + f, cnt,     extra,       tol};
        const int* live = D.gpass + f;
        // the probe: the split of A (read by every pass of the wave), G0, its Cholesky factor, the
        // features, the network, the routes
        OQR_TRY(tc_batch_split_a(plan, w, D.tab, D.scratch, s));
        OQR_TRY(tc_batch_gram(plan, w, 0, D.tab, D.scratch, ctx->st, limit, ctx->sm_count, s));
        OQR_TRY(tc_batch_norms(plan, w, D.tab, D.scratch, sel.anorm2, sel.znorm2, s));
        OQR_TRY(launch_batched_gram_chol(dw, cnt, sw, s));
        OQR_TRY(launch_features_batched(dw, cnt, sw, D.wtab, D.feat + (size_t)f * MLP_IN, s));
        OQR_TRY(launch_mlp_forward(cnt, D.feat + (size_t)f * MLP_IN, params, 1, nullptr, D.choice + f, s));
        OQR_TRY(launch_sel_route(sel, D.choice + f, s));
        // the first factor: R1 = chol(G0 + s I) on the shifted route (elsewhere the probe's R1 stands),
        // then Q1 = Z R1^{-1}
        OQR_TRY(launch_batched_shifts(dw, cnt, sel.mask, sel.anorm2, sel.znorm2, 11.0, U64, sel.shifts, s));
        OQR_TRY(launch_sel_shift_g(sel, s));
        OQR_TRY(launch_batched_chol_solve(dw, cnt, sw, sel.mask, nullptr, s));
        OQR_TRY(launch_sel_after_factor(sel, 0, s));
        // passes 1..3 (4: the extra check of a late instance)
        for (int pass = 1; pass < 4 + extra; ++pass) {
            OQR_TRY(tc_batch_gram(plan, w, pass, D.tab, D.scratch, ctx->st, limit, ctx->sm_count, s, live));
            OQR_TRY(launch_sel_decide(sel, pass, s));
            OQR_TRY(launch_batched_factor(dw, cnt, sw, pass, nullptr, s));
            if (pass == 1) {  // the late refactor: R1 = chol(G0 + s I), Q1 = Z R1^{-1}
                OQR_TRY(launch_sel_late_mask(sel, s));
                OQR_TRY(launch_batched_shifts(dw, cnt, sel.mask, sel.anorm2, sel.znorm2, 11.0, U64, sel.shifts, s));
                OQR_TRY(launch_sel_late_prep(sel, s));
                OQR_TRY(launch_batched_chol_solve(dw, cnt, sw, sel.mask, sel.mask, s));
            }
            OQR_TRY(launch_sel_after_factor(sel, pass, s));
        }
        OQR_TRY(launch_batched_rfinal(dw, cnt, sw, s));
    }
    OQR_TRY(cudaMemcpyAsync(P.sts, D.sts, sizeof(int) * count, cudaMemcpyDeviceToHost, s));
    OQR_TRY(cudaMemcpyAsync(P.opt, D.opt, sizeof(int) * count, cudaMemcpyDeviceToHost, s));
    OQR_TRY(cudaMemcpyAsync(P.orth, D.orth, sizeof(double) * count, cudaMemcpyDeviceToHost, s));
    OQR_TRY(cudaMemcpyAsync(P.st, ctx->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    if (cudaStreamSynchronize(s) != cudaSuccess) return OQR_ERR_CUDA;
    const bool timed_out = P.st->code != 0;
    res->status.assign((size_t)count, 0);
    res->choice.assign((size_t)count, 0);
    res->orth.assign((size_t)count, std::nan(""));
    for (int i = 0; i < count; ++i) {
        const int b = S.perm[i];
        res->status[b] = timed_out ? -1 : P.sts[i];
        res->choice[b] = P.opt[i];
        res->orth[b] = P.orth[i];
    }
    return timed_out ? OQR_ERR_TIMEOUT : OQR_OK;
}

// FP64 A-CholQR2 over a sub-batch (the fallback and the network's FP64 choices): outputs into the
// caller's Q and R of those instances, statuses through the context's small selector buffer.
oqr_status selector_fp64(oqr_ctx* ctx, const SelInputs& I, const std::vector<int>& idx, SelResult* res,
                         cudaStream_t s)
{
    const int k = (int)idx.size();
    if (k == 0) return OQR_OK;
    std::vector<int> m(k), n(k);
    std::vector<const double*> A(k), Z(k);
    std::vector<double*> Q(k), R(k);
    std::vector<long> lda(k), ldz(k), ldq(k), ldr(k);
    for (int j = 0; j < k; ++j) {
        const int b = idx[j];
        m[j] = I.m[b];
        n[j] = I.n[b];
        A[j] = I.A[b];
        Z[j] = I.Z[b];
        Q[j] = I.Q[b];
        R[j] = I.R[b];
        lda[j] = I.lda[b];
        ldz[j] = I.ldz[b];
        ldq[j] = I.ldq[b];
        ldr[j] = I.ldr[b];
    }
    const size_t need = (size_t)k * sizeof(int) + 256;
    if (ctx->sel_bytes < need) {
        if (ctx->sel_buf) {
            cudaStreamSynchronize(s);
            cudaFree(ctx->sel_buf);
            ctx->sel_buf = nullptr;
            ctx->sel_bytes = 0;
        }
        if (cudaMalloc(&ctx->sel_buf, need) != cudaSuccess) {
            cudaGetLastError();
            return OQR_ERR_NO_MEMORY;
        }
        ctx->sel_bytes = need;
    }
    int* dst = static_cast<int*>(ctx->sel_buf);
    oqr_status v = batched_fp64_impl(ctx, k, m.data(), n.data(), A.data(), lda.data(), Z.data(), ldz.data(),
                                     Q.data(), ldq.data(), R.data(), ldr.data(), nullptr, dst, s);
    if (v != OQR_OK) return v;
    std::vector<int> hst(k);
    OQR_TRY(cudaMemcpyAsync(hst.data(), dst, sizeof(int) * k, cudaMemcpyDeviceToHost, s));
    if (cudaStreamSynchronize(s) != cudaSuccess) return OQR_ERR_CUDA;
    for (int j = 0; j < k; ++j) {
        const int b = idx[j];
        res->status[b] = hst[j];
        res->choice[b] = SEL_FP64;
        res->orth[b] = std::nan("");
    }
    return OQR_OK;
}

oqr_status selector_batch(oqr_ctx* ctx, const SelInputs& I, const oqr_opts& o, int* status, cudaStream_t s)
{
    if (!o.selector_params) return OQR_ERR_INVALID_ARG;
    const double tol = o.selector_tol > 0 ? o.selector_tol : 1e-12;
    SelResult res;
    oqr_status v = selector_run(ctx, I, o.selector_params, tol, o.selector_check != 0, &res, s);
    if (v != OQR_OK && v != OQR_ERR_TIMEOUT) return v;
    if (v == OQR_OK) {
        // FP64 A-CholQR2 for the network's FP64 choices, a breakdown, a failed last-pass check, or a
        // failed extra check
        std::vector<int> fb;
        for (int b = 0; b < I.count; ++b)
            if (res.choice[b] == SEL_FP64 || res.status[b] != 0 || (!std::isnan(res.orth[b]) && !(res.orth[b] <= tol)))
                fb.push_back(b);
        if ((v = selector_fp64(ctx, I, fb, &res, s)) != OQR_OK) return v;
    }
    OQR_TRY(cudaMemcpy(status, res.status.data(), sizeof(int) * I.count, cudaMemcpyHostToDevice));
    if (o.batch_orth)
        OQR_TRY(cudaMemcpy(o.batch_orth, res.orth.data(), sizeof(double) * I.count, cudaMemcpyHostToDevice));
    if (o.batch_choice)
        OQR_TRY(cudaMemcpy(o.batch_choice, res.choice.data(), sizeof(int) * I.count, cudaMemcpyHostToDevice));
    return v;
}
}  // namespace

extern "C" {

void oqr_default_opts(oqr_opts* opts)
{
    if (opts) fill_defaults(opts);
}

const char* oqr_status_string(oqr_status s)
{
    switch (s) {
        case OQR_OK: return "OQR_OK";
        case OQR_ERR_INVALID_ARG: return "OQR_ERR_INVALID_ARG: invalid argument";
        case OQR_ERR_NOT_SPD: return "OQR_ERR_NOT_SPD: Cholesky breakdown (matrix not numerically SPD)";
        case OQR_ERR_CHECK_FAILED: return "OQR_ERR_CHECK_FAILED: orthogonality check failed";
        case OQR_ERR_CUDA: return "OQR_ERR_CUDA: CUDA runtime error";
        case OQR_ERR_NO_MEMORY: return "OQR_ERR_NO_MEMORY: workspace unavailable";
        case OQR_ERR_TIMEOUT: return "OQR_ERR_TIMEOUT: device-side wait timed out";
        case OQR_ERR_UNSUPPORTED: return "OQR_ERR_UNSUPPORTED: size or option not supported by the library";
    }
    return "unknown oqr_status";
}

oqr_status oqr_create(oqr_ctx** out, int device)
{
    if (!out) return OQR_ERR_INVALID_ARG;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
        cudaGetLastError();
        return OQR_ERR_INVALID_ARG;
    }
    if (cudaSetDevice(device) != cudaSuccess) return OQR_ERR_CUDA;
    oqr_ctx* ctx = new (std::nothrow) oqr_ctx;
    if (!ctx) return OQR_ERR_NO_MEMORY;
    ctx->device = device;
    cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (cudaMalloc(&ctx->st, sizeof(DevStatus)) != cudaSuccess) {
        delete ctx;
        return OQR_ERR_NO_MEMORY;
    }
    cudaMemset(ctx->st, 0, sizeof(DevStatus));
    *out = ctx;
    return OQR_OK;
}

oqr_status oqr_destroy(oqr_ctx* ctx)
{
    if (!ctx) return OQR_OK;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    if (ctx->batch_exec) cudaGraphExecDestroy(ctx->batch_exec);
    if (ctx->mixed_exec) cudaGraphExecDestroy(ctx->mixed_exec);
    if (ctx->stage) cudaFree(ctx->stage);
    if (ctx->sel_buf) cudaFree(ctx->sel_buf);
    if (ctx->pin) cudaFreeHost(ctx->pin);
    for (cudaEvent_t e : ctx->sel_ev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : ctx->events) cudaEventDestroy(e);
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    if (ctx->ws && ctx->ws_owned) cudaFree(ctx->ws);
    if (ctx->st) cudaFree(ctx->st);
    delete ctx;
    return OQR_OK;
}

oqr_status oqr_workspace_size(oqr_ctx* ctx, int algo, int m, int n, const oqr_opts* opts, size_t* bytes)
{
    if (!ctx || !bytes || m < 1 || n < 1 || n > m) return OQR_ERR_INVALID_ARG;
    const oqr_opts o = resolve(opts);
    const GramPlan gp = gram_plan(m, n, ctx->sm_count);
    Carve c(nullptr);
    double *partials, *G, *work, *R1, *R2, *R3, *scratch;
    layout_cholqr(c, gp, &partials, &G, &work, &R1, &R2, &R3, &scratch);
    if (algo == OQR_ALGO_CGS2) {
        CgsLayout L;
        L.b = std::min(o.block, n);
        L.gp = gram_plan(m, L.b, ctx->sm_count);
        L.splits = CGS_MAX_SPLITS;
        layout_cgs2(c, L, m, n);
        *bytes = c.off;
        return OQR_OK;
    }
    if (algo < 0 || algo > OQR_ALGO_CGS2) return OQR_ERR_INVALID_ARG;
    // the normal-equation algorithms: the same plan as the call itself, tensor-core regions included
    oqr_opts oa = o;
    if (algo == OQR_ALGO_SCHOLQR3) oa.shifted = 1;
    NePlan P;
    oqr_status v = ne_plan(oa, algo == OQR_ALGO_CHOLQR ? 1 : 0, m, n, &P);
    if (v != OQR_OK) return v;
    NeBuffers B;
    *bytes = ne_carve(nullptr, gp, P, &B);
    return OQR_OK;
}

oqr_status oqr_set_workspace(oqr_ctx* ctx, void* ptr, size_t bytes)
{
    if (!ctx) return OQR_ERR_INVALID_ARG;
    if (ptr && (reinterpret_cast<uintptr_t>(ptr) % 256 != 0)) return OQR_ERR_INVALID_ARG;
    if (ctx->ws && ctx->ws_owned) {
        cudaDeviceSynchronize();
        cudaFree(ctx->ws);
    }
    ctx->ws = ptr;
    ctx->ws_bytes = ptr ? bytes : 0;
    ctx->ws_owned = ptr == nullptr;
    return OQR_OK;
}

oqr_status oqr_get_status(oqr_ctx* ctx, void* stream, int* info)
{
    if (!ctx) return OQR_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return OQR_ERR_CUDA;
    DevStatus h;
    if (cudaMemcpy(&h, ctx->st, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return OQR_ERR_CUDA;
    if (info) *info = h.info;
    return static_cast<oqr_status>(h.code);
}

oqr_status oqr_cholqr(oqr_ctx* ctx, int m, int n, const double* A, long lda, const double* Z, long ldz, double* Q,
                      long ldq, double* R, long ldr, const oqr_opts* opts, oqr_info* info, void* stream)
{
    return normal_equation(ctx, m, n, dense_op(A, lda), Z, ldz, Q, ldq, R, ldr, opts, info, stream, 1);
}

oqr_status oqr_cholqr2(oqr_ctx* ctx, int m, int n, const double* A, long lda, const double* Z, long ldz,
                       double* Q, long ldq, double* R, long ldr, const oqr_opts* opts, oqr_info* info, void* stream)
{
    if (opts && opts->reuse_w)
        return cholqr2_reuse_w(ctx, m, n, A, lda, Z, ldz, Q, ldq, R, ldr, resolve(opts), info,
                               static_cast<cudaStream_t>(stream));
    return normal_equation(ctx, m, n, dense_op(A, lda), Z, ldz, Q, ldq, R, ldr, opts, info, stream, 0);
}

oqr_status oqr_cholqr2_host(oqr_ctx* ctx, int m, int n, const double* A, long lda, const double* Z, long ldz,
                            double* Q, long ldq, double* R, long ldr, const oqr_opts* opts, oqr_info* info,
                            void* stream)
{
    if (!ctx || m < 1 || n < 1 || n > m || !A || !Z || !Q || !R || lda < m || ldz < m || ldq < m || ldr < n)
        return OQR_ERR_INVALID_ARG;
    const oqr_opts o = resolve(opts);
    NePlan P;
    oqr_status v = ne_plan(o, 0, m, n, &P);
    if (v != OQR_OK) return v;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaSetDevice(ctx->device) != cudaSuccess) return OQR_ERR_CUDA;
    // device staging: A (lower triangle only is copied; leading dimension even for 16-byte columns), Z, Q, R
    const long ldA = (m + 1) & ~1L;
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t bA = al((size_t)ldA * m * 8), bZ = al((size_t)m * n * 8), bR = al((size_t)n * n * 8);
    const size_t need = bA + 2 * bZ + bR;
    if (ctx->stage_bytes < need) {
        if (ctx->stage) {
            cudaStreamSynchronize(s);
            cudaFree(ctx->stage);
            ctx->stage = nullptr;
            ctx->stage_bytes = 0;
        }
        if (cudaMalloc(&ctx->stage, need) != cudaSuccess) {
            cudaGetLastError();
            return OQR_ERR_NO_MEMORY;
        }
        ctx->stage_bytes = need;
    }
    char* sb = static_cast<char*>(ctx->stage);
    double* Ad = reinterpret_cast<double*>(sb);
    double* Zd = reinterpret_cast<double*>(sb + bA);
    double* Qd = reinterpret_cast<double*>(sb + bA + bZ);
    double* Rd = reinterpret_cast<double*>(sb + bA + 2 * bZ);
    // the factorization's workspace, planned exactly as the call below plans it
    const GramPlan gp = gram_plan(m, n, ctx->sm_count);
    NeBuffers B;
    if ((v = ensure_ws(ctx, ne_carve(nullptr, gp, P, &B))) != OQR_OK) return v;
    ne_carve(ctx->ws, gp, P, &B);
    const int panels = (m + KCH_PANEL - 1) / KCH_PANEL;
    if (!ctx->copy_stream && cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
        return OQR_ERR_CUDA;
    while ((int)ctx->events.size() < panels + 2) {
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return OQR_ERR_CUDA;
        ctx->events.push_back(e);
    }
    cudaStream_t cs = ctx->copy_stream;
    cudaEvent_t ev_start = ctx->events[panels], ev_z = ctx->events[panels + 1];
    // the copies start after the work already queued on `stream` (which may still use the staging)
    OQR_TRY(cudaEventRecord(ev_start, s));
    OQR_TRY(cudaStreamWaitEvent(cs, ev_start, 0));
    OQR_TRY(cudaMemcpy2DAsync(Zd, (size_t)m * 8, Z, (size_t)ldz * 8, (size_t)m * 8, n, cudaMemcpyHostToDevice, cs));
    OQR_TRY(cudaEventRecord(ev_z, cs));
    // A's lower triangle in panels of KCH_PANEL columns (rows j0..m-1 of each), each split on `stream`
    // as soon as it has arrived when the first pass takes the EMU64-family split
    const bool split_early = emu_family(P.prec_first);
    const TcPlan tp = tc_plan(m, n, tc_mode_of(P.prec_first), emu_family(P.prec_first) ? P.sa : 0);
    if (split_early) OQR_TRY(tc_split_a_begin(tp, B.tcws, s));
    for (int k = 0; k < panels; ++k) {
        const long j0 = (long)k * KCH_PANEL;
        const long w = std::min<long>(KCH_PANEL, m - j0);
        OQR_TRY(cudaMemcpy2DAsync(Ad + j0 + j0 * ldA, (size_t)ldA * 8, A + j0 + j0 * lda, (size_t)lda * 8,
                                  (size_t)(m - j0) * 8, (size_t)w, cudaMemcpyHostToDevice, cs));
        OQR_TRY(cudaEventRecord(ctx->events[k], cs));
        if (split_early) {
            OQR_TRY(cudaStreamWaitEvent(s, ctx->events[k], 0));
            OQR_TRY(tc_split_a_chunk(tp, Ad, ldA, k, B.tcws, s));
        }
    }
    if (!split_early) OQR_TRY(cudaStreamWaitEvent(s, ctx->events[panels - 1], 0));
    OQR_TRY(cudaStreamWaitEvent(s, ev_z, 0));
    if ((v = normal_equation(ctx, m, n, dense_op(Ad, ldA), Zd, m, Qd, m, Rd, n, &o, nullptr, stream, 0,
                             split_early)) != OQR_OK)
        return v;
    OQR_TRY(cudaMemcpy2DAsync(Q, (size_t)ldq * 8, Qd, (size_t)m * 8, (size_t)m * 8, n, cudaMemcpyDeviceToHost, s));
    OQR_TRY(cudaMemcpy2DAsync(R, (size_t)ldr * 8, Rd, (size_t)n * 8, (size_t)n * 8, n, cudaMemcpyDeviceToHost, s));
    return finish(ctx, s, info, P.passes, o.check != 0);
}

oqr_status oqr_cgs2(oqr_ctx* ctx, int m, int n, const double* A, long lda, const double* Z, long ldz, double* Q,
                    long ldq, double* R, long ldr, const oqr_opts* opts, oqr_info* info, void* stream)
{
    return cgs2_impl(ctx, m, n, A, lda, Z, ldz, Q, ldq, R, ldr, opts, info, stream);
}

oqr_status oqr_gram(oqr_ctx* ctx, int m, int n, const double* A, long lda, const double* Z, long ldz, double* G,
                    long ldg, int prec, void* stream)
{
    if (!ctx || m < 1 || n < 1 || n > m || bad_matrix(A, lda, m, m) || bad_matrix(Z, ldz, m, n) ||
        bad_matrix(G, ldg, n, n))
        return OQR_ERR_INVALID_ARG;
    if (!prec_ok(prec)) return OQR_ERR_INVALID_ARG;
    if (n > 1024) return OQR_ERR_UNSUPPORTED;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const GramPlan gp = gram_plan(m, n, ctx->sm_count);
    if (prec == OQR_FP64) {
        oqr_status v = ensure_ws(ctx, align256(gram_partials_bytes(gp)));
        if (v != OQR_OK) return v;
        if ((v = reset_status(ctx, s)) != OQR_OK) return v;
        OQR_TRY(launch_gram_f64(gp, A, lda, Z, ldz, static_cast<double*>(ctx->ws), ctx->st, 4000000000ull, s));
        OQR_TRY(launch_gram_reduce(gp, static_cast<double*>(ctx->ws), G, ldg, nullptr, ctx->st, s));
        return OQR_OK;
    }
    const TcPlan tp = tc_plan(m, n, tc_mode_of(prec));
    oqr_status v = ensure_ws(ctx, align256(tc_workspace_bytes(tp)) + align256((size_t)n * n * 8));
    if (v != OQR_OK) return v;
    if ((v = reset_status(ctx, s)) != OQR_OK) return v;
    // the tensor-core path writes G with leading dimension n into the workspace tail, then copies out
    double* Gt = reinterpret_cast<double*>(static_cast<char*>(ctx->ws) + align256(tc_workspace_bytes(tp)));
    OQR_TRY(launch_tc_gram(tp, A, lda, Z, ldz, Gt, n, nullptr, ctx->ws, ctx->st, 4000000000ull, ctx->sm_count, s));
    OQR_TRY(cudaMemcpy2DAsync(G, ldg * sizeof(double), Gt, n * sizeof(double), n * sizeof(double), n,
                              cudaMemcpyDeviceToDevice, s));
    return OQR_OK;
}

int oqr_batched_default_splits(int m, int n)
{
    (void)n;
    if (m < 1) return 1;
    const long nb = (m + 63) / 64;
    const long steps = 2 * (nb - 1) * nb + ((std::min<long>((long)nb * 64, m) + 15) / 16);
    long sp = (steps + 255) / 256;
    return (int)std::max(1L, std::min(64L, sp));
}

oqr_status oqr_batched(oqr_ctx* ctx, int count, const int* m, const int* n, const double* const* A, const long* lda,
                       const double* const* Z, const long* ldz, double* const* Q, const long* ldq, double* const* R,
                       const long* ldr, int mode, const oqr_opts* opts, int* status, void* stream)
{
    if (!ctx || count < 1 || count > 65535 || !m || !n || !A || !lda || !Z || !ldz || !Q || !ldq || !R || !ldr ||
        !status)
        return OQR_ERR_INVALID_ARG;
    const oqr_opts o = resolve(opts);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (mode >= OQR_BATCHED_TC && mode <= OQR_BATCHED_SHIFTED_TC) {
        const int prog = mode == OQR_BATCHED_TC ? OQR_BATCH_CHOLQR2_TC
                         : mode == OQR_BATCHED_TC2_FIRST ? OQR_BATCH_CHOLQR2_TC2
                                                         : OQR_BATCH_SCHOLQR3_TC;
        std::vector<int> pr((size_t)count, prog);
        return oqr_batched_mixed(ctx, count, m, n, A, lda, Z, ldz, Q, ldq, R, ldr, pr.data(), status, o.batch_orth,
                                 stream);
    }
    if (mode == OQR_BATCHED_FP64)
        return batched_fp64_impl(ctx, count, m, n, A, lda, Z, ldz, Q, ldq, R, ldr, o.batch_splits, status, s);
    if (mode != OQR_BATCHED_SELECTOR) return OQR_ERR_INVALID_ARG;
    for (int b = 0; b < count; ++b) {
        const int mb = m[b], nb = n[b];
        if (mb < 1 || nb < 1 || nb > mb || nb > BATCH_MAX_N || mb > BATCH_MAX_M) return OQR_ERR_INVALID_ARG;
        if (bad_matrix(A[b], lda[b], mb, mb) || bad_matrix(Z[b], ldz[b], mb, nb) || bad_matrix(Q[b], ldq[b], mb, nb) ||
            bad_matrix(R[b], ldr[b], nb, nb))
            return OQR_ERR_INVALID_ARG;
    }
    const SelInputs in{count, m, n, A, lda, Z, ldz, Q, ldq, R, ldr};
    return selector_batch(ctx, in, o, status, s);
}

oqr_status oqr_batched_features(oqr_ctx* ctx, int count, const int* m, const int* n, const double* const* A,
                                const long* lda, const double* const* Z, const long* ldz, float* feat, void* stream)
{
    if (!ctx || count < 1 || count > 65535 || !m || !n || !A || !lda || !Z || !ldz || !feat) return OQR_ERR_INVALID_ARG;
    for (int b = 0; b < count; ++b) {
        const int mb = m[b], nb = n[b];
        if (mb < 1 || nb < 1 || nb > mb || nb > BATCH_MAX_N || mb > BATCH_MAX_M) return OQR_ERR_INVALID_ARG;
        if (bad_matrix(A[b], lda[b], mb, mb) || bad_matrix(Z[b], ldz[b], mb, nb)) return OQR_ERR_INVALID_ARG;
    }
    const SelInputs in{count, m, n, A, lda, Z, ldz, nullptr, nullptr, nullptr, nullptr};
    return features_waves(ctx, in, feat, static_cast<cudaStream_t>(stream));
}

oqr_status oqr_batched_mixed(oqr_ctx* ctx, int count, const int* m, const int* n, const double* const* A,
                             const long* lda, const double* const* Z, const long* ldz, double* const* Q,
                             const long* ldq, double* const* R, const long* ldr, const int* program, int* status,
                             double* orth, void* stream)
{
    if (!ctx || count < 1 || count > 65535 || !m || !n || !A || !lda || !Z || !ldz || !Q || !ldq || !R || !ldr ||
        !status)
        return OQR_ERR_INVALID_ARG;
    for (int b = 0; b < count; ++b) {
        const int mb = m[b], nb = n[b];
        if (mb < 1 || nb < 1 || nb > mb || nb > BATCH_MAX_N || mb > BATCH_MAX_M) return OQR_ERR_INVALID_ARG;
        if (bad_matrix(A[b], lda[b], mb, mb) || bad_matrix(Z[b], ldz[b], mb, nb) || bad_matrix(Q[b], ldq[b], mb, nb) ||
            bad_matrix(R[b], ldr[b], nb, nb))
            return OQR_ERR_INVALID_ARG;
        if (program && (program[b] < OQR_BATCH_CHOLQR_TC || program[b] > OQR_BATCH_SCHOLQR3_TC))
            return OQR_ERR_INVALID_ARG;
    }
    // largest m first: a wave's plane pitch is its first instance's m
    std::vector<int> perm((size_t)count);
    for (int b = 0; b < count; ++b) perm[b] = b;
    std::stable_sort(perm.begin(), perm.end(), [&](int x, int y) { return m[x] > m[y]; });
    std::vector<TcBatchShape> sh((size_t)count);
    std::vector<int> shifted((size_t)count, 0);
    // the graph writes status (and orth) directly: their addresses are part of its signature
    std::vector<long> key{count, 0, (long)reinterpret_cast<uintptr_t>(status), (long)reinterpret_cast<uintptr_t>(orth)};
    size_t pool_doubles = 0;
    for (int i = 0; i < count; ++i) {
        const int b = perm[i];
        const int pr = program ? program[b] : OQR_BATCH_CHOLQR2_TC;
        const int npass = pr == OQR_BATCH_CHOLQR_TC ? 1 : pr == OQR_BATCH_SCHOLQR3_TC ? 3 : 2;
        sh[i] = TcBatchShape{m[b], n[b], pr == OQR_BATCH_CHOLQR2_TC2 ? 3 : 1, npass + (orth ? 1 : 0)};
        shifted[i] = pr == OQR_BATCH_SCHOLQR3_TC;
        key.push_back(((long)m[b] << 32) | ((long)n[b] << 8) | (orth ? 4 : 0) | pr);
        pool_doubles += align256((size_t)4 * n[b] * n[b] * sizeof(double)) / sizeof(double);
    }
    const size_t budget = ctx->batch_budget ? ctx->batch_budget : BATCH_WAVE_BYTES;
    key.push_back((long)budget);
    const TcBatchPlan plan = tc_batch_plan(sh, budget);
    auto layout = [&](Carve& c, char** tab, BatchDesc** d, int** sts, int** dperm, int** dshifted, double** anorm2,
                      double** shifts, double** orths, double** pool, double** upool, void** scratch) {
        *tab = c.take<char>(plan.table_bytes);
        *orths = c.take<double>((size_t)count);
        *d = c.take<BatchDesc>((size_t)count);
        *sts = c.take<int>((size_t)count);
        *dperm = c.take<int>((size_t)count);
        *dshifted = c.take<int>((size_t)count);
        *anorm2 = c.take<double>((size_t)2 * count);  // ||A_b||_F^2, then ||Z_b||_F^2
        *shifts = c.take<double>((size_t)count);
        *pool = c.take<double>(pool_doubles);
        *upool = c.take<double>((size_t)plan.upool_doubles);
        *scratch = c.take<char>(plan.scratch_bytes);
    };
    char* tab;
    BatchDesc* ddesc;
    int *sts, *dperm, *dshifted;
    double *anorm2, *shifts, *orths, *pool, *upool;
    void* scratch;
    Carve probe(nullptr);
    layout(probe, &tab, &ddesc, &sts, &dperm, &dshifted, &anorm2, &shifts, &orths, &pool, &upool, &scratch);
    oqr_status v = ensure_ws(ctx, probe.off);
    if (v != OQR_OK) return v;
    Carve cv(ctx->ws);
    layout(cv, &tab, &ddesc, &sts, &dperm, &dshifted, &anorm2, &shifts, &orths, &pool, &upool, &scratch);
    key[1] = (long)reinterpret_cast<uintptr_t>(ctx->ws);
    // per instance (sorted order): its descriptor (one Gram partial = the product's half C) and tensor-core inputs
    std::vector<BatchDesc> desc((size_t)count);
    std::vector<TcBatchIn> in((size_t)count);
    double* q = pool;
    for (int i = 0; i < count; ++i) {
        const int b = perm[i];
        const size_t nn = (size_t)n[b] * n[b];
        BatchDesc& d = desc[i];
        d.A = A[b];
        d.Z = Z[b];
        d.Q = Q[b];
        d.R = R[b];
        d.lda = lda[b];
        d.ldz = ldz[b];
        d.ldq = ldq[b];
        d.ldr = ldr[b];
        d.m = m[b];
        d.n = n[b];
        d.splits = 1;
        d.npass = sh[i].npass - (orth ? 1 : 0);  // factor passes
        d.partials = q;
        d.G = q + nn;
        d.R1 = d.G + nn;
        d.R2 = d.R1 + nn;
        q += align256(4 * nn * sizeof(double)) / sizeof(double);
        in[i] = TcBatchIn{A[b], lda[b], Z[b], ldz[b], Q[b], ldq[b], d.partials};
    }
    std::vector<char> image;
    tc_batch_tables(plan, sh, in, tab, upool, image);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    OQR_TRY(cudaMemcpyAsync(tab, image.data(), image.size(), cudaMemcpyHostToDevice, s));
    OQR_TRY(cudaMemcpyAsync(ddesc, desc.data(), sizeof(BatchDesc) * count, cudaMemcpyHostToDevice, s));
    OQR_TRY(cudaMemcpyAsync(dperm, perm.data(), sizeof(int) * count, cudaMemcpyHostToDevice, s));
    OQR_TRY(cudaMemcpyAsync(dshifted, shifted.data(), sizeof(int) * count, cudaMemcpyHostToDevice, s));
    OQR_TRY(cudaMemsetAsync(sts, 0, sizeof(int) * count, s));
    if ((v = reset_status(ctx, s)) != OQR_OK) return v;
    const uint64_t limit = 4000000000ull;
    auto seq = [&]() -> cudaError_t {
        cudaError_t e;
        for (int w = 0; w < (int)plan.waves.size(); ++w) {
            const NvtxRange range("oqr: batched wave %d", w);
            const TcBatchWave& W = plan.waves[w];
            const BatchDesc* dw = ddesc + W.first;
            int* sw = sts + W.first;
            bool any_shift = false;
            for (int i = W.first; i < W.first + W.count; ++i) any_shift = any_shift || shifted[i];
            if ((e = tc_batch_split_a(plan, w, tab, scratch, s)) != cudaSuccess) return e;
            for (int pass = 0; pass < W.maxpass; ++pass) {
                if ((e = tc_batch_gram(plan, w, pass, tab, scratch, ctx->st, limit, ctx->sm_count, s)) != cudaSuccess)
                    return e;
                if (pass == 0 && any_shift &&
                    ((e = tc_batch_norms(plan, w, tab, scratch, anorm2 + W.first, anorm2 + count + W.first, s)) !=
                         cudaSuccess ||
                     (e = launch_batched_shifts(dw, W.count, dshifted + W.first, anorm2 + W.first,
                                                anorm2 + count + W.first, 11.0, U64, shifts + W.first, s)) !=
                         cudaSuccess))
                    return e;
                if ((e = launch_batched_factor(dw, W.count, sw, pass, any_shift ? shifts + W.first : nullptr, s)) !=
                    cudaSuccess)
                    return e;
                if (orth && (e = launch_batched_check(dw, W.count, sw, pass, orths + W.first, s)) != cudaSuccess)
                    return e;
            }
            if ((e = launch_batched_rfinal(dw, W.count, sw, s)) != cudaSuccess) return e;
        }
        if (orth && (e = launch_batch_scatter_f64(orths, dperm, count, orth, s)) != cudaSuccess) return e;
        return launch_batch_status_scatter(sts, dperm, count, ctx->st, status, s);
    };
    return run_cached_graph(ctx, key, seq, s);
}

oqr_status oqr_features(oqr_ctx* ctx, int m, int n, const double* A, long lda, const double* Z, long ldz, float* feat,
                        void* stream)
{
    if (!ctx || !feat || m < 1 || n < 1 || n > m || bad_matrix(A, lda, m, m) || bad_matrix(Z, ldz, m, n))
        return OQR_ERR_INVALID_ARG;
    if (n > 1024) return OQR_ERR_UNSUPPORTED;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const TcPlan tp = tc_plan(m, n, 0);
    const size_t tb = align256(tc_workspace_bytes(tp));
    oqr_status v = ensure_ws(ctx, tb + 2 * align256((size_t)n * n * 8) + align256(2 * SHIFT_PARTS * 8));
    if (v != OQR_OK) return v;
    if ((v = reset_status(ctx, s)) != OQR_OK) return v;
    char* w = static_cast<char*>(ctx->ws);
    double* G = reinterpret_cast<double*>(w + tb);
    double* C = reinterpret_cast<double*>(w + tb + align256((size_t)n * n * 8));
    double* scratch = reinterpret_cast<double*>(w + tb + 2 * align256((size_t)n * n * 8));
    OQR_TRY(launch_tc_gram(tp, A, lda, Z, ldz, G, n, nullptr, ctx->ws, ctx->st, 4000000000ull, ctx->sm_count, s));
    OQR_TRY(launch_norms_and_shift(m, n, A, lda, Z, ldz, 0.0, U64, scratch, 2 * SHIFT_PARTS, ctx->st, s));
    OQR_TRY(launch_features(m, n, G, n, C, ctx->st, feat, s));
    return OQR_OK;
}

int oqr_mlp_param_count(void) { return MLP_PARAMS; }

oqr_status oqr_mlp_forward(oqr_ctx* ctx, int B, const float* X, const float* params, int bf16, float* logits,
                           int* choice, void* stream)
{
    if (!ctx || B < 1 || !X || !params || (!logits && !choice)) return OQR_ERR_INVALID_ARG;
    OQR_TRY(launch_mlp_forward(B, X, params, bf16, logits, choice, static_cast<cudaStream_t>(stream)));
    return OQR_OK;
}

oqr_status oqr_mlp_grad(oqr_ctx* ctx, int B, const float* X, const int* y, const float* params, float* grad,
                        float* loss, void* stream)
{
    if (!ctx || B < 1 || !X || !y || !params || !grad) return OQR_ERR_INVALID_ARG;
    oqr_status v = ensure_ws(ctx, align256(mlp_scratch_bytes(B)));
    if (v != OQR_OK) return v;
    OQR_TRY(launch_mlp_grad(B, X, y, params, grad, loss, static_cast<float*>(ctx->ws),
                            static_cast<cudaStream_t>(stream)));
    return OQR_OK;
}

oqr_status oqr_mlp_adam(oqr_ctx* ctx, float* params, const float* grad, float* m, float* v, float lr, float beta1,
                        float beta2, float eps, int t, void* stream)
{
    if (!ctx || !params || !grad || !m || !v || t < 1) return OQR_ERR_INVALID_ARG;
    OQR_TRY(launch_adam(MLP_PARAMS, params, grad, m, v, lr, beta1, beta2, eps, t, static_cast<cudaStream_t>(stream)));
    return OQR_OK;
}

oqr_status oqr_gram_phases(oqr_ctx* ctx, int m, int n, const double* A, long lda, const double* Z, long ldz,
                           double* G, long ldg, int prec, float* phase_ms, int* nphase, void* stream)
{
    if (!ctx || !phase_ms || !nphase || m < 1 || n < 1 || n > m || bad_matrix(A, lda, m, m) ||
        bad_matrix(Z, ldz, m, n) || bad_matrix(G, ldg, n, n))
        return OQR_ERR_INVALID_ARG;
    if (!prec_ok(prec)) return OQR_ERR_INVALID_ARG;
    if (n > 1024) return OQR_ERR_UNSUPPORTED;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t ev[7];
    for (int i = 0; i < 7; ++i)
        if (cudaEventCreate(&ev[i]) != cudaSuccess) return OQR_ERR_CUDA;
    oqr_status v = OQR_OK;
    if (prec == OQR_FP64) {
        const GramPlan gp = gram_plan(m, n, ctx->sm_count);
        v = ensure_ws(ctx, align256(gram_partials_bytes(gp)));
        if (v == OQR_OK) v = reset_status(ctx, s);
        if (v == OQR_OK) {
            cudaEventRecord(ev[0], s);
            launch_gram_f64(gp, A, lda, Z, ldz, static_cast<double*>(ctx->ws), ctx->st, 4000000000ull, s);
            cudaEventRecord(ev[1], s);
            launch_gram_reduce(gp, static_cast<double*>(ctx->ws), G, ldg, nullptr, ctx->st, s);
            cudaEventRecord(ev[2], s);
            *nphase = 2;
        }
    } else {
        const TcPlan tp = tc_plan(m, n, tc_mode_of(prec));
        v = ensure_ws(ctx, align256(tc_workspace_bytes(tp)) + align256((size_t)n * n * 8));
        if (v == OQR_OK) v = reset_status(ctx, s);
        if (v == OQR_OK) {
            double* Gt = reinterpret_cast<double*>(static_cast<char*>(ctx->ws) + align256(tc_workspace_bytes(tp)));
            if (launch_tc_gram(tp, A, lda, Z, ldz, Gt, n, nullptr, ctx->ws, ctx->st, 4000000000ull, ctx->sm_count, s,
                               ev) != cudaSuccess)
                v = OQR_ERR_CUDA;
            else if (cudaMemcpy2DAsync(G, ldg * sizeof(double), Gt, n * sizeof(double), n * sizeof(double), n,
                                       cudaMemcpyDeviceToDevice, s) != cudaSuccess)
                v = OQR_ERR_CUDA;
            *nphase = 5;
        }
    }
    if (v == OQR_OK) {
        if (cudaStreamSynchronize(s) != cudaSuccess) v = OQR_ERR_CUDA;
        for (int i = 0; v == OQR_OK && i < *nphase; ++i)
            if (cudaEventElapsedTime(&phase_ms[i], ev[i], ev[i + 1]) != cudaSuccess) v = OQR_ERR_CUDA;
    }
    for (int i = 0; i < 7; ++i) cudaEventDestroy(ev[i]);
    return v;
}

oqr_status oqr_potrf(oqr_ctx* ctx, int n, const double* G, long ldg, double shift, double* R, long ldr, int* info,
                     void* stream)
{
    if (!ctx || n < 1 || bad_matrix(G, ldg, n, n) || bad_matrix(R, ldr, n, n) || G == R) return OQR_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    oqr_status v = reset_status(ctx, s);
    if (v != OQR_OK) return v;
    OQR_TRY(cudaMemcpyAsync(&ctx->st->shift, &shift, sizeof(double), cudaMemcpyHostToDevice, s));
    OQR_TRY(launch_potrf(n, G, ldg, R, ldr, &ctx->st->shift, ctx->st, s));
    if (!info) return OQR_OK;
    int col = 0;
    v = oqr_get_status(ctx, stream, &col);
    *info = v == OQR_ERR_NOT_SPD ? col : 0;
    return v;
}

oqr_status oqr_trsm(oqr_ctx* ctx, int m, int n, const double* Z, long ldz, const double* R, long ldr, double* Q,
                    long ldq, void* stream)
{
    if (!ctx || m < 1 || n < 1 || bad_matrix(Z, ldz, m, n) || bad_matrix(R, ldr, n, n) || bad_matrix(Q, ldq, m, n))
        return OQR_ERR_INVALID_ARG;
    if (n > 1024) return OQR_ERR_UNSUPPORTED;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    oqr_status v = reset_status(ctx, s);
    if (v != OQR_OK) return v;
    OQR_TRY(launch_trsm(m, n, Z, ldz, R, ldr, Q, ldq, ctx->st, s));
    return OQR_OK;
}

oqr_status oqr_trsm_tc(oqr_ctx* ctx, int m, int n, const double* Z, long ldz, const double* R, long ldr, double* Q,
                       long ldq, void* stream)
{
    if (!ctx || m < 1 || n < 1 || bad_matrix(Z, ldz, m, n) || bad_matrix(R, ldr, n, n) || bad_matrix(Q, ldq, m, n))
        return OQR_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    oqr_status v = ensure_ws(ctx, trsm_tc_workspace_bytes(m, n));
    if (v != OQR_OK) return v;
    if ((v = reset_status(ctx, s)) != OQR_OK) return v;
    OQR_TRY(launch_trsm_tc(m, n, Z, ldz, R, ldr, Q, ldq, ctx->ws, ctx->st, 4000000000ull, ctx->sm_count, s));
    return OQR_OK;
}

oqr_status oqr_trsm_last(oqr_ctx* ctx, int m, int n, const double* G, long ldg, const double* Z, long ldz,
                         const double* R, long ldr, double* Q, long ldq, void* stream)
{
    if (!ctx || m < 1 || n < 1 || bad_matrix(G, ldg, n, n) || bad_matrix(Z, ldz, m, n) || bad_matrix(R, ldr, n, n) ||
        bad_matrix(Q, ldq, m, n))
        return OQR_ERR_INVALID_ARG;
    if (n > TRINV_MAX_N) return OQR_ERR_UNSUPPORTED;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    LastSolve L;
    Carve sz(nullptr);
    carve_last(sz, m, n, true, &L);
    oqr_status v = ensure_ws(ctx, sz.off);
    if (v != OQR_OK) return v;
    Carve c(ctx->ws);
    carve_last(c, m, n, true, &L);
    if ((v = reset_status(ctx, s)) != OQR_OK) return v;
    OQR_TRY(launch_last_solve(ctx, m, n, G, ldg, Z, ldz, R, ldr, Q, ldq, L, 4000000000ull, s));
    return OQR_OK;
}

oqr_status oqr_rprod(oqr_ctx* ctx, int n, const double* U, long ldu, const double* S, long lds, double* R, long ldr,
                     void* stream)
{
    if (!ctx || n < 1 || bad_matrix(U, ldu, n, n) || bad_matrix(S, lds, n, n) || bad_matrix(R, ldr, n, n) ||
        R == U || R == S)
        return OQR_ERR_INVALID_ARG;
    OQR_TRY(launch_rprod(n, U, ldu, S, lds, R, ldr, static_cast<cudaStream_t>(stream)));
    return OQR_OK;
}

oqr_status oqr_check(oqr_ctx* ctx, int m, int n, const double* A, long lda, const double* Q, long ldq, double* E,
                     long lde, double* orth2, double* orthF, void* stream)
{
    if (!ctx || m < 1 || n < 1 || n > m || bad_matrix(A, lda, m, m) || bad_matrix(Q, ldq, m, n) ||
        (E && lde < n))
        return OQR_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const GramPlan gp = gram_plan(m, n, ctx->sm_count);
    Carve probe(nullptr);
    double *partials, *G, *work, *R1, *R2, *R3, *scratch;
    layout_cholqr(probe, gp, &partials, &G, &work, &R1, &R2, &R3, &scratch);
    oqr_status v = ensure_ws(ctx, probe.off);
    if (v != OQR_OK) return v;
    Carve c(ctx->ws);
    layout_cholqr(c, gp, &partials, &G, &work, &R1, &R2, &R3, &scratch);
    if ((v = reset_status(ctx, s)) != OQR_OK) return v;
    if ((v = run_check(ctx, gp, A, lda, Q, ldq, partials, G, work, E, lde, 4000000000ull, s)) != OQR_OK) return v;
    if (orth2 || orthF) {
        if (cudaStreamSynchronize(s) != cudaSuccess) return OQR_ERR_CUDA;
        DevStatus h;
        if (cudaMemcpy(&h, ctx->st, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return OQR_ERR_CUDA;
        if (orth2) *orth2 = h.orth2;
        if (orthF) *orthF = h.orthF;
        return static_cast<oqr_status>(h.code);
    }
    return OQR_OK;
}

oqr_status oqr_set_batch_budget(oqr_ctx* ctx, size_t bytes)
{
    if (!ctx) return OQR_ERR_INVALID_ARG;
    ctx->batch_budget = bytes;
    return OQR_OK;
}

oqr_status oqr_diag_timeout(oqr_ctx* ctx, long limit_ns, void* stream)
{
    if (!ctx || limit_ns < 1 || limit_ns > 10000000000L) return OQR_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    oqr_status v = reset_status(ctx, s);
    if (v != OQR_OK) return v;
    OQR_TRY(launch_timeout_probe(ctx->st, (uint64_t)limit_ns, s));
    return OQR_OK;
}

oqr_status oqr_repres(oqr_ctx* ctx, int m, int n, const double* Z, long ldz, const double* Q, long ldq,
                      const double* R, long ldr, double* res2, double* resF, void* stream)
{
    if (!ctx || m < 1 || n < 1 || n > m || bad_matrix(Z, ldz, m, n) || bad_matrix(Q, ldq, m, n) ||
        bad_matrix(R, ldr, n, n))
        return OQR_ERR_INVALID_ARG;
    if (n > 1024) return OQR_ERR_UNSUPPORTED;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // D = Z - Q R (m x n), S = D^T D and T = Z^T Z (split along m), then their largest eigenvalues and traces
    const int splits = std::max(1, std::min(64, m / 512));
    Carve probe(nullptr);
    auto layout = [&](Carve& c, double** D, double** S, double** T, double** ws, double** work, double** out) {
        *D = c.take<double>((size_t)m * n);
        *S = c.take<double>((size_t)n * n);
        *T = c.take<double>((size_t)n * n);
        *ws = c.take<double>(gemm_splitk_bytes(n, n, splits) / sizeof(double) + 1);
        *work = c.take<double>((size_t)2 * n);
        *out = c.take<double>(4);
    };
    double *D, *S, *T, *ws, *work, *out;
    layout(probe, &D, &S, &T, &ws, &work, &out);
    oqr_status v = ensure_ws(ctx, probe.off);
    if (v != OQR_OK) return v;
    Carve c(ctx->ws);
    layout(c, &D, &S, &T, &ws, &work, &out);
    OQR_TRY(cudaMemcpy2DAsync(D, (size_t)m * 8, Z, (size_t)ldz * 8, (size_t)m * 8, n, cudaMemcpyDeviceToDevice, s));
    OQR_TRY(launch_gemm_f64(GEMM_N, m, n, n, -1.0, Q, ldq, R, ldr, 1.0, D, m, nullptr, 1, s));
    OQR_TRY(launch_gemm_f64(GEMM_T, n, n, m, 1.0, D, m, D, m, 0.0, S, n, ws, splits, s));
    OQR_TRY(launch_gemm_f64(GEMM_T, n, n, m, 1.0, Z, ldz, Z, ldz, 0.0, T, n, ws, splits, s));
    OQR_TRY(launch_lambda_max(n, S, n, work, out, s));
    OQR_TRY(launch_lambda_max(n, T, n, work, out + 2, s));
    double h[4];
    OQR_TRY(cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, s));
    if (cudaStreamSynchronize(s) != cudaSuccess) return OQR_ERR_CUDA;
    if (res2) *res2 = h[2] > 0.0 ? std::sqrt(h[0] / h[2]) : 0.0;
    if (resF) *resF = h[3] > 0.0 ? std::sqrt(h[1] / h[3]) : 0.0;
    return OQR_OK;
}

oqr_status oqr_cholqr2_tridiag(oqr_ctx* ctx, int m, int n, const double* d, const double* e, const double* Z, long ldz,
                               double* Q, long ldq, double* R, long ldr, const oqr_opts* opts, oqr_info* info,
                               void* stream)
{
    if (!d) return OQR_ERR_INVALID_ARG;
    AOp op;
    op.d = d;
    op.e = e;
    return normal_equation(ctx, m, n, op, Z, ldz, Q, ldq, R, ldr, opts, info, stream, 0);
}

oqr_status oqr_gram_tridiag(oqr_ctx* ctx, int m, int n, const double* d, const double* e, const double* Z, long ldz,
                            double* G, long ldg, int prec, void* stream)
{
    if (!ctx || !d || (m > 1 && !e) || m < 1 || n < 1 || n > m || bad_matrix(Z, ldz, m, n) ||
        bad_matrix(G, ldg, n, n))
        return OQR_ERR_INVALID_ARG;
    if (!prec_ok(prec)) return OQR_ERR_INVALID_ARG;
    if (n > 1024) return OQR_ERR_UNSUPPORTED;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const GramPlan gp = gram_plan(m, n, ctx->sm_count);
    AOp op;
    op.d = d;
    op.e = e;
    const size_t tcb = prec == OQR_FP64 ? 0 : tc_workspace_bytes(tc_plan(m, n, tc_mode_of(prec), 0, true));
    auto layout = [&](Carve& c, double** part, double** Ub, double** Cb, double** Gt, void** tcws) {
        *part = c.take<double>(gram_partials_bytes(gp) / sizeof(double));
        *Ub = c.take<double>((size_t)m * n);
        *Cb = c.take<double>((size_t)n * n);
        *Gt = c.take<double>((size_t)n * n);
        *tcws = c.take<char>(tcb);
    };
    double *part, *Ub, *Cb, *Gt;
    void* tcws;
    Carve probe(nullptr);
    layout(probe, &part, &Ub, &Cb, &Gt, &tcws);
    oqr_status v = ensure_ws(ctx, probe.off);
    if (v != OQR_OK) return v;
    Carve c(ctx->ws);
    layout(c, &part, &Ub, &Cb, &Gt, &tcws);
    if ((v = reset_status(ctx, s)) != OQR_OK) return v;
    OQR_TRY(form_gram(ctx, prec, gp, op, Z, ldz, part, Gt, nullptr, tcws, 4000000000ull, s, nullptr, Ub, Cb));
    OQR_TRY(cudaMemcpy2DAsync(G, ldg * sizeof(double), Gt, n * sizeof(double), n * sizeof(double), n,
                              cudaMemcpyDeviceToDevice, s));
    return OQR_OK;
}

oqr_status oqr_precholqr(oqr_ctx* ctx, int m, int n, const double* A, long lda, const double* Z, long ldz, double* Q,
                         long ldq, double* R, long ldr, const oqr_opts* opts, oqr_info* info, void* stream)
{
    return precholqr_impl(ctx, m, n, dense_op(A, lda), Z, ldz, Q, ldq, R, ldr, opts, info,
                          static_cast<cudaStream_t>(stream));
}

oqr_status oqr_precholqr_tridiag(oqr_ctx* ctx, int m, int n, const double* d, const double* e, const double* Z,
                                 long ldz, double* Q, long ldq, double* R, long ldr, const oqr_opts* opts,
                                 oqr_info* info, void* stream)
{
    if (!d) return OQR_ERR_INVALID_ARG;
    AOp op;
    op.d = d;
    op.e = e;
    return precholqr_impl(ctx, m, n, op, Z, ldz, Q, ldq, R, ldr, opts, info, static_cast<cudaStream_t>(stream));
}

oqr_status oqr_tsqr(oqr_ctx* ctx, int m, int n, const double* Z, long ldz, double* Y, long ldy, double* S, long lds,
                    void* stream)
{
    if (!ctx || m < 1 || n < 1 || n > m || bad_matrix(Z, ldz, m, n) || bad_matrix(Y, ldy, m, n) ||
        bad_matrix(S, lds, n, n))
        return OQR_ERR_INVALID_ARG;
    if (n > 1024) return OQR_ERR_UNSUPPORTED;
    oqr_status v = ensure_ws(ctx, euclid_qr_bytes(m, n, ctx->sm_count));
    if (v != OQR_OK) return v;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if ((v = reset_status(ctx, s)) != OQR_OK) return v;
    const oqr_opts o = resolve(nullptr);
    OQR_TRY(launch_euclid_qr(m, n, Z, ldz, Y, ldy, S, lds, static_cast<double*>(ctx->ws), ctx->sm_count, ctx->st,
                             (uint64_t)o.spin_limit, s));
    oqr_info info;
    return finish(ctx, s, &info, 0, false);
}

oqr_status oqr_symm(oqr_ctx* ctx, int m, int k, const double* A, long lda, const double* B, long ldb, double* C,
                    long ldc, void* stream)
{
    if (!ctx || m < 1 || k < 1 || bad_matrix(A, lda, m, m) || bad_matrix(B, ldb, m, k) || bad_matrix(C, ldc, m, k))
        return OQR_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    oqr_status v = ensure_ws(ctx, align256(symm_workspace_doubles(m, k) * sizeof(double)));
    if (v != OQR_OK) return v;
    OQR_TRY(launch_symm(m, k, A, lda, B, ldb, C, ldc, static_cast<double*>(ctx->ws), ctx->sm_count, s));
    return OQR_OK;
}

oqr_status oqr_glls(oqr_ctx* ctx, int m, int n, int k, const double* A, long lda, const double* Q, long ldq,
                    const double* R, long ldr, const double* B, long ldb, double* X, long ldx, void* stream)
{
    if (!ctx || m < 1 || n < 1 || n > m || k < 1 || bad_matrix(A, lda, m, m) || bad_matrix(Q, ldq, m, n) ||
        bad_matrix(R, ldr, n, n) || bad_matrix(B, ldb, m, k) || bad_matrix(X, ldx, n, k))
        return OQR_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // C = A B (m x k), Y = Q^T C (n x k, split along m), X = R^{-1} Y
    const int tiles = ((n + 63) / 64) * ((k + 63) / 64);
    const int splits = std::max(1, std::min(64, 2 * ctx->sm_count / tiles));
    auto layout = [&](Carve& c, double** part, double** Cm, double** Y, double** ws) {
        *part = c.take<double>(symm_workspace_doubles(m, k));
        *Cm = c.take<double>((size_t)m * k);
        *Y = c.take<double>((size_t)n * k);
        *ws = c.take<double>(gemm_splitk_bytes(n, k, splits) / sizeof(double) + 1);
    };
    Carve probe(nullptr);
    double *part, *Cm, *Y, *ws;
    layout(probe, &part, &Cm, &Y, &ws);
    oqr_status v = ensure_ws(ctx, probe.off);
    if (v != OQR_OK) return v;
    Carve c(ctx->ws);
    layout(c, &part, &Cm, &Y, &ws);
    OQR_TRY(launch_symm(m, k, A, lda, B, ldb, Cm, m, part, ctx->sm_count, s));
    OQR_TRY(launch_gemm_f64(GEMM_T, n, k, m, 1.0, Q, ldq, Cm, m, 0.0, Y, n, ws, splits, s));
    OQR_TRY(launch_upper_solve(n, k, R, ldr, Y, n, X, ldx, s));
    return OQR_OK;
}

}  // extern "C"

// --------------------------------------------------------- tensor maps ------
namespace oqr {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        cudaGetLastError();
    }
    return fn;
}

bool make_tensor_map_2d(CUtensorMap* map, CUtensorMapDataType dtype, int elem_bytes, const void* base, long rows,
                        long cols, long ld, int box_rows, int box_cols)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
    cuuint64_t strides[1] = {(cuuint64_t)ld * (cuuint64_t)elem_bytes};
    cuuint32_t box[2] = {(cuuint32_t)box_rows, (cuuint32_t)box_cols};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, dtype, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace oqr
