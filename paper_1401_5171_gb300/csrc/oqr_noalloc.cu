// Allocation-free variant of the fused Gram entry point.
//
// Some callers cannot call cudaMalloc at all: a plug-in running under another
// framework whose caching allocator has already reserved the device memory
// (a direct allocation would fail or fragment it), and real-time or embedded
// hosts that fix their memory at start-up and cannot afford an allocation's
// latency or the device synchronization that cudaMalloc and cudaFree may
// imply.  oqr_gram_noalloc serves them: it computes the same G = Z^T A Z as
// oqr_gram, but its split-K partial sums and its status word live in one
// file-scope device array of fixed size instead of a context workspace, and
// the call takes no context (creating one allocates).
//
// The first call on a device looks up the array's device address
// (cudaGetSymbolAddress, with that device current) and caches it; make that
// first call before any stream capture on the device.
//
// The array is NOALLOC_SCRATCH_BYTES (8 MiB + 256 B) on every device that
// loads this library, held until the process exits.  It limits the number of
// split-K partials to floor(8 MiB / (8 n^2)); n above 1024 is rejected.
// Every call on a device shares the array, so calls that overlap on the GPU
// (different streams, no ordering) race on it; the status word is cleared at
// the start of every call and the partials are overwritten, never
// accumulated into, so nothing is left over from an earlier call.
//
// There is no context to report a device-side failure to, so a failure is
// made visible in the result itself: if a time-limited wait of the Gram
// kernel gives up, every element of G is set to NaN (the reduction then
// skips its writes, and the last kernel of the call fills G).
//
// The cached address belongs to the device's primary context as it was at the
// first call; cudaDeviceReset after that call is not supported (the module
// reloads and the array may move).
#include <mutex>

#include "oqr_internal.cuh"

using namespace oqr;

namespace {

constexpr size_t NOALLOC_HEADER_BYTES = 256;  // DevStatus, padded
constexpr size_t NOALLOC_SCRATCH_BYTES = NOALLOC_HEADER_BYTES + (size_t(8) << 20);
constexpr int NOALLOC_MAX_N = 1024;
constexpr int NOALLOC_MAX_DEVICES = 64;
static_assert(sizeof(DevStatus) <= NOALLOC_HEADER_BYTES, "status header");

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[NOALLOC_MAX_DEVICES];  // device address of g_noalloc_scratch, per device

// The device address of the array on the current device, looked up once per
// device (with that device current).  In host code g_noalloc_scratch names a
// host-side shadow, never the device memory, so kernels only ever receive this
// looked-up address.
oqr_status scratch_on_current_device(void** out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return OQR_ERR_CUDA;
    }
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return OQR_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return OQR_ERR_CUDA;
        }
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return OQR_OK;
}

// G (n x n, ldg) = NaN everywhere when the call's status word records an error.
__global__ void noalloc_fail_fill_kernel(int n, double* G, long ldg, const DevStatus* st)
{
    if (*(volatile const int*)&st->code == 0) return;
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long)n * n) return;
    G[(e % n) + (e / n) * ldg] = __longlong_as_double(0x7FF8000000000000LL);
}

}  // namespace

extern "C" oqr_status oqr_gram_noalloc(int m, int n, const double* A, long lda, const double* Z, long ldz,
                                       double* G, long ldg, void* stream)
{
    if (m < 1 || n < 1 || n > m || !A || !Z || !G || lda < m || ldz < m || ldg < n) return OQR_ERR_INVALID_ARG;
    if (n > NOALLOC_MAX_N) return OQR_ERR_UNSUPPORTED;
    void* base = nullptr;
    oqr_status v = scratch_on_current_device(&base);
    if (v != OQR_OK) return v;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess) {
        cudaGetLastError();
        return OQR_ERR_CUDA;
    }
    DevStatus* st = static_cast<DevStatus*>(base);
    double* partials = reinterpret_cast<double*>(static_cast<char*>(base) + NOALLOC_HEADER_BYTES);
    const size_t capacity = (NOALLOC_SCRATCH_BYTES - NOALLOC_HEADER_BYTES) / sizeof(double);
    GramPlan p = gram_plan(m, n, sms);
    const size_t max_splits = capacity / ((size_t)n * n);
    if (max_splits < 1) return OQR_ERR_UNSUPPORTED;
    if ((size_t)p.splits > max_splits) p.splits = (int)max_splits;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(st, 0, sizeof(DevStatus), s) != cudaSuccess) return OQR_ERR_CUDA;
    if (launch_gram_f64(p, A, lda, Z, ldz, partials, st, 4000000000ull, s) != cudaSuccess) return OQR_ERR_CUDA;
    if (launch_gram_reduce(p, partials, G, ldg, nullptr, st, s) != cudaSuccess) return OQR_ERR_CUDA;
    const long tot = (long)n * n;
    noalloc_fail_fill_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(n, G, ldg, st);
    if (cudaGetLastError() != cudaSuccess) return OQR_ERR_CUDA;
    return OQR_OK;
}
