// rtd_noalloc.cu - scoring entry point that allocates no memory.
//
// Some callers cannot allocate device memory at the moment they score:
// a real-time sorting line that must not stall on the allocator between
// frames, code running inside a pre-reserved memory budget, or a host
// process whose device memory is handed out by another component.  For them
// rtdetmcd_distances_noalloc computes the same squared distances as
// rtdetmcd_distances, but keeps its small working state (the factorised
// fit and a status word) in the fixed-size array below instead of a
// caller-provided workspace.
//
// The array is a file-scope __device__ variable: every GPU that loads this
// library holds RTD_NOALLOC_SCRATCH_BYTES of it until the process exits.  In
// host code its name is only a host-side stand-in, not a device address, so
// the address used for the kernels is looked up once per device with
// cudaGetSymbolAddress (with that device current) and cached.  All calls on a
// device share the array and it keeps the last call's contents; calls whose
// device work overlaps (several host threads or streams at once) race on it.
#include <mutex>
#include <string.h>

#include "rtd_internal.cuh"

using namespace rtd;

namespace {

struct NoAllocState {
    Status st;
    double mu[RTD_MAX_P];
    double sigma[RTD_MAX_P * RTD_MAX_P];
    RowParams rp;
};

}  // namespace

static_assert(sizeof(NoAllocState) <= RTD_NOALLOC_SCRATCH_BYTES, "no-alloc scratch too small");

static __device__ __align__(256) unsigned char g_noalloc_scratch[RTD_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int MAX_DEVICES = 64;
std::mutex g_lock;
void* g_addr[MAX_DEVICES] = {};

// Device address of the scratch array on the current device (looked up on
// the first call per device).
int scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RTD_ECUDA;
    if (dev < 0 || dev >= MAX_DEVICES) return RTD_EINVAL;
    std::lock_guard<std::mutex> g(g_lock);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return RTD_ECUDA;
        }
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return RTD_OK;
}

// Device (or managed) memory that the current device's kernels may read as
// their own: memory of another device is refused, not read as peer memory.
bool on_device(const void* ptr) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) { cudaGetLastError(); return false; }
    if (a.type == cudaMemoryTypeManaged) return true;
    if (a.type != cudaMemoryTypeDevice) return false;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return false; }
    return a.device == dev;
}

}  // namespace

extern "C" int rtdetmcd_distances_noalloc(const float* X, int64_t n, int32_t p, int64_t ld,
                                          const double* mu_host, const double* sigma_host,
                                          int32_t precision, float* d2_out, void* stream) {
    if (!X || !mu_host || !sigma_host || !d2_out || n < 1 || n >= (1LL << 31) || ld < p ||
        (precision != RTD_FP32 && precision != RTD_FP64))
        return RTD_EINVAL;
    if (p < 1 || p > RTD_MAX_P) return RTD_EINVAL;          // beyond what the array holds
    // host data would need staging memory; another device's memory is not
    // this device's to write
    if (!on_device(X) || !on_device(d2_out)) return RTD_EINVAL;
    void* base = nullptr;
    int e = scratch_address(&base);
    if (e) return e;
    NoAllocState* S = reinterpret_cast<NoAllocState*>(base);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // the status word must start at zero; mu and sigma are overwritten
    if (cudaMemsetAsync(&S->st, 0, sizeof(Status), s) != cudaSuccess) return RTD_ECUDA;
    if (cudaMemcpyAsync(S->mu, mu_host, (size_t)p * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return RTD_ECUDA;
    if (cudaMemcpyAsync(S->sigma, sigma_host, (size_t)p * p * sizeof(double), cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
        return RTD_ECUDA;
    launch_score_prep(S->mu, S->sigma, p, &S->rp, &S->st, s);
    launch_score(X, n, p, ld, &S->rp, precision, d2_out, s);
    Status hs;
    if (cudaMemcpyAsync(&hs, &S->st, sizeof(Status), cudaMemcpyDeviceToHost, s) != cudaSuccess) return RTD_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return RTD_ECUDA;
    if (cudaGetLastError() != cudaSuccess) return RTD_ECUDA;
    return hs.code;
}
