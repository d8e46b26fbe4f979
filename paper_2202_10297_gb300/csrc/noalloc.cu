// adpar_vjp_scan_noalloc: the scan VJP for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the
// point where they need a gradient: code running inside a custom memory
// manager or allocator hook that must not re-enter it, real-time loops
// that forbid allocation after start-up, or hosts that hand the library
// fixed buffers and nothing else.  adpar_vjp_scan needs a caller-supplied
// workspace; this entry point instead uses one static device array that
// every GPU loading the library holds from module load until process exit.
//
// The array's name is a host-side stand-in in host code, not a device
// address, so every call looks up its device address on the current device
// with cudaGetSymbolAddress.  Nothing is cached: a context that is torn down
// and re-created (cudaDeviceReset) may load the module at another address.
#include "common.cuh"

namespace adpar {
size_t scan_workspace_size(adpar_opdesc d, int64_t n, bool minimal);
}

namespace {

// 8 MiB: enough for every scan VJP up to 2^28 FP32 elements of a width-1
// operator and 2^26 FP64 pairs of the linear recurrence.
constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;

static __device__ __align__(256) unsigned char g_scan_scratch[kNoAllocScratchBytes];

// Device address of the static scratch on the current device.  The first
// lookup on a device loads the module there; later ones are cheap.
int scratch_on_current_device(void** out) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scan_scratch) != cudaSuccess || p == nullptr) return ADPAR_ERR_CUDA;
    *out = p;
    return ADPAR_OK;
}

}  // namespace

extern "C" size_t adpar_noalloc_scratch_bytes(void) { return kNoAllocScratchBytes; }

extern "C" int adpar_vjp_scan_noalloc(adpar_opdesc d, int64_t n, const void* a, const void* b,
                                      const void* ybar_a, const void* ybar_b, void* abar, void* bbar,
                                      void* ys_a, void* ys_b, uint32_t flags, void* stream) {
    // size first: a request beyond the static array is refused before any
    // pointer is looked at or anything is enqueued
    const size_t need = adpar::scan_workspace_size(d, n, true);
    if (need == (size_t)-1) return ADPAR_ERR_INVALID;
    if (need > kNoAllocScratchBytes) return ADPAR_ERR_TOO_LARGE;
    void* scratch = nullptr;
    const int st = scratch_on_current_device(&scratch);
    if (st != ADPAR_OK) return st;
    // the scan clears its own flags and counters at the start of every
    // call, so stale contents from the previous call do no harm
    return adpar_vjp_scan(d, n, a, b, ybar_a, ybar_b, abar, bbar, ys_a, ys_b, flags, scratch,
                          kNoAllocScratchBytes, stream);
}

extern "C" int adpar_noalloc_status(void* stream, int* device_status) {
    if (!device_status) return ADPAR_ERR_INVALID;
    void* scratch = nullptr;
    const int st = scratch_on_current_device(&scratch);
    if (st != ADPAR_OK) return st;
    // the status word is the first word of the scan's workspace header,
    // which adpar_vjp_scan_noalloc places at the start of the static array
    return adpar_workspace_status(scratch, stream, device_status);
}

extern "C" int adpar_noalloc_selftest_timeout(void* stream) {
    void* scratch = nullptr;
    const int st = scratch_on_current_device(&scratch);
    if (st != ADPAR_OK) return st;
    return adpar_selftest_timeout(scratch, kNoAllocScratchBytes, stream);
}
