// Library-wide entry points of the adpar C ABI: status strings, version,
// workspace sizing and the device status word.
#include "common.cuh"

namespace adpar {
size_t scan_workspace_size(adpar_opdesc d, int64_t n, bool minimal);
size_t reduce_general_workspace_size(adpar_opdesc d, int64_t n, bool minimal);
size_t reduce_workspace_size(adpar_opdesc d);
size_t hist_workspace_size(adpar_opdesc d, int64_t m);
size_t kmeans_workspace_size(int64_t k);
size_t scan_vec_workspace_size(adpar_opdesc d, int64_t n, int64_t m);
size_t hist_general_workspace_size(adpar_opdesc d, int64_t n, int64_t m);
size_t scan_wide_workspace_size(adpar_opdesc d, int64_t n);
size_t jvp_reduce_workspace_size(adpar_opdesc d);
size_t jvp_hist_workspace_size(adpar_opdesc d, int64_t m);
size_t kmeans_fwd_rev_workspace_size(int64_t N, int64_t k);
}

extern "C" const char* adpar_status_string(int status) {
    switch (status) {
    case ADPAR_OK: return "ok";
    case ADPAR_ERR_INVALID: return "invalid argument";
    case ADPAR_ERR_UNSUPPORTED: return "unsupported combination";
    case ADPAR_ERR_ALIGN: return "array not 16-byte aligned";
    case ADPAR_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case ADPAR_ERR_CUDA: return "CUDA error";
    case ADPAR_ERR_TIMEOUT: return "device-side wait timed out";
    case ADPAR_ERR_TOO_LARGE: return "problem needs more than the static no-allocation scratch";
    }
    return "unknown status";
}

extern "C" const char* adpar_version(void) { return "adpar 0.1 (sm_103a)"; }

extern "C" size_t adpar_workspace_size(int rule, adpar_opdesc d, int64_t n, int64_t m) {
    const bool minimal = (rule & ADPAR_WS_MINIMAL) != 0;
    rule &= ~ADPAR_WS_MINIMAL;
    switch (rule) {
    case ADPAR_RULE_SCAN: return adpar::scan_workspace_size(d, n, minimal);
    case ADPAR_RULE_REDUCE_GENERAL: return adpar::reduce_general_workspace_size(d, n, minimal);
    case ADPAR_RULE_SCAN_VEC: return adpar::scan_vec_workspace_size(d, n, m);
    case ADPAR_RULE_HIST_GENERAL: return adpar::hist_general_workspace_size(d, n, m);
    case ADPAR_RULE_SCAN_WIDE: return adpar::scan_wide_workspace_size(d, n);
    case ADPAR_RULE_REDUCE: return n < 0 ? (size_t)-1 : adpar::reduce_workspace_size(d);
    case ADPAR_RULE_HIST: return n < 0 ? (size_t)-1 : adpar::hist_workspace_size(d, m);
    case ADPAR_RULE_KMEANS: return n < 0 ? (size_t)-1 : adpar::kmeans_workspace_size(m);
    case ADPAR_RULE_JVP_REDUCE: return n < 0 ? (size_t)-1 : adpar::jvp_reduce_workspace_size(d);
    case ADPAR_RULE_JVP_HIST: return n < 0 ? (size_t)-1 : adpar::jvp_hist_workspace_size(d, m);
    case ADPAR_RULE_KMEANS_FWD_REV: return adpar::kmeans_fwd_rev_workspace_size(n, m);
    }
    return (size_t)-1;
}

extern "C" int adpar_workspace_status(const void* work, void* stream, int* device_status) {
    if (!work || !device_status) return ADPAR_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(s) != cudaSuccess) return ADPAR_ERR_CUDA;
    uint32_t v = 0;
    if (cudaMemcpy(&v, work, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) return ADPAR_ERR_CUDA;
    *device_status = (int)v;
    return ADPAR_OK;
}

namespace {
__global__ void selftest_init_kernel(uint32_t* words) { words[threadIdx.x] = 0u; }
// one bounded wait on a flag that nothing sets: it gives up after the
// wait limit and records ADPAR_ERR_TIMEOUT in the workspace header
__global__ void selftest_wait_kernel(adpar::WsHeader* hdr, const uint32_t* flag) {
    if (threadIdx.x == 0) (void)adpar::wait_flag(flag, hdr);
}
}  // namespace

extern "C" int adpar_selftest_timeout(void* work, size_t work_bytes, void* stream) {
    if (!work || work_bytes < 512 || (reinterpret_cast<uintptr_t>(work) & 255u)) return ADPAR_ERR_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint32_t* w = static_cast<uint32_t*>(work);
    selftest_init_kernel<<<1, 128, 0, s>>>(w);  // header and the flag word at byte 256
    selftest_wait_kernel<<<1, 32, 0, s>>>(reinterpret_cast<adpar::WsHeader*>(w), w + 64);
    return cudaGetLastError() == cudaSuccess ? ADPAR_OK : ADPAR_ERR_CUDA;
}
