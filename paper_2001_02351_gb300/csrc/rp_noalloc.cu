// rp_contract_chi0_static: the BF16x3 chi0 contraction with all of its scratch memory in a
// fixed array of this file, so that a call allocates nothing.
//
// Some callers cannot allocate device memory at the point where they need chi0: for example
// an application that reserves the whole device memory budget for its own pool at start-up and
// forbids further cudaMalloc calls, or a latency-critical loop in which a device allocation
// (which can synchronise the whole device) is not allowed.  They pass inputs and outputs that
// they own; the bf16 split of M, the float copy of the weights and the wait-timeout flag live
// in g_static_scratch below.  That array is held by every GPU that loads this library, for as
// long as the process runs.  rp_contract_chi0_static_status reads (and clears) the timeout flag
// the last call left there, also without allocating.
#include <cuda_runtime.h>

#include <mutex>

#include "rp_internal.h"

namespace {

// 64 MiB: bf16 hi part (24 MiB), bf16 lo part (24 MiB), complex-float weights (8 MiB), flags.
constexpr size_t kSplitBytes = (size_t)24 << 20;
constexpr size_t kW32Bytes = (size_t)8 << 20;
constexpr size_t kFlagBytes = 256;
constexpr size_t kScratchBytes = 2 * kSplitBytes + kW32Bytes + kFlagBytes;

static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// device address of g_static_scratch on the current device (looked up once per device)
int scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RP_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return RP_ERR_CUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return RP_OK;
}

// the timeout flag inside the array
int* static_flag(void* base) { return (int*)((unsigned char*)base + 2 * kSplitBytes + kW32Bytes); }

}  // namespace

extern "C" int rp_contract_chi0_static_status(void* cuda_stream) {
    void* base = nullptr;
    int s = scratch_address(&base);
    if (s != RP_OK) return s;
    int* flag = static_flag(base);
    if (cudaStreamSynchronize((cudaStream_t)cuda_stream) != cudaSuccess) {
        cudaGetLastError();
        return RP_ERR_CUDA;
    }
    int v = 0;
    if (cudaMemcpy(&v, flag, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return RP_ERR_CUDA;
    }
    if (v) {
        if (cudaMemset(flag, 0, sizeof(int)) != cudaSuccess) return RP_ERR_CUDA;
        return RP_ERR_TIMEOUT;
    }
    return RP_OK;
}

extern "C" int rp_contract_chi0_static(int ng, long long K, int nfreq, const double* M, const double* w,
                                       double* chi_out, void* cuda_stream) {
    if (ng < 1 || K < 1 || nfreq < 1 || !M || !w || !chi_out) return RP_ERR_ARG;
    const long long kp2 = rp::tc_kp2(K);
    if ((unsigned long long)ng * (unsigned long long)kp2 * 2ULL > kSplitBytes) return RP_ERR_ARG;
    if ((unsigned long long)rp::tc_wrows(nfreq) * (unsigned long long)(kp2 / 2) * 8ULL > kW32Bytes)
        return RP_ERR_ARG;
    void* base = nullptr;
    int s = scratch_address(&base);
    if (s != RP_OK) return s;
    unsigned char* p = (unsigned char*)base;
    void* hi = p;
    void* lo = p + kSplitBytes;
    void* w32 = p + 2 * kSplitBytes;
    int* flag = static_flag(base);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int nsm = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return RP_ERR_CUDA;
    // the output accumulates and the flag records a wait that gave up: both start at zero
    if (cudaMemsetAsync(flag, 0, sizeof(int), st) != cudaSuccess) return RP_ERR_CUDA;
    if (cudaMemsetAsync(chi_out, 0, (size_t)nfreq * ng * ng * sizeof(double2), st) != cudaSuccess) return RP_ERR_CUDA;
    cudaError_t e = rp::launch_split_bf16(M, false, K, 0, K, ng, hi, lo, st);
    if (e == cudaSuccess)
        e = rp::launch_contract_bf16x3(hi, lo, K, ng, (const double2*)w, K, 0, nfreq, w32, (double2*)chi_out, flag,
                                       nsm, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return RP_ERR_CUDA;
    }
    return RP_OK;
}
