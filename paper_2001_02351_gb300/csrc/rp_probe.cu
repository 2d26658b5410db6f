// Peak probes (measurement aid, no counterpart in the paper): the rates the rooflines of the FP64
// kernels and of the BF16x3 contraction are quoted against, measured on the device that runs them.
//   k_probe_dfma   FP64 FMA pipe: eight independent FMA chains per thread, no memory traffic;
//   k_probe_dmma   FP64 tensor path: back-to-back mma.sync m8n8k4 f64 on register operands, four
//                  independent accumulators per warp;
//   k_probe_bf16   tcgen05.mma kind::f16 (bf16 in, f32 accumulate) M = 128, N = 256, K = 16, issued
//                  back to back by one thread per CTA on shared-memory operands (zeros) into TMEM,
//                  the same descriptors as the contraction kernel; one CTA per SM.
// Each is timed with CUDA events around one launch after a warm-up launch; results are written to
// sinks so that nothing is optimised away.
#include <cuda_runtime.h>

#include "rp_internal.h"

namespace rp {

__global__ void __launch_bounds__(256) k_probe_dfma(int iters, double seed, double* sink) {
    double a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = seed + i + threadIdx.x;
    const double b = 1.0 - 1e-12, c = 1e-12;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = fma(a[i], b, c);
    }
    double s = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += a[i];
    if (s == 1234.5) sink[threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_probe_dmma(int iters, double seed, double* sink) {
    double acc[4][2];
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[i][0] = acc[i][1] = 0.0;
    const double a = seed + threadIdx.x * 1e-3, b = seed - threadIdx.x * 1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                         : "+d"(acc[i][0]), "+d"(acc[i][1])
                         : "d"(a), "d"(b));
    }
    double s = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) s += acc[i][0] + acc[i][1];
    if (s == 1234.5) sink[threadIdx.x] = s;
}

__device__ __forceinline__ uint64_t probe_desc(uint32_t addr) {
    // K-major, 128B swizzle, 8-row groups 1024 B apart (as the contraction kernel)
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// A: 128 rows x 64 bf16, B: 256 rows x 64 bf16 (zeros), 4 K steps of 16 per pass
__global__ void __launch_bounds__(128, 1) k_probe_bf16(int iters, int* sink) {
    extern __shared__ unsigned char sm_probe[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)sm_probe + 1023) & ~(uintptr_t)1023);
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
    const uint32_t sb = sa + 128 * 128;
    const uint32_t bar = sb + 256 * 128;
    __shared__ uint32_t taddr;
    for (int i = threadIdx.x; i < (128 + 256) * 128 / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(smem)[i] = make_uint4(0, 0, 0, 0);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(
                         (uint32_t)__cvta_generic_to_shared(&taddr)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = taddr;
    // D f32, A bf16, B bf16, K-major, N = 256, M = 128
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(256 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    if (threadIdx.x == 0) {
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const uint64_t da = probe_desc(sa + kk * 32), db = probe_desc(sb + kk * 32);
                const uint32_t acc = (it | kk) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(da), "l"(db), "r"(idesc), "r"(acc));
            }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                     : "memory");
        // bounded wait for the MMAs (they complete in milliseconds; give up after 2 s of global time)
        uint32_t ok = 0;
        uint64_t t0, t1;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
        while (!ok) {
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(ok)
                : "r"(bar)
                : "memory");
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
            if (t1 - t0 > 2000000000ULL) break;
        }
        if (!ok) atomicExch(sink, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (threadIdx.x < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem));
}

int probe_peaks(double* out, int num_sms, cudaStream_t st) {
    double* sink = nullptr;
    if (cudaMalloc(&sink, 4096 * sizeof(double)) != cudaSuccess) return RP_ERR_OOM;
    cudaMemset(sink, 0, 4096 * sizeof(double));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int status = RP_OK;
    auto time_it = [&](auto launch) -> double {
        launch();                                  // warm-up
        cudaEventRecord(e0, st);
        launch();
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms * 1e-3;
    };
    const int blocks = num_sms * 8, threads = 256;
    const int it_f = 1 << 16, it_m = 1 << 14, it_t = 1 << 12;
    double t = time_it([&] { k_probe_dfma<<<blocks, threads, 0, st>>>(it_f, 1.0, sink); });
    out[0] = 2.0 * 8 * it_f * (double)blocks * threads / t / 1e12;
    t = time_it([&] { k_probe_dmma<<<blocks, threads, 0, st>>>(it_m, 1.0, sink); });
    out[1] = 2.0 * 8 * 8 * 4 * 4 * (double)it_m * blocks * (threads / 32) / t / 1e12;
    // more shared memory than two CTAs can share: one CTA per SM, as the rate assumes
    const size_t smem = 120 * 1024;
    if (cudaFuncSetAttribute(k_probe_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess) {
        t = time_it([&] { k_probe_bf16<<<num_sms, 128, smem, st>>>(it_t, (int*)sink); });
        out[2] = 2.0 * 128 * 256 * 16 * 4 * (double)it_t * num_sms / t / 1e12;
    } else {
        out[2] = 0.0;
    }
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaGetLastError();
    int flag = 0;
    if (e == cudaSuccess) cudaMemcpy(&flag, sink, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) status = RP_ERR_CUDA;
    else if (flag) status = RP_ERR_TIMEOUT;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    return status;
}

}  // namespace rp
