// Measured ALU throughput of the device: the denominators for kernels bound by plain
// FP32 FMA or INT32 add issue.  Each thread runs 16 independent dependency chains (no
// memory traffic in the loop) and the grid fills every SM several times over; one
// warm-up launch, then one launch timed with CUDA events.  The packed form runs the
// paired fma.rn.f32x2 that the fp32 dedispersion kernels issue.
#include <cstdint>

#include "dd_internal.h"
#include "dd_packed.cuh"

namespace dd {
namespace {

constexpr int kChains = 16;

__global__ void __launch_bounds__(256) k_fma_peak(float* sink, int iters, float m, float b) {
    float a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = threadIdx.x * 1e-3f + i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = fmaf(a[i], m, b);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += a[i];
    if (s == 1234.5f) sink[0] = s;  // keeps the loop alive
}

// Packed pairs: each chain is one 64-bit register of two fp32 lanes, one fma.rn.f32x2
// (two FMAs) per chain per step.
__global__ void __launch_bounds__(256) k_fma2_peak(float* sink, int iters, float m, float b) {
    uint64_t a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = pk2(threadIdx.x * 1e-3f + i, threadIdx.x * 2e-3f - i);
    const uint64_t mm = pk_dup(m), bb = pk_dup(b);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i)  // a = a * m + b, both lanes
            asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(a[i]) : "l"(a[i]), "l"(mm), "l"(bb));
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
        float lo, hi;
        unpk(a[i], lo, hi);
        s += lo + hi;
    }
    if (s == 1234.5f) sink[0] = s;  // keeps the loop alive
}

__global__ void __launch_bounds__(256) k_iadd_peak(int* sink, int iters, int u, int v) {
    int a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = (int)threadIdx.x + i;
    for (int it = 0; it < iters; ++it) {
        // each chain adds its neighbour's previous value: one three-input add per chain
        // per step, and no closed form the compiler could substitute for the loop
        const int t0 = a[0];
#pragma unroll
        for (int i = 0; i < kChains - 1; ++i) a[i] = a[i] + a[i + 1] + u;
        a[kChains - 1] = a[kChains - 1] + t0 + v;
    }
    int s = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s ^= a[i];
    if (s == 0x7fffabcd) sink[0] = s;
}

}  // namespace
}  // namespace dd

extern "C" dd_status dd_alu_peak(int32_t kind, double* ops_per_s, void* stream) {
    if (!ops_per_s || kind < 0 || kind > 2) return DD_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return dd::cuda_status(e);
    void* sink = nullptr;
    e = cudaMalloc(&sink, 16);
    if (e != cudaSuccess) return dd::cuda_status(e);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int blocks = sms * 8, threads = 256, iters = 20000;
    float ms = 0.f;
    if (e == cudaSuccess) {
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
            cudaEventRecord(e0, s);
            if (kind == 0)
                dd::k_fma_peak<<<blocks, threads, 0, s>>>((float*)sink, rep ? iters : 200, 1.0000001f, 1e-7f);
            else if (kind == 2)
                dd::k_fma2_peak<<<blocks, threads, 0, s>>>((float*)sink, rep ? iters : 200, 1.0000001f, 1e-7f);
            else
                dd::k_iadd_peak<<<blocks, threads, 0, s>>>((int*)sink, rep ? iters : 200, 3, 5);
            cudaEventRecord(e1, s);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        }
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess) return dd::cuda_status(e);
    // FP32: 2 flops per FMA (two FMAs per packed instruction); INT32: 2 additions per
    // three-input add
    const double ops = (kind == 2 ? 4.0 : 2.0) * dd::kChains * (double)iters * blocks * threads;
    *ops_per_s = ops / (ms * 1e-3);
    return DD_OK;
}
