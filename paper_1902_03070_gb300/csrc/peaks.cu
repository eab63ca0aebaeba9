// Throughput of the CUDA-core FMA pipes: the roofline denominators of the
// Jacobi kernels, measured on the device they run on.  Every thread runs
// eight independent FMA chains x <- x b + c (b just below 1, so the chains
// settle at c / (1 - b) and never reach subnormals or overflow); a grid of
// eight 256-thread blocks per SM keeps every scheduler issuing.  The packed
// form issues fma.rn.f32x2 (two FP32 FMAs per instruction).
#include <cuda_runtime.h>

#include <stdint.h>

#include "tnn_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kUnroll = 16;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_chains_kernel(T* out, int iters, T b, T c)
{
    T x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = T(threadIdx.x + i) * T(1e-3);
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int i = 0; i < kChains; ++i) x[i] = fma(x[i], b, c);
    T s = T(0);
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    if (s == T(-1)) out[blockIdx.x * kThreads + threadIdx.x] = s;  // never true; keeps the chains
}

__global__ void __launch_bounds__(kThreads) fma2_chains_kernel(float* out, int iters, float b, float c)
{
    uint64_t x[kChains], bb, cc;
    asm("mov.b64 %0, {%1, %1};" : "=l"(bb) : "f"(b));
    asm("mov.b64 %0, {%1, %1};" : "=l"(cc) : "f"(c));
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
        const float lo = float(threadIdx.x + i) * 1e-3f, hi = lo + 0.5f;
        asm("mov.b64 %0, {%1, %2};" : "=l"(x[i]) : "f"(lo), "f"(hi));
    }
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int i = 0; i < kChains; ++i) asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[i]) : "l"(bb), "l"(cc));
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[i]));
        s += lo + hi;
    }
    if (s == -1.f) out[blockIdx.x * kThreads + threadIdx.x] = s;
}

}  // namespace

extern "C" tnn_status tnn_fma_peak(int32_t device, int32_t kind, double* flops_per_s)
{
    if (!flops_per_s || kind < 0 || kind > 2) return TNN_EINVAL;
    *flops_per_s = 0.0;
    int sms = 0;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        cudaGetLastError();
        return TNN_ECUDA;
    }
    const int blocks = 8 * sms;
    const int iters = kind == 2 ? 64 : 1024;  // FP64 runs at a small fraction of the FP32 rate
    void* out = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    tnn_status st = TNN_ECUDA;
    if (cudaMalloc(&out, (size_t)blocks * kThreads * 8) == cudaSuccess &&
        cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess &&
        cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
        auto launch = [&]() {
            if (kind == 0)
                fma_chains_kernel<float><<<blocks, kThreads, 0, s>>>((float*)out, iters, 0.999999f, 1e-6f);
            else if (kind == 1)
                fma2_chains_kernel<<<blocks, kThreads, 0, s>>>((float*)out, iters, 0.999999f, 1e-6f);
            else
                fma_chains_kernel<double><<<blocks, kThreads, 0, s>>>((double*)out, iters, 0.999999, 1e-6);
        };
        for (int w = 0; w < 3; ++w) launch();
        cudaEventRecord(e0, s);
        const int reps = 10;
        for (int r = 0; r < reps; ++r) launch();
        cudaEventRecord(e1, s);
        float ms = 0.f;
        if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
            ms > 0.f) {
            const double fmas = (double)reps * blocks * kThreads * iters * kUnroll * kChains * (kind == 1 ? 2 : 1);
            *flops_per_s = 2.0 * fmas / (ms * 1e-3);
            st = TNN_OK;
        }
    }
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    if (out) cudaFree(out);
    return st;
}
