// Launch plumbing for the Jacobi kernels: block width K, rows per lane R and
// lanes per block pair L are compile-time; a plan picks them from the shape.
#pragma once

#include "jacobi.cuh"

namespace tnn {
namespace jac {

// K for a given element type, rows per lane and mode (register budget: 2K
// columns of R rows, twice that with V).
__host__ __device__ constexpr int pick_K(int elem, int R, bool withv)
{
    return elem == 4 ? (withv ? (R <= 8 ? 4 : 2) : 4) : (withv ? (R <= 4 ? 4 : 2) : (R <= 8 ? 4 : 2));
}

// A64: the FP64-angle instantiation (FP32 SVT, slice in shared memory; the
// plan must have in_smem set).
template <typename T, int K, int R, int L, bool WITHV, bool ITEMS = false, bool A64 = false>
cudaError_t launch_one(const JacobiPlan& p, KArgs<T> a, cudaStream_t s)
{
    void (*kern)(KArgs<T>);
    if constexpr (A64) kern = jacobi_kernel<T, K, R, L, true, false, false, true>;
    else kern = p.in_smem ? jacobi_kernel<T, K, R, L, true, WITHV, ITEMS> : jacobi_kernel<T, K, R, L, false, WITHV, ITEMS>;
    cudaFuncAttributes attr;
    cudaError_t e = cudaFuncGetAttributes(&attr, kern);
    if (e != cudaSuccess) return e;
    const int wmax = attr.maxThreadsPerBlock / 32;
    const int gpw = 32 / L;
    int W = (p.nb / 2 + gpw - 1) / gpw;  // one block pair per group
    if (W > wmax) W = wmax;
    if (W < 1) W = 1;
    const int npad = p.nb * K;
    size_t wsz = (size_t)p.ldA * npad * sizeof(T);
    size_t big = p.in_smem ? (WITHV ? 2 : 1) * ((wsz + 255) & ~(size_t)255) : 0;
    size_t smem = big + smem_small_bytes(npad, W, (int)sizeof(T));
    if (smem > 48 * 1024) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<(unsigned)p.n3, W * 32, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace jac
}  // namespace tnn

// One supported (L, R, K) variant of a (T, WITHV) family; the plan's key is
// L * 1000 + R * 10 + K.
#define TNN_JAC_CASE(T, L, R, WITHV) \
    case L * 1000 + R * 10 + jac::pick_K((int)sizeof(T), R, WITHV): \
        return jac::launch_one<T, jac::pick_K((int)sizeof(T), R, WITHV), R, L, WITHV>(p, a, s);
#define TNN_JAC_CASE_K(T, L, R, K, WITHV) \
    case L * 1000 + R * 10 + K:           \
        return jac::launch_one<T, K, R, L, WITHV>(p, a, s);
// The FP64-angle SVT kernels (FP32, slice in shared memory).
#define TNN_JAC_CASE_A64(T, L, R) \
    case L * 1000 + R * 10 + jac::pick_K((int)sizeof(T), R, false): \
        return jac::launch_one<T, jac::pick_K((int)sizeof(T), R, false), R, L, false, false, true>(p, a, s);
#define TNN_JAC_CASE_K_A64(T, L, R, K) \
    case L * 1000 + R * 10 + K:         \
        return jac::launch_one<T, K, R, L, false, false, true>(p, a, s);
namespace tnn {
// FP32 SVT with FP64 rotation angles (jacobi_svt_f32_a64.cu), for plans with
// angle64 and in_smem set.
cudaError_t launch_jacobi_svt_f32_a64(const JacobiPlan& p, const jac::KArgs<float>& a, cudaStream_t s);
}  // namespace tnn
// The same for the batched (item-table) SVT kernels.
#define TNN_JAC_CASE_I(T, L, R) \
    case L * 1000 + R * 10 + jac::pick_K((int)sizeof(T), R, false): \
        return jac::launch_one<T, jac::pick_K((int)sizeof(T), R, false), R, L, false, true>(p, a, s);
#define TNN_JAC_CASE_KI(T, L, R, K) \
    case L * 1000 + R * 10 + K:     \
        return jac::launch_one<T, K, R, L, false, true>(p, a, s);
