// Launch plumbing for the Jacobi kernels: the block width K and rows per lane
// RA are compile-time; a plan picks them from the slice shape.
#pragma once

#include "jacobi.cuh"

namespace tnn {
namespace jac {

// K for a given element type, RA and mode (register budget: 2K columns of
// RA rows, twice that with V).
__host__ __device__ constexpr int pick_K(int elem, int RA, bool withv)
{
    return elem == 4 ? (withv ? (RA <= 8 ? 4 : 2) : 4) : (RA <= 4 ? 4 : 2);
}

template <typename T, int K, int RA, bool WITHV>
cudaError_t launch_one(const JacobiPlan& p, KArgs<T> a, cudaStream_t s)
{
    void (*kern)(KArgs<T>) = p.in_smem ? jacobi_kernel<T, K, RA, true, WITHV> : jacobi_kernel<T, K, RA, false, WITHV>;
    cudaFuncAttributes attr;
    cudaError_t e = cudaFuncGetAttributes(&attr, kern);
    if (e != cudaSuccess) return e;
    int wmax = attr.maxThreadsPerBlock / 32;
    int W = p.nb / 2;
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

// Switch over the supported RA values for one (T, WITHV) family.
#define TNN_JAC_CASE(T, RA, WITHV)                                                              \
    case RA:                                                                                    \
        return jac::launch_one<T, jac::pick_K((int)sizeof(T), RA, WITHV), RA, WITHV>(p, a, s);
