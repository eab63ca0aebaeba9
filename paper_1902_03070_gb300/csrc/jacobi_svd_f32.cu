// Jacobi SVD launches (singular vectors kept), float slices.
#include "jacobi_launch.cuh"

namespace tnn {

template <>
cudaError_t launch_jacobi_svd<float>(const JacobiPlan& p, const float* data, float* U, float* sigma, float* V,
                                   int max_sweeps, void* work, SliceStats* stats, cudaStream_t s)
{
    jac::KArgs<float> a{};
    a.data = const_cast<float*>(data); a.n1 = p.n1; a.n2 = p.n2; a.n3 = p.n3;
    a.m = p.m; a.n = p.n; a.tr = p.tr; a.nb = p.nb; a.ldA = p.ldA;
    a.tau = 0.0; a.ctl = nullptr; a.max_sweeps = max_sweeps; a.small_stop = p.small_stop;
    a.work = reinterpret_cast<float*>(work); a.stats = stats;
    a.U = U; a.S = sigma; a.V = V;
    switch (p.L * 1000 + p.RA * 10 + p.K) {
        TNN_JAC_CASE(float, 32, 2, true)
        TNN_JAC_CASE(float, 32, 4, true)
        TNN_JAC_CASE(float, 32, 6, true)
        TNN_JAC_CASE(float, 32, 8, true)
        TNN_JAC_CASE(float, 32, 12, true)
        TNN_JAC_CASE(float, 32, 16, true)
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace tnn
