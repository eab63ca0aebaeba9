// Batched Jacobi SVT launches (one CTA per SliceItem), float slices.
#include "jacobi_cluster.cuh"
#include "jacobi_launch.cuh"

namespace tnn {

template <>
cudaError_t launch_jacobi_svt_items<float>(const JacobiPlan& plan, const SliceItem* items, int count, int max_sweeps,
                                        void* work, cudaStream_t s)
{
    JacobiPlan p = plan;  // one CTA per item
    p.n3 = count;
    jac::KArgs<float> a{};
    a.items = items;
    a.nb = p.nb; a.ldA = p.ldA; a.n3 = count;
    a.max_sweeps = max_sweeps; a.small_stop = p.small_stop;
    a.work = reinterpret_cast<float*>(work);
    if (p.cluster > 1) return launch_jacobi_svt_cluster<float>(p, a, true, s);
    switch (p.L * 1000 + p.RA * 10 + p.K) {
        TNN_JAC_CASE_I(float, 16, 4)
        TNN_JAC_CASE_I(float, 16, 8)
        TNN_JAC_CASE_I(float, 16, 12)
        TNN_JAC_CASE_I(float, 32, 8)
        TNN_JAC_CASE_I(float, 32, 12)
        TNN_JAC_CASE_I(float, 32, 16)
        TNN_JAC_CASE_I(float, 32, 4)
        TNN_JAC_CASE_I(float, 32, 6)
        TNN_JAC_CASE_KI(float, 16, 12, 2)
        TNN_JAC_CASE_KI(float, 32, 6, 8)
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace tnn
