// Batched Jacobi SVT launches (one CTA per SliceItem), double slices.
#include "jacobi_cluster.cuh"
#include "jacobi_launch.cuh"

namespace tnn {

template <>
cudaError_t launch_jacobi_svt_items<double>(const JacobiPlan& plan, const SliceItem* items, int count, int max_sweeps,
                                        void* work, cudaStream_t s)
{
    JacobiPlan p = plan;  // one CTA per item
    p.n3 = count;
    jac::KArgs<double> a{};
    a.items = items;
    a.nb = p.nb; a.ldA = p.ldA; a.n3 = count;
    a.max_sweeps = max_sweeps; a.small_stop = p.small_stop;
    a.work = reinterpret_cast<double*>(work);
    if (p.cluster > 1) return launch_jacobi_svt_cluster<double>(p, a, true, s);
    switch (p.L * 1000 + p.RA * 10 + p.K) {
        TNN_JAC_CASE_I(double, 16, 2)
        TNN_JAC_CASE_I(double, 16, 4)
        TNN_JAC_CASE_I(double, 16, 6)
        TNN_JAC_CASE_I(double, 32, 4)
        TNN_JAC_CASE_I(double, 32, 6)
        TNN_JAC_CASE_I(double, 32, 8)
        TNN_JAC_CASE_I(double, 32, 16)
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace tnn
