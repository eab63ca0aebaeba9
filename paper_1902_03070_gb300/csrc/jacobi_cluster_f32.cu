// Jacobi SVT launches with a slice spread over a thread-block cluster, float slices.
#include "jacobi_cluster.cuh"

namespace tnn {

template <>
cudaError_t launch_jacobi_svt_cluster<float>(const JacobiPlan& p, jac::KArgs<float> a, bool items, cudaStream_t s)
{
    switch (p.L * 1000 + p.RA * 10 + p.K) {
        TNN_JAC_CLUSTER_CASE(float, 16, 12, 4)
        TNN_JAC_CLUSTER_CASE(float, 32, 8, 4)
        TNN_JAC_CLUSTER_CASE(float, 32, 12, 4)
        TNN_JAC_CLUSTER_CASE(float, 32, 16, 4)
    default: return cudaErrorInvalidValue;
    }
}

bool jacobi_cluster_variant_f32(int L, int R, int K)
{
    switch (L * 1000 + R * 10 + K) {
    case 16124:
    case 32084:
    case 32124:
    case 32164:
        return true;
    default: return false;
    }
}

}  // namespace tnn
