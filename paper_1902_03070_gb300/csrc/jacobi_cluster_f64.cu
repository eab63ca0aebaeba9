// Jacobi SVT launches with a slice spread over a thread-block cluster, double slices.
#include "jacobi_cluster.cuh"

namespace tnn {

template <>
cudaError_t launch_jacobi_svt_cluster<double>(const JacobiPlan& p, jac::KArgs<double> a, bool items, cudaStream_t s)
{
    switch (p.L * 1000 + p.RA * 10 + p.K) {
        TNN_JAC_CLUSTER_CASE(double, 32, 6, 4)
        TNN_JAC_CLUSTER_CASE(double, 32, 8, 4)
        TNN_JAC_CLUSTER_CASE(double, 32, 16, 2)
    default: return cudaErrorInvalidValue;
    }
}

bool jacobi_cluster_variant_f64(int L, int R, int K)
{
    switch (L * 1000 + R * 10 + K) {
    case 32064:
    case 32084:
    case 32162:
        return true;
    default: return false;
    }
}

}  // namespace tnn
