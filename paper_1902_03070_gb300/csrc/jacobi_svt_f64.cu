// Jacobi SVT launches, double slices.
#include "jacobi_cluster.cuh"
#include "jacobi_launch.cuh"

namespace tnn {

template <>
cudaError_t launch_jacobi_svt<double>(const JacobiPlan& p, double* data, double tau, const AdmmCtl* ctl, int max_sweeps,
                                   void* work, SliceStats* stats, cudaStream_t s,
                                   const WarmPtrs* warm)
{
    jac::KArgs<double> a{};
    a.data = data; a.n1 = p.n1; a.n2 = p.n2; a.n3 = p.n3;
    a.m = p.m; a.n = p.n; a.tr = p.tr; a.nb = p.nb; a.ldA = p.ldA;
    a.tau = tau; a.ctl = ctl; a.max_sweeps = max_sweeps; a.small_stop = p.small_stop; a.sweep_log = p.sweep_log;
    a.work = reinterpret_cast<double*>(work); a.stats = stats;
    if (p.cluster > 1) return launch_jacobi_svt_cluster<double>(p, a, false, s);
    switch (p.L * 1000 + p.RA * 10 + p.K) {
        TNN_JAC_CASE(double, 16, 2, false)
        TNN_JAC_CASE(double, 16, 4, false)
        TNN_JAC_CASE(double, 16, 6, false)
        TNN_JAC_CASE(double, 32, 4, false)
        TNN_JAC_CASE(double, 32, 6, false)
        TNN_JAC_CASE(double, 32, 8, false)
        TNN_JAC_CASE(double, 32, 16, false)
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace tnn
