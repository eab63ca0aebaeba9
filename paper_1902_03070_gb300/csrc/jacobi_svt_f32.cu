// Jacobi SVT launches, float slices.
#include "jacobi_cluster.cuh"
#include "jacobi_launch.cuh"

namespace tnn {

template <>
cudaError_t launch_jacobi_svt<float>(const JacobiPlan& p, float* data, double tau, const AdmmCtl* ctl, int max_sweeps,
                                   void* work, SliceStats* stats, cudaStream_t s,
                                   const WarmPtrs* warm)
{
    jac::KArgs<float> a{};
    a.data = data; a.n1 = p.n1; a.n2 = p.n2; a.n3 = p.n3;
    a.m = p.m; a.n = p.n; a.tr = p.tr; a.nb = p.nb; a.ldA = p.ldA;
    a.tau = tau; a.ctl = ctl; a.max_sweeps = max_sweeps; a.small_stop = p.small_stop; a.sweep_log = p.sweep_log;
    a.work = reinterpret_cast<float*>(work); a.stats = stats;
    if (warm) {
        a.w0 = static_cast<const float*>(warm->w0);
        a.wflag = warm->wflag;
        a.vrec = static_cast<float*>(warm->vrec);
        a.wrec = warm->wrec;
        a.tail_s = static_cast<float*>(warm->tail_s);
        a.tail_info = warm->tail_info;
    }
    if (p.cluster > 1) return launch_jacobi_svt_cluster<float>(p, a, false, s);
    if (p.angle64 && p.in_smem) return launch_jacobi_svt_f32_a64(p, a, s);
    switch (p.L * 1000 + p.RA * 10 + p.K) {
        TNN_JAC_CASE(float, 16, 4, false)
        TNN_JAC_CASE(float, 16, 8, false)
        TNN_JAC_CASE(float, 16, 12, false)
        TNN_JAC_CASE(float, 32, 8, false)
        TNN_JAC_CASE(float, 32, 12, false)
        TNN_JAC_CASE(float, 32, 16, false)
        TNN_JAC_CASE(float, 32, 4, false)
        TNN_JAC_CASE(float, 32, 6, false)
        TNN_JAC_CASE_K(float, 16, 12, 2, false)
        TNN_JAC_CASE_K(float, 32, 6, 8, false)
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace tnn
