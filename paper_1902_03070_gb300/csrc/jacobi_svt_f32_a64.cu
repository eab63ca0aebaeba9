// Jacobi SVT launches, float slices in shared memory, with the rotation
// angles and convergence tests in FP64 (TNN_OPT_JACOBI_FP64_ANGLES); a
// translation unit of its own so that it compiles beside the default ones.
#include "jacobi_launch.cuh"

namespace tnn {

cudaError_t launch_jacobi_svt_f32_a64(const JacobiPlan& p, const jac::KArgs<float>& a, cudaStream_t s)
{
    switch (p.L * 1000 + p.RA * 10 + p.K) {
        TNN_JAC_CASE_A64(float, 16, 4)
        TNN_JAC_CASE_A64(float, 16, 8)
        TNN_JAC_CASE_A64(float, 16, 12)
        TNN_JAC_CASE_A64(float, 32, 8)
        TNN_JAC_CASE_A64(float, 32, 12)
        TNN_JAC_CASE_A64(float, 32, 16)
        TNN_JAC_CASE_A64(float, 32, 4)
        TNN_JAC_CASE_A64(float, 32, 6)
        TNN_JAC_CASE_K_A64(float, 16, 12, 2)
        TNN_JAC_CASE_K_A64(float, 32, 6, 8)
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace tnn
