// tsvt_dct_static: the t-SVT of tsvt_dct for callers that cannot allocate
// device memory (the paper has no counterpart).  Some callers have no allocation available at the moment
// they need a t-SVT: a serving loop that runs under a fixed device-memory
// budget owned by another allocator (a surprise cudaMalloc could fail or
// fragment that pool), code that must not create a context and workspace of
// its own, or a host thread that may not block on the allocator's implicit
// device synchronisation.  This entry point uses no context and calls no
// cudaMalloc, cudaFree or other allocating routine: its scratch (the two DCT
// operators, the transformed tensor, per-slice statistics, status counters
// and, for slices too large for shared memory, the Jacobi working copies)
// lives in one file-scope device array of TNN_STATIC_SCRATCH_BYTES, which
// every GPU that loads the library keeps until the process exits.  It runs
// the kernels tsvt_dct runs for the same precision (the tensor-core
// transforms for 3xTF32 and BF16 split) and, like tsvt_dct with a tnn_out,
// waits for them to report a sweep cap or a non-finite value.
#include <cuda_runtime.h>

#include <mutex>

#include "tnn_internal.h"

namespace {

constexpr size_t kScratchBytes = TNN_STATIC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

// The scratch array.  In host code its name is only a host-side stand-in;
// the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// Device address of g_scratch on the current device (looked up once per
// device, with that device current).
tnn_status scratch_address(void** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return TNN_ENODEV;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return TNN_ECUDA;
        }
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return TNN_OK;
}

// A pointer the kernels may use: device memory of the current device, or
// managed memory.
bool on_current_device(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    if (a.type != cudaMemoryTypeDevice) return false;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.device == dev;
}

// Folds the per-slice statistics into two counters at the front of the
// scratch: slices that hit the sweep cap and slices that met a non-finite
// value (one thread; n3 is small).
__global__ void summarise_stats(const tnn::SliceStats* st, int64_t n3, int* out)
{
    int unconv = 0, nonfin = 0;
    for (int64_t k = 0; k < n3; ++k) {
        unconv += st[k].converged ? 0 : 1;
        nonfin += st[k].nonfinite ? 1 : 0;
    }
    out[0] = unconv;
    out[1] = nonfin;
}

template <typename T>
tnn_status run(const T* Z, const tnn_shape& sh, double tau, tnn_precision prec, T* Y, cudaStream_t s)
{
    using namespace tnn;
    // sizes are checked against the scratch before any product that could wrap
    const size_t cap = kScratchBytes / sizeof(T);
    if ((size_t)sh.n3 > cap || (size_t)sh.n1 > cap || (size_t)sh.n2 > cap) return TNN_EINVAL;
    if ((size_t)sh.n1 > cap / (size_t)sh.n2) return TNN_EINVAL;
    if ((size_t)sh.n3 > cap / ((size_t)sh.n1 * (size_t)sh.n2)) return TNN_EINVAL;
    JacobiPlan jp;
    if (!jacobi_plan(sh.n1, sh.n2, sh.n3, (int)sizeof(T), &jp)) return TNN_EINVAL;
    const size_t N = (size_t)sh.n1 * sh.n2 * sh.n3;
    // the tensor-core forms of tsvt_dct (3xTF32, BF16 split) where it uses them
    const bool tc = sizeof(T) == 4 && (prec == TNN_FP32_TF32X3 || prec == TNN_FP32_BF16SPLIT) &&
                    tube_tc_supported(sh.n3);
    const bool bf = prec == TNN_FP32_BF16SPLIT;
    const size_t b_hdr = 256;  // status counters and the tensor-core timeout flag
    const size_t b_op = tc ? up256(tube_tc_image_floats(sh.n3, bf) * sizeof(float))
                           : up256((size_t)sh.n3 * sh.n3 * sizeof(T));
    const size_t b_st = up256(sizeof(SliceStats) * (size_t)sh.n3);
    const size_t b_w = up256(N * sizeof(T));
    const size_t b_j = up256(jp.work_bytes);
    if (b_j > kScratchBytes || b_hdr + 2 * b_op + b_st + b_w + b_j > kScratchBytes) return TNN_EINVAL;
    void* base = nullptr;
    tnn_status st = scratch_address(&base);
    if (st != TNN_OK) return st;
    char* c = static_cast<char*>(base);
    int* counters = reinterpret_cast<int*>(c);   // [0] sweep-cap slices, [1] non-finite slices, [2] timeout flag
    char* opf = c + b_hdr;
    char* opi = opf + b_op;
    SliceStats* stats = reinterpret_cast<SliceStats*>(opi + b_op);
    T* W = reinterpret_cast<T*>(opi + b_op + b_st);
    void* jw = opi + b_op + b_st + b_w;
    // Every scratch byte read below is written first in the same call (the
    // flag cleared, the operators, the transformed tensor, the statistics),
    // so nothing left by an earlier call is used.
    if (cudaMemsetAsync(counters, 0, 3 * sizeof(int), s) != cudaSuccess) return TNN_ECUDA;
    const int64_t P = sh.n1 * sh.n2;
    if (tc) {
        if (launch_build_operator_tc((float*)opf, sh.n3, 0, 0, bf, s) != cudaSuccess) return TNN_ECUDA;
        if (launch_build_operator_tc((float*)opi, sh.n3, 1, 0, bf, s) != cudaSuccess) return TNN_ECUDA;
        if (launch_tube_tc((const float*)Z, (float*)W, (const float*)opf, P, sh.n3, bf, counters + 2, s) !=
            cudaSuccess)
            return TNN_ECUDA;
    } else {
        if (launch_build_operator<T>((T*)opf, sh.n3, 0, 0, s) != cudaSuccess) return TNN_ECUDA;
        if (launch_build_operator<T>((T*)opi, sh.n3, 1, 0, s) != cudaSuccess) return TNN_ECUDA;
        if (launch_tube_op<T>(Z, W, (const T*)opf, P, sh.n3, s) != cudaSuccess) return TNN_ECUDA;
    }
    if (launch_jacobi_svt<T>(jp, W, tau, nullptr, 0, jw, stats, s) != cudaSuccess) return TNN_ECUDA;
    if (tc) {
        if (launch_tube_tc((const float*)W, (float*)Y, (const float*)opi, P, sh.n3, bf, counters + 2, s) !=
            cudaSuccess)
            return TNN_ECUDA;
    } else if (launch_tube_op<T>(W, Y, (const T*)opi, P, sh.n3, s) != cudaSuccess) {
        return TNN_ECUDA;
    }
    summarise_stats<<<1, 1, 0, s>>>(stats, sh.n3, counters);
    if (cudaGetLastError() != cudaSuccess) return TNN_ECUDA;
    // the status comes back through a host variable (no allocation)
    int h[3] = {0, 0, 0};
    if (cudaMemcpyAsync(h, counters, sizeof h, cudaMemcpyDeviceToHost, s) != cudaSuccess) return TNN_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return TNN_ECUDA;
    if (h[2]) return TNN_ECUDA;
    if (h[1]) return TNN_ENONFINITE;
    if (h[0]) return TNN_ENOCONV;
    return TNN_OK;
}

}  // namespace

extern "C" tnn_status tsvt_dct_static(const void* Z, tnn_shape sh, double tau, tnn_precision prec, void* Y,
                                      void* stream)
{
    if (!Z || !Y || sh.n1 <= 0 || sh.n2 <= 0 || sh.n3 <= 0 || !(tau >= 0.0) || !(tau < 1e300)) return TNN_EINVAL;
    if (!(prec == TNN_FP64 || prec == TNN_FP32 || prec == TNN_FP32_TF32X3 || prec == TNN_FP32_BF16SPLIT))
        return TNN_EINVAL;
    if (!on_current_device(Z) || !on_current_device(Y)) return TNN_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (prec == TNN_FP64) return run<double>((const double*)Z, sh, tau, prec, (double*)Y, s);
    return run<float>((const float*)Z, sh, tau, prec, (float*)Y, s);
}
