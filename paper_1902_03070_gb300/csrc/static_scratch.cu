// tsvt_dct_static: the t-SVT of tsvt_dct for callers that cannot allocate
// device memory.  Some callers have no allocation available at the moment
// they need a t-SVT: a serving loop that runs under a fixed device-memory
// budget owned by another allocator (a surprise cudaMalloc could fail or
// fragment that pool), code that must not create a context and workspace of
// its own, or a host thread that may not block on the allocator's implicit
// device synchronisation.  This entry point uses no context and calls no
// cudaMalloc, cudaFree or other allocating routine: its scratch (the two DCT
// operators, the transformed tensor, per-slice statistics and, for slices too
// large for shared memory, the Jacobi working copies) lives in one file-scope
// device array of TNN_STATIC_SCRATCH_BYTES, which every GPU that loads the
// library keeps until the process exits.
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

bool on_device(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <typename T>
tnn_status run(const T* Z, const tnn_shape& sh, double tau, T* Y, cudaStream_t s)
{
    using namespace tnn;
    JacobiPlan jp;
    if (!jacobi_plan(sh.n1, sh.n2, sh.n3, (int)sizeof(T), &jp)) return TNN_EINVAL;
    const size_t N = (size_t)sh.n1 * sh.n2 * sh.n3;
    const size_t b_op = up256((size_t)sh.n3 * sh.n3 * sizeof(T));
    const size_t b_st = up256(sizeof(SliceStats) * (size_t)sh.n3);
    const size_t b_w = up256(N * sizeof(T));
    const size_t b_j = up256(jp.work_bytes);
    if (2 * b_op + b_st + b_w + b_j > kScratchBytes) return TNN_EINVAL;  // beyond the static scratch
    void* base = nullptr;
    tnn_status st = scratch_address(&base);
    if (st != TNN_OK) return st;
    char* c = static_cast<char*>(base);
    T* opf = reinterpret_cast<T*>(c);
    T* opi = reinterpret_cast<T*>(c + b_op);
    SliceStats* stats = reinterpret_cast<SliceStats*>(c + 2 * b_op);
    T* W = reinterpret_cast<T*>(c + 2 * b_op + b_st);
    void* jw = c + 2 * b_op + b_st + b_w;
    // Every scratch byte read below is written first in the same call (the
    // operators, the transformed tensor, the statistics), so nothing left by
    // an earlier call is used and nothing needs clearing.
    if (launch_build_operator<T>(opf, sh.n3, 0, 0, s) != cudaSuccess) return TNN_ECUDA;
    if (launch_build_operator<T>(opi, sh.n3, 1, 0, s) != cudaSuccess) return TNN_ECUDA;
    const int64_t P = sh.n1 * sh.n2;
    if (launch_tube_op<T>(Z, W, opf, P, sh.n3, s) != cudaSuccess) return TNN_ECUDA;
    if (launch_jacobi_svt<T>(jp, W, tau, nullptr, 0, jw, stats, s) != cudaSuccess) return TNN_ECUDA;
    if (launch_tube_op<T>(W, Y, opi, P, sh.n3, s) != cudaSuccess) return TNN_ECUDA;
    return TNN_OK;
}

}  // namespace

extern "C" tnn_status tsvt_dct_static(const void* Z, tnn_shape sh, double tau, tnn_precision prec, void* Y,
                                      void* stream)
{
    if (!Z || !Y || sh.n1 <= 0 || sh.n2 <= 0 || sh.n3 <= 0 || !(tau >= 0.0) || !(tau < 1e300)) return TNN_EINVAL;
    if (!(prec == TNN_FP64 || prec == TNN_FP32 || prec == TNN_FP32_TF32X3 || prec == TNN_FP32_BF16SPLIT))
        return TNN_EINVAL;
    if (!on_device(Z) || !on_device(Y)) return TNN_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (prec == TNN_FP64) return run<double>((const double*)Z, sh, tau, (double*)Y, s);
    return run<float>((const float*)Z, sh, tau, (float*)Y, s);
}
