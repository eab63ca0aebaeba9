// Warm start of the per-slice Jacobi SVT across ADMM iterations.
//
// One-sided Jacobi on A0 Q, Q orthogonal, has the singular values and left
// singular vectors of A0, so the SVT of Algorithm 1 (rebuilt from A0 itself)
// does not depend on Q; but with Q the previous iteration's right singular
// vectors, A0 Q already has nearly orthogonal columns and the sweeps drop
// from 10-19 to a few in the late iterations of a completion, where the
// slices change little from one iteration to the next.
//
// Per iteration and slice k (FP32; slices held by one CTA):
//   warm_gemm_kernel: W0_k = A0_k Q_k (A0 oriented as the Jacobi kernel
//     orients it; W0 in its working-copy layout, padded with zeros) for the
//     slices whose Q is valid;
//   the Jacobi kernel starts from W0_k and, after its sweeps, writes
//     V_k = A0^T s_c / sigma_c (columns by descending sigma) over W0_k;
//   warm_qr_kernel: Q_k = the orthogonal factor of a Householder QR of V_k
//     (the reliable columns, those of the large singular values, first: Q's
//     leading columns are theirs).  Q is a product of reflectors, orthogonal
//     to rounding whatever V_k is, so a poor V only costs sweeps.
// The state is Q (n x n per slice) followed by one int flag per slice
// (0: no Q yet, start from A0); a zero-filled state is a cold start.
#include <cuda_runtime.h>

#include "tnn_internal.h"

namespace tnn {
namespace {

constexpr int WT = 256;   // threads per CTA of the QR
constexpr int WTG = 384;  // threads per CTA of the GEMM (12 warps)
constexpr int WCB = 6;    // output columns per warp pass of the GEMM
constexpr int WMR = 8;    // most rows per lane of the GEMM (m <= 256)
constexpr int WQR = 7;    // rows per lane of a Q column (n <= 224)

template <typename T, int MR>
__global__ void __launch_bounds__(WTG) warm_gemm_kernel(const T* __restrict__ data, int64_t n1, int64_t n2, int m,
                                                      int n, int tr, int ldA, int npad, size_t stride,
                                                      const T* __restrict__ Q, const int* __restrict__ flag,
                                                      T* __restrict__ w0, const AdmmCtl* __restrict__ ctl)
{
    if (ctl && ctl->done) return;
    const int k = blockIdx.x;
    if (!flag[k]) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* As = reinterpret_cast<T*>(smem_raw);  // oriented slice, column j at As + j * m
    T* Qs = As + (size_t)m * n;              // Q_k, column c at Qs + c * n
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, W = WTG / 32;
    const T* src = data + (size_t)k * n1 * n2;
    const int64_t S = n1 * n2;
    for (int64_t e = tid; e < S; e += WTG) {
        const int i = (int)(e % n1), j = (int)(e / n1);
        const int r = tr ? j : i, c = tr ? i : j;
        As[(size_t)c * m + r] = src[e];
    }
    const T* Qk = Q + (size_t)k * n * n;
    for (int e = tid; e < n * n; e += WTG) Qs[e] = Qk[e];
    __syncthreads();
    T* out = w0 + (size_t)k * stride;
    for (int c0 = warp * WCB; c0 < npad; c0 += W * WCB) {
        T acc[MR][WCB];
#pragma unroll
        for (int q = 0; q < MR; ++q)
#pragma unroll
            for (int b = 0; b < WCB; ++b) acc[q][b] = T(0);
#pragma unroll 4
        for (int j = 0; j < n; ++j) {
            T av[MR], qv[WCB];
#pragma unroll
            for (int q = 0; q < MR; ++q) {
                const int r = q * 32 + lane;
                av[q] = r < m ? As[(size_t)j * m + r] : T(0);
            }
#pragma unroll
            for (int b = 0; b < WCB; ++b) qv[b] = (c0 + b < n) ? Qs[(size_t)(c0 + b) * n + j] : T(0);
#pragma unroll
            for (int q = 0; q < MR; ++q)
#pragma unroll
                for (int b = 0; b < WCB; ++b) acc[q][b] = fma(av[q], qv[b], acc[q][b]);
        }
#pragma unroll
        for (int b = 0; b < WCB; ++b) {
            const int c = c0 + b;
            if (c >= npad) break;
            T* col = out + (size_t)c * ldA;
#pragma unroll
            for (int q = 0; q < MR; ++q) {
                const int r = q * 32 + lane;
                if (r < ldA) col[r] = (r < m && c < n) ? acc[q][b] : T(0);
            }
            for (int r = MR * 32 + lane; r < ldA; r += 32) col[r] = T(0);
        }
    }
}

// Reflector of column c (rows c..n-1, norm^2 s2 given): alpha = -sign(x_c)
// |x|, v = x - alpha e_c stored over x (only x_c changes), beta = 2 / |v|^2
// (0, H = I, for a zero column).
template <typename T>
__device__ __forceinline__ void make_reflector(T* x, int c, T s2, T* bet)
{
    const T x0 = x[c];
    const T nx = sqrt(s2);
    const T alpha = x0 >= T(0) ? -nx : nx;
    x[c] = x0 - alpha;
    const T vn2 = T(2) * nx * (nx + fabs(x0));  // |x - alpha e_c|^2, no cancellation
    bet[c] = vn2 > T(0) ? T(2) / vn2 : T(0);
}

template <typename T>
__global__ void __launch_bounds__(WT) warm_qr_kernel(T* __restrict__ vrec, int n, size_t stride, int* __restrict__ wrec,
                                                    T* __restrict__ Q, int* __restrict__ flag,
                                                    const AdmmCtl* __restrict__ ctl)
{
    if (ctl && ctl->done) return;
    const int k = blockIdx.x;
    if (!wrec[k]) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* Vs = reinterpret_cast<T*>(smem_raw);  // n x n, column c at Vs + c * n; Householder vectors below the diagonal
    T* bet = Vs + (size_t)n * n;             // beta of each reflector
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, W = WT / 32;
    const T* V = vrec + (size_t)k * stride;
    for (int e = tid; e < n * n; e += WT) Vs[e] = V[e];
    __syncthreads();
    // Householder QR, one barrier per column: in step c every warp applies
    // reflector c to its columns j > c (column j belongs to warp j mod W,
    // four columns at a time so that four reductions overlap), and the warp
    // holding column c + 1 then forms reflector c + 1 from it
    if (warp == 0) {
        T s2 = T(0);
        for (int r = lane; r < n; r += 32) s2 = fma(Vs[r], Vs[r], s2);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        if (lane == 0) make_reflector(Vs, 0, s2, bet);
    }
    __syncthreads();
    for (int c = 0; c < n; ++c) {
        const T b = bet[c];
        const T* x = Vs + (size_t)c * n;
        T xv[WQR];
#pragma unroll
        for (int i = 0; i < WQR; ++i) {
            const int r = i * 32 + lane;
            xv[i] = (r >= c && r < n) ? x[r] : T(0);
        }
        // this warp's columns j > c: j = j0 + W q, j0 the first of them
        const int j0 = c + 1 + ((warp - (c + 1)) % W + W) % W;
        for (int jb = j0; jb < n; jb += 4 * W) {
            T* y[4];
            T yv[4][WQR];
            T d[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = jb + u * W;
                y[u] = Vs + (size_t)(j < n ? j : c) * n;
                d[u] = T(0);
#pragma unroll
                for (int i = 0; i < WQR; ++i) {
                    const int r = i * 32 + lane;
                    yv[u][i] = (j < n && r < n) ? y[u][r] : T(0);
                    d[u] = fma(xv[i], yv[u][i], d[u]);
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                for (int u = 0; u < 4; ++u) d[u] += __shfl_xor_sync(0xffffffffu, d[u], o);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = jb + u * W;
                if (j >= n) continue;
                const T f = b * d[u];
                T s2 = T(0);
#pragma unroll
                for (int i = 0; i < WQR; ++i) {
                    const int r = i * 32 + lane;
                    const T v = fma(-f, xv[i], yv[u][i]);
                    if (r >= c && r < n) y[u][r] = v;
                    if (j == c + 1 && r >= c + 1 && r < n) s2 = fma(v, v, s2);
                }
                if (j == c + 1) {  // the next reflector, from the column just updated
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
                    __syncwarp();
                    if (lane == 0) make_reflector(y[u], c + 1, s2, bet);
                }
            }
        }
        __syncthreads();
    }
    // Q = H_0 H_1 ... H_{n-1}; its column j is H_0 ... H_j e_j (the later
    // reflectors leave e_j alone).  Each warp takes four consecutive columns
    // at a time (in registers, row r = 32 i + lane) and applies reflectors
    // from the group's last column down to 0 (a reflector past a column's
    // own leaves it unchanged).
    T* Qk = Q + (size_t)k * n * n;
    for (int g0 = warp * 4; g0 < n; g0 += 4 * W) {
        T qv[4][WQR];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int i = 0; i < WQR; ++i) qv[u][i] = (i * 32 + lane == g0 + u) ? T(1) : T(0);
        const int cmax = g0 + 3 < n - 1 ? g0 + 3 : n - 1;
        for (int c = cmax; c >= 0; --c) {
            const T b = bet[c];
            if (b == T(0)) continue;
            const T* x = Vs + (size_t)c * n;
            T xv[WQR];
            T d[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
            for (int i = 0; i < WQR; ++i) {
                const int r = i * 32 + lane;
                xv[i] = (r >= c && r < n) ? x[r] : T(0);
#pragma unroll
                for (int u = 0; u < 4; ++u) d[u] = fma(xv[i], qv[u][i], d[u]);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                for (int u = 0; u < 4; ++u) d[u] += __shfl_xor_sync(0xffffffffu, d[u], o);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const T f = b * d[u];
#pragma unroll
                for (int i = 0; i < WQR; ++i) qv[u][i] = fma(-f, xv[i], qv[u][i]);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (g0 + u >= n) break;
            T* qc = Qk + (size_t)(g0 + u) * n;
#pragma unroll
            for (int i = 0; i < WQR; ++i) {
                const int r = i * 32 + lane;
                if (r < n) qc[r] = qv[u][i];
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        flag[k] = 1;
        wrec[k] = 0;
    }
}

}  // namespace

size_t warm_gemm_smem(int m, int n, int elem) { return ((size_t)m * n + (size_t)n * n) * elem; }
size_t warm_qr_smem(int n, int elem) { return ((size_t)n * n + n) * elem; }

bool warm_supported(const JacobiPlan& p)
{
    return p.cluster <= 1 && p.elem == 4 && p.m <= WMR * 32 && p.n <= WQR * 32 &&
           warm_gemm_smem(p.m, p.n, p.elem) <= 200 * 1024 &&
           warm_qr_smem(p.n, p.elem) <= 200 * 1024;
}

size_t warm_state_bytes(int64_t n3, int n, int elem)
{
    return ((size_t)n3 * n * n * elem + 255) / 256 * 256 + ((size_t)n3 * sizeof(int) + 255) / 256 * 256;
}

template <typename T>
cudaError_t launch_warm_gemm(const JacobiPlan& p, const T* data, const T* Q, const int* flag, T* w0,
                             const AdmmCtl* ctl, cudaStream_t s)
{
    const size_t sm = warm_gemm_smem(p.m, p.n, sizeof(T));
    auto kern = p.m <= 192 ? warm_gemm_kernel<T, 6> : warm_gemm_kernel<T, WMR>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const size_t stride = (size_t)p.ldA * p.nb * p.K;
    kern<<<(unsigned)p.n3, WTG, sm, s>>>(data, p.n1, p.n2, p.m, p.n, p.tr, p.ldA, p.nb * p.K, stride, Q, flag, w0, ctl);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_warm_qr(const JacobiPlan& p, T* vrec, int* wrec, T* Q, int* flag, const AdmmCtl* ctl, cudaStream_t s)
{
    const size_t sm = warm_qr_smem(p.n, sizeof(T));
    auto kern = warm_qr_kernel<T>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const size_t stride = (size_t)p.ldA * p.nb * p.K;
    kern<<<(unsigned)p.n3, WT, sm, s>>>(vrec, p.n, stride, wrec, Q, flag, ctl);
    return cudaGetLastError();
}

template cudaError_t launch_warm_gemm<float>(const JacobiPlan&, const float*, const float*, const int*, float*,
                                             const AdmmCtl*, cudaStream_t);
template cudaError_t launch_warm_qr<float>(const JacobiPlan&, float*, int*, float*, int*, const AdmmCtl*,
                                           cudaStream_t);

}  // namespace tnn
