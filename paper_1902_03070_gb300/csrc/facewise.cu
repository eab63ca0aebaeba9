// Facewise (per frontal slice) matrix products in the transform domain, the
// core of the t-product of Eq. 14 and of the t-SVD recomposition (Theorem 4).
// C_k = op(A_k) diag(dscale_k) op(B_k), a batched SIMT GEMM: 64 x 64 output
// tile per CTA, 4 x 4 per thread, operands staged in shared memory.
#include <cuda_runtime.h>
#include <stdint.h>

#include "tnn_internal.h"

namespace tnn {
namespace {

constexpr int TM = 64, TN = 64, TK = 16;

template <typename T>
__global__ void __launch_bounds__(256)
facewise_kernel(const T* __restrict__ A, const T* __restrict__ B, T* __restrict__ C, int64_t m, int64_t n, int64_t kk,
                int transA, int transB, const T* __restrict__ dscale)
{
    __shared__ T As[TK][TM];
    __shared__ T Bs[TK][TN];
    const int64_t bz = blockIdx.z;
    const T* Ak = A + bz * m * kk;
    const T* Bk = B + bz * kk * n;
    T* Ck = C + bz * m * n;
    const T* dk = dscale ? dscale + bz * kk : nullptr;
    const int tid = threadIdx.x;
    const int ti = tid & 15, tj = tid >> 4;
    const int64_t i0 = (int64_t)blockIdx.x * TM, j0 = (int64_t)blockIdx.y * TN;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
    for (int64_t l0 = 0; l0 < kk; l0 += TK) {
        __syncthreads();
        for (int e = tid; e < TK * TM; e += 256) {
            int ll = e / TM, ii = e % TM;
            int64_t i = i0 + ii, l = l0 + ll;
            T v = T(0);
            if (i < m && l < kk) {
                v = transA ? Ak[l + kk * i] : Ak[i + m * l];
                if (dk) v *= dk[l];
            }
            As[ll][ii] = v;
        }
        for (int e = tid; e < TK * TN; e += 256) {
            int ll = e / TN, jj = e % TN;
            int64_t j = j0 + jj, l = l0 + ll;
            Bs[ll][jj] = (j < n && l < kk) ? (transB ? Bk[j + n * l] : Bk[l + kk * j]) : T(0);
        }
        __syncthreads();
#pragma unroll 4
        for (int ll = 0; ll < TK; ++ll) {
            T a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) a[u] = As[ll][ti + 16 * u];
#pragma unroll
            for (int u = 0; u < 4; ++u) b[u] = Bs[ll][tj + 16 * u];
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) acc[x][y] = fma(a[x], b[y], acc[x][y]);
        }
    }
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
            int64_t i = i0 + ti + 16 * x, j = j0 + tj + 16 * y;
            if (i < m && j < n) Ck[i + m * j] = acc[x][y];
        }
}

}  // namespace

template <typename T>
cudaError_t launch_facewise(const T* A, const T* B, T* C, int64_t m, int64_t n, int64_t kk, int64_t nbatch,
                            int transA, int transB, const T* dscale, cudaStream_t s)
{
    dim3 g((unsigned)((m + TM - 1) / TM), (unsigned)((n + TN - 1) / TN), (unsigned)nbatch);
    facewise_kernel<T><<<g, 256, 0, s>>>(A, B, C, m, n, kk, transA, transB, dscale);
    return cudaGetLastError();
}

template cudaError_t launch_facewise<float>(const float*, const float*, float*, int64_t, int64_t, int64_t, int64_t,
                                            int, int, const float*, cudaStream_t);
template cudaError_t launch_facewise<double>(const double*, const double*, double*, int64_t, int64_t, int64_t,
                                             int64_t, int, int, const double*, cudaStream_t);

}  // namespace tnn
