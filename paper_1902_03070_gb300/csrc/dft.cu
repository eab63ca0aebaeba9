// The DFT-based comparison path: t-SVT under the Fourier transform along
// the tubes (the t-SVD the paper compares against, with TNN-F).
//
// For a real tensor the DFT slices k and n3 - k are complex conjugates, so
// only the nh = floor(n3/2) + 1 slices k = 0..nh-1 are computed.  Forward:
// a real GEMM per pixel tube with an n3 x 2nh operator (cos, -sin columns),
// writing slice k as two real planes (real part, imaginary part).  Each
// complex slice gets a one-sided Jacobi SVT (Hestenes with complex column
// pairs: the pair's inner product gamma = a_i^H a_j is turned real by a
// unit phase on a_j, then the real Rutishauser rotation applies) and the
// V-free rebuild Y = sum_{sigma > tau} (1 - tau/sigma) / sigma^2
// a_q (a_q^H A0).  Inverse: a real GEMM with a 2nh x n3 operator that folds
// in the conjugate slices (weights 1 for k = 0 and k = n3/2, 2 otherwise).
//
// The Jacobi kernel here is deliberately plain (one warp per column pair,
// columns in shared memory, one CTA per slice) and also runs on real slices,
// so that tsvt_dct_plain measures the DCT path with the same kernel design:
// the DCT/DFT ratio then compares the transforms' arithmetic, not two
// kernels of different tuning.
#include <cuda_runtime.h>
#include <math.h>

#include <vector>

#include "tnn_internal.h"

namespace tnn {
namespace {

constexpr int RBM = 128;  // pixels per tile
constexpr int RBN = 64;   // outputs per pass
constexpr int RBK = 16;   // inputs per stage
constexpr int RNT = 256;

// out(p, q) = sum_j in(p, j) op(j, q), q < nout (op: nin x nout, column-major).
template <typename T>
__global__ void __launch_bounds__(RNT) tube_rect_kernel(const T* __restrict__ in, T* __restrict__ out,
                                                        const T* __restrict__ op, int64_t P, int nin, int nout)
{
    const int64_t p0 = (int64_t)blockIdx.x * RBM;
    __shared__ __align__(16) T As[RBK][RBM];
    __shared__ T Ts[RBK][RBN];
    const int tid = threadIdx.x, tp = tid & 31, tq = tid >> 5;
    for (int q0 = 0; q0 < nout; q0 += RBN) {
        T acc[8][4];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[i][c] = T(0);
        for (int j0 = 0; j0 < nin; j0 += RBK) {
            __syncthreads();
            for (int e = tid; e < RBK * RBM; e += RNT) {
                const int jj = e / RBM, pp = e % RBM;
                const int64_t p = p0 + pp;
                const int j = j0 + jj;
                As[jj][pp] = (p < P && j < nin) ? in[(size_t)p + (size_t)P * j] : T(0);
            }
            for (int e = tid; e < RBK * RBN; e += RNT) {
                const int jj = e / RBN, qq = e % RBN;
                const int j = j0 + jj, q = q0 + qq;
                Ts[jj][qq] = (j < nin && q < nout) ? op[j + (size_t)nin * q] : T(0);
            }
            __syncthreads();
#pragma unroll 4
            for (int jj = 0; jj < RBK; ++jj) {
                T av[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) av[c] = As[jj][tp * 4 + c];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const T t = Ts[jj][tq + 8 * i];
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[i][c] = fma(av[c], t, acc[i][c]);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int q = q0 + tq + 8 * i;
            if (q >= nout) continue;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int64_t p = p0 + tp * 4 + c;
                if (p < P) out[(size_t)p + (size_t)P * q] = acc[i][c];
            }
        }
        __syncthreads();
    }
}

// DFT operators.  Forward (n3 x 2nh): column 2k = cos(2 pi j k / n3), column
// 2k + 1 = -sin(2 pi j k / n3).  Inverse (2nh x n3): row 2k = w_k cos / n3,
// row 2k + 1 = -w_k sin / n3, w_k = 1 for k = 0 and k = n3/2, else 2.
// Angles reduced exactly: (j k) mod n3.
template <typename T>
__global__ void build_dft_ops(T* fwd, T* inv, int n3, int nh)
{
    const int total = n3 * nh;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
        const int j = idx % n3, k = idx / n3;
        const long long r = ((long long)j * k) % n3;
        double sn, cs;
        sincospi(2.0 * (double)r / (double)n3, &sn, &cs);
        fwd[j + (size_t)n3 * (2 * k)] = (T)cs;
        fwd[j + (size_t)n3 * (2 * k + 1)] = (T)(-sn);
        const double w = (k == 0 || 2 * k == n3) ? 1.0 : 2.0;
        inv[(2 * k) + (size_t)(2 * nh) * j] = (T)(w * cs / n3);
        inv[(2 * k + 1) + (size_t)(2 * nh) * j] = (T)(-w * sn / n3);
    }
}

template <int L, typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Plain one-sided Jacobi SVT of one slice per CTA (real, or complex stored
// as a real plane and an imaginary plane `im_off` elements after it).
// RR rows per lane (m <= 32 RR).  Slice s starts at data + s * slice_stride.
template <typename T, bool CPLX, int RR, bool SMEM>
__global__ void __launch_bounds__(RR >= 16 ? 256 : 512) jacobi_plain_kernel(T* data, int64_t slice_stride, int64_t im_off, int n1,
                                                          int n2, double tau, int max_sweeps, T* work,
                                                          SliceStats* stats)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, W = blockDim.x >> 5;
    const int slice = blockIdx.x;
    const bool tr = n1 < n2;
    const int m = tr ? n2 : n1, n = tr ? n1 : n2;
    const int np = n + (n & 1);  // columns, padded to even
    const int ldA = m;
    const size_t plane = (size_t)ldA * np;
    T* base = SMEM ? reinterpret_cast<T*>(smem_raw) : work + (size_t)slice * plane * (CPLX ? 2 : 1);
    T* Are = base;
    T* Aim = CPLX ? base + plane : nullptr;
    int* kidx = reinterpret_cast<int*>(SMEM ? smem_raw + plane * sizeof(T) * (CPLX ? 2 : 1) : smem_raw);
    T* kcf = reinterpret_cast<T*>(kidx + ((np + 3) & ~3));
    T* sig = kcf + np;
    __shared__ int s_rot, s_keep, s_nonfinite;
    __shared__ double s_nuc;
    __shared__ unsigned long long s_pairs, s_rots;

    T* src_re = data + (size_t)slice * slice_stride;
    T* src_im = CPLX ? src_re + im_off : nullptr;
    // oriented element (r, c): A(r, c), or conj(A(c, r)) when transposed
    for (size_t e = tid; e < plane; e += blockDim.x) {
        const int c = (int)(e / ldA), r = (int)(e % ldA);
        T vr = T(0), vi = T(0);
        if (c < n) {
            const size_t g = tr ? (size_t)c + (size_t)n1 * r : (size_t)r + (size_t)n1 * c;
            vr = src_re[g];
            if (CPLX) vi = tr ? -src_im[g] : src_im[g];
        }
        Are[e] = vr;
        if (CPLX) Aim[e] = vi;
    }
    if (tid == 0) {
        s_pairs = 0;
        s_rots = 0;
        s_nonfinite = 0;
        s_nuc = 0.0;
        s_keep = 0;
    }
    __syncthreads();

    const T tol = sqrt((T)m) * (sizeof(T) == 4 ? T(5.9604645e-8) : T(1.1102230246251565e-16));
    int sweeps = 0, converged = 0;
    unsigned long long pairs = 0, rots = 0;
    const int msw = max_sweeps > 0 ? max_sweeps : 30;
    while (sweeps < msw) {
        if (tid == 0) s_rot = 0;
        __syncthreads();
        int big = 0;
        for (int step = 0; step < np - 1; ++step) {
            for (int pr = warp; pr < np / 2; pr += W) {
                // circle method over the np columns: position 0 fixed
                auto at = [&](int t) {
                    if (t == 0) return 0;
                    int v = t - 1 + step;
                    if (v >= np - 1) v -= np - 1;
                    return 1 + v;
                };
                const int ci = at(pr), cj = at(np - 1 - pr);
                T ar[RR], ai[RR], br[RR], bi[RR];
                T al = T(0), be = T(0), gr = T(0), gi = T(0);
#pragma unroll
                for (int q = 0; q < RR; ++q) {
                    const int r = q * 32 + lane;
                    const bool in = r < m;
                    ar[q] = in ? Are[(size_t)ci * ldA + r] : T(0);
                    br[q] = in ? Are[(size_t)cj * ldA + r] : T(0);
                    ai[q] = (CPLX && in) ? Aim[(size_t)ci * ldA + r] : T(0);
                    bi[q] = (CPLX && in) ? Aim[(size_t)cj * ldA + r] : T(0);
                    al = fma(ar[q], ar[q], al);
                    be = fma(br[q], br[q], be);
                    gr = fma(ar[q], br[q], gr);
                    if (CPLX) {
                        al = fma(ai[q], ai[q], al);
                        be = fma(bi[q], bi[q], be);
                        gr = fma(ai[q], bi[q], gr);
                        gi = fma(ar[q], bi[q], gi);
                        gi = fma(-ai[q], br[q], gi);
                    }
                }
                al = warp_sum<32>(al);
                be = warp_sum<32>(be);
                gr = warp_sum<32>(gr);
                if (CPLX) gi = warp_sum<32>(gi);
                const T ag = CPLX ? sqrt(fma(gr, gr, gi * gi)) : fabs(gr);
                const T den = sqrt(al * be);
                const bool rot = den > T(0) && ag > tol * den;  // uniform across the warp
                if (lane == 0) ++pairs;
                if (rot) {
                    if (ag > T(2) * tol * den) big = 1;
                    if (lane == 0) ++rots;
                    // real rotation for |gamma|; the phase u = conj(gamma)/|gamma| goes onto a_j
                    const T zeta = (be - al) / (T(2) * ag);
                    const T t = (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + sqrt(fma(zeta, zeta, T(1))));
                    const T c = T(1) / sqrt(fma(t, t, T(1)));
                    const T s = c * t;
                    const T ur = gr / ag, ui = CPLX ? -gi / ag : T(0);
#pragma unroll
                    for (int q = 0; q < RR; ++q) {
                        const T vr = CPLX ? fma(ur, br[q], -ui * bi[q]) : ur * br[q];
                        const T vi = CPLX ? fma(ur, bi[q], ui * br[q]) : T(0);
                        const T nr = fma(c, ar[q], -s * vr), nj = fma(s, ar[q], c * vr);
                        ar[q] = nr;
                        br[q] = nj;
                        if (CPLX) {
                            const T mi = fma(c, ai[q], -s * vi), mj = fma(s, ai[q], c * vi);
                            ai[q] = mi;
                            bi[q] = mj;
                        }
                    }
#pragma unroll
                    for (int q = 0; q < RR; ++q) {
                        const int r = q * 32 + lane;
                        if (r < m) {
                            Are[(size_t)ci * ldA + r] = ar[q];
                            Are[(size_t)cj * ldA + r] = br[q];
                            if (CPLX) {
                                Aim[(size_t)ci * ldA + r] = ai[q];
                                Aim[(size_t)cj * ldA + r] = bi[q];
                            }
                        }
                    }
                }
            }
            __syncthreads();
        }
        if (big) atomicOr(&s_rot, 1);
        __syncthreads();
        const int any = s_rot;
        ++sweeps;
        __syncthreads();
        if (!any) {
            converged = 1;
            break;
        }
    }
    if (lane == 0 && pairs) atomicAdd(&s_pairs, pairs);
    if (lane == 0 && rots) atomicAdd(&s_rots, rots);

    // sigma_c = |a_c| (warp per column)
    for (int c = warp; c < np; c += W) {
        T s2 = T(0);
        for (int r = lane; r < m; r += 32) {
            const T x = Are[(size_t)c * ldA + r];
            s2 = fma(x, x, s2);
            if (CPLX) {
                const T y = Aim[(size_t)c * ldA + r];
                s2 = fma(y, y, s2);
            }
        }
        s2 = warp_sum<32>(s2);
        if (lane == 0) {
            sig[c] = sqrt(s2);
            if (!isfinite(s2)) s_nonfinite = 1;
        }
    }
    __syncthreads();
    const T tt = (T)tau;
    if (tid == 0) {
        int kk = 0;
        double nuc = 0.0;
        for (int c = 0; c < np; ++c) {
            const T sg = sig[c];
            if (sg > tt) {
                kidx[kk] = c;
                kcf[kk] = (T(1) - tt / sg) / (sg * sg);
                nuc += (double)(sg - tt);
                ++kk;
            }
        }
        s_keep = kk;
        s_nuc = nuc;
    }
    __syncthreads();
    const int keep = s_keep;
    // rebuild, warp per output column: y_j = sum_q cf_q a_q (a_q^H a0_j)
    for (int j = warp; j < n; j += W) {
        T xr[RR], xi[RR], yr[RR], yi[RR];
#pragma unroll
        for (int q = 0; q < RR; ++q) {
            const int r = q * 32 + lane;
            xr[q] = T(0);
            xi[q] = T(0);
            yr[q] = T(0);
            yi[q] = T(0);
            if (r < m) {
                const size_t g = tr ? (size_t)j + (size_t)n1 * r : (size_t)r + (size_t)n1 * j;
                xr[q] = src_re[g];
                if (CPLX) xi[q] = tr ? -src_im[g] : src_im[g];
            }
        }
        for (int k = 0; k < keep; ++k) {
            const int c = kidx[k];
            T vr[RR], vi[RR];
            T dr = T(0), di = T(0);
#pragma unroll
            for (int q = 0; q < RR; ++q) {
                const int r = q * 32 + lane;
                vr[q] = r < m ? Are[(size_t)c * ldA + r] : T(0);
                vi[q] = (CPLX && r < m) ? Aim[(size_t)c * ldA + r] : T(0);
                dr = fma(vr[q], xr[q], dr);
                if (CPLX) {
                    dr = fma(vi[q], xi[q], dr);
                    di = fma(vr[q], xi[q], di);
                    di = fma(-vi[q], xr[q], di);
                }
            }
            dr = warp_sum<32>(dr) * kcf[k];
            if (CPLX) di = warp_sum<32>(di) * kcf[k];
#pragma unroll
            for (int q = 0; q < RR; ++q) {
                yr[q] = fma(dr, vr[q], yr[q]);
                if (CPLX) {
                    yr[q] = fma(-di, vi[q], yr[q]);
                    yi[q] = fma(dr, vi[q], yi[q]);
                    yi[q] = fma(di, vr[q], yi[q]);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < RR; ++q) {
            const int r = q * 32 + lane;
            if (r < m) {
                const size_t g = tr ? (size_t)j + (size_t)n1 * r : (size_t)r + (size_t)n1 * j;
                src_re[g] = yr[q];
                if (CPLX) src_im[g] = tr ? -yi[q] : yi[q];
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        SliceStats st;
        st.nuc = s_nuc;
        st.pairs = (int64_t)s_pairs;
        st.rotations = (int64_t)s_rots;
        st.sweeps = sweeps;
        st.converged = converged;
        st.nonfinite = s_nonfinite;
        st.kept = keep;
        stats[slice] = st;
    }
}

// Shared memory of the plain kernel: the working copy (when it fits), the
// kept list, coefficients and sigmas.
size_t plain_small_bytes(int np, int elem) { return (size_t)((np + 3) & ~3) * 4 + (size_t)2 * np * elem + 64; }

template <typename T, bool CPLX, int RR>
cudaError_t launch_plain_rr(T* data, int64_t stride, int64_t im_off, int n3s, int n1, int n2, double tau, T* work,
                            bool smem_copy, SliceStats* stats, cudaStream_t s)
{
    const int m = n1 > n2 ? n1 : n2, n = n1 > n2 ? n2 : n1;
    const int np = n + (n & 1);
    const size_t plane = (size_t)m * np * sizeof(T) * (CPLX ? 2 : 1);
    int W = np / 2;
    const int wcap = RR >= 16 ? 8 : 16;  // the kernels' thread bounds (registers: RR rows x 6 planes per lane)
    if (W > wcap) W = wcap;
    if (W < 1) W = 1;
    const size_t small = plain_small_bytes(np, (int)sizeof(T));
    if (smem_copy) {
        auto k = jacobi_plain_kernel<T, CPLX, RR, true>;
        const size_t smem = plane + small;
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        k<<<n3s, W * 32, smem, s>>>(data, stride, im_off, n1, n2, tau, 0, nullptr, stats);
    } else {
        auto k = jacobi_plain_kernel<T, CPLX, RR, false>;
        k<<<n3s, W * 32, small, s>>>(data, stride, im_off, n1, n2, tau, 0, work, stats);
    }
    return cudaGetLastError();
}

}  // namespace

size_t jacobi_plain_work_bytes(int64_t n1, int64_t n2, int64_t n3s, int elem, bool cplx, bool* smem_copy)
{
    const int64_t m = n1 > n2 ? n1 : n2, n = n1 > n2 ? n2 : n1;
    const int64_t np = n + (n & 1);
    const size_t plane = (size_t)m * np * elem * (cplx ? 2 : 1);
    *smem_copy = plane + plain_small_bytes((int)np, elem) <= 226 * 1024;
    return *smem_copy ? 0 : plane * (size_t)n3s;
}

template <typename T>
cudaError_t launch_jacobi_plain(T* data, int64_t stride, int64_t im_off, int n3s, int n1, int n2, double tau,
                                bool cplx, T* work, bool smem_copy, SliceStats* stats, cudaStream_t s)
{
    const int m = n1 > n2 ? n1 : n2;
    if (m > 512) return cudaErrorInvalidValue;
    const int rr = (m + 31) / 32;
#define TNN_PLAIN(RRV)                                                                                             \
    return cplx ? launch_plain_rr<T, true, RRV>(data, stride, im_off, n3s, n1, n2, tau, work, smem_copy, stats, s) \
                : launch_plain_rr<T, false, RRV>(data, stride, im_off, n3s, n1, n2, tau, work, smem_copy, stats, s);
    if (rr <= 2) { TNN_PLAIN(2) }
    if (rr <= 4) { TNN_PLAIN(4) }
    if (rr <= 8) { TNN_PLAIN(8) }
    TNN_PLAIN(16)
#undef TNN_PLAIN
}
template cudaError_t launch_jacobi_plain<float>(float*, int64_t, int64_t, int, int, int, double, bool, float*, bool,
                                                SliceStats*, cudaStream_t);
template cudaError_t launch_jacobi_plain<double>(double*, int64_t, int64_t, int, int, int, double, bool, double*,
                                                 bool, SliceStats*, cudaStream_t);

template <typename T>
cudaError_t launch_tube_rect(const T* in, T* out, const T* op, int64_t P, int nin, int nout, cudaStream_t s)
{
    const unsigned grid = (unsigned)((P + RBM - 1) / RBM);
    if (grid == 0) return cudaSuccess;
    tube_rect_kernel<T><<<grid, RNT, 0, s>>>(in, out, op, P, nin, nout);
    return cudaGetLastError();
}
template cudaError_t launch_tube_rect<float>(const float*, float*, const float*, int64_t, int, int, cudaStream_t);
template cudaError_t launch_tube_rect<double>(const double*, double*, const double*, int64_t, int, int,
                                              cudaStream_t);

template <typename T>
cudaError_t launch_build_dft_ops(T* fwd, T* inv, int n3, cudaStream_t s)
{
    const int nh = n3 / 2 + 1;
    const int total = n3 * nh;
    build_dft_ops<T><<<(total + 255) / 256, 256, 0, s>>>(fwd, inv, n3, nh);
    return cudaGetLastError();
}
template cudaError_t launch_build_dft_ops<float>(float*, float*, int, cudaStream_t);
template cudaError_t launch_build_dft_ops<double>(double*, double*, int, cudaStream_t);

}  // namespace tnn
