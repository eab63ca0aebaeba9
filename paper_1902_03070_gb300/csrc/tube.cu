// Tube transforms along mode 3 on CUDA cores (FP64 and FP32 paths), with the
// ADMM prologue / epilogue of Algorithm 1 fused in.
//
// The transform is the contraction out(p, q) = sum_j in(p, j) * T(j, q) over
// the tube index, p = i + n1*j the pixel (P = n1*n2 pixels, contiguous in
// memory for a fixed tube index) and T the n3 x n3 DCT operator.  One CTA
// computes a 128-pixel x 64-frequency tile; the input strip and the operator
// chunk are staged in shared memory, every pixel is read from HBM once per
// 64-wide frequency tile and written once.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "tnn_internal.h"

namespace tnn {

namespace {

constexpr int BM = 128;  // pixels per CTA tile
constexpr int BN = 64;   // output tube positions per CTA tile
constexpr int BK = 16;   // input tube positions per stage
constexpr int NT = 256;  // threads per CTA: 32 pixel groups x 8 frequency groups

// The DCT operator of the requested direction, T(j, q) column-major in an
// n3 x n3 array (T[j + n3*q]), computed in FP64 from the definition
// C[k, j] = a_k cos(pi (2j+1) k / (2 n3)), a_0 = sqrt(1/n3), a_k = sqrt(2/n3).
template <typename T>
__global__ void build_operator(T* op, int n3, int inverse, int scaled)
{
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n3 * n3) return;
    int j = idx % n3, q = idx / n3;
    auto Cf = [n3](int k, int jj) {
        double a = (k == 0) ? sqrt(1.0 / n3) : sqrt(2.0 / n3);
        return a * cospi((double)((2 * jj + 1) * k) / (2.0 * n3));
    };
    double v;
    if (!inverse) {
        v = Cf(q, j);                       // forward: out_q = sum_j C[q, j] in_j
        if (scaled) v /= Cf(q, 0);          // L: divide frequency q by w_q = C[q, 0]
    } else {
        v = Cf(j, q);                       // inverse: out_q = sum_k C[k, q] in_k (k = j here)
        if (scaled) v *= Cf(j, 0);          // L^-1: input frequency k scaled by w_k
    }
    op[j + (size_t)n3 * q] = (T)v;
}

struct NoPro {};

// One 128-pixel x 64-frequency tile (pixels p0.., output positions q0..).
// MODE 0: plain; MODE 1: forward with prologue Z = X - M/beta; MODE 2:
// inverse with the ADMM epilogue, its four partial sums written to
// partials[4 tile .. 4 tile + 3].  Shared by the per-tensor kernel (one tile
// per CTA of a 2-D grid) and the batched ADMM step (tiles of many tensors
// from an item table), so both compute the same bits.
template <typename T, int MODE>
__device__ __forceinline__ void tube_tile(const T* __restrict__ in, const T* __restrict__ in2, T* __restrict__ out,
                                          const T* __restrict__ op, int64_t P, int n3,
                                          const AdmmCtl* __restrict__ ctl, T* __restrict__ Xs, T* __restrict__ Ms,
                                          const T* __restrict__ Bs, const uint8_t* __restrict__ mask,
                                          double* __restrict__ partials, int64_t p0, int q0, int64_t tile)
{
    __shared__ __align__(16) T As[BK][BM];
    __shared__ T Ts[BK][BN];

    const int tid = threadIdx.x;
    const int tp = tid & 31;     // pixel group: pixels tp*4 .. tp*4+3 of the tile
    const int tq = tid >> 5;     // frequency group: q = tq + 8*i

    T rbeta = T(0);
    double beta = 0.0;
    if (MODE != 0) {
        beta = ctl->beta;
        rbeta = (T)beta;
    }

    T acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[i][c] = T(0);

    for (int j0 = 0; j0 < n3; j0 += BK) {
        __syncthreads();
        // stage the input strip: BK tube positions x BM pixels
        for (int e = tid; e < BK * BM; e += NT) {
            int jj = e / BM, pp = e % BM;
            int64_t p = p0 + pp;
            int j = j0 + jj;
            T v = T(0);
            if (p < P && j < n3) {
                size_t g = (size_t)p + (size_t)P * j;
                v = in[g];
                if (MODE == 1) v = v - in2[g] / rbeta;  // Z = X - M / beta
            }
            As[jj][pp] = v;
        }
        for (int e = tid; e < BK * BN; e += NT) {
            int jj = e / BN, qq = e % BN;
            int j = j0 + jj, q = q0 + qq;
            Ts[jj][qq] = (j < n3 && q < n3) ? op[j + (size_t)n3 * q] : T(0);
        }
        __syncthreads();
#pragma unroll 4
        for (int jj = 0; jj < BK; ++jj) {
            T a[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) a[c] = As[jj][tp * 4 + c];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                T t = Ts[jj][tq + 8 * i];
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[i][c] = fma(a[c], t, acc[i][c]);
            }
        }
    }

    if (MODE != 2) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            int q = q0 + tq + 8 * i;
            if (q >= n3) continue;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                int64_t p = p0 + tp * 4 + c;
                if (p < P) out[(size_t)p + (size_t)P * q] = acc[i][c];
            }
        }
        return;
    }

    // ADMM epilogue (Algorithm 1; Eq. 25 and the multiplier update of Eq. 20):
    //   X+ = mask ? B : Y + M/beta,  M+ = M + beta (Y - X+)
    //   residual sums in FP64 per thread, FP32 only within a row of 4 pixels
    double sdx = 0, sxx = 0, syx = 0, snx = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        int q = q0 + tq + 8 * i;
        if (q >= n3) continue;
        T cdx = 0, cxx = 0, cyx = 0, cnx = 0;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            int64_t p = p0 + tp * 4 + c;
            if (p >= P) continue;
            size_t g = (size_t)p + (size_t)P * q;
            T y = acc[i][c];
            T x = Xs[g], mm = Ms[g];
            T xn = mask[g] ? Bs[g] : y + mm / rbeta;
            T mn = mm + rbeta * (y - xn);
            T dx = xn - x, dy = y - xn;
            cdx = fma(dx, dx, cdx);
            cxx = fma(x, x, cxx);
            cyx = fma(dy, dy, cyx);
            cnx = fma(xn, xn, cnx);
            Xs[g] = xn;
            Ms[g] = mn;
        }
        sdx += (double)cdx;
        sxx += (double)cxx;
        syx += (double)cyx;
        snx += (double)cnx;
    }
    double s[4] = {sdx, sxx, syx, snx};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int v = 0; v < 4; ++v) s[v] += __shfl_xor_sync(0xffffffffu, s[v], o);
    __shared__ double red[NT / 32][4];
    if (tp == 0)
#pragma unroll
        for (int v = 0; v < 4; ++v) red[tq][v] = s[v];
    __syncthreads();
    if (tid < 4) {
        double t = 0.0;
        for (int w = 0; w < NT / 32; ++w) t += red[w][tid];
        partials[(size_t)tile * 4 + tid] = t;
    }
}

template <typename T, int MODE>
__global__ void __launch_bounds__(NT)
tube_kernel(const T* __restrict__ in, const T* __restrict__ in2, T* __restrict__ out, const T* __restrict__ op,
            int64_t P, int n3, const AdmmCtl* __restrict__ ctl, T* __restrict__ Xs, T* __restrict__ Ms,
            const T* __restrict__ Bs, const uint8_t* __restrict__ mask, double* __restrict__ partials)
{
    if (MODE != 0 && ctl->done) return;
    tube_tile<T, MODE>(in, in2, out, op, P, n3, ctl, Xs, Ms, Bs, mask, partials, (int64_t)blockIdx.x * BM,
                       (int)blockIdx.y * BN, (int64_t)blockIdx.y * gridDim.x + blockIdx.x);
}

// Batched ADMM step: tiles of many tensors, one CTA each (AdmmTileItem).
template <typename T, int MODE>
__global__ void __launch_bounds__(NT) tube_admm_batched_kernel(const AdmmTileItem* __restrict__ items)
{
    const AdmmTileItem it = items[blockIdx.x];
    if (it.ctl->done) return;
    tube_tile<T, MODE>(static_cast<const T*>(it.in), static_cast<const T*>(it.in2), static_cast<T*>(it.out),
                       static_cast<const T*>(it.op), it.P, it.n3, it.ctl, static_cast<T*>(it.X),
                       static_cast<T*>(it.M), static_cast<const T*>(it.B), it.mask, it.partials, it.p0, it.q0,
                       it.tile);
}

template <typename T>
__global__ void admm_init_kernel(const T* __restrict__ B, const uint8_t* __restrict__ mask, T* __restrict__ X,
                                 T* __restrict__ M, int64_t N)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
        X[e] = mask[e] ? B[e] : T(0);
        M[e] = T(0);
    }
}

__global__ void ctl_init_kernel(AdmmCtl* ctl, double beta, double rho, double beta_max, double tol, int max_iter)
{
    AdmmCtl c;
    c.beta = beta;
    c.rho = rho;
    c.beta_max = beta_max;
    c.tol = tol;
    c.iter = 0;
    c.max_iter = max_iter;
    c.done = (max_iter <= 0) ? 1 : 0;
    c.converged = 0;
    c.rel_change = 0.0;
    c.primal_res = 0.0;
    c.sweeps_max = 0;
    c.unconverged = 0;
    c.nonfinite = 0;
    c.pad_ = 0;
    *ctl = c;
}

// One block, fixed-order reduction: results do not depend on timing.
__device__ __forceinline__ void admm_finalize_block(AdmmCtl* ctl, const double* __restrict__ partials, int nblocks,
                                                    const SliceStats* __restrict__ stats, int64_t n3)
{
    __shared__ double red[256][4];
    __shared__ int sw[256], un[256], nf[256];
    const int t = threadIdx.x;
    double s[4] = {0, 0, 0, 0};
    for (int b = t; b < nblocks; b += 256)
        for (int v = 0; v < 4; ++v) s[v] += partials[(size_t)b * 4 + v];
    for (int v = 0; v < 4; ++v) red[t][v] = s[v];
    int smax = 0, uc = 0, nfin = 0;
    for (int64_t k = t; k < n3; k += 256) {
        smax = max(smax, stats[k].sweeps);
        uc += stats[k].converged ? 0 : 1;
        nfin |= stats[k].nonfinite;
    }
    sw[t] = smax; un[t] = uc; nf[t] = nfin;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (t < h) {
            for (int v = 0; v < 4; ++v) red[t][v] += red[t + h][v];
            sw[t] = max(sw[t], sw[t + h]);
            un[t] += un[t + h];
            nf[t] |= nf[t + h];
        }
        __syncthreads();
    }
    if (t == 0) {
        double dx = red[0][0], xx = red[0][1], yx = red[0][2], nx = red[0][3];
        double rc = (xx > 0.0) ? sqrt(dx) / sqrt(xx) : sqrt(dx);
        double pr = (nx > 0.0) ? sqrt(yx) / sqrt(nx) : sqrt(yx);
        AdmmCtl c = *ctl;
        c.rel_change = rc;
        c.primal_res = pr;
        c.sweeps_max = sw[0];
        c.unconverged += un[0];
        c.nonfinite |= nf[0] | (isfinite(rc) && isfinite(pr) ? 0 : 1);
        double nb = c.rho * c.beta;
        c.beta = (nb < c.beta_max) ? nb : c.beta_max;
        c.iter += 1;
        if (rc <= c.tol && pr <= c.tol) {
            c.converged = 1;
            c.done = 1;
        }
        if (c.iter >= c.max_iter || c.nonfinite) c.done = 1;
        *ctl = c;
    }
}

__global__ void admm_finalize_kernel(AdmmCtl* ctl, const double* __restrict__ partials, int nblocks,
                                     const SliceStats* __restrict__ stats, int64_t n3)
{
    if (ctl->done) return;
    admm_finalize_block(ctl, partials, nblocks, stats, n3);
}

// Batched ADMM step: one block per job.
__global__ void admm_finalize_batched_kernel(const AdmmJobItem* __restrict__ jobs)
{
    const AdmmJobItem j = jobs[blockIdx.x];
    if (j.ctl->done) return;
    admm_finalize_block(j.ctl, j.partials, j.nblocks, j.stats, j.n3);
}

inline dim3 tube_grid(int64_t P, int64_t n3)
{
    return dim3((unsigned)((P + BM - 1) / BM), (unsigned)((n3 + BN - 1) / BN), 1);
}

}  // namespace

// Operator cache lives in api.cu; these entry points take it ready-made.
template <typename T>
cudaError_t launch_build_operator(T* op, int64_t n3, int inverse, int scaled, cudaStream_t s)
{
    int n = (int)(n3 * n3);
    build_operator<T><<<(n + 255) / 256, 256, 0, s>>>(op, (int)n3, inverse, scaled);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_tube_op(const T* X, T* Y, const T* op, int64_t P, int64_t n3, cudaStream_t s)
{
    tube_kernel<T, 0><<<tube_grid(P, n3), NT, 0, s>>>(X, nullptr, Y, op, P, (int)n3, nullptr, nullptr, nullptr,
                                                     nullptr, nullptr, nullptr);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_tube_fwd_admm_op(const T* X, const T* M, T* Zbar, const T* op, int64_t P, int64_t n3,
                                    const AdmmCtl* ctl, cudaStream_t s)
{
    tube_kernel<T, 1><<<tube_grid(P, n3), NT, 0, s>>>(X, M, Zbar, op, P, (int)n3, ctl, nullptr, nullptr, nullptr,
                                                     nullptr, nullptr);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_tube_inv_admm_op(const T* Ybar, T* X, T* M, const T* B, const uint8_t* mask, const T* op,
                                    int64_t P, int64_t n3, const AdmmCtl* ctl, double* partials, int* nblocks,
                                    cudaStream_t s)
{
    dim3 g = tube_grid(P, n3);
    *nblocks = (int)(g.x * g.y);
    tube_kernel<T, 2><<<g, NT, 0, s>>>(Ybar, nullptr, nullptr, op, P, (int)n3, ctl, X, M, B, mask, partials);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_tube_admm_batched(const AdmmTileItem* items, int count, int mode, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    if (mode == 1) tube_admm_batched_kernel<T, 1><<<count, NT, 0, s>>>(items);
    else tube_admm_batched_kernel<T, 2><<<count, NT, 0, s>>>(items);
    return cudaGetLastError();
}

cudaError_t launch_admm_finalize_batched(const AdmmJobItem* jobs, int count, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    admm_finalize_batched_kernel<<<count, 256, 0, s>>>(jobs);
    return cudaGetLastError();
}

int tube_tiles_x(int64_t P) { return (int)((P + BM - 1) / BM); }
int tube_tiles_y(int64_t n3) { return (int)((n3 + BN - 1) / BN); }
int tube_tile_pixels() { return BM; }
int tube_tile_outputs() { return BN; }

int tube_partials_count(int64_t P, int64_t n3)
{
    dim3 g = tube_grid(P, n3);
    return (int)(g.x * g.y);
}

template <typename T>
cudaError_t launch_admm_init(const T* B, const uint8_t* mask, T* X, T* M, int64_t N, cudaStream_t s)
{
    int64_t blocks = (N + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    admm_init_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(B, mask, X, M, N);
    return cudaGetLastError();
}

cudaError_t launch_ctl_init(AdmmCtl* ctl, double beta, double rho, double beta_max, double tol, int max_iter,
                            cudaStream_t s)
{
    ctl_init_kernel<<<1, 1, 0, s>>>(ctl, beta, rho, beta_max, tol, max_iter);
    return cudaGetLastError();
}

cudaError_t launch_admm_finalize(AdmmCtl* ctl, const double* partials, int nblocks, const SliceStats* stats,
                                 int64_t n3, cudaStream_t s)
{
    admm_finalize_kernel<<<1, 256, 0, s>>>(ctl, partials, nblocks, stats, n3);
    return cudaGetLastError();
}

#define TNN_INST(T)                                                                                              \
    template cudaError_t launch_build_operator<T>(T*, int64_t, int, int, cudaStream_t);                         \
    template cudaError_t launch_tube_op<T>(const T*, T*, const T*, int64_t, int64_t, cudaStream_t);              \
    template cudaError_t launch_tube_fwd_admm_op<T>(const T*, const T*, T*, const T*, int64_t, int64_t,          \
                                                    const AdmmCtl*, cudaStream_t);                               \
    template cudaError_t launch_tube_inv_admm_op<T>(const T*, T*, T*, const T*, const uint8_t*, const T*,        \
                                                    int64_t, int64_t, const AdmmCtl*, double*, int*,             \
                                                    cudaStream_t);                                               \
    template cudaError_t launch_admm_init<T>(const T*, const uint8_t*, T*, T*, int64_t, cudaStream_t);      \
    template cudaError_t launch_tube_admm_batched<T>(const AdmmTileItem*, int, int, cudaStream_t);
TNN_INST(float)
TNN_INST(double)
#undef TNN_INST

}  // namespace tnn
