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

#include "async_copy.cuh"
#include "tnn_internal.h"

namespace tnn {
namespace {

constexpr int WQ = 512;   // threads per CTA of the QR (16 warps: room on its SMs for other kernels' CTAs)
template <int NB> constexpr int qr_threads() { return WQ; }
constexpr int WGM = 640;  // most threads per CTA of the GEMM (20 warps)
constexpr int WCB = 8;    // output columns per warp tile of the GEMM
constexpr int WMR = 8;    // most rows per lane of the GEMM (m <= 256)
constexpr int WQN = 224; // most columns of the QR (28 rows per lane)

// Leading dimensions of the GEMM's shared-memory operands: A is held with
// lda = 32 MR + 1 rows (odd, so that the transposing stores of a slice with
// tr = 1 hit distinct banks; rows m..32 MR - 1 are zero), and Q transposed,
// Qt[j * ldq + c] = Q[c * n + j], with ldq = n rounded up to the tile width
// plus 4 (a multiple of 4 floats, so each warp reads its 8 entries of a row
// as two 16-byte loads; columns n.. are zero).
__host__ __device__ inline int gemm_lda(int mr) { return 32 * mr + 1; }
__host__ __device__ inline int gemm_ldq(int n) { return (n + WCB - 1) / WCB * WCB + 4; }

// Cooperative copy of `cols` columns of `rows` elements (source column j at
// src + j * lds) into shared memory: dst[j * ldd + i] (tr: dst[i * ldd + j]).
// A warp takes eight columns at a time, lanes over the rows, so each thread
// keeps eight loads in flight.
template <typename T>
__device__ __forceinline__ void load_cols(T* dst, int ldd, const T* __restrict__ src, int64_t lds, int rows,
                                          int cols, bool tr, int warp, int W, int lane)
{
    constexpr int U = 8;
    for (int j0 = warp * U; j0 < cols; j0 += W * U)
        for (int i = lane; i < rows; i += 32) {
            T v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) v[u] = (j0 + u < cols) ? src[(size_t)(j0 + u) * lds + i] : T(0);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (j0 + u >= cols) break;
                if (tr) dst[(size_t)i * ldd + j0 + u] = v[u];
                else dst[(size_t)(j0 + u) * ldd + i] = v[u];
            }
        }
}

// W0 = A0 Q for one slice per CTA, both operands in shared memory; each warp
// computes 32 MR x 8 output tiles (lane rows r = 32 q + lane, eight columns),
// so one k step costs MR + 2 shared loads for 8 MR FMAs.
template <typename T, int MR>
__global__ void __launch_bounds__(WGM) warm_gemm_kernel(const T* __restrict__ data, int64_t n1, int64_t n2, int m,
                                                      int n, int tr, int ldA, int npad, size_t stride,
                                                      const T* __restrict__ Q, const int* __restrict__ flag,
                                                      T* __restrict__ w0, const AdmmCtl* __restrict__ ctl)
{
    static_assert(sizeof(T) == 4, "FP32 only");
    if (ctl && ctl->done) return;
    const int k = blockIdx.x;
    if (!flag[k]) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int lda = 32 * MR + 1;
    const int ldq = gemm_ldq(n);
    T* As = reinterpret_cast<T*>(smem_raw);             // column c at As + c * lda
    T* Qt = As + ((size_t)lda * n + 3) / 4 * 4;         // row j (all c) at Qt + j * ldq
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, W = blockDim.x >> 5;
    // the oriented slice (source columns j, n1 rows each; tr: A's rows) and
    // Q transposed (4-way bank conflicts on those stores), zero-padded
    load_cols(As, lda, data + (size_t)k * n1 * n2, n1, (int)n1, (int)n2, tr != 0, warp, W, lane);
    load_cols(Qt, ldq, Q + (size_t)k * n * n, n, n, n, true, warp, W, lane);
    for (int c = warp; c < n; c += W)
        for (int r = m + lane; r < 32 * MR; r += 32) As[(size_t)c * lda + r] = T(0);
    for (int j = warp; j < n; j += W)
        for (int c = n + lane; c < ldq; c += 32) Qt[(size_t)j * ldq + c] = T(0);
    __syncthreads();
    T* out = w0 + (size_t)k * stride;
    const int ntile = (n + WCB - 1) / WCB;
    for (int t = warp; t < ntile; t += W) {
        const int c0 = t * WCB;
        float acc[MR][WCB];
#pragma unroll
        for (int q = 0; q < MR; ++q)
#pragma unroll
            for (int b = 0; b < WCB; ++b) acc[q][b] = 0.0f;
        const T* ap = As + lane;
        const T* qp = Qt + c0;
#pragma unroll 2
        for (int j = 0; j < n; ++j) {
            float av[MR];
#pragma unroll
            for (int q = 0; q < MR; ++q) av[q] = ap[q * 32];
            const float4 q0 = *reinterpret_cast<const float4*>(qp);
            const float4 q1 = *reinterpret_cast<const float4*>(qp + 4);
            const float qv[WCB] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
#pragma unroll
            for (int q = 0; q < MR; ++q)
#pragma unroll
                for (int b = 0; b < WCB; ++b) acc[q][b] = fmaf(av[q], qv[b], acc[q][b]);
            ap += lda;
            qp += ldq;
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
    // padding columns past the last tile
    for (int c = ntile * WCB + warp; c < npad; c += W)
        for (int r = lane; r < ldA; r += 32) out[(size_t)c * ldA + r] = T(0);
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
    T r;  // 1 / vn2, correctly rounded (the reciprocal is cheaper than a division on the reflector's chain)
    if constexpr (sizeof(T) == 4) r = __frcp_rn(vn2);
    else r = T(1) / vn2;
    bet[c] = vn2 > T(0) ? T(2) * r : T(0);
}

// The QR keeps the n x n matrix in shared memory, column c at Vs + c * ldv
// (rows n.. zero).  A column is worked on by 8 lanes (lane l8 = lane % 8
// holds rows r = 8 i + l8, i < NB), so a warp takes four consecutive columns
// at once and a dot product is a 3-level reduction within 8 lanes; ldv is
// 8 or 24 modulo 32, so the four columns fall in distinct banks.  Reflector
// c touches rows c.. only: the work with c in a 16-row segment runs over the
// row blocks from that segment on (the template argument I0 = 2 (c / 16);
// the segment's own two blocks are masked to rows >= c).

// Factorisation step c: the columns j > c go in chunks of four (chunk q =
// columns c + 1 + 4 q .. c + 4 + 4 q) and get reflector c.  Warp 0 takes
// chunk 0 alone, which holds column c + 1, and then forms reflector c + 1;
// the other chunks go to warps 1 .. W - 1 in turn.
template <typename T, int NB, int I0>
__device__ __forceinline__ void qr_step(T* Vs, T* bet, int ldv, int n, int c, int warp, int W, int lane)
{
    const int l8 = lane & 7, sg = lane >> 3;
    const T b = bet[c];
    const T* x = Vs + (size_t)c * ldv + l8;
    T xv[NB];
#pragma unroll
    for (int i = I0; i < NB; ++i) xv[i] = (i >= I0 + 2 || 8 * i + l8 >= c) ? x[8 * i] : T(0);
    const int nq = (n - 1 - c + 3) >> 2;
    for (int q = warp; q < (warp == 0 ? 1 : nq); q += W - 1) {
        const int j = c + 1 + 4 * q + sg;
        const bool valid = j < n;
        T* y = Vs + (size_t)(valid ? j : c) * ldv + l8;  // a lane past the last column reads column c, stores nothing
        T yv[NB];
        T d0 = T(0), d1 = T(0);
#pragma unroll
        for (int i = I0; i < NB; ++i) {
            yv[i] = y[8 * i];
            if ((i - I0) & 1) d1 = fma(xv[i], yv[i], d1);
            else d0 = fma(xv[i], yv[i], d0);
        }
        T d = d0 + d1;
        d += __shfl_xor_sync(0xffffffffu, d, 4);
        d += __shfl_xor_sync(0xffffffffu, d, 2);
        d += __shfl_xor_sync(0xffffffffu, d, 1);
        const T f = b * d;
        T s2 = T(0);
#pragma unroll
        for (int i = I0; i < NB; ++i) {
            const T v = fma(-f, xv[i], yv[i]);  // rows < c: xv = 0, the value is kept
            if (valid) y[8 * i] = v;
            if (8 * i + l8 > c) s2 = fma(v, v, s2);
        }
        if (q == 0) {  // lanes 0-7 hold column c + 1: the next reflector
            s2 += __shfl_xor_sync(0xffffffffu, s2, 4);
            s2 += __shfl_xor_sync(0xffffffffu, s2, 2);
            s2 += __shfl_xor_sync(0xffffffffu, s2, 1);
            __syncwarp();
            if (lane == 0) make_reflector(Vs + (size_t)(c + 1) * ldv, c + 1, s2, bet);
        }
    }
}

template <typename T, int NB, int I0 = 0>
__device__ __forceinline__ void qr_step_at(int I, T* Vs, T* bet, int ldv, int n, int c, int warp, int W, int lane)
{
    if constexpr (I0 < NB) {
        if (I == I0) qr_step<T, NB, I0>(Vs, bet, ldv, n, c, warp, W, lane);
        else qr_step_at<T, NB, I0 + 2>(I, Vs, bet, ldv, n, c, warp, W, lane);
    }
}

// Q formation: reflectors chi down to clo (one 16-row segment, I0 its first
// block) applied to the column this lane's group of 8 holds.
template <typename T, int NB, int I0>
__device__ __forceinline__ void q_apply(T (&qv)[NB], const T* Vs, const T* bet, int ldv, int chi, int clo, int l8)
{
    for (int c = chi; c >= clo; --c) {
        const T b = bet[c];
        if (b == T(0)) continue;
        const T* x = Vs + (size_t)c * ldv + l8;
        T xv[NB];
        T d0 = T(0), d1 = T(0);
#pragma unroll
        for (int i = I0; i < NB; ++i) {
            xv[i] = (i >= I0 + 2 || 8 * i + l8 >= c) ? x[8 * i] : T(0);
            if ((i - I0) & 1) d1 = fma(xv[i], qv[i], d1);
            else d0 = fma(xv[i], qv[i], d0);
        }
        T d = d0 + d1;
        d += __shfl_xor_sync(0xffffffffu, d, 4);
        d += __shfl_xor_sync(0xffffffffu, d, 2);
        d += __shfl_xor_sync(0xffffffffu, d, 1);
        const T f = b * d;
#pragma unroll
        for (int i = I0; i < NB; ++i) qv[i] = fma(-f, xv[i], qv[i]);
    }
}

template <typename T, int NB, int I0 = 0>
__device__ __forceinline__ void q_apply_at(int I, T (&qv)[NB], const T* Vs, const T* bet, int ldv, int chi, int clo,
                                           int l8)
{
    if constexpr (I0 < NB) {
        if (I == I0) q_apply<T, NB, I0>(qv, Vs, bet, ldv, chi, clo, l8);
        else q_apply_at<T, NB, I0 + 2>(I, qv, Vs, bet, ldv, chi, clo, l8);
    }
}

// Shared-memory leading dimension of the QR: at least 8 NB rows, 8 or 24
// modulo 32 (see above).
__host__ __device__ inline int qr_ldv(int nb)
{
    const int r = 8 * nb;
    return (r % 32 == 0 || r % 32 == 16) ? r + 8 : r;
}

template <typename T, int NB>
__global__ void __launch_bounds__(qr_threads<NB>()) warm_qr_kernel(const T* __restrict__ vrec, int n, size_t stride, int* __restrict__ wrec,
                                                    T* __restrict__ Q, int* __restrict__ flag,
                                                    const AdmmCtl* __restrict__ ctl)
{
    if (ctl && ctl->done) return;
    const int k = blockIdx.x;
    if (!wrec[k]) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ldv = qr_ldv(NB);
    T* Vs = reinterpret_cast<T*>(smem_raw);  // Householder vectors below the diagonal, R on and above it
    T* bet = Vs + (size_t)ldv * n;           // beta of each reflector
    __shared__ int s_next;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, W = blockDim.x >> 5;
    const int l8 = lane & 7, sg = lane >> 3;
    load_cols(Vs, ldv, vrec + (size_t)k * stride, n, n, n, false, warp, W, lane);
    for (int c = warp; c < n; c += W)
        for (int r = n + lane; r < ldv; r += 32) Vs[(size_t)c * ldv + r] = T(0);
    if (tid == 0) s_next = 0;
    __syncthreads();
    // Householder QR, one barrier per column
    if (warp == 0) {
        T s2 = T(0);
        for (int r = lane; r < n; r += 32) s2 = fma(Vs[r], Vs[r], s2);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        if (lane == 0) make_reflector(Vs, 0, s2, bet);
    }
    __syncthreads();
    for (int c = 0; c < n - 1; ++c) {
        qr_step_at<T, NB>(2 * (c >> 4), Vs, bet, ldv, n, c, warp, W, lane);
        __syncthreads();
    }
    // Q = H_0 H_1 ... H_{n-1}; its column j is H_0 ... H_j e_j (the later
    // reflectors leave e_j alone).  A warp takes four consecutive columns (a
    // group of 8 lanes each, in registers) and applies the reflectors from
    // the last column's down to 0; the groups go out largest first (their
    // work grows with their columns) from a shared counter.
    T* Qk = Q + (size_t)k * n * n;
    const int ng = (n + 3) / 4;
    for (;;) {
        int idx = 0;
        if (lane == 0) idx = atomicAdd(&s_next, 1);
        idx = __shfl_sync(0xffffffffu, idx, 0);
        if (idx >= ng) break;
        const int g0 = 4 * (ng - 1 - idx);
        const int j = g0 + sg;
        T qv[NB];
#pragma unroll
        for (int i = 0; i < NB; ++i) qv[i] = (8 * i + l8 == j) ? T(1) : T(0);
        const int cmax = g0 + 3 < n - 1 ? g0 + 3 : n - 1;
        for (int seg = cmax >> 4; seg >= 0; --seg) {
            const int chi = cmax < 16 * seg + 15 ? cmax : 16 * seg + 15;
            q_apply_at<T, NB>(2 * seg, qv, Vs, bet, ldv, chi, 16 * seg, l8);
        }
        if (j < n) {
            T* qc = Qk + (size_t)j * n;
#pragma unroll
            for (int i = 0; i < NB; ++i) {
                const int r = 8 * i + l8;
                if (r < n) qc[r] = qv[i];
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        flag[k] = 1;
        wrec[k] = 0;
    }
}

// The tail of the warm-started SVT of one slice after its sweeps, on all
// SMs: CTA (t, k) takes the JT output columns j0 = JT t .. of slice k, with
// S the converged columns (s_c, m rows), A0 the oriented slice (overwritten
// by Y) and the Jacobi kernel's record (coef, recovery scale, rank, kept
// columns; tail_info_stride):
//   R = S^T A0[:, tile]                         (n x JT, in shared memory)
//   V[j, rank_c] = R[c, j] / (d_c |s_c|^2)      (the recovered right vectors)
//   Y[:, tile] = sum_q S[:, kidx_q] coef_q R[kidx_q, tile]
// with coef_q = (1 - tau / sigma_q) / |s_q|^2: the V-free rebuild of the
// shrunk slice, Y = sum_{sigma > tau} (1 - tau / sigma) u u^T A0.  Each warp
// computes 8 output columns (lanes over rows) for one half of the rows, as
// in the A Q product, so that 12 warps share a tile.
constexpr int TJ = 48;            // output columns per CTA
constexpr int TWC = TJ / WCB;     // column tiles per CTA
constexpr int TW = 2 * TWC;       // warps per CTA: each column tile's rows in two halves
constexpr int TLD = TJ + 4;       // leading dimension of the row-major tiles (16-byte rows)

// shared memory: S as the Jacobi kernel laid it out (ldA rows per column), the
// A0 tile (later the Y tile) and the R tile (32 MR rows of TLD), then per
// column the recovery scale and rank and per kept column its coef and index
__host__ __device__ inline size_t tail_smem_floats(int n, int ldA, int npad, int mrc, int mrr)
{
    return ((size_t)n * ldA + 3) / 4 * 4 + (size_t)32 * mrr * TLD + (size_t)32 * mrc * TLD + 4 * (size_t)npad;
}

template <int MRC, int MRR>
__global__ void __launch_bounds__(32 * TW) warm_tail_kernel(float* __restrict__ data, int64_t n1, int64_t n2, int m,
                                                            int n, int tr, int ldA, int npad, size_t stride,
                                                            const float* __restrict__ S, const float* __restrict__ info,
                                                            float* __restrict__ V, int* __restrict__ wrec,
                                                            const AdmmCtl* __restrict__ ctl)
{
    if (ctl && ctl->done) return;
    const int t = blockIdx.x, k = blockIdx.y;
    const int j0 = t * TJ;
    if (j0 >= n) return;
    const int jn = n - j0 < TJ ? n - j0 : TJ;
    const float* inf = info + (size_t)k * tail_info_stride(npad);
    const int* iinf = reinterpret_cast<const int*>(inf);
    const int keep = iinf[4 * npad], hasv = iinf[4 * npad + 1];
    float* src = data + (size_t)k * n1 * n2;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    auto at = [&](int r, int j) -> float& {  // element (r, j) of the oriented slice
        return tr ? src[(size_t)j + (size_t)n1 * r] : src[(size_t)r + (size_t)n1 * j];
    };
    if (!hasv && keep == 0) {  // a slice without sweeps keeps nothing: Y = 0
        for (int e = tid; e < m * jn; e += 32 * TW) {
            const int r = tr ? e / jn : e % m, j = tr ? e % jn : e / m;
            at(r, j0 + j) = 0.0f;
        }
        return;
    }
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lds = ldA;  // rows m .. ldA - 1 of the Jacobi kernel's columns are zero, and ldA >= 32 MRR
    float* Ss = reinterpret_cast<float*>(smem_raw);                // column c at Ss + c * lds
    float* At = Ss + ((size_t)n * lds + 3) / 4 * 4;                // A0 tile, row r at At + r * TLD (rows m.., columns jn.. zero)
    float* Rt = At + (size_t)32 * MRR * TLD;                       // R tile, row c at Rt + c * TLD
    float* cq = Rt + (size_t)32 * MRC * TLD;                       // coef of the kept columns
    int* kq = reinterpret_cast<int*>(cq + npad);                   // the kept columns
    float* rsm = cq + 2 * npad;                                    // recovery scale by column
    int* rkm = reinterpret_cast<int*>(cq + 3 * npad);              // rank by column
    // S in one contiguous asynchronous copy (16-byte chunks)
    copy_to_shared(Ss, S + (size_t)k * stride, (size_t)n * lds, tid, 32 * TW);
    if (tr && ((reinterpret_cast<uintptr_t>(src) & 15u) == 0) && n1 % 4 == 0) {
        // A0 rows are source columns: TJ contiguous j per r, 16-byte chunks
        for (int e = tid; e < 32 * MRR * (TJ / 4); e += 32 * TW) {
            const int r = e / (TJ / 4), q = 4 * (e % (TJ / 4));
            float* d = At + (size_t)r * TLD + q;
            if (r < m && q + 3 < jn) cp_async16(d, src + (size_t)(j0 + q) + (size_t)n1 * r);
            else
                for (int u = 0; u < 4; ++u) d[u] = (r < m && q + u < jn) ? src[(size_t)(j0 + q + u) + (size_t)n1 * r] : 0.0f;
        }
    } else if (tr) {
        for (int e = tid; e < 32 * MRR * TJ; e += 32 * TW) {
            const int r = e / TJ, j = e % TJ;
            At[(size_t)r * TLD + j] = (r < m && j < jn) ? src[(size_t)(j0 + j) + (size_t)n1 * r] : 0.0f;
        }
    } else {  // A0 columns are source columns: eight loads in flight per thread
        load_cols(At, TLD, src + (size_t)n1 * j0, n1, m, jn, true, warp, TW, lane);
        for (int j = jn + warp; j < TJ; j += TW)
            for (int r = lane; r < m; r += 32) At[(size_t)r * TLD + j] = 0.0f;
        for (int e = tid; e < (32 * MRR - m) * TJ; e += 32 * TW) At[(size_t)(m + e / TJ) * TLD + e % TJ] = 0.0f;
    }
    for (int q = tid; q < keep; q += 32 * TW) {
        cq[q] = inf[q];
        kq[q] = iinf[3 * npad + q];
    }
    if (hasv)
        for (int c = tid; c < n; c += 32 * TW) {
            rsm[c] = inf[npad + c];
            rkm[c] = iinf[2 * npad + c];
        }
    cp_async_wait_all();
    __syncthreads();
    const int jj = (warp % TWC) * WCB;  // this warp's 8 columns of the tile
    const int h = warp / TWC;           // and its half of the rows
    {   // R = S^T A0: rows c = 32 q + lane, q in this half's blocks
        constexpr int QH = (MRC + 1) / 2;
        float acc[QH][WCB];
#pragma unroll
        for (int q = 0; q < QH; ++q)
#pragma unroll
            for (int b = 0; b < WCB; ++b) acc[q][b] = 0.0f;
        const float* sp[QH];
        bool cv[QH];
#pragma unroll
        for (int q = 0; q < QH; ++q) {
            const int c = 32 * (h * QH + q) + lane;
            cv[q] = h * QH + q < MRC && c < n;
            sp[q] = Ss + (size_t)(cv[q] ? c : 0) * lds;
        }
#pragma unroll 2
        for (int r = 0; r < m; ++r) {
            float av[QH];
#pragma unroll
            for (int q = 0; q < QH; ++q) av[q] = cv[q] ? sp[q][r] : 0.0f;
            const float4 b0 = *reinterpret_cast<const float4*>(At + (size_t)r * TLD + jj);
            const float4 b1 = *reinterpret_cast<const float4*>(At + (size_t)r * TLD + jj + 4);
            const float bv[WCB] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int q = 0; q < QH; ++q)
#pragma unroll
                for (int b = 0; b < WCB; ++b) acc[q][b] = fmaf(av[q], bv[b], acc[q][b]);
        }
        float* Vk = V + (size_t)k * n * n;
#pragma unroll
        for (int q = 0; q < QH; ++q) {
            if (!cv[q]) continue;
            const int c = 32 * (h * QH + q) + lane;
#pragma unroll
            for (int b = 0; b < WCB; ++b) Rt[(size_t)c * TLD + jj + b] = acc[q][b];
            if (hasv) {
                const float rs = rsm[c];
                float* vrow = Vk + (size_t)rkm[c] * n + j0 + jj;
#pragma unroll
                for (int b = 0; b < WCB; ++b)
                    if (jj + b < jn) vrow[b] = acc[q][b] * rs;
            }
        }
    }
    __syncthreads();
    {   // Y = sum_q coef_q s_{kidx_q} R[kidx_q, :]: rows r = 32 p + lane, p in this half's blocks
        constexpr int PH = MRR / 2;
        float acc[PH][WCB];
#pragma unroll
        for (int p = 0; p < PH; ++p)
#pragma unroll
            for (int b = 0; b < WCB; ++b) acc[p][b] = 0.0f;
#pragma unroll 2
        for (int q = 0; q < keep; ++q) {
            const int c = kq[q];
            const float w = cq[q];
            const float* col = Ss + (size_t)c * lds + 32 * h * PH + lane;
            float av[PH];
#pragma unroll
            for (int p = 0; p < PH; ++p) av[p] = col[32 * p] * w;
            const float4 g0 = *reinterpret_cast<const float4*>(Rt + (size_t)c * TLD + jj);
            const float4 g1 = *reinterpret_cast<const float4*>(Rt + (size_t)c * TLD + jj + 4);
            const float gv[WCB] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
#pragma unroll
            for (int p = 0; p < PH; ++p)
#pragma unroll
                for (int b = 0; b < WCB; ++b) acc[p][b] = fmaf(av[p], gv[b], acc[p][b]);
        }
        // the Y tile into the A0 tile's place (phase 1 is done with it)
#pragma unroll
        for (int p = 0; p < PH; ++p) {
            const int r = 32 * (h * PH + p) + lane;
            float* yrow = At + (size_t)r * TLD + jj;
            *reinterpret_cast<float4*>(yrow) = make_float4(acc[p][0], acc[p][1], acc[p][2], acc[p][3]);
            *reinterpret_cast<float4*>(yrow + 4) = make_float4(acc[p][4], acc[p][5], acc[p][6], acc[p][7]);
        }
    }
    __syncthreads();
    // coalesced stores of the Y tile
    if (tr && ((reinterpret_cast<uintptr_t>(src) & 15u) == 0) && n1 % 4 == 0) {
        for (int e = tid; e < m * (TJ / 4); e += 32 * TW) {
            const int r = e / (TJ / 4), q = 4 * (e % (TJ / 4));
            const float* y = At + (size_t)r * TLD + q;
            float* d = src + (size_t)(j0 + q) + (size_t)n1 * r;
            if (q + 3 < jn) *reinterpret_cast<float4*>(d) = *reinterpret_cast<const float4*>(y);
            else
                for (int u = 0; u < 4 && q + u < jn; ++u) d[u] = y[u];
        }
    } else if (tr) {
        for (int e = tid; e < m * TJ; e += 32 * TW) {
            const int r = e / TJ, j = e % TJ;
            if (j < jn) src[(size_t)(j0 + j) + (size_t)n1 * r] = At[(size_t)r * TLD + j];
        }
    } else {
        for (int j = warp; j < jn; j += TW)
            for (int r = lane; r < m; r += 32) src[(size_t)r + (size_t)n1 * (j0 + j)] = At[(size_t)r * TLD + j];
    }
    if (hasv && t == 0 && tid == 0) wrec[k] = 1;
}

}  // namespace

// rows per lane of the GEMM's tiles (even, 2..8) and of the QR's columns (even, 2..28)
int gemm_mr(int m) { return ((m + 31) / 32 + 1) / 2 * 2; }
int qr_nb(int n) { return ((n + 7) / 8 + 1) / 2 * 2; }

size_t warm_gemm_smem(int m, int n, int elem)
{
    return (((size_t)gemm_lda(gemm_mr(m)) * n + 3) / 4 * 4 + (size_t)n * gemm_ldq(n)) * elem;
}
size_t warm_qr_smem(int n, int elem) { return ((size_t)qr_ldv(qr_nb(n)) * n + n) * elem; }

constexpr size_t kMaxDynSmem = 227 * 1024;

bool warm_supported(const JacobiPlan& p)
{
    return p.cluster <= 1 && p.elem == 4 && p.m >= 1 && p.n >= 1 && p.m <= WMR * 32 && p.n <= WQN &&
           warm_gemm_smem(p.m, p.n, p.elem) <= kMaxDynSmem && warm_qr_smem(p.n, p.elem) <= kMaxDynSmem;
}

size_t warm_state_bytes(int64_t n3, int n, int elem)
{
    return ((size_t)n3 * n * n * elem + 255) / 256 * 256 + ((size_t)n3 * sizeof(int) + 255) / 256 * 256;
}

template <typename T>
cudaError_t launch_warm_gemm(const JacobiPlan& p, const T* data, const T* Q, const int* flag, T* w0,
                             const AdmmCtl* ctl, cudaStream_t s)
{
    if (!warm_supported(p)) return cudaErrorInvalidValue;
    const size_t sm = warm_gemm_smem(p.m, p.n, sizeof(T));
    decltype(&warm_gemm_kernel<T, 2>) kern;
    switch (gemm_mr(p.m)) {
    case 2: kern = warm_gemm_kernel<T, 2>; break;
    case 4: kern = warm_gemm_kernel<T, 4>; break;
    case 6: kern = warm_gemm_kernel<T, 6>; break;
    default: kern = warm_gemm_kernel<T, 8>; break;
    }
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const int ntile = (p.n + WCB - 1) / WCB;
    const int warps = ntile < WGM / 32 ? ntile : WGM / 32;
    const size_t stride = (size_t)p.ldA * p.nb * p.K;
    kern<<<(unsigned)p.n3, 32 * warps, sm, s>>>(data, p.n1, p.n2, p.m, p.n, p.tr, p.ldA, p.nb * p.K, stride, Q, flag,
                                               w0, ctl);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_warm_qr(const JacobiPlan& p, const T* vrec, size_t vstride, int* wrec, T* Q, int* flag,
                           const AdmmCtl* ctl, cudaStream_t s)
{
    if (!warm_supported(p)) return cudaErrorInvalidValue;
    const size_t sm = warm_qr_smem(p.n, sizeof(T));
    decltype(&warm_qr_kernel<T, 2>) kern;
    switch (qr_nb(p.n)) {
    case 2: kern = warm_qr_kernel<T, 2>; break;
    case 4: kern = warm_qr_kernel<T, 4>; break;
    case 6: kern = warm_qr_kernel<T, 6>; break;
    case 8: kern = warm_qr_kernel<T, 8>; break;
    case 10: kern = warm_qr_kernel<T, 10>; break;
    case 12: kern = warm_qr_kernel<T, 12>; break;
    case 14: kern = warm_qr_kernel<T, 14>; break;
    case 16: kern = warm_qr_kernel<T, 16>; break;
    case 18: kern = warm_qr_kernel<T, 18>; break;
    case 20: kern = warm_qr_kernel<T, 20>; break;
    case 22: kern = warm_qr_kernel<T, 22>; break;
    case 24: kern = warm_qr_kernel<T, 24>; break;
    case 26: kern = warm_qr_kernel<T, 26>; break;
    default: kern = warm_qr_kernel<T, 28>; break;
    }
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    // a warp per chunk of four columns, 4 to 16 warps
    int warps = (p.n + 3) / 4;
    warps = warps < 4 ? 4 : (warps > WQ / 32 ? WQ / 32 : warps);
    kern<<<(unsigned)p.n3, 32 * warps, sm, s>>>(vrec, p.n, vstride, wrec, Q, flag, ctl);
    return cudaGetLastError();
}

bool tail_supported(const JacobiPlan& p)
{
    if (!warm_supported(p)) return false;
    const int mrr = gemm_mr(p.m), mrc = (p.n + 31) / 32;
    return mrc <= mrr && mrc >= mrr - 1 && 32 * mrr <= p.ldA &&
           tail_smem_floats(p.n, p.ldA, p.nb * p.K, mrc, mrr) * sizeof(float) <= kMaxDynSmem;
}

template <typename T>
cudaError_t launch_warm_tail(const JacobiPlan& p, T* data, const T* S, const float* info, T* V, int* wrec,
                             const AdmmCtl* ctl, cudaStream_t s)
{
    static_assert(sizeof(T) == 4, "FP32 only");
    if (!tail_supported(p)) return cudaErrorInvalidValue;
    const int mrr = gemm_mr(p.m), mrc = (p.n + 31) / 32;
    decltype(&warm_tail_kernel<1, 2>) kern = nullptr;
    switch (mrr * 10 + mrc) {
    case 21: kern = warm_tail_kernel<1, 2>; break;
    case 22: kern = warm_tail_kernel<2, 2>; break;
    case 43: kern = warm_tail_kernel<3, 4>; break;
    case 44: kern = warm_tail_kernel<4, 4>; break;
    case 65: kern = warm_tail_kernel<5, 6>; break;
    case 66: kern = warm_tail_kernel<6, 6>; break;
    case 87: kern = warm_tail_kernel<7, 8>; break;
    case 88: kern = warm_tail_kernel<8, 8>; break;
    default: return cudaErrorInvalidValue;  // a shape whose n is far below m keeps the in-kernel tail
    }
    const size_t sm = tail_smem_floats(p.n, p.ldA, p.nb * p.K, mrc, mrr) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const size_t stride = (size_t)p.ldA * p.nb * p.K;
    const dim3 grid((unsigned)((p.n + TJ - 1) / TJ), (unsigned)p.n3);
    kern<<<grid, 32 * TW, sm, s>>>(reinterpret_cast<float*>(data), p.n1, p.n2, p.m, p.n, p.tr, p.ldA, p.nb * p.K,
                                   stride, reinterpret_cast<const float*>(S), info, reinterpret_cast<float*>(V), wrec,
                                   ctl);
    return cudaGetLastError();
}

template cudaError_t launch_warm_gemm<float>(const JacobiPlan&, const float*, const float*, const int*, float*,
                                             const AdmmCtl*, cudaStream_t);
template cudaError_t launch_warm_qr<float>(const JacobiPlan&, const float*, size_t, int*, float*, int*,
                                           const AdmmCtl*, cudaStream_t);
template cudaError_t launch_warm_tail<float>(const JacobiPlan&, float*, const float*, const float*, float*, int*,
                                             const AdmmCtl*, cudaStream_t);

}  // namespace tnn
