// Per-slice one-sided Jacobi SVD / SVT on CUDA cores (sm_103a).
//
// One CTA owns one frontal slice.  The slice is oriented so that it has at
// least as many rows as columns (m >= n; a wide slice is transposed on load)
// and kept in shared memory (or, if it does not fit, in an L2-resident global
// scratch area with the same layout).  Its n columns are cut into nb blocks of
// K columns.  A sweep is a round-robin tournament over the blocks (the circle
// method: nb - 1 steps, each pairing every block with another); in a step each
// warp loads its two blocks (2K columns, RA rows per lane) into registers and
// applies the rotations of all K x K cross pairs (plus, in the first step of a
// sweep, the pairs inside each block) in rounds of K disjoint pairs, then
// writes them back.  Column dot products are warp butterfly reductions, which
// leave bitwise-identical sums in every lane, so every branch on them is
// warp-uniform.
//
// Rotations are Rutishauser's formula (Demmel and Veselic, SIAM J. Matrix
// Anal. Appl. 13, 1992) in the scaled ("fast") form: a column is held as
// d_i * s_i, so the rotation of a pair costs two FMAs per row,
//   s_i <- s_i - t (d_j/d_i) s_j,   s_j <- s_j + t (d_i/d_j) s_i,   d <- c d,
// and squared column norms are carried along (alpha' = alpha - t gamma, beta'
// = beta + t gamma) and recomputed when a column loses most of its norm.  A
// pair is rotated when |gamma| > tol sqrt(alpha beta), tol = sqrt(m) * unit
// roundoff; a sweep without rotation ends the iteration.
//
// SVT rebuild without V (Algorithm 1's U (S - tau)_+ V^T):  with converged
// columns s_i (orthogonal, sigma_i = d_i |s_i|) and U = [s_i / |s_i|], the
// slice A0 satisfies U^T A0 = S V^T, so
//     Y = U diag((sigma - tau)_+) V^T = sum_{sigma_i > tau} (1 - tau/sigma_i)
//         / |s_i|^2 * s_i (s_i^T A0).
// Y is built column by column from the original slice (re-read from memory),
// which is then overwritten in place.  The error of this form is bounded by
// the backward error of the orthogonalisation, like the U D V^T form, and it
// needs no V: V updates would cost 2n FMAs per rotation.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <utility>

#include "tnn_internal.h"

namespace tnn {
namespace jac {

template <typename T> struct Num;
template <> struct Num<float> {
    static __device__ __forceinline__ float unit() { return 5.9604645e-8f; }      // 2^-24
    static __device__ __forceinline__ float fold() { return 9.094947e-13f; }      // 2^-40
};
template <> struct Num<double> {
    static __device__ __forceinline__ double unit() { return 1.1102230246251565e-16; }  // 2^-53
    static __device__ __forceinline__ double fold() { return 6.223015277861142e-61; }    // 2^-200
};

template <typename T> struct Vec;           // VEC consecutive rows per lane access
template <> struct Vec<float> { static constexpr int N = 2; typedef float2 V; };
template <> struct Vec<double> { static constexpr int N = 1; typedef double V; };

// IEEE round-to-nearest reciprocal (intrinsic form).
__device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp(double x) { return __drcp_rn(x); }

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Row index of register (q, v) of lane l: rows come in groups of VEC
// consecutive rows, lane-interleaved, so a warp-wide vector access touches
// 32*VEC consecutive elements.
template <typename T>
__device__ __forceinline__ int row_of(int lane, int g, int v) { return (g * 32 + lane) * Vec<T>::N + v; }

// Circle-method position for the pairs inside a block of K columns.
__host__ __device__ constexpr int wpos(int K, int r, int t) { return t == 0 ? 0 : 1 + (t - 1 + r) % (K - 1); }
__host__ __device__ constexpr int within_i(int K, int r, int p)
{
    return p < K / 2 ? wpos(K, r, p) : K + wpos(K, r, p - K / 2);
}
__host__ __device__ constexpr int within_j(int K, int r, int p)
{
    return p < K / 2 ? wpos(K, r, K - 1 - p) : K + wpos(K, r, K - 1 - (p - K / 2));
}
__host__ __device__ constexpr int cross_i(int K, int r, int p) { return p; }
__host__ __device__ constexpr int cross_j(int K, int r, int p) { return K + (p + r) % K; }

// Block at position t of the circle at step s (nb blocks; position 0 fixed).
__device__ __forceinline__ int block_at(int nb, int t, int s) { return t == 0 ? 0 : 1 + (t - 1 + s) % (nb - 1); }

struct Counters {
    int64_t pairs;
    int64_t rots;
    int recomputes;
};

// Registers of one warp: 2K columns of A (and of V when WITHV).
template <typename T, int K, int RA, bool WITHV>
struct Regs {
    T a[2 * K][RA];
    T v[WITHV ? 2 * K : 1][WITHV ? RA : 1];
    T d[2 * K];   // column scales
    T al[2 * K];  // true squared norms d^2 |s|^2
};

template <typename T, int K, int RA, bool WITHV>
__device__ __forceinline__ void recompute_norm(Regs<T, K, RA, WITHV>& R, int c)
{
    T s = T(0);
#pragma unroll
    for (int q = 0; q < RA; ++q) s = fma(R.a[c][q], R.a[c][q], s);
    s = warp_sum(s);
    R.al[c] = R.d[c] * R.d[c] * s;
}

// Rutishauser's rotation for the 2 x 2 Gram matrix [[ai, gam], [gam, aj]]:
// zeta = (aj - ai) / (2 gam), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
// c = 1 / sqrt(1 + t^2).  Written with reciprocals and reciprocal square roots
// (no division or square-root slow paths, whose calls would force the
// register-resident columns out to local memory); c gets one Newton step
// y <- y (3 - x y^2) / 2 so that c^2 (1 + t^2) = 1 to working precision.
template <typename T>
__device__ __forceinline__ void rot_params(T ai, T aj, T gam, T& t, T& c)
{
    const T zeta = (aj - ai) * (T(0.5) * rcp(gam));
    const T az = fabs(zeta);
    const T q = T(1) + az * az;
    T tt = (az > T(1e15)) ? T(0.5) * rcp(az) : rcp(az + q * rsqrt(q));
    t = copysign(tt, zeta);
    const T x = T(1) + t * t;
    T y = rsqrt(x);
    y = y * (T(1.5) - T(0.5) * x * y * y);
    c = y;
}

// Rotate columns i, j of the register set with tangent t and cosine c.
template <typename T, int K, int RA, bool WITHV>
__device__ __forceinline__ void apply_rot(Regs<T, K, RA, WITHV>& R, int i, int j, T t, T c)
{
    const T t1 = t * (R.d[j] * rcp(R.d[i]));
    const T t2 = t * (R.d[i] * rcp(R.d[j]));
#pragma unroll
    for (int q = 0; q < RA; ++q) {
        T x = R.a[i][q], y = R.a[j][q];
        R.a[i][q] = fma(-t1, y, x);
        R.a[j][q] = fma(t2, x, y);
    }
    if (WITHV) {
#pragma unroll
        for (int q = 0; q < RA; ++q) {
            T x = R.v[i][q], y = R.v[j][q];
            R.v[i][q] = fma(-t1, y, x);
            R.v[j][q] = fma(t2, x, y);
        }
    }
    R.d[i] *= c;
    R.d[j] *= c;
}

// One round: K disjoint pairs (I(p), J(p)).  The round index is a template
// parameter so that every register index below is a compile-time constant.
template <typename T, int K, int RA, bool WITHV, bool CROSS, int r>
__device__ __forceinline__ void do_round(Regs<T, K, RA, WITHV>& R, const T tol, Counters& cnt)
{
    T g[K];
#pragma unroll
    for (int p = 0; p < K; ++p) {
        const int i = CROSS ? cross_i(K, r, p) : within_i(K, r, p);
        const int j = CROSS ? cross_j(K, r, p) : within_j(K, r, p);
        T s = T(0);
#pragma unroll
        for (int q = 0; q < RA; ++q) s = fma(R.a[i][q], R.a[j][q], s);
        g[p] = s;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int p = 0; p < K; ++p) g[p] += __shfl_xor_sync(0xffffffffu, g[p], o);
    cnt.pairs += K;
#pragma unroll
    for (int p = 0; p < K; ++p) {
        const int i = CROSS ? cross_i(K, r, p) : within_i(K, r, p);
        const int j = CROSS ? cross_j(K, r, p) : within_j(K, r, p);
        const T ai = R.al[i], aj = R.al[j];
        const T gam = (R.d[i] * R.d[j]) * g[p];
        if (fabs(gam) * rsqrt(ai) * rsqrt(aj) > tol) {  // warp-uniform (false for a zero column)
            T t, c;
            rot_params(ai, aj, gam, t, c);
            apply_rot(R, i, j, t, c);
            const T tg = t * gam;
            R.al[i] = ai - tg;
            R.al[j] = aj + tg;
            // the carried norm loses accuracy when a column loses most of its norm
            if (R.al[i] < T(0.25) * ai) { recompute_norm(R, i); ++cnt.recomputes; }
            if (R.al[j] < T(0.25) * aj) { recompute_norm(R, j); ++cnt.recomputes; }
            ++cnt.rots;
        }
    }
}

template <typename T, int K, int RA, bool WITHV, bool CROSS, int... Rs>
__device__ __forceinline__ void do_rounds(Regs<T, K, RA, WITHV>& R, const T tol, Counters& cnt,
                                          std::integer_sequence<int, Rs...>)
{
    (do_round<T, K, RA, WITHV, CROSS, Rs>(R, tol, cnt), ...);
}

template <typename T, int K, int RA, bool WITHV>
__device__ __forceinline__ void load_cols(Regs<T, K, RA, WITHV>& R, const T* Aw, const T* Vw, const T* dsc,
                                          int ldA, int bI, int bJ, int lane)
{
    typedef typename Vec<T>::V VT;
    constexpr int VN = Vec<T>::N;
#pragma unroll
    for (int c = 0; c < 2 * K; ++c) {
        const int col = (c < K) ? bI * K + c : bJ * K + (c - K);
        const T* src = Aw + (size_t)col * ldA;
#pragma unroll
        for (int g = 0; g < RA / VN; ++g) {
            VT x = *reinterpret_cast<const VT*>(src + row_of<T>(lane, g, 0));
            const T* xs = reinterpret_cast<const T*>(&x);
#pragma unroll
            for (int v = 0; v < VN; ++v) R.a[c][g * VN + v] = xs[v];
        }
        if (WITHV) {
            const T* vs = Vw + (size_t)col * ldA;
#pragma unroll
            for (int g = 0; g < RA / VN; ++g) {
                VT x = *reinterpret_cast<const VT*>(vs + row_of<T>(lane, g, 0));
                const T* xs = reinterpret_cast<const T*>(&x);
#pragma unroll
                for (int v = 0; v < VN; ++v) R.v[c][g * VN + v] = xs[v];
            }
        }
        R.d[c] = dsc[col];
    }
    T s[2 * K];
#pragma unroll
    for (int c = 0; c < 2 * K; ++c) {
        T acc = T(0);
#pragma unroll
        for (int q = 0; q < RA; ++q) acc = fma(R.a[c][q], R.a[c][q], acc);
        s[c] = acc;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int c = 0; c < 2 * K; ++c) s[c] += __shfl_xor_sync(0xffffffffu, s[c], o);
#pragma unroll
    for (int c = 0; c < 2 * K; ++c) R.al[c] = R.d[c] * R.d[c] * s[c];
}

template <typename T, int K, int RA, bool WITHV>
__device__ __forceinline__ void store_cols(Regs<T, K, RA, WITHV>& R, T* Aw, T* Vw, T* dsc, int ldA, int bI, int bJ,
                                           int lane)
{
    typedef typename Vec<T>::V VT;
    constexpr int VN = Vec<T>::N;
#pragma unroll
    for (int c = 0; c < 2 * K; ++c) {
        const int col = (c < K) ? bI * K + c : bJ * K + (c - K);
        if (R.d[c] < Num<T>::fold()) {  // fold a tiny scale into the stored column
#pragma unroll
            for (int q = 0; q < RA; ++q) R.a[c][q] *= R.d[c];
            if (WITHV) {
#pragma unroll
                for (int q = 0; q < RA; ++q) R.v[c][q] *= R.d[c];
            }
            R.d[c] = T(1);
        }
        T* dst = Aw + (size_t)col * ldA;
#pragma unroll
        for (int g = 0; g < RA / VN; ++g) {
            VT x;
            T* xs = reinterpret_cast<T*>(&x);
#pragma unroll
            for (int v = 0; v < VN; ++v) xs[v] = R.a[c][g * VN + v];
            *reinterpret_cast<VT*>(dst + row_of<T>(lane, g, 0)) = x;
        }
        if (WITHV) {
            T* vd = Vw + (size_t)col * ldA;
#pragma unroll
            for (int g = 0; g < RA / VN; ++g) {
                VT x;
                T* xs = reinterpret_cast<T*>(&x);
#pragma unroll
                for (int v = 0; v < VN; ++v) xs[v] = R.v[c][g * VN + v];
                *reinterpret_cast<VT*>(vd + row_of<T>(lane, g, 0)) = x;
            }
        }
        if (lane == 0) dsc[col] = R.d[c];
    }
}

template <typename T>
struct KArgs {
    T* data;            // SVT: slices in/out;  SVD: slices in
    int64_t n1, n2, n3;
    int m, n, tr, nb, ldA;
    double tau;
    const AdmmCtl* ctl;
    int max_sweeps;
    T* work;            // global scratch (working copies when not in shared memory)
    SliceStats* stats;
    T* U;               // SVD outputs
    T* S;
    T* V;
};

// Shared-memory carve-up (bytes) for a launch.
__host__ __device__ inline size_t smem_small_bytes(int npad, int W, int elem)
{
    // dsc, sig, cf (elem each), kidx (int), gbuf W x npad (elem), rank (int)
    size_t b = (size_t)npad * (3 * elem + 8) + (size_t)W * npad * elem;
    return (b + 255) & ~(size_t)255;
}

// Threads per CTA the register file allows for one instantiation: the 2K
// register-resident columns (twice that with V) plus about 48 values of
// scales, norms and angle temporaries, plus addressing.
template <typename T, int K, int RA, bool WITHV>
struct Bound {
    static constexpr int regs = (2 * K * RA * (WITHV ? 2 : 1) + 48) * (int)(sizeof(T) / 4) + 16;
    static constexpr int t = (65536 / regs) / 32 * 32;
    static constexpr int value = t > 1024 ? 1024 : t;
};

template <typename T, int K, int RA, bool SMEM, bool WITHV>
__global__ void __launch_bounds__(Bound<T, K, RA, WITHV>::value) jacobi_kernel(KArgs<T> a)
{
    if (a.ctl && a.ctl->done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int W = blockDim.x >> 5;
    const int nthr = blockDim.x;
    const int slice = blockIdx.x;
    const int m = a.m, n = a.n, nb = a.nb, ldA = a.ldA, tr = a.tr;
    const int npad = nb * K;
    const int64_t n1 = a.n1;
    const size_t wsz = (size_t)ldA * npad;

    T* Aw;
    T* Vw = nullptr;
    unsigned char* rest;
    if (SMEM) {
        Aw = reinterpret_cast<T*>(smem_raw);
        if (WITHV) Vw = Aw + wsz;
        rest = smem_raw + (WITHV ? 2 : 1) * ((wsz * sizeof(T) + 255) & ~(size_t)255);
    } else {
        Aw = a.work + (size_t)slice * (WITHV ? 2 : 1) * wsz;
        if (WITHV) Vw = Aw + wsz;
        rest = smem_raw;
    }
    T* dsc = reinterpret_cast<T*>(rest);
    T* sig = dsc + npad;
    T* cf = sig + npad;
    int* kidx = reinterpret_cast<int*>(cf + npad);
    int* rank = kidx + npad;
    T* gbuf = reinterpret_cast<T*>(rank + npad);
    __shared__ int s_rot, s_keep, s_nonfinite;
    __shared__ double s_nuc;
    __shared__ unsigned long long s_pairs, s_rots;

    T* src = a.data + (size_t)slice * n1 * a.n2;

    // ---- load the oriented slice; pad rows and columns with zeros
    for (size_t e = tid; e < wsz; e += nthr) Aw[e] = T(0);
    if (WITHV)
        for (size_t e = tid; e < wsz; e += nthr) {
            int c = (int)(e / ldA), r = (int)(e % ldA);
            Vw[e] = (r == c && c < n) ? T(1) : T(0);
        }
    __syncthreads();
    const int64_t S = n1 * a.n2;
    for (int64_t e = tid; e < S; e += nthr) {
        int i = (int)(e % n1), j = (int)(e / n1);
        // oriented (row, col): (i, j) if n1 >= n2 else (j, i)
        int r = tr ? j : i, c = tr ? i : j;
        Aw[(size_t)c * ldA + r] = src[e];
    }
    for (int c = tid; c < npad; c += nthr) dsc[c] = T(1);
    if (tid == 0) { s_pairs = 0; s_rots = 0; s_nonfinite = 0; s_nuc = 0.0; s_keep = 0; }
    __syncthreads();

    // ---- sweeps
    const T tol = sqrt((T)m) * Num<T>::unit();
    Counters cnt{0, 0, 0};
    int sweeps = 0, converged = 0;
    const int max_sweeps = a.max_sweeps > 0 ? a.max_sweeps : 30;
    const int npairs = nb / 2;
    while (sweeps < max_sweeps) {
        if (tid == 0) s_rot = 0;
        __syncthreads();
        const int64_t rot0 = cnt.rots;
        for (int step = 0; step < nb - 1; ++step) {
            for (int pr = warp; pr < npairs; pr += W) {
                const int bI = block_at(nb, pr, step), bJ = block_at(nb, nb - 1 - pr, step);
                Regs<T, K, RA, WITHV> R;
                load_cols<T, K, RA, WITHV>(R, Aw, Vw, dsc, ldA, bI, bJ, lane);
                if (step == 0)
                    do_rounds<T, K, RA, WITHV, false>(R, tol, cnt, std::make_integer_sequence<int, K - 1>{});
                do_rounds<T, K, RA, WITHV, true>(R, tol, cnt, std::make_integer_sequence<int, K>{});
                store_cols<T, K, RA, WITHV>(R, Aw, Vw, dsc, ldA, bI, bJ, lane);
            }
            __syncthreads();
        }
        if (lane == 0 && cnt.rots != rot0) atomicAdd(&s_rot, (int)(cnt.rots - rot0));
        __syncthreads();
        const int nrot = s_rot;
        ++sweeps;
        __syncthreads();
        if (nrot == 0) { converged = 1; break; }
    }
    if (lane == 0) {
        atomicAdd(&s_pairs, (unsigned long long)cnt.pairs);
        atomicAdd(&s_rots, (unsigned long long)cnt.rots);
    }

    // ---- singular values sigma_c = d_c |s_c| (warp per column)
    for (int c = warp; c < npad; c += W) {
        const T* col = Aw + (size_t)c * ldA;
        T s = T(0);
        for (int r = lane; r < ldA; r += 32) s = fma(col[r], col[r], s);
        s = warp_sum(s);
        if (lane == 0) {
            T sg = dsc[c] * sqrt(s);
            sig[c] = sg;
            cf[c] = s;  // |s_c|^2 for now
            if (!isfinite(sg)) s_nonfinite = 1;
        }
    }
    __syncthreads();

    const T tau = a.ctl ? (T)(1.0 / a.ctl->beta) : (T)a.tau;

    if (!WITHV) {
        // ---- SVT: kept columns (sigma > tau) and their coefficients
        if (tid == 0) {
            int kk = 0;
            double nuc = 0.0;
            for (int c = 0; c < npad; ++c) {
                T sg = sig[c];
                if (sg > tau && cf[c] > T(0)) {
                    kidx[kk] = c;
                    cf[kk] = (T(1) - tau / sg) / cf[c];
                    nuc += (double)(sg - tau);
                    ++kk;
                }
            }
            s_keep = kk;
            s_nuc = nuc;
        }
        __syncthreads();
        const int keep = s_keep;
        // ---- rebuild Y = sum_q cf_q s_q (s_q^T a0_j), column j at a time, in place
        T* gb = gbuf + (size_t)warp * npad;
        for (int j = warp; j < n; j += W) {
            T x[RA];
#pragma unroll
            for (int q = 0; q < RA; ++q) {
                const int r = row_of<T>(lane, q / Vec<T>::N, q % Vec<T>::N);
                x[q] = (r < m) ? (tr ? src[(size_t)j + (size_t)n1 * r] : src[(size_t)r + (size_t)n1 * j]) : T(0);
            }
            // coefficients g_q = cf_q * (s_q . a0_j), four at a time
            for (int q0 = 0; q0 < keep; q0 += 4) {
                T g[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    T s = T(0);
                    if (q0 + u < keep) {
                        const T* col = Aw + (size_t)kidx[q0 + u] * ldA;
#pragma unroll
                        for (int q = 0; q < RA; ++q) s = fma(col[row_of<T>(lane, q / Vec<T>::N, q % Vec<T>::N)], x[q], s);
                    }
                    g[u] = s;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                    for (int u = 0; u < 4; ++u) g[u] += __shfl_xor_sync(0xffffffffu, g[u], o);
                if (lane < 4 && q0 + lane < keep) gb[q0 + lane] = g[lane] * cf[q0 + lane];
            }
            __syncwarp();
            T y[RA];
#pragma unroll
            for (int q = 0; q < RA; ++q) y[q] = T(0);
            for (int u = 0; u < keep; ++u) {
                const T coef = gb[u];
                const T* col = Aw + (size_t)kidx[u] * ldA;
#pragma unroll
                for (int q = 0; q < RA; ++q) y[q] = fma(coef, col[row_of<T>(lane, q / Vec<T>::N, q % Vec<T>::N)], y[q]);
            }
#pragma unroll
            for (int q = 0; q < RA; ++q) {
                const int r = row_of<T>(lane, q / Vec<T>::N, q % Vec<T>::N);
                if (r < m) {
                    if (tr) src[(size_t)j + (size_t)n1 * r] = y[q];
                    else src[(size_t)r + (size_t)n1 * j] = y[q];
                }
            }
            __syncwarp();
        }
    } else {
        // ---- SVD outputs, columns ordered by descending sigma (ties by index)
        for (int c = tid; c < n; c += nthr) {
            int rk = 0;
            const T sc = sig[c];
            for (int o = 0; o < n; ++o) {
                const T so = sig[o];
                rk += (so > sc || (so == sc && o < c)) ? 1 : 0;
            }
            rank[c] = rk;
        }
        __syncthreads();
        const int r = n;  // thin: r = min(n1, n2) = n
        const int64_t n2 = a.n2;
        for (int c = warp; c < n; c += W) {
            const int pos = rank[c];
            const T nrm = sqrt(cf[c]);
            const T inv = nrm > T(0) ? T(1) / nrm : T(0);
            const T* col = Aw + (size_t)c * ldA;
            const T* vcol = Vw + (size_t)c * ldA;
            const T dv = dsc[c];
            // U_A (m rows) and V_A (n rows); slice U = U_A, V = V_A unless transposed
            T* Uo = tr ? a.V : a.U;
            T* Vo = tr ? a.U : a.V;
            const int64_t ldU = tr ? n2 : n1;   // rows of the output holding U_A
            const int64_t ldV = tr ? n1 : n2;
            T* ucol = Uo + (size_t)slice * ldU * r + (size_t)pos * ldU;
            T* vout = Vo + (size_t)slice * ldV * r + (size_t)pos * ldV;
            for (int q = lane; q < m; q += 32) ucol[q] = col[q] * inv;
            for (int q = lane; q < n; q += 32) vout[q] = vcol[q] * dv;
            if (lane == 0) a.S[(size_t)slice * r + pos] = sig[c];
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
        st.kept = WITHV ? n : s_keep;
        a.stats[slice] = st;
    }
}

}  // namespace jac
}  // namespace tnn
