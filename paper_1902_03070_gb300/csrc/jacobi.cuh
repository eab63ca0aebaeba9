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

#include "async_copy.cuh"
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

// Reciprocal: the hardware's approximate FP32 reciprocal (rcp.approx.f32,
// subnormals kept), within about one unit in the last place; FP64 is the IEEE
// round-to-nearest intrinsic.
__device__ __forceinline__ float rcp(float x)
{
    float y;
    asm("rcp.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ double rcp(double x) { return __drcp_rn(x); }

// sum_q x[q] y[q] over a lane's R rows as two FMA chains (even and odd rows)
// added at the end: half the dependent chain of one accumulator.
template <typename T, int R>
__device__ __forceinline__ T dot_rows(const T (&x)[R], const T (&y)[R])
{
    T e = T(0), o = T(0);
#pragma unroll
    for (int q = 0; q + 1 < R; q += 2) {
        e = fma(x[q], y[q], e);
        o = fma(x[q + 1], y[q + 1], o);
    }
    if (R % 2) e = fma(x[R - 1], y[R - 1], e);
    return e + o;
}

// Lane layout.  A block pair is owned by a group of L lanes (L = 16: two
// groups per warp; L = 32: one).  Register q of group lane hl holds row
//   ((q / VN) * L + hl) * VN + q % VN,
// VN consecutive rows per vector access (2 for float when R is even).
template <typename T, int R>
struct VecOf {
    static constexpr int N = (sizeof(T) == 4 && R % 2 == 0) ? 2 : 1;
};
template <typename T, int N> struct VecT;
template <> struct VecT<float, 2> { typedef float2 V; };
template <> struct VecT<float, 1> { typedef float V; };
template <> struct VecT<double, 1> { typedef double V; };

template <int L, int VN>
__device__ __forceinline__ int grow(int hl, int q) { return ((q / VN) * L + hl) * VN + q % VN; }

constexpr unsigned FULL = 0xffffffffu;

// Sum over the L lanes of a group; every lane of the group gets the same bits.
template <int L, typename T>
__device__ __forceinline__ T group_sum(T v)
{
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// Reduce-scatter of K partial sums over the L lanes of a group: the result in
// lane hl is the group sum of g[hl / (L / K)], bitwise identical across the
// L / K lanes that hold it.  Each halving stage sends half of the live values
// to the partner lane, so K sums cost about K + log2(L / K) shuffles.
template <typename T, int K, int L>
__device__ __forceinline__ T reduce_scatter(const T (&g)[K], int hl)
{
    constexpr int G = L / K;
    T v[K];
#pragma unroll
    for (int p = 0; p < K; ++p) v[p] = g[p];
#pragma unroll
    for (int h = L / 2, c = K; h >= G; h >>= 1, c >>= 1) {
        const bool up = (hl & h) != 0;
#pragma unroll
        for (int t = 0; t < c / 2; ++t) {
            const T send = up ? v[t] : v[t + c / 2];
            const T keep = up ? v[t + c / 2] : v[t];
            v[t] = keep + __shfl_xor_sync(FULL, send, h);
        }
    }
    T s = v[0];
#pragma unroll
    for (int h = G / 2; h >= 1; h >>= 1) s += __shfl_xor_sync(FULL, s, h);
    return s;
}

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
template <bool CROSS>
__host__ __device__ constexpr int pair_i(int K, int r, int p) { return CROSS ? cross_i(K, r, p) : within_i(K, r, p); }
template <bool CROSS>
__host__ __device__ constexpr int pair_j(int K, int r, int p) { return CROSS ? cross_j(K, r, p) : within_j(K, r, p); }

// Block at position t of the circle at step s (nb blocks; position 0 fixed).
__device__ __forceinline__ int block_at(int nb, int t, int s)
{
    if (t == 0) return 0;
    int v = t - 1 + s;  // < 2 (nb - 1): one conditional subtraction instead of a modulo
    if (v >= nb - 1) v -= nb - 1;
    return 1 + v;
}

// pairs visited, rotations applied, and rotations of pairs whose relative
// off-diagonality exceeded twice the threshold (only those keep a sweep from
// counting as the last one: right after a rotation a pair sits at rounding
// level, about the threshold itself, and could otherwise be rotated again
// and again).
struct Counters {
    int pairs;
    int rots;
    int big;
    int bigll;  // the part of big whose two columns both had squared norms below tau^2
    int wide;   // rotations applied with |gamma| / sqrt(alpha beta) or |t| above theta (the small-rotation stop)
    float cbig, tbig, tall;  // sweep log: largest |gamma| / sqrt(alpha beta) and |t| of the big rotations, |t| of all
};

// Registers of one group: 2K columns of A (and of V when WITHV), with the
// column scales d and the true squared norms al = d^2 |s|^2 (the same value
// in every lane of the group).
template <typename T, int K, int R, bool WITHV>
struct Regs {
    T a[2 * K][R];
    T v[WITHV ? 2 * K : 1][WITHV ? R : 1];
    T d[2 * K];
    T al[2 * K];
};

// Rutishauser's rotation for the Gram matrix [[ai, gam], [gam, aj]] of a
// column pair: zeta = (aj - ai) / (2 gam), t = sign(zeta) / (|zeta| +
// sqrt(1 + zeta^2)), c = 1 / sqrt(1 + t^2); reciprocal and reciprocal-square-
// root forms (no division or square-root slow paths), and one Newton step
// y <- y (3 - x y^2) / 2 on c so that c^2 (1 + t^2) = 1 to working precision.
//
// The tangent is evaluated as t = 2 gam / (D + sign(D) sqrt(D^2 + 4 gam^2))
// with D = aj - ai (the same value: multiply Rutishauser's numerator and
// denominator by 2 |gam|), which needs one reciprocal square root and one
// reciprocal; if D^2 + 4 gam^2 overflows, the zeta form is used.
template <typename T>
__device__ __forceinline__ void rot_params(T ai, T aj, T gam, T& t, T& c)
{
    const T D = aj - ai, g2 = gam + gam;
    const T h2 = fma(D, D, g2 * g2);
    if (h2 < T(INFINITY)) {
        const T h = h2 * rsqrt(h2);
        t = g2 * rcp(D + copysign(h, D));
    } else {
        const T zeta = D * (T(0.5) * rcp(gam));
        const T az = fabs(zeta);
        const T q = T(1) + az * az;
        const T tt = (az > T(1e15)) ? T(0.5) * rcp(az) : rcp(az + q * rsqrt(q));
        t = copysign(tt, zeta);
    }
    const T x = T(1) + t * t;
    T y = rsqrt(x);
    y = y * (T(1.5) - T(0.5) * x * y * y);
    c = y;
}

// Factors of the scaled rotation for tangent t: t1 = t d_j / d_i, t2 = t d_i /
// d_j and c = 1 / sqrt(1 + t^2).  The angle t itself need not be accurate
// (any t gives an orthogonal rotation), but c must belong to the t that is
// applied and t1, t2 must match the scales: their errors act as a column
// scaling that builds up in d over the thousands of rotations a column takes
// part in, and d |s| is the singular value the shrinkage uses.  What matters
// is bias: a systematic error adds up linearly over the rotations, a random
// one only as their square root.  Measured on GB300 over 2^24 random
// arguments (bias / RMS in units of the last place): c from the approximate
// reciprocal square root and one Newton step +0.08 / 0.46 (without the step
// +0.14 / 0.76), correctly rounded +0.01 / 0.35; t1, t2 from the approximate
// reciprocal refined by one FMA Newton step 0.00 / 0.73, correctly rounded
// division 0.00 / 0.60.  So FP32 takes the correctly rounded reciprocal square
// root for c and the refined reciprocal for t1, t2 (with the biased c the
// t-SVT error reached 1e-5..3e-5 of ||Y|| where tau is large); FP64 the IEEE
// reciprocal.
__device__ __forceinline__ void rot_factors(float t, float di, float dj, float& t1, float& t2, float& c)
{
    float ri = rcp(di), rj = rcp(dj);
    ri = fmaf(ri, fmaf(-di, ri, 1.0f), ri);
    rj = fmaf(rj, fmaf(-dj, rj, 1.0f), rj);
    t1 = (t * dj) * ri;
    t2 = (t * di) * rj;
    c = __frsqrt_rn(fmaf(t, t, 1.0f));
}
__device__ __forceinline__ void rot_factors(double t, double di, double dj, double& t1, double& t2, double& c)
{
    const double rd = rcp(di * dj);
    t1 = t * (dj * dj) * rd;
    t2 = t * (di * di) * rd;
    c = 1.0 / sqrt(fma(t, t, 1.0));
}

// The same rotation evaluated in FP64 (from FP32 or FP64 column sums): the
// FP64-angle option of the FP32 kernels.
__device__ __forceinline__ void rot_params64(double ai, double aj, double gam, double& t, double& c)
{
    const double D = aj - ai, g2 = gam + gam;
    const double h = sqrt(fma(D, D, g2 * g2));
    t = g2 / (D + copysign(h, D));
    c = 1.0 / sqrt(fma(t, t, 1.0));
}

// Relative off-diagonality |gam| / sqrt(ai aj) of a pair in FP64; NaN (no
// rotation) for a zero column or a carried norm gone negative, as in the
// FP32 form.
__device__ __forceinline__ double off64(double ai, double aj, double gam)
{
    return (ai > 0.0 && aj > 0.0) ? fabs(gam) / sqrt(ai * aj) : __longlong_as_double(0x7ff8000000000000ll);
}

template <typename T, int K, int R, int L, bool WITHV>
__device__ __forceinline__ void recompute_norm(Regs<T, K, R, WITHV>& S, int c)
{
    T s = T(0);
#pragma unroll
    for (int q = 0; q < R; ++q) s = fma(S.a[c][q], S.a[c][q], s);
    s = group_sum<L>(s);
    S.al[c] = S.d[c] * S.d[c] * s;
}

// One round: K disjoint pairs (pair_i(p), pair_j(p)) of the 2K register
// columns.  Each of the K slots of L/K lanes computes one pair's rotation and
// the group learns all K of them by shuffles.
// lm: the group's 2K column flags (bit c: register column c belongs to the
// sweep's set of small columns); a pair of two flagged columns is left alone.
template <typename T, int K, int R, int L, bool WITHV, bool CROSS, int r>
__device__ __forceinline__ void do_round(Regs<T, K, R, WITHV>& S, const T tol, const int hl, Counters& cnt,
                                         const unsigned lm, const bool a64, const T tau2, const T theta)
{
    constexpr int G = L / K;
    const int slot = hl / G;
    T g[K];
#pragma unroll
    for (int p = 0; p < K; ++p) {
        const int i = pair_i<CROSS>(K, r, p), j = pair_j<CROSS>(K, r, p);
        g[p] = dot_rows<T, R>(S.a[i], S.a[j]);
    }
    const T gs = reduce_scatter<T, K, L>(g, hl);
    // this slot's pair state
    T ai = S.al[pair_i<CROSS>(K, r, 0)], aj = S.al[pair_j<CROSS>(K, r, 0)];
    T di = S.d[pair_i<CROSS>(K, r, 0)], dj = S.d[pair_j<CROSS>(K, r, 0)];
    unsigned lo = (lm >> pair_i<CROSS>(K, r, 0)) & (lm >> pair_j<CROSS>(K, r, 0)) & 1u;
#pragma unroll
    for (int p = 1; p < K; ++p) {
        const bool me = slot == p;
        ai = me ? S.al[pair_i<CROSS>(K, r, p)] : ai;
        aj = me ? S.al[pair_j<CROSS>(K, r, p)] : aj;
        di = me ? S.d[pair_i<CROSS>(K, r, p)] : di;
        dj = me ? S.d[pair_j<CROSS>(K, r, p)] : dj;
        lo = me ? ((lm >> pair_i<CROSS>(K, r, p)) & (lm >> pair_j<CROSS>(K, r, p)) & 1u) : lo;
    }
    const T gam = (di * dj) * gs;
    T t1 = T(0), t2 = T(0), cc = T(1), tg = T(0);
    bool bigp, rotp, widep = false;
    if (a64) {
        const double off = lo ? 0.0 : off64((double)ai, (double)aj, (double)gam);
        bigp = off > 2.0 * (double)tol;
        rotp = off > (double)tol;
        widep = off > (double)theta;
        if (bigp) cnt.cbig = fmaxf(cnt.cbig, (float)off);
    } else {
        const T off = lo ? T(0) : fabs(gam) * rsqrt(ai) * rsqrt(aj);
        bigp = off > T(2) * tol;
        rotp = off > tol;  // false for a zero column (0 * inf = NaN) and for a carried norm gone negative
        widep = off > theta;
        if (bigp) cnt.cbig = fmaxf(cnt.cbig, (float)off);
    }
    if (rotp) {
        if (a64) {
            double t, c;
            rot_params64((double)ai, (double)aj, (double)gam, t, c);
            t1 = (T)(t * ((double)dj / (double)di));
            t2 = (T)(t * ((double)di / (double)dj));
            cc = (T)c;
            tg = (T)(t * (double)gam);
            widep = widep || fabs(t) > (double)theta;
            cnt.tall = fmaxf(cnt.tall, (float)fabs(t));
            if (bigp) cnt.tbig = fmaxf(cnt.tbig, (float)fabs(t));
        } else {
            T t, c;
            rot_params(ai, aj, gam, t, c);
            rot_factors(t, di, dj, t1, t2, cc);
            tg = t * gam;
            widep = widep || fabs(t) > theta;
            cnt.tall = fmaxf(cnt.tall, (float)fabs(t));
            if (bigp) cnt.tbig = fmaxf(cnt.tbig, (float)fabs(t));
        }
    } else {
        widep = false;
    }
    T T1[K], T2[K], CC[K], TG[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
        T1[q] = __shfl_sync(FULL, t1, q * G, L);
        T2[q] = __shfl_sync(FULL, t2, q * G, L);
        CC[q] = __shfl_sync(FULL, cc, q * G, L);
        TG[q] = __shfl_sync(FULL, tg, q * G, L);
    }
    if (bigp && hl % G == 0) {
        ++cnt.big;
        if (ai < tau2 && aj < tau2) ++cnt.bigll;
    }
    if (widep && hl % G == 0) ++cnt.wide;
    if (hl == 0) cnt.pairs += K;
    unsigned need = 0;
#pragma unroll
    for (int q = 0; q < K; ++q) {
        const int i = pair_i<CROSS>(K, r, q), j = pair_j<CROSS>(K, r, q);
        const bool rot = (T1[q] != T(0)) || (T2[q] != T(0));
        if (hl == 0) cnt.rots += rot ? 1 : 0;
        if (__any_sync(FULL, rot)) {
#pragma unroll
            for (int k = 0; k < R; ++k) {
                const T x = S.a[i][k], y = S.a[j][k];
                S.a[i][k] = fma(-T1[q], y, x);
                S.a[j][k] = fma(T2[q], x, y);
            }
            if (WITHV) {
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    const T x = S.v[i][k], y = S.v[j][k];
                    S.v[i][k] = fma(-T1[q], y, x);
                    S.v[j][k] = fma(T2[q], x, y);
                }
            }
        }
        const T oi = S.al[i], oj = S.al[j];
        S.d[i] *= CC[q];
        S.d[j] *= CC[q];
        S.al[i] = oi - TG[q];
        S.al[j] = oj + TG[q];
        // a carried norm loses accuracy when the column loses most of its norm
        if (S.al[i] < T(0.25) * oi) need |= 1u << i;
        if (S.al[j] < T(0.25) * oj) need |= 1u << j;
    }
    if (__any_sync(FULL, need != 0)) {
#pragma unroll
        for (int c = 0; c < 2 * K; ++c)
            if (__any_sync(FULL, (need >> c) & 1u)) recompute_norm<T, K, R, L, WITHV>(S, c);
    }
}

// Column state of one slot of L/K lanes during the cross rounds of a step:
// the slot owns column I_p of the first block for the whole step and, in
// round r, column J_{(p+r) mod K} of the second block, whose state moves one
// slot down after every round.
template <typename T>
struct Slot {
    T aI, dI, aJ, dJ;
};

// Cross round r: slot p rotates the pair (I_p, J_{(p+r) mod K}).  Only the
// slot's lanes touch the pair's state; the group learns the K rotations
// (t1, t2) by shuffles.
template <typename T, int K, int R, int L, bool WITHV, int r>
__device__ __forceinline__ void cross_round(Regs<T, K, R, WITHV>& S, Slot<T>& st, const T tol, const int hl,
                                            Counters& cnt, const unsigned lm, const bool a64, const T tau2,
                                            const T theta)
{
    constexpr int G = L / K;
    const int slot = hl / G;
    T g[K];
#pragma unroll
    for (int p = 0; p < K; ++p) {
        const int j = K + (p + r) % K;
        g[p] = dot_rows<T, R>(S.a[p], S.a[j]);
    }
    const T gs = reduce_scatter<T, K, L>(g, hl);
    const T gam = (st.dI * st.dJ) * gs;
    T t1 = T(0), t2 = T(0);
    bool needI = false, needJ = false;
    const unsigned lo = (lm >> slot) & (lm >> (K + (slot + r) % K)) & 1u;
    bool bigp, rotp, widep;
    if (a64) {
        const double off = lo ? 0.0 : off64((double)st.aI, (double)st.aJ, (double)gam);
        bigp = off > 2.0 * (double)tol;
        rotp = off > (double)tol;
        widep = off > (double)theta;
        if (bigp) cnt.cbig = fmaxf(cnt.cbig, (float)off);
    } else {
        const T off = lo ? T(0) : fabs(gam) * rsqrt(st.aI) * rsqrt(st.aJ);
        bigp = off > T(2) * tol;
        rotp = off > tol;  // false for a zero column (0 * inf = NaN) and for a carried norm gone negative
        widep = off > theta;
        if (bigp) cnt.cbig = fmaxf(cnt.cbig, (float)off);
    }
    if (bigp && hl % G == 0) {
        ++cnt.big;
        if (st.aI < tau2 && st.aJ < tau2) ++cnt.bigll;
    }
    if (rotp) {
        T c, tg;
        if (a64) {
            double td, cd;
            rot_params64((double)st.aI, (double)st.aJ, (double)gam, td, cd);
            t1 = (T)(td * ((double)st.dJ / (double)st.dI));
            t2 = (T)(td * ((double)st.dI / (double)st.dJ));
            c = (T)cd;
            tg = (T)(td * (double)gam);
            widep = widep || fabs(td) > (double)theta;
            cnt.tall = fmaxf(cnt.tall, (float)fabs(td));
            if (bigp) cnt.tbig = fmaxf(cnt.tbig, (float)fabs(td));
        } else {
            T t;
            rot_params(st.aI, st.aJ, gam, t, c);
            rot_factors(t, st.dI, st.dJ, t1, t2, c);
            tg = t * gam;
            widep = widep || fabs(t) > theta;
            cnt.tall = fmaxf(cnt.tall, (float)fabs(t));
            if (bigp) cnt.tbig = fmaxf(cnt.tbig, (float)fabs(t));
        }
        if (widep && hl % G == 0) ++cnt.wide;
        const T oI = st.aI, oJ = st.aJ;
        st.aI = oI - tg;
        st.aJ = oJ + tg;
        st.dI *= c;
        st.dJ *= c;
        // a carried norm loses accuracy when the column loses most of its norm
        needI = st.aI < T(0.25) * oI;
        needJ = st.aJ < T(0.25) * oJ;
        if (hl % G == 0) ++cnt.rots;
    }
    if (hl == 0) cnt.pairs += K;
    T T1[K], T2[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
        T1[q] = __shfl_sync(FULL, t1, q * G, L);
        T2[q] = __shfl_sync(FULL, t2, q * G, L);
    }
    // one vote per round; a pair without a rotation has t1 = t2 = 0 and is left exactly as it is
    if (__any_sync(FULL, t1 != T(0) || t2 != T(0))) {
#pragma unroll
        for (int q = 0; q < K; ++q) {
            const int j = K + (q + r) % K;
#pragma unroll
            for (int k = 0; k < R; ++k) {
                const T x = S.a[q][k], y = S.a[j][k];
                S.a[q][k] = fma(-T1[q], y, x);
                S.a[j][k] = fma(T2[q], x, y);
            }
            if (WITHV) {
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    const T x = S.v[q][k], y = S.v[j][k];
                    S.v[q][k] = fma(-T1[q], y, x);
                    S.v[j][k] = fma(T2[q], x, y);
                }
            }
        }
    }
    // recompute flagged norms from the rotated columns (a group that did not
    // flag the column just refreshes it)
    const unsigned bi = __ballot_sync(FULL, needI), bj = __ballot_sync(FULL, needJ);
    if ((bi | bj) != 0u) {
#pragma unroll
        for (int q = 0; q < K; ++q) {
            const unsigned sq = ((1u << G) - 1u) << (q * G);   // slot q's lanes in a group
            const unsigned wq = (L == 32) ? sq : (sq | (sq << 16));
            if ((bi & wq) != 0u) {
                T acc = T(0);
#pragma unroll
                for (int k = 0; k < R; ++k) acc = fma(S.a[q][k], S.a[q][k], acc);
                acc = group_sum<L>(acc);
                if (slot == q) st.aI = st.dI * st.dI * acc;
            }
            if ((bj & wq) != 0u) {
                const int j = K + (q + r) % K;
                T acc = T(0);
#pragma unroll
                for (int k = 0; k < R; ++k) acc = fma(S.a[j][k], S.a[j][k], acc);
                acc = group_sum<L>(acc);
                if (slot == q) st.aJ = st.dJ * st.dJ * acc;
            }
        }
    }
    // the second-block column state moves one slot down (slot p takes slot p+1's)
    const int srcl = ((slot + 1) % K) * G + hl % G;
    st.aJ = __shfl_sync(FULL, st.aJ, srcl, L);
    st.dJ = __shfl_sync(FULL, st.dJ, srcl, L);
}

template <typename T, int K, int R, int L, bool WITHV, int... Rs>
__device__ __forceinline__ void cross_rounds(Regs<T, K, R, WITHV>& S, Slot<T>& st, const T tol, const int hl,
                                             Counters& cnt, std::integer_sequence<int, Rs...>, const unsigned lm = 0u,
                                             const bool a64 = false, const T tau2 = T(0), const T theta = T(0))
{
    (cross_round<T, K, R, L, WITHV, Rs>(S, st, tol, hl, cnt, lm, a64, tau2, theta), ...);
}

template <typename T, int K, int R, int L, bool WITHV, bool CROSS, int... Rs>
__device__ __forceinline__ void do_rounds(Regs<T, K, R, WITHV>& S, const T tol, const int hl, Counters& cnt,
                                          std::integer_sequence<int, Rs...>, const unsigned lm = 0u,
                                          const bool a64 = false, const T tau2 = T(0), const T theta = T(0))
{
    (do_round<T, K, R, L, WITHV, CROSS, Rs>(S, tol, hl, cnt, lm, a64, tau2, theta), ...);
}

// Load the 2K columns of blocks bI, bJ into the group's registers and the
// slot state (carried squared norm and scale of I_p and J_p) into the slot.
template <typename T, int K, int R, int L, bool WITHV>
// Block bI's columns are read from AwI (scales dscI), block bJ's from AwJ
// (dscJ): the same array for a slice held by one CTA; for a slice spread over
// a cluster, each base is the owning CTA's array (offset so that global
// column indices address it).
// With anorm set, the slot's squared norms are the ones carried from the
// previous step (anorm[c] = d_c^2 |s_c|^2, written by store_cols); without
// it they are recomputed from the loaded columns.
__device__ __forceinline__ void load_cols(Regs<T, K, R, WITHV>& S, Slot<T>& st, const T* AwI, const T* AwJ,
                                          const T* Vw, const T* dscI, const T* dscJ, int ldA, int bI, int bJ,
                                          int hl, bool active, const T* anorm = nullptr)
{
    constexpr int VN = VecOf<T, R>::N;
    constexpr int G = L / K;
    typedef typename VecT<T, VN>::V VT;
#pragma unroll
    for (int c = 0; c < 2 * K; ++c) {
        const int col = (c < K) ? bI * K + c : bJ * K + (c - K);
        const T* src = ((c < K) ? AwI : AwJ) + (size_t)col * ldA;
#pragma unroll
        for (int g = 0; g < R / VN; ++g) {
            const VT x = *reinterpret_cast<const VT*>(src + grow<L, VN>(hl, g * VN));
            const T* xs = reinterpret_cast<const T*>(&x);
#pragma unroll
            for (int u = 0; u < VN; ++u) S.a[c][g * VN + u] = xs[u];
        }
        if (WITHV) {
            const T* vs = Vw + (size_t)col * ldA;
#pragma unroll
            for (int g = 0; g < R / VN; ++g) {
                const VT x = *reinterpret_cast<const VT*>(vs + grow<L, VN>(hl, g * VN));
                const T* xs = reinterpret_cast<const T*>(&x);
#pragma unroll
                for (int u = 0; u < VN; ++u) S.v[c][g * VN + u] = xs[u];
            }
        }
    }
    const int slot = hl / G;
    const int cI = bI * K + slot, cJ = bJ * K + slot;
    st.dI = dscI[cI];
    st.dJ = dscJ[cJ];
    if (anorm) {
        st.aI = active ? anorm[cI] : T(-1);
        st.aJ = active ? anorm[cJ] : T(-1);
        return;
    }
    // fresh squared norms of the 2K columns, ordered (I_0, J_0, I_1, J_1, ...)
    // so that the reduce-scatter leaves I_p and J_p in the two halves of slot p
    T nv[2 * K];
#pragma unroll
    for (int c = 0; c < K; ++c) {
        T a0 = T(0), a1 = T(0);
#pragma unroll
        for (int q = 0; q < R; ++q) {
            a0 = fma(S.a[c][q], S.a[c][q], a0);
            a1 = fma(S.a[K + c][q], S.a[K + c][q], a1);
        }
        nv[2 * c] = a0;
        nv[2 * c + 1] = a1;
    }
    constexpr int H = L / (2 * K);  // lanes per reduced value
    const T mine = reduce_scatter<T, 2 * K, L>(nv, hl);
    const T other = __shfl_xor_sync(FULL, mine, H);
    const bool upper = (hl & H) != 0;
    const T sI = upper ? other : mine, sJ = upper ? mine : other;
    // an inactive group (no block pair left) works on block 0 with negative
    // norms: every off-diagonality test is then NaN, so it never rotates
    st.aI = active ? st.dI * st.dI * sI : T(-1);
    st.aJ = active ? st.dJ * st.dJ * sJ : T(-1);
}

// Redundant copy of the 2K column states in every lane (for the within-block
// rounds of a sweep's first step).
template <typename T, int K, int R, int L, bool WITHV>
__device__ __forceinline__ void gather_state(Regs<T, K, R, WITHV>& S, const Slot<T>& st)
{
    constexpr int G = L / K;
#pragma unroll
    for (int c = 0; c < K; ++c) {
        S.al[c] = __shfl_sync(FULL, st.aI, c * G, L);
        S.d[c] = __shfl_sync(FULL, st.dI, c * G, L);
        S.al[K + c] = __shfl_sync(FULL, st.aJ, c * G, L);
        S.d[K + c] = __shfl_sync(FULL, st.dJ, c * G, L);
    }
}

template <typename T, int K, int R, int L, bool WITHV>
__device__ __forceinline__ void scatter_state(const Regs<T, K, R, WITHV>& S, Slot<T>& st, int hl)
{
    constexpr int G = L / K;
    const int slot = hl / G;
#pragma unroll
    for (int c = 0; c < K; ++c) {
        if (slot == c) {
            st.aI = S.al[c];
            st.dI = S.d[c];
            st.aJ = S.al[K + c];
            st.dJ = S.d[K + c];
        }
    }
}

// Write the columns and the slot state back; fold tiny scales into the data.
template <typename T, int K, int R, int L, bool WITHV>
__device__ __forceinline__ void store_cols(Regs<T, K, R, WITHV>& S, Slot<T>& st, T* AwI, T* AwJ, T* Vw, T* dscI,
                                           T* dscJ, int ldA, int bI, int bJ, int hl, bool active,
                                           T* anorm = nullptr)
{
    constexpr int VN = VecOf<T, R>::N;
    constexpr int G = L / K;
    typedef typename VecT<T, VN>::V VT;
    const int slot = hl / G;
    const bool fold_any = __any_sync(FULL, st.dI < Num<T>::fold() || st.dJ < Num<T>::fold());
    if (fold_any) {
#pragma unroll
        for (int c = 0; c < K; ++c) {
            const T fI = __shfl_sync(FULL, st.dI, c * G, L);
            const T fJ = __shfl_sync(FULL, st.dJ, c * G, L);
            const T sI = fI < Num<T>::fold() ? fI : T(1);
            const T sJ = fJ < Num<T>::fold() ? fJ : T(1);
#pragma unroll
            for (int q = 0; q < R; ++q) {
                S.a[c][q] *= sI;
                S.a[K + c][q] *= sJ;
                if (WITHV) {
                    S.v[c][q] *= sI;
                    S.v[K + c][q] *= sJ;
                }
            }
        }
        if (st.dI < Num<T>::fold()) st.dI = T(1);
        if (st.dJ < Num<T>::fold()) st.dJ = T(1);
    }
    if (!active) return;
#pragma unroll
    for (int c = 0; c < 2 * K; ++c) {
        const int col = (c < K) ? bI * K + c : bJ * K + (c - K);
        T* dst = ((c < K) ? AwI : AwJ) + (size_t)col * ldA;
#pragma unroll
        for (int g = 0; g < R / VN; ++g) {
            VT x;
            T* xs = reinterpret_cast<T*>(&x);
#pragma unroll
            for (int u = 0; u < VN; ++u) xs[u] = S.a[c][g * VN + u];
            *reinterpret_cast<VT*>(dst + grow<L, VN>(hl, g * VN)) = x;
        }
        if (WITHV) {
            T* vd = Vw + (size_t)col * ldA;
#pragma unroll
            for (int g = 0; g < R / VN; ++g) {
                VT x;
                T* xs = reinterpret_cast<T*>(&x);
#pragma unroll
                for (int u = 0; u < VN; ++u) xs[u] = S.v[c][g * VN + u];
                *reinterpret_cast<VT*>(vd + grow<L, VN>(hl, g * VN)) = x;
            }
        }
    }
    if (hl % G == 0) {
        dscI[bI * K + slot] = st.dI;
        dscJ[bJ * K + slot] = st.dJ;
        if (anorm) {
            anorm[bI * K + slot] = st.aI;
            anorm[bJ * K + slot] = st.aJ;
        }
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
    const SliceItem* items;  // batched SVT: per-CTA slice parameters (replace the fields above)
    // warm start (single-tensor SVT): slice k starts from w0 + k * stride (the
    // slice times an orthogonal Q, in the working copy's layout) when
    // wflag[k] is set; after the sweeps A0^T s_i / sigma_i of every column is
    // written to vrec + k * stride (n x n, columns by descending sigma) and
    // wrec[k] set.  vrec may alias w0: each CTA reads its w0 before writing.
    const T* w0;
    const int* wflag;
    T* vrec;
    int* wrec;
    int small_stop;     // 1: stop after a sweep of small rotations only (see theta in the kernel)
    float* sweep_log;   // optional: per slice and sweep s < kSweepLogSweeps, kSweepLogVals values (see the sweep loop)
    // offloaded tail (warm-started single-tensor SVT): instead of the
    // recovery and the rebuild, the kernel writes its converged columns to
    // tail_s + k * stride (its working-copy layout) and, at tail_info + k *
    // tail_info_stride(npad), what warm_tail_kernel needs (see there)
    T* tail_s;
    float* tail_info;
};

// Shared-memory carve-up (bytes) for a launch: dsc, sig, cf, carried norms
// (elem each), kidx and rank (int), and per warp a coefficient buffer of
// 4 x npad.
__host__ __device__ inline size_t smem_small_bytes(int npad, int W, int elem)
{
    size_t b = (size_t)npad * (4 * elem + 8) + (size_t)W * 4 * npad * elem;
    return (b + 255) & ~(size_t)255;
}

// Threads per CTA the register file allows for one instantiation: the 2K
// register-resident columns (twice that with V), about 3 x 2K values of
// column state and broadcast rotations, 40 temporaries, plus addressing.
template <typename T, int K, int R, bool WITHV>
struct Bound {
    static constexpr int regs = (2 * K * R * (WITHV ? 2 : 1) + 6 * K + 40) * (int)(sizeof(T) / 4) + 24;
    static constexpr int t = (65536 / regs) / 32 * 32;
    static constexpr int value = t > 1024 ? 1024 : t;
};

// A64: the FP32 rotation angles and convergence tests in FP64 (a separate
// instantiation, so the default kernels carry no FP64 code).
template <typename T, int K, int R, int L, bool SMEM, bool WITHV, bool ITEMS = false, bool A64 = false>
__global__ void __launch_bounds__(Bound<T, K, R, WITHV>::value) jacobi_kernel(KArgs<T> a)
{
    if (a.ctl && a.ctl->done) return;
    const long long t_start = clock64();  // phase times for the sweep log
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int W = blockDim.x >> 5;
    const int nthr = blockDim.x;
    const int slice = blockIdx.x;
    const SliceItem* item = ITEMS ? a.items + slice : nullptr;  // batched: per-CTA slice parameters
    // a batched ADMM job that has stopped: its slices are left as they are
    const AdmmCtl* ictl = item ? item->ctl : nullptr;
    if (ictl && ictl->done) return;
    const int m = item ? item->m : a.m, n = item ? item->n : a.n, nb = item ? item->nb : a.nb;
    const int ldA = a.ldA, tr = item ? item->tr : a.tr;
    const int npad = nb * K;
    const int64_t n1 = item ? item->n1 : a.n1, n2 = item ? item->n2 : a.n2;
    const size_t wsz = (size_t)ldA * npad;
    // per-CTA working copy stride in global scratch: sized for the launch's largest slice
    const size_t wstride = (size_t)ldA * a.nb * K;
    constexpr int GPW = 32 / L;  // groups per warp
    const int hl = lane % L;
    const int NG = W * GPW;

    T* Aw;
    T* Vw = nullptr;
    unsigned char* rest;
    if (SMEM) {
        Aw = reinterpret_cast<T*>(smem_raw);
        if (WITHV) Vw = Aw + wsz;
        rest = smem_raw + (WITHV ? 2 : 1) * ((wsz * sizeof(T) + 255) & ~(size_t)255);
    } else {
        Aw = a.work + (size_t)slice * (WITHV ? 2 : 1) * wstride;
        if (WITHV) Vw = Aw + wsz;
        rest = smem_raw;
    }
    T* dsc = reinterpret_cast<T*>(rest);
    T* sig = dsc + npad;
    T* cf = sig + npad;
    T* anorm = cf + npad;  // squared norms d^2 |s|^2 carried from step to step within a sweep
    int* kidx = reinterpret_cast<int*>(anorm + npad);
    int* rank = kidx + npad;
    T* gbuf = reinterpret_cast<T*>(rank + npad);
    __shared__ int s_rot, s_rotll, s_wide, s_keep, s_nonfinite, s_nlo, s_cnt;
    __shared__ int s_lg[3];
    __shared__ double s_nuc, s_fro, s_lo, s_s1, s_yn;
    __shared__ unsigned long long s_maxb;  // bits of a nonnegative double (ordered as integers)
    __shared__ unsigned long long s_pairs, s_rots;

    T* src = item ? static_cast<T*>(item->data) : a.data + (size_t)slice * n1 * n2;

    // ---- load the oriented slice; pad rows and columns with zeros
    const bool warm_in = !WITHV && !ITEMS && a.w0 && a.wflag && a.wflag[slice];
    T fro = T(0);  // this thread's share of ||A||_F^2
    if (warm_in) {
        // warm start: the slice times the previous iteration's right singular
        // vectors (orthogonal), already oriented, padded and laid out as here;
        // the same singular values, columns nearly orthogonal
        const T* w0 = a.w0 + (size_t)slice * wstride;
        if constexpr (SMEM && sizeof(T) == 4) {  // all chunks in flight at once, then the norm from shared memory
            copy_to_shared(reinterpret_cast<float*>(Aw), reinterpret_cast<const float*>(w0), wsz, tid, nthr);
            cp_async_wait_all();
            __syncthreads();
            for (size_t e = tid; e < wsz; e += nthr) fro = fma(Aw[e], Aw[e], fro);
        } else {
            for (size_t e = tid; e < wsz; e += nthr) {
                const T v = w0[e];
                Aw[e] = v;
                fro = fma(v, v, fro);
            }
        }
    } else {
        for (size_t e = tid; e < wsz; e += nthr) Aw[e] = T(0);
        if (WITHV)
            for (size_t e = tid; e < wsz; e += nthr) {
                int c = (int)(e / ldA), r = (int)(e % ldA);
                Vw[e] = (r == c && c < n) ? T(1) : T(0);
            }
        __syncthreads();
        const int64_t S = n1 * n2;
        for (int64_t e = tid; e < S; e += nthr) {
            int i = (int)(e % n1), j = (int)(e / n1);
            // oriented (row, col): (i, j) if n1 >= n2 else (j, i)
            int r = tr ? j : i, c = tr ? i : j;
            const T v = src[e];
            Aw[(size_t)c * ldA + r] = v;
            fro = fma(v, v, fro);
        }
    }
    for (int c = tid; c < npad; c += nthr) dsc[c] = T(1);
    if (tid == 0) { s_pairs = 0; s_rots = 0; s_nonfinite = 0; s_nuc = 0.0; s_keep = 0; s_fro = 0.0; }
    __syncthreads();
    fro = group_sum<32>(fro);
    if (lane == 0) atomicAdd(&s_fro, (double)fro);
    __syncthreads();

    // SVT of a slice whose Frobenius norm is below the threshold: every
    // singular value is at most ||A||_F <= tau, so Y = 0 and the sweeps can
    // be skipped (the rebuild below then keeps nothing and writes zeros, as
    // the full computation would).  The margin covers the rounding of the sum.
    bool skip = false;
    if (!WITHV) {
        const double tau0 = a.ctl ? 1.0 / a.ctl->beta : (ictl ? 1.0 / ictl->beta : (item ? item->tau : a.tau));
        skip = s_fro * (1.0 + 1e-3) < tau0 * tau0;
    }

    // ---- sweeps
    //
    // SVT: columns whose squared norms sum to at most tau^2 need no rotation
    // among themselves.  If, at the end, every pair involving another column
    // has converged, the slice is S_H V_H^T + S_Lo V_Lo^T with S_H's columns
    // orthogonal to each other and to S_Lo's, so its SVT is that of the
    // first term plus that of the second, and the second is zero because
    // ||S_Lo||_2 <= ||S_Lo||_F <= tau; the rebuild below keeps only columns
    // with sigma > tau, none of them in S_Lo.  Each sweep flags the columns
    // with alpha < tau^2 / 4 (from the carried squared norms) and, if their
    // alphas sum to at most 0.9 tau^2, leaves pairs of two flagged columns
    // alone (when at least half of the columns are flagged).  A sweep without
    // rotation ends the iteration only if the flagged
    // columns' alphas still sum below tau^2 (a rotation with a column that
    // has shrunk below them can grow them); otherwise full sweeps follow.
    const T tol = sqrt((T)m) * Num<T>::unit();
    // The small-rotation stop.  A pair rotated in a sweep is left orthogonal
    // to rounding; a later rotation of one of its columns with a third
    // column k by the tangent t changes the pair's normalised dot product by
    // at most about max(|t|, |gamma_ik| / sqrt(alpha_i alpha_k)) times column
    // k's normalised dot product with the other column (the column-norm
    // ratio that enters is offset by the small angle: t ~ gamma / (alpha_k -
    // alpha_i)), and each column meets fewer than n partners in a sweep.  So
    // a sweep whose rotations all had both quantities at most theta leaves
    // every pair within tol + 4 n theta^2 of orthogonal, and with theta =
    // sqrt(tol / (4 n)) within 2 tol: the level the stopping rule (no
    // rotation above 2 tol in a sweep) accepts, without the extra sweep that
    // rule spends confirming it.  theta = 0 turns the stop off.
    const T theta = a.small_stop ? sqrt(tol / (T(4) * (T)n)) : T(0);
    constexpr bool a64 = A64 && sizeof(T) == 4;
    Counters cnt{0, 0, 0, 0, 0, 0.f, 0.f, 0.f};
    int sweeps = 0, converged = skip ? 1 : 0;
    const int max_sweeps = a.max_sweeps > 0 ? a.max_sweeps : 30;
    const int npairs = nb / 2;
    const double tau_s = WITHV ? 0.0
                               : (a.ctl ? 1.0 / a.ctl->beta : (ictl ? 1.0 / ictl->beta : (item ? item->tau : a.tau)));
    bool full_only = WITHV;
    int cert_left = WITHV ? 0 : 2;  // zero-SVT certificate attempts (below)
    int* loflag = kidx;  // free until the rebuild
    const T tau2 = (T)(tau_s * tau_s);
    bool gmode = false;           // low block certified (below): pairs of two low columns are left alone
    int gm_left = WITHV ? 0 : 4;  // low-block certificate attempts

    // Low-block certificate (SVT).  The columns whose squared norms are
    // below tau^2 form a block S_L whose singular values the SVT discards as
    // long as they are at most tau.  By Gershgorin on its Gram matrix
    // G = S_L^T S_L, sigma_max(S_L)^2 <= max_i sum_{j in L} |G_ij|.  The bound,
    // with the rounding of the computed G (|dG_ij| <= m u |a_i| |a_j|) and of
    // the row sums added as for the zero-SVT certificate, is accepted if it is
    // at most (tau + eps)^2 with eps = 1e-7 ||Y_slice|| (estimated from the
    // other columns' norms): a singular value of S_L above tau by at most eps
    // would change Y by at most eps.  Once certified, pairs of two low columns
    // are left alone; a sweep without rotation ends the iteration only if the
    // certificate still holds on the current columns.  Columns of S_L are
    // listed in rank[] (free in the SVT).
    auto low_cert = [&](const bool zero) -> bool {
        if (tid == 0) { s_cnt = 0; s_maxb = 0ull; s_s1 = 0.0; s_yn = 0.0; }
        __syncthreads();
        double yn = 0.0, s1 = 0.0;
        for (int c = tid; c < n; c += nthr) {
            const double an = (double)anorm[c];
            if (an < tau_s * tau_s) {
                rank[atomicAdd(&s_cnt, 1)] = c;
                s1 += sqrt(fmax(an, 0.0));
            } else {
                const double e = sqrt(an) - tau_s;
                yn += e * e;
            }
        }
        yn = group_sum<32>(yn);
        s1 = group_sum<32>(s1);
        if (lane == 0) {
            if (yn != 0.0) atomicAdd(&s_yn, yn);
            if (s1 != 0.0) atomicAdd(&s_s1, s1);
        }
        __syncthreads();
        const int nl = s_cnt;
        const double S1 = 1.01 * s_s1;
        // zero: the zero-SVT certificate below (every column in the set, bound below tau^2)
        const double lim = zero ? (1.0 - 1e-4) * tau_s * tau_s
                                : (tau_s + 1e-7 * sqrt(s_yn)) * (tau_s + 1e-7 * sqrt(s_yn));
        // The Gram G = S_lo^T S_lo (true scales: G_ij = d_i d_j s_i.s_j) in 4 x 4
        // blocks, a thread per block of its upper triangle, each entry a
        // column-pair dot product over the m rows.  Each block writes its
        // row sums of |G_ij| (and, off the diagonal, those of its transpose)
        // into its own slot of part[row][block], and each row's slots are
        // added in block order, so the bound does not depend on thread
        // timing; the summation's rounding is covered by the (1 + 2 nl u)
        // factor below.  All in the kernel's precision (FP64 here would run
        // at a small fraction of the FP32 rate).
        const double uu = (double)Num<T>::unit();
        double wmax = 0.0;
        const int B = (nl + 3) / 4, nblk = B * (B + 1) / 2;
        T* part = gbuf;  // nl x B (gbuf is free during the sweeps)
        if ((size_t)nl * B > (size_t)W * 4 * npad) {  // no room: no certificate
            __syncthreads();
            return false;
        }
        for (int blk = tid; blk < nblk; blk += nthr) {
            int bi = 0, rem = blk;  // blk -> (bi, bj), bi <= bj, row by row of the upper triangle
            while (rem >= B - bi) { rem -= B - bi; ++bi; }
            const int bj = bi + rem;
            const T* ci[4];
            const T* cj[4];
            bool vi[4], vj[4];
            T di[4], dj[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                vi[u] = 4 * bi + u < nl;
                vj[u] = 4 * bj + u < nl;
                const int a = rank[vi[u] ? 4 * bi + u : 0], b = rank[vj[u] ? 4 * bj + u : 0];
                ci[u] = Aw + (size_t)a * ldA;
                cj[u] = Aw + (size_t)b * ldA;
                di[u] = vi[u] ? dsc[a] : T(0);
                dj[u] = vj[u] ? dsc[b] : T(0);
            }
            T acc[4][4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
            for (int r = 0; r < m; ++r) {
                T x[4], y[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    x[u] = ci[u][r];
                    y[u] = cj[u][r];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[u][v] = fma(x[u], y[v], acc[u][v]);
            }
            T rs[4] = {T(0), T(0), T(0), T(0)}, cs[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const T g = fabs(acc[u][v]) * di[u] * dj[v];  // zero outside the list
                    rs[u] += g;
                    cs[v] += g;
                }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (vi[u]) part[(size_t)(4 * bi + u) * B + bj] = rs[u];
                if (bi != bj && vj[u]) part[(size_t)(4 * bj + u) * B + bi] = cs[u];
            }
        }
        __syncthreads();
        for (int i = tid; i < nl; i += nthr) {
            const int c = rank[i];
            T rsum = T(0);
            for (int q = 0; q < B; ++q) rsum += part[(size_t)i * B + q];
            const double b = (double)rsum * (1.0 + 2.0 * nl * uu) +
                             2.0 * m * uu * sqrt(fmax((double)anorm[c], 0.0)) * S1;
            wmax = fmax(wmax, b);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wmax = fmax(wmax, __shfl_xor_sync(FULL, wmax, o));
        if (lane == 0) atomicMax(&s_maxb, (unsigned long long)__double_as_longlong(wmax));
        __syncthreads();
        const bool ok = __longlong_as_double((long long)s_maxb) <= lim;
        __syncthreads();  // the shared words are reused after this
        return ok;
    };
    if (!WITHV && !skip) {
        for (int c = warp; c < npad; c += W) {
            const T* col = Aw + (size_t)c * ldA;
            T s2 = T(0);
            for (int r = lane; r < ldA; r += 32) s2 = fma(col[r], col[r], s2);
            s2 = group_sum<32>(s2);
            if (lane == 0) anorm[c] = s2;  // the scales are all 1 here
        }
    }
    const long long t_load = clock64();
    while (!skip && sweeps < max_sweeps) {
        const long long t_sweep = clock64();
        if (tid == 0) { s_rot = 0; s_rotll = 0; s_wide = 0; s_lo = 0.0; s_nlo = 0; s_lg[0] = s_lg[1] = s_lg[2] = 0; }
        cnt.cbig = cnt.tbig = cnt.tall = 0.f;
        __syncthreads();
        if (!full_only || gmode) {
            // columns flagged: below tau^2 / 4 (small-column sweeps) or, with
            // the low block certified, below tau^2
            const double thr = gmode ? tau_s * tau_s : 0.25 * tau_s * tau_s;
            double part = 0.0;
            int nf = 0;
            for (int c = tid; c < npad; c += nthr) {
                const double an = (double)anorm[c];
                const int f = an < thr ? 1 : 0;
                loflag[c] = f;
                part += f ? fabs(an) : 0.0;  // a carried alpha gone negative counts by its size
                nf += (f && c < n) ? 1 : 0;
            }
            part = group_sum<32>(part);
            nf = group_sum<32>(nf);
            if (lane == 0) {
                if (part != 0.0) atomicAdd(&s_lo, part);
                if (nf) atomicAdd(&s_nlo, nf);
            }
        }
        __syncthreads();
        // flagged sweeps only where they pay: most columns flagged (a few
        // tiny columns save nothing and can cost a closing full sweep)
        const bool partial = gmode || (!full_only && s_lo <= 0.9 * tau_s * tau_s && 2 * s_nlo >= n);
        const int big0 = cnt.big, bigll0 = cnt.bigll, wide0 = cnt.wide;
        // one sweep; compiled twice, so that a sweep without flagged columns
        // runs code without the flag tests
        auto sweep = [&](auto flagged) {
            constexpr bool FL = decltype(flagged)::value;
            for (int step = 0; step < nb - 1; ++step) {
                // iterations are warp-uniform: a group without a block pair works on block 0 with zero norms
                for (int base = warp * GPW; base < npairs; base += NG) {
                    const int pr = base + lane / L;
                    const bool active = pr < npairs;
                    const int bI = active ? block_at(nb, pr, step) : 0;
                    const int bJ = active ? block_at(nb, nb - 1 - pr, step) : 0;
                    Regs<T, K, R, WITHV> Sr;
                    Slot<T> st;
                    const Counters cnt0 = cnt;
                    // squared norms: recomputed at a sweep's first step, carried after it
                    load_cols<T, K, R, L, WITHV>(Sr, st, Aw, Aw, Vw, dsc, dsc, ldA, bI, bJ, hl, active,
                                                 step == 0 ? nullptr : anorm);
                    unsigned lm = 0u;  // flags of the 2K columns (I block: bits 0..K-1, J block: K..2K-1)
                    if constexpr (FL) {
#pragma unroll
                        for (int c = 0; c < K; ++c)
                            lm |= ((unsigned)loflag[bI * K + c] << c) | ((unsigned)loflag[bJ * K + c] << (K + c));
                    }
                    if (step == 0) {
                        gather_state<T, K, R, L, WITHV>(Sr, st);
                        do_rounds<T, K, R, L, WITHV, false>(Sr, tol, hl, cnt,
                                                            std::make_integer_sequence<int, K - 1>{}, lm, a64, tau2,
                                                            theta);
                        scatter_state<T, K, R, L, WITHV>(Sr, st, hl);
                    }
                    cross_rounds<T, K, R, L, WITHV>(Sr, st, tol, hl, cnt, std::make_integer_sequence<int, K>{}, lm,
                                                    a64, tau2, theta);
                    store_cols<T, K, R, L, WITHV>(Sr, st, Aw, Aw, Vw, dsc, dsc, ldA, bI, bJ, hl, active, anorm);
                    if (!active) cnt = cnt0;  // an inactive group's work is discarded, and so are its counts
                }
                __syncthreads();
            }
        };
        if (!WITHV && partial) sweep(std::true_type{});
        else sweep(std::false_type{});
        if (cnt.big != big0) atomicAdd(&s_rot, cnt.big - big0);
        if (cnt.bigll != bigll0) atomicAdd(&s_rotll, cnt.bigll - bigll0);
        if (cnt.wide != wide0) atomicAdd(&s_wide, cnt.wide - wide0);
        if (a.sweep_log) {  // the sweep's largest rotations, as float bits (nonnegative: ordered as integers)
            atomicMax(&s_lg[0], __float_as_int(cnt.cbig));
            atomicMax(&s_lg[1], __float_as_int(cnt.tbig));
            atomicMax(&s_lg[2], __float_as_int(cnt.tall));
        }
        __syncthreads();
        const int nrot = s_rot, nrotll = s_rotll;
        long long t_dec = 0;
        float* lg = (a.sweep_log && tid == 0 && sweeps < kSweepLogSweeps && !item)
                        ? a.sweep_log + ((size_t)slice * (kSweepLogSweeps + 1) + sweeps) * kSweepLogVals
                        : nullptr;
        if (lg) {
            // big rotations, wide ones (the small-rotation stop), big low-low
            // ones, largest |gamma| / sqrt(alpha beta) of the big ones,
            // largest |t| of the big ones and of all, then the sweep's cycles
            // (thread 0's clock) and those of the stopping tests after it
            t_dec = clock64();
            lg[0] = (float)nrot; lg[1] = (float)s_wide; lg[2] = (float)nrotll;
            lg[3] = __int_as_float(s_lg[0]); lg[4] = __int_as_float(s_lg[1]); lg[5] = __int_as_float(s_lg[2]);
            lg[6] = (float)(t_dec - t_sweep);
        }
        ++sweeps;
        // converged: no big rotation in the sweep, or only small ones (every
        // rotation applied had |gamma| / sqrt(alpha beta) <= theta and
        // |t| <= theta, so what they left between any two columns is at most
        // about 4 n theta^2 <= tol; see theta above)
        bool done = nrot == 0 || s_wide == 0;
        if (done && partial && !gmode) {
            // the flagged columns' alphas after the sweep
            if (tid == 0) s_lo = 0.0;
            __syncthreads();
            double part = 0.0;
            for (int c = tid; c < npad; c += nthr) part += loflag[c] ? fabs((double)anorm[c]) : 0.0;
            part = group_sum<32>(part);
            if (lane == 0 && part != 0.0) atomicAdd(&s_lo, part);
            __syncthreads();
            done = s_lo <= (1.0 - 1e-3) * tau_s * tau_s;
            if (!done) full_only = true;
        }
        // the low-block certificate: re-checked on the current columns when a
        // sweep that left low pairs alone ends without rotation; attempted once
        // rotations of low pairs are at least half of a sweep's big ones
        if (!WITHV && done && gmode) {
            --gm_left;
            done = low_cert(false);
            if (!done) gmode = false;
        } else if (!WITHV && !done && !gmode && gm_left > 0 && sweeps >= 2 && 2 * nrotll >= nrot) {
            --gm_left;
            gmode = low_cert(false);
        }
        // Zero-SVT certificate.  sigma_1^2 is the largest eigenvalue of the
        // Gram matrix G = S^T S of the current columns (V orthogonal), so by
        // Gershgorin sigma_1^2 <= max_i sum_j |G_ij|.  A slice whose columns
        // are all below tau after a sweep (necessary for sigma_1 <= tau) gets
        // that bound, with the rounding of the computed G (|dG_ij| <= m u
        // |a_i| |a_j|) and of the row sums added; if it is below tau^2, every
        // singular value is at most tau, the SVT is zero and the sweeps stop
        // (the rebuild keeps no column: each column's norm is at most
        // sigma_1).  Tried after the first two sweeps only.
        if (!WITHV && !done && cert_left > 0) {
            --cert_left;
            if (tid == 0) s_maxb = 0ull;
            __syncthreads();
            double amx = 0.0;
            for (int c = tid; c < n; c += nthr) amx = fmax(amx, fmax((double)anorm[c], 0.0));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) amx = fmax(amx, __shfl_xor_sync(FULL, amx, o));
            if (lane == 0) atomicMax(&s_maxb, (unsigned long long)__double_as_longlong(amx));
            __syncthreads();
            const double amax = __longlong_as_double((long long)s_maxb);
            __syncthreads();
            if (amax < 0.999 * tau_s * tau_s) done = low_cert(true);  // every column is in the low set
        }
        __syncthreads();
        if (lg) lg[7] = (float)(clock64() - t_dec);
        if (done) { converged = 1; break; }
    }
    const long long t_sweeps = clock64();
    if (cnt.pairs) atomicAdd(&s_pairs, (unsigned long long)cnt.pairs);
    if (cnt.rots) atomicAdd(&s_rots, (unsigned long long)cnt.rots);

    // ---- singular values sigma_c = d_c |s_c| (warp per column)
    for (int c = warp; c < npad; c += W) {
        const T* col = Aw + (size_t)c * ldA;
        T s2 = T(0);
        for (int r = lane; r < ldA; r += 32) s2 = fma(col[r], col[r], s2);
        s2 = group_sum<32>(s2);
        if (lane == 0) {
            T sg = dsc[c] * sqrt(s2);
            sig[c] = sg;
            cf[c] = s2;  // |s_c|^2 for now
            if (!isfinite(sg)) s_nonfinite = 1;
        }
    }
    __syncthreads();

    // ---- offloaded tail: the converged columns, each column's rank by
    // descending sigma (ties by index) and its recovery scale 1 / (d_c
    // |s_c|^2) go to global memory; the kept columns and their coefficients
    // follow below
    const bool offload = !WITHV && !ITEMS && a.tail_info != nullptr;
    float* tinfo = offload ? a.tail_info + (size_t)slice * tail_info_stride(npad) : nullptr;
    if (offload && !skip) {
        int* irank = reinterpret_cast<int*>(tinfo + 2 * npad);
        for (int c = tid; c < n; c += nthr) {
            int rk = 0;
            const T sc = sig[c];
            for (int o = 0; o < n; ++o) {
                const T so = sig[o];
                rk += (so > sc || (so == sc && o < c)) ? 1 : 0;
            }
            irank[c] = rk;
            const T den = dsc[c] * cf[c];
            tinfo[npad + c] = den > T(0) ? (float)(T(1) / den) : 0.0f;
        }
        T* so = a.tail_s + (size_t)slice * wstride;
        for (size_t e = tid; e < (size_t)ldA * n; e += nthr) so[e] = Aw[e];
    }

    // ---- warm start for the next iteration: v_c = A0^T s_c / (d_c |s_c|^2)
    // = A0^T u_c / sigma_c for every column, columns by descending sigma
    // (the reliable ones first for the orthogonalisation that follows).  A
    // slice that ran no sweep has no new vectors.
    if (!WITHV && !ITEMS && a.vrec && !skip && !offload) {
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
        T* vr = a.vrec + (size_t)slice * wstride;  // this slice's w0, read before the sweeps
        constexpr int RR = (R * L + 31) / 32;
        constexpr int JB = (RR <= 6) ? 4 : (RR <= 12 ? 2 : 1);
        constexpr int NV = 4 * JB;
        constexpr int GV = 32 / NV;
        for (int j0 = warp * JB; j0 < n; j0 += JB * W) {
            T x[JB][RR];
#pragma unroll
            for (int u = 0; u < JB; ++u)
#pragma unroll
                for (int q = 0; q < RR; ++q) {
                    const int r = q * 32 + lane, j = j0 + u;
                    x[u][q] = (r < m && j < n) ? (tr ? src[(size_t)j + (size_t)n1 * r] : src[(size_t)r + (size_t)n1 * j])
                                               : T(0);
                }
            for (int k0 = 0; k0 < n; k0 += 4) {
                T g[NV];
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    T sv[RR];
                    const T* col = Aw + (size_t)(k0 + v < n ? k0 + v : 0) * ldA;
#pragma unroll
                    for (int q = 0; q < RR; ++q) {
                        const int r = q * 32 + lane;
                        sv[q] = (r < ldA && k0 + v < n) ? col[r] : T(0);
                    }
#pragma unroll
                    for (int u = 0; u < JB; ++u) {
                        T acc = T(0);
#pragma unroll
                        for (int q = 0; q < RR; ++q) acc = fma(sv[q], x[u][q], acc);
                        g[v * JB + u] = acc;
                    }
                }
                const T tot = reduce_scatter<T, NV, 32>(g, lane);  // lane holds value lane / GV
                const int idx = lane / GV, vv = idx / JB, uu = idx % JB;
                const int k = k0 + vv, j = j0 + uu;
                if (lane % GV == 0 && k < n && j < n) {
                    const T den = dsc[k] * cf[k];
                    vr[(size_t)rank[k] * n + j] = den > T(0) ? tot / den : T(0);
                }
            }
        }
        if (tid == 0) a.wrec[slice] = 1;
        __syncthreads();
    }

    const T tau = a.ctl ? (T)(1.0 / a.ctl->beta) : (ictl ? (T)(1.0 / ictl->beta) : (T)(item ? item->tau : a.tau));

    if (!WITHV) {
        // ---- SVT: kept columns (sigma > tau) and their coefficients, compacted
        // in column order by warp 0, 32 columns at a time (each chunk's values
        // are read before any of its writes, and a kept column's new position
        // is never past its own, so no value is overwritten before it is read)
        if (warp == 0) {
            int kk = 0;
            double nuc = 0.0;
            for (int c0 = 0; c0 < npad; c0 += 32) {
                const int c = c0 + lane;
                const T sg = c < npad ? sig[c] : T(0);
                const T s2 = c < npad ? cf[c] : T(0);
                const bool kp = c < npad && sg > tau && s2 > T(0);
                const unsigned mask = __ballot_sync(FULL, kp);
                const int pos = kk + __popc(mask & ((1u << lane) - 1u));
                __syncwarp();
                if (kp) {
                    kidx[pos] = c;
                    cf[pos] = (T(1) - tau / sg) / s2;
                    nuc += (double)(sg - tau);
                }
                kk += __popc(mask);
                __syncwarp();
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) nuc += __shfl_xor_sync(FULL, nuc, o);
            if (lane == 0) {
                s_keep = kk;
                s_nuc = nuc;
            }
        }
        __syncthreads();
        const int keep = s_keep;
        if (offload) {  // the kept columns and their coefficients, for the tail kernel
            int* ikidx = reinterpret_cast<int*>(tinfo + 3 * npad);
            for (int q = tid; q < keep; q += nthr) {
                ikidx[q] = kidx[q];
                tinfo[q] = (float)cf[q];
            }
            if (tid == 0) {
                reinterpret_cast<int*>(tinfo)[4 * npad] = keep;
                reinterpret_cast<int*>(tinfo)[4 * npad + 1] = skip ? 0 : 1;
            }
        }
        // ---- rebuild Y = sum_q cf_q s_q (s_q^T a0_j), JB output columns per
        // warp (each shared-memory load of a kept column feeds JB FMAs); the
        // slice is overwritten in place (each warp reads only the columns it
        // writes).  Rows are lane-strided, RR = ceil(ldA / 32) per lane.
        constexpr int RR = (R * L + 31) / 32;
        constexpr int JB = (RR <= 6) ? 4 : (RR <= 12 ? 2 : 1);
        constexpr int NV = 4 * JB;     // partial sums per batch: 4 kept columns x JB
        constexpr int GV = 32 / NV;    // lanes holding each reduced value
        T* gb = gbuf + (size_t)warp * 4 * npad;
        for (int j0 = warp * JB; j0 < (offload ? 0 : n); j0 += JB * W) {
            T x[JB][RR];
#pragma unroll
            for (int u = 0; u < JB; ++u)
#pragma unroll
                for (int q = 0; q < RR; ++q) {
                    const int r = q * 32 + lane, j = j0 + u;
                    x[u][q] = (r < m && j < n) ? (tr ? src[(size_t)j + (size_t)n1 * r] : src[(size_t)r + (size_t)n1 * j])
                                               : T(0);
                }
            // coefficients gb[u * npad + k] = cf_k (s_k . a0_{j0+u}), four kept columns at a time
            for (int k0 = 0; k0 < keep; k0 += 4) {
                T g[NV];
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    T sv[RR];
                    const int kc = (k0 + v < keep) ? kidx[k0 + v] : kidx[0];
                    const T* col = Aw + (size_t)kc * ldA;
#pragma unroll
                    for (int q = 0; q < RR; ++q) {
                        const int r = q * 32 + lane;
                        sv[q] = (r < ldA && k0 + v < keep) ? col[r] : T(0);
                    }
#pragma unroll
                    for (int u = 0; u < JB; ++u) {
                        T acc = T(0);
#pragma unroll
                        for (int q = 0; q < RR; ++q) acc = fma(sv[q], x[u][q], acc);
                        g[v * JB + u] = acc;
                    }
                }
                const T tot = reduce_scatter<T, NV, 32>(g, lane);  // lane holds value lane / GV
                const int idx = lane / GV, vv = idx / JB, uu = idx % JB;
                if (lane % GV == 0 && k0 + vv < keep) gb[uu * npad + k0 + vv] = tot * cf[k0 + vv];
            }
            __syncwarp();
            T y[JB][RR];
#pragma unroll
            for (int u = 0; u < JB; ++u)
#pragma unroll
                for (int q = 0; q < RR; ++q) y[u][q] = T(0);
            for (int k = 0; k < keep; ++k) {
                const T* col = Aw + (size_t)kidx[k] * ldA;
                T sv[RR];
#pragma unroll
                for (int q = 0; q < RR; ++q) {
                    const int r = q * 32 + lane;
                    sv[q] = (r < ldA) ? col[r] : T(0);
                }
#pragma unroll
                for (int u = 0; u < JB; ++u) {
                    const T coef = gb[u * npad + k];
#pragma unroll
                    for (int q = 0; q < RR; ++q) y[u][q] = fma(coef, sv[q], y[u][q]);
                }
            }
#pragma unroll
            for (int u = 0; u < JB; ++u)
#pragma unroll
                for (int q = 0; q < RR; ++q) {
                    const int r = q * 32 + lane, j = j0 + u;
                    if (r < m && j < n) {
                        if (tr) src[(size_t)j + (size_t)n1 * r] = y[u][q];
                        else src[(size_t)r + (size_t)n1 * j] = y[u][q];
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
            const int64_t ldU = tr ? n2 : n1;  // rows of the output holding U_A
            const int64_t ldV = tr ? n1 : n2;
            T* ucol = Uo + (size_t)slice * ldU * r + (size_t)pos * ldU;
            T* vout = Vo + (size_t)slice * ldV * r + (size_t)pos * ldV;
            for (int q = lane; q < m; q += 32) ucol[q] = col[q] * inv;
            for (int q = lane; q < n; q += 32) vout[q] = vcol[q] * dv;
            if (lane == 0) a.S[(size_t)slice * r + pos] = sig[c];
        }
    }
    __syncthreads();
    if (a.sweep_log && tid == 0 && !item) {  // phase cycles: load, sweeps, tail, total
        float* ph = a.sweep_log + ((size_t)slice * (kSweepLogSweeps + 1) + kSweepLogSweeps) * kSweepLogVals;
        const long long t_end = clock64();
        ph[0] = (float)(t_load - t_start);
        ph[1] = (float)(t_sweeps - t_load);
        ph[2] = (float)(t_end - t_sweeps);
        ph[3] = (float)(t_end - t_start);
    }
    if (tid == 0) {
        SliceStats st;
        st.nuc = s_nuc;
        st.pairs = (int64_t)s_pairs;
        st.rotations = (int64_t)s_rots;
        st.sweeps = sweeps;
        st.converged = converged;
        st.nonfinite = s_nonfinite;
        st.kept = WITHV ? n : s_keep;
        if (item) *item->stats = st;
        else a.stats[slice] = st;
    }
}

}  // namespace jac
}  // namespace tnn
