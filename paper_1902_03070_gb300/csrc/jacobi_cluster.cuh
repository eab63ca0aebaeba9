// Per-slice Jacobi SVT with the slice spread over a thread-block cluster.
//
// A slice whose working copy does not fit in one CTA's shared memory is cut
// by columns into 2C super-blocks of s column blocks (K columns each) over
// the C CTAs of a cluster, two super-blocks per CTA.  The sweep is a two-level
// cyclic ordering: the super-blocks follow the circle method over 2C - 1
// super-steps, and in each super-step every CTA rotates, in its own shared
// memory, all block pairs between its two super-blocks (s rounds of s
// disjoint pairs; in the first super-step of a sweep also the pairs inside
// each super-block and inside each block).  Every column pair is visited once
// per sweep, as in the single-CTA kernel, with the same rotations and
// convergence test (jacobi.cuh); the rounds of a super-step touch only local
// shared memory.
//
// Between super-steps the super-blocks move one place around the circle:
// each CTA pulls its new super-blocks out of its neighbours' shared memory
// (distributed shared memory) into free buffers.  Three buffers per CTA are
// enough with a two-phase pull (tops, then bottoms) between cluster
// barriers; the buffers' roles then follow a fixed pattern, so every CTA
// knows which buffer of a neighbour holds what.  After 2C - 1 moves every
// super-block is back home, where the sweep vote (one counter per CTA, fed
// by every CTA) and, at the end, the rebuild read them.
#pragma once

#include <cooperative_groups.h>

#include "jacobi.cuh"

namespace tnn {
namespace jac {

// Rows per lane and output columns per warp of the SVT rebuild.
__host__ __device__ constexpr int rebuild_rows(int R, int L) { return (R * L + 31) / 32; }
__host__ __device__ constexpr int rebuild_jb(int R, int L)
{
    return rebuild_rows(R, L) <= 6 ? 4 : (rebuild_rows(R, L) <= 12 ? 2 : 1);
}

// Elements of one super-block buffer: sK columns of ldA, then their sK
// scales, rounded up to 16 bytes.
__host__ __device__ inline size_t cluster_buf_elems(int ldA, int sK, int elem)
{
    const size_t e = (size_t)ldA * sK + sK;
    const size_t per16 = 16 / elem;
    return (e + per16 - 1) / per16 * per16;
}

// Dynamic shared memory of one cluster CTA: three super-block buffers, then
// sigma and |s|^2 of its two home super-blocks (2 sK each) and the kept
// list and coefficients (npad each).  The rebuild's per-warp coefficients
// (W x JB x npad) use the spare buffer, which must hold them.
__host__ __device__ inline size_t cluster_smem_bytes(int ldA, int sK, int npad, int elem)
{
    const size_t bufs = 3 * cluster_buf_elems(ldA, sK, elem) * elem;
    const size_t small = (size_t)4 * sK * elem + (size_t)npad * (elem + 4);
    return bufs + ((small + 255) & ~(size_t)255);
}

constexpr int kMaxCluster = 16;  // 16 is a non-portable cluster size (opted into at launch)

// Thread bound of the cluster kernels: the single-CTA bound rounded down to
// a multiple of 128 threads, since registers are granted for whole groups of
// four warps (a bound of 288 threads leaves no more registers than 384).
template <typename T, int K, int R>
struct ClusterBound {
    static constexpr int b = Bound<T, K, R, false>::value;
    static constexpr int value = b >= 128 ? b / 128 * 128 : b;
};

// Buffer roles (top, bottom, spare) of CTA `rank` after k super-block moves.
// CTA 0 keeps its top and swaps bottom and spare; every other CTA takes the
// spare as its top, the old top buffer as its bottom, the old bottom as spare.
__device__ __forceinline__ void cluster_roles(int rank, int k, int& top, int& bot, int& spare)
{
    if (rank == 0) {
        top = 0;
        bot = (k & 1) ? 2 : 1;
        spare = (k & 1) ? 1 : 2;
    } else {
        const int q = k % 3;
        top = q == 0 ? 0 : (q == 1 ? 2 : 1);
        bot = q == 0 ? 1 : (q == 1 ? 0 : 2);
        spare = q == 0 ? 2 : (q == 1 ? 1 : 0);
    }
}

// Copy `elems` (a multiple of 16 bytes) from another CTA's shared memory.
template <typename T>
__device__ __forceinline__ void pull_block(T* dst, const T* src, size_t elems, int tid, int nthr)
{
    const float4* s4 = reinterpret_cast<const float4*>(src);
    float4* d4 = reinterpret_cast<float4*>(dst);
    const size_t n4 = elems * sizeof(T) / 16;
    for (size_t e = tid; e < n4; e += nthr) d4[e] = s4[e];
}

// One round of s disjoint block pairs of the CTA's two super-blocks.
// kind 0: cross pairs (p_i, q_(i+t) mod s), with the within-block rounds when
// `within`; kind 1: the circle-method step t inside the top (pairs < s/2)
// and inside the bottom super-block (pairs >= s/2).
template <typename T, int K, int R, int L>
__device__ __forceinline__ void cluster_round(T* topA, T* topD, T* botA, T* botD, int s, int ldA, int kind, int t,
                                              bool within, T tol, int hl, int warp, int lane, int NG,
                                              Counters& cnt)
{
    constexpr int GPW = 32 / L;
    for (int base = warp * GPW; base < s; base += NG) {
        const int pr = base + lane / L;
        const bool active = pr < s;
        int bI = 0, bJ = 0;
        T *AI = topA, *AJ = botA, *DI = topD, *DJ = botD;
        if (active) {
            if (kind == 0) {
                bI = pr;
                bJ = pr + t < s ? pr + t : pr + t - s;
            } else {
                const int h = s / 2;
                const int p = pr < h ? pr : pr - h;
                bI = block_at(s, p, t);
                bJ = block_at(s, s - 1 - p, t);
                if (pr >= h) {
                    AI = botA;
                    DI = botD;
                } else {
                    AJ = topA;
                    DJ = topD;
                }
            }
        }
        Regs<T, K, R, false> Sr;
        Slot<T> st;
        const Counters cnt0 = cnt;
        load_cols<T, K, R, L, false>(Sr, st, AI, AJ, nullptr, DI, DJ, ldA, bI, bJ, hl, active);
        if (within) {
            gather_state<T, K, R, L, false>(Sr, st);
            do_rounds<T, K, R, L, false, false>(Sr, tol, hl, cnt, std::make_integer_sequence<int, K - 1>{});
            scatter_state<T, K, R, L, false>(Sr, st, hl);
        }
        cross_rounds<T, K, R, L, false>(Sr, st, tol, hl, cnt, std::make_integer_sequence<int, K>{});
        store_cols<T, K, R, L, false>(Sr, st, AI, AJ, nullptr, DI, DJ, ldA, bI, bJ, hl, active);
        if (!active) cnt = cnt0;
    }
    __syncthreads();
}

template <typename T, int K, int R, int L, bool ITEMS>
__global__ void __launch_bounds__(ClusterBound<T, K, R>::value) jacobi_cluster_kernel(KArgs<T> a)
{
    namespace cg = cooperative_groups;
    // every CTA of a cluster reads the same flag before its first barrier:
    // all of them return here or none does
    if (a.ctl && a.ctl->done) return;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int C = (int)cl.num_blocks(), rank = (int)cl.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int W = blockDim.x >> 5, nthr = blockDim.x;
    const int slice = blockIdx.x / C;
    // batched: per-cluster slice parameters from the item table
    const SliceItem* item = ITEMS ? a.items + slice : nullptr;
    // a batched ADMM job that has stopped (the same flag for every CTA of the cluster)
    const AdmmCtl* ictl = item ? item->ctl : nullptr;
    if (ictl && ictl->done) return;
    const int m = item ? item->m : a.m, n = item ? item->n : a.n, nb = item ? item->nb : a.nb;
    const int ldA = a.ldA, tr = item ? item->tr : a.tr;
    const int npad = nb * K;
    const int s = nb / (2 * C), sK = s * K;  // blocks and columns per super-block
    const int64_t n1 = item ? item->n1 : a.n1, n2 = item ? item->n2 : a.n2;
    constexpr int GPW = 32 / L;
    const int hl = lane % L;
    const int NG = W * GPW;
    constexpr int RR = rebuild_rows(R, L);
    constexpr int JB = rebuild_jb(R, L);

    const size_t BS = cluster_buf_elems(ldA, sK, (int)sizeof(T));
    T* buf0 = reinterpret_cast<T*>(smem_raw);
    auto buf = [&](int b) { return buf0 + (size_t)b * BS; };
    T* sig = buf0 + 3 * BS;  // home super-blocks: top [0, sK), bottom [sK, 2 sK)
    T* nrm = sig + 2 * sK;
    T* kcf = nrm + 2 * sK;
    int* kidx = reinterpret_cast<int*>(kcf + npad);
    __shared__ T* s_col[2 * kMaxCluster];  // per super-block id: its columns, at home
    __shared__ T* s_sig[kMaxCluster];
    __shared__ T* s_nrm[kMaxCluster];
    __shared__ int s_rotv[2], s_keep, s_nonfinite;
    __shared__ double s_nuc, s_fro;
    __shared__ unsigned long long s_pairs, s_rots;

    if (tid == 0) {
        s_fro = 0.0;
        s_rotv[0] = 0;
        s_rotv[1] = 0;
        s_pairs = 0;
        s_rots = 0;
        s_nonfinite = 0;
        s_nuc = 0.0;
        s_keep = 0;
    }
    T* src = item ? static_cast<T*>(item->data) : a.data + (size_t)slice * n1 * n2;

    // ---- load the two home super-blocks: id rank (top, buffer 0) and id
    // 2C - 1 - rank (bottom, buffer 1); pad rows and columns with zeros
    for (size_t e = tid; e < 2 * BS; e += nthr) buf0[e] = T(0);
    __syncthreads();
    for (int c = tid; c < sK; c += nthr) {
        buf(0)[(size_t)ldA * sK + c] = T(1);
        buf(1)[(size_t)ldA * sK + c] = T(1);
    }
    T fro = T(0);  // this thread's share of ||A||_F^2
    for (int h = 0; h < 2; ++h) {
        const int c0 = (h == 0 ? rank : 2 * C - 1 - rank) * sK;
        const int nloc = n - c0 < sK ? (n - c0 > 0 ? n - c0 : 0) : sK;
        T* A = buf(h);
        const int64_t tot = (int64_t)m * nloc;
        for (int64_t e = tid; e < tot; e += nthr) {
            int r, c;
            if (tr) { r = (int)(e / nloc); c = (int)(e % nloc); }  // source row c0 + c, column r
            else { c = (int)(e / m); r = (int)(e % m); }
            const T v = tr ? src[(size_t)(c0 + c) + (size_t)n1 * r] : src[(size_t)r + (size_t)n1 * (c0 + c)];
            A[(size_t)c * ldA + r] = v;
            fro = fma(v, v, fro);
        }
    }
    fro = group_sum<32>(fro);
    if (lane == 0) atomicAdd(&s_fro, (double)fro);
    cl.sync();
    // ||A||_F^2 of the whole slice, summed over the cluster in rank order (the
    // same value, hence the same decision, in every CTA): a slice whose
    // Frobenius norm is below the threshold has every singular value below
    // it, so Y = 0 and the sweeps are skipped (the rebuild keeps nothing)
    const T tau = a.ctl ? (T)(1.0 / a.ctl->beta) : (ictl ? (T)(1.0 / ictl->beta) : (T)(item ? item->tau : a.tau));
    double fro_all = 0.0;
    for (int r = 0; r < C; ++r) fro_all += *cl.map_shared_rank(&s_fro, r);
    const bool skip = fro_all * (1.0 + 1e-3) < (double)tau * (double)tau;

    // ---- sweeps
    const T tol = sqrt((T)m) * Num<T>::unit();
    Counters cnt{0, 0, 0};
    int sweeps = 0, converged = skip ? 1 : 0;
    const int max_sweeps = a.max_sweeps > 0 ? a.max_sweeps : 30;
    const int nss = 2 * C - 1;
    int k = 0;  // super-block moves so far
    while (!skip && sweeps < max_sweeps) {
        const int par = sweeps & 1;
        const int big0 = cnt.big;
        for (int ss = 0; ss < nss; ++ss, ++k) {
            int it, ib, is;
            cluster_roles(rank, k, it, ib, is);
            T* PA = buf(it);
            T* QA = buf(ib);
            T* PD = PA + (size_t)ldA * sK;
            T* QD = QA + (size_t)ldA * sK;
            if (ss == 0) {
                cluster_round<T, K, R, L>(PA, PD, QA, QD, s, ldA, 0, 0, true, tol, hl, warp, lane, NG, cnt);
                for (int t = 0; t < s - 1; ++t)
                    cluster_round<T, K, R, L>(PA, PD, QA, QD, s, ldA, 1, t, false, tol, hl, warp, lane, NG, cnt);
                for (int t = 1; t < s; ++t)
                    cluster_round<T, K, R, L>(PA, PD, QA, QD, s, ldA, 0, t, false, tol, hl, warp, lane, NG, cnt);
            } else {
                for (int t = 0; t < s; ++t)
                    cluster_round<T, K, R, L>(PA, PD, QA, QD, s, ldA, 0, t, false, tol, hl, warp, lane, NG, cnt);
            }
            // ---- move the super-blocks one place around the circle
            cl.sync();  // every CTA's rounds are done
            if (ss == 0 && tid == 0) s_rotv[par ^ 1] = 0;  // last read before this barrier
            if (rank >= 1) {  // phase A: new top <- left neighbour's top (CTA 0's bottom for CTA 1)
                int nt, nbt, nsp;
                const int from = rank == 1 ? 0 : rank - 1;
                cluster_roles(from, k, nt, nbt, nsp);
                const T* srcb = cl.map_shared_rank(buf(rank == 1 ? nbt : nt), from);
                pull_block(buf(is), srcb, BS, tid, nthr);
            }
            cl.sync();
            if (rank <= C - 2) {  // phase B: new bottom <- right neighbour's bottom
                int nt, nbt, nsp;
                cluster_roles(rank + 1, k, nt, nbt, nsp);
                const T* srcb = cl.map_shared_rank(buf(nbt), rank + 1);
                pull_block(buf(rank == 0 ? is : it), srcb, BS, tid, nthr);
            }
            cl.sync();
        }
        // vote: one increment per rotating warp into the counter of every CTA
        if (__any_sync(FULL, cnt.big != big0) && lane == 0)
            for (int r = 0; r < C; ++r) atomicAdd(cl.map_shared_rank(&s_rotv[par], r), 1);
        cl.sync();
        const int nrot = s_rotv[par];
        ++sweeps;
        if (nrot == 0) {
            converged = 1;
            break;
        }
    }
    if (cnt.pairs) atomicAdd(&s_pairs, (unsigned long long)cnt.pairs);
    if (cnt.rots) atomicAdd(&s_rots, (unsigned long long)cnt.rots);

    // ---- home again: sigma and |s|^2 of the two home super-blocks
    int it, ib, is;
    cluster_roles(rank, k, it, ib, is);
    for (int c = warp; c < 2 * sK; c += W) {
        const T* A = c < sK ? buf(it) : buf(ib);
        const int lc = c < sK ? c : c - sK;
        const T* col = A + (size_t)lc * ldA;
        T s2 = T(0);
        for (int r = lane; r < ldA; r += 32) s2 = fma(col[r], col[r], s2);
        s2 = group_sum<32>(s2);
        if (lane == 0) {
            const T sg = A[(size_t)ldA * sK + lc] * sqrt(s2);
            sig[c] = sg;
            nrm[c] = s2;
            if (!isfinite(sg)) s_nonfinite = 1;
        }
    }
    // where each super-block's columns live (every CTA follows the same role pattern)
    if (tid < 2 * C) {
        const int g = tid;
        const int o = g < C ? g : 2 * C - 1 - g;
        int ot, ob, os;
        cluster_roles(o, k, ot, ob, os);
        s_col[g] = cl.map_shared_rank(buf(g < C ? ot : ob), o);
    }
    if (tid < C) {
        s_sig[tid] = cl.map_shared_rank(sig, tid);
        s_nrm[tid] = cl.map_shared_rank(nrm, tid);
    }
    cl.sync();

    // ---- kept columns (sigma > tau) in ascending order, the same list in every CTA
    if (warp == 0) {
        int kk = 0;
        double nuc = 0.0;
        for (int cb = 0; cb < npad; cb += 32) {
            const int c = cb + lane;
            T sg = T(0), s2 = T(0);
            if (c < npad) {
                const int g = c / sK;
                const int o = g < C ? g : 2 * C - 1 - g;
                const int idx = (g < C ? 0 : sK) + (c - g * sK);
                sg = s_sig[o][idx];
                s2 = s_nrm[o][idx];
            }
            const bool keepf = c < npad && sg > tau && s2 > T(0);
            const unsigned bal = __ballot_sync(FULL, keepf);
            const int pos = kk + __popc(bal & ((1u << lane) - 1u));
            if (keepf) {
                kidx[pos] = c;
                kcf[pos] = (T(1) - tau / sg) / s2;
            }
            nuc += group_sum<32>(keepf ? (double)(sg - tau) : 0.0);
            kk += __popc(bal);
        }
        if (lane == 0) {
            s_keep = kk;
            s_nuc = nuc;
        }
    }
    unsigned long long pairs_all = 0, rots_all = 0;
    int nonfinite_all = 0;
    if (rank == 0 && tid == 0) {
        for (int r = 0; r < C; ++r) {
            pairs_all += *cl.map_shared_rank(&s_pairs, r);
            rots_all += *cl.map_shared_rank(&s_rots, r);
            nonfinite_all |= *cl.map_shared_rank(&s_nonfinite, r);
        }
    }
    __syncthreads();
    const int keep = s_keep;

    // ---- rebuild Y = sum_q cf_q s_q (s_q^T a0_j) over the cluster's warps;
    // each warp reads and then overwrites only its own output columns.  The
    // spare buffer holds the per-warp coefficients.
    constexpr int NV = 4 * JB;
    constexpr int GV = 32 / NV;
    T* gb = buf(is) + (size_t)warp * JB * npad;
    const int gw = rank * W + warp, GW = W * C;
    for (int j0 = gw * JB; j0 < n; j0 += JB * GW) {
        T x[JB][RR];
#pragma unroll
        for (int u = 0; u < JB; ++u)
#pragma unroll
            for (int q = 0; q < RR; ++q) {
                const int r = q * 32 + lane, j = j0 + u;
                x[u][q] = (r < m && j < n) ? (tr ? src[(size_t)j + (size_t)n1 * r] : src[(size_t)r + (size_t)n1 * j])
                                           : T(0);
            }
        for (int k0 = 0; k0 < keep; k0 += 4) {
            T g[NV];
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                T sv[RR];
                const int kc = (k0 + v < keep) ? kidx[k0 + v] : kidx[0];
                const T* col = s_col[kc / sK] + (size_t)(kc % sK) * ldA;
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
            const T tot = reduce_scatter<T, NV, 32>(g, lane);
            const int idx = lane / GV, vv = idx / JB, uu = idx % JB;
            if (lane % GV == 0 && k0 + vv < keep) gb[uu * npad + k0 + vv] = tot * kcf[k0 + vv];
        }
        __syncwarp();
        T y[JB][RR];
#pragma unroll
        for (int u = 0; u < JB; ++u)
#pragma unroll
            for (int q = 0; q < RR; ++q) y[u][q] = T(0);
        for (int kq = 0; kq < keep; ++kq) {
            const int kc = kidx[kq];
            const T* col = s_col[kc / sK] + (size_t)(kc % sK) * ldA;
            T sv[RR];
#pragma unroll
            for (int q = 0; q < RR; ++q) {
                const int r = q * 32 + lane;
                sv[q] = (r < ldA) ? col[r] : T(0);
            }
#pragma unroll
            for (int u = 0; u < JB; ++u) {
                const T coef = gb[u * npad + kq];
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
    cl.sync();  // no CTA leaves while another may still read its shared memory
    if (rank == 0 && tid == 0) {
        SliceStats st;
        st.nuc = s_nuc;
        st.pairs = (int64_t)pairs_all;
        st.rotations = (int64_t)rots_all;
        st.sweeps = sweeps;
        st.converged = converged;
        st.nonfinite = nonfinite_all;
        st.kept = keep;
        if (item) *item->stats = st;
        else a.stats[slice] = st;
    }
}

// Launch over p.n3 slices (items), clusters of p.cluster CTAs; p.nb is the
// largest block count of the launch.
template <typename T, int K, int R, int L, bool ITEMS>
cudaError_t launch_cluster(const JacobiPlan& p, KArgs<T> a, cudaStream_t s)
{
    void (*kern)(KArgs<T>) = jacobi_cluster_kernel<T, K, R, L, ITEMS>;
    cudaFuncAttributes attr;
    cudaError_t e = cudaFuncGetAttributes(&attr, kern);
    if (e != cudaSuccess) return e;
    const int C = p.cluster;
    if (C < 2 || C > kMaxCluster || p.nb % (4 * C) != 0) return cudaErrorInvalidValue;
    const int wmax = attr.maxThreadsPerBlock / 32;
    const int gpw = 32 / L;
    const int s_blocks = p.nb / (2 * C);  // block pairs per round
    int W = (s_blocks + gpw - 1) / gpw;
    if (W > wmax) W = wmax;
    if (W < 1) W = 1;
    const int npad = p.nb * K, sK = s_blocks * K;
    // the rebuild's per-warp coefficients live in the spare super-block buffer
    if ((size_t)W * rebuild_jb(R, L) * npad > cluster_buf_elems(p.ldA, sK, (int)sizeof(T)))
        return cudaErrorInvalidValue;
    const size_t smem = cluster_smem_bytes(p.ldA, sK, npad, (int)sizeof(T));
    if (C > 8) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    if (smem > 48 * 1024) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(p.n3 * C), 1, 1);
    cfg.blockDim = dim3((unsigned)(W * 32), 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kern, a);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace jac
}  // namespace tnn

namespace tnn {
// Cluster launches of one element type (jacobi_cluster_f32.cu / _f64.cu);
// `items` selects the item-table kernels of batched plans.
template <typename T>
cudaError_t launch_jacobi_svt_cluster(const JacobiPlan& p, jac::KArgs<T> a, bool items, cudaStream_t s);
}  // namespace tnn

// One cluster variant of a type; the plan's key is L * 1000 + R * 10 + K.
#define TNN_JAC_CLUSTER_CASE(T, L, R, K)                                                              \
    case L * 1000 + R * 10 + K:                                                                       \
        return items ? jac::launch_cluster<T, K, R, L, true>(p, a, s) : jac::launch_cluster<T, K, R, L, false>(p, a, s);
