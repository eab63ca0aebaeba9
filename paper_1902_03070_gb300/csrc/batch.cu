// Batched t-SVT over many tensors of different shapes (the slices of many
// uneven tensors through one launch sequence, recorded as a CUDA graph).
//
// A plan holds, on the device: an item table of 128-pixel tiles for the
// forward and the inverse tube transform of every tensor (one grid covers
// every tile of every tensor), and the frontal slices of all tensors grouped
// by Jacobi variant (one launch per group, one CTA per slice, per-slice
// shapes and thresholds from an item table).  A run is forward transforms ->
// one Jacobi launch per group -> inverse transforms on one stream, or one
// graph launch replaying them.  Creating a plan with autotuning times every
// compiled Jacobi variant that covers a group's slices on the plan's own data
// and keeps the fastest (cached per shape class for the process).
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "tnn_internal.h"

namespace tnn {
namespace {

constexpr int BBM = 128;  // pixels per tile
constexpr int BBN = 64;   // output tube positions per pass
constexpr int BBK = 16;   // input tube positions per stage
constexpr int BNT = 256;

template <typename T>
__global__ void __launch_bounds__(BNT) tube_batched_kernel(const TubeItem* __restrict__ items)
{
    const TubeItem it = items[blockIdx.x];
    const T* __restrict__ in = static_cast<const T*>(it.in);
    T* __restrict__ out = static_cast<T*>(it.out);
    const T* __restrict__ op = static_cast<const T*>(it.op);
    const int64_t P = it.P, p0 = it.p0;
    const int n3 = it.n3;
    __shared__ __align__(16) T As[BBK][BBM];
    __shared__ T Ts[BBK][BBN];
    const int tid = threadIdx.x, tp = tid & 31, tq = tid >> 5;
    for (int q0 = 0; q0 < n3; q0 += BBN) {
        T acc[8][4];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[i][c] = T(0);
        for (int j0 = 0; j0 < n3; j0 += BBK) {
            __syncthreads();
            for (int e = tid; e < BBK * BBM; e += BNT) {
                const int jj = e / BBM, pp = e % BBM;
                const int64_t p = p0 + pp;
                const int j = j0 + jj;
                As[jj][pp] = (p < P && j < n3) ? in[(size_t)p + (size_t)P * j] : T(0);
            }
            for (int e = tid; e < BBK * BBN; e += BNT) {
                const int jj = e / BBN, qq = e % BBN;
                const int j = j0 + jj, q = q0 + qq;
                Ts[jj][qq] = (j < n3 && q < n3) ? op[j + (size_t)n3 * q] : T(0);
            }
            __syncthreads();
#pragma unroll 4
            for (int jj = 0; jj < BBK; ++jj) {
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
            if (q >= n3) continue;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int64_t p = p0 + tp * 4 + c;
                if (p < P) out[(size_t)p + (size_t)P * q] = acc[i][c];
            }
        }
        __syncthreads();
    }
}

}  // namespace

template <typename T>
cudaError_t launch_tube_batched(const TubeItem* items, int count, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    tube_batched_kernel<T><<<count, BNT, 0, s>>>(items);
    return cudaGetLastError();
}
template cudaError_t launch_tube_batched<float>(const TubeItem*, int, cudaStream_t);
template cudaError_t launch_tube_batched<double>(const TubeItem*, int, cudaStream_t);

int tube_batched_tile() { return BBM; }

}  // namespace tnn

// ---- the plan --------------------------------------------------------------------
using namespace tnn;

struct tnn_tsvt_batch {
    struct Group {
        JacobiPlan plan;  // variant, largest block count, in_smem; n3 = slices
        int off = 0;      // first SliceItem of the group
        int count = 0;
        void* work = nullptr;
        double cost = 0;  // m n^2 of the group's largest slice (launch order)
    };
    int device = 0;
    int elem = 4;
    int flags = 0;
    std::vector<tnn_tsvt_item> items;
    std::vector<Group> groups;
    void* mem = nullptr;     // transformed tensors, operators, statistics, launch tables
    void* mem_w = nullptr;   // Jacobi working copies of groups kept in global memory
    TubeItem* d_fwd = nullptr;
    TubeItem* d_inv = nullptr;
    int ntiles = 0;
    SliceItem* d_slices = nullptr;
    SliceStats* d_stats = nullptr;
    int nslices = 0;
    static constexpr int kStreams = 8;
    cudaStream_t side[kStreams] = {};
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[kStreams] = {};
    cudaStream_t cap = nullptr;  // private stream the graph is captured on
    cudaGraphExec_t exec = nullptr;
    int launches = 0;
};

namespace {

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Shape {
    int n1, n2, n3;
    int m, n, tr;
};

Shape shape_of(const tnn_shape& sh)
{
    Shape s;
    s.n1 = (int)sh.n1; s.n2 = (int)sh.n2; s.n3 = (int)sh.n3;
    s.m = s.n1 >= s.n2 ? s.n1 : s.n2;
    s.n = s.n1 >= s.n2 ? s.n2 : s.n1;
    s.tr = s.n1 < s.n2 ? 1 : 0;
    return s;
}

int variant_key(const JacobiPlan& p) { return p.L * 1000 + p.RA * 10 + p.K; }

// Slice table of one group under the variant of `gp`: every slice of every
// tensor in `tensors`, largest (m n^2) first so the block scheduler starts
// the long slices before the short ones.
std::vector<SliceItem> group_slices(const tnn_tsvt_batch& b, const std::vector<int>& tensors,
                                    const std::vector<char*>& wbuf, const JacobiPlan& gp, int stats_off)
{
    std::vector<int> order(tensors);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        Shape a = shape_of(b.items[x].shape), c = shape_of(b.items[y].shape);
        return (double)a.m * a.n * a.n > (double)c.m * c.n * c.n;
    });
    std::vector<SliceItem> out;
    int so = stats_off;
    // block count of a slice: even; with clusters of C, a multiple of 4C
    const int q = gp.cluster > 1 ? 4 * gp.cluster : 2;
    for (int t : order) {
        const Shape s = shape_of(b.items[t].shape);
        const int nb = q * ((s.n + q * gp.K - 1) / (q * gp.K));
        for (int k = 0; k < s.n3; ++k) {
            SliceItem it{};
            it.data = wbuf[t] + (size_t)k * s.n1 * s.n2 * b.elem;
            it.n1 = s.n1; it.n2 = s.n2;
            it.m = s.m; it.n = s.n; it.tr = s.tr; it.nb = nb;
            it.tau = b.items[t].tau;
            it.stats = b.d_stats + so++;
            out.push_back(it);
        }
    }
    return out;
}

// Group plan of a variant over the group's largest oriented shape.
bool group_plan(int elem, int L, int R, int K, int mmax, int nmax, int count, JacobiPlan* gp)
{
    return jacobi_plan_variant(mmax, nmax, count, elem, L, R, K, gp);
}

cudaError_t jacobi_items(int elem, const JacobiPlan& gp, const SliceItem* d, int count, void* work, cudaStream_t s)
{
    return elem == 8 ? launch_jacobi_svt_items<double>(gp, d, count, 0, work, s)
                     : launch_jacobi_svt_items<float>(gp, d, count, 0, work, s);
}

cudaError_t tube_items(int elem, const TubeItem* d, int count, cudaStream_t s)
{
    return elem == 8 ? launch_tube_batched<double>(d, count, s) : launch_tube_batched<float>(d, count, s);
}

// Forward transforms, then each group on a side stream (groups spread over
// the side streams, longest slices first), then the inverse transforms after all
// groups.  Valid both in a captured stream and on a live one.
cudaError_t enqueue(tnn_tsvt_batch* b, cudaStream_t s, bool inverse = true)
{
    cudaError_t e;
    if ((e = tube_items(b->elem, b->d_fwd, b->ntiles, s)) != cudaSuccess) return e;
    const int ns = std::min<int>(tnn_tsvt_batch::kStreams, (int)b->groups.size());
    if (ns <= 1) {
        for (auto& g : b->groups)
            if ((e = jacobi_items(b->elem, g.plan, b->d_slices + g.off, g.count, g.work, s)) != cudaSuccess) return e;
    } else {
        if ((e = cudaEventRecord(b->fork, s)) != cudaSuccess) return e;
        for (int i = 0; i < ns; ++i)
            if ((e = cudaStreamWaitEvent(b->side[i], b->fork, 0)) != cudaSuccess) return e;
        for (size_t gi = 0; gi < b->groups.size(); ++gi) {
            auto& g = b->groups[gi];
            if ((e = jacobi_items(b->elem, g.plan, b->d_slices + g.off, g.count, g.work, b->side[gi % ns])) !=
                cudaSuccess)
                return e;
        }
        for (int i = 0; i < ns; ++i) {
            if ((e = cudaEventRecord(b->join[i], b->side[i])) != cudaSuccess) return e;
            if ((e = cudaStreamWaitEvent(s, b->join[i], 0)) != cudaSuccess) return e;
        }
    }
    return inverse ? tube_items(b->elem, b->d_inv, b->ntiles, s) : cudaSuccess;
}

// Autotuner: time every compiled variant that covers a group on the plan's
// own slices (forward transforms re-run before each timing, since the SVT
// works in place) and keep the fastest.  Results are cached for the process
// by (element size, largest m, largest n, slices).
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, std::tuple<int, int, int>> g_tune;

void free_plan(tnn_tsvt_batch* b)
{
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (int i = 0; i < tnn_tsvt_batch::kStreams; ++i) {
        if (b->side[i]) cudaStreamDestroy(b->side[i]);
        if (b->join[i]) cudaEventDestroy(b->join[i]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->mem) cudaFree(b->mem);
    if (b->mem_w) cudaFree(b->mem_w);
    delete b;
}

}  // namespace

extern "C" {

tnn_status tnn_tsvt_batch_create(tnn_ctx* ctx, const tnn_tsvt_item* items, int32_t count, tnn_precision prec,
                                 int32_t flags, void* stream, tnn_tsvt_batch** out)
{
    if (!ctx || !out) return TNN_EINVAL;
    *out = nullptr;
    if (!items || count <= 0) return ctx_fail(ctx, TNN_EINVAL, "batch: no items");
    if (!(prec == TNN_FP64 || prec == TNN_FP32 || prec == TNN_FP32_TF32X3 || prec == TNN_FP32_BF16SPLIT))
        return ctx_fail(ctx, TNN_EINVAL, "batch: unknown precision");
    if (flags & ~(TNN_BATCH_GRAPH | TNN_BATCH_AUTOTUNE)) return ctx_fail(ctx, TNN_EINVAL, "batch: unknown flags");
    if (cudaSetDevice(ctx_device(ctx)) != cudaSuccess) {
        cudaGetLastError();
        return ctx_fail(ctx, TNN_ECUDA, "batch: cannot select the context's device");
    }
    const int elem = prec == TNN_FP64 ? 8 : 4;
    for (int i = 0; i < count; ++i) {
        const tnn_tsvt_item& it = items[i];
        if (!it.Z || !it.Y || it.shape.n1 <= 0 || it.shape.n2 <= 0 || it.shape.n3 <= 0 || !(it.tau >= 0.0) ||
            !(it.tau < 1e300) || it.shape.n1 > (1 << 20) || it.shape.n2 > (1 << 20) || it.shape.n3 > (1 << 20))
            return ctx_fail(ctx, TNN_EINVAL, "batch: invalid item");
        if (!is_device_pointer(it.Z) || !is_device_pointer(it.Y))
            return ctx_fail(ctx, TNN_EINVAL, "batch: item buffers must be device memory");
        JacobiPlan jp;
        if (!jacobi_plan(it.shape.n1, it.shape.n2, it.shape.n3, elem, &jp))
            return ctx_fail(ctx, TNN_EINVAL, "batch: slice too large");
    }
    cudaStream_t s = (cudaStream_t)stream;
    tnn_tsvt_batch* b = new tnn_tsvt_batch;
    b->device = ctx_device(ctx);
    b->elem = elem;
    b->flags = flags;
    b->items.assign(items, items + count);
    auto bail = [&](tnn_status st, const char* msg) {
        cudaGetLastError();
        free_plan(b);
        return ctx_fail(ctx, st, msg);
    };
#define BCK(call, msg)                          \
    do {                                        \
        if ((call) != cudaSuccess) return bail(TNN_ECUDA, msg); \
    } while (0)

    // ---- groups: tensors by the plan each would get alone: variant,
    // whether its working copies fit in one CTA's shared memory, and the
    // cluster that holds a slice too large for one CTA (a slice that fits is
    // never moved to global memory or a cluster by a larger one in its group)
    std::map<std::tuple<int, int, int>, std::vector<int>> by_variant;
    for (int i = 0; i < count; ++i) {
        JacobiPlan jp;
        jacobi_plan_mode(items[i].shape.n1, items[i].shape.n2, items[i].shape.n3, elem, false, &jp, true);
        by_variant[std::make_tuple(variant_key(jp), (int)jp.in_smem, jp.cluster)].push_back(i);
    }

    // ---- memory A: transformed tensors, operators, statistics, tube tables
    const int tile = tube_batched_tile();
    std::map<int, std::pair<size_t, size_t>> op_off;  // n3 -> (forward, inverse) offsets
    std::vector<size_t> w_off(count);
    size_t total = 0;
    int ntiles = 0, nslices = 0;
    for (int i = 0; i < count; ++i) {
        const tnn_shape& sh = items[i].shape;
        w_off[i] = total;
        total += up256((size_t)sh.n1 * sh.n2 * sh.n3 * elem);
        ntiles += (int)((sh.n1 * sh.n2 + tile - 1) / tile);
        nslices += (int)sh.n3;
        if (!op_off.count((int)sh.n3)) op_off[(int)sh.n3] = {0, 0};
    }
    for (auto& kv : op_off) {
        const size_t ob = up256((size_t)kv.first * kv.first * elem);
        kv.second.first = total;
        kv.second.second = total + ob;
        total += 2 * ob;
    }
    const size_t o_stats = total;
    total += up256(sizeof(SliceStats) * nslices);
    const size_t o_fwd = total;
    total += up256(sizeof(TubeItem) * ntiles);
    const size_t o_inv = total;
    total += up256(sizeof(TubeItem) * ntiles);
    const size_t o_sl = total;
    total += up256(sizeof(SliceItem) * nslices);
    if (cudaMalloc(&b->mem, total) != cudaSuccess) return bail(TNN_ENOMEM, "batch: device allocation failed");
    char* base = static_cast<char*>(b->mem);
    b->d_stats = reinterpret_cast<SliceStats*>(base + o_stats);
    b->d_fwd = reinterpret_cast<TubeItem*>(base + o_fwd);
    b->d_inv = reinterpret_cast<TubeItem*>(base + o_inv);
    b->d_slices = reinterpret_cast<SliceItem*>(base + o_sl);
    b->ntiles = ntiles;
    b->nslices = nslices;
    std::vector<char*> wbuf(count);
    for (int i = 0; i < count; ++i) wbuf[i] = base + w_off[i];

    for (auto& kv : op_off) {
        if (elem == 8) {
            BCK(launch_build_operator<double>((double*)(base + kv.second.first), kv.first, 0, 0, s), "batch: operator");
            BCK(launch_build_operator<double>((double*)(base + kv.second.second), kv.first, 1, 0, s), "batch: operator");
        } else {
            BCK(launch_build_operator<float>((float*)(base + kv.second.first), kv.first, 0, 0, s), "batch: operator");
            BCK(launch_build_operator<float>((float*)(base + kv.second.second), kv.first, 1, 0, s), "batch: operator");
        }
    }
    {
        std::vector<TubeItem> f, v;
        f.reserve(ntiles);
        v.reserve(ntiles);
        for (int i = 0; i < count; ++i) {
            const tnn_shape& sh = items[i].shape;
            const int64_t P = sh.n1 * sh.n2;
            const auto& oo = op_off[(int)sh.n3];
            for (int64_t p0 = 0; p0 < P; p0 += tile) {
                f.push_back(TubeItem{items[i].Z, wbuf[i], base + oo.first, P, p0, (int)sh.n3, 0});
                v.push_back(TubeItem{wbuf[i], items[i].Y, base + oo.second, P, p0, (int)sh.n3, 0});
            }
        }
        BCK(cudaMemcpyAsync(b->d_fwd, f.data(), sizeof(TubeItem) * ntiles, cudaMemcpyHostToDevice, s), "batch: table");
        BCK(cudaMemcpyAsync(b->d_inv, v.data(), sizeof(TubeItem) * ntiles, cudaMemcpyHostToDevice, s), "batch: table");
        BCK(cudaStreamSynchronize(s), "batch: table");
    }

    // ---- group plans (default variant, or the autotuner's choice)
    struct G { std::vector<int> tensors; int mmax = 0, nmax = 0, count = 0; double cost = 0; int key = 0, cluster = 0; };
    std::vector<G> gs;
    for (auto& kv : by_variant) {
        G g;
        g.tensors = kv.second;
        g.key = std::get<0>(kv.first);
        g.cluster = std::get<2>(kv.first);
        for (int t : g.tensors) {
            Shape sh = shape_of(items[t].shape);
            g.mmax = std::max(g.mmax, sh.m);
            g.nmax = std::max(g.nmax, sh.n);
            g.count += sh.n3;
            g.cost = std::max(g.cost, (double)sh.m * sh.n * sh.n);
        }
        gs.push_back(g);
    }
    // groups with the longest slices first, so they start at once
    std::sort(gs.begin(), gs.end(), [](const G& x, const G& y) { return x.cost > y.cost; });

    std::vector<std::tuple<int, int, int>> chosen(gs.size());
    for (size_t gi = 0; gi < gs.size(); ++gi)
        chosen[gi] = std::make_tuple(gs[gi].key / 1000, (gs[gi].key / 10) % 100, gs[gi].key % 10);

    if (flags & TNN_BATCH_AUTOTUNE) {
        int VL[32], VR[32], VK[32];
        const int nv = std::min(32, jacobi_svt_variants(elem, VL, VR, VK, 32));
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        BCK(cudaEventCreate(&e0), "batch: event");
        BCK(cudaEventCreate(&e1), "batch: event");
        int stats_off = 0;
        for (size_t gi = 0; gi < gs.size(); ++gi) {
            const G& g = gs[gi];
            if (g.cluster > 1) {  // cluster groups keep their variant
                stats_off += g.count;
                continue;
            }
            const auto key = std::make_tuple(elem, g.mmax, g.nmax, g.count);
            {
                std::lock_guard<std::mutex> lk(g_tune_mu);
                auto it = g_tune.find(key);
                if (it != g_tune.end()) {
                    chosen[gi] = it->second;
                    stats_off += g.count;
                    continue;
                }
            }
            float best = 1e30f;
            for (int v = 0; v < nv; ++v) {
                JacobiPlan gp;
                if (!group_plan(elem, VL[v], VR[v], VK[v], g.mmax, g.nmax, g.count, &gp)) continue;
                if (gp.L * gp.RA >= 4 * std::max(g.mmax, 32)) continue;  // far too tall for these slices
                std::vector<SliceItem> sl = group_slices(*b, g.tensors, wbuf, gp, stats_off);
                void* work = nullptr;
                if (gp.work_bytes && cudaMalloc(&work, gp.work_bytes) != cudaSuccess) {
                    cudaGetLastError();
                    continue;
                }
                bool ok = cudaMemcpyAsync(b->d_slices, sl.data(), sizeof(SliceItem) * sl.size(),
                                          cudaMemcpyHostToDevice, s) == cudaSuccess;
                float t_min = 1e30f;
                for (int rep = 0; ok && rep < 2; ++rep) {
                    ok = tube_items(elem, b->d_fwd, ntiles, s) == cudaSuccess &&
                         cudaEventRecord(e0, s) == cudaSuccess &&
                         jacobi_items(elem, gp, b->d_slices, g.count, work, s) == cudaSuccess &&
                         cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
                    float ms = 0.f;
                    if (ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) t_min = std::min(t_min, ms);
                }
                if (!ok) cudaGetLastError();
                if (work) cudaFree(work);
                if (ok && t_min < best) {
                    best = t_min;
                    chosen[gi] = std::make_tuple(VL[v], VR[v], VK[v]);
                }
            }
            {
                std::lock_guard<std::mutex> lk(g_tune_mu);
                g_tune[key] = chosen[gi];
            }
            stats_off += g.count;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }

    // ---- final slice table and working copies
    std::vector<SliceItem> all;
    all.reserve(nslices);
    size_t wtotal = 0;
    std::vector<size_t> woff(gs.size(), 0);
    for (size_t gi = 0; gi < gs.size(); ++gi) {
        tnn_tsvt_batch::Group grp;
        if (gs[gi].cluster > 1) {
            if (!jacobi_plan_mode(gs[gi].mmax, gs[gi].nmax, gs[gi].count, elem, false, &grp.plan, true) ||
                grp.plan.cluster != gs[gi].cluster || variant_key(grp.plan) != gs[gi].key)
                return bail(TNN_EINVAL, "batch: no cluster plan covers a group");
        } else if (!group_plan(elem, std::get<0>(chosen[gi]), std::get<1>(chosen[gi]), std::get<2>(chosen[gi]),
                               gs[gi].mmax, gs[gi].nmax, gs[gi].count, &grp.plan)) {
            return bail(TNN_EINVAL, "batch: no variant covers a group");
        }
        grp.off = (int)all.size();
        grp.count = gs[gi].count;
        grp.cost = gs[gi].cost;
        std::vector<SliceItem> sl = group_slices(*b, gs[gi].tensors, wbuf, grp.plan, grp.off);
        all.insert(all.end(), sl.begin(), sl.end());
        woff[gi] = wtotal;
        wtotal += up256(grp.plan.work_bytes);
        b->groups.push_back(grp);
    }
    if (wtotal) {
        if (cudaMalloc(&b->mem_w, wtotal) != cudaSuccess) return bail(TNN_ENOMEM, "batch: device allocation failed");
        for (size_t gi = 0; gi < gs.size(); ++gi)
            if (b->groups[gi].plan.work_bytes) b->groups[gi].work = static_cast<char*>(b->mem_w) + woff[gi];
    }
    BCK(cudaMemcpyAsync(b->d_slices, all.data(), sizeof(SliceItem) * all.size(), cudaMemcpyHostToDevice, s),
        "batch: table");
    BCK(cudaStreamSynchronize(s), "batch: table");

    for (int i = 0; i < tnn_tsvt_batch::kStreams; ++i) {
        BCK(cudaStreamCreateWithFlags(&b->side[i], cudaStreamNonBlocking), "batch: stream");
        BCK(cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming), "batch: event");
    }
    BCK(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming), "batch: event");
    b->launches = 2 + (int)b->groups.size();

    if (flags & TNN_BATCH_GRAPH) {
        // one uncaptured pass first (without the inverse transforms, so no
        // item buffer is written): it sets every Jacobi kernel's
        // shared-memory attribute outside the capture
        BCK(enqueue(b, s, false), "batch: launch");
        BCK(cudaStreamSynchronize(s), "batch: launch");
        BCK(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking), "batch: stream");
        cudaGraph_t graph = nullptr;
        BCK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal), "batch: capture");
        cudaError_t ce = enqueue(b, b->cap);
        cudaError_t ee = cudaStreamEndCapture(b->cap, &graph);
        if (ce != cudaSuccess || ee != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return bail(TNN_ECUDA, "batch: capture failed");
        }
        cudaError_t ie = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) return bail(TNN_ECUDA, "batch: graph instantiation failed");
        b->launches = 1;
    }
#undef BCK
    *out = b;
    return TNN_OK;
}

tnn_status tnn_tsvt_batch_run(tnn_tsvt_batch* b, void* stream)
{
    if (!b) return TNN_EINVAL;
    if (cudaSetDevice(b->device) != cudaSuccess) {
        cudaGetLastError();
        return TNN_ECUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = b->exec ? cudaGraphLaunch(b->exec, s) : enqueue(b, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return TNN_ECUDA;
    }
    return TNN_OK;
}

tnn_status tnn_tsvt_batch_info(const tnn_tsvt_batch* b, int32_t out[4])
{
    if (!b || !out) return TNN_EINVAL;
    out[0] = (int32_t)b->groups.size();
    out[1] = b->exec ? 1 : b->launches;
    out[2] = b->nslices;
    out[3] = b->exec ? 1 : 0;
    return TNN_OK;
}

tnn_status tnn_tsvt_batch_group(const tnn_tsvt_batch* b, int32_t g, int32_t out[6])
{
    if (!b || !out || g < 0 || g >= (int32_t)b->groups.size()) return TNN_EINVAL;
    const auto& gr = b->groups[g];
    out[0] = gr.plan.L;
    out[1] = gr.plan.RA;
    out[2] = gr.plan.K;
    out[3] = gr.count;
    out[4] = gr.plan.cluster > 1 ? 1 + gr.plan.cluster : gr.plan.in_smem;
    out[5] = gr.plan.m;
    return TNN_OK;
}

tnn_status tnn_tsvt_batch_profile(tnn_tsvt_batch* b, void* stream, double* ms)
{
    if (!b || !ms) return TNN_EINVAL;
    if (cudaSetDevice(b->device) != cudaSuccess) {
        cudaGetLastError();
        return TNN_ECUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int n = (int)b->groups.size() + 2;
    std::vector<cudaEvent_t> ev(n + 1, nullptr);
    bool ok = true;
    for (auto& e : ev) ok = ok && cudaEventCreate(&e) == cudaSuccess;
    ok = ok && cudaEventRecord(ev[0], s) == cudaSuccess && tube_items(b->elem, b->d_fwd, b->ntiles, s) == cudaSuccess &&
         cudaEventRecord(ev[1], s) == cudaSuccess;
    for (size_t gi = 0; ok && gi < b->groups.size(); ++gi) {
        auto& g = b->groups[gi];
        ok = jacobi_items(b->elem, g.plan, b->d_slices + g.off, g.count, g.work, s) == cudaSuccess &&
             cudaEventRecord(ev[gi + 2], s) == cudaSuccess;
    }
    ok = ok && tube_items(b->elem, b->d_inv, b->ntiles, s) == cudaSuccess && cudaEventRecord(ev[n], s) == cudaSuccess &&
         cudaEventSynchronize(ev[n]) == cudaSuccess;
    for (int i = 0; ok && i < n; ++i) {
        float t = 0.f;
        ok = cudaEventElapsedTime(&t, ev[i], ev[i + 1]) == cudaSuccess;
        ms[i] = t;
    }
    for (auto& e : ev)
        if (e) cudaEventDestroy(e);
    if (!ok) {
        cudaGetLastError();
        return TNN_ECUDA;
    }
    return TNN_OK;
}

tnn_status tnn_tsvt_batch_stats(tnn_tsvt_batch* b, void* stream, int64_t out[4])
{
    if (!b || !out) return TNN_EINVAL;
    if (cudaSetDevice(b->device) != cudaSuccess || cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) {
        cudaGetLastError();
        return TNN_ECUDA;
    }
    std::vector<SliceStats> h(b->nslices);
    if (cudaMemcpy(h.data(), b->d_stats, sizeof(SliceStats) * h.size(), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return TNN_ECUDA;
    }
    int64_t unconv = 0, nonfin = 0, rots = 0, smax = 0;
    for (const auto& st : h) {
        unconv += st.converged ? 0 : 1;
        nonfin += st.nonfinite ? 1 : 0;
        rots += st.rotations;
        smax = std::max<int64_t>(smax, st.sweeps);
    }
    out[0] = unconv;
    out[1] = nonfin;
    out[2] = rots;
    out[3] = smax;
    return nonfin ? TNN_ENONFINITE : TNN_OK;
}

void tnn_tsvt_batch_destroy(tnn_tsvt_batch* b)
{
    if (!b) return;
    cudaSetDevice(b->device);
    cudaDeviceSynchronize();
    free_plan(b);
}

}  // extern "C"
