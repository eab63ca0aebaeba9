// Batched ADMM steps: Algorithm 1 for many completion problems of different
// shapes at once, one CUDA-graph launch per iteration of all of them.
//
// A step is: the forward transforms with the Z = X - M/beta prologue of
// every tile of every tensor (one grid), the Jacobi SVTs of all slices (one
// launch per group of slices sharing a kernel variant and residency, groups
// on parallel streams; threshold 1/beta read from each job's control block),
// the inverse transforms with the fused X/M update and partial sums (one
// grid), and the per-job stop test and beta update (one block per job).
// Every kernel a job's tile, slice or finalize runs is the one tnn_complete
// runs for that job alone (the same device functions, the same per-tile
// partial-sum slots, the same Jacobi variant), so each job's iterates are
// those of a separate tnn_complete with the CUDA-core transforms, bit for
// bit; a job that has stopped is skipped by every kernel of later steps.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <memory>
#include <vector>

#include "tnn_internal.h"

using namespace tnn;

namespace tnn {

void build_admm_tiles(const std::vector<const AdmmJob*>& jobs, std::vector<AdmmTileItem>& fwd,
                      std::vector<AdmmTileItem>& inv, std::vector<AdmmJobItem>& jt)
{
    const int tp = tube_tile_pixels(), tq = tube_tile_outputs();
    fwd.clear();
    inv.clear();
    jt.assign(jobs.size(), AdmmJobItem{});
    for (size_t i = 0; i < jobs.size(); ++i) {
        const AdmmJob& j = *jobs[i];
        const int64_t P = j.sh.n1 * j.sh.n2;
        const int tx = tube_tiles_x(P), ty = tube_tiles_y(j.sh.n3);
        for (int y = 0; y < ty; ++y)
            for (int x = 0; x < tx; ++x) {
                AdmmTileItem a{};
                a.P = P;
                a.n3 = (int)j.sh.n3;
                a.p0 = (int64_t)x * tp;
                a.q0 = y * tq;
                a.tile = (int64_t)y * tx + x;
                a.ctl = j.ctl;
                a.partials = j.partials;
                AdmmTileItem fw = a, iv = a;
                fw.in = j.X;
                fw.in2 = j.M;
                fw.out = j.W;
                fw.op = j.opf.op;
                iv.in = j.W;
                iv.op = j.opi.op;
                iv.X = j.X;
                iv.M = j.M;
                iv.B = j.B;
                iv.mask = j.mask;
                fwd.push_back(fw);
                inv.push_back(iv);
            }
        jt[i].ctl = j.ctl;
        jt[i].partials = j.partials;
        jt[i].stats = j.stats;
        jt[i].n3 = j.sh.n3;
        jt[i].nblocks = tx * ty;
    }
}

bool build_admm_slices(int elem, const std::vector<const AdmmJob*>& jobs, std::vector<SliceGroup>& groups,
                       std::vector<SliceItem>& slices)
{
    groups.clear();
    slices.clear();
    auto vkey = [](const JacobiPlan& p) { return p.L * 1000 + p.RA * 10 + p.K; };
    std::map<std::tuple<int, int, int>, std::vector<int>> byv;
    for (size_t i = 0; i < jobs.size(); ++i) {
        const tnn_shape& sh = jobs[i]->sh;
        JacobiPlan jp;
        if (!jacobi_plan_mode(sh.n1, sh.n2, sh.n3, elem, false, &jp, true)) return false;
        byv[std::make_tuple(vkey(jp), (int)jp.in_smem, jp.cluster)].push_back((int)i);
    }
    struct G { std::vector<int> tensors; int mmax = 0, nmax = 0, count = 0, key = 0, cluster = 0; double cost = 0; };
    std::vector<G> gs;
    for (auto& kv : byv) {
        G g;
        g.tensors = kv.second;
        g.key = std::get<0>(kv.first);
        g.cluster = std::get<2>(kv.first);
        for (int t : g.tensors) {
            const tnn_shape& sh = jobs[t]->sh;
            const int m = (int)std::max(sh.n1, sh.n2), n = (int)std::min(sh.n1, sh.n2);
            g.mmax = std::max(g.mmax, m);
            g.nmax = std::max(g.nmax, n);
            g.count += (int)sh.n3;
            g.cost = std::max(g.cost, (double)m * n * n);
        }
        gs.push_back(g);
    }
    // groups with the longest slices first, so they start at once
    std::sort(gs.begin(), gs.end(), [](const G& x, const G& y) { return x.cost > y.cost; });
    for (const G& g : gs) {
        SliceGroup grp;
        bool ok;
        if (g.cluster > 1) {
            ok = jacobi_plan_mode(g.mmax, g.nmax, g.count, elem, false, &grp.plan, true) &&
                 grp.plan.cluster == g.cluster && vkey(grp.plan) == g.key;
        } else {
            ok = jacobi_plan_variant(g.mmax, g.nmax, g.count, elem, g.key / 1000, (g.key / 10) % 100, g.key % 10,
                                     &grp.plan);
        }
        if (!ok) return false;
        grp.off = (int)slices.size();
        grp.count = g.count;
        // longest slices first within the group as well
        std::vector<int> order(g.tensors);
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
            const tnn_shape &a = jobs[x]->sh, &c = jobs[y]->sh;
            const double ma = (double)std::max(a.n1, a.n2), na = (double)std::min(a.n1, a.n2);
            const double mc = (double)std::max(c.n1, c.n2), nc = (double)std::min(c.n1, c.n2);
            return ma * na * na > mc * nc * nc;
        });
        const int q = grp.plan.cluster > 1 ? 4 * grp.plan.cluster : 2;
        for (int t : order) {
            const AdmmJob& j = *jobs[t];
            const int n1 = (int)j.sh.n1, n2 = (int)j.sh.n2;
            const int m = std::max(n1, n2), n = std::min(n1, n2);
            const int nb = q * ((n + q * grp.plan.K - 1) / (q * grp.plan.K));
            for (int k = 0; k < (int)j.sh.n3; ++k) {
                SliceItem it{};
                it.data = static_cast<char*>(j.W) + (size_t)k * n1 * n2 * elem;
                it.n1 = n1;
                it.n2 = n2;
                it.m = m;
                it.n = n;
                it.tr = n1 < n2 ? 1 : 0;
                it.nb = nb;
                it.tau = 0.0;
                it.ctl = j.ctl;
                it.stats = j.stats + k;
                slices.push_back(it);
            }
        }
        groups.push_back(grp);
    }
    return true;
}

cudaError_t enqueue_admm_iteration(int elem, const AdmmTileItem* fwd, const AdmmTileItem* inv, int ntiles,
                                   const AdmmJobItem* jobs, int njobs, const std::vector<SliceGroup>& groups,
                                   const SliceItem* slices, int sweeps, cudaStream_t s, const cudaStream_t* side,
                                   int nside, cudaEvent_t fork, const cudaEvent_t* join)
{
    cudaError_t e;
    auto tiles = [&](const AdmmTileItem* d, int mode, cudaStream_t st) {
        return elem == 8 ? launch_tube_admm_batched<double>(d, ntiles, mode, st)
                         : launch_tube_admm_batched<float>(d, ntiles, mode, st);
    };
    auto jac = [&](const SliceGroup& g, cudaStream_t st) {
        return elem == 8 ? launch_jacobi_svt_items<double>(g.plan, slices + g.off, g.count, sweeps, g.work, st)
                         : launch_jacobi_svt_items<float>(g.plan, slices + g.off, g.count, sweeps, g.work, st);
    };
    if ((e = tiles(fwd, 1, s)) != cudaSuccess) return e;
    const int ns = std::min<int>(nside, (int)groups.size());
    if (ns <= 1) {
        for (const auto& g : groups)
            if ((e = jac(g, s)) != cudaSuccess) return e;
    } else {
        if ((e = cudaEventRecord(fork, s)) != cudaSuccess) return e;
        for (int i = 0; i < ns; ++i)
            if ((e = cudaStreamWaitEvent(side[i], fork, 0)) != cudaSuccess) return e;
        for (size_t gi = 0; gi < groups.size(); ++gi)
            if ((e = jac(groups[gi], side[gi % ns])) != cudaSuccess) return e;
        for (int i = 0; i < ns; ++i) {
            if ((e = cudaEventRecord(join[i], side[i])) != cudaSuccess) return e;
            if ((e = cudaStreamWaitEvent(s, join[i], 0)) != cudaSuccess) return e;
        }
    }
    if ((e = tiles(inv, 2, s)) != cudaSuccess) return e;
    return launch_admm_finalize_batched(jobs, njobs, s);
}

}  // namespace tnn

struct tnn_admm_batch {
    int device = 0, elem = 4, count = 0;
    tnn_admm_params prm{};
    std::vector<tnn_admm_item> items;
    std::vector<SliceGroup> groups;
    void* mem = nullptr;
    void* mem_w = nullptr;
    AdmmTileItem* d_fwd = nullptr;
    AdmmTileItem* d_inv = nullptr;
    AdmmJobItem* d_jobs = nullptr;
    SliceItem* d_slices = nullptr;
    AdmmCtl* d_ctl = nullptr;
    AdmmCtl* h_ctl = nullptr;  // pinned mirror
    int ntiles = 0, nslices = 0;
    static constexpr int kStreams = 8;
    cudaStream_t side[kStreams] = {};
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[kStreams] = {};
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec = nullptr;
    int synced = 0;  // h_ctl holds the state after the last sync
};

namespace {

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// One iteration of every job (valid on a live stream and under capture).
cudaError_t enqueue_step(tnn_admm_batch* b, cudaStream_t s)
{
    return enqueue_admm_iteration(b->elem, b->d_fwd, b->d_inv, b->ntiles, b->d_jobs, b->count, b->groups,
                                  b->d_slices, b->prm.jacobi_max_sweeps, s, b->side, tnn_admm_batch::kStreams,
                                  b->fork, b->join);
}

cudaError_t enqueue_reset(tnn_admm_batch* b, cudaStream_t s)
{
    cudaError_t e;
    for (int i = 0; i < b->count; ++i) {
        const tnn_admm_item& it = b->items[i];
        const int64_t N = it.shape.n1 * it.shape.n2 * it.shape.n3;
        e = b->elem == 8 ? launch_admm_init<double>((const double*)it.B, it.mask, (double*)it.X, (double*)it.M, N, s)
                         : launch_admm_init<float>((const float*)it.B, it.mask, (float*)it.X, (float*)it.M, N, s);
        if (e != cudaSuccess) return e;
        e = launch_ctl_init(b->d_ctl + i, b->prm.beta0, b->prm.rho, b->prm.beta_max, b->prm.tol, b->prm.max_iter, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

void free_plan(tnn_admm_batch* b)
{
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (int i = 0; i < tnn_admm_batch::kStreams; ++i) {
        if (b->side[i]) cudaStreamDestroy(b->side[i]);
        if (b->join[i]) cudaEventDestroy(b->join[i]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->mem) cudaFree(b->mem);
    if (b->mem_w) cudaFree(b->mem_w);
    if (b->h_ctl) cudaFreeHost(b->h_ctl);
    delete b;
}

}  // namespace

extern "C" {

tnn_status tnn_admm_batch_create(tnn_ctx* ctx, const tnn_admm_item* items, int32_t count,
                                 const tnn_admm_params* prm, tnn_precision prec, int32_t flags, void* stream,
                                 tnn_admm_batch** out)
{
    if (!ctx || !out) return TNN_EINVAL;
    *out = nullptr;
    if (!items || count <= 0 || !prm) return ctx_fail(ctx, TNN_EINVAL, "admm batch: no items or parameters");
    if (!(prec == TNN_FP64 || prec == TNN_FP32 || prec == TNN_FP32_TF32X3 || prec == TNN_FP32_BF16SPLIT))
        return ctx_fail(ctx, TNN_EINVAL, "admm batch: unknown precision");
    if (flags & ~TNN_BATCH_GRAPH) return ctx_fail(ctx, TNN_EINVAL, "admm batch: unknown flags");
    if (!(prm->beta0 > 0.0) || !(prm->rho > 0.0) || !(prm->beta_max > 0.0) || prm->tol != prm->tol ||
        prm->max_iter < 0 || prm->jacobi_max_sweeps < 0)
        return ctx_fail(ctx, TNN_EINVAL, "admm batch: invalid ADMM parameters");
    if (cudaSetDevice(ctx_device(ctx)) != cudaSuccess) {
        cudaGetLastError();
        return ctx_fail(ctx, TNN_ECUDA, "admm batch: cannot select the context's device");
    }
    const int elem = prec == TNN_FP64 ? 8 : 4;
    for (int i = 0; i < count; ++i) {
        const tnn_admm_item& it = items[i];
        if (!it.B || !it.mask || !it.X || !it.M || it.shape.n1 <= 0 || it.shape.n2 <= 0 || it.shape.n3 <= 0 ||
            it.shape.n1 > (1 << 20) || it.shape.n2 > (1 << 20) || it.shape.n3 > (1 << 20))
            return ctx_fail(ctx, TNN_EINVAL, "admm batch: invalid item");
        if (!is_device_pointer(it.B) || !is_device_pointer(it.mask) || !is_device_pointer(it.X) ||
            !is_device_pointer(it.M))
            return ctx_fail(ctx, TNN_EINVAL, "admm batch: item buffers must be device memory");
        JacobiPlan jp;
        if (!jacobi_plan(it.shape.n1, it.shape.n2, it.shape.n3, elem, &jp))
            return ctx_fail(ctx, TNN_EINVAL, "admm batch: slice too large");
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::unique_ptr<tnn_admm_batch> bp(new tnn_admm_batch);
    tnn_admm_batch* b = bp.get();
    b->device = ctx_device(ctx);
    b->elem = elem;
    b->count = count;
    b->prm = *prm;
    b->items.assign(items, items + count);
    auto bail = [&](tnn_status st, const char* msg) {
        cudaGetLastError();
        free_plan(bp.release());
        return ctx_fail(ctx, st, msg);
    };
#define BCK(call, msg)                                          \
    do {                                                        \
        if ((call) != cudaSuccess) return bail(TNN_ECUDA, msg); \
    } while (0)

    // ---- device layout: per job W, partials, statistics, control block;
    // operators per tube length; tile, job and slice tables
    std::vector<size_t> oW(count), oP(count), oS(count);
    std::vector<int> ntile(count);
    std::map<int64_t, std::pair<size_t, size_t>> ops;
    size_t total = 0;
    int ntiles = 0, nslices = 0;
    for (int i = 0; i < count; ++i) {
        const tnn_shape& sh = items[i].shape;
        const int64_t P = sh.n1 * sh.n2;
        ntile[i] = tube_tiles_x(P) * tube_tiles_y(sh.n3);
        oW[i] = total;
        total += up256((size_t)P * sh.n3 * elem);
        oP[i] = total;
        total += up256((size_t)ntile[i] * 4 * sizeof(double));
        oS[i] = total;
        total += up256(sizeof(SliceStats) * sh.n3);
        ntiles += ntile[i];
        nslices += (int)sh.n3;
        ops[sh.n3] = {0, 0};
    }
    for (auto& kv : ops) {
        const size_t ob = up256((size_t)kv.first * kv.first * elem);
        kv.second = {total, total + ob};
        total += 2 * ob;
    }
    const size_t oC = total;
    total += up256(sizeof(AdmmCtl) * count);
    const size_t oF = total;
    total += up256(sizeof(AdmmTileItem) * ntiles);
    const size_t oI = total;
    total += up256(sizeof(AdmmTileItem) * ntiles);
    const size_t oJ = total;
    total += up256(sizeof(AdmmJobItem) * count);
    const size_t oL = total;
    total += up256(sizeof(SliceItem) * nslices);
    if (cudaMalloc(&b->mem, total) != cudaSuccess) return bail(TNN_ENOMEM, "admm batch: device allocation failed");
    if (cudaHostAlloc((void**)&b->h_ctl, sizeof(AdmmCtl) * count, cudaHostAllocDefault) != cudaSuccess) {
        b->h_ctl = nullptr;
        return bail(TNN_ENOMEM, "admm batch: pinned allocation failed");
    }
    char* base = static_cast<char*>(b->mem);
    b->d_ctl = reinterpret_cast<AdmmCtl*>(base + oC);
    b->d_fwd = reinterpret_cast<AdmmTileItem*>(base + oF);
    b->d_inv = reinterpret_cast<AdmmTileItem*>(base + oI);
    b->d_jobs = reinterpret_cast<AdmmJobItem*>(base + oJ);
    b->d_slices = reinterpret_cast<SliceItem*>(base + oL);
    b->ntiles = ntiles;
    b->nslices = nslices;
    for (auto& kv : ops) {
        if (elem == 8) {
            BCK(launch_build_operator<double>((double*)(base + kv.second.first), kv.first, 0, 0, s), "operator");
            BCK(launch_build_operator<double>((double*)(base + kv.second.second), kv.first, 1, 0, s), "operator");
        } else {
            BCK(launch_build_operator<float>((float*)(base + kv.second.first), kv.first, 0, 0, s), "operator");
            BCK(launch_build_operator<float>((float*)(base + kv.second.second), kv.first, 1, 0, s), "operator");
        }
    }
    std::vector<AdmmJob> jobs(count);
    std::vector<const AdmmJob*> jp(count);
    for (int i = 0; i < count; ++i) {
        const tnn_admm_item& it = items[i];
        AdmmJob& j = jobs[i];
        j = AdmmJob{};
        j.sh = it.shape;
        j.prec = prec;
        j.elem = elem;
        j.B = it.B;
        j.mask = it.mask;
        j.X = it.X;
        j.M = it.M;
        j.W = base + oW[i];
        j.ctl = b->d_ctl + i;
        j.partials = reinterpret_cast<double*>(base + oP[i]);
        j.stats = reinterpret_cast<SliceStats*>(base + oS[i]);
        j.opf.op = base + ops[it.shape.n3].first;
        j.opi.op = base + ops[it.shape.n3].second;
        jp[i] = &j;
    }
    {
        std::vector<AdmmTileItem> f, v;
        std::vector<AdmmJobItem> jt;
        build_admm_tiles(jp, f, v, jt);
        BCK(cudaMemcpyAsync(b->d_fwd, f.data(), sizeof(AdmmTileItem) * ntiles, cudaMemcpyHostToDevice, s), "table");
        BCK(cudaMemcpyAsync(b->d_inv, v.data(), sizeof(AdmmTileItem) * ntiles, cudaMemcpyHostToDevice, s), "table");
        BCK(cudaMemcpyAsync(b->d_jobs, jt.data(), sizeof(AdmmJobItem) * count, cudaMemcpyHostToDevice, s), "table");
    }

    // ---- Jacobi groups: tensors by the plan each would get alone
    std::vector<SliceItem> all;
    if (!build_admm_slices(elem, jp, b->groups, all)) return bail(TNN_EINVAL, "admm batch: no plan covers a group");
    size_t wtotal = 0;
    std::vector<size_t> woff(b->groups.size(), 0);
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
        woff[gi] = wtotal;
        wtotal += up256(b->groups[gi].plan.work_bytes);
    }
    if (wtotal) {
        if (cudaMalloc(&b->mem_w, wtotal) != cudaSuccess) return bail(TNN_ENOMEM, "admm batch: allocation failed");
        for (size_t gi = 0; gi < b->groups.size(); ++gi)
            if (b->groups[gi].plan.work_bytes) b->groups[gi].work = static_cast<char*>(b->mem_w) + woff[gi];
    }
    BCK(cudaMemcpyAsync(b->d_slices, all.data(), sizeof(SliceItem) * all.size(), cudaMemcpyHostToDevice, s),
        "table");
    for (int i = 0; i < tnn_admm_batch::kStreams; ++i) {
        BCK(cudaStreamCreateWithFlags(&b->side[i], cudaStreamNonBlocking), "stream");
        BCK(cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming), "event");
    }
    BCK(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming), "event");
    BCK(enqueue_reset(b, s), "admm batch: state init");
    BCK(cudaStreamSynchronize(s), "admm batch: setup");

    if (flags & TNN_BATCH_GRAPH) {
        // one step's kernels need their shared-memory attributes set outside
        // a capture: set them by a launch on a throwaway control state (every
        // kernel returns at once on a stopped job)
        std::vector<AdmmCtl> stop(count);
        for (auto& c : stop) {
            c = AdmmCtl{};
            c.beta = 1.0;
            c.done = 1;
        }
        BCK(cudaMemcpyAsync(b->d_ctl, stop.data(), sizeof(AdmmCtl) * count, cudaMemcpyHostToDevice, s), "table");
        BCK(enqueue_step(b, s), "admm batch: launch");
        BCK(enqueue_reset(b, s), "admm batch: state init");
        BCK(cudaStreamSynchronize(s), "admm batch: setup");
        BCK(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking), "stream");
        cudaGraph_t graph = nullptr;
        BCK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal), "capture");
        const cudaError_t ce = enqueue_step(b, b->cap);
        const cudaError_t ee = cudaStreamEndCapture(b->cap, &graph);
        if (ce != cudaSuccess || ee != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return bail(TNN_ECUDA, "admm batch: capture failed");
        }
        const cudaError_t ie = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) return bail(TNN_ECUDA, "admm batch: graph instantiation failed");
    }
#undef BCK
    *out = bp.release();
    return TNN_OK;
}

tnn_status tnn_admm_batch_reset(tnn_admm_batch* b, void* stream)
{
    if (!b) return TNN_EINVAL;
    if (cudaSetDevice(b->device) != cudaSuccess || enqueue_reset(b, (cudaStream_t)stream) != cudaSuccess) {
        cudaGetLastError();
        return TNN_ECUDA;
    }
    b->synced = 0;
    return TNN_OK;
}

tnn_status tnn_admm_batch_step(tnn_admm_batch* b, int32_t iters, void* stream)
{
    if (!b || iters < 0) return TNN_EINVAL;
    if (cudaSetDevice(b->device) != cudaSuccess) {
        cudaGetLastError();
        return TNN_ECUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    for (int i = 0; i < iters; ++i) {
        const cudaError_t e = b->exec ? cudaGraphLaunch(b->exec, s) : enqueue_step(b, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return TNN_ECUDA;
        }
    }
    b->synced = 0;
    return TNN_OK;
}

tnn_status tnn_admm_batch_sync(tnn_admm_batch* b, void* stream, int32_t* running)
{
    if (!b) return TNN_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaSetDevice(b->device) != cudaSuccess ||
        cudaMemcpyAsync(b->h_ctl, b->d_ctl, sizeof(AdmmCtl) * b->count, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return TNN_ECUDA;
    }
    b->synced = 1;
    int r = 0;
    for (int i = 0; i < b->count; ++i) r += b->h_ctl[i].done ? 0 : 1;
    if (running) *running = r;
    return TNN_OK;
}

tnn_status tnn_admm_batch_run(tnn_admm_batch* b, void* stream)
{
    if (!b) return TNN_EINVAL;
    int32_t running = 1, queued = 0, chunk = 1;
    tnn_status st;
    if ((st = tnn_admm_batch_sync(b, stream, &running))) return st;
    while (running > 0 && queued < b->prm.max_iter) {
        const int n = std::min(chunk, b->prm.max_iter - queued);
        if ((st = tnn_admm_batch_step(b, n, stream))) return st;
        queued += n;
        if ((st = tnn_admm_batch_sync(b, stream, &running))) return st;
        if (chunk < 16) chunk *= 2;
    }
    return TNN_OK;
}

tnn_status tnn_admm_batch_report(const tnn_admm_batch* b, int32_t i, tnn_admm_report* rep)
{
    if (!b || !rep || i < 0 || i >= b->count || !b->synced) return TNN_EINVAL;
    const AdmmCtl& c = b->h_ctl[i];
    rep->iters = c.iter;
    rep->converged = c.converged;
    rep->rel_change = c.rel_change;
    rep->primal_res = c.primal_res;
    rep->beta_final = c.beta;
    rep->jacobi_sweeps_max = c.sweeps_max;
    rep->jacobi_unconverged = c.unconverged;
    return c.nonfinite ? TNN_ENONFINITE : (c.converged ? TNN_OK : TNN_ENOCONV);
}

void tnn_admm_batch_destroy(tnn_admm_batch* b)
{
    if (!b) return;
    cudaSetDevice(b->device);
    cudaDeviceSynchronize();
    free_plan(b);
}

}  // extern "C"
