// Completion server: continuous batching of Algorithm 1 jobs on one GPU.
//
// Jobs wait in submission order until their device footprint fits under the
// HBM cap; an admitted job gets one stream-ordered allocation holding B, the
// mask, X, M, the transformed tensor, its partial sums, Jacobi statistics
// and control block (beta, iteration, stop test), which stay resident until
// the result is taken.  Every scheduling pass queues the next chunk of
// iterations of every running job on its stream (jobs are spread over a
// fixed set of streams, so different jobs' kernels overlap), then reads the
// control block back asynchronously; a job whose stop test held or whose
// iteration cap was reached leaves at the next pass, and its room goes to
// the next queued job.  The host never waits on the GPU inside a pass.
//
// Each job runs exactly the kernels of tnn_complete, on its own buffers, so
// its result is the same bit for bit whatever else is running.  With
// TNN_SERVER_BATCH_KERNELS, the running jobs of a CUDA-core precision (FP32,
// FP64) instead share one launch sequence per iteration on a batch stream of
// their precision: the tables of the batched ADMM iteration (forward and
// inverse tiles, finalize items, slice groups) are rebuilt whenever the set
// of jobs in it changes, and every job still gets the iterates it would get
// alone, bit for bit.
#include <cuda_runtime.h>

#include <string.h>

#include <chrono>
#include <deque>
#include <map>
#include <memory>
#include <vector>

#include "tnn_internal.h"

using namespace tnn;

namespace {

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

struct SJob {
    int64_t id = 0;
    int state = 0;  // 0 queued, 1 running, 2 finished, 3 failed
    tnn_status result = TNN_OK;
    tnn_shape sh{};
    tnn_precision prec = TNN_FP32;
    tnn_admm_params prm{};
    const void* B_user = nullptr;
    const uint8_t* mask_user = nullptr;
    size_t bytes = 0;
    void* mem = nullptr;
    AdmmJob aj{};
    int lane = -1;
    int queued = 0;
    bool in_flight = false;
    cudaEvent_t ev = nullptr;
    AdmmCtl* h_ctl = nullptr;  // pinned slot
    AdmmCtl last{};
    double t_submit = 0, t_admit = -1, t_finish = -1;
    double work = 0;  // estimated: iterations x slices x m n^2 (one-sided Jacobi sweep cost)
    void* stage = nullptr;  // pinned copy of pageable host inputs (from the server's pool)
    size_t stage_size = 0;
    int batch = -1;  // batch lane (0 FP32, 1 FP64) when its iterations run batched
};

// One launch sequence per iteration for the running jobs of one precision.
struct BatchLane {
    static constexpr int kSide = 8;
    int elem = 4;
    int lane = -1;  // index of its stream among the server's lanes
    cudaStream_t side[kSide] = {};
    cudaEvent_t fork = nullptr, join[kSide] = {}, done = nullptr;
    bool in_flight = false;
    std::vector<int64_t> ids;  // jobs the device tables describe, in order
    std::vector<SliceGroup> groups;
    void* dmem = nullptr;  // tables and Jacobi scratch
    size_t dcap = 0;
    void* hstage = nullptr;  // pinned staging of the tables
    size_t hcap = 0;
    AdmmTileItem *d_fwd = nullptr, *d_inv = nullptr;
    AdmmJobItem* d_jobs = nullptr;
    SliceItem* d_slices = nullptr;
    int ntiles = 0, njobs = 0;
    int64_t passes = 0, rebuilds = 0;
};

// True for pageable host memory (a copy from it would block the host until
// the stream reaches it).
bool pageable(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return a.type == cudaMemoryTypeUnregistered;
}

// Device layout of one job (offsets into its allocation).
struct Layout {
    size_t B, mask, X, M, W, partials, stats, ctl, jwork, warm, wscr, wrec, tinfo, total;
};

// A job warm-starts its Jacobi from the previous iteration's right singular
// vectors (as tnn_complete does) when it runs on its own kernels: FP32
// precisions, slices one CTA holds, not a TNN_FP32 job of a server that
// batches those (the batched kernels start cold).
bool job_warm(tnn_precision prec, const JacobiPlan& jp, bool batching)
{
    return prec != TNN_FP64 && warm_supported(jp) && !(batching && prec == TNN_FP32);
}

Layout layout_of(const tnn_shape& sh, int elem, const JacobiPlan& jp, bool warm)
{
    const size_t N = (size_t)sh.n1 * sh.n2 * sh.n3, bytes = N * elem;
    Layout L;
    size_t o = 0;
    auto add = [&](size_t b) {
        const size_t at = o;
        o += up256(b);
        return at;
    };
    L.B = add(bytes);
    L.mask = add(N);
    L.X = add(bytes);
    L.M = add(bytes);
    L.W = add(bytes);
    L.partials = add((size_t)tube_partials_count(sh.n1 * sh.n2, sh.n3) * 4 * sizeof(double));
    L.stats = add(sizeof(SliceStats) * sh.n3);
    L.ctl = add(sizeof(AdmmCtl));
    L.jwork = add(jp.work_bytes);
    L.warm = warm ? add(warm_state_bytes(sh.n3, jp.n, elem)) : 0;
    L.wscr = warm ? add((size_t)sh.n3 * jp.ldA * jp.nb * jp.K * elem) : 0;
    L.wrec = warm ? add(sizeof(int) * sh.n3) : 0;
    const bool tail = warm && tail_supported(jp);  // the offloaded SVT tail's per-slice record
    L.tinfo = tail ? add(sizeof(float) * sh.n3 * tail_info_stride(jp.nb * jp.K)) : 0;
    L.total = o;
    return L;
}

}  // namespace

struct tnn_server {
    tnn_server_params p{};
    tnn_ctx* ctx = nullptr;
    std::vector<cudaStream_t> lanes;
    std::vector<int> lane_load;
    std::deque<int64_t> queue;
    std::map<int64_t, std::unique_ptr<SJob>> jobs;
    int64_t next_id = 1;
    size_t bytes = 0, peak = 0;
    int running = 0;
    int64_t completed = 0;
    std::vector<AdmmCtl*> pinned_blocks;  // 64 control-block slots each
    std::vector<AdmmCtl*> free_slots;
    // pinned staging buffers, kept for reuse (freeing pinned memory can
    // synchronise the device): size -> buffer
    std::multimap<size_t, void*> stage_free;
    std::vector<void*> stage_all;

    void* stage_get(size_t bytes, size_t* got)
    {
        auto it = stage_free.lower_bound(bytes);
        if (it != stage_free.end()) {
            void* p = it->second;
            *got = it->first;
            stage_free.erase(it);
            return p;
        }
        size_t sz = 1 << 20;
        while (sz < bytes) sz <<= 1;
        void* p = nullptr;
        if (cudaHostAlloc(&p, sz, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        stage_all.push_back(p);
        *got = sz;
        return p;
    }
    void stage_put(void* p, size_t sz) { stage_free.emplace(sz, p); }
    BatchLane batch[2];  // FP32, FP64 (TNN_SERVER_BATCH_KERNELS)
    cudaStream_t xfer = nullptr;  // result copies
    std::chrono::steady_clock::time_point t0;

    double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }

    AdmmCtl* slot()
    {
        if (free_slots.empty()) {
            AdmmCtl* blk = nullptr;
            if (cudaHostAlloc((void**)&blk, 64 * sizeof(AdmmCtl), cudaHostAllocDefault) != cudaSuccess) {
                cudaGetLastError();
                return nullptr;
            }
            pinned_blocks.push_back(blk);
            for (int i = 63; i >= 0; --i) free_slots.push_back(blk + i);
        }
        AdmmCtl* s = free_slots.back();
        free_slots.pop_back();
        return s;
    }
};

namespace {

// Admit the job at the head of the queue; false if it must wait.
bool admit(tnn_server* sv, SJob& j)
{
    const int elem = j.prec == TNN_FP64 ? 8 : 4;
    JacobiPlan jp;
    jacobi_plan(j.sh.n1, j.sh.n2, j.sh.n3, elem, &jp);
    const bool warm = job_warm(j.prec, jp, (sv->p.flags & TNN_SERVER_BATCH_KERNELS) != 0);
    const Layout L = layout_of(j.sh, elem, jp, warm);
    int lane = 0;
    const int bl = (sv->p.flags & TNN_SERVER_BATCH_KERNELS) && (j.prec == TNN_FP32 || j.prec == TNN_FP64)
                       ? (j.prec == TNN_FP64 ? 1 : 0)
                       : -1;
    if (bl >= 0) {
        lane = sv->batch[bl].lane;
    } else {
        for (int i = 1; i < sv->p.streams; ++i)
            if (sv->lane_load[i] < sv->lane_load[lane]) lane = i;
    }
    cudaStream_t s = sv->lanes[lane];
    void* mem = nullptr;
    if (cudaMallocAsync(&mem, L.total, s) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    AdmmCtl* hs = sv->slot();
    cudaEvent_t ev = nullptr;
    if (!hs || cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        if (hs) sv->free_slots.push_back(hs);
        cudaFreeAsync(mem, s);
        return false;
    }
    char* c = static_cast<char*>(mem);
    const size_t N = (size_t)j.sh.n1 * j.sh.n2 * j.sh.n3, bytes = N * elem;
    j.mem = mem;
    j.bytes = L.total;
    j.lane = lane;
    j.ev = ev;
    j.h_ctl = hs;
    j.aj.sh = j.sh;
    j.aj.prec = j.prec;
    j.aj.elem = elem;
    j.aj.prm = j.prm;
    j.aj.B = c + L.B;
    j.aj.mask = reinterpret_cast<const uint8_t*>(c + L.mask);
    j.aj.X = c + L.X;
    j.aj.M = c + L.M;
    j.aj.W = c + L.W;
    j.aj.ctl = reinterpret_cast<AdmmCtl*>(c + L.ctl);
    j.aj.partials = reinterpret_cast<double*>(c + L.partials);
    j.aj.stats = reinterpret_cast<SliceStats*>(c + L.stats);
    j.aj.jwork = jp.work_bytes ? c + L.jwork : nullptr;
    j.aj.jp = jp;
    if (warm) {
        j.aj.warm = c + L.warm;
        j.aj.wscr = c + L.wscr;
        j.aj.wrec = reinterpret_cast<int*>(c + L.wrec);
        if (tail_supported(jp)) j.aj.tinfo = reinterpret_cast<float*>(c + L.tinfo);
    }
    bool ok = cudaMemcpyAsync(c + L.B, j.B_user, bytes, cudaMemcpyDefault, s) == cudaSuccess &&
              cudaMemcpyAsync(c + L.mask, j.mask_user, N, cudaMemcpyDefault, s) == cudaSuccess;
    if (ok && warm)  // a cold start: no slice has its vectors yet
        ok = cudaMemsetAsync(c + L.warm, 0, L.wscr - L.warm, s) == cudaSuccess &&
             cudaMemsetAsync(c + L.wrec, 0, sizeof(int) * j.sh.n3, s) == cudaSuccess;
    if (ok) {
        ok = (elem == 8 ? launch_admm_init<double>((const double*)j.aj.B, j.aj.mask, (double*)j.aj.X,
                                                   (double*)j.aj.M, (int64_t)N, s)
                        : launch_admm_init<float>((const float*)j.aj.B, j.aj.mask, (float*)j.aj.X, (float*)j.aj.M,
                                                  (int64_t)N, s)) == cudaSuccess &&
             launch_ctl_init(j.aj.ctl, j.prm.beta0, j.prm.rho, j.prm.beta_max, j.prm.tol, j.prm.max_iter, s) ==
                 cudaSuccess &&
             admm_prepare_job(sv->ctx, j.aj, s) == TNN_OK;
    }
    // batched iterations take the CUDA-core operators; a job given
    // tensor-core ones runs alone on the batch stream
    j.batch = ok && bl >= 0 && !j.aj.opf.tc && !j.aj.opi.tc ? bl : -1;
    sv->bytes += L.total;
    if (sv->bytes > sv->peak) sv->peak = sv->bytes;
    sv->lane_load[lane] += 1;
    sv->running += 1;
    j.state = 1;
    j.t_admit = sv->now();
    if (!ok) {
        cudaGetLastError();
        j.state = 3;
        j.result = TNN_ECUDA;
        j.t_finish = j.t_admit;
        sv->running -= 1;
        sv->lane_load[lane] -= 1;
    }
    return true;
}

// Bytes a job would hold on the device.
size_t footprint(const tnn_shape& sh, tnn_precision prec)
{
    const int elem = prec == TNN_FP64 ? 8 : 4;
    JacobiPlan jp;
    if (!jacobi_plan(sh.n1, sh.n2, sh.n3, elem, &jp)) return 0;
    return layout_of(sh, elem, jp, job_warm(prec, jp, false)).total;
}

void release(tnn_server* sv, SJob& j)
{
    if (j.mem) {
        cudaFreeAsync(j.mem, sv->lanes[j.lane]);
        sv->bytes -= j.bytes;
        j.mem = nullptr;
    }
    if (j.ev) {
        cudaEventDestroy(j.ev);
        j.ev = nullptr;
    }
    if (j.h_ctl) {
        sv->free_slots.push_back(j.h_ctl);
        j.h_ctl = nullptr;
    }
    if (j.stage) {
        // a job that failed at admission may still have its copies in flight
        if (j.state == 3) cudaStreamSynchronize(sv->lanes[j.lane]);
        sv->stage_put(j.stage, j.stage_size);
        j.stage = nullptr;
    }
}

void fail_job(tnn_server* sv, SJob& j, int* nfin)
{
    j.state = 3;
    j.result = TNN_ECUDA;
    j.t_finish = sv->now();
    j.in_flight = false;
    sv->running -= 1;
    sv->lane_load[j.lane] -= 1;
    sv->completed += 1;
    ++*nfin;
}

// Point the batch lane's device tables at the jobs `ids` (uploaded through
// pinned staging on the batch stream).  The previous pass has completed.
cudaError_t batch_tables(tnn_server* sv, BatchLane& b, const std::vector<int64_t>& ids)
{
    std::vector<const AdmmJob*> jobs;
    for (int64_t id : ids) jobs.push_back(&sv->jobs[id]->aj);
    std::vector<AdmmTileItem> f, v;
    std::vector<AdmmJobItem> jt;
    std::vector<SliceItem> sl;
    build_admm_tiles(jobs, f, v, jt);
    if (!build_admm_slices(b.elem, jobs, b.groups, sl)) return cudaErrorInvalidValue;
    const size_t sf = up256(sizeof(AdmmTileItem) * f.size()), sj = up256(sizeof(AdmmJobItem) * jt.size()),
                 ss = up256(sizeof(SliceItem) * sl.size());
    const size_t tables = 2 * sf + sj + ss;
    size_t work = 0;
    for (auto& g : b.groups) work += up256(g.plan.work_bytes);
    cudaStream_t s = sv->lanes[b.lane];
    cudaError_t e;
    if (tables + work > b.dcap) {
        if (b.dmem) {
            cudaFreeAsync(b.dmem, s);
            sv->bytes -= b.dcap;
            b.dmem = nullptr;
            b.dcap = 0;
        }
        const size_t cap = (tables + work) * 5 / 4;
        if ((e = cudaMallocAsync(&b.dmem, cap, s)) != cudaSuccess) return e;
        b.dcap = cap;
        sv->bytes += cap;
        if (sv->bytes > sv->peak) sv->peak = sv->bytes;
    }
    if (tables > b.hcap) {
        if (b.hstage) sv->stage_put(b.hstage, b.hcap);
        b.hstage = sv->stage_get(tables, &b.hcap);
        if (!b.hstage) {
            b.hcap = 0;
            return cudaErrorMemoryAllocation;
        }
    }
    char* h = static_cast<char*>(b.hstage);
    char* d = static_cast<char*>(b.dmem);
    memcpy(h, f.data(), sizeof(AdmmTileItem) * f.size());
    memcpy(h + sf, v.data(), sizeof(AdmmTileItem) * v.size());
    memcpy(h + 2 * sf, jt.data(), sizeof(AdmmJobItem) * jt.size());
    memcpy(h + 2 * sf + sj, sl.data(), sizeof(SliceItem) * sl.size());
    if ((e = cudaMemcpyAsync(d, h, tables, cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
    b.d_fwd = reinterpret_cast<AdmmTileItem*>(d);
    b.d_inv = reinterpret_cast<AdmmTileItem*>(d + sf);
    b.d_jobs = reinterpret_cast<AdmmJobItem*>(d + 2 * sf);
    b.d_slices = reinterpret_cast<SliceItem*>(d + 2 * sf + sj);
    size_t w = tables;
    for (auto& g : b.groups) {
        g.work = g.plan.work_bytes ? d + w : nullptr;
        w += up256(g.plan.work_bytes);
    }
    b.ntiles = (int)f.size();
    b.njobs = (int)jt.size();
    b.ids = ids;
    b.rebuilds += 1;
    return cudaSuccess;
}

// Queue the next chunk of iterations of the batch lane's running jobs.
// Jobs with another Jacobi sweep cap than the first one wait for a later
// pass (the cap is one launch argument).
void batch_pass(tnn_server* sv, BatchLane& b, int* nfin)
{
    if (b.in_flight) return;
    std::vector<int64_t> ids;
    int sweeps = -1;
    for (auto& kv : sv->jobs) {
        const SJob& j = *kv.second;
        if (j.state != 1 || j.in_flight || j.batch != (int)(&b - sv->batch)) continue;
        if (sweeps < 0) sweeps = j.prm.jacobi_max_sweeps;
        if (j.prm.jacobi_max_sweeps == sweeps) ids.push_back(kv.first);
    }
    if (ids.empty()) return;
    cudaStream_t s = sv->lanes[b.lane];
    cudaError_t e = ids == b.ids ? cudaSuccess : batch_tables(sv, b, ids);
    if (e != cudaSuccess) b.ids.clear();
    for (int it = 0; e == cudaSuccess && it < sv->p.chunk; ++it)
        e = enqueue_admm_iteration(b.elem, b.d_fwd, b.d_inv, b.ntiles, b.d_jobs, b.njobs, b.groups, b.d_slices,
                                   sweeps, s, b.side, BatchLane::kSide, b.fork,
                                   b.join);
    for (int64_t id : ids) {
        SJob& j = *sv->jobs[id];
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(j.h_ctl, j.aj.ctl, sizeof(AdmmCtl), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaEventRecord(j.ev, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            fail_job(sv, j, nfin);
            continue;
        }
        j.queued += std::min(sv->p.chunk, std::max(0, j.prm.max_iter - j.queued));
        j.in_flight = true;
    }
    if (e == cudaSuccess && cudaEventRecord(b.done, s) == cudaSuccess) {
        b.in_flight = true;
        b.passes += 1;
    } else {
        cudaGetLastError();
        b.ids.clear();
    }
}

}  // namespace

extern "C" {

tnn_status tnn_server_footprint(tnn_shape sh, tnn_precision prec, uint64_t* bytes)
{
    if (!bytes) return TNN_EINVAL;
    *bytes = 0;
    if (sh.n1 <= 0 || sh.n2 <= 0 || sh.n3 <= 0) return TNN_EINVAL;
    if (!(prec == TNN_FP64 || prec == TNN_FP32 || prec == TNN_FP32_TF32X3 || prec == TNN_FP32_BF16SPLIT))
        return TNN_EINVAL;
    const size_t fp = footprint(sh, prec);
    if (fp == 0) return TNN_EINVAL;
    *bytes = fp;
    return TNN_OK;
}

tnn_status tnn_server_create(const tnn_server_params* p, tnn_server** out)
{
    if (!out) return TNN_EINVAL;
    *out = nullptr;
    tnn_server_params q{};
    if (p) q = *p;
    if (q.max_active < 0 || q.streams < 0 || q.chunk < 0) return TNN_EINVAL;
    if (q.policy != TNN_SERVER_FIFO && q.policy != TNN_SERVER_SHORTEST_FIRST) return TNN_EINVAL;
    if (q.flags & ~TNN_SERVER_BATCH_KERNELS) return TNN_EINVAL;
    if (q.hbm_cap_bytes == 0) q.hbm_cap_bytes = 150ull * 1000 * 1000 * 1000;
    if (q.streams == 0) q.streams = 8;
    if (q.chunk == 0) q.chunk = 8;
    std::unique_ptr<tnn_server> sv(new tnn_server);
    sv->p = q;
    tnn_status st = tnn_create(&sv->ctx, q.device);
    if (st != TNN_OK) return st;
    // keep freed job memory in the stream-ordered pool for the next jobs
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, q.device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
    const int nbl = (q.flags & TNN_SERVER_BATCH_KERNELS) ? 2 : 0;
    bool ok = true;
    for (int i = 0; ok && i < q.streams + nbl; ++i) {
        cudaStream_t s = nullptr;
        ok = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess;
        if (!ok) break;
        sv->lanes.push_back(s);
        sv->lane_load.push_back(0);
    }
    ok = ok && cudaStreamCreateWithFlags(&sv->xfer, cudaStreamNonBlocking) == cudaSuccess;
    for (int b = 0; ok && b < nbl; ++b) {
        BatchLane& L = sv->batch[b];
        L.elem = b == 1 ? 8 : 4;
        L.lane = q.streams + b;
        for (int i = 0; ok && i < BatchLane::kSide; ++i)
            ok = cudaStreamCreateWithFlags(&L.side[i], cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&L.join[i], cudaEventDisableTiming) == cudaSuccess;
        ok = ok && cudaEventCreateWithFlags(&L.fork, cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        tnn_server_destroy(sv.release());
        return TNN_ECUDA;
    }
    sv->t0 = std::chrono::steady_clock::now();
    *out = sv.release();
    return TNN_OK;
}

tnn_status tnn_server_submit(tnn_server* sv, const void* B, const uint8_t* mask, tnn_shape sh,
                             const tnn_admm_params* prm, tnn_precision prec, int64_t* job_id)
{
    if (!sv || !B || !mask || !prm || !job_id) return TNN_EINVAL;
    if (sh.n1 <= 0 || sh.n2 <= 0 || sh.n3 <= 0) return TNN_EINVAL;
    if (!(prec == TNN_FP64 || prec == TNN_FP32 || prec == TNN_FP32_TF32X3 || prec == TNN_FP32_BF16SPLIT))
        return TNN_EINVAL;
    if (!(prm->beta0 > 0.0) || !(prm->rho > 0.0) || !(prm->beta_max > 0.0) || prm->tol != prm->tol ||
        prm->max_iter < 0 || prm->jacobi_max_sweeps < 0)
        return TNN_EINVAL;
    const size_t fp = footprint(sh, prec);
    if (fp == 0 || fp > sv->p.hbm_cap_bytes) return TNN_EINVAL;  // slice too large, or never fits the cap
    std::unique_ptr<SJob> j(new SJob);
    j->id = sv->next_id++;
    j->sh = sh;
    j->prec = prec;
    j->prm = *prm;
    j->B_user = B;
    j->mask_user = mask;
    j->bytes = fp;
    {
        const double m = (double)(sh.n1 > sh.n2 ? sh.n1 : sh.n2), n = (double)(sh.n1 > sh.n2 ? sh.n2 : sh.n1);
        j->work = (double)prm->max_iter * (double)sh.n3 * m * n * n;
    }
    // pageable host inputs are copied now into pinned memory, so that the
    // admission copies never block the scheduling pass
    const size_t N = (size_t)sh.n1 * sh.n2 * sh.n3, bytes = N * (prec == TNN_FP64 ? 8 : 4);
    const bool pb = pageable(B), pm = pageable(mask);
    if (pb || pm) {
        const size_t sz = (pb ? (bytes + 255) / 256 * 256 : 0) + (pm ? N : 0);
        j->stage = sv->stage_get(sz, &j->stage_size);
        if (!j->stage) return TNN_ENOMEM;
        char* c = static_cast<char*>(j->stage);
        if (pb) {
            memcpy(c, B, bytes);
            j->B_user = c;
            c += (bytes + 255) / 256 * 256;
        }
        if (pm) {
            memcpy(c, mask, N);
            j->mask_user = reinterpret_cast<const uint8_t*>(c);
        }
    }
    j->t_submit = sv->now();
    *job_id = j->id;
    sv->queue.push_back(j->id);
    sv->jobs[j->id] = std::move(j);
    return TNN_OK;
}

tnn_status tnn_server_step(tnn_server* sv, int32_t* finished)
{
    if (!sv) return TNN_EINVAL;
    if (cudaSetDevice(sv->p.device) != cudaSuccess) {
        cudaGetLastError();
        return TNN_ECUDA;
    }
    int nfin = 0;
    // a finished batch pass: its jobs' events have completed too
    for (auto& b : sv->batch)
        if (b.in_flight) {
            const cudaError_t q = cudaEventQuery(b.done);
            if (q != cudaErrorNotReady) b.in_flight = false;
            if (q != cudaSuccess) cudaGetLastError();
        }
    // retire: running jobs whose last chunk has landed and that stopped
    for (auto& kv : sv->jobs) {
        SJob& j = *kv.second;
        if (j.state != 1 || !j.in_flight) continue;
        const cudaError_t q = cudaEventQuery(j.ev);
        if (q == cudaErrorNotReady) continue;
        j.in_flight = false;
        if (q != cudaSuccess) {
            cudaGetLastError();
            j.state = 3;
            j.result = TNN_ECUDA;
        } else {
            if (j.stage) {  // the admission copies came before this chunk
                sv->stage_put(j.stage, j.stage_size);
                j.stage = nullptr;
            }
            j.last = *j.h_ctl;
            if (!(j.last.done || j.queued >= j.prm.max_iter)) continue;
            j.state = 2;
            j.result = j.last.nonfinite ? TNN_ENONFINITE : (j.last.converged ? TNN_OK : TNN_ENOCONV);
        }
        j.t_finish = sv->now();
        sv->running -= 1;
        sv->lane_load[j.lane] -= 1;
        sv->completed += 1;
        ++nfin;
    }
    // admit while the footprint fits: in submission order, or the queued job
    // with the least estimated work first
    while (!sv->queue.empty()) {
        if (sv->p.policy == TNN_SERVER_SHORTEST_FIRST) {
            auto best = sv->queue.begin();
            for (auto it = sv->queue.begin(); it != sv->queue.end(); ++it)
                if (sv->jobs[*it]->work < sv->jobs[*best]->work) best = it;
            const int64_t id = *best;
            sv->queue.erase(best);
            sv->queue.push_front(id);
        }
        SJob& j = *sv->jobs[sv->queue.front()];
        if (sv->p.max_active > 0 && sv->running >= sv->p.max_active) break;
        if (sv->bytes + j.bytes > sv->p.hbm_cap_bytes) break;
        if (!admit(sv, j)) {
            if (sv->running > 0) break;  // retry when running jobs have released memory
            j.state = 3;                 // nothing left to wait for
            j.result = TNN_ENOMEM;
            j.t_finish = sv->now();
            sv->queue.pop_front();
            sv->completed += 1;
            ++nfin;
            continue;
        }
        sv->queue.pop_front();
        if (j.state == 3) {
            sv->completed += 1;
            ++nfin;
        }
    }
    // queue the next chunk of every running job that is not in flight
    for (auto& kv : sv->jobs) {
        SJob& j = *kv.second;
        if (j.state != 1 || j.in_flight || j.batch >= 0) continue;
        cudaStream_t s = sv->lanes[j.lane];
        int n = j.prm.max_iter - j.queued;
        if (n > sv->p.chunk) n = sv->p.chunk;
        if (n > 0 && admm_enqueue_iters(sv->ctx, j.aj, n, s) != TNN_OK) {
            j.state = 3;
            j.result = TNN_ECUDA;
            j.t_finish = sv->now();
            sv->running -= 1;
            sv->lane_load[j.lane] -= 1;
            sv->completed += 1;
            ++nfin;
            continue;
        }
        j.queued += n;
        if (cudaMemcpyAsync(j.h_ctl, j.aj.ctl, sizeof(AdmmCtl), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaEventRecord(j.ev, s) != cudaSuccess) {
            cudaGetLastError();
            j.state = 3;
            j.result = TNN_ECUDA;
            j.t_finish = sv->now();
            sv->running -= 1;
            sv->lane_load[j.lane] -= 1;
            sv->completed += 1;
            ++nfin;
            continue;
        }
        j.in_flight = true;
    }
    if (sv->p.flags & TNN_SERVER_BATCH_KERNELS)
        for (auto& b : sv->batch) batch_pass(sv, b, &nfin);
    if (finished) *finished = nfin;
    return TNN_OK;
}

tnn_status tnn_server_job_state(tnn_server* sv, int64_t id, int32_t* state)
{
    if (!sv || !state) return TNN_EINVAL;
    auto it = sv->jobs.find(id);
    if (it == sv->jobs.end()) return TNN_EINVAL;
    *state = it->second->state;
    return TNN_OK;
}

tnn_status tnn_server_take(tnn_server* sv, int64_t id, void* X_out, tnn_admm_report* rep, double times[3])
{
    if (!sv) return TNN_EINVAL;
    auto it = sv->jobs.find(id);
    if (it == sv->jobs.end()) return TNN_EINVAL;
    SJob& j = *it->second;
    if (j.state < 2) return TNN_EINVAL;  // not finished yet
    tnn_status res = j.result;
    if (j.state == 2 && X_out) {
        const size_t bytes = (size_t)j.sh.n1 * j.sh.n2 * j.sh.n3 * (j.prec == TNN_FP64 ? 8 : 4);
        // on the transfer stream, after the job's last chunk only (its lane
        // may already run other jobs' iterations)
        cudaStream_t s = sv->xfer;
        if (cudaStreamWaitEvent(s, j.ev, 0) != cudaSuccess ||
            cudaMemcpyAsync(X_out, j.aj.X, bytes, cudaMemcpyDefault, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            cudaGetLastError();
            res = TNN_ECUDA;
        } else if (ctx_check_tc(sv->ctx) != TNN_OK) {
            res = TNN_ECUDA;
        }
    }
    if (rep) {
        rep->iters = j.last.iter;
        rep->converged = j.last.converged;
        rep->rel_change = j.last.rel_change;
        rep->primal_res = j.last.primal_res;
        rep->beta_final = j.last.beta;
        rep->jacobi_sweeps_max = j.last.sweeps_max;
        rep->jacobi_unconverged = j.last.unconverged;
    }
    if (times) {
        times[0] = j.t_submit;
        times[1] = j.t_admit;
        times[2] = j.t_finish;
    }
    if (j.lane >= 0) release(sv, j);
    if (j.stage) {
        sv->stage_put(j.stage, j.stage_size);
        j.stage = nullptr;
    }
    sv->jobs.erase(it);
    return res;
}

tnn_status tnn_server_stats(const tnn_server* sv, int64_t out[6])
{
    if (!sv || !out) return TNN_EINVAL;
    int64_t fin = 0;
    for (auto& kv : sv->jobs) fin += kv.second->state >= 2 ? 1 : 0;
    out[0] = (int64_t)sv->queue.size();
    out[1] = sv->running;
    out[2] = fin;
    out[3] = (int64_t)sv->bytes;
    out[4] = (int64_t)sv->peak;
    out[5] = sv->completed;
    return TNN_OK;
}

void tnn_server_destroy(tnn_server* sv)
{
    if (!sv) return;
    cudaSetDevice(sv->p.device);
    for (auto s : sv->lanes) cudaStreamSynchronize(s);
    for (auto& kv : sv->jobs)
        if (kv.second->lane >= 0) release(sv, *kv.second);
    for (auto& b : sv->batch) {
        if (b.dmem && b.lane >= 0) cudaFreeAsync(b.dmem, sv->lanes[b.lane]);
        for (int i = 0; i < BatchLane::kSide; ++i) {
            if (b.side[i]) cudaStreamSynchronize(b.side[i]);
            if (b.side[i]) cudaStreamDestroy(b.side[i]);
            if (b.join[i]) cudaEventDestroy(b.join[i]);
        }
        if (b.fork) cudaEventDestroy(b.fork);
        if (b.done) cudaEventDestroy(b.done);
    }
    for (auto s : sv->lanes) cudaStreamSynchronize(s);
    for (auto s : sv->lanes) cudaStreamDestroy(s);
    if (sv->xfer) cudaStreamDestroy(sv->xfer);
    for (auto b : sv->pinned_blocks) cudaFreeHost(b);
    for (auto b : sv->stage_all) cudaFreeHost(b);
    tnn_destroy(sv->ctx);
    delete sv;
}

}  // extern "C"
