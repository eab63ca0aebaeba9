// C ABI of libtnn (declared in include/tnn.h): argument checks, the context
// and its device workspace, host/device staging, and the drivers that chain
// the kernels of each call on the caller's stream.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "tnn_internal.h"

using namespace tnn;

struct tnn_ctx {
    int device = 0;
    std::string err;
    void* ws = nullptr;          // device workspace
    size_t ws_size = 0;
    size_t ws_off = 0;           // bump offset during one call
    AdmmCtl* h_ctl = nullptr;    // pinned host mirror of the control block
    std::map<std::tuple<int64_t, int, int, int>, void*> ops;  // (n3, elem, inverse, scaled) -> operator
    std::map<std::tuple<int64_t, int, int, int>, float*> tc_ops;  // (n3, inverse, scaled, bf16) -> tensor-core images
    int* d_err = nullptr;        // set by a tensor-core kernel whose bounded wait timed out
    int opt_jacobi_sweeps = 0;   // TNN_OPT_JACOBI_MAX_SWEEPS (0: the kernels' default)
    int opt_tc_polls = -1;       // TNN_OPT_TC_WAIT_POLLS (negative: the default limit)
    int opt_angle64 = 0;         // TNN_OPT_JACOBI_FP64_ANGLES
    int opt_small_stop = 1;      // TNN_OPT_JACOBI_SMALL_STOP
    int opt_sweep_log = 0;       // TNN_OPT_JACOBI_SWEEP_LOG
    float* d_sweep_log = nullptr;  // the log's device buffer (grown on demand)
    int64_t sweep_log_cap = 0;   // slices it holds
    float* last_sweep_log = nullptr;  // the log of the last Jacobi launch, if it kept one
    // the warm-start QR's side stream and its two events (none if their creation failed)
    cudaStream_t qr_stream = nullptr;
    cudaEvent_t ev_tail = nullptr, ev_qr = nullptr;
    int opt_warm = 1;            // TNN_OPT_ADMM_WARM_START (tnn_complete)
    SliceStats* last_stats = nullptr;
    int64_t last_n3 = 0;
    cudaStream_t last_stream = nullptr;
    // tracing: CUDA events around every kernel launch while enabled
    bool prof = false;
    struct Rec { int kind; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
};

namespace {

tnn_status fail(tnn_ctx* c, tnn_status s, const char* fmt, ...)
{
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return s;
}

#define CK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) return fail(ctx, TNN_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

bool is_device_ptr(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

// Workspace planning: a call first adds up what it needs, grows the
// workspace once if needed, then carves it.
struct Carve {
    size_t total = 0;
    size_t add(size_t b)
    {
        size_t off = total;
        total += align_up(b);
        return off;
    }
};

tnn_status ensure_ws(tnn_ctx* ctx, size_t bytes)
{
    if (bytes <= ctx->ws_size) return TNN_OK;
    // queued work may still use the old buffer
    CK(cudaDeviceSynchronize());
    if (ctx->ws) CK(cudaFree(ctx->ws));
    ctx->ws = nullptr;
    ctx->ws_size = 0;
    size_t b = align_up(bytes);
    if (cudaMalloc(&ctx->ws, b) != cudaSuccess) {
        cudaGetLastError();
        ctx->ws = nullptr;
        return fail(ctx, TNN_ENOMEM, "workspace allocation of %zu bytes failed", b);
    }
    ctx->ws_size = b;
    return TNN_OK;
}

inline void* at(tnn_ctx* ctx, size_t off) { return static_cast<char*>(ctx->ws) + off; }

// Tracing.  Each traced launch is bracketed by two events on its stream.
cudaEvent_t pool_event(tnn_ctx* ctx)
{
    if (!ctx->pool.empty()) {
        cudaEvent_t e = ctx->pool.back();
        ctx->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

struct Trace {
    tnn_ctx* ctx;
    int kind;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    Trace(tnn_ctx* c, int k, cudaStream_t st) : ctx(c), kind(k), s(st)
    {
        if (ctx->prof) {
            a = pool_event(ctx);
            cudaEventRecord(a, s);
        }
    }
    ~Trace()
    {
        if (a) {
            cudaEvent_t b = pool_event(ctx);
            cudaEventRecord(b, s);
            ctx->recs.push_back({kind, a, b});
        }
    }
};

// Kernel kinds reported by tnn_profile_read (array index, listed in tnn.h).
enum { K_TUBE = 0, K_TUBE_FWD_ADMM, K_JACOBI_SVT, K_TUBE_INV_ADMM, K_FINALIZE, K_CTL_INIT, K_ADMM_INIT,
       K_JACOBI_SVD, K_FACEWISE, K_DFT, K_JACOBI_PLAIN, K_WARM, K_SVT_TAIL, K_NKINDS };
#define TRACE_CAT2(a, b) a##b
#define TRACE_CAT(a, b) TRACE_CAT2(a, b)
#define TRACE(kind) Trace TRACE_CAT(trace_, __LINE__)(ctx, kind, s)

int elem_of(tnn_precision p) { return p == TNN_FP64 ? 8 : 4; }

bool prec_ok(tnn_precision p)
{
    return p == TNN_FP64 || p == TNN_FP32 || p == TNN_FP32_TF32X3 || p == TNN_FP32_BF16SPLIT;
}

bool shape_ok(const tnn_shape& s) { return s.n1 > 0 && s.n2 > 0 && s.n3 > 0; }

tnn_status set_device(tnn_ctx* ctx)
{
    CK(cudaSetDevice(ctx->device));
    return TNN_OK;
}

// Operator matrix for (n3, elem, inverse, scaled), built once per context.
tnn_status get_op(tnn_ctx* ctx, int64_t n3, int elem, int inverse, int scaled, cudaStream_t s, const void** out)
{
    auto key = std::make_tuple(n3, elem, inverse, scaled);
    auto it = ctx->ops.find(key);
    if (it != ctx->ops.end()) {
        *out = it->second;
        return TNN_OK;
    }
    void* p = nullptr;
    if (cudaMalloc(&p, (size_t)n3 * n3 * elem) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, TNN_ENOMEM, "operator allocation failed");
    }
    cudaError_t e = elem == 8 ? launch_build_operator<double>((double*)p, n3, inverse, scaled, s)
                              : launch_build_operator<float>((float*)p, n3, inverse, scaled, s);
    if (e != cudaSuccess) {
        cudaFree(p);
        return fail(ctx, TNN_ECUDA, "build_operator: %s", cudaGetErrorString(e));
    }
    // other streams may use the operator later: make it complete now
    CK(cudaStreamSynchronize(s));
    ctx->ops[key] = p;
    *out = p;
    return TNN_OK;
}

// Tensor-core operator images for (n3, inverse, scaled, BF16 or TF32 split),
// built once per context.
tnn_status get_op_tc(tnn_ctx* ctx, int64_t n3, int inverse, int scaled, bool bf, cudaStream_t s, const float** out)
{
    auto key = std::make_tuple(n3, inverse, scaled, bf ? 1 : 0);
    auto it = ctx->tc_ops.find(key);
    if (it != ctx->tc_ops.end()) {
        *out = it->second;
        return TNN_OK;
    }
    float* p = nullptr;
    if (cudaMalloc(&p, tube_tc_image_floats(n3, bf) * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, TNN_ENOMEM, "operator image allocation failed");
    }
    cudaError_t e = launch_build_operator_tc(p, n3, inverse, scaled, bf, s);
    if (e != cudaSuccess) {
        cudaFree(p);
        return fail(ctx, TNN_ECUDA, "build_operator_tc: %s", cudaGetErrorString(e));
    }
    CK(cudaStreamSynchronize(s));
    ctx->tc_ops[key] = p;
    *out = p;
    return TNN_OK;
}

bool use_tc(tnn_precision prec, int64_t n3)
{
    return (prec == TNN_FP32_TF32X3 || prec == TNN_FP32_BF16SPLIT) && tube_tc_supported(n3);
}

tnn_status get_tube(tnn_ctx* ctx, tnn_precision prec, int elem, int64_t n3, int inverse, int scaled, cudaStream_t s,
                    TubeOp* t)
{
    t->tc = use_tc(prec, n3);
    t->bf = prec == TNN_FP32_BF16SPLIT;
    if (t->tc) return get_op_tc(ctx, n3, inverse, scaled, t->bf, s, &t->img);
    return get_op(ctx, n3, elem, inverse, scaled, s, &t->op);
}

cudaError_t tube_any(tnn_ctx* ctx, int elem, const void* X, void* Y, const TubeOp& t, int64_t P, int64_t n3,
                     cudaStream_t s)
{
    if (t.tc) return launch_tube_tc((const float*)X, (float*)Y, t.img, P, n3, t.bf, ctx->d_err, s, ctx->opt_tc_polls);
    return elem == 8 ? launch_tube_op<double>((const double*)X, (double*)Y, (const double*)t.op, P, n3, s)
                     : launch_tube_op<float>((const float*)X, (float*)Y, (const float*)t.op, P, n3, s);
}

// After a synchronisation: report (and clear) a tensor-core kernel timeout.
tnn_status check_tc_error(tnn_ctx* ctx)
{
    int h = 0;
    CK(cudaMemcpy(&h, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) {
        CK(cudaMemset(ctx->d_err, 0, sizeof(int)));
        return fail(ctx, TNN_ECUDA, "a tensor-core transform timed out waiting for its copies");
    }
    return TNN_OK;
}

// A tensor argument: the device pointer the kernels use, plus where it came from.
struct Arg {
    const void* user;
    void* dev;
    size_t bytes;
    bool host;
};

}  // namespace

extern "C" {

const char* tnn_status_string(tnn_status s)
{
    switch (s) {
    case TNN_OK: return "TNN_OK";
    case TNN_EINVAL: return "TNN_EINVAL (invalid argument)";
    case TNN_ENOMEM: return "TNN_ENOMEM (allocation failed)";
    case TNN_ECUDA: return "TNN_ECUDA (CUDA call failed)";
    case TNN_ENOCONV: return "TNN_ENOCONV (iteration cap reached)";
    case TNN_ENONFINITE: return "TNN_ENONFINITE (NaN or infinity)";
    case TNN_ENODEV: return "TNN_ENODEV (no sm_103 device)";
    }
    return "unknown tnn_status";
}

const char* tnn_last_error(const tnn_ctx* ctx) { return ctx ? ctx->err.c_str() : ""; }

tnn_status tnn_create(tnn_ctx** out, int device)
{
    if (!out) return TNN_EINVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return TNN_ENODEV;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return TNN_ENODEV;
    if (!(prop.major == 10 && prop.minor == 3)) return TNN_ENODEV;
    tnn_ctx* ctx = new tnn_ctx();
    ctx->device = device;
    if (cudaSetDevice(device) != cudaSuccess || cudaMallocHost(&ctx->h_ctl, sizeof(AdmmCtl)) != cudaSuccess ||
        cudaMalloc(&ctx->d_err, 256) != cudaSuccess || cudaMemset(ctx->d_err, 0, 256) != cudaSuccess) {
        cudaGetLastError();
        if (ctx->h_ctl) cudaFreeHost(ctx->h_ctl);
        if (ctx->d_err) cudaFree(ctx->d_err);
        delete ctx;
        return TNN_ENOMEM;
    }
    if (cudaStreamCreateWithFlags(&ctx->qr_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_tail, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_qr, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();  // no side stream: the QR stays on the call's stream
        if (ctx->ev_tail) cudaEventDestroy(ctx->ev_tail);
        if (ctx->qr_stream) cudaStreamDestroy(ctx->qr_stream);
        ctx->qr_stream = nullptr;
        ctx->ev_tail = ctx->ev_qr = nullptr;
    }
    *out = ctx;
    return TNN_OK;
}

void tnn_destroy(tnn_ctx* ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    if (ctx->ws) cudaFree(ctx->ws);
    for (auto& kv : ctx->ops) cudaFree(kv.second);
    for (auto& kv : ctx->tc_ops) cudaFree(kv.second);
    if (ctx->d_err) cudaFree(ctx->d_err);
    if (ctx->d_sweep_log) cudaFree(ctx->d_sweep_log);
    if (ctx->ev_tail) cudaEventDestroy(ctx->ev_tail);
    if (ctx->ev_qr) cudaEventDestroy(ctx->ev_qr);
    if (ctx->qr_stream) cudaStreamDestroy(ctx->qr_stream);
    for (auto& r : ctx->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : ctx->pool) cudaEventDestroy(e);
    if (ctx->h_ctl) cudaFreeHost(ctx->h_ctl);
    delete ctx;
}

tnn_status tnn_set_option(tnn_ctx* ctx, int option, int64_t value)
{
    if (!ctx) return TNN_EINVAL;
    switch (option) {
    case TNN_OPT_JACOBI_MAX_SWEEPS:
        if (value < 0 || value > 1000) return fail(ctx, TNN_EINVAL, "sweep cap %lld out of range", (long long)value);
        ctx->opt_jacobi_sweeps = (int)value;
        return TNN_OK;
    case TNN_OPT_TC_WAIT_POLLS:
        if (value > (int64_t)1 << 30) return fail(ctx, TNN_EINVAL, "poll limit %lld out of range", (long long)value);
        ctx->opt_tc_polls = value < 0 ? -1 : (int)value;
        return TNN_OK;
    case TNN_OPT_JACOBI_FP64_ANGLES:
        if (value != 0 && value != 1) return fail(ctx, TNN_EINVAL, "FP64-angle flag must be 0 or 1");
        ctx->opt_angle64 = (int)value;
        return TNN_OK;
    case TNN_OPT_ADMM_WARM_START:
        if (value != 0 && value != 1) return fail(ctx, TNN_EINVAL, "warm-start flag must be 0 or 1");
        ctx->opt_warm = (int)value;
        return TNN_OK;
    case TNN_OPT_JACOBI_SMALL_STOP:
        if (value != 0 && value != 1) return fail(ctx, TNN_EINVAL, "small-rotation stop flag must be 0 or 1");
        ctx->opt_small_stop = (int)value;
        return TNN_OK;
    case TNN_OPT_JACOBI_SWEEP_LOG:
        if (value != 0 && value != 1) return fail(ctx, TNN_EINVAL, "sweep-log flag must be 0 or 1");
        ctx->opt_sweep_log = (int)value;
        return TNN_OK;
    default: return fail(ctx, TNN_EINVAL, "unknown option %d", option);
    }
}

tnn_status tnn_reserve(tnn_ctx* ctx, size_t bytes)
{
    if (!ctx) return TNN_EINVAL;
    tnn_status st = set_device(ctx);
    if (st != TNN_OK) return st;
    return ensure_ws(ctx, bytes);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Drivers
// ---------------------------------------------------------------------------
namespace {

// Stage arguments: device pointers pass through, host pointers get a slot
// in the workspace (assigned by the caller's Carve).
struct Stager {
    tnn_ctx* ctx;
    cudaStream_t s;
    std::vector<Arg> outs;
    bool any_host = false;

    tnn_status in(Arg& a, size_t off)
    {
        if (!a.host) return TNN_OK;
        any_host = true;
        a.dev = at(ctx, off);
        if (a.bytes) CK(cudaMemcpyAsync(a.dev, a.user, a.bytes, cudaMemcpyHostToDevice, s));
        return TNN_OK;
    }
    void out(Arg& a, size_t off)
    {
        if (!a.host) return;
        any_host = true;
        a.dev = at(ctx, off);
        outs.push_back(a);
    }
    tnn_status finish()
    {
        for (auto& a : outs)
            if (a.bytes) CK(cudaMemcpyAsync(const_cast<void*>(a.user), a.dev, a.bytes, cudaMemcpyDeviceToHost, s));
        if (any_host) CK(cudaStreamSynchronize(s));
        return TNN_OK;
    }
};

Arg make_arg(const void* p, size_t bytes)
{
    Arg a;
    a.user = p;
    a.bytes = bytes;
    a.host = !is_device_ptr(p);
    a.dev = a.host ? nullptr : const_cast<void*>(p);
    return a;
}

tnn_status jacobi_status(tnn_ctx* ctx, const SliceStats* d_stats, int64_t n3, cudaStream_t s, double* nuc_out)
{
    std::vector<SliceStats> h((size_t)n3);
    CK(cudaMemcpyAsync(h.data(), d_stats, sizeof(SliceStats) * n3, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    double nuc = 0.0;
    bool unconv = false, nonfin = false;
    for (auto& x : h) {
        nuc += x.nuc;
        if (!x.converged) unconv = true;
        if (x.nonfinite) nonfin = true;
    }
    if (nuc_out) *nuc_out = nuc;
    if (nonfin) return fail(ctx, TNN_ENONFINITE, "non-finite singular value met");
    if (unconv) return fail(ctx, TNN_ENOCONV, "a Jacobi SVD reached its sweep cap");
    return TNN_OK;
}

}  // namespace

extern "C" {

tnn_status tnn_workspace_size(tnn_ctx* ctx, int op, tnn_shape sh, tnn_precision prec, size_t* bytes)
{
    if (!ctx || !bytes || !shape_ok(sh) || !prec_ok(prec)) return fail(ctx, TNN_EINVAL, "invalid argument");
    const int elem = elem_of(prec);
    const size_t N = (size_t)sh.n1 * sh.n2 * sh.n3;
    Carve cv;
    JacobiPlan jp;
    switch (op) {
    case TNN_OP_TDCT3: break;
    case TNN_OP_TSVT:
        if (!jacobi_plan(sh.n1, sh.n2, sh.n3, elem, &jp)) return fail(ctx, TNN_EINVAL, "slice too large");
        cv.add(N * elem); cv.add(sizeof(SliceStats) * sh.n3); cv.add(jp.work_bytes);
        break;
    case TNN_OP_TSVD: {
        if (!jacobi_plan_mode(sh.n1, sh.n2, sh.n3, elem, true, &jp)) return fail(ctx, TNN_EINVAL, "slice too large");
        int64_t r = sh.n1 < sh.n2 ? sh.n1 : sh.n2;
        cv.add(N * elem); cv.add((size_t)sh.n1 * r * sh.n3 * elem); cv.add((size_t)sh.n2 * r * sh.n3 * elem);
        cv.add((size_t)r * sh.n3 * elem); cv.add(sizeof(SliceStats) * sh.n3); cv.add(jp.work_bytes);
        break;
    }
    case TNN_OP_TPROD:
        cv.add(N * elem); cv.add(N * elem); cv.add(N * elem);
        break;
    case TNN_OP_COMPLETE:
        if (!jacobi_plan(sh.n1, sh.n2, sh.n3, elem, &jp)) return fail(ctx, TNN_EINVAL, "slice too large");
        cv.add(N * elem); cv.add(N * elem);
        cv.add((size_t)tube_partials_count(sh.n1 * sh.n2, sh.n3) * 4 * sizeof(double));
        cv.add(sizeof(SliceStats) * sh.n3); cv.add(sizeof(AdmmCtl)); cv.add(jp.work_bytes);
        break;
    default: return fail(ctx, TNN_EINVAL, "unknown op %d", op);
    }
    *bytes = cv.total;
    return TNN_OK;
}

tnn_status tdct3(tnn_ctx* ctx, const void* X, tnn_shape sh, int inverse, int scaled, tnn_precision prec, void* Y,
                 void* stream)
{
    if (!ctx) return TNN_EINVAL;
    if (!X || !Y || !shape_ok(sh) || !prec_ok(prec)) return fail(ctx, TNN_EINVAL, "invalid argument");
    tnn_status st = set_device(ctx);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int elem = elem_of(prec);
    const size_t bytes = (size_t)sh.n1 * sh.n2 * sh.n3 * elem;
    Arg ax = make_arg(X, bytes), ay = make_arg(Y, bytes);
    Carve cv;
    size_t ox = ax.host ? cv.add(bytes) : 0, oy = ay.host ? cv.add(bytes) : 0;
    if ((st = ensure_ws(ctx, cv.total))) return st;
    TubeOp op;
    if ((st = get_tube(ctx, prec, elem, sh.n3, inverse ? 1 : 0, scaled ? 1 : 0, s, &op))) return st;
    Stager sg{ctx, s};
    if ((st = sg.in(ax, ox))) return st;
    sg.out(ay, oy);
    {
        TRACE(K_TUBE);
        CK(tube_any(ctx, elem, ax.dev, ay.dev, op, sh.n1 * sh.n2, sh.n3, s));
    }
    ctx->last_stream = s;
    return sg.finish();
}

// TNN_OPT_JACOBI_SWEEP_LOG: the plan's log buffer (sweep_log_floats per
// slice, grown here, outside any stream capture; the launches that use it
// clear it first); none when the option is off.
static tnn_status attach_sweep_log(tnn_ctx* ctx, JacobiPlan& jp)
{
    jp.sweep_log = nullptr;
    if (!ctx->opt_sweep_log) return TNN_OK;
    if (jp.n3 > ctx->sweep_log_cap) {
        if (ctx->d_sweep_log) CK(cudaFree(ctx->d_sweep_log));
        ctx->d_sweep_log = nullptr;
        ctx->sweep_log_cap = 0;
        CK(cudaMalloc(&ctx->d_sweep_log, sizeof(float) * sweep_log_floats * (size_t)jp.n3));
        ctx->sweep_log_cap = jp.n3;
    }
    jp.sweep_log = ctx->d_sweep_log;
    return TNN_OK;
}

tnn_status tsvt_dct(tnn_ctx* ctx, const void* Z, tnn_shape sh, double tau, tnn_precision prec, void* Y,
                    double* tnn_out, void* stream)
{
    if (!ctx) return TNN_EINVAL;
    if (!Z || !Y || !shape_ok(sh) || !prec_ok(prec) || !(tau >= 0.0) || !(tau < 1e300))
        return fail(ctx, TNN_EINVAL, "invalid argument");
    tnn_status st = set_device(ctx);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int elem = elem_of(prec);
    JacobiPlan jp;
    if (!jacobi_plan(sh.n1, sh.n2, sh.n3, elem, &jp)) return fail(ctx, TNN_EINVAL, "slice %lldx%lld too large",
                                                                (long long)sh.n1, (long long)sh.n2);
    jp.angle64 = ctx->opt_angle64;
    jp.small_stop = ctx->opt_small_stop;
    if ((st = attach_sweep_log(ctx, jp))) return st;
    const size_t bytes = (size_t)sh.n1 * sh.n2 * sh.n3 * elem;
    Arg az = make_arg(Z, bytes), ay = make_arg(Y, bytes);
    Carve cv;
    size_t ow = cv.add(bytes), ost = cv.add(sizeof(SliceStats) * sh.n3), ojw = cv.add(jp.work_bytes);
    size_t oz = az.host ? cv.add(bytes) : 0, oy = ay.host ? cv.add(bytes) : 0;
    if ((st = ensure_ws(ctx, cv.total))) return st;
    TubeOp opf, opi;
    if ((st = get_tube(ctx, prec, elem, sh.n3, 0, 0, s, &opf))) return st;
    if ((st = get_tube(ctx, prec, elem, sh.n3, 1, 0, s, &opi))) return st;
    Stager sg{ctx, s};
    if ((st = sg.in(az, oz))) return st;
    sg.out(ay, oy);
    void* W = at(ctx, ow);
    SliceStats* stats = (SliceStats*)at(ctx, ost);
    const int64_t P = sh.n1 * sh.n2;
    {
        TRACE(K_TUBE);
        CK(tube_any(ctx, elem, az.dev, W, opf, P, sh.n3, s));
    }
    {
        TRACE(K_JACOBI_SVT);
        const int sw = ctx->opt_jacobi_sweeps;
        if (jp.sweep_log) CK(cudaMemsetAsync(jp.sweep_log, 0, sizeof(float) * sweep_log_floats * sh.n3, s));
        if (elem == 8) CK(launch_jacobi_svt<double>(jp, (double*)W, tau, nullptr, sw, at(ctx, ojw), stats, s));
        else CK(launch_jacobi_svt<float>(jp, (float*)W, tau, nullptr, sw, at(ctx, ojw), stats, s));
    }
    {
        TRACE(K_TUBE);
        CK(tube_any(ctx, elem, W, ay.dev, opi, P, sh.n3, s));
    }
    ctx->last_sweep_log = jp.sweep_log;
    ctx->last_stats = stats;
    ctx->last_n3 = sh.n3;
    ctx->last_stream = s;
    if ((st = sg.finish())) return st;
    if (tnn_out || sg.any_host) {
        if ((st = check_tc_error(ctx))) return st;
        return jacobi_status(ctx, stats, sh.n3, s, tnn_out);
    }
    return TNN_OK;
}

tnn_status tsvd_dct_forward(tnn_ctx* ctx, const void* X, tnn_shape sh, tnn_precision prec, void* U, void* S,
                            void* V, void* stream)
{
    if (!ctx) return TNN_EINVAL;
    if (!X || !U || !S || !V || !shape_ok(sh) || !prec_ok(prec)) return fail(ctx, TNN_EINVAL, "invalid argument");
    tnn_status st = set_device(ctx);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int elem = elem_of(prec);
    JacobiPlan jp;
    if (!jacobi_plan_mode(sh.n1, sh.n2, sh.n3, elem, true, &jp)) return fail(ctx, TNN_EINVAL, "slice too large");
    const int64_t r = sh.n1 < sh.n2 ? sh.n1 : sh.n2;
    const size_t bx = (size_t)sh.n1 * sh.n2 * sh.n3 * elem;
    const size_t bu = (size_t)sh.n1 * r * sh.n3 * elem, bv = (size_t)sh.n2 * r * sh.n3 * elem;
    const size_t bs = (size_t)r * sh.n3 * elem;
    Arg ax = make_arg(X, bx), au = make_arg(U, bu), as = make_arg(S, bs), av = make_arg(V, bv);
    Carve cv;
    size_t ow = cv.add(bx), ou = cv.add(bu), ov = cv.add(bv), os = cv.add(bs);
    size_t ost = cv.add(sizeof(SliceStats) * sh.n3), ojw = cv.add(jp.work_bytes);
    size_t ohx = ax.host ? cv.add(bx) : 0, ohu = au.host ? cv.add(bu) : 0, ohs = as.host ? cv.add(bs) : 0,
           ohv = av.host ? cv.add(bv) : 0;
    if ((st = ensure_ws(ctx, cv.total))) return st;
    TubeOp opf, opi;
    if ((st = get_tube(ctx, prec, elem, sh.n3, 0, 1, s, &opf))) return st;
    if ((st = get_tube(ctx, prec, elem, sh.n3, 1, 1, s, &opi))) return st;
    Stager sg{ctx, s};
    if ((st = sg.in(ax, ohx))) return st;
    sg.out(au, ohu);
    sg.out(as, ohs);
    sg.out(av, ohv);
    void *W = at(ctx, ow), *Uh = at(ctx, ou), *Vh = at(ctx, ov), *Sh = at(ctx, os);
    SliceStats* stats = (SliceStats*)at(ctx, ost);
    CK(tube_any(ctx, elem, ax.dev, W, opf, sh.n1 * sh.n2, sh.n3, s));
    if (elem == 8) {
        TRACE(K_JACOBI_SVD);
        CK(launch_jacobi_svd<double>(jp, (const double*)W, (double*)Uh, (double*)Sh, (double*)Vh, 0, at(ctx, ojw),
                                     stats, s));
    } else {
        TRACE(K_JACOBI_SVD);
        CK(launch_jacobi_svd<float>(jp, (const float*)W, (float*)Uh, (float*)Sh, (float*)Vh, 0, at(ctx, ojw), stats,
                                    s));
    }
    CK(tube_any(ctx, elem, Uh, au.dev, opi, sh.n1 * r, sh.n3, s));
    CK(tube_any(ctx, elem, Vh, av.dev, opi, sh.n2 * r, sh.n3, s));
    CK(tube_any(ctx, elem, Sh, as.dev, opi, r, sh.n3, s));
    ctx->last_sweep_log = nullptr;
    ctx->last_stats = stats;
    ctx->last_n3 = sh.n3;
    ctx->last_stream = s;
    if ((st = sg.finish())) return st;
    if (sg.any_host) return jacobi_status(ctx, stats, sh.n3, s, nullptr);
    return TNN_OK;
}

tnn_status tsvd_dct_inverse(tnn_ctx* ctx, const void* U, const void* S, const void* V, tnn_shape sh,
                            tnn_precision prec, void* X, void* stream)
{
    if (!ctx) return TNN_EINVAL;
    if (!X || !U || !S || !V || !shape_ok(sh) || !prec_ok(prec)) return fail(ctx, TNN_EINVAL, "invalid argument");
    tnn_status st = set_device(ctx);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int elem = elem_of(prec);
    const int64_t r = sh.n1 < sh.n2 ? sh.n1 : sh.n2;
    const size_t bx = (size_t)sh.n1 * sh.n2 * sh.n3 * elem;
    const size_t bu = (size_t)sh.n1 * r * sh.n3 * elem, bv = (size_t)sh.n2 * r * sh.n3 * elem;
    const size_t bs = (size_t)r * sh.n3 * elem;
    Arg ax = make_arg(X, bx), au = make_arg(U, bu), as = make_arg(S, bs), av = make_arg(V, bv);
    Carve cv;
    size_t ou = cv.add(bu), ov = cv.add(bv), os = cv.add(bs), ot = cv.add(bx);
    size_t ohx = ax.host ? cv.add(bx) : 0, ohu = au.host ? cv.add(bu) : 0, ohs = as.host ? cv.add(bs) : 0,
           ohv = av.host ? cv.add(bv) : 0;
    if ((st = ensure_ws(ctx, cv.total))) return st;
    TubeOp opf, opi;
    if ((st = get_tube(ctx, prec, elem, sh.n3, 0, 1, s, &opf))) return st;
    if ((st = get_tube(ctx, prec, elem, sh.n3, 1, 1, s, &opi))) return st;
    Stager sg{ctx, s};
    if ((st = sg.in(au, ohu))) return st;
    if ((st = sg.in(as, ohs))) return st;
    if ((st = sg.in(av, ohv))) return st;
    sg.out(ax, ohx);
    void *Lu = at(ctx, ou), *Lv = at(ctx, ov), *Ls = at(ctx, os), *Tt = at(ctx, ot);
    CK(tube_any(ctx, elem, au.dev, Lu, opf, sh.n1 * r, sh.n3, s));
    CK(tube_any(ctx, elem, av.dev, Lv, opf, sh.n2 * r, sh.n3, s));
    CK(tube_any(ctx, elem, as.dev, Ls, opf, r, sh.n3, s));
    // L(X)_k = L(U)_k diag(L(S)_k) L(V)_k^T
    TRACE(K_FACEWISE);
    if (elem == 8)
        CK(launch_facewise<double>((const double*)Lu, (const double*)Lv, (double*)Tt, sh.n1, sh.n2, r, sh.n3, 0, 1,
                                   (const double*)Ls, s));
    else
        CK(launch_facewise<float>((const float*)Lu, (const float*)Lv, (float*)Tt, sh.n1, sh.n2, r, sh.n3, 0, 1,
                                  (const float*)Ls, s));
    CK(tube_any(ctx, elem, Tt, ax.dev, opi, sh.n1 * sh.n2, sh.n3, s));
    ctx->last_stream = s;
    return sg.finish();
}

tnn_status tprod_dct(tnn_ctx* ctx, const void* X, const void* Y, int64_t m1, int64_t m2, int64_t m4, int64_t m3,
                     tnn_precision prec, void* Z, void* stream)
{
    if (!ctx) return TNN_EINVAL;
    if (!X || !Y || !Z || m1 <= 0 || m2 <= 0 || m4 <= 0 || m3 <= 0 || !prec_ok(prec))
        return fail(ctx, TNN_EINVAL, "invalid argument");
    tnn_status st = set_device(ctx);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int elem = elem_of(prec);
    const size_t bx = (size_t)m1 * m2 * m3 * elem, by = (size_t)m2 * m4 * m3 * elem, bz = (size_t)m1 * m4 * m3 * elem;
    Arg ax = make_arg(X, bx), ay = make_arg(Y, by), az = make_arg(Z, bz);
    Carve cv;
    size_t olx = cv.add(bx), oly = cv.add(by), olz = cv.add(bz);
    size_t ohx = ax.host ? cv.add(bx) : 0, ohy = ay.host ? cv.add(by) : 0, ohz = az.host ? cv.add(bz) : 0;
    if ((st = ensure_ws(ctx, cv.total))) return st;
    TubeOp opf, opi;
    if ((st = get_tube(ctx, prec, elem, m3, 0, 1, s, &opf))) return st;
    if ((st = get_tube(ctx, prec, elem, m3, 1, 1, s, &opi))) return st;
    Stager sg{ctx, s};
    if ((st = sg.in(ax, ohx))) return st;
    if ((st = sg.in(ay, ohy))) return st;
    sg.out(az, ohz);
    void *Lx = at(ctx, olx), *Ly = at(ctx, oly), *Lz = at(ctx, olz);
    CK(tube_any(ctx, elem, ax.dev, Lx, opf, m1 * m2, m3, s));
    CK(tube_any(ctx, elem, ay.dev, Ly, opf, m2 * m4, m3, s));
    TRACE(K_FACEWISE);
    if (elem == 8)
        CK(launch_facewise<double>((const double*)Lx, (const double*)Ly, (double*)Lz, m1, m4, m2, m3, 0, 0, nullptr, s));
    else
        CK(launch_facewise<float>((const float*)Lx, (const float*)Ly, (float*)Lz, m1, m4, m2, m3, 0, 0, nullptr, s));
    CK(tube_any(ctx, elem, Lz, az.dev, opi, m1 * m4, m3, s));
    ctx->last_stream = s;
    return sg.finish();
}

}  // extern "C"

namespace {

// ADMM driver shared by tnn_complete and tnn_admm_iterate.  X, M device
// pointers already hold the state; B and mask are device pointers.
AdmmJob make_job(const tnn_shape& sh, tnn_precision prec, const tnn_admm_params& prm, const void* B, const void* mask,
                 void* X, void* M, void* W, AdmmCtl* ctl, double* partials, SliceStats* stats, void* jwork,
                 const JacobiPlan& jp)
{
    AdmmJob j;
    j.sh = sh;
    j.prec = prec;
    j.elem = elem_of(prec);
    j.prm = prm;
    j.B = B;
    j.mask = (const uint8_t*)mask;
    j.X = X;
    j.M = M;
    j.W = W;
    j.ctl = ctl;
    j.partials = partials;
    j.stats = stats;
    j.jwork = jwork;
    j.jp = jp;
    return j;
}

}  // namespace

namespace tnn {

// The job's transform operators (built once per context and n3).
tnn_status admm_prepare_job(tnn_ctx* ctx, AdmmJob& j, cudaStream_t s)
{
    tnn_status st;
    if ((st = get_tube(ctx, j.prec, j.elem, j.sh.n3, 0, 0, s, &j.opf))) return st;
    return get_tube(ctx, j.prec, j.elem, j.sh.n3, 1, 0, s, &j.opi);
}

// Queue `iters` iterations of Algorithm 1 for one job on stream s (every
// kernel reads beta and `done` from the job's device control block).
tnn_status admm_enqueue_iters(tnn_ctx* ctx, const AdmmJob& j, int iters, cudaStream_t s)
{
    const int64_t P = j.sh.n1 * j.sh.n2, n3 = j.sh.n3;
    const int sweeps = j.prm.jacobi_max_sweeps;
    const TubeOp& opf = j.opf;
    const TubeOp& opi = j.opi;
    for (int q = 0; q < iters; ++q) {
        int nblk = 0;
        if (j.elem == 8) {
            { TRACE(K_TUBE_FWD_ADMM);
              CK(launch_tube_fwd_admm_op<double>((const double*)j.X, (const double*)j.M, (double*)j.W,
                                                 (const double*)opf.op, P, n3, j.ctl, s)); }
            { TRACE(K_JACOBI_SVT);
              if (j.jp.sweep_log)
                  CK(cudaMemsetAsync(j.jp.sweep_log, 0, sizeof(float) * sweep_log_floats * n3, s));
              CK(launch_jacobi_svt<double>(j.jp, (double*)j.W, 0.0, j.ctl, sweeps, j.jwork, j.stats, s)); }
            { TRACE(K_TUBE_INV_ADMM);
              CK(launch_tube_inv_admm_op<double>((const double*)j.W, (double*)j.X, (double*)j.M, (const double*)j.B,
                                                 j.mask, (const double*)opi.op, P, n3, j.ctl, j.partials, &nblk, s)); }
        } else {
            { TRACE(K_TUBE_FWD_ADMM);
              if (opf.tc)
                  CK(launch_tube_tc_fwd_admm((const float*)j.X, (const float*)j.M, (float*)j.W, opf.img, P, n3, opf.bf,
                                             j.ctl, ctx->d_err, s, ctx->opt_tc_polls));
              else
                  CK(launch_tube_fwd_admm_op<float>((const float*)j.X, (const float*)j.M, (float*)j.W,
                                                    (const float*)opf.op, P, n3, j.ctl, s)); }
            // warm start: the slices times the previous iteration's right
            // singular vectors before the sweeps, the new vectors after them
            const bool warm = j.warm != nullptr;
            float* Q = (float*)j.warm;
            int* wflag = warm ? (int*)((char*)j.warm + ((size_t)n3 * j.jp.n * j.jp.n * 4 + 255) / 256 * 256) : nullptr;
            if (warm) {
                TRACE(K_WARM);
                if (j.qs) CK(cudaStreamWaitEvent(s, j.ev_qr, 0));  // the previous iteration's QR
                CK(launch_warm_gemm<float>(j.jp, (const float*)j.W, Q, wflag, (float*)j.wscr, j.ctl, s));
            }
            // with the offloaded tail the Jacobi kernel leaves its columns in
            // the scratch, the tail kernel writes the recovered vectors over
            // Q (consumed above) and the QR turns them into the next Q in place
            const bool tail = warm && j.tinfo != nullptr;
            { TRACE(K_JACOBI_SVT);
              if (j.jp.sweep_log)
                  CK(cudaMemsetAsync(j.jp.sweep_log, 0, sizeof(float) * sweep_log_floats * n3, s));
              WarmPtrs wp{j.wscr, wflag, j.wscr, j.wrec};
              if (tail) { wp.tail_s = j.wscr; wp.tail_info = j.tinfo; }
              CK(launch_jacobi_svt<float>(j.jp, (float*)j.W, 0.0, j.ctl, sweeps, j.jwork, j.stats, s,
                                          warm ? &wp : nullptr)); }
            if (tail) {
                TRACE(K_SVT_TAIL);
                CK(launch_warm_tail<float>(j.jp, (float*)j.W, (const float*)j.wscr, j.tinfo, Q, j.wrec, j.ctl, s));
            }
            if (warm && tail && j.qs) {
                // on the side stream, after the tail; it checks no stop flag (the
                // tail marks the slices it wrote, and the finalize that may set
                // the flag runs alongside)
                CK(cudaEventRecord(j.ev_tail, s));
                CK(cudaStreamWaitEvent(j.qs, j.ev_tail, 0));
                {
                    Trace tq(ctx, K_WARM, j.qs);
                    CK(launch_warm_qr<float>(j.jp, Q, (size_t)j.jp.n * j.jp.n, j.wrec, Q, wflag, nullptr, j.qs));
                }
                CK(cudaEventRecord(j.ev_qr, j.qs));
            } else if (warm) {
                TRACE(K_WARM);
                const size_t wstride = (size_t)j.jp.ldA * j.jp.nb * j.jp.K;
                CK(launch_warm_qr<float>(j.jp, tail ? Q : (const float*)j.wscr, tail ? (size_t)j.jp.n * j.jp.n : wstride,
                                         j.wrec, Q, wflag, j.ctl, s));
            }
            { TRACE(K_TUBE_INV_ADMM);
              if (opi.tc)
                  CK(launch_tube_tc_inv_admm((const float*)j.W, (float*)j.X, (float*)j.M, (const float*)j.B, j.mask,
                                             opi.img, P, n3, opi.bf, j.ctl, j.partials, &nblk, ctx->d_err, s,
                                             ctx->opt_tc_polls));
              else
                  CK(launch_tube_inv_admm_op<float>((const float*)j.W, (float*)j.X, (float*)j.M, (const float*)j.B,
                                                    j.mask, (const float*)opi.op, P, n3, j.ctl, j.partials, &nblk, s)); }
        }
        { TRACE(K_FINALIZE); CK(launch_admm_finalize(j.ctl, j.partials, nblk, j.stats, n3, s)); }
    }
    if (j.qs) CK(cudaStreamWaitEvent(s, j.ev_qr, 0));  // the last QR before the call's stream goes on
    return TNN_OK;
}

}  // namespace tnn

namespace {

tnn_status admm_run(tnn_ctx* ctx, AdmmJob& j, double beta0, int max_iter, cudaStream_t s, AdmmCtl* out)
{
    tnn_status st;
    if ((st = admm_prepare_job(ctx, j, s))) return st;
    {
        TRACE(K_CTL_INIT);
        CK(launch_ctl_init(j.ctl, beta0, j.prm.rho, j.prm.beta_max, j.prm.tol, max_iter, s));
    }
    int queued = 0, chunk = 1;
    for (;;) {
        const int n = chunk < max_iter - queued ? chunk : max_iter - queued;
        if ((st = admm_enqueue_iters(ctx, j, n, s))) return st;
        queued += n;
        CK(cudaMemcpyAsync(ctx->h_ctl, j.ctl, sizeof(AdmmCtl), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (ctx->h_ctl->done || queued >= max_iter) break;
        if (chunk < 16) chunk *= 2;
    }
    if ((st = check_tc_error(ctx))) return st;
    *out = *ctx->h_ctl;
    ctx->last_sweep_log = j.jp.sweep_log;
    ctx->last_stats = j.stats;
    ctx->last_n3 = j.sh.n3;
    ctx->last_stream = s;
    return TNN_OK;
}

tnn_status check_params(tnn_ctx* ctx, const tnn_admm_params* p)
{
    if (!p) return fail(ctx, TNN_EINVAL, "params is NULL");
    if (!(p->beta0 > 0.0) || !(p->rho > 0.0) || !(p->beta_max > 0.0) || p->tol != p->tol || p->max_iter < 0 ||
        p->jacobi_max_sweeps < 0)
        return fail(ctx, TNN_EINVAL, "invalid ADMM parameters");
    return TNN_OK;
}

void fill_report(tnn_admm_report* rep, const AdmmCtl& c)
{
    if (!rep) return;
    rep->iters = c.iter;
    rep->converged = c.converged;
    rep->rel_change = c.rel_change;
    rep->primal_res = c.primal_res;
    rep->beta_final = c.beta;
    rep->jacobi_sweeps_max = c.sweeps_max;
    rep->jacobi_unconverged = c.unconverged;
}

}  // namespace

extern "C" {

tnn_status tnn_complete(tnn_ctx* ctx, const void* B, const uint8_t* mask, tnn_shape sh,
                        const tnn_admm_params* params, tnn_precision prec, void* X_out, tnn_admm_report* rep,
                        void* stream)
{
    if (!ctx) return TNN_EINVAL;
    if (!B || !mask || !X_out || !shape_ok(sh) || !prec_ok(prec)) return fail(ctx, TNN_EINVAL, "invalid argument");
    tnn_status st = check_params(ctx, params);
    if (st) return st;
    if ((st = set_device(ctx))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int elem = elem_of(prec);
    JacobiPlan jp;
    if (!jacobi_plan(sh.n1, sh.n2, sh.n3, elem, &jp)) return fail(ctx, TNN_EINVAL, "slice too large");
    jp.angle64 = ctx->opt_angle64;
    jp.small_stop = ctx->opt_small_stop;
    if ((st = attach_sweep_log(ctx, jp))) return st;
    const size_t N = (size_t)sh.n1 * sh.n2 * sh.n3, bytes = N * elem;
    Arg ab = make_arg(B, bytes), am = make_arg(mask, N), ax = make_arg(X_out, bytes);
    const int nparts = tube_partials_count(sh.n1 * sh.n2, sh.n3);
    Carve cv;
    size_t oM = cv.add(bytes), oW = cv.add(bytes), oP = cv.add((size_t)nparts * 4 * sizeof(double));
    size_t oS = cv.add(sizeof(SliceStats) * sh.n3), oC = cv.add(sizeof(AdmmCtl)), oJ = cv.add(jp.work_bytes);
    size_t ohb = ab.host ? cv.add(bytes) : 0, ohm = am.host ? cv.add(N) : 0, ohx = ax.host ? cv.add(bytes) : 0;
    // warm start across the run's iterations: state, scratch and flags
    const bool warm = ctx->opt_warm && elem == 4 && warm_supported(jp);
    const size_t wstate = warm ? warm_state_bytes(sh.n3, jp.n, elem) : 0;
    const size_t wscr = warm ? (size_t)sh.n3 * jp.ldA * jp.nb * jp.K * elem : 0;
    size_t oWs = warm ? cv.add(wstate) : 0, oWc = warm ? cv.add(wscr) : 0;
    size_t oWr = warm ? cv.add(sizeof(int) * sh.n3) : 0;
    const bool tail = warm && tail_supported(jp);
    size_t oWt = tail ? cv.add(sizeof(float) * sh.n3 * tail_info_stride(jp.nb * jp.K)) : 0;
    if ((st = ensure_ws(ctx, cv.total))) return st;
    Stager sg{ctx, s};
    if ((st = sg.in(ab, ohb))) return st;
    if ((st = sg.in(am, ohm))) return st;
    sg.out(ax, ohx);
    void* X = ax.dev;
    void* M = at(ctx, oM);
    TRACE(K_ADMM_INIT);
    if (elem == 8) CK(launch_admm_init<double>((const double*)ab.dev, (const uint8_t*)am.dev, (double*)X, (double*)M,
                                               (int64_t)N, s));
    else CK(launch_admm_init<float>((const float*)ab.dev, (const uint8_t*)am.dev, (float*)X, (float*)M, (int64_t)N, s));
    AdmmCtl res;
    AdmmJob job = make_job(sh, prec, *params, ab.dev, am.dev, X, M, at(ctx, oW), (AdmmCtl*)at(ctx, oC),
                           (double*)at(ctx, oP), (SliceStats*)at(ctx, oS), at(ctx, oJ), jp);
    if (warm) {
        CK(cudaMemsetAsync(at(ctx, oWs), 0, wstate, s));
        CK(cudaMemsetAsync(at(ctx, oWr), 0, sizeof(int) * sh.n3, s));
        job.warm = at(ctx, oWs);
        job.wscr = at(ctx, oWc);
        job.wrec = (int*)at(ctx, oWr);
        if (tail) job.tinfo = (float*)at(ctx, oWt);
        if (tail && ctx->qr_stream) {
            job.qs = ctx->qr_stream;
            job.ev_tail = ctx->ev_tail;
            job.ev_qr = ctx->ev_qr;
        }
    }
    st = admm_run(ctx, job, params->beta0, params->max_iter, s, &res);
    if (st) return st;
    if ((st = sg.finish())) return st;
    fill_report(rep, res);
    if (res.nonfinite) return fail(ctx, TNN_ENONFINITE, "non-finite value met in iteration %d", res.iter);
    if (!res.converged) return fail(ctx, TNN_ENOCONV, "max_iter reached after %d iterations", res.iter);
    return TNN_OK;
}

tnn_status tnn_admm_iterate(tnn_ctx* ctx, const void* B, const uint8_t* mask, tnn_shape sh,
                            const tnn_admm_params* params, tnn_precision prec, void* X, void* M, double* beta,
                            int32_t iters, void* warm_state, tnn_admm_report* rep, void* stream)
{
    if (!ctx) return TNN_EINVAL;
    if (!B || !mask || !X || !M || !beta || !(*beta > 0.0) || iters < 0 || !shape_ok(sh) || !prec_ok(prec))
        return fail(ctx, TNN_EINVAL, "invalid argument");
    tnn_status st = check_params(ctx, params);
    if (st) return st;
    if ((st = set_device(ctx))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int elem = elem_of(prec);
    JacobiPlan jp;
    if (!jacobi_plan(sh.n1, sh.n2, sh.n3, elem, &jp)) return fail(ctx, TNN_EINVAL, "slice too large");
    jp.angle64 = ctx->opt_angle64;
    jp.small_stop = ctx->opt_small_stop;
    if ((st = attach_sweep_log(ctx, jp))) return st;
    const size_t N = (size_t)sh.n1 * sh.n2 * sh.n3, bytes = N * elem;
    Arg ab = make_arg(B, bytes), am = make_arg(mask, N), ax = make_arg(X, bytes), amm = make_arg(M, bytes);
    const int nparts = tube_partials_count(sh.n1 * sh.n2, sh.n3);
    Carve cv;
    size_t oW = cv.add(bytes), oP = cv.add((size_t)nparts * 4 * sizeof(double));
    size_t oS = cv.add(sizeof(SliceStats) * sh.n3), oC = cv.add(sizeof(AdmmCtl)), oJ = cv.add(jp.work_bytes);
    size_t ohb = ab.host ? cv.add(bytes) : 0, ohm = am.host ? cv.add(N) : 0;
    size_t ohx = ax.host ? cv.add(bytes) : 0, ohmm = amm.host ? cv.add(bytes) : 0;
    // warm start from the caller's state (device memory), when this precision
    // and slice size use it
    const bool warm = warm_state && elem == 4 && warm_supported(jp);
    if (warm && !is_device_ptr(warm_state)) return fail(ctx, TNN_EINVAL, "warm state must be device memory");
    const size_t wscr = warm ? (size_t)sh.n3 * jp.ldA * jp.nb * jp.K * elem : 0;
    size_t oWc = warm ? cv.add(wscr) : 0, oWr = warm ? cv.add(sizeof(int) * sh.n3) : 0;
    const bool tail = warm && tail_supported(jp);
    size_t oWt = tail ? cv.add(sizeof(float) * sh.n3 * tail_info_stride(jp.nb * jp.K)) : 0;
    if ((st = ensure_ws(ctx, cv.total))) return st;
    Stager sg{ctx, s};
    if ((st = sg.in(ab, ohb))) return st;
    if ((st = sg.in(am, ohm))) return st;
    if ((st = sg.in(ax, ohx))) return st;
    if ((st = sg.in(amm, ohmm))) return st;
    sg.out(ax, ohx);
    sg.out(amm, ohmm);
    int max_iter = params->max_iter < iters ? params->max_iter : iters;
    AdmmCtl res;
    AdmmJob job = make_job(sh, prec, *params, ab.dev, am.dev, ax.dev, amm.dev, at(ctx, oW), (AdmmCtl*)at(ctx, oC),
                           (double*)at(ctx, oP), (SliceStats*)at(ctx, oS), at(ctx, oJ), jp);
    if (warm) {
        CK(cudaMemsetAsync(at(ctx, oWr), 0, sizeof(int) * sh.n3, s));
        job.warm = warm_state;
        job.wscr = at(ctx, oWc);
        job.wrec = (int*)at(ctx, oWr);
        if (tail) job.tinfo = (float*)at(ctx, oWt);
        if (tail && ctx->qr_stream) {
            job.qs = ctx->qr_stream;
            job.ev_tail = ctx->ev_tail;
            job.ev_qr = ctx->ev_qr;
        }
    }
    st = admm_run(ctx, job, *beta, max_iter, s, &res);
    if (st) return st;
    if ((st = sg.finish())) return st;
    *beta = res.beta;
    fill_report(rep, res);
    if (res.nonfinite) return fail(ctx, TNN_ENONFINITE, "non-finite value met in iteration %d", res.iter);
    return TNN_OK;
}

tnn_status tnn_admm_warm_size(tnn_shape sh, tnn_precision prec, size_t* bytes)
{
    if (!bytes || !shape_ok(sh) || !prec_ok(prec)) return TNN_EINVAL;
    *bytes = 0;
    const int elem = elem_of(prec);
    JacobiPlan jp;
    if (!jacobi_plan(sh.n1, sh.n2, sh.n3, elem, &jp)) return TNN_EINVAL;
    if (elem == 4 && warm_supported(jp)) *bytes = warm_state_bytes(sh.n3, jp.n, elem);
    return TNN_OK;
}

// The DFT comparison path and its like-for-like DCT counterpart: transform,
// plain per-slice Jacobi SVT, inverse transform.
static tnn_status tsvt_plain_run(tnn_ctx* ctx, const void* Z, tnn_shape sh, double tau, tnn_precision prec, void* Y,
                                 double* tnn_out, void* stream, bool dft)
{
    if (!ctx) return TNN_EINVAL;
    if (!Z || !Y || !shape_ok(sh) || !prec_ok(prec) || !(tau >= 0.0) || !(tau < 1e300))
        return fail(ctx, TNN_EINVAL, "invalid argument");
    if (sh.n1 > 512 || sh.n2 > 512 || sh.n3 > (1 << 20)) return fail(ctx, TNN_EINVAL, "slice too large");
    tnn_status st = set_device(ctx);
    if (st) return st;
    if (!is_device_ptr(Z) || !is_device_ptr(Y)) return fail(ctx, TNN_EINVAL, "device pointers required");
    cudaStream_t s = (cudaStream_t)stream;
    const int elem = elem_of(prec);
    const int64_t P = sh.n1 * sh.n2, n3 = sh.n3, nh = n3 / 2 + 1;
    const int64_t planes = dft ? 2 * nh : n3;
    const int64_t nsl = dft ? nh : n3;
    bool smem_copy = true;
    const size_t wbytes = jacobi_plain_work_bytes(sh.n1, sh.n2, nsl, elem, dft, &smem_copy);
    Carve cv;
    const size_t oW = cv.add((size_t)planes * P * elem), oS = cv.add(sizeof(SliceStats) * nsl);
    const size_t oF = dft ? cv.add((size_t)n3 * 2 * nh * elem) : 0, oI = dft ? cv.add((size_t)n3 * 2 * nh * elem) : 0;
    const size_t oJ = cv.add(wbytes);
    if ((st = ensure_ws(ctx, cv.total))) return st;
    void* W = at(ctx, oW);
    SliceStats* stats = (SliceStats*)at(ctx, oS);
    if (dft) {
        {
            TRACE(K_DFT);
            if (elem == 8) {
                CK(launch_build_dft_ops<double>((double*)at(ctx, oF), (double*)at(ctx, oI), (int)n3, s));
                CK(launch_tube_rect<double>((const double*)Z, (double*)W, (const double*)at(ctx, oF), P, (int)n3,
                                            (int)(2 * nh), s));
            } else {
                CK(launch_build_dft_ops<float>((float*)at(ctx, oF), (float*)at(ctx, oI), (int)n3, s));
                CK(launch_tube_rect<float>((const float*)Z, (float*)W, (const float*)at(ctx, oF), P, (int)n3,
                                           (int)(2 * nh), s));
            }
        }
        {
            TRACE(K_JACOBI_PLAIN);
            if (elem == 8)
                CK(launch_jacobi_plain<double>((double*)W, 2 * P, P, (int)nh, (int)sh.n1, (int)sh.n2, tau, true,
                                               (double*)at(ctx, oJ), smem_copy, stats, s));
            else
                CK(launch_jacobi_plain<float>((float*)W, 2 * P, P, (int)nh, (int)sh.n1, (int)sh.n2, tau, true,
                                              (float*)at(ctx, oJ), smem_copy, stats, s));
        }
        {
            TRACE(K_DFT);
            if (elem == 8)
                CK(launch_tube_rect<double>((const double*)W, (double*)Y, (const double*)at(ctx, oI), P, (int)(2 * nh),
                                            (int)n3, s));
            else
                CK(launch_tube_rect<float>((const float*)W, (float*)Y, (const float*)at(ctx, oI), P, (int)(2 * nh),
                                           (int)n3, s));
        }
    } else {
        const void *opf = nullptr, *opi = nullptr;
        if ((st = get_op(ctx, n3, elem, 0, 0, s, &opf))) return st;
        if ((st = get_op(ctx, n3, elem, 1, 0, s, &opi))) return st;
        {
            TRACE(K_TUBE);
            CK(elem == 8 ? launch_tube_op<double>((const double*)Z, (double*)W, (const double*)opf, P, n3, s)
                         : launch_tube_op<float>((const float*)Z, (float*)W, (const float*)opf, P, n3, s));
        }
        {
            TRACE(K_JACOBI_PLAIN);
            if (elem == 8)
                CK(launch_jacobi_plain<double>((double*)W, P, 0, (int)n3, (int)sh.n1, (int)sh.n2, tau, false,
                                               (double*)at(ctx, oJ), smem_copy, stats, s));
            else
                CK(launch_jacobi_plain<float>((float*)W, P, 0, (int)n3, (int)sh.n1, (int)sh.n2, tau, false,
                                              (float*)at(ctx, oJ), smem_copy, stats, s));
        }
        {
            TRACE(K_TUBE);
            CK(elem == 8 ? launch_tube_op<double>((const double*)W, (double*)Y, (const double*)opi, P, n3, s)
                         : launch_tube_op<float>((const float*)W, (float*)Y, (const float*)opi, P, n3, s));
        }
    }
    ctx->last_sweep_log = nullptr;
    ctx->last_stats = stats;
    ctx->last_n3 = nsl;
    ctx->last_stream = s;
    if (!tnn_out) return TNN_OK;
    std::vector<SliceStats> h((size_t)nsl);
    CK(cudaMemcpyAsync(h.data(), stats, sizeof(SliceStats) * nsl, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    double nuc = 0.0;
    bool unconv = false, nonfin = false;
    for (int64_t k = 0; k < nsl; ++k) {
        // TNN-F sums all n3 DFT slices: slice k and its conjugate n3 - k count twice
        const double w = !dft ? 1.0 : ((k == 0 || 2 * k == n3) ? 1.0 : 2.0);
        nuc += w * h[k].nuc;
        unconv |= !h[k].converged;
        nonfin |= h[k].nonfinite != 0;
    }
    *tnn_out = dft ? nuc / (double)n3 : nuc;
    if (nonfin) return fail(ctx, TNN_ENONFINITE, "non-finite singular value met");
    if (unconv) return fail(ctx, TNN_ENOCONV, "a Jacobi SVD reached its sweep cap");
    return TNN_OK;
}

tnn_status tsvt_dft(tnn_ctx* ctx, const void* Z, tnn_shape sh, double tau, tnn_precision prec, void* Y,
                    double* tnn_out, void* stream)
{
    return tsvt_plain_run(ctx, Z, sh, tau, prec, Y, tnn_out, stream, true);
}

tnn_status tsvt_dct_plain(tnn_ctx* ctx, const void* Z, tnn_shape sh, double tau, tnn_precision prec, void* Y,
                          double* tnn_out, void* stream)
{
    return tsvt_plain_run(ctx, Z, sh, tau, prec, Y, tnn_out, stream, false);
}

tnn_status tnn_last_jacobi_stats(tnn_ctx* ctx, int64_t out[6])
{
    if (!ctx || !out) return TNN_EINVAL;
    for (int i = 0; i < 6; ++i) out[i] = 0;
    if (!ctx->last_stats) return TNN_OK;
    tnn_status st = set_device(ctx);
    if (st) return st;
    std::vector<SliceStats> h((size_t)ctx->last_n3);
    CK(cudaStreamSynchronize(ctx->last_stream));
    CK(cudaMemcpy(h.data(), ctx->last_stats, sizeof(SliceStats) * ctx->last_n3, cudaMemcpyDeviceToHost));
    out[0] = ctx->last_n3;
    for (auto& x : h) {
        out[1] += x.pairs;
        out[2] += x.rotations;
        if (x.sweeps > out[3]) out[3] = x.sweeps;
        out[4] += x.converged ? 0 : 1;
        out[5] += x.kept;
    }
    return TNN_OK;
}

tnn_status tnn_last_sweep_log(tnn_ctx* ctx, int64_t n, float* out)
{
    if (!ctx || n < 0 || (n > 0 && !out)) return TNN_EINVAL;
    if (!ctx->last_stats || !ctx->last_sweep_log) return fail(ctx, TNN_EINVAL, "no sweep log was recorded");
    tnn_status st = set_device(ctx);
    if (st) return st;
    const int64_t cnt = n < ctx->last_n3 ? n : ctx->last_n3;
    CK(cudaStreamSynchronize(ctx->last_stream));
    if (cnt > 0)
        CK(cudaMemcpy(out, ctx->last_sweep_log, sizeof(float) * sweep_log_floats * cnt, cudaMemcpyDeviceToHost));
    return TNN_OK;
}

tnn_status tnn_last_slice_stats(tnn_ctx* ctx, int64_t n, int32_t* sweeps, int32_t* kept, int64_t* rotations)
{
    if (!ctx || n < 0) return TNN_EINVAL;
    if (!ctx->last_stats || n == 0) return TNN_OK;
    tnn_status st = set_device(ctx);
    if (st) return st;
    std::vector<SliceStats> h((size_t)ctx->last_n3);
    CK(cudaStreamSynchronize(ctx->last_stream));
    CK(cudaMemcpy(h.data(), ctx->last_stats, sizeof(SliceStats) * ctx->last_n3, cudaMemcpyDeviceToHost));
    const int64_t cnt = n < ctx->last_n3 ? n : ctx->last_n3;
    for (int64_t k = 0; k < cnt; ++k) {
        if (sweeps) sweeps[k] = h[(size_t)k].sweeps;
        if (kept) kept[k] = h[(size_t)k].kept;
        if (rotations) rotations[k] = h[(size_t)k].rotations;
    }
    return TNN_OK;
}

}  // extern "C"

namespace tnn {
tnn_status ctx_fail(tnn_ctx* ctx, tnn_status s, const char* msg) { return fail(ctx, s, "%s", msg); }
tnn_status ctx_check_tc(tnn_ctx* ctx) { return check_tc_error(ctx); }
int ctx_device(const tnn_ctx* ctx) { return ctx->device; }
bool is_device_pointer(const void* p) { return is_device_ptr(p); }
}  // namespace tnn

extern "C" {

tnn_status tnn_profile(tnn_ctx* ctx, int enable)
{
    if (!ctx) return TNN_EINVAL;
    ctx->prof = enable != 0;
    return TNN_OK;
}

tnn_status tnn_profile_read(tnn_ctx* ctx, double ms[TNN_NKERNELS], int64_t launches[TNN_NKERNELS])
{
    if (!ctx || !ms || !launches) return TNN_EINVAL;
    tnn_status st = set_device(ctx);
    if (st) return st;
    for (int i = 0; i < TNN_NKERNELS; ++i) { ms[i] = 0.0; launches[i] = 0; }
    for (auto& r : ctx->recs) {
        CK(cudaEventSynchronize(r.b));
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, r.a, r.b));
        if (r.kind >= 0 && r.kind < TNN_NKERNELS) {
            ms[r.kind] += t;
            launches[r.kind] += 1;
        }
        ctx->pool.push_back(r.a);
        ctx->pool.push_back(r.b);
    }
    ctx->recs.clear();
    return TNN_OK;
}

}  // extern "C"
