// Shape planning for the Jacobi kernels (host only).  The variants compiled
// (L lanes per block pair, R rows per lane) are listed here and in the
// jacobi_sv*_*.cu dispatch files.
#include <stdio.h>
#include <stdlib.h>

#include "jacobi_cluster.cuh"
#include "jacobi_launch.cuh"

namespace tnn {

namespace {

struct Variant {
    int L, R, K;  // K = 0: the default block width for (elem, R)
};

// Smallest variant whose L * R rows cover m (the first listed wins), unless
// TNN_JACOBI_VARIANT="L,R[,K]" names a compiled variant that covers m (a
// tuning override for benchmarking the variants against each other).
bool pick_variant(int m, int elem, bool withv, Variant* out)
{
    static const Variant f32_svt[] = {{16, 4, 0}, {16, 8, 0}, {16, 12, 0}, {32, 8, 0}, {32, 12, 0},
                                       {32, 16, 0}, {32, 4, 0}, {32, 6, 0}, {16, 12, 2}, {32, 6, 8}};
    static const Variant f64_svt[] = {{16, 2, 0}, {16, 4, 0}, {16, 6, 0}, {32, 4, 0}, {32, 6, 0}, {32, 8, 0},
                                       {32, 16, 0}};
    static const Variant f32_svd[] = {{32, 2, 0}, {32, 4, 0}, {32, 6, 0}, {32, 8, 0}, {32, 12, 0}, {32, 16, 0}};
    static const Variant f64_svd[] = {{32, 1, 0}, {32, 2, 0}, {32, 4, 0}, {32, 6, 0}, {32, 8, 0}};
    const Variant* t;
    int cnt;
    if (elem == 4) {
        t = withv ? f32_svd : f32_svt;
        cnt = withv ? 6 : 10;
    } else {
        t = withv ? f64_svd : f64_svt;
        cnt = withv ? 5 : 7;
    }
    if (const char* env = getenv("TNN_JACOBI_VARIANT")) {
        int L = 0, R = 0, K = 0;
        if (sscanf(env, "%d,%d,%d", &L, &R, &K) >= 2)
            for (int i = 0; i < cnt; ++i)
                if (t[i].L == L && t[i].R == R && t[i].K == K && L * R >= m) {
                    *out = t[i];
                    return true;
                }
    }
    for (int i = 0; i < cnt; ++i)
        if (t[i].L * t[i].R >= m) {
            *out = t[i];
            return true;
        }
    return false;
}

}  // namespace

static bool plan_with(int64_t n1, int64_t n2, int64_t n3, int elem, bool withv, Variant v, bool cluster,
                      JacobiPlan* p);

bool jacobi_plan_mode(int64_t n1, int64_t n2, int64_t n3, int elem, bool withv, JacobiPlan* p, bool cluster)
{
    if (n1 <= 0 || n2 <= 0 || n3 <= 0) return false;
    const int64_t m = n1 >= n2 ? n1 : n2;
    if (m > 512) return false;
    Variant v;
    if (!pick_variant((int)m, elem, withv, &v)) return false;
    return plan_with(n1, n2, n3, elem, withv, v, cluster, p);
}

int jacobi_svt_variants(int elem, int* L, int* R, int* K, int max)
{
    static const Variant f32[] = {{16, 4, 4}, {16, 8, 4}, {16, 12, 4}, {32, 8, 4}, {32, 12, 4},
                                  {32, 16, 4}, {32, 4, 4}, {32, 6, 4}, {16, 12, 2}, {32, 6, 8}};
    static const Variant f64[] = {{16, 2, 4}, {16, 4, 4}, {16, 6, 4}, {32, 4, 4}, {32, 6, 4}, {32, 8, 4},
                                  {32, 16, 2}};
    const Variant* t = elem == 4 ? f32 : f64;
    const int cnt = elem == 4 ? 10 : 7;
    for (int i = 0; i < cnt && i < max; ++i) {
        L[i] = t[i].L;
        R[i] = t[i].R;
        K[i] = t[i].K;
    }
    return cnt;
}

bool jacobi_plan_variant(int64_t n1, int64_t n2, int64_t n3, int elem, int L, int R, int K, JacobiPlan* p)
{
    if (n1 <= 0 || n2 <= 0 || n3 <= 0) return false;
    const int64_t m = n1 >= n2 ? n1 : n2;
    if (m > (int64_t)L * R) return false;
    Variant v{L, R, K};
    return plan_with(n1, n2, n3, elem, false, v, false, p);
}

bool jacobi_cluster_variant_f32(int L, int R, int K);
bool jacobi_cluster_variant_f64(int L, int R, int K);

static bool plan_with(int64_t n1, int64_t n2, int64_t n3, int elem, bool withv, Variant v, bool cluster,
                      JacobiPlan* p)
{
    const int64_t m = n1 >= n2 ? n1 : n2;
    const int64_t n = n1 >= n2 ? n2 : n1;
    const int K = v.K ? v.K : jac::pick_K(elem, v.R, withv);
    p->n1 = n1; p->n2 = n2; p->n3 = n3;
    p->m = (int)m; p->n = (int)n; p->tr = n1 < n2 ? 1 : 0;
    p->K = K; p->RA = v.R; p->L = v.L;
    p->nb = 2 * (int)((n + 2 * K - 1) / (2 * K));
    p->ldA = v.L * v.R + (elem == 4 ? 2 : 1);
    p->elem = elem;
    const int npad = p->nb * K;
    const int gpw = 32 / v.L;
    int Wguess = (p->nb / 2 + gpw - 1) / gpw;
    if (Wguess > 32) Wguess = 32;
    size_t wsz = (size_t)p->ldA * npad * elem;
    size_t big = (withv ? 2 : 1) * ((wsz + 255) & ~(size_t)255);
    size_t small = jac::smem_small_bytes(npad, Wguess, elem);
    p->in_smem = (big + small) <= 226 * 1024 ? 1 : 0;  // static shared memory needs a little room
    p->smem_bytes = p->in_smem ? big + small : small;
    p->work_bytes = p->in_smem ? 0 : (size_t)n3 * (withv ? 2 : 1) * wsz;
    p->W = Wguess;
    p->cluster = 0;
    // A slice too large for one CTA's shared memory is spread over a cluster
    // (the smallest of 2, 4, 8 CTAs that holds it).  TNN_JACOBI_CLUSTER=C
    // spreads every slice over C CTAs where the variant allows (a tuning
    // override for benchmarking).
    const bool has = !withv && (elem == 4 ? jacobi_cluster_variant_f32(v.L, v.R, K)
                                          : jacobi_cluster_variant_f64(v.L, v.R, K));
    int force = 0;
    if (const char* env = getenv("TNN_JACOBI_CLUSTER")) force = atoi(env);
    if (cluster && has && (!p->in_smem || force > 1)) {
        for (int C = 2; C <= jac::kMaxCluster; C *= 2) {
            if (force > 1 && C != force) continue;
            // 2C super-blocks of an even number s of blocks
            const int nbC = 4 * C * (int)((n + 4 * C * K - 1) / (4 * C * K));
            const int npadC = nbC * K, sK = nbC / (2 * C) * K;
            int W = (nbC / (2 * C) + gpw - 1) / gpw;
            if (W > 32) W = 32;
            const size_t smem = jac::cluster_smem_bytes(p->ldA, sK, npadC, elem);
            if (smem > 226 * 1024) continue;
            if ((size_t)W * jac::rebuild_jb(v.R, v.L) * npadC > jac::cluster_buf_elems(p->ldA, sK, elem)) continue;
            p->cluster = C;
            p->nb = nbC;
            p->in_smem = 1;
            p->smem_bytes = smem;
            p->work_bytes = 0;
            p->W = W;
            break;
        }
    }
    return true;
}

bool jacobi_plan(int64_t n1, int64_t n2, int64_t n3, int elem, JacobiPlan* plan)
{
    return jacobi_plan_mode(n1, n2, n3, elem, false, plan);
}

}  // namespace tnn

extern "C" tnn_status tnn_jacobi_plan_info(tnn_shape shape, tnn_precision prec, int64_t out[9])
{
    if (!out) return TNN_EINVAL;
    if (!(prec == TNN_FP64 || prec == TNN_FP32 || prec == TNN_FP32_TF32X3 || prec == TNN_FP32_BF16SPLIT))
        return TNN_EINVAL;
    tnn::JacobiPlan p;
    if (!tnn::jacobi_plan(shape.n1, shape.n2, shape.n3, prec == TNN_FP64 ? 8 : 4, &p)) return TNN_EINVAL;
    out[0] = p.L;
    out[1] = p.RA;
    out[2] = p.K;
    out[3] = p.nb;
    out[4] = p.W;
    out[5] = p.in_smem;
    out[6] = p.cluster > 1 ? p.cluster : 1;
    out[7] = (int64_t)p.smem_bytes;
    out[8] = (int64_t)p.work_bytes;
    return TNN_OK;
}
