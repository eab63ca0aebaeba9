// Shape planning for the Jacobi kernels (host only).
#include "jacobi_launch.cuh"

namespace tnn {

static int pick_RA(int m, int elem)
{
    static const int ra32[] = {2, 4, 6, 8, 12, 16};
    static const int ra64[] = {1, 2, 4, 6, 8, 12, 16};
    const int* t = elem == 4 ? ra32 : ra64;
    int cnt = elem == 4 ? 6 : 7;
    for (int i = 0; i < cnt; ++i)
        if (32 * t[i] >= m) return t[i];
    return 0;
}

bool jacobi_plan_mode(int64_t n1, int64_t n2, int64_t n3, int elem, bool withv, JacobiPlan* p)
{
    if (n1 <= 0 || n2 <= 0 || n3 <= 0) return false;
    const int64_t m = n1 >= n2 ? n1 : n2;
    const int64_t n = n1 >= n2 ? n2 : n1;
    if (m > 512) return false;
    if (withv && elem == 8 && m > 256) return false;
    int RA = pick_RA((int)m, elem);
    if (RA == 0) return false;
    int K = jac::pick_K(elem, RA, withv);
    p->n1 = n1; p->n2 = n2; p->n3 = n3;
    p->m = (int)m; p->n = (int)n; p->tr = n1 < n2 ? 1 : 0;
    p->K = K; p->RA = RA;
    p->nb = 2 * (int)((n + 2 * K - 1) / (2 * K));
    p->ldA = 32 * RA + (elem == 4 ? 2 : 1);
    p->elem = elem;
    const int npad = p->nb * K;
    const int Wguess = p->nb / 2 < 32 ? p->nb / 2 : 32;
    size_t wsz = (size_t)p->ldA * npad * elem;
    size_t big = (withv ? 2 : 1) * ((wsz + 255) & ~(size_t)255);
    size_t small = jac::smem_small_bytes(npad, Wguess, elem);
    p->in_smem = (big + small) <= 226 * 1024 ? 1 : 0;  // static shared memory needs a little room
    p->smem_bytes = p->in_smem ? big + small : small;
    p->work_bytes = p->in_smem ? 0 : (size_t)n3 * (withv ? 2 : 1) * wsz;
    p->W = Wguess;
    return true;
}

bool jacobi_plan(int64_t n1, int64_t n2, int64_t n3, int elem, JacobiPlan* plan)
{
    return jacobi_plan_mode(n1, n2, n3, elem, false, plan);
}

}  // namespace tnn
