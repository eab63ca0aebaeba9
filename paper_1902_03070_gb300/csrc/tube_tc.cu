// Tube transforms on the tcgen05 tensor cores (FP32 data, 3xTF32 split or
// three-part BF16 split).
//
// out(p, q) = sum_j in(p, j) op(j, q) as a GEMM with M = pixels (a CTA owns
// 128 of them, the MMA's M), N = output tube positions (n3 rounded up to 16,
// all of them in one TMEM accumulator) and K = input tube positions, taken in
// chunks of 32.  FP32 accuracy from TF32 products: x = x_hi + x_lo with x_hi
// x rounded to TF32 (10 mantissa bits) and x_lo = x - x_hi (exact in FP32,
// at most 2^-11 |x|), and out = A_hi B_hi + A_hi B_lo + A_lo B_hi (the
// dropped A_lo B_lo term is below 2^-22 relative).  The BF16 form splits
// each value into three BF16 parts x = x0 + x1 + x2 (8 significant bits
// each; x1 at most 2^-9 |x|, x2 at most 2^-17 |x|, the rest below 2^-25 |x|)
// and runs the six products of total order at most two (A0 B0, A0 B1,
// A1 B0, A0 B2, A1 B1, A2 B0) as kind::f16 MMAs with FP32 accumulation:
// what it drops is below about 2^-24 relative, FP32 accuracy.  (With two
// parts and three products the dropped terms are of order 2^-16, a transform
// error of a few 1e-6, which shows in the t-SVT at the 1e-5 level.)
//
// Staging: 256 threads, two per pixel row (each takes half of a K chunk), load
// the input strip with coalesced loads (the ADMM prologue Z = X - M/beta is
// applied here), split it and write the K-major core-matrix layout (8 rows x
// 16 bytes per core matrix, no swizzle);
// the operator's hi/lo images are prebuilt in the same layout, chunk by chunk,
// and each chunk is copied in by bulk asynchronous copies (TMA engine) that
// complete on an mbarrier.  One thread issues the MMAs and commits them to a
// second mbarrier; the epilogue reads the accumulator with tcgen05.ld (warp w
// reads TMEM lanes 32 (w % 4) .. + 31 = pixels, the two warps of a lane
// quarter taking alternate 16-column chunks, so twice the loads are in
// flight) and writes the output coalesced, with the ADMM update fused in the
// inverse direction.
//
// Every mbarrier wait is bounded: on timeout the kernel records an error,
// stops issuing work, waits (bounded) for what it has in flight, frees its
// TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "tnn_internal.h"

namespace tnn {
namespace {

constexpr int TBM = 128;          // pixels per CTA (MMA M)
constexpr int TKC = 32;           // K chunk (input tube positions per stage)
constexpr int TTHREADS = 256;     // two threads per pixel row (each stages half of a K chunk)
constexpr int TKH = TKC / 2;      // K values a thread stages per chunk
constexpr uint32_t kSpinLimit = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// x rounded to the nearest TF32 value (10 mantissa bits), ties away from zero.
__device__ __forceinline__ float tf32_hi(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Shared-memory matrix descriptor, K-major, no swizzle: start address, byte
// offset between core matrices adjacent along K (lbo) and along M/N (sbo).
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
    d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version
    return d;
}

// Instruction descriptor: D in F32, A and B in TF32, both K-major, M x N.
__host__ __device__ constexpr uint32_t make_idesc_tf32(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// The same for kind::f16 with A and B both BF16.
__host__ __device__ constexpr uint32_t make_idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// BF16 bits of x rounded to nearest even, and the rounded value.
__device__ __forceinline__ uint16_t bf16_bits(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float bf16_val(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// Bounded wait for the given phase parity (at most `limit` polls); false on
// timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit)
{
    const uint32_t a = smem_u32(bar);
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(
            dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
            dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Byte offset of element (row, k) of a K-major tile of TKC columns: core
// matrices of 8 rows x 16 bytes (4 TF32 or 8 BF16 values of K per row).
template <bool BF>
__host__ __device__ __forceinline__ uint32_t kmajor_off(int row, int k)
{
    constexpr int E = BF ? 8 : 4;  // K values per 16-byte core-matrix row
    constexpr int ES = BF ? 2 : 4;
    return (uint32_t)((k / E) * 128 + (row >> 3) * (TKC / E * 128) + (row & 7) * 16 + (k % E) * ES);
}

// MODE 0: plain; MODE 1: forward with Z = X - M/beta; MODE 2: inverse with the
// ADMM update.  BF: three-part BF16 split (kind::f16) instead of 3xTF32.
template <int MODE, bool BF>
__global__ void __launch_bounds__(TTHREADS, 2)
tube_tc_kernel(const float* __restrict__ in, const float* __restrict__ in2, float* __restrict__ out,
               const float* __restrict__ bimg, int64_t P, int n3, int NP, int nchunks, uint32_t tmem_cols,
               const AdmmCtl* __restrict__ ctl, float* __restrict__ Xs, float* __restrict__ Ms,
               const float* __restrict__ Bs, const uint8_t* __restrict__ mask, double* __restrict__ partials,
               int* __restrict__ err, uint32_t spin)
{
    if (MODE != 0 && ctl->done) return;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar_b[2], bar_mma;
    __shared__ uint32_t s_taddr;
    __shared__ double red[TTHREADS / 32][4];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t p0 = (int64_t)blockIdx.x * TBM;
    constexpr uint32_t ES = BF ? 2 : 4;                // bytes per staged value
    constexpr int NPART = BF ? 3 : 2;                  // split parts per value
    const uint32_t a_bytes = TBM * TKC * ES;           // one A tile (one part)
    const uint32_t b_bytes = (uint32_t)NP * TKC * ES;  // one B tile (one part)
    unsigned char* Ahi = smem;
    unsigned char* Alo = smem + a_bytes;
    unsigned char* Alo2 = smem + 2 * a_bytes;          // BF16: third part
    // two stages of operator tiles: stage t holds the NPART parts from Bst(t) on
    auto Bst = [&](int t) { return smem + NPART * a_bytes + (size_t)t * NPART * b_bytes; };

    float rbeta = 1.f, rinv = 1.f;
    if (MODE != 0) {
        rbeta = (float)ctl->beta;
        rinv = (float)(1.0 / ctl->beta);  // M / beta as M * (1 / beta): within an ulp, no division per element
    }

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_taddr)),
                     "r"(tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        mbar_init(&bar_b[0], 1);
        mbar_init(&bar_b[1], 1);
        mbar_init(&bar_mma, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t taddr = s_taddr;
    const uint32_t idesc = BF ? make_idesc_bf16(TBM, NP) : make_idesc_tf32(TBM, NP);
    const int row = tid & (TBM - 1), half = tid / TBM;  // staging: pixel row, half of the K chunk
    const int64_t p = p0 + row;
    const bool prow = p < P;

    uint32_t phase_b[2] = {0u, 0u}, phase_m = 0;
    bool b_pending[2] = {false, false};  // thread 0: a stage copy not yet awaited
    bool mma_pending = false;            // thread 0: a commit not yet awaited
    bool ok = true;
    auto issue_b = [&](int chunk) {
        const int t = chunk & 1;
        mbar_expect_tx(&bar_b[t], NPART * b_bytes);
        const unsigned char* src = reinterpret_cast<const unsigned char*>(bimg) + (size_t)chunk * NPART * b_bytes;
#pragma unroll
        for (int q = 0; q < NPART; ++q) bulk_g2s(Bst(t) + q * b_bytes, src + q * b_bytes, b_bytes, &bar_b[t]);
        b_pending[t] = true;
    };
    if (tid == 0) issue_b(0);
    // a chunk's inputs, loaded into registers (issued early: see the loop below)
    auto load_chunk = [&](int c, float (&v)[TKH], float (&w)[TKH]) {
        const int k0 = c * TKC + half * TKH;
#pragma unroll
        for (int u = 0; u < TKH; ++u) {
            const int j = k0 + u;
            const bool ld = prow && j < n3;
            const size_t e = (size_t)p + (size_t)P * (ld ? j : 0);
            v[u] = ld ? __ldg(in + e) : 0.f;
            if (MODE == 1) w[u] = ld ? __ldg(in2 + e) : 0.f;
        }
    };
    // split chunk c into the A tiles and issue its MMAs; false on a timeout
    auto run_chunk = [&](int c, float (&v)[TKH], float (&w)[TKH]) -> bool {
        if (c > 0) {
            // the A tiles are rewritten only after the previous chunk's MMAs completed
            const int late = mbar_wait(&bar_mma, phase_m, spin) ? 0 : 1;
            phase_m ^= 1;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (__syncthreads_or(late)) return false;
            if (tid == 0) mma_pending = false;
        }
        if (!BF) {
#pragma unroll
            for (int g = 0; g < TKH / 4; ++g) {
                float x[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) x[u] = (MODE == 1) ? fmaf(-w[g * 4 + u], rinv, v[g * 4 + u]) : v[g * 4 + u];
                float4 hi, lo;
                hi.x = tf32_hi(x[0]); lo.x = x[0] - hi.x;
                hi.y = tf32_hi(x[1]); lo.y = x[1] - hi.y;
                hi.z = tf32_hi(x[2]); lo.z = x[2] - hi.z;
                hi.w = tf32_hi(x[3]); lo.w = x[3] - hi.w;
                const uint32_t off = kmajor_off<false>(row, half * TKH + g * 4);
                *reinterpret_cast<float4*>(Ahi + off) = hi;
                *reinterpret_cast<float4*>(Alo + off) = lo;
            }
        } else {
#pragma unroll
            for (int g = 0; g < TKH / 8; ++g) {
                // x = x0 + x1 + x2, each part rounded to BF16 from what the
                // parts before it leave (x - x0 and x - x0 - x1 are exact in FP32)
                uint32_t hw[4], mw[4], lw[4];
#pragma unroll
                for (int u = 0; u < 8; u += 2) {
                    float x0 = v[g * 8 + u], x1 = v[g * 8 + u + 1];
                    if (MODE == 1) {
                        x0 = fmaf(-w[g * 8 + u], rinv, x0);
                        x1 = fmaf(-w[g * 8 + u + 1], rinv, x1);
                    }
                    const uint16_t h0 = bf16_bits(x0), h1 = bf16_bits(x1);
                    const float r0 = x0 - bf16_val(h0), r1 = x1 - bf16_val(h1);
                    const uint16_t m0 = bf16_bits(r0), m1 = bf16_bits(r1);
                    const uint16_t l0 = bf16_bits(r0 - bf16_val(m0)), l1 = bf16_bits(r1 - bf16_val(m1));
                    hw[u / 2] = (uint32_t)h0 | ((uint32_t)h1 << 16);
                    mw[u / 2] = (uint32_t)m0 | ((uint32_t)m1 << 16);
                    lw[u / 2] = (uint32_t)l0 | ((uint32_t)l1 << 16);
                }
                const uint32_t off = kmajor_off<true>(row, half * TKH + g * 8);
                *reinterpret_cast<uint4*>(Ahi + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                *reinterpret_cast<uint4*>(Alo + off) = make_uint4(mw[0], mw[1], mw[2], mw[3]);
                *reinterpret_cast<uint4*>(Alo2 + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
            }
        }
        // make the generic-proxy writes visible to the tensor cores
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        int fail = 0;
        if (tid == 0) {
            const int t = c & 1;
            if (!mbar_wait(&bar_b[t], phase_b[t], spin)) {
                fail = 1;
            } else {
                b_pending[t] = false;
                phase_b[t] ^= 1;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                // an MMA takes 32 bytes of K (8 TF32 or 16 BF16 values): two core matrices
                const uint32_t sbo = TKC / (BF ? 8 : 4) * 128, lbo = 128;
                const uint32_t bh0 = smem_u32(Bst(t)), bl0 = bh0 + b_bytes, bl20 = bl0 + b_bytes;
#pragma unroll
                for (int s = 0; s < TKC * (int)ES / 32; ++s) {
                    const uint32_t koff = (uint32_t)s * 2 * 128;
                    const uint64_t ah = make_desc(smem_u32(Ahi) + koff, lbo, sbo);
                    const uint64_t al = make_desc(smem_u32(Alo) + koff, lbo, sbo);
                    const uint64_t bh = make_desc(bh0 + koff, lbo, sbo);
                    const uint64_t bl = make_desc(bl0 + koff, lbo, sbo);
                    if (BF) {
                        // parts 0, 1, 2 of each operand: every product of total
                        // order at most 2 (what is dropped is below 2^-24 relative)
                        const uint64_t al2 = make_desc(smem_u32(Alo2) + koff, lbo, sbo);
                        const uint64_t bl2 = make_desc(bl20 + koff, lbo, sbo);
                        mma_bf16(taddr, ah, bh, idesc, (c > 0 || s > 0) ? 1u : 0u);
                        mma_bf16(taddr, ah, bl, idesc, 1u);
                        mma_bf16(taddr, al, bh, idesc, 1u);
                        mma_bf16(taddr, ah, bl2, idesc, 1u);
                        mma_bf16(taddr, al, bl, idesc, 1u);
                        mma_bf16(taddr, al2, bh, idesc, 1u);
                    } else {
                        mma_tf32(taddr, ah, bh, idesc, (c > 0 || s > 0) ? 1u : 0u);
                        mma_tf32(taddr, ah, bl, idesc, 1u);
                        mma_tf32(taddr, al, bh, idesc, 1u);
                    }
                }
                mma_commit(&bar_mma);
                mma_pending = true;
                // the other stage was read by chunk c-1's MMAs, which completed above
                if (c + 1 < nchunks) issue_b(c + 1);
            }
        }
        if (__syncthreads_or(fail)) return false;
        return true;
    };
    // software pipeline: the loads of chunk c + 1 are in flight while chunk c
    // waits for the MMAs of chunk c - 1, is split and is issued (two register
    // buffers, used alternately, so no load result is copied)
    {
        float va[TKH], wa[TKH], vb[TKH], wb[TKH];
        load_chunk(0, va, wa);
        for (int c = 0; c < nchunks; c += 2) {
            if (c + 1 < nchunks) load_chunk(c + 1, vb, wb);
            if (!run_chunk(c, va, wa)) {
                ok = false;
                break;
            }
            if (c + 1 >= nchunks) break;
            if (c + 2 < nchunks) load_chunk(c + 2, va, wa);
            if (!run_chunk(c + 1, vb, wb)) {
                ok = false;
                break;
            }
        }
    }
    // epilogue lanes: warp w reads TMEM lanes 32 (w % 4) .. + 31 (its pixels),
    // 16 columns at a time, the two warps of a lane quarter alternating chunks
    const int quarter = warp & 3, qhalf = warp >> 2;
    const int64_t pe = p0 + quarter * 32 + lane;
    const bool erow = pe < P;
    // inverse with the ADMM update: the X, M, B, mask values of a 16-column
    // chunk (B is loaded everywhere, no wait on the mask, but only selected on it)
    float xv[16], mv[16], bv[16];
    uint8_t kv[16];
    auto load_epi = [&](int q0) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int q = q0 + u;
            const bool ld = erow && q < n3;
            const size_t e = (size_t)pe + (size_t)P * (ld ? q : 0);
            xv[u] = ld ? Xs[e] : 0.f;
            mv[u] = ld ? Ms[e] : 0.f;
            kv[u] = ld ? mask[e] : (uint8_t)0;
            bv[u] = ld ? __ldg(Bs + e) : 0.f;
        }
    };
    // the first chunk's loads are in flight while the last MMAs finish
    if (MODE == 2 && ok) load_epi(qhalf * 16);
    if (ok) {
        const int late = mbar_wait(&bar_mma, phase_m, spin) ? 0 : 1;
        phase_m ^= 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (__syncthreads_or(late)) ok = false;
        else if (tid == 0) mma_pending = false;
    }

    if (ok) {
        // residual sums in FP64 per thread, FP32 only within a chunk of 16
        double sdx = 0.0, sxx = 0.0, syx = 0.0, snx = 0.0;
        for (int q0 = qhalf * 16; q0 < NP; q0 += 32) {
            float v[16];
            tmem_ld16(taddr + ((uint32_t)(quarter * 32) << 16) + (uint32_t)q0, v);
            if (MODE != 2) {
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int q = q0 + u;
                    if (erow && q < n3) out[(size_t)pe + (size_t)P * q] = v[u];
                }
            } else {
                // Algorithm 1's update (Eq. 25 and the multiplier update of Eq. 20)
                if (q0 > qhalf * 16) load_epi(q0);  // the first chunk's were loaded before the MMA wait
                float cdx = 0.f, cxx = 0.f, cyx = 0.f, cnx = 0.f;
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int q = q0 + u;
                    if (!erow || q >= n3) continue;
                    const size_t e = (size_t)pe + (size_t)P * q;
                    const float y = v[u];
                    const float x = xv[u], mm = mv[u];
                    const float xn = kv[u] ? bv[u] : fmaf(mm, rinv, y);
                    const float mn = fmaf(rbeta, y - xn, mm);
                    const float dx = xn - x, dy = y - xn;
                    cdx = fmaf(dx, dx, cdx);
                    cxx = fmaf(x, x, cxx);
                    cyx = fmaf(dy, dy, cyx);
                    cnx = fmaf(xn, xn, cnx);
                    Xs[e] = xn;
                    Ms[e] = mn;
                }
                sdx += (double)cdx;
                sxx += (double)cxx;
                syx += (double)cyx;
                snx += (double)cnx;
            }
        }
        if (MODE == 2) {
            double sv[4] = {sdx, sxx, syx, snx};
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                for (int t = 0; t < 4; ++t) sv[t] += __shfl_xor_sync(0xffffffffu, sv[t], o);
            if (lane == 0)
#pragma unroll
                for (int t = 0; t < 4; ++t) red[warp][t] = sv[t];
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (MODE == 2 && tid < 4) {
        double t = 0.0;
        for (int w = 0; w < TTHREADS / 32; ++w) t += ok ? red[w][tid] : 0.0;
        partials[(size_t)blockIdx.x * 4 + tid] = t;
    }
    if (!ok && tid == 0) {
        atomicExch(err, 1);
        // let in-flight copies and MMAs land before the shared memory goes
        // away: bounded by the full limit, whatever limit the waits above had
        for (int t = 0; t < 2; ++t)
            if (b_pending[t]) mbar_wait(&bar_b[t], phase_b[t], kSpinLimit);
        if (mma_pending) mbar_wait(&bar_mma, phase_m, kSpinLimit);
    }
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(tmem_cols));
}

// Operator images: for each K chunk, the hi and lo parts (TF32, or BF16
// when bf) of op(k, n) (k = input position, n = output position) in the
// K-major core-matrix layout of an NP x TKC tile; zero outside n3 x n3.
__global__ void build_operator_tc(float* img, int n3, int NP, int nchunks, int inverse, int scaled, int bf)
{
    const int total = nchunks * NP * TKC;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
        const int c = idx / (NP * TKC), r = idx % (NP * TKC);
        const int n = r / TKC, kk = r % TKC, k = c * TKC + kk;
        double v = 0.0;
        if (n < n3 && k < n3) {
            auto Cf = [n3](int a, int b) {
                const double s = (a == 0) ? sqrt(1.0 / n3) : sqrt(2.0 / n3);
                return s * cospi((double)((2 * b + 1) * a) / (2.0 * n3));
            };
            if (!inverse) {  // out_n = sum_k C[n, k] in_k
                v = Cf(n, k);
                if (scaled) v /= Cf(n, 0);
            } else {         // out_n = sum_k C[k, n] in_k
                v = Cf(k, n);
                if (scaled) v *= Cf(k, 0);
            }
        }
        if (!bf) {
            const float hi = tf32_hi((float)v);
            const float lo = tf32_hi((float)(v - (double)hi));
            const uint32_t off = kmajor_off<false>(n, kk) / 4;
            img[(size_t)c * 2 * NP * TKC + off] = hi;
            img[(size_t)c * 2 * NP * TKC + (size_t)NP * TKC + off] = lo;
        } else {
            // three BF16 parts, each rounded from what the parts before it leave
            const uint16_t hi = bf16_bits((float)v);
            const double r = v - (double)bf16_val(hi);
            const uint16_t mid = bf16_bits((float)r);
            const uint16_t lo = bf16_bits((float)(r - (double)bf16_val(mid)));
            uint16_t* b16 = reinterpret_cast<uint16_t*>(img);
            const uint32_t off = kmajor_off<true>(n, kk) / 2;
            b16[(size_t)c * 3 * NP * TKC + off] = hi;
            b16[(size_t)c * 3 * NP * TKC + (size_t)NP * TKC + off] = mid;
            b16[(size_t)c * 3 * NP * TKC + (size_t)2 * NP * TKC + off] = lo;
        }
    }
}

}  // namespace

bool tube_tc_supported(int64_t n3) { return n3 >= 1 && n3 <= 256; }

int tube_tc_np(int64_t n3) { return (int)((n3 + 15) / 16 * 16); }
int tube_tc_chunks(int64_t n3) { return (int)((n3 + TKC - 1) / TKC); }
size_t tube_tc_image_floats(int64_t n3, bool bf)
{
    // TF32: two 4-byte parts per value; BF16: three 2-byte parts
    return bf ? (size_t)tube_tc_chunks(n3) * 3 * tube_tc_np(n3) * TKC / 2
              : (size_t)tube_tc_chunks(n3) * 2 * tube_tc_np(n3) * TKC;
}
int tube_tc_partials_count(int64_t P) { return (int)((P + TBM - 1) / TBM); }

cudaError_t launch_build_operator_tc(float* img, int64_t n3, int inverse, int scaled, bool bf, cudaStream_t s)
{
    const int NP = tube_tc_np(n3), nc = tube_tc_chunks(n3);
    const int total = nc * NP * TKC;
    build_operator_tc<<<(total + 255) / 256, 256, 0, s>>>(img, (int)n3, NP, nc, inverse, scaled, bf ? 1 : 0);
    return cudaGetLastError();
}

template <int MODE, bool BF>
static cudaError_t launch_tc_as(const float* in, const float* in2, float* out, const float* img, int64_t P,
                                int64_t n3, const AdmmCtl* ctl, float* X, float* M, const float* B,
                                const uint8_t* mask, double* partials, int* err, int spin, cudaStream_t s)
{
    const int NP = tube_tc_np(n3), nc = tube_tc_chunks(n3);
    uint32_t cols = 32;
    while ((int)cols < NP) cols <<= 1;
    const size_t es = BF ? 2 : 4;
    const size_t np = BF ? 3 : 2;  // split parts
    const size_t smem = np * (size_t)TBM * TKC * es + 2 * np * (size_t)NP * TKC * es;  // A parts + two B stages
    auto kern = tube_tc_kernel<MODE, BF>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)((P + TBM - 1) / TBM);
    kern<<<grid, TTHREADS, smem, s>>>(in, in2, out, img, P, (int)n3, NP, nc, cols, ctl, X, M, B, mask, partials, err,
                                      spin < 0 ? kSpinLimit : (uint32_t)spin);
    return cudaGetLastError();
}

template <int MODE>
static cudaError_t launch_tc(bool bf, const float* in, const float* in2, float* out, const float* img, int64_t P,
                             int64_t n3, const AdmmCtl* ctl, float* X, float* M, const float* B, const uint8_t* mask,
                             double* partials, int* err, int spin, cudaStream_t s)
{
    return bf ? launch_tc_as<MODE, true>(in, in2, out, img, P, n3, ctl, X, M, B, mask, partials, err, spin, s)
              : launch_tc_as<MODE, false>(in, in2, out, img, P, n3, ctl, X, M, B, mask, partials, err, spin, s);
}

cudaError_t launch_tube_tc(const float* X, float* Y, const float* img, int64_t P, int64_t n3, bool bf, int* err,
                           cudaStream_t s, int spin)
{
    return launch_tc<0>(bf, X, nullptr, Y, img, P, n3, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, err, spin,
                        s);
}

cudaError_t launch_tube_tc_fwd_admm(const float* X, const float* M, float* Zbar, const float* img, int64_t P, int64_t n3,
                                    bool bf, const AdmmCtl* ctl, int* err, cudaStream_t s, int spin)
{
    return launch_tc<1>(bf, X, M, Zbar, img, P, n3, ctl, nullptr, nullptr, nullptr, nullptr, nullptr, err, spin, s);
}

cudaError_t launch_tube_tc_inv_admm(const float* Ybar, float* X, float* M, const float* B, const uint8_t* mask,
                                    const float* img, int64_t P, int64_t n3, bool bf, const AdmmCtl* ctl,
                                    double* partials, int* nblocks, int* err, cudaStream_t s, int spin)
{
    *nblocks = tube_tc_partials_count(P);
    return launch_tc<2>(bf, Ybar, nullptr, nullptr, img, P, n3, ctl, X, M, B, mask, partials, err, spin, s);
}

}  // namespace tnn
