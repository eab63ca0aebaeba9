// Internal declarations shared by the libtnn CUDA sources.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/tnn.h"

namespace tnn {

// Device-resident control block of an ADMM run (Algorithm 1).  Every kernel
// of an iteration reads beta and `done` from here, and the finalize kernel
// advances it, so iterations can be queued ahead of the host's stop test:
// once `done` is set, queued iterations exit at their first instruction.
struct AdmmCtl {
    double beta;       // beta of the iteration about to run
    double rho, beta_max, tol;
    int32_t iter;      // iterations completed in this run
    int32_t max_iter;
    int32_t done;      // 1: the run has stopped; kernels return immediately
    int32_t converged; // 1: the tol test stopped the run
    double rel_change; // ||X+ - X|| / ||X|| of the last completed iteration
    double primal_res; // ||Y - X+|| / ||X+|| of the last completed iteration
    int32_t sweeps_max;       // most Jacobi sweeps of a slice, last iteration
    int32_t unconverged;      // slices that hit the sweep cap, whole run
    int32_t nonfinite;        // a NaN/Inf was met
    int32_t pad_;
};

// Per-slice Jacobi statistics, written by the SVT/SVD kernels.
// Per-sweep log of the single-CTA Jacobi SVT (TNN_OPT_JACOBI_SWEEP_LOG): for
// each slice, kSweepLogSweeps rows (one per sweep) and a row of phase times,
// kSweepLogVals floats each.
constexpr int kSweepLogSweeps = 8;
constexpr int kSweepLogVals = 8;
constexpr int sweep_log_floats = (kSweepLogSweeps + 1) * kSweepLogVals;

// Per-slice record the Jacobi SVT leaves for the offloaded tail
// (warm_tail_kernel), in 32-bit words: coef[q] (q < keep), 1 / (d_c |s_c|^2)
// by column, rank_c by column (int), kidx[q] (int), keep (int), has_vec (int:
// the slice ran sweeps, so its recovered vectors are valid).
__host__ __device__ inline size_t tail_info_stride(int npad) { return 4 * (size_t)npad + 4; }

struct SliceStats {
    double nuc;        // sum_i (sigma_i - tau)_+ of the slice
    int64_t pairs;     // column pairs visited
    int64_t rotations; // rotations applied
    int32_t sweeps;    // sweeps run
    int32_t converged; // 1 if the last sweep applied no rotation
    int32_t nonfinite; // 1 if a NaN/Inf was met
    int32_t kept;      // singular values above tau (SVT) / singular values (SVD)
};

// ---- tube transforms (tube.cu) ----------------------------------------------
// out(p, q) = sum_j in(p, j) * op(j, q) over the tube index (P pixels, n3
// tube positions), op the n3 x n3 operator built by launch_build_operator
// from the DCT definition:
//   forward (inverse = 0): op(j, q) = C[q, j]      (divided by w_q if scaled)
//   inverse (inverse = 1): op(k, q) = C[k, q]      (times w_k if scaled)
template <typename T>
cudaError_t launch_build_operator(T* op, int64_t n3, int inverse, int scaled, cudaStream_t s);

template <typename T>
cudaError_t launch_tube_op(const T* X, T* Y, const T* op, int64_t P, int64_t n3, cudaStream_t s);

// Forward transform with the ADMM prologue Z = X - M / beta (beta from ctl).
template <typename T>
cudaError_t launch_tube_fwd_admm_op(const T* X, const T* M, T* Zbar, const T* op, int64_t P, int64_t n3,
                                    const AdmmCtl* ctl, cudaStream_t s);

// Inverse transform with the ADMM epilogue of Algorithm 1: Y = idct(Ybar);
//   X+ = mask ? B : Y + M / beta;  M+ = M + beta (Y - X+);  X <- X+, M <- M+;
// per-block FP64 partial sums of ||X+ - X||^2, ||X||^2, ||Y - X+||^2, ||X+||^2
// into `partials` (4 doubles per block); *nblocks receives the block count.
template <typename T>
cudaError_t launch_tube_inv_admm_op(const T* Ybar, T* X, T* M, const T* B, const uint8_t* mask, const T* op,
                                    int64_t P, int64_t n3, const AdmmCtl* ctl, double* partials, int* nblocks,
                                    cudaStream_t s);

// Number of partial-sum blocks launch_tube_inv_admm_op writes.
int tube_partials_count(int64_t P, int64_t n3);

// Finalize one ADMM iteration: reduce the partials (fixed order), set
// rel_change / primal_res, advance beta and iter, set done.  One block.
cudaError_t launch_admm_finalize(AdmmCtl* ctl, const double* partials, int nblocks, const SliceStats* stats,
                                 int64_t n3, cudaStream_t s);

// X = mask ? B : 0,  M = 0.
template <typename T>
cudaError_t launch_admm_init(const T* B, const uint8_t* mask, T* X, T* M, int64_t N, cudaStream_t s);
cudaError_t launch_ctl_init(AdmmCtl* ctl, double beta, double rho, double beta_max, double tol, int max_iter,
                            cudaStream_t s);

// ---- tube transforms on tcgen05 tensor cores (tube_tc.cu), FP32 data -------
// 3xTF32 split, or BF16 hi/lo split when bf; the operator is passed as
// prebuilt hi/lo images in the MMA's shared-memory layout
// (launch_build_operator_tc, tube_tc_image_floats floats of storage).
// *err is set to 1 if a bounded wait timed out; `spin` bounds the polls of
// each wait (negative: the default limit, about 4e6 polls).
bool tube_tc_supported(int64_t n3);
size_t tube_tc_image_floats(int64_t n3, bool bf);
int tube_tc_partials_count(int64_t P);
cudaError_t launch_build_operator_tc(float* img, int64_t n3, int inverse, int scaled, bool bf, cudaStream_t s);
cudaError_t launch_tube_tc(const float* X, float* Y, const float* img, int64_t P, int64_t n3, bool bf, int* err,
                           cudaStream_t s, int spin = -1);
cudaError_t launch_tube_tc_fwd_admm(const float* X, const float* M, float* Zbar, const float* img, int64_t P,
                                    int64_t n3, bool bf, const AdmmCtl* ctl, int* err, cudaStream_t s,
                                    int spin = -1);
cudaError_t launch_tube_tc_inv_admm(const float* Ybar, float* X, float* M, const float* B, const uint8_t* mask,
                                    const float* img, int64_t P, int64_t n3, bool bf, const AdmmCtl* ctl,
                                    double* partials, int* nblocks, int* err, cudaStream_t s, int spin = -1);

// ---- Jacobi SVT / SVD (jacobi.cu) -------------------------------------------
// One frontal slice of a batched SVT launch (slices of different tensors and
// shapes in one grid, one CTA each).
struct SliceItem {
    void* data;         // the slice (n1 x n2, leading dimension n1), overwritten by its SVT
    int n1, n2;         // slice shape
    int m, n, tr, nb;   // oriented shape (m >= n), transposed flag, column blocks
    double tau;         // threshold (when ctl is null)
    SliceStats* stats;  // where the slice's statistics go
    const AdmmCtl* ctl; // batched ADMM: threshold 1/beta from here; nothing runs once done
};

enum JacobiMode { JAC_SVT = 0, JAC_SVD = 1 };

struct JacobiPlan {
    int64_t n1, n2, n3;
    int m, n;          // oriented slice: m >= n (m = max(n1,n2))
    int tr;            // 1 if the slice is transposed (n1 < n2)
    int K, RA, W;      // block width, rows per lane, warps per CTA
    int L;             // lanes per block pair (16 or 32)
    int nb;            // number of column blocks (even)
    int ldA;           // leading dimension of the working copy (rows, padded)
    int in_smem;       // working copy in shared memory
    size_t smem_bytes; // dynamic shared memory per CTA
    size_t work_bytes; // global scratch per launch
    int elem;          // sizeof(T)
    int cluster;       // > 1: each slice spread over a cluster of this many CTAs (SVT only)
    int angle64 = 0;   // FP32 SVT of slices in shared memory: rotation angles and convergence tests in FP64
    int small_stop = 1; // Jacobi: stop after a sweep whose rotations were all small (KArgs::small_stop)
    float* sweep_log = nullptr;  // single-CTA SVT: per-sweep rotation log (KArgs::sweep_log), or none
};

// Plan a Jacobi launch for n1 x n2 slices of element size elem (4 or 8).
// Returns false if the shape is beyond what the kernels support.
bool jacobi_plan(int64_t n1, int64_t n2, int64_t n3, int elem, JacobiPlan* plan);
// Same, for the SVD launch (singular vectors kept) when withv is true.
bool jacobi_plan_mode(int64_t n1, int64_t n2, int64_t n3, int elem, bool withv, JacobiPlan* plan,
                      bool cluster = true);

// SVT of every frontal slice of `data` in place:  data_k <- U (S - tau)_+ V^T.
// tau = 1 / ctl->beta when ctl is not null (and the launch exits if ctl->done).
// Warm start of the SVT (warm.cu): w0 = start columns (per slice, working-
// copy layout, launch stride ldA * nb * K), wflag = slices whose w0 is valid,
// vrec / wrec = the recovered right vectors and their flags (vrec may be w0).
struct WarmPtrs {
    void* w0;
    const int* wflag;
    void* vrec;
    int* wrec;
    void* tail_s = nullptr;       // offloaded tail: the converged columns go here (may be w0) ...
    float* tail_info = nullptr;   // ... and the per-slice record (tail_info_stride words each)
};

template <typename T>
cudaError_t launch_jacobi_svt(const JacobiPlan& plan, T* data, double tau, const AdmmCtl* ctl, int max_sweeps,
                              void* work, SliceStats* stats, cudaStream_t s, const WarmPtrs* warm = nullptr);

// Warm start across ADMM iterations (FP32, slices held by one CTA).  State:
// n3 orthogonal n x n matrices Q followed by n3 int flags (warm_state_bytes);
// zero-filled = cold.  Scratch: n3 * ldA * nb * K elements (W0, then the
// recovered vectors) and n3 int flags.
bool warm_supported(const JacobiPlan& p);
size_t warm_state_bytes(int64_t n3, int n, int elem);
template <typename T>
cudaError_t launch_warm_gemm(const JacobiPlan& p, const T* data, const T* Q, const int* flag, T* w0,
                             const AdmmCtl* ctl, cudaStream_t s);
template <typename T>
cudaError_t launch_warm_qr(const JacobiPlan& p, const T* vrec, size_t vstride, int* wrec, T* Q, int* flag,
                           const AdmmCtl* ctl, cudaStream_t s);
// The offloaded tail of the warm-started SVT (recovered vectors into V, n x n
// per slice; the rebuild over the slices in `data`), from the Jacobi
// kernel's columns S and record `info`; tail_supported says whether the
// shape fits (else the Jacobi kernel keeps its own tail).
bool tail_supported(const JacobiPlan& p);
template <typename T>
cudaError_t launch_warm_tail(const JacobiPlan& p, T* data, const T* S, const float* info, T* V, int* wrec,
                             const AdmmCtl* ctl, cudaStream_t s);

// SVT of a list of slices (device array of `count` SliceItems) that all use
// the variant of `plan` (K, RA, L, ldA, in_smem); plan.nb and plan.n3 must be
// the largest block count and the item count.  `work` holds count x the
// per-slice working copy when the variant does not keep it in shared memory.
template <typename T>
cudaError_t launch_jacobi_svt_items(const JacobiPlan& plan, const SliceItem* items, int count, int max_sweeps,
                                    void* work, cudaStream_t s);

// SVD of every frontal slice of `data` (not modified):  U (n1 x r per slice),
// sigma (r per slice, descending), V (n2 x r per slice), r = min(n1, n2).
template <typename T>
cudaError_t launch_jacobi_svd(const JacobiPlan& plan, const T* data, T* U, T* sigma, T* V, int max_sweeps,
                              void* work, SliceStats* stats, cudaStream_t s);

// Compiled SVT variants for an element size: fills up to `max` (L, R, K)
// triples, returns how many exist.
int jacobi_svt_variants(int elem, int* L, int* R, int* K, int max);
// Plan for one given variant (false if it does not cover the shape).
bool jacobi_plan_variant(int64_t n1, int64_t n2, int64_t n3, int elem, int L, int R, int K, JacobiPlan* plan);

// ---- batched tube transforms (batch.cu) -------------------------------------
// One 128-pixel tile of one tensor's plain tube transform.
struct TubeItem {
    const void* in;
    void* out;
    const void* op;  // that tensor's n3 x n3 operator (launch_build_operator)
    int64_t P;       // pixels of the tensor
    int64_t p0;      // first pixel of the tile
    int n3;
    int pad_;
};
template <typename T>
cudaError_t launch_tube_batched(const TubeItem* items, int count, cudaStream_t s);
int tube_batched_tile();

// ---- batched ADMM steps (tube.cu kernels, batch.cu plans) -----------------------
// One 128-pixel x 64-position tile of one tensor's forward (MODE 1: in = X,
// in2 = M, out = W) or inverse (MODE 2: in = W, ADMM update of X, M from B
// and the mask, partial sums to partials[4 tile ..]) transform.
struct AdmmTileItem {
    const void* in;
    const void* in2;
    void* out;
    const void* op;
    void* X;
    void* M;
    const void* B;
    const uint8_t* mask;
    double* partials;
    const AdmmCtl* ctl;
    int64_t P, p0, tile;
    int n3, q0;
};
// One job's finalize (the per-iteration stop test and beta update).
struct AdmmJobItem {
    AdmmCtl* ctl;
    const double* partials;
    const SliceStats* stats;
    int64_t n3;
    int nblocks, pad_;
};
template <typename T>
cudaError_t launch_tube_admm_batched(const AdmmTileItem* items, int count, int mode, cudaStream_t s);
cudaError_t launch_admm_finalize_batched(const AdmmJobItem* jobs, int count, cudaStream_t s);
// A group of slices sharing one Jacobi launch (plan: variant, residency,
// largest block count; n3 = slices).
struct SliceGroup {
    JacobiPlan plan;
    int off = 0, count = 0;
    void* work = nullptr;  // plan.work_bytes of scratch when not in shared memory
};
struct AdmmJob;
// Launch tables of one batched ADMM iteration over `jobs` (CUDA-core
// transforms: opf.op / opi.op): forward and inverse tiles, finalize items,
// and the slice items grouped by the plan each job's slices would get alone
// (longest slices first).  false if a shape has no plan.
void build_admm_tiles(const std::vector<const AdmmJob*>& jobs, std::vector<AdmmTileItem>& fwd,
                      std::vector<AdmmTileItem>& inv, std::vector<AdmmJobItem>& jt);
bool build_admm_slices(int elem, const std::vector<const AdmmJob*>& jobs, std::vector<SliceGroup>& groups,
                       std::vector<SliceItem>& slices);
// One iteration from device tables: forward tiles, the groups (spread over
// the side streams between fork and join events when more than one), inverse
// tiles, finalize.
cudaError_t enqueue_admm_iteration(int elem, const AdmmTileItem* fwd, const AdmmTileItem* inv, int ntiles,
                                   const AdmmJobItem* jobs, int njobs, const std::vector<SliceGroup>& groups,
                                   const SliceItem* slices, int sweeps, cudaStream_t s, const cudaStream_t* side,
                                   int nside, cudaEvent_t fork, const cudaEvent_t* join);

// Tile grid of the CUDA-core transforms: tile (x, y) covers pixels
// [x tube_tile_pixels(), ..) and positions [y tube_tile_outputs(), ..);
// its partial-sum index is y tube_tiles_x(P) + x.
int tube_tiles_x(int64_t P);
int tube_tiles_y(int64_t n3);
int tube_tile_pixels();
int tube_tile_outputs();

// ---- DFT comparison path (dft.cu) ------------------------------------------------
// out(p, q) = sum_j in(p, j) op(j, q), q < nout; op nin x nout column-major.
template <typename T>
cudaError_t launch_tube_rect(const T* in, T* out, const T* op, int64_t P, int nin, int nout, cudaStream_t s);
// Forward (n3 x 2nh) and inverse (2nh x n3) real DFT operators, nh = n3/2 + 1:
// slice k of the half spectrum as planes 2k (real part) and 2k + 1 (imaginary).
template <typename T>
cudaError_t launch_build_dft_ops(T* fwd, T* inv, int n3, cudaStream_t s);
// Plain one-sided Jacobi SVT of n3s slices (n1 x n2, slice s at data + s *
// stride; complex slices keep their imaginary plane im_off elements after the
// real one), threshold tau, in place.  Scratch bytes when the working copy
// does not fit in shared memory (smem_copy = false).
size_t jacobi_plain_work_bytes(int64_t n1, int64_t n2, int64_t n3s, int elem, bool cplx, bool* smem_copy);
template <typename T>
cudaError_t launch_jacobi_plain(T* data, int64_t stride, int64_t im_off, int n3s, int n1, int n2, double tau,
                                bool cplx, T* work, bool smem_copy, SliceStats* stats, cudaStream_t s);

// ---- one completion job's device state (api.cu) ---------------------------------
// One tube transform direction: CUDA-core operator or tensor-core images.
struct TubeOp {
    const void* op = nullptr;    // CUDA-core operator (n3 x n3)
    const float* img = nullptr;  // tensor-core images
    bool tc = false;
    bool bf = false;             // BF16 hi/lo split (else 3xTF32)
};

// Everything an ADMM run (Algorithm 1) touches on the device.
struct AdmmJob {
    tnn_shape sh;
    tnn_precision prec;
    int elem;
    tnn_admm_params prm;
    const void* B;
    const uint8_t* mask;
    void* X;
    void* M;
    void* W;               // transformed tensor (N elements)
    AdmmCtl* ctl;          // device control block
    double* partials;      // tube_partials_count(P, n3) x 4
    SliceStats* stats;     // n3
    void* jwork;           // plan.work_bytes
    JacobiPlan jp;
    TubeOp opf, opi;       // filled by admm_prepare_job
    // warm start (FP32, warm_supported(jp)): the state (Q per slice, then
    // flags), the scratch (n3 * ldA * nb * K elements) and its n3 flags
    void* warm = nullptr;
    void* wscr = nullptr;
    int* wrec = nullptr;
    // offloaded SVT tail (tail_supported(jp)): n3 x tail_info_stride(npad) words
    float* tinfo = nullptr;
    // with the tail: the QR on this side stream (it needs only the tail's
    // output, so it overlaps the inverse and next forward transforms); the
    // next A Q waits for ev_qr
    cudaStream_t qs = nullptr;
    cudaEvent_t ev_tail = nullptr, ev_qr = nullptr;
};

// The job's transform operators, from the context's caches (built on first use).
tnn_status admm_prepare_job(tnn_ctx* ctx, AdmmJob& j, cudaStream_t s);
// Queue `iters` iterations on stream s; each exits at once if the job is done.
tnn_status admm_enqueue_iters(tnn_ctx* ctx, const AdmmJob& j, int iters, cudaStream_t s);

// ---- context hooks for entry points outside api.cu ------------------------------
tnn_status ctx_fail(tnn_ctx* ctx, tnn_status s, const char* msg);
tnn_status ctx_check_tc(tnn_ctx* ctx);  // after a synchronisation: a tensor-core wait that timed out
int ctx_device(const tnn_ctx* ctx);
bool is_device_pointer(const void* p);

// ---- facewise products (facewise.cu) -------------------------------------------
// C_k = op(A_k) * B_k for k < nb, A_k m x kk (or kk x m if transA), B_k kk x n,
// all column-major and contiguous per slice.  Optional per-slice column scale
// of A: if dscale != null, A_k(:, q) is multiplied by dscale[q + kk*k].
template <typename T>
cudaError_t launch_facewise(const T* A, const T* B, T* C, int64_t m, int64_t n, int64_t kk, int64_t nbatch,
                            int transA, int transB, const T* dscale, cudaStream_t s);

}  // namespace tnn
