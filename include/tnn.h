/*
 * tnn.h - C ABI of libtnn, a GB300 (sm_103a) implementation of the DCT-based
 * tensor SVD, t-product, tensor singular value thresholding (t-SVT) and TNN-C
 * tensor completion of Xu, Zhao and Ng, "A Fast Algorithm for Cosine
 * Transform Based Tensor Singular Value Decomposition" (arXiv 1902.03070).
 *
 * Layout.  A third-order tensor X of size n1 x n2 x n3 is one contiguous
 * array in the paper's MATLAB order, element (i, j, k) at i + n1*(j + n2*k):
 * each frontal slice X(:,:,k) is a column-major n1 x n2 matrix and the tube
 * X(i,j,:) has stride n1*n2 (Section 2).  Element type: double for
 * TNN_FP64, float for every other precision.
 *
 * Pointers.  Tensor arguments of the single-tensor calls may be device
 * pointers or host pointers; the library asks the CUDA runtime which (the
 * batched plans and the DFT comparison path take device pointers only, the
 * server copies its jobs' inputs itself).  Host buffers are staged through the
 * context's device workspace with copies on the given stream (pinned host
 * memory makes those copies asynchronous) and the call then synchronises the
 * stream before it returns.  The caller owns every buffer it passes; the
 * library never frees or keeps them.  The library allocates device memory only
 * inside tnn_create, tnn_reserve and when a call finds the context's workspace
 * too small (the workspace then grows and never shrinks).
 *
 * Streams.  `stream` is a cudaStream_t passed as void* (NULL = legacy default
 * stream).  Calls on device buffers are stream-ordered and return before the
 * GPU finishes, except where a result is returned in host memory (tnn_out,
 * the report of tnn_complete / tnn_admm_iterate): those calls synchronise
 * the stream.
 *
 * Errors.  No call aborts or prints.  Invalid arguments (a NULL tensor
 * pointer, a non-positive size, tau < 0, beta <= 0, ...) return TNN_EINVAL
 * before anything is launched.  A failing CUDA call returns TNN_ECUDA.  A
 * Jacobi SVD that reached its sweep cap, or an ADMM run that reached max_iter
 * without meeting tol, returns TNN_ENOCONV with every output written.  A NaN
 * or infinity met by a kernel returns TNN_ENONFINITE (outputs written but
 * meaningless).  tnn_last_error() gives a one-line description of the last
 * failure on a context.
 *
 * Threads.  A context may be used from one host thread at a time.
 *
 * Transforms.  dct denotes the orthonormal DCT-II along the tubes (MATLAB's
 * dct(X,[],3), used by Algorithm 1): C[k,j] = a_k cos(pi (2j+1) k / (2 n3)),
 * a_0 = sqrt(1/n3), a_k = sqrt(2/n3).  L denotes the scaled transform under
 * which Theorem 3 and Example 1 hold as printed: L(X)_k = dct(X)_k / w_k with
 * w = C e_1, the first column of C.  The t-product (Eq. 13) and the t-SVD
 * (Theorem 4) use L; the t-SVT and Algorithm 1 use dct as written.
 */
#ifndef TNN_H
#define TNN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TNN_OK = 0,
    TNN_EINVAL = 1,     /* invalid argument; nothing was launched */
    TNN_ENOMEM = 2,     /* device or pinned host allocation failed */
    TNN_ECUDA = 3,      /* a CUDA runtime or driver call failed */
    TNN_ENOCONV = 4,    /* Jacobi sweep cap or ADMM max_iter reached (outputs written) */
    TNN_ENONFINITE = 5, /* NaN or infinity met */
    TNN_ENODEV = 6      /* no usable sm_103 device */
} tnn_status;

typedef enum {
    TNN_FP64 = 0,           /* double data, FP64 arithmetic everywhere (the plain path) */
    TNN_FP32 = 1,           /* float data, FP32 arithmetic on CUDA cores */
    TNN_FP32_TF32X3 = 2,    /* float data, tube DCT on tcgen05 tensor cores, 3xTF32 split */
    TNN_FP32_BF16SPLIT = 3  /* float data, tube DCT on tcgen05 tensor cores, three-part BF16 split (six
                               products accumulated in FP32) */
} tnn_precision;

typedef struct {
    int64_t n1, n2, n3;
} tnn_shape;

/* Algorithm 1 parameters.  beta follows beta <- min(rho beta, beta_max) after
 * every iteration (rho = 1: the paper's fixed beta).  The run stops when both
 * ||X+ - X||_F / ||X||_F <= tol (the paper's test) and ||Y - X+||_F /
 * ||X+||_F <= tol (the residual of the splitting Y = X), or after max_iter
 * iterations.  jacobi_max_sweeps caps the sweeps of every per-slice Jacobi
 * SVD (0 selects 30). */
typedef struct {
    double beta0, rho, beta_max, tol;
    int32_t max_iter;
    int32_t jacobi_max_sweeps;
} tnn_admm_params;

typedef struct {
    int32_t iters;              /* iterations run */
    int32_t converged;          /* 1 if the tol test stopped the run */
    double rel_change;          /* ||X+ - X||_F / ||X||_F of the last iteration */
    double primal_res;          /* ||Y - X+||_F / ||X+||_F of the last iteration */
    double beta_final;          /* beta after the last update */
    int32_t jacobi_sweeps_max;  /* most sweeps any slice needed in the last iteration */
    int32_t jacobi_unconverged; /* slices that hit the sweep cap, summed over the run */
} tnn_admm_report;

typedef struct tnn_ctx tnn_ctx;

/* Create a context on CUDA device `device` (made current for the call).
 * Returns TNN_ENODEV if the device is not compute capability 10.3. */
tnn_status tnn_create(tnn_ctx** ctx, int device);

/* Free the context and its workspace.  NULL is accepted. */
void tnn_destroy(tnn_ctx* ctx);

/* Static string naming a status code. */
const char* tnn_status_string(tnn_status s);

/* One-line description of the last failure on ctx ("" if none). */
const char* tnn_last_error(const tnn_ctx* ctx);

/* Grow the context's device workspace to at least `bytes` (never shrinks). */
tnn_status tnn_reserve(tnn_ctx* ctx, size_t bytes);

/* Per-context options (no counterpart in the paper).
 * TNN_OPT_JACOBI_MAX_SWEEPS: sweep cap of the per-slice Jacobi SVT in
 *   tsvt_dct (0 = the kernels' default of 30; 1 ... 1000).  A slice that
 *   reaches the cap still gets its shrinkage and rebuild from the columns
 *   as they are; the call reports TNN_ENOCONV when it reports a status.
 * TNN_OPT_TC_WAIT_POLLS: how many times each bounded mbarrier wait of the
 *   tensor-core transforms polls before it gives up (negative = the default,
 *   about 4e6).  A wait that gives up makes the kernel set the context's
 *   error flag, stop issuing work, let its own copies and MMAs in flight
 *   finish (waiting with the default bound), free its tensor memory and
 *   return; the next call that checks the flag returns TNN_ECUDA and clears
 *   it.  For exercising that path; the output of a call that timed out is
 *   undefined.
 * TNN_OPT_JACOBI_FP64_ANGLES: 1 = the FP32 Jacobi SVT of tsvt_dct,
 *   tnn_complete and tnn_admm_iterate computes each pair's convergence test
 *   and rotation (Rutishauser's angle and the scaled-rotation factors) in
 *   FP64 from its FP32 dot products, for slices whose working copy fits in
 *   one CTA's shared memory (larger slices keep the FP32 form); 0 (default)
 *   = in FP32.  The columns, the dot products and the rotations applied stay
 *   FP32.  (Measured on the video-shaped workload: about 5x the time per
 *   iteration for errors within 1.2x of the FP32 form's.)
 * TNN_OPT_ADMM_WARM_START: 1 (default) = tnn_complete warm-starts the
 *   per-slice Jacobi of each iteration from the previous iteration's right
 *   singular vectors (FP32 precisions, slices one CTA holds; the state lives
 *   in the workspace; see tnn_admm_iterate); 0 = every iteration starts from
 *   the slices themselves, as the batched plans and the completion server
 *   do, whose iterates tnn_complete then reproduces bit for bit.
 * TNN_OPT_JACOBI_SMALL_STOP: 1 (default) = the Jacobi kernels of tsvt_dct,
 *   tnn_complete and tnn_admm_iterate also stop after a sweep whose
 *   rotations all had |gamma| / sqrt(alpha beta) and |t| at most
 *   theta = sqrt(tol / (4 n)) (tol = sqrt(m) u, n the slice's smaller
 *   side): such a sweep leaves every pair within 2 tol of orthogonal, the
 *   level the plain rule (a sweep without rotation above 2 tol) accepts, so
 *   the sweep that rule spends confirming it is skipped.  0 = the plain rule
 *   only.  The batched plans and the server always use 1.
 * TNN_OPT_JACOBI_SWEEP_LOG: 1 = the single-CTA Jacobi SVT launches of
 *   tsvt_dct, tnn_complete and tnn_admm_iterate on ctx record, per slice and
 *   sweep, the counts and largest rotations that drive the stopping rules
 *   (read with tnn_last_sweep_log; the buffer is device memory the context
 *   allocates); 0 (default) = no log.  A tracing aid: the log costs a
 *   device clear per launch.
 * Returns TNN_EINVAL for an unknown option or a value out of range. */
#define TNN_OPT_JACOBI_MAX_SWEEPS 1
#define TNN_OPT_TC_WAIT_POLLS 2
#define TNN_OPT_JACOBI_FP64_ANGLES 3
#define TNN_OPT_ADMM_WARM_START 4
#define TNN_OPT_JACOBI_SMALL_STOP 5
#define TNN_OPT_JACOBI_SWEEP_LOG 6
tnn_status tnn_set_option(tnn_ctx* ctx, int option, int64_t value);

enum { TNN_OP_TDCT3 = 0, TNN_OP_TSVT = 1, TNN_OP_TSVD = 2, TNN_OP_TPROD = 3, TNN_OP_COMPLETE = 4 };

/* Device workspace `op` needs for `shape` at `prec` with device buffers (host
 * buffers add their staging).  For TNN_OP_TPROD the shape is (m1, m2, m3) and
 * m4 = m2 is assumed; pass the largest of m2, m4 as n2 for a bound. */
tnn_status tnn_workspace_size(tnn_ctx* ctx, int op, tnn_shape shape, tnn_precision prec, size_t* bytes);

/* Tube transform (Section 3; Algorithm 1).
 *   inverse = 0, scaled = 0:  Y = dct(X,[],3)
 *   inverse = 1, scaled = 0:  Y = idct(X,[],3)
 *   inverse = 0, scaled = 1:  Y = L(X)
 *   inverse = 1, scaled = 1:  Y = L^-1(X)
 * X and Y are n1 x n2 x n3; Y must not overlap X. */
tnn_status tdct3(tnn_ctx* ctx, const void* X, tnn_shape shape, int inverse, int scaled,
                 tnn_precision prec, void* Y, void* stream);

/* Tensor singular value thresholding (Theorem 5, as Algorithm 1 computes it):
 *   Zbar = dct(Z,[],3);  for every frontal slice k, Zbar_k = U S V^T (SVD)
 *   and Ybar_k = U (S - tau)_+ V^T;  Y = idct(Ybar,[],3).
 * Y is the proximal point of tau * sum_k ||dct(.)_k||_* at Z.  Z and Y are
 * n1 x n2 x n3 and may be the same buffer.  tau >= 0.  If tnn_out is not
 * NULL it receives sum_k ||Ybar_k||_* (the slice nuclear norms, without the
 * 1/n3 of the TNN-C definition, Eq. 16) and the call synchronises. */
tnn_status tsvt_dct(tnn_ctx* ctx, const void* Z, tnn_shape shape, double tau, tnn_precision prec,
                    void* Y, double* tnn_out, void* stream);

/* Thin DCT-based t-SVD (Theorem 4), r = min(n1, n2):  X = U * S * V^T under
 * the t-product of Eq. 13, with U (n1 x r x n3) and V (n2 x r x n3)
 * orthogonal in the sense U^T * U = V^T * V = I (identity tensor) and S
 * f-diagonal (Definition 4).  S is returned as its r x n3 diagonal tubes:
 * S(i,i,k) = S[i + r*k].  Computed as the SVD of every frontal slice of L(X)
 * (singular values in descending order per slice) mapped back by L^-1. */
tnn_status tsvd_dct_forward(tnn_ctx* ctx, const void* X, tnn_shape shape, tnn_precision prec,
                            void* U, void* S, void* V, void* stream);

/* Inverse of tsvd_dct_forward: X = U * S * V^T (Eq. 13 t-products) for U
 * (n1 x r x n3), S (r x n3 diagonal tubes), V (n2 x r x n3), r = min(n1, n2). */
tnn_status tsvd_dct_inverse(tnn_ctx* ctx, const void* U, const void* S, const void* V, tnn_shape shape,
                            tnn_precision prec, void* X, void* stream);

/* DCT-based t-product (Definition 7, Eq. 13): Z = X * Y = fold(btph(A) unfold(Y))
 * for X (m1 x m2 x m3) and Y (m2 x m4 x m3); Z is m1 x m4 x m3.  Computed
 * facewise in the transform domain (Eq. 14): L(Z)_k = L(X)_k L(Y)_k.
 * Z must not overlap X or Y. */
tnn_status tprod_dct(tnn_ctx* ctx, const void* X, const void* Y, int64_t m1, int64_t m2, int64_t m4,
                     int64_t m3, tnn_precision prec, void* Z, void* stream);

/* Algorithm 1: ADMM for the completion model (Eq. 17) from X = B on the
 * mask, M = 0, beta = beta0.  B (n1 x n2 x n3, a full-size buffer) may be
 * read everywhere but its values off the mask never affect the result.
 * mask is n1*n2*n3 bytes in the tensor's layout (nonzero = observed).
 * X_out receives the recovered tensor and may be the same buffer as B.
 * rep (may be NULL) receives the run's report.  Synchronises the stream.
 * Returns TNN_ENOCONV if max_iter was reached before the tol test passed.
 * The FP32 precisions warm-start each iteration's per-slice Jacobi from the
 * previous iteration's right singular vectors (see tnn_admm_warm_size); the
 * orthogonalisation of those vectors runs on a stream the context owns,
 * ordered after the iteration's work and before the next one's by events,
 * and joined back to `stream` before the call returns. */
tnn_status tnn_complete(tnn_ctx* ctx, const void* B, const uint8_t* mask, tnn_shape shape,
                        const tnn_admm_params* params, tnn_precision prec, void* X_out,
                        tnn_admm_report* rep, void* stream);

/* Run up to `iters` iterations of Algorithm 1 from a caller-held state:
 * X and M (n1 x n2 x n3, device or host, updated in place), *beta (host,
 * updated) and, optionally, the warm-start state `warm` (NULL: none).  The
 * iteration counter starts from 0 for this call; params->tol and
 * params->max_iter still stop the run (max_iter counts iterations of this
 * call).  A run split over several calls computes exactly what one call
 * does (checkpoint and resume; the same warm buffer is part of the state).
 * rep may be NULL.  Synchronises the stream.  Returns TNN_OK when all
 * requested iterations ran or tol was met.
 *
 * warm: a device buffer of tnn_admm_warm_size bytes, zero-filled before the
 * job's first iteration, then left to the library, which keeps there each
 * slice's right singular vectors (an orthogonal n x n matrix Q per slice,
 * n = min(n1, n2)) from the last iteration that rotated it.  One-sided
 * Jacobi on A Q has the singular values and left singular vectors of A, so
 * the SVT (rebuilt from A) does not depend on Q up to rounding; a Q from the
 * previous iteration makes the columns of A Q nearly orthogonal and cuts the
 * sweeps severalfold late in a completion.  Any orthogonal Q is correct, so
 * a zero-filled or stale buffer only costs sweeps.  Used by the FP32
 * precisions for slices one CTA holds; otherwise not touched.  Within a call
 * the buffer briefly holds the unorthogonalised vectors (the context's side
 * stream turns them into Q); the call joins that stream back to `stream`
 * before it returns, so between calls the buffer always holds Q. */
tnn_status tnn_admm_iterate(tnn_ctx* ctx, const void* B, const uint8_t* mask, tnn_shape shape,
                            const tnn_admm_params* params, tnn_precision prec, void* X, void* M,
                            double* beta, int32_t iters, void* warm, tnn_admm_report* rep, void* stream);

/* Host only: bytes of the warm-start state of tnn_admm_iterate for this
 * shape and precision; 0 when the precision or slice size does not use it
 * (FP64, or slices spread over thread-block clusters). */
tnn_status tnn_admm_warm_size(tnn_shape shape, tnn_precision prec, size_t* bytes);

/* Kernel statistics of the last tsvt_dct / tsvd_dct_forward / ADMM iteration
 * on ctx: out[0] = slices, out[1] = column pairs visited, out[2] = rotations
 * applied, out[3] = most sweeps of any slice, out[4] = slices that hit the
 * sweep cap, out[5] = singular values kept (above tau) over all slices.
 * For the SVT, a slice whose Frobenius norm is below tau runs no sweep, a
 * slice whose top singular value is certified below tau stops after the
 * sweep that certified it, and pairs of small columns left unrotated are
 * still counted as visited (their dot products are computed).
 * Synchronises the last stream used. */
tnn_status tnn_last_jacobi_stats(tnn_ctx* ctx, int64_t out[6]);

/* Per-slice statistics of the same launch as tnn_last_jacobi_stats: for each
 * slice k < min(n, slices), sweeps[k] (sweeps run), kept[k] (singular values
 * above tau) and rotations[k] (rotations applied).  Host arrays of n
 * entries, any of them NULL to skip it; entries k >= slices are left alone.
 * TNN_EINVAL for a null ctx or n < 0; all zero-work (nothing written) when
 * no Jacobi launch has run on ctx.  Synchronises the last stream used. */
tnn_status tnn_last_slice_stats(tnn_ctx* ctx, int64_t n, int32_t* sweeps, int32_t* kept, int64_t* rotations);

/* The per-sweep log of the last Jacobi launch on ctx, recorded when
 * TNN_OPT_JACOBI_SWEEP_LOG was 1 for it: for each slice k < min(n, slices),
 * nine rows of eight floats at out[(k * 9 + row) * 8 ...].  Row s < 8 is
 * sweep s: its big rotations (|gamma| > 2 tol sqrt(alpha beta)), its wide
 * rotations (those that block the small-rotation stop), its big rotations
 * between two columns below tau, the largest |gamma| / sqrt(alpha beta) of
 * its big rotations, the largest |t| of its big rotations and of all its
 * rotations, the sweep's SM clock cycles and those of the stopping tests
 * after it (certificates included); all zero for sweeps not run.  Row 8 is
 * the slice's cycles in the load (start columns and norms), the sweeps, the
 * tail (singular values, recovery or record, rebuild) and in all.  Slices
 * spread over a cluster keep no log.  out is a host array of n * 72 floats.
 * TNN_EINVAL if the last launch kept no log.  Synchronises the last stream
 * used. */
tnn_status tnn_last_sweep_log(tnn_ctx* ctx, int64_t n, float* out);

/* tsvt_dct without a context and without any device allocation (no
 * counterpart in the paper).  For callers that cannot allocate device memory
 * when they need a t-SVT: a serving loop bound to a fixed memory budget owned
 * by another allocator, code that must not create a context of its own, or a
 * thread that may not wait on the allocator's implicit synchronisation.
 * Computes what tsvt_dct computes for the same precision, with the same
 * kernels (the tensor-core transforms for TNN_FP32_TF32X3 and
 * TNN_FP32_BF16SPLIT, the CUDA-core ones for TNN_FP32 and TNN_FP64), without
 * tnn_out.  Z and Y must be device pointers of the current device (or
 * managed memory); Y may be Z; anything else returns TNN_EINVAL.
 * Scratch: one file-scope device array of TNN_STATIC_SCRATCH_BYTES that every
 * GPU loading the library holds until the process exits.  The call needs
 * 256 bytes + the two DCT operators (2 n3^2 elements, or the tensor-core
 * images of them) + n1 n2 n3 elements + 32 n3 bytes (each part rounded up to
 * 256 bytes), plus the Jacobi working copies when a frontal slice does not
 * fit in shared memory; a larger problem (or a size whose byte count would
 * not fit in size_t) returns TNN_EINVAL before anything is launched (at most
 * about 4.1e6 float or 2.0e6 double elements when the slices fit in shared
 * memory).  The first call on a device looks the array's device address up
 * with cudaGetSymbolAddress (device current); make that first call before
 * any stream capture.  All calls share the array and the call writes every
 * scratch byte it reads, so nothing carries over from an earlier call; calls
 * whose GPU work overlaps (other streams, other threads) race on the scratch
 * and must be ordered by the caller.  The call synchronises the stream at
 * the end and returns TNN_ENOCONV when a slice's Jacobi SVD hit its sweep
 * cap, TNN_ENONFINITE when a NaN or infinity was met (Y is written in both
 * cases) and TNN_ECUDA when a tensor-core transform timed out. */
#define TNN_STATIC_SCRATCH_BYTES ((size_t)16 << 20)
tnn_status tsvt_dct_static(const void* Z, tnn_shape shape, double tau, tnn_precision prec, void* Y, void* stream);

/* The DFT comparison path (Section 2: the t-SVD of Kilmer and Martin that
 * the paper compares against).  tsvt_dft is the proximal operator of
 * tau * TNN-F (Definition 6): Y = ifft(SVT_tau(fft(Z))) along the tubes,
 * each DFT slice shrunk by tau; for real Z only the slices
 * k = 0..floor(n3/2) are computed (the others are their conjugates) and Y is
 * real.  *tnn_out (may be NULL) receives TNN-F(Y).  tsvt_dct_plain is the
 * DCT t-SVT of tsvt_dct computed with the same plain per-slice Jacobi kernel
 * as tsvt_dft (one warp per column pair), so that the two differ only in the
 * transform and the arithmetic it implies (real against complex slices):
 * the pair measures the paper's DCT-against-DFT cost comparison (Table 2).
 * Device pointers only (TNN_EINVAL otherwise); Y may alias Z; slices up to
 * 512 x 512; TNN_FP64 runs in FP64, every other precision in plain FP32.
 * Synchronises the stream only when tnn_out is requested. */
tnn_status tsvt_dft(tnn_ctx* ctx, const void* Z, tnn_shape shape, double tau, tnn_precision prec, void* Y,
                    double* tnn_out, void* stream);
tnn_status tsvt_dct_plain(tnn_ctx* ctx, const void* Z, tnn_shape shape, double tau, tnn_precision prec, void* Y,
                          double* tnn_out, void* stream);

/* Batched t-SVT: one t-SVT (as tsvt_dct) for each of `count` tensors of
 * different shapes, with the slices of all tensors in the same launches.
 * A plan is built once for fixed device buffers (items[i].Z in, items[i].Y
 * out, may be the same buffer; shapes; thresholds tau >= 0) and then run any
 * number of times on the buffers' current contents.  The plan owns device
 * memory for the transformed tensors and its launch tables (allocated here,
 * freed by tnn_tsvt_batch_destroy).  A run launches, on one stream, the
 * forward tube transforms of all tensors (one grid), one Jacobi SVT launch
 * per group of slices sharing a kernel variant and residency (one CTA per
 * slice, or one thread-block cluster per slice too large for one CTA; the
 * groups on parallel streams), and the inverse transforms;
 * with TNN_BATCH_GRAPH the sequence is recorded once as a CUDA graph and a
 * run is a single graph launch.  With TNN_BATCH_AUTOTUNE the plan times
 * every compiled Jacobi variant that covers a group on its own data when it
 * is created and keeps the fastest (cached per shape class for the process).
 * Precisions: TNN_FP64 and TNN_FP32 (the tensor-core forms TNN_FP32_TF32X3
 * and TNN_FP32_BF16SPLIT run as TNN_FP32 here).
 * Host pointers are rejected (TNN_EINVAL).  Creation synchronises `stream`
 * and writes no item buffer; runs are stream-ordered and must not overlap one
 * another (they share the plan's buffers).  Slices are 512 x 512 at most. */
typedef struct {
    const void* Z;
    void* Y;
    tnn_shape shape;
    double tau;
} tnn_tsvt_item;
typedef struct tnn_tsvt_batch tnn_tsvt_batch;
#define TNN_BATCH_GRAPH 1
#define TNN_BATCH_AUTOTUNE 2
tnn_status tnn_tsvt_batch_create(tnn_ctx* ctx, const tnn_tsvt_item* items, int32_t count, tnn_precision prec,
                                 int32_t flags, void* stream, tnn_tsvt_batch** plan);
tnn_status tnn_tsvt_batch_run(tnn_tsvt_batch* plan, void* stream);
/* out[0] = Jacobi launch groups, out[1] = launches per run (1 with a graph),
 * out[2] = slices, out[3] = 1 if runs replay a CUDA graph. */
tnn_status tnn_tsvt_batch_info(const tnn_tsvt_batch* plan, int32_t out[4]);
/* Group g (0 <= g < groups): out = {L, R, K, slices, 1 if the working
 * copies are in shared memory, largest m}; (L, R, K) names the Jacobi
 * variant (L lanes per column-block pair, R rows per lane, K columns per
 * block).  Slices too large for one CTA are spread over thread-block
 * clusters (their group reports in_smem = 1 + cluster size). */
tnn_status tnn_tsvt_batch_group(const tnn_tsvt_batch* plan, int32_t g, int32_t out[6]);
/* One run without the graph, every launch in order on `stream` with CUDA
 * events between them; ms[0] = forward transforms, ms[1 + g] = group g's
 * Jacobi launch, ms[groups + 1] = inverse transforms (groups + 2 values).
 * Synchronises `stream`; writes the item outputs like a run. */
tnn_status tnn_tsvt_batch_profile(tnn_tsvt_batch* plan, void* stream, double* ms);
/* Synchronises `stream`, then sums the statistics of the last run:
 * out = {slices that hit the sweep cap, slices with a NaN/Inf, rotations,
 * most sweeps of a slice}.  Returns TNN_ENONFINITE if out[1] > 0. */
tnn_status tnn_tsvt_batch_stats(tnn_tsvt_batch* plan, void* stream, int64_t out[4]);
void tnn_tsvt_batch_destroy(tnn_tsvt_batch* plan);

/* Batched ADMM: Algorithm 1 for many completion problems of different
 * shapes at once, each iteration of all of them one launch sequence (one
 * CUDA-graph launch with TNN_BATCH_GRAPH): the forward transforms with the
 * Z = X - M/beta prologue of every tensor (one grid), the per-slice Jacobi
 * SVTs of all tensors (one launch per group of slices sharing a kernel
 * variant and residency, threshold 1/beta from each job's control block),
 * the inverse transforms with the fused X/M update (one grid) and every
 * job's stop test and beta update.  Each job computes exactly what
 * tnn_complete computes for it alone with TNN_FP32 (or TNN_FP64) transforms,
 * iterate for iterate, and a job that has stopped is skipped.  Items: device
 * buffers B, mask (as tnn_complete), X and M (n1 x n2 x n3, the job's state,
 * owned by the caller and updated in place); one parameter set for all jobs.
 * Create initialises X = B on the mask, M = 0 and the control blocks (as
 * tnn_admm_batch_reset does) and synchronises `stream`.  step queues `iters`
 * iterations (stream-ordered, no host wait); sync waits for them and gives
 * the number of jobs still running; run steps in growing chunks until every
 * job stopped or max_iter; report reads job i's state after a sync (returns
 * TNN_ENOCONV for a job that stopped on max_iter).  TNN_FP32_TF32X3 and
 * TNN_FP32_BF16SPLIT run as TNN_FP32 here.  The plan owns the transformed
 * tensors, partial sums, statistics, control blocks and launch tables. */
typedef struct {
    const void* B;
    const uint8_t* mask;
    void* X;
    void* M;
    tnn_shape shape;
} tnn_admm_item;
typedef struct tnn_admm_batch tnn_admm_batch;
tnn_status tnn_admm_batch_create(tnn_ctx* ctx, const tnn_admm_item* items, int32_t count,
                                 const tnn_admm_params* params, tnn_precision prec, int32_t flags, void* stream,
                                 tnn_admm_batch** plan);
tnn_status tnn_admm_batch_reset(tnn_admm_batch* plan, void* stream);
tnn_status tnn_admm_batch_step(tnn_admm_batch* plan, int32_t iters, void* stream);
tnn_status tnn_admm_batch_sync(tnn_admm_batch* plan, void* stream, int32_t* running);
tnn_status tnn_admm_batch_run(tnn_admm_batch* plan, void* stream);
tnn_status tnn_admm_batch_report(const tnn_admm_batch* plan, int32_t job, tnn_admm_report* rep);
void tnn_admm_batch_destroy(tnn_admm_batch* plan);

/* Completion server (no counterpart in the paper: the serving layer around
 * Algorithm 1).  A job is a completion problem with tnn_complete's
 * arguments.  Queued jobs are admitted in submission order while the device
 * footprint of the admitted ones stays within hbm_cap_bytes (and at most
 * max_active run), or least estimated work first; an admitted job keeps B, the mask, X, M, the transformed
 * tensor and its control block (beta, iteration, stop test) resident on the
 * device until its result is taken.  Each tnn_server_step retires the jobs
 * that stopped (stop test or max_iter), admits what now fits, and queues the
 * next `chunk` iterations of every running job; jobs are spread over
 * `streams` CUDA streams so their kernels overlap, and a step never waits on
 * the GPU.  A job runs exactly tnn_complete's kernels on its own buffers, so
 * its result does not depend on what else is running.  With
 * TNN_SERVER_BATCH_KERNELS in flags, the running FP32 and FP64 jobs (CUDA-core
 * transforms) run batched instead: per precision, one launch sequence per
 * iteration covers all of them (the kernels of tnn_admm_batch, tables
 * rebuilt whenever a job joins or leaves), on one extra stream per
 * precision; each job still gets the iterates it would get alone, bit for
 * bit, and jobs with another jacobi_max_sweeps than the first running one
 * wait for a later pass.  The tables and Jacobi scratch of a batch count
 * towards the footprint.  Not thread-safe: one host thread drives a
 * server. */
#define TNN_SERVER_FIFO 0           /* admit in submission order */
#define TNN_SERVER_SHORTEST_FIRST 1 /* admit the least estimated work first (iterations x n3 x m n^2) */
#define TNN_SERVER_BATCH_KERNELS 1  /* flags: batched iterations for FP32 and FP64 jobs */
typedef struct {
    uint64_t hbm_cap_bytes; /* 0: 150e9 */
    int32_t max_active;     /* 0: no limit beyond the footprint cap */
    int32_t streams;        /* 0: 8 */
    int32_t chunk;          /* iterations queued per job per step; 0: 8 */
    int32_t device;
    int32_t policy;         /* TNN_SERVER_FIFO or TNN_SERVER_SHORTEST_FIRST */
    int32_t flags;          /* 0 or TNN_SERVER_BATCH_KERNELS; other bits: TNN_EINVAL */
} tnn_server_params;
typedef struct tnn_server tnn_server;
tnn_status tnn_server_create(const tnn_server_params* params, tnn_server** server);
/* Host only: the device bytes a job of this shape and precision holds while
 * admitted (B, mask, X, M, the transformed tensor, partial sums, Jacobi
 * statistics and scratch, control block; each 256-byte aligned), the figure
 * admission compares with hbm_cap_bytes.  TNN_EINVAL for a null pointer, an
 * unknown precision, a non-positive extent or slices too large to plan. */
tnn_status tnn_server_footprint(tnn_shape shape, tnn_precision prec, uint64_t* bytes);
/* B (FP64 for TNN_FP64, else FP32) and mask (uint8, 1 = observed): pageable
 * host memory is copied at submission (into pinned memory the job owns);
 * pinned host or device memory is read at admission and must stay valid and
 * unchanged until then (state 1).  TNN_EINVAL if the job could never fit
 * the cap or its slices are too large. */
tnn_status tnn_server_submit(tnn_server* server, const void* B, const uint8_t* mask, tnn_shape shape,
                             const tnn_admm_params* params, tnn_precision prec, int64_t* job_id);
/* *finished = jobs that finished (or failed) in this pass (may be NULL). */
tnn_status tnn_server_step(tnn_server* server, int32_t* finished);
/* *state: 0 queued, 1 running, 2 finished (result waiting), 3 failed. */
tnn_status tnn_server_job_state(tnn_server* server, int64_t job_id, int32_t* state);
/* For a finished or failed job: copies X (host or device X_out, may be NULL),
 * fills the report and times = {submitted, admitted, finished} in seconds
 * since the server was created (either may be NULL), frees the job and
 * returns its status (TNN_OK, TNN_ENOCONV, TNN_ENONFINITE, ...).  TNN_EINVAL
 * while the job is still queued or running. */
tnn_status tnn_server_take(tnn_server* server, int64_t job_id, void* X_out, tnn_admm_report* rep, double times[3]);
/* out = {queued, running, finished not yet taken, device bytes admitted,
 * peak device bytes admitted, jobs finished so far}. */
tnn_status tnn_server_stats(const tnn_server* server, int64_t out[6]);
void tnn_server_destroy(tnn_server* server);

/* Tracing (no counterpart in the paper).  While enabled, every kernel a call
 * launches is bracketed by two CUDA events on the call's stream.
 * tnn_profile_read synchronises on those events, returns per kernel kind the
 * summed device time (ms) and the launch count since the last read, and
 * clears the record.  Kinds (array index):
 *   0 tube transform            1 forward transform + ADMM prologue
 *   2 Jacobi SVT                3 inverse transform + ADMM epilogue
 *   4 ADMM iteration finalize   5 ADMM control init
 *   6 ADMM state init           7 Jacobi SVD
 *   8 facewise product          9 DFT / rectangular tube transform
 *  10 plain Jacobi SVT (comparison path)
 *  11 warm start of the Jacobi SVT (A Q before it, Q after it)
 *  12 tail of the warm-started SVT (recovered vectors and rebuild) */
#define TNN_NKERNELS 13
tnn_status tnn_profile(tnn_ctx* ctx, int enable);
tnn_status tnn_profile_read(tnn_ctx* ctx, double ms[TNN_NKERNELS], int64_t launches[TNN_NKERNELS]);

/* Host only (no device needed): the Jacobi SVT launch the library plans for
 * the slices of a tensor of this shape and precision (one-sided Jacobi,
 * Algorithm 1's per-slice SVD).  out = {L lanes per column-block pair, R rows
 * per lane, K columns per block, nb column blocks (after padding), W warps per
 * CTA, 1 if a slice's working copy is in shared memory, cluster size (1: one
 * CTA per slice; > 1: each slice spread over a thread-block cluster), dynamic
 * shared memory bytes per CTA, global scratch bytes for the tensor}.  Honours
 * the same tuning overrides as the launches.  TNN_EINVAL for a null out, an
 * unknown precision, a non-positive extent or max(n1, n2) > 512. */
tnn_status tnn_jacobi_plan_info(tnn_shape shape, tnn_precision prec, int64_t out[9]);

/* Measured peak of a CUDA-core FMA pipe on `device` (no counterpart in the
 * paper: the roofline denominator of the Jacobi kernels).  kind 0: FP32 FMA,
 * 1: packed FP32 FMA (fma.rn.f32x2, two per instruction), 2: FP64 FMA.
 * Runs eight independent FMA chains per thread on eight 256-thread blocks per
 * SM for a few milliseconds (10 timed launches after 3 warm-ups, CUDA events)
 * and writes the rate in flop/s (2 per FMA) to *flops_per_s.  Allocates and
 * frees a small device buffer; synchronises.  TNN_EINVAL for a null pointer
 * or an unknown kind, TNN_ECUDA on a CUDA error. */
tnn_status tnn_fma_peak(int32_t device, int32_t kind, double* flops_per_s);

#ifdef __cplusplus
}
#endif

#endif /* TNN_H */
