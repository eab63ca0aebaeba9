/*
 * FP64 CPU oracle for the DCT-based tensor SVD, t-product, t-SVT and TNN-C
 * completion of Xu, Zhao and Ng, "A Fast Algorithm for Cosine Transform Based
 * Tensor Singular Value Decomposition" (arXiv 1902.03070).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA library is checked against.  Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant generator with the CUDA path.
 *
 * Conventions (Section 2 of the paper, MATLAB indexing):
 *   - a third-order tensor X of size n1 x n2 x n3 is stored column-major,
 *     x[i + n1*(j + n2*k)], so the frontal slice X^(k) = X(:,:,k) is a
 *     contiguous column-major n1 x n2 matrix and the tube X(i,j,:) has stride
 *     n1*n2;
 *   - matrices are column-major, a[i + m*j].
 *
 * Everything is IEEE double.  No blocking, fusion or reordering beyond what the
 * definitions state: each function writes out the definition it cites.
 *
 * Parity status of each function (what pins it, see tests/test_oracle_*.py):
 *   or_dct_matrix          pinned: orthogonality, scipy DCT-II (ortho), Example 1
 *   or_tube_transform      pinned: scipy DCT along axis 2, Example 1, Theorem 3
 *   or_btph                pinned: Example 1 printed matrix, Theorem 3 brute force
 *   or_tprod_btph          pinned: Eq. 13 vs Eq. 14 (two independent routes)
 *   or_tprod               pinned: Eq. 13 vs Eq. 14, identity tensor is the unit
 *   or_jacobi_svd          pinned: LAPACK singular values, orthogonality, A = U S V^T
 *   or_svt_matrix          pinned: prox optimality certificate, perturbation,
 *                                  tau = 0, tau >= sigma_max, rank-1 closed form
 *   or_tsvt                pinned: as or_svt_matrix plus n3 = 1 reduction
 *   or_tsvd                pinned: X = U*S*V^T, U^T*U = I, f-diagonal S
 *   or_admm                pinned: invariants X_Omega = B_Omega and
 *                                  M_{Omega^c} = 0 (bit-exact), full observation,
 *                                  exact recovery of a low-tubal-rank tensor
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef int64_t i64;

static double or_pi(void) { return acos(-1.0); }

/* ------------------------------------------------------------------------ */
/* DCT matrix.  The paper's transform is MATLAB's dct (Section 3, used in    */
/* Algorithm 1), the orthonormal DCT-II:                                      */
/*   C[k,j] = a_k cos(pi (2j+1) k / (2 n)),  a_0 = sqrt(1/n), a_k = sqrt(2/n). */
/* Column-major: C[k + n*j].                                                  */
/* ------------------------------------------------------------------------ */
void or_dct_matrix(i64 n, double* C)
{
    const double pi = or_pi();
    for (i64 k = 0; k < n; ++k) {
        double a = (k == 0) ? sqrt(1.0 / (double)n) : sqrt(2.0 / (double)n);
        for (i64 j = 0; j < n; ++j)
            C[k + n * j] = a * cos(pi * (double)(2 * j + 1) * (double)k / (2.0 * (double)n));
    }
}

/* ------------------------------------------------------------------------ */
/* Transform along the tubes (mode 3).                                       */
/*   inverse = 0: Y(:,:,k) = sum_j C[k,j] X(:,:,j)      (dct(X,[],3))         */
/*   inverse = 1: Y(:,:,j) = sum_k C[k,j] X(:,:,k)      (idct(X,[],3); C^-1 = C^T) */
/* scaled = 1 selects the transform L that makes Theorem 3 and Example 1     */
/* hold as printed: L(X)_k = dct(X)_k / w_k with w = C e_1 (first column of C), */
/* and L^-1(Y) = idct(w .* Y).  w_k > 0 for every k < n3.                     */
/* ------------------------------------------------------------------------ */
void or_tube_transform(i64 n1, i64 n2, i64 n3, const double* X, int inverse, int scaled, double* Y)
{
    const i64 P = n1 * n2;
    double* C = (double*)malloc(sizeof(double) * (size_t)(n3 * n3));
    or_dct_matrix(n3, C);
    for (i64 p = 0; p < P; ++p) {
        for (i64 q = 0; q < n3; ++q) {
            double s = 0.0;
            if (!inverse) {
                /* output frequency q, input position j */
                for (i64 j = 0; j < n3; ++j) s += C[q + n3 * j] * X[p + P * j];
                if (scaled) s /= C[q + n3 * 0];
            } else {
                /* output position q, input frequency k */
                for (i64 k = 0; k < n3; ++k) {
                    double xv = X[p + P * k];
                    if (scaled) xv *= C[k + n3 * 0];
                    s += C[k + n3 * q] * xv;
                }
            }
            Y[p + P * q] = s;
        }
    }
    free(C);
}

/* ------------------------------------------------------------------------ */
/* Block Toeplitz-plus-Hankel matrix btph(A) of Section 3 (Eqs. 9-11), with  */
/* X = A + sigma(A):  A^(m3) = X^(m3),  A^(k) = X^(k) - A^(k+1).              */
/* With 1-based block indices r, c in 1..m3:                                  */
/*   bt block (r,c) = A^(|r-c|+1)                                   (Eq. 9)   */
/*   bh block (r,c) = A^(r+c)        if r+c <= m3                             */
/*                  = O              if r+c == m3+1                           */
/*                  = A^(2m3+2-r-c)  otherwise                      (Eq. 10)  */
/* Output: dense (m1 m3) x (m2 m3) column-major matrix, row index i + m1*(r-1),*/
/* column index j + m2*(c-1).                                                 */
/* ------------------------------------------------------------------------ */
void or_btph(i64 m1, i64 m2, i64 m3, const double* X, double* out)
{
    const i64 S = m1 * m2;
    double* A = (double*)malloc(sizeof(double) * (size_t)(S * m3));
    /* shift decomposition, slices 1-based in the comments, 0-based here */
    for (i64 e = 0; e < S; ++e) A[e + S * (m3 - 1)] = X[e + S * (m3 - 1)];
    for (i64 k = m3 - 2; k >= 0; --k)
        for (i64 e = 0; e < S; ++e) A[e + S * k] = X[e + S * k] - A[e + S * (k + 1)];

    const i64 R = m1 * m3;
    memset(out, 0, sizeof(double) * (size_t)(R * m2 * m3));
    for (i64 r = 1; r <= m3; ++r) {
        for (i64 c = 1; c <= m3; ++c) {
            i64 bt = (r > c ? r - c : c - r) + 1; /* 1-based slice of A for bt */
            i64 s = r + c, bh;                     /* 1-based slice of A for bh, 0 = O */
            if (s <= m3) bh = s;
            else if (s == m3 + 1) bh = 0;
            else bh = 2 * m3 + 2 - s;
            for (i64 j = 0; j < m2; ++j) {
                for (i64 i = 0; i < m1; ++i) {
                    double v = A[i + m1 * j + S * (bt - 1)];
                    if (bh > 0) v += A[i + m1 * j + S * (bh - 1)];
                    out[(i + m1 * (r - 1)) + R * (j + m2 * (c - 1))] = v;
                }
            }
        }
    }
    free(A);
}

/* ------------------------------------------------------------------------ */
/* DCT-based t-product by its definition (Definition 7, Eq. 13):             */
/*   Z = fold(btph(A) * unfold(Y)),  X (m1 x m2 x m3), Y (m2 x m4 x m3).      */
/* unfold stacks the frontal slices vertically (Eq. 3).                       */
/* ------------------------------------------------------------------------ */
void or_tprod_btph(i64 m1, i64 m2, i64 m4, i64 m3, const double* X, const double* Y, double* Z)
{
    const i64 R = m1 * m3, K = m2 * m3;
    double* B = (double*)malloc(sizeof(double) * (size_t)(R * K));
    or_btph(m1, m2, m3, X, B);
    /* unfold(Y) is (m2 m3) x m4 with row j + m2*k, column l  <->  Y[j + m2*(l + m4*k)] */
    for (i64 l = 0; l < m4; ++l) {
        for (i64 row = 0; row < R; ++row) {
            double s = 0.0;
            for (i64 col = 0; col < K; ++col) {
                i64 j = col % m2, k = col / m2;
                s += B[row + R * col] * Y[j + m2 * (l + m4 * k)];
            }
            i64 i = row % m1, k = row / m1;
            Z[i + m1 * (l + m4 * k)] = s; /* fold back to m1 x m4 x m3 */
        }
    }
    free(B);
}

/* ------------------------------------------------------------------------ */
/* DCT-based t-product through the transform (Eq. 14): with the scaled       */
/* transform L of Theorem 3,  L(Z)_k = L(X)_k L(Y)_k  (facewise product).     */
/* ------------------------------------------------------------------------ */
void or_tprod(i64 m1, i64 m2, i64 m4, i64 m3, const double* X, const double* Y, double* Z)
{
    double* Xh = (double*)malloc(sizeof(double) * (size_t)(m1 * m2 * m3));
    double* Yh = (double*)malloc(sizeof(double) * (size_t)(m2 * m4 * m3));
    double* Zh = (double*)malloc(sizeof(double) * (size_t)(m1 * m4 * m3));
    or_tube_transform(m1, m2, m3, X, 0, 1, Xh);
    or_tube_transform(m2, m4, m3, Y, 0, 1, Yh);
    for (i64 k = 0; k < m3; ++k) {
        const double* a = Xh + m1 * m2 * k;
        const double* b = Yh + m2 * m4 * k;
        double* c = Zh + m1 * m4 * k;
        for (i64 l = 0; l < m4; ++l)
            for (i64 i = 0; i < m1; ++i) {
                double s = 0.0;
                for (i64 j = 0; j < m2; ++j) s += a[i + m1 * j] * b[j + m2 * l];
                c[i + m1 * l] = s;
            }
    }
    or_tube_transform(m1, m4, m3, Zh, 1, 1, Z);
    free(Xh); free(Yh); free(Zh);
}

/* ------------------------------------------------------------------------ */
/* One-sided (Hestenes) Jacobi SVD of an m x n matrix with m >= n, the SVD   */
/* the paper calls per frontal slice (Algorithm 1, Section 3 cost remark).   */
/* The method: J. Demmel and K. Veselic, "Jacobi's method is more accurate   */
/* than QR", SIAM J. Matrix Anal. Appl. 13 (1992); rotation formula of       */
/* Rutishauser.  Cyclic-by-rows pair order (i < j).  For each pair:          */
/*   alpha = |a_i|^2, beta = |a_j|^2, gamma = a_i . a_j ;                      */
/*   skip if |gamma| <= tol sqrt(alpha beta)  (tol = sqrt(m) * 2^-53);        */
/*   zeta = (beta - alpha) / (2 gamma), t = sign(zeta)/(|zeta| + sqrt(1+zeta^2)), */
/*   c = 1/sqrt(1+t^2), s = c t ;                                             */
/*   a_i <- c a_i - s a_j,  a_j <- s a_i + c a_j  (same on V).                */
/* Stops after a sweep without rotation or after max_sweeps sweeps.          */
/* Output: sigma (n, descending), U (m x n, u_i = a_i / sigma_i, zero column  */
/* if sigma_i == 0), V (n x n).  A is read with leading dimension lda.       */
/* Returns the number of sweeps run; *converged is 1 iff the last sweep made */
/* no rotation.                                                              */
/* ------------------------------------------------------------------------ */
int or_jacobi_svd(i64 m, i64 n, const double* A, i64 lda, double* sigma, double* U, double* V,
                  int max_sweeps, int* converged)
{
    double* W = (double*)malloc(sizeof(double) * (size_t)(m * n));
    double* Vw = (double*)malloc(sizeof(double) * (size_t)(n * n));
    for (i64 j = 0; j < n; ++j)
        for (i64 i = 0; i < m; ++i) W[i + m * j] = A[i + lda * j];
    for (i64 j = 0; j < n; ++j)
        for (i64 i = 0; i < n; ++i) Vw[i + n * j] = (i == j) ? 1.0 : 0.0;

    const double tol = sqrt((double)m) * ldexp(1.0, -53);
    int sweeps = 0, conv = 0;
    while (sweeps < max_sweeps) {
        ++sweeps;
        int rotated = 0;
        for (i64 i = 0; i < n - 1; ++i) {
            for (i64 j = i + 1; j < n; ++j) {
                double* ai = W + m * i;
                double* aj = W + m * j;
                double alpha = 0.0, beta = 0.0, gamma = 0.0;
                for (i64 r = 0; r < m; ++r) {
                    alpha += ai[r] * ai[r];
                    beta += aj[r] * aj[r];
                    gamma += ai[r] * aj[r];
                }
                if (!(fabs(gamma) > tol * sqrt(alpha * beta))) continue;
                double zeta = (beta - alpha) / (2.0 * gamma);
                double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double c = 1.0 / sqrt(1.0 + t * t);
                double s = c * t;
                for (i64 r = 0; r < m; ++r) {
                    double x = ai[r], y = aj[r];
                    ai[r] = c * x - s * y;
                    aj[r] = s * x + c * y;
                }
                double* vi = Vw + n * i;
                double* vj = Vw + n * j;
                for (i64 r = 0; r < n; ++r) {
                    double x = vi[r], y = vj[r];
                    vi[r] = c * x - s * y;
                    vj[r] = s * x + c * y;
                }
                rotated = 1;
            }
        }
        if (!rotated) { conv = 1; break; }
    }

    /* singular values are the column norms; order them descending */
    double* nrm = (double*)malloc(sizeof(double) * (size_t)n);
    i64* ord = (i64*)malloc(sizeof(i64) * (size_t)n);
    for (i64 j = 0; j < n; ++j) {
        double s = 0.0;
        for (i64 r = 0; r < m; ++r) s += W[r + m * j] * W[r + m * j];
        nrm[j] = sqrt(s);
        ord[j] = j;
    }
    for (i64 a = 1; a < n; ++a) { /* insertion sort, stable */
        i64 key = ord[a], b = a - 1;
        while (b >= 0 && nrm[ord[b]] < nrm[key]) { ord[b + 1] = ord[b]; --b; }
        ord[b + 1] = key;
    }
    for (i64 q = 0; q < n; ++q) {
        i64 j = ord[q];
        sigma[q] = nrm[j];
        for (i64 r = 0; r < m; ++r) U[r + m * q] = (nrm[j] > 0.0) ? W[r + m * j] / nrm[j] : 0.0;
        for (i64 r = 0; r < n; ++r) V[r + n * q] = Vw[r + n * j];
    }
    free(nrm); free(ord); free(W); free(Vw);
    if (converged) *converged = conv;
    return sweeps;
}

/* ------------------------------------------------------------------------ */
/* Matrix singular value thresholding (the per-slice part of Theorem 5 and   */
/* of Algorithm 1):  A = U S V^T,  Y = U (S - tau)_+ V^T.                     */
/* A is m x n with leading dimension lda; Y is m x n with leading dimension   */
/* ldy.  If m < n the SVD is taken of A^T and the factors swap roles.         */
/* Returns the sum of (sigma_i - tau)_+ (the nuclear norm of Y) in *nuc and   */
/* the sweep count; *converged as in or_jacobi_svd.                           */
/* ------------------------------------------------------------------------ */
int or_svt_matrix(i64 m, i64 n, const double* A, i64 lda, double tau, double* Y, i64 ldy,
                  double* nuc, int max_sweeps, int* converged)
{
    const int tr = (m < n);
    const i64 mm = tr ? n : m, nn = tr ? m : n; /* mm >= nn */
    double* At = (double*)malloc(sizeof(double) * (size_t)(mm * nn));
    for (i64 j = 0; j < nn; ++j)
        for (i64 i = 0; i < mm; ++i) At[i + mm * j] = tr ? A[j + lda * i] : A[i + lda * j];
    double* sg = (double*)malloc(sizeof(double) * (size_t)nn);
    double* U = (double*)malloc(sizeof(double) * (size_t)(mm * nn));
    double* V = (double*)malloc(sizeof(double) * (size_t)(nn * nn));
    int sw = or_jacobi_svd(mm, nn, At, mm, sg, U, V, max_sweeps, converged);
    double nsum = 0.0;
    for (i64 q = 0; q < nn; ++q) {
        double d = sg[q] - tau;
        sg[q] = d > 0.0 ? d : 0.0;
        nsum += sg[q];
    }
    /* Yt = U diag(d) V^T  (mm x nn); Y = Yt or Yt^T */
    for (i64 j = 0; j < nn; ++j)
        for (i64 i = 0; i < mm; ++i) {
            double s = 0.0;
            for (i64 q = 0; q < nn; ++q) s += U[i + mm * q] * sg[q] * V[j + nn * q];
            if (tr) Y[j + ldy * i] = s;
            else Y[i + ldy * j] = s;
        }
    if (nuc) *nuc = nsum;
    free(At); free(sg); free(U); free(V);
    return sw;
}

/* ------------------------------------------------------------------------ */
/* t-SVT, the proximal step of Theorem 5 as Algorithm 1 computes it:         */
/*   Zbar = dct(Z,[],3); per slice Ybar_k = U_k (S_k - tau)_+ V_k^T;           */
/*   Y = idct(Ybar,[],3).                                                     */
/* Output *tnn = sum_k ||Ybar_k||_*  (no 1/n3 factor).  nthreads > 1 runs the */
/* independent slices on OpenMP threads (no change to any arithmetic).       */
/* Returns the largest sweep count; *all_converged is 1 iff every slice      */
/* converged.                                                                */
/* ------------------------------------------------------------------------ */
int or_tsvt(i64 n1, i64 n2, i64 n3, const double* Z, double tau, double* Y, double* tnn,
            int max_sweeps, int nthreads, int* all_converged, int* sweeps_per_slice)
{
    const i64 S = n1 * n2;
    double* Zb = (double*)malloc(sizeof(double) * (size_t)(S * n3));
    double* Yb = (double*)malloc(sizeof(double) * (size_t)(S * n3));
    double* nuc = (double*)malloc(sizeof(double) * (size_t)n3);
    int* sw = (int*)malloc(sizeof(int) * (size_t)n3);
    int* cv = (int*)malloc(sizeof(int) * (size_t)n3);
    or_tube_transform(n1, n2, n3, Z, 0, 0, Zb);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (i64 k = 0; k < n3; ++k)
        sw[k] = or_svt_matrix(n1, n2, Zb + S * k, n1, tau, Yb + S * k, n1, &nuc[k], max_sweeps, &cv[k]);
    (void)nthreads;
    or_tube_transform(n1, n2, n3, Yb, 1, 0, Y);
    double t = 0.0;
    int swmax = 0, allc = 1;
    for (i64 k = 0; k < n3; ++k) {
        t += nuc[k];
        if (sw[k] > swmax) swmax = sw[k];
        if (!cv[k]) allc = 0;
        if (sweeps_per_slice) sweeps_per_slice[k] = sw[k];
    }
    if (tnn) *tnn = t;
    if (all_converged) *all_converged = allc;
    free(Zb); free(Yb); free(nuc); free(sw); free(cv);
    return swmax;
}

/* ------------------------------------------------------------------------ */
/* Thin DCT-based t-SVD (Theorem 4) with r = min(m1, m2):                    */
/*   L(X)_k = Uh_k Sh_k Vh_k^T  (SVD of each slice of the scaled transform),  */
/*   U = L^-1(Uh) (m1 x r x m3), V = L^-1(Vh) (m2 x r x m3),                  */
/*   S(i,i,:) = L^-1 of the tube of singular values, stored S[i + r*k].       */
/* Then X = U * S * V^T under the t-product of Eq. 13.                       */
/* ------------------------------------------------------------------------ */
int or_tsvd(i64 m1, i64 m2, i64 m3, const double* X, double* U, double* S, double* V,
            int max_sweeps, int nthreads)
{
    const i64 r = m1 < m2 ? m1 : m2;
    const i64 P = m1 * m2;
    double* Xh = (double*)malloc(sizeof(double) * (size_t)(P * m3));
    double* Uh = (double*)malloc(sizeof(double) * (size_t)(m1 * r * m3));
    double* Vh = (double*)malloc(sizeof(double) * (size_t)(m2 * r * m3));
    double* Sh = (double*)malloc(sizeof(double) * (size_t)(r * m3));
    int* sw = (int*)malloc(sizeof(int) * (size_t)m3);
    or_tube_transform(m1, m2, m3, X, 0, 1, Xh);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (i64 k = 0; k < m3; ++k) {
        const double* a = Xh + P * k;
        if (m1 >= m2) {
            /* columns of the slice: U is m1 x r, V is m2 x r */
            sw[k] = or_jacobi_svd(m1, m2, a, m1, Sh + r * k, Uh + m1 * r * k, Vh + m2 * r * k, max_sweeps, NULL);
        } else {
            /* SVD of the transpose: slice^T = U' S V'^T, so slice = V' S U'^T */
            double* at = (double*)malloc(sizeof(double) * (size_t)(m2 * m1));
            for (i64 j = 0; j < m1; ++j)
                for (i64 i = 0; i < m2; ++i) at[i + m2 * j] = a[j + m1 * i];
            sw[k] = or_jacobi_svd(m2, m1, at, m2, Sh + r * k, Vh + m2 * r * k, Uh + m1 * r * k, max_sweeps, NULL);
            free(at);
        }
    }
    (void)nthreads;
    or_tube_transform(m1, r, m3, Uh, 1, 1, U);
    or_tube_transform(m2, r, m3, Vh, 1, 1, V);
    or_tube_transform(r, 1, m3, Sh, 1, 1, S);
    int swmax = 0;
    for (i64 k = 0; k < m3; ++k) if (sw[k] > swmax) swmax = sw[k];
    free(Xh); free(Uh); free(Vh); free(Sh); free(sw);
    return swmax;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 (ADMM for the completion model, Eq. 17), with the penalty    */
/* schedule beta <- min(rho beta, beta_max) after each iteration (rho = 1    */
/* is the paper's fixed beta).  Per iteration l:                             */
/*   Z = X - M / beta                                                         */
/*   Y = t-SVT(Z, 1/beta)                                 (Theorem 5)         */
/*   X+ = (Y + M / beta) on the complement of Omega, B on Omega   (Eq. 25)   */
/*   M+ = M + beta (Y - X+)                                (Eq. 20, step 3)   */
/*   relchg = ||X+ - X||_F / ||X||_F  (absolute change if ||X||_F = 0)        */
/*   pres   = ||Y - X+||_F / ||X+||_F (the residual of the splitting Y = X    */
/*            of Eq. 19; absolute if ||X+||_F = 0)                            */
/*   beta <- min(rho beta, beta_max);  l <- l + 1                             */
/* until (relchg <= tol and pres <= tol) or l >= max_iter, at least one      */
/* iteration.  The paper's loop test has only relchg; alone it stops at the  */
/* first iteration whenever the first Y is 0 (1/beta above every singular    */
/* value), since X then does not move while M grows.  The residual of the    */
/* constraint Y = X is ADMM's primal residual.                                */
/* Init: X = B on Omega and 0 elsewhere, M = 0.  mask[e] != 0 marks Omega.   */
/* X (out) and M (out) are caller buffers of n1 n2 n3 doubles.               */
/* out[0] = iterations, out[1] = last relchg, out[2] = last pres,            */
/* out[3] = beta after the last update, out[4] = converged.                  */
/* ------------------------------------------------------------------------ */
void or_admm(i64 n1, i64 n2, i64 n3, const double* B, const uint8_t* mask, double beta0, double rho,
             double beta_max, double tol, int max_iter, int max_sweeps, int nthreads, int resume,
             double* X, double* M, double* out)
{
    const i64 N = n1 * n2 * n3;
    double* Z = (double*)malloc(sizeof(double) * (size_t)N);
    double* Y = (double*)malloc(sizeof(double) * (size_t)N);
    /* Algorithm 1 starts from X = B on the mask and M = 0; with resume set the
       iterations continue from the (X, M) passed in, beta0 being the beta the
       next iteration uses. */
    if (!resume)
        for (i64 e = 0; e < N; ++e) { X[e] = mask[e] ? B[e] : 0.0; M[e] = 0.0; }
    double beta = beta0, relchg = 0.0, pres = 0.0;
    int l = 0, conv = 0;
    for (;;) {
        for (i64 e = 0; e < N; ++e) Z[e] = X[e] - M[e] / beta;
        or_tsvt(n1, n2, n3, Z, 1.0 / beta, Y, NULL, max_sweeps, nthreads, NULL, NULL);
        double dx = 0.0, xx = 0.0, yx = 0.0, nx = 0.0;
        for (i64 e = 0; e < N; ++e) {
            double xn = mask[e] ? B[e] : Y[e] + M[e] / beta;
            double mn = M[e] + beta * (Y[e] - xn);
            dx += (xn - X[e]) * (xn - X[e]);
            xx += X[e] * X[e];
            yx += (Y[e] - xn) * (Y[e] - xn);
            nx += xn * xn;
            X[e] = xn;
            M[e] = mn;
        }
        relchg = (xx > 0.0) ? sqrt(dx) / sqrt(xx) : sqrt(dx);
        pres = (nx > 0.0) ? sqrt(yx) / sqrt(nx) : sqrt(yx);
        beta = (rho * beta < beta_max) ? rho * beta : beta_max;
        ++l;
        if (relchg <= tol && pres <= tol) { conv = 1; break; }
        if (l >= max_iter) break;
    }
    out[0] = (double)l;
    out[1] = relchg;
    out[2] = pres;
    out[3] = beta;
    out[4] = (double)conv;
    free(Z); free(Y);
}

/* Threads the OpenMP runtime grants for a request of nthreads. */
int or_threads(int nthreads)
{
#ifdef _OPENMP
    int got = 1;
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1)
    {
#pragma omp single
        got = omp_get_num_threads();
    }
    return got;
#else
    (void)nthreads;
    return 1;
#endif
}
