/*
 * Plain FP64 CPU oracle for ANLS-NMF with block principal pivoting (BPP).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path links, loads or calls
 * this file: it is used by tests/, by the smoke check and by the benchmark's
 * CPU-baseline leg. It shares no code with the CUDA library.
 *
 * Everything is written as the plain definition (or the algorithm's steps in
 * order), with naive loops in double precision and no blocking. OpenMP only
 * splits independent rows / right-hand sides across threads; every value is
 * computed by the same sequential loop whatever the thread count, so results
 * are bitwise reproducible.
 *
 * Paper: Kannan, Ballard, Park, "A High-Performance Parallel Algorithm for
 * Nonnegative Matrix Factorization" (arXiv 1509.09313).
 *   Eq. 1   f(W,H) = ||A - W H||_F^2, W >= 0 (m x k), H >= 0 (k x n).
 *   Eq. 2   the two-block alternating scheme (W first, then H).
 *   Alg. 1  ANLS: update W from (H H^T, A H^T), then H from (W^T W, W^T A).
 *   Eq. 3   the single right-hand-side NLS min_{x>=0} ||C x - b||_2^2.
 *   Eq. 4   its KKT conditions y = C^T C x - C^T b, y >= 0, x >= 0, x^T y = 0.
 *   Sec. 4.2 BPP: exchange indices between the active set (x_i = 0) and the
 *           passive set until the partition satisfies Eq. 4; passive values
 *           come from the normal equations restricted to the passive set. The
 *           exchange rules are those of the cited method (Kim, He and Park,
 *           SIAM J. Sci. Comput. 2011): full exchange of all infeasible
 *           indices while their count keeps dropping, up to three more full
 *           exchanges after it stops dropping, then single exchange of the
 *           largest infeasible index (the backup rule).
 *
 * Alternative local updates the paper names for the same two steps (Sec. 3):
 *   Eq. 5   MU: every entry of W scaled by (A H^T)_ij / (W H H^T)_ij, all from
 *           the iterate before the update; likewise H with (W^T A) and W^T W H.
 *   Eq. 6   HALS: column i of W (row i of H) replaced by
 *           [(A H^T)^i - sum_{l != i} (H H^T)_li w^l]_+ / (H H^T)_ii, the columns
 *           taken in order 1..k with the newest values of the others.
 *
 * Storage: A is float32 row-major (the stored input both paths read); W is
 * m x k row-major; H is kept as H^T, n x k row-major, so each right-hand side
 * of either half-step is one contiguous k-vector.
 *
 * Parity pins (tests/test_oracle_*.py): brute force over all 2^k partitions,
 * scipy's Lawson-Hanson NNLS, closed forms (k = 1, diagonal Gram, all-positive
 * unconstrained solution, non-positive RHS), KKT residuals of every solve,
 * numpy products, the non-increasing objective of exact block minimisation,
 * and planted exact recovery. Pivot-round counts have no printed value in the
 * paper: beyond the closed cases (0 rounds for g <= 0, 1 round when the
 * unconstrained solution is positive) they are parity unpinned.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum {
    OR_OK = 0,
    OR_NOT_CONVERGED = 4,
    OR_SINGULAR = 5,
};

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Gram of the rows of X (rows x k, row-major): G = X^T X, k x k.
 * With X = H^T this is H H^T; with X = W it is W^T W (Alg. 1). */
void oracle_gram(const double *X, int64_t rows, int k, double *G)
{
    for (int a = 0; a < k; ++a)
        for (int b = 0; b < k; ++b) {
            double s = 0.0;
            for (int64_t i = 0; i < rows; ++i)
                s += X[i * k + a] * X[i * k + b];
            G[a * k + b] = s;
        }
}

/* Dense products of Alg. 1 with A (m x n, float32 row-major, leading dim lda).
 * trans = 0: out (m x k) = A F with F = H^T (n x k): row i is sum_j A_ij h_j.
 * trans = 1: out (n x k) = A^T F with F = W (m x k): row j is sum_i A_ij w_i,
 *            i.e. the columns of W^T A stored as rows. */
void oracle_mm_dense(const float *A, int64_t m, int64_t n, int64_t lda,
                     const double *F, int k, int trans, double *out)
{
    if (trans == 0) {
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < m; ++i)
            for (int r = 0; r < k; ++r) {
                double s = 0.0;
                for (int64_t j = 0; j < n; ++j)
                    s += (double)A[i * lda + j] * F[j * k + r];
                out[i * k + r] = s;
            }
    } else {
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < n; ++j)
            for (int r = 0; r < k; ++r) {
                double s = 0.0;
                for (int64_t i = 0; i < m; ++i)
                    s += (double)A[i * lda + j] * F[i * k + r];
                out[j * k + r] = s;
            }
    }
}

/* Sparse (CSR) counterpart. trans = 0: out (m x k) = A F; trans = 1:
 * out (n x k) = A^T F, accumulated over the rows of A in index order. */
void oracle_mm_csr(const int64_t *rowptr, const int32_t *colidx, const float *vals,
                   int64_t m, int64_t n, const double *F, int k, int trans, double *out)
{
    if (trans == 0) {
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < m; ++i)
            for (int r = 0; r < k; ++r) {
                double s = 0.0;
                for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p)
                    s += (double)vals[p] * F[(int64_t)colidx[p] * k + r];
                out[i * k + r] = s;
            }
    } else {
        memset(out, 0, sizeof(double) * (size_t)n * (size_t)k);
        for (int64_t i = 0; i < m; ++i)
            for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p)
                for (int r = 0; r < k; ++r)
                    out[(int64_t)colidx[p] * k + r] += (double)vals[p] * F[i * k + r];
    }
}

/* Eq. 1, dense: sum over all (i, j) of (A_ij - w_i . h_j)^2. */
double oracle_objective_dense(const float *A, int64_t m, int64_t n, int64_t lda,
                              const double *W, const double *Ht, int k)
{
    double f = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : f)
    for (int64_t i = 0; i < m; ++i) {
        double fi = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double wh = 0.0;
            for (int r = 0; r < k; ++r)
                wh += W[i * k + r] * Ht[j * k + r];
            double d = (double)A[i * lda + j] - wh;
            fi += d * d;
        }
        f += fi;
    }
    return f;
}

/* Eq. 1, sparse A. Summing (A_ij - (WH)_ij)^2 over all m*n positions splits
 * exactly into the stored entries and the rest:
 *   f = sum_{(i,j) stored} (A_ij - (WH)_ij)^2 + sum_{(i,j) not stored} (WH)_ij^2
 *     = sum_{stored} [(A_ij - (WH)_ij)^2 - (WH)_ij^2] + ||W H||_F^2,
 * and ||W H||_F^2 = trace((W^T W)(H H^T)). All three in FP64. Pinned against the
 * all-positions sum on small matrices. */
double oracle_objective_csr(const int64_t *rowptr, const int32_t *colidx, const float *vals,
                            int64_t m, int64_t n, const double *W, const double *Ht, int k)
{
    double *GW = (double *)malloc(sizeof(double) * (size_t)k * (size_t)k);
    double *GH = (double *)malloc(sizeof(double) * (size_t)k * (size_t)k);
    oracle_gram(W, m, k, GW);
    oracle_gram(Ht, n, k, GH);
    double full = 0.0;
    for (int a = 0; a < k; ++a)
        for (int b = 0; b < k; ++b)
            full += GW[a * k + b] * GH[b * k + a];
    free(GW);
    free(GH);
    double stored = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : stored)
    for (int64_t i = 0; i < m; ++i) {
        double si = 0.0;
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            double wh = 0.0;
            for (int r = 0; r < k; ++r)
                wh += W[i * k + r] * Ht[(int64_t)colidx[p] * k + r];
            double d = (double)vals[p] - wh;
            si += d * d - wh * wh;
        }
        stored += si;
    }
    return stored + full;
}

/* ---------------------------------------------------------------------------
 * One NLS in normal-equations form (Eq. 3 with G = C^T C, g = C^T b):
 *   minimise 0.5 x^T G x - g^T x subject to x >= 0.
 * The partition (passive set F, active set = the rest) determines the
 * candidate point: x_F solves G_FF x_F = g_F, x = 0 off F; y = G x - g with
 * y_F = 0 (Eq. 4's y, since C^T C x - C^T b = G x - g).
 * ------------------------------------------------------------------------- */

/* Cholesky of the |F| x |F| principal submatrix and the two triangular solves.
 * L is p x p row-major scratch. Returns 0, or OR_SINGULAR on a pivot <= 0. */
static int solve_partition(const double *G, int k, const double *g, const uint8_t *F,
                           double *x, double *y, int *idx, double *L, double *z)
{
    int p = 0;
    for (int i = 0; i < k; ++i)
        if (F[i])
            idx[p++] = i;
    /* Cholesky G_FF = L L^T (row-oriented textbook form). */
    for (int a = 0; a < p; ++a) {
        for (int b = 0; b <= a; ++b) {
            double s = G[idx[a] * k + idx[b]];
            for (int c = 0; c < b; ++c)
                s -= L[a * p + c] * L[b * p + c];
            if (a == b) {
                if (!(s > 0.0))
                    return OR_SINGULAR;
                L[a * p + a] = sqrt(s);
            } else {
                L[a * p + b] = s / L[b * p + b];
            }
        }
    }
    /* L z = g_F, then L^T x_F = z. */
    for (int a = 0; a < p; ++a) {
        double s = g[idx[a]];
        for (int c = 0; c < a; ++c)
            s -= L[a * p + c] * z[c];
        z[a] = s / L[a * p + a];
    }
    for (int a = p - 1; a >= 0; --a) {
        double s = z[a];
        for (int c = a + 1; c < p; ++c)
            s -= L[c * p + a] * z[c];
        z[a] = s / L[a * p + a];
    }
    for (int i = 0; i < k; ++i)
        x[i] = 0.0;
    for (int a = 0; a < p; ++a)
        x[idx[a]] = z[a];
    /* y = G x - g off F, zero on F. */
    for (int i = 0; i < k; ++i) {
        if (F[i]) {
            y[i] = 0.0;
            continue;
        }
        double s = -g[i];
        for (int a = 0; a < p; ++a)
            s += G[i * k + idx[a]] * z[a];
        y[i] = s;
    }
    return OR_OK;
}

/* BPP for one right-hand side (Sec. 4.2 and the cited method).
 * F (k bytes) holds the starting passive set when warm != 0 and receives the
 * final one. Indices with G_ii <= 0 (a zero row of the factor, so G_i* = 0 and
 * g_i = 0 for data-derived problems) can never be passive: they stay active at
 * x_i = 0 and are never counted as infeasible.
 * Returns the status; *rounds = number of exchange-and-solve steps. */
static int bpp_one(const double *G, int k, const double *g, double *x, uint8_t *F,
                   int warm, int max_rounds, int *rounds, double *work, int *idx)
{
    double *y = work;
    double *z = y + k;
    double *L = z + k;
    uint8_t usable[1024];
    for (int i = 0; i < k; ++i) {
        usable[i] = G[i * k + i] > 0.0;
        F[i] = (warm && F[i] && usable[i]) ? 1 : 0;
    }
    int st = solve_partition(G, k, g, F, x, y, idx, L, z);
    *rounds = 0;
    if (st != OR_OK)
        return st;
    int alpha = 3, beta = k + 1;
    for (;;) {
        int nv = 0, vmax = -1;
        for (int i = 0; i < k; ++i) {
            int inf = usable[i] && ((F[i] && x[i] < 0.0) || (!F[i] && y[i] < 0.0));
            if (inf) {
                ++nv;
                vmax = i;
            }
        }
        if (nv == 0)
            return OR_OK;
        if (*rounds >= max_rounds)
            return OR_NOT_CONVERGED;
        if (nv < beta) {
            beta = nv;
            alpha = 3;
            for (int i = 0; i < k; ++i)
                if (usable[i] && ((F[i] && x[i] < 0.0) || (!F[i] && y[i] < 0.0)))
                    F[i] ^= 1;
        } else if (alpha >= 1) {
            alpha -= 1;
            for (int i = 0; i < k; ++i)
                if (usable[i] && ((F[i] && x[i] < 0.0) || (!F[i] && y[i] < 0.0)))
                    F[i] ^= 1;
        } else {
            F[vmax] ^= 1;
        }
        *rounds += 1;
        st = solve_partition(G, k, g, F, x, y, idx, L, z);
        if (st != OR_OK)
            return st;
    }
}

/* Batched BPP: nrhs independent problems sharing G (the multi right-hand-side
 * NLS of Alg. 1 lines "update W" / "update H"). B and X are nrhs x k row-major.
 * passive (nrhs x k bytes, nullable) carries the warm start in and the final
 * passive sets out; rounds / status (nullable) receive per-RHS results.
 * Returns the worst status (0 if all converged). */
int oracle_bpp(const double *G, int k, const double *B, int64_t nrhs, double *X,
               uint8_t *passive, int warm, int max_rounds, int32_t *rounds, int8_t *status)
{
    if (k < 1 || k > 1024)
        return 1;
    int worst = OR_OK;
#pragma omp parallel
    {
        double *work = (double *)malloc(sizeof(double) * (size_t)(2 * k + k * k));
        int *idx = (int *)malloc(sizeof(int) * (size_t)k);
        uint8_t *Fl = (uint8_t *)malloc((size_t)k);
        int wl = OR_OK;
#pragma omp for schedule(dynamic, 64)
        for (int64_t j = 0; j < nrhs; ++j) {
            int r = 0;
            if (passive && warm)
                memcpy(Fl, passive + j * k, (size_t)k);
            int st = bpp_one(G, k, B + j * k, X + j * k, Fl, warm && passive, max_rounds, &r,
                             work, idx);
            if (passive)
                memcpy(passive + j * k, Fl, (size_t)k);
            if (rounds)
                rounds[j] = r;
            if (status)
                status[j] = (int8_t)st;
            if (st > wl)
                wl = st;
        }
#pragma omp critical
        if (wl > worst)
            worst = wl;
        free(work);
        free(idx);
        free(Fl);
    }
    return worst;
}

/* MU step of Eq. 5 for the rows of X (rows x k): with R the matching rows of
 * A H^T (or of (W^T A)^T) and G = H H^T (or W^T W),
 *   x_ij <- x_ij R_ij / (X G)_ij,
 * every (X G)_ij from the X before the step. Where (X G)_ij is not positive
 * (only when x_ij = 0 or G_jj = 0 for nonnegative data) x_ij is left as it is:
 * Eq. 5 is silent there and 0 is a fixed point of the rule. */
void oracle_mu(const double *G, int k, const double *R, int64_t rows, double *X)
{
#pragma omp parallel
    {
        double *den = (double *)malloc(sizeof(double) * (size_t)k);
#pragma omp for schedule(static)
        for (int64_t r = 0; r < rows; ++r) {
            double *x = X + r * k;
            for (int j = 0; j < k; ++j) {
                double d = 0.0;
                for (int l = 0; l < k; ++l)
                    d += x[l] * G[l * k + j];
                den[j] = d;
            }
            for (int j = 0; j < k; ++j)
                if (den[j] > 0.0)
                    x[j] = x[j] * R[r * k + j] / den[j];
        }
        free(den);
    }
}

/* HALS step of Eq. 6 for the rows of X: for i = 0..k-1 in order,
 *   x_i <- [R_i - sum_{l != i} G_li x_l]_+ / G_ii,
 * the sum using the values of x already updated for l < i. A column with
 * G_ii <= 0 (its factor row or column is zero) is set to 0: Eq. 6 divides by
 * G_ii, and such a column does not change f. */
void oracle_hals(const double *G, int k, const double *R, int64_t rows, double *X)
{
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < rows; ++r) {
        double *x = X + r * k;
        for (int i = 0; i < k; ++i) {
            const double gii = G[i * k + i];
            if (!(gii > 0.0)) {
                x[i] = 0.0;
                continue;
            }
            double num = R[r * k + i];
            for (int l = 0; l < k; ++l)
                if (l != i)
                    num -= G[l * k + i] * x[l];
            x[i] = (num > 0.0 ? num : 0.0) / gii;
        }
    }
}

/* Squared norm of the projected gradient of f with respect to the rows of X
 * (the stopping measure of Lin 2007, used for ANLS by Kim and Park): with
 * grad = X G - R (half the gradient of Eq. 1 in X when G and R are the other
 * factor's Gram and right-hand sides), each entry counts as grad_ij where
 * x_ij > 0 and as min(0, grad_ij) where x_ij = 0. */
double oracle_pgrad_sq(const double *G, int k, const double *R, int64_t rows, const double *X)
{
    double total = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : total)
    for (int64_t r = 0; r < rows; ++r) {
        const double *x = X + r * k;
        double row = 0.0;
        for (int j = 0; j < k; ++j) {
            double gj = -R[r * k + j];
            for (int l = 0; l < k; ++l)
                gj += x[l] * G[l * k + j];
            const double pj = x[j] > 0.0 ? gj : (gj < 0.0 ? gj : 0.0);
            row += pj * pj;
        }
        total += row;
    }
    return total;
}

/* One local update of X from (G, R) by the chosen method: 0 BPP (x = the exact
 * NLS minimiser), 1 MU, 2 HALS. */
static int local_update(int solver, const double *G, int k, const double *R, int64_t rows,
                        double *X, uint8_t *passive, int warm, int max_rounds, int32_t *rounds)
{
    if (solver == 1) {
        oracle_mu(G, k, R, rows, X);
        return OR_OK;
    }
    if (solver == 2) {
        oracle_hals(G, k, R, rows, X);
        return OR_OK;
    }
    return oracle_bpp(G, k, R, rows, X, passive, warm, max_rounds, rounds, NULL);
}

/* ---------------------------------------------------------------------------
 * ANLS (Alg. 1 with Eq. 2): T iterations, W-update then H-update, each an
 * exact block minimisation solved row by row with BPP.
 *   kind = 0: dense A (float32, lda); kind = 1: CSR A (rowptr/colidx/vals).
 *   W (m x k) and Ht (n x k): starting point in, final factors out.
 *   f_hist (iters + 1 values): f before the first iteration, then after each.
 *   pW (m x k bytes) / pH (n x k bytes), nullable: passive sets; with warm = 1
 *   each solve starts from the previous iteration's sets (first solve cold).
 *   rounds_hist (nullable, 2 * iters): total exchange rounds per half-step.
 *   solver: 0 BPP (the paper's method), 1 MU (Eq. 5), 2 HALS (Eq. 6); for MU and
 *   HALS each half-step is one update of the factor, and W, Ht are read as the
 *   iterate being updated (rounds are 0).
 * Returns the worst BPP status seen.
 * ------------------------------------------------------------------------- */
int oracle_anls(int kind, const float *A, int64_t lda, const int64_t *rowptr,
                const int32_t *colidx, const float *vals, int64_t m, int64_t n, int k,
                double *W, double *Ht, int iters, int warm, int max_rounds, double *f_hist,
                uint8_t *pW, uint8_t *pH, int64_t *rounds_hist, int solver)
{
    double *G = (double *)malloc(sizeof(double) * (size_t)k * (size_t)k);
    double *V = (double *)malloc(sizeof(double) * (size_t)m * (size_t)k);
    double *Y = (double *)malloc(sizeof(double) * (size_t)n * (size_t)k);
    int32_t *rw = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > n ? m : n));
    uint8_t *ownW = pW ? NULL : (uint8_t *)calloc((size_t)m * (size_t)k, 1);
    uint8_t *ownH = pH ? NULL : (uint8_t *)calloc((size_t)n * (size_t)k, 1);
    uint8_t *PW = pW ? pW : ownW;
    uint8_t *PH = pH ? pH : ownH;
    int worst = OR_OK;
    if (f_hist)
        f_hist[0] = kind == 0 ? oracle_objective_dense(A, m, n, lda, W, Ht, k)
                              : oracle_objective_csr(rowptr, colidx, vals, m, n, W, Ht, k);
    for (int t = 0; t < iters; ++t) {
        int w = warm && t > 0;
        /* W <- argmin_{W>=0} ||A - W H||: Gram H H^T and right-hand sides A H^T. */
        oracle_gram(Ht, n, k, G);
        if (kind == 0)
            oracle_mm_dense(A, m, n, lda, Ht, k, 0, V);
        else
            oracle_mm_csr(rowptr, colidx, vals, m, n, Ht, k, 0, V);
        memset(rw, 0, sizeof(int32_t) * (size_t)m);
        int st = local_update(solver, G, k, V, m, W, PW, w, max_rounds, rw);
        if (st > worst)
            worst = st;
        if (rounds_hist) {
            int64_t s = 0;
            for (int64_t i = 0; i < m; ++i)
                s += rw[i];
            rounds_hist[2 * t] = s;
        }
        /* H <- argmin_{H>=0} ||A - W H||: Gram W^T W and right-hand sides (W^T A)^T. */
        oracle_gram(W, m, k, G);
        if (kind == 0)
            oracle_mm_dense(A, m, n, lda, W, k, 1, Y);
        else
            oracle_mm_csr(rowptr, colidx, vals, m, n, W, k, 1, Y);
        memset(rw, 0, sizeof(int32_t) * (size_t)n);
        st = local_update(solver, G, k, Y, n, Ht, PH, w, max_rounds, rw);
        if (st > worst)
            worst = st;
        if (rounds_hist) {
            int64_t s = 0;
            for (int64_t j = 0; j < n; ++j)
                s += rw[j];
            rounds_hist[2 * t + 1] = s;
        }
        if (f_hist)
            f_hist[t + 1] = kind == 0 ? oracle_objective_dense(A, m, n, lda, W, Ht, k)
                                      : oracle_objective_csr(rowptr, colidx, vals, m, n, W, Ht, k);
    }
    free(G);
    free(V);
    free(Y);
    free(rw);
    free(ownW);
    free(ownH);
    return worst;
}
