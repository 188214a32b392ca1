/*
 * bqrrp_oracle.c -- plain, slow, obviously-correct FP64 CPU oracle for BQRRP.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this file; only the test-suite, the smoke check and the timed CPU baseline of
 * the benchmark do.  It shares no code, header, table or helper with the CUDA
 * library: every routine below is written out from the paper
 * ("Anatomy of High-Performance Column-Pivoted QR Decomposition", arXiv
 * 2507.00976) or from the textbook definition it names, as plain loops over
 * column-major arrays, with no blocking, fusion or reordering.
 *
 * Conventions: column-major, A(i,j) = A[i + j*lda], 0-based indices inside,
 * 1-based permutation vector on output (GEQP3 format, Sec. 1.3).
 *
 * Readings of the paper that this file commits to (each is also a pin in the
 * tests):
 *  - the sketching operator is d x m (Sec. 3.2; Alg. 1 writes d x n);
 *  - its entries are +-1 drawn from Philox4x32-10 (dense) or a sparse-sign
 *    operator with nnz nonzeros per column, both with unit scale (the paper
 *    says the variance is inessential, Alg. 1 footnote);
 *  - qrcp_wide is Alg. 2 (LUPP on the transposed sketch, piv_transform,
 *    permutation, unpivoted Householder QR) with all min(n-s, d) LU steps;
 *  - tri_rank is a diagonal inspection: k is the largest j <= w such that
 *    |Rsk(t,t)| > 10*d*u*|Rsk0(0,0)| for all t < j, u = 2^-53, where Rsk0 is
 *    the sketch's R factor of the FIRST iteration (a global scale, so that a
 *    trailing block made of rounding noise is not judged against itself);
 *    Sec. 2.2 defers the estimator to prior work, so this is our reading;
 *  - R11 = diag(D) * Rchol * Rsk(0:k, 0:w)  (Alg. 3, with D applied to rows,
 *    which is what makes Q_curr * R11 reproduce the panel);
 *  - the Householder reconstruction is the modified-LU construction of
 *    Ballard et al. (cited as BD2015, Alg. 5): Qc - [S;0] = Y*U with S chosen
 *    during elimination, T = -U*S*Y1^{-T}, D = S;
 *  - the rank-revealing truncation of the batched and serving workloads (not
 *    in the paper) is a post-pass on the computed R: the smallest i with
 *    ||R(i:, i:)||_F <= tol * ||A||_F, the residual measure of Sec. 6, with the
 *    rows at and below the factorization's rank counted as zero.
 *
 * Threads: the loops over independent columns (or rows) carry an OpenMP
 * "parallel for"; each iteration runs the same plain loop in the same order
 * as before, so the results are bit for bit the same for any thread count.
 * The thread count is 1 unless bqrrp_ref_set_threads() raises it.
 *
 * Parity status: every routine here is pinned by tests/test_oracle_*.py
 * (library cross-checks, closed forms, brute force, invariants) except the
 * numeric ratio curves of the Kahan experiment (Sec. 6), whose figures are
 * not in the text: parity unpinned for that experiment only.
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define AT(A, i, j, ld) ((A)[(size_t)(i) + (size_t)(j) * (size_t)(ld)])

/* Return codes, mirrored (not shared) by the CUDA library's own header. */
enum { REF_OK = 0, REF_ENOMEM = 1, REF_ENUMERIC = 3 };

/* Thread count of the parallel loops (1 = serial, the default). */
static int g_threads = 1;
void bqrrp_ref_set_threads(int t) { g_threads = t > 0 ? t : 1; }
int bqrrp_ref_get_threads(void) { return g_threads; }
#define PAR_FOR _Pragma("omp parallel for schedule(static) num_threads(g_threads)")

/* ------------------------------------------------------------------------ */
/* Philox4x32-10: Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as    */
/* easy as 1, 2, 3", SC'11.  Counter of four 32-bit words, key of two.        */
/* ------------------------------------------------------------------------ */
void bqrrp_ref_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;   /* round multipliers */
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;   /* key schedule (Weyl) */
    uint32_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * x0;
        uint64_t p1 = (uint64_t)M1 * x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ------------------------------------------------------------------------ */
/* Sketching operators (Alg. 1 sample step; Sec. 3.2).  S is d x m, ld = d.   */
/* ------------------------------------------------------------------------ */

/* Dense +-1: key = (seed lo, seed hi); for column j and row r the counter is
 * (j, r/128, 0, 0) and bit (r mod 128) of the 128-bit output (word (r%128)/32,
 * bit r%32) selects -1 when set.  Rows are prefix-stable in d. */
void bqrrp_ref_sketch_dense(int64_t d, int64_t m, uint64_t seed, double* S)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    PAR_FOR
    for (int64_t j = 0; j < m; ++j) {
        for (int64_t r = 0; r < d; ++r) {
            uint32_t ctr[4] = {(uint32_t)j, (uint32_t)(r / 128), 0u, 0u};
            uint32_t out[4];
            bqrrp_ref_philox4x32_10(ctr, key, out);
            int q = (int)(r % 128);
            uint32_t bit = (out[q / 32] >> (q % 32)) & 1u;
            AT(S, r, j, d) = bit ? -1.0 : 1.0;
        }
    }
}

/* Sparse sign: column j of S holds exactly nnz entries +-1 at distinct rows.
 * Draw t = 0,1,2,... uses counter (j, 1+t, 0, 0); each of the four output
 * words w gives a candidate row ((w>>1) * d) >> 31 and a sign (w & 1 -> -1);
 * candidates whose row is already taken are rejected. */
int bqrrp_ref_sketch_sparse(int64_t d, int64_t m, uint64_t seed, int64_t nnz, double* S)
{
    if (nnz < 1 || nnz > d) return -4;
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    int64_t* rows = (int64_t*)malloc(sizeof(int64_t) * (size_t)nnz);
    if (!rows) return REF_ENOMEM;
    for (int64_t j = 0; j < m; ++j) {
        for (int64_t r = 0; r < d; ++r) AT(S, r, j, d) = 0.0;
        int64_t got = 0;
        for (uint32_t t = 0; got < nnz; ++t) {
            uint32_t ctr[4] = {(uint32_t)j, 1u + t, 0u, 0u};
            uint32_t out[4];
            bqrrp_ref_philox4x32_10(ctr, key, out);
            for (int q = 0; q < 4 && got < nnz; ++q) {
                uint32_t w = out[q];
                int64_t row = (int64_t)(((uint64_t)(w >> 1) * (uint64_t)d) >> 31);
                int taken = 0;
                for (int64_t e = 0; e < got; ++e) if (rows[e] == row) taken = 1;
                if (taken) continue;
                rows[got++] = row;
                AT(S, row, j, d) = (w & 1u) ? -1.0 : 1.0;
            }
        }
    }
    free(rows);
    return REF_OK;
}

/* Msk = S * A  (d x n), plain triple loop, sum over i in increasing order. */
void bqrrp_ref_sketch_apply(int64_t d, int64_t m, int64_t n, const double* S,
                            const double* A, int64_t lda, double* Msk, int64_t ldsk)
{
    PAR_FOR
    for (int64_t j = 0; j < n; ++j)
        for (int64_t r = 0; r < d; ++r) {
            double acc = 0.0;
            for (int64_t i = 0; i < m; ++i) acc += AT(S, r, i, d) * AT(A, i, j, lda);
            AT(Msk, r, j, ldsk) = acc;
        }
}

/* ------------------------------------------------------------------------ */
/* Householder reflector in the LAPACK dlarfg convention (GEQRF/GEQP3 output */
/* format of Sec. 1.3): H = I - tau*v*v^T, v(0) = 1, H*[alpha; x] = [beta;0].*/
/* ------------------------------------------------------------------------ */
static double house(int64_t len, double* x /* x[0]=alpha, x[1..] tail */, double* tau)
{
    double alpha = x[0];
    double xn2 = 0.0;
    for (int64_t i = 1; i < len; ++i) xn2 += x[i] * x[i];
    if (xn2 == 0.0) { *tau = 0.0; return alpha; }
    double nrm = sqrt(alpha * alpha + xn2);
    double beta = (alpha >= 0.0) ? -nrm : nrm;
    *tau = (beta - alpha) / beta;
    double scal = 1.0 / (alpha - beta);
    for (int64_t i = 1; i < len; ++i) x[i] *= scal;
    x[0] = beta;
    return beta;
}

/* Apply H = I - tau v v^T (v(0)=1 implicit, v tail in vtail) to the rows
 * [0, len) of columns of C starting at C (ld ldc), ncols columns. */
static void apply_house(int64_t len, const double* vtail, double tau,
                        double* C, int64_t ldc, int64_t ncols)
{
    if (tau == 0.0) return;
    PAR_FOR
    for (int64_t c = 0; c < ncols; ++c) {
        double* col = C + (size_t)c * (size_t)ldc;
        double w = col[0];
        for (int64_t i = 1; i < len; ++i) w += vtail[i - 1] * col[i];
        w *= tau;
        col[0] -= w;
        for (int64_t i = 1; i < len; ++i) col[i] -= w * vtail[i - 1];
    }
}

/* Unpivoted Householder QR (GEQRF, LAWN 41 count 2mn^2 - 2n^3/3 for m >= n). */
void bqrrp_ref_geqrf(int64_t m, int64_t n, double* A, int64_t lda, double* tau)
{
    int64_t kk = m < n ? m : n;
    for (int64_t j = 0; j < kk; ++j) {
        double* col = &AT(A, j, j, lda);
        house(m - j, col, &tau[j]);
        apply_house(m - j, col + 1, tau[j], &AT(A, j, j + 1, lda), lda, n - j - 1);
    }
}

/* Businger-Golub QRCP (GEQP3 semantics, Sec. 1): at step j the pivot is the
 * first column of largest 2-norm of the trailing block A(j:m, j:n), recomputed
 * exactly (no norm downdating).  jpvt is 1-based on output. */
void bqrrp_ref_qrcp_bg(int64_t m, int64_t n, double* A, int64_t lda, int64_t* jpvt, double* tau)
{
    for (int64_t j = 0; j < n; ++j) jpvt[j] = j;
    int64_t kk = m < n ? m : n;
    for (int64_t j = 0; j < kk; ++j) {
        int64_t p = j;
        double best = -1.0;
        for (int64_t t = j; t < n; ++t) {
            double s = 0.0;
            for (int64_t i = j; i < m; ++i) s += AT(A, i, t, lda) * AT(A, i, t, lda);
            if (s > best) { best = s; p = t; }
        }
        if (p != j) {
            for (int64_t i = 0; i < m; ++i) {
                double tmp = AT(A, i, j, lda); AT(A, i, j, lda) = AT(A, i, p, lda); AT(A, i, p, lda) = tmp;
            }
            int64_t tj = jpvt[j]; jpvt[j] = jpvt[p]; jpvt[p] = tj;
        }
        double* col = &AT(A, j, j, lda);
        house(m - j, col, &tau[j]);
        apply_house(m - j, col + 1, tau[j], &AT(A, j, j + 1, lda), lda, n - j - 1);
    }
    for (int64_t j = kk; j < n; ++j) tau[j] = 0.0;
    for (int64_t j = 0; j < n; ++j) jpvt[j] += 1;
}

/* ------------------------------------------------------------------------ */
/* Alg. 2 pieces: LU with partial pivoting (GETRF semantics) and the pivot   */
/* format conversion piv_transform.                                          */
/* ------------------------------------------------------------------------ */

/* Row-pivoted LU of X (N x d), min(N,d) steps, in place.  The pivot of step j
 * is the FIRST row t >= j of largest |X(t,j)| (IDAMAX rule).  If the pivot is
 * zero the step performs no elimination (GETRF info > 0 behaviour).  margin,
 * if non-null, receives min over steps of (|top1|-|top2|)/|top1| (1 when a
 * step has a single candidate or an exact zero column).  Returns the number of
 * steps. */
int64_t bqrrp_ref_lupp(int64_t N, int64_t d, double* X, int64_t ldx, int64_t* ipiv, double* margin)
{
    int64_t steps = N < d ? N : d;
    double mg = 1.0;
    for (int64_t j = 0; j < steps; ++j) {
        int64_t p = j;
        double best = fabs(AT(X, j, j, ldx));
        for (int64_t t = j + 1; t < N; ++t) {
            double v = fabs(AT(X, t, j, ldx));
            if (v > best) { best = v; p = t; }
        }
        if (margin && best > 0.0) {
            double second = -1.0;
            for (int64_t t = j; t < N; ++t) if (t != p) {
                double v = fabs(AT(X, t, j, ldx));
                if (v > second) second = v;
            }
            if (second >= 0.0) {
                double g = (best - second) / best;
                if (g < mg) mg = g;
            }
        }
        ipiv[j] = p;
        if (p != j)
            for (int64_t c = 0; c < d; ++c) {
                double tmp = AT(X, j, c, ldx); AT(X, j, c, ldx) = AT(X, p, c, ldx); AT(X, p, c, ldx) = tmp;
            }
        double piv = AT(X, j, j, ldx);
        if (piv != 0.0) {
            for (int64_t t = j + 1; t < N; ++t) AT(X, t, j, ldx) /= piv;
            PAR_FOR
            for (int64_t c = j + 1; c < d; ++c) {
                double u = AT(X, j, c, ldx);
                for (int64_t t = j + 1; t < N; ++t) AT(X, t, c, ldx) -= AT(X, t, j, ldx) * u;
            }
        }
    }
    if (margin) *margin = mg;
    return steps;
}

/* piv_transform (Alg. 2, Sec. 2.1): start from the identity on N entries and
 * swap positions j and ipiv[j] for j = 0 .. steps-1, in order.  Jqr[t] is then
 * the original index of the entry that ends at position t (0-based). */
void bqrrp_ref_piv_transform(int64_t N, int64_t steps, const int64_t* ipiv, int64_t* Jqr)
{
    for (int64_t t = 0; t < N; ++t) Jqr[t] = t;
    for (int64_t j = 0; j < steps; ++j) {
        int64_t p = ipiv[j];
        int64_t tmp = Jqr[j]; Jqr[j] = Jqr[p]; Jqr[p] = tmp;
    }
}

/* col_perm_parallel (Alg. 5) on 0-based indices: out(:, t) = in(:, J[t]). */
static void col_gather(int64_t rows, int64_t ncols, const double* in, int64_t ldin,
                       const int64_t* J, double* out, int64_t ldout)
{
    PAR_FOR
    for (int64_t t = 0; t < ncols; ++t)
        for (int64_t i = 0; i < rows; ++i) AT(out, i, t, ldout) = AT(in, i, J[t], ldin);
}

/* ------------------------------------------------------------------------ */
/* Alg. 3 pieces: triangular solve, Cholesky QR, Householder reconstruction.  */
/* ------------------------------------------------------------------------ */

/* X <- X * R^{-1}, R upper triangular k x k (ld ldr), X rows x k (ld ldx);
 * row-wise forward substitution. */
static void trsm_right_upper(int64_t rows, int64_t k, const double* R, int64_t ldr, double* X, int64_t ldx)
{
    PAR_FOR
    for (int64_t i = 0; i < rows; ++i)
        for (int64_t j = 0; j < k; ++j) {
            double s = AT(X, i, j, ldx);
            for (int64_t t = 0; t < j; ++t) s -= AT(X, i, t, ldx) * AT(R, t, j, ldr);
            AT(X, i, j, ldx) = s / AT(R, j, j, ldr);
        }
}

/* Upper Cholesky G = R^T R of a k x k SPD matrix; returns the number of
 * successful columns (k on success, j < k when the pivot of column j is not
 * positive or not finite).  R's strictly-lower part is zeroed. */
static int64_t chol_upper(int64_t k, const double* G, int64_t ldg, double* R, int64_t ldr)
{
    for (int64_t j = 0; j < k; ++j)
        for (int64_t i = 0; i < k; ++i) AT(R, i, j, ldr) = 0.0;
    for (int64_t j = 0; j < k; ++j) {
        double s = AT(G, j, j, ldg);
        for (int64_t t = 0; t < j; ++t) s -= AT(R, t, j, ldr) * AT(R, t, j, ldr);
        if (!(s > 0.0) || !isfinite(s)) return j;
        double rjj = sqrt(s);
        AT(R, j, j, ldr) = rjj;
        for (int64_t l = j + 1; l < k; ++l) {
            double v = AT(G, j, l, ldg);
            for (int64_t t = 0; t < j; ++t) v -= AT(R, t, j, ldr) * AT(R, t, l, ldr);
            AT(R, j, l, ldr) = v / rjj;
        }
    }
    return k;
}

/* Householder reconstruction (ORHR_COL; BD2015 Alg. 5 as cited in Sec. 2.3).
 * In: Q (rows x k, orthonormal columns), overwritten by Y (unit lower
 * trapezoidal, unit diagonal stored explicitly, zeros above).  Out: T (k x k
 * upper, ld ldt) and D (k signs).  Modified LU: for j = 0..k-1,
 * s_j = -sign(A(j,j)) (sign(0) = +1), A(j,j) -= s_j, then ordinary
 * elimination of column j without pivoting; this yields Q - [S;0] = Y*U.
 * Finally T = -U*S*Y1^{-T}. */
void bqrrp_ref_orhr_col(int64_t rows, int64_t k, double* Q, int64_t ldq, double* T, int64_t ldt, double* D)
{
    double* U = (double*)calloc((size_t)k * (size_t)k + 1, sizeof(double));
    for (int64_t j = 0; j < k; ++j) {
        double a = AT(Q, j, j, ldq);
        double s = (a >= 0.0) ? -1.0 : 1.0;       /* s_j = -sign(a), sign(0)=+1 */
        D[j] = s;
        AT(Q, j, j, ldq) = a - s;
        double piv = AT(Q, j, j, ldq);
        for (int64_t i = j + 1; i < rows; ++i) AT(Q, i, j, ldq) /= piv;
        PAR_FOR
        for (int64_t c = j + 1; c < k; ++c) {
            double u = AT(Q, j, c, ldq);
            for (int64_t i = j + 1; i < rows; ++i) AT(Q, i, c, ldq) -= AT(Q, i, j, ldq) * u;
        }
    }
    /* split into U (upper, incl. diagonal) and unit-lower Y */
    for (int64_t j = 0; j < k; ++j)
        for (int64_t i = 0; i <= j; ++i) {
            AT(U, i, j, k) = AT(Q, i, j, ldq);
            AT(Q, i, j, ldq) = (i == j) ? 1.0 : 0.0;
        }
    /* T = -U*S*Y1^{-T}:  solve T * Y1^T = B with B = -U*S (columns of U
     * scaled by -s_j); Y1^T is unit upper, so T is found row by row. */
    PAR_FOR
    for (int64_t i = 0; i < k; ++i)
        for (int64_t j = 0; j < k; ++j) {
            double bij = -AT(U, i, j, k) * D[j];
            /* (T Y1^T)(i,j) = sum_t T(i,t) Y1(j,t) = T(i,j) + sum_{t<j} T(i,t) Y1(j,t) */
            double s = bij;
            for (int64_t t = 0; t < j; ++t) s -= AT(T, i, t, ldt) * AT(Q, j, t, ldq);
            AT(T, i, j, ldt) = s;
        }
    free(U);
}

/* ------------------------------------------------------------------------ */
/* BQRRP (Alg. 1), CholQR panel (Alg. 3) or Householder panel (Sec. 3.5).    */
/* ------------------------------------------------------------------------ */

static int has_nonfinite(int64_t rows, int64_t cols, const double* X, int64_t ld)
{
    for (int64_t j = 0; j < cols; ++j)
        for (int64_t i = 0; i < rows; ++i)
            if (!isfinite(AT(X, i, j, ld))) return 1;
    return 0;
}

/* Apply Q_curr^T = (H_1 ... H_k)^T to C (rows x ncols): H_1 first (ORMQR,
 * Sec. 2.4).  Y holds the reflectors (unit diagonal explicit), tau their
 * scalars.  Only the first `keep_rows` rows of the result are written back. */
static void apply_qt_col(int64_t rows, int64_t k, const double* Y, int64_t ldy, const double* tau,
                         double* col, int64_t keep_rows, double* scratch)
{
    for (int64_t i = 0; i < rows; ++i) scratch[i] = col[i];
    for (int64_t j = 0; j < k; ++j) {
        double w = 0.0;
        for (int64_t i = j; i < rows; ++i) w += AT(Y, i, j, ldy) * scratch[i];
        w *= tau[j];
        for (int64_t i = j; i < rows; ++i) scratch[i] -= w * AT(Y, i, j, ldy);
    }
    for (int64_t i = 0; i < keep_rows; ++i) col[i] = scratch[i];
}

static void apply_qt(int64_t rows, int64_t k, const double* Y, int64_t ldy, const double* tau,
                     double* C, int64_t ldc, int64_t ncols, int64_t keep_rows, double* scratch)
{
    const int nt = g_threads;
    double* all = nt > 1 ? (double*)malloc(sizeof(double) * (size_t)(rows > 0 ? rows : 1) * (size_t)nt) : NULL;
    if (!all) {
        for (int64_t c = 0; c < ncols; ++c)
            apply_qt_col(rows, k, Y, ldy, tau, &AT(C, 0, c, ldc), keep_rows, scratch);
        return;
    }
    /* one scratch column per thread */
    #pragma omp parallel num_threads(nt)
    {
        double* sc = all + (size_t)omp_get_thread_num() * (size_t)(rows > 0 ? rows : 1);
        #pragma omp for schedule(static)
        for (int64_t c = 0; c < ncols; ++c)
            apply_qt_col(rows, k, Y, ldy, tau, &AT(C, 0, c, ldc), keep_rows, sc);
    }
    free(all);
}

/* Alg. 3 on one panel.  Mp: rows x w permuted panel (read only); Rsk: upper
 * triangle of the sketch's R (ld ldr).  Pre = Mp(:, 0:k) Rsk11^{-1}; G =
 * Pre^T Pre; Rchol = chol(G); Qc = Pre Rchol^{-1}; (Y, T, D) = ORHR_COL(Qc)
 * with Y left in Y (rows x k, ld ldy); R11 = diag(D) Rchol Rsk(0:k, 0:w) in
 * R11 (k x w, ld ldb).  G, Rc, T are k x k with ld ldb.  Returns the number of
 * columns kept (k, or the column where the Cholesky factorization broke down;
 * on breakdown Y, T and R11 are not formed). */
static int64_t ref_cholqr_panel(int64_t rows, int64_t w, int64_t k, const double* Mp, int64_t ldm,
                                const double* Rsk, int64_t ldr, double* Y, int64_t ldy, double* G,
                                double* Rc, double* T, double* D, double* R11, int64_t ldb)
{
    for (int64_t j = 0; j < k; ++j)
        for (int64_t i = 0; i < rows; ++i) AT(Y, i, j, ldy) = AT(Mp, i, j, ldm);
    trsm_right_upper(rows, k, Rsk, ldr, Y, ldy);                  /* Pre = M(:,0:k) Rsk11^{-1} */
    PAR_FOR
    for (int64_t j = 0; j < k; ++j)                                /* G = Pre^T Pre */
        for (int64_t l = 0; l < k; ++l) {
            double acc = 0.0;
            for (int64_t i = 0; i < rows; ++i) acc += AT(Y, i, j, ldy) * AT(Y, i, l, ldy);
            AT(G, j, l, ldb) = acc;
        }
    int64_t kc = chol_upper(k, G, ldb, Rc, ldb);
    if (kc < k) return kc;
    trsm_right_upper(rows, k, Rc, ldb, Y, ldy);                   /* Qc = Pre Rchol^{-1} */
    bqrrp_ref_orhr_col(rows, k, Y, ldy, T, ldb, D);               /* Y, T, D */
    /* R11 = diag(D) * Rchol * Rsk(0:k, 0:w)  (k x w) */
    PAR_FOR
    for (int64_t j = 0; j < w; ++j)
        for (int64_t i = 0; i < k; ++i) {
            double acc = 0.0;
            int64_t tmax = j < k - 1 ? j : k - 1;                 /* Rsk(t,j) = 0 for t > j */
            for (int64_t t = i; t <= tmax; ++t) acc += AT(Rc, i, t, ldb) * AT(Rsk, t, j, ldr);
            AT(R11, i, j, ldb) = D[i] * acc;
        }
    return k;
}

/* Test hook: Alg. 3 on a panel with the same layout as above; also writes R11
 * into the upper trapezoid of Mp's first k rows and the reflectors below the
 * diagonal (the storage the factorization uses).  tau = diag(T). */
int64_t bqrrp_ref_cholqr_panel(int64_t rows, int64_t w, int64_t k, double* Mp, int64_t ldm,
                               const double* Rsk, int64_t ldr, double* T, int64_t ldt, double* tau)
{
    int64_t kb = k > 0 ? k : 1;
    double* Y = (double*)malloc(sizeof(double) * (size_t)(rows > 0 ? rows : 1) * (size_t)kb);
    double* G = (double*)malloc(sizeof(double) * (size_t)kb * (size_t)kb);
    double* Rc = (double*)malloc(sizeof(double) * (size_t)kb * (size_t)kb);
    double* Tk = (double*)malloc(sizeof(double) * (size_t)kb * (size_t)kb);
    double* D = (double*)malloc(sizeof(double) * (size_t)kb);
    double* R11 = (double*)malloc(sizeof(double) * (size_t)kb * (size_t)(w > 0 ? w : 1));
    int64_t kc = -1;
    if (Y && G && Rc && Tk && D && R11) {
        kc = ref_cholqr_panel(rows, w, k, Mp, ldm, Rsk, ldr, Y, rows, G, Rc, Tk, D, R11, kb);
        if (kc == k) {
            for (int64_t j = 0; j < w; ++j)
                for (int64_t i = 0; i < k && i <= j; ++i) AT(Mp, i, j, ldm) = AT(R11, i, j, kb);
            for (int64_t j = 0; j < k; ++j)
                for (int64_t i = j + 1; i < rows; ++i) AT(Mp, i, j, ldm) = AT(Y, i, j, rows);
            for (int64_t j = 0; j < k; ++j) {
                tau[j] = AT(Tk, j, j, kb);
                for (int64_t i = 0; i < k; ++i) AT(T, i, j, ldt) = AT(Tk, i, j, kb);
            }
        }
    }
    free(Y); free(G); free(Rc); free(Tk); free(D); free(R11);
    return kc;
}

/* sketch_kind: 0 dense +-1 Philox operator, 1 sparse sign (nnz per column),
 * 2 test hook only: S = I_m (requires d = m) together with qrcp_wide by
 * Businger-Golub, the special case in which BQRRP reduces to Businger-Golub
 * QRCP (derived from the sketch update of Alg. 1; pinned against LAPACK's
 * dgeqp3 in the tests).
 * trace (nullable): for iteration i, trace[4*i + 0] = k, [1] = min LU margin,
 * [2] = 1 if the sketch was non-finite (identity pivots), [3] = w.
 * Test hooks: max_iters > 0 stops after that many full iterations (the sketch
 * update of the last one included) and returns rank = s of the next block;
 * sketch_out (nullable, d x n, ld d) receives the sketch buffer on exit. */
int bqrrp_ref_factor(int64_t m, int64_t n, double* A, int64_t lda, int64_t b, int64_t d,
                     uint64_t seed, int sketch_kind, int64_t nnz, int panel_kind,
                     int64_t* jpvt, double* tau, int64_t* rank,
                     double* trace, int64_t trace_iters, int64_t max_iters, double* sketch_out)
{
    if (m < 0 || m < n) return -1;
    if (n < 0) return -2;
    if (lda < (m > 1 ? m : 1)) return -4;
    if (b < 1) return -5;
    if (d < b) return -6;
    if (sketch_kind != 0 && sketch_kind != 1 && sketch_kind != 2) return -8;
    if (sketch_kind == 1 && (nnz < 1 || nnz > d)) return -9;
    if (sketch_kind == 2 && d != m) return -6;
    *rank = 0;
    if (n == 0) return REF_OK;
    if (has_nonfinite(m, n, A, lda)) return REF_ENUMERIC;

    /* Alg. 1: sample S (d x m) and sketch Msk = S*M (d x n). */
    double* S = (double*)malloc(sizeof(double) * (size_t)d * (size_t)m);
    double* Msk = (double*)malloc(sizeof(double) * (size_t)d * (size_t)n);
    double* X = (double*)malloc(sizeof(double) * (size_t)n * (size_t)d);
    double* tmp = (double*)malloc(sizeof(double) * (size_t)(d > m ? d : m) * (size_t)n);
    int64_t* ipiv = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int64_t* Jsk = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int64_t* J = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int64_t* Jt = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    double* Pre = (double*)malloc(sizeof(double) * (size_t)m * (size_t)b);
    double* G = (double*)malloc(sizeof(double) * (size_t)b * (size_t)b);
    double* Rc = (double*)malloc(sizeof(double) * (size_t)b * (size_t)b);
    double* T = (double*)malloc(sizeof(double) * (size_t)b * (size_t)b);
    double* D = (double*)malloc(sizeof(double) * (size_t)b);
    double* R11 = (double*)malloc(sizeof(double) * (size_t)b * (size_t)b);
    double* Z = (double*)malloc(sizeof(double) * (size_t)b * (size_t)b);
    double* scratch = (double*)malloc(sizeof(double) * (size_t)(m + d + 1));
    double* sktau = (double*)malloc(sizeof(double) * (size_t)(n + d + 1));
    int rc = REF_OK;
    if (!S || !Msk || !X || !tmp || !ipiv || !Jsk || !J || !Jt || !Pre || !G || !Rc || !T || !D ||
        !R11 || !Z || !scratch || !sktau) { rc = REF_ENOMEM; goto done; }

    if (sketch_kind == 0) bqrrp_ref_sketch_dense(d, m, seed, S);
    else if (sketch_kind == 2) {                       /* S = I_m (test hook, see below) */
        for (int64_t j = 0; j < m; ++j)
            for (int64_t r = 0; r < d; ++r) AT(S, r, j, d) = (r == j) ? 1.0 : 0.0;
    }
    else { int e = bqrrp_ref_sketch_sparse(d, m, seed, nnz, S); if (e) { rc = e == REF_ENOMEM ? e : -9; goto done; } }
    bqrrp_ref_sketch_apply(d, m, n, S, A, lda, Msk, d);

    for (int64_t j = 0; j < n; ++j) J[j] = j;
    for (int64_t j = 0; j < n; ++j) tau[j] = 0.0;
    int64_t ell = 0;
    double r00_first = 0.0;

    for (int64_t it = 0;; ++it) {
        int64_t s = it * b;
        int64_t c = (s + b < n) ? s + b : n;
        int64_t w = c - s;
        int64_t N = n - s;
        double* Ssk = &AT(Msk, 0, s, d);           /* working sketch d x N */

        /* ---- Alg. 2: qrcp_wide on the sketch ---- */
        int nonfinite = has_nonfinite(d, N, Ssk, d);
        double margin = 1.0;
        if (nonfinite) {
            for (int64_t t = 0; t < N; ++t) Jsk[t] = t;       /* identity pivots */
        } else if (sketch_kind == 2) {
            /* Test hook: qrcp_wide by Businger-Golub instead of Alg. 2.  With
             * S = I the sketch is M itself, Rsk11 = D R11 (D = +-1), so the
             * sketch update zeroes rows 0..w-1 and leaves the trailing R of
             * the pivoted QR: BQRRP then makes Businger-Golub's choices. */
            bqrrp_ref_qrcp_bg(d, N, Ssk, d, Jsk, sktau);     /* R of the permuted sketch, in place */
            for (int64_t t = 0; t < N; ++t) Jsk[t] -= 1;
        } else {
            PAR_FOR
            for (int64_t t = 0; t < N; ++t)                    /* X = Ssk^T, N x d */
                for (int64_t r = 0; r < d; ++r) AT(X, t, r, N) = AT(Ssk, r, t, d);
            int64_t steps = bqrrp_ref_lupp(N, d, X, N, ipiv, &margin);
            bqrrp_ref_piv_transform(N, steps, ipiv, Jsk);
        }
        if (sketch_kind != 2 || nonfinite) {
            col_gather(d, N, Ssk, d, Jsk, tmp, d);
            for (int64_t t = 0; t < N; ++t)
                for (int64_t r = 0; r < d; ++r) AT(Ssk, r, t, d) = AT(tmp, r, t, d);
            bqrrp_ref_geqrf(d, N, Ssk, d, sktau);             /* Rsk in place */
        }
        for (int64_t t = 0; t < N; ++t)
            for (int64_t r = t + 1; r < d; ++r) AT(Ssk, r, t, d) = 0.0;

        /* ---- tri_rank (Sec. 2.2, our reading) ---- */
        int64_t k = 0;
        {
            if (it == 0) r00_first = fabs(AT(Ssk, 0, 0, d));
            double thr = 10.0 * (double)d * 1.1102230246251565e-16 * r00_first; /* 10 d u |R0(0,0)| */
            if (r00_first > 0.0 && isfinite(r00_first))
                while (k < w && isfinite(AT(Ssk, k, k, d)) && fabs(AT(Ssk, k, k, d)) > thr) ++k;
        }
        if (trace && it < trace_iters) {
            trace[4 * it + 0] = (double)k; trace[4 * it + 1] = margin;
            trace[4 * it + 2] = (double)nonfinite; trace[4 * it + 3] = (double)w;
        }

        /* ---- permute M(:, s:) and J(s:) (Alg. 1 permute steps, merged) ---- */
        col_gather(m, N, &AT(A, 0, s, lda), lda, Jsk, tmp, m);
        PAR_FOR
        for (int64_t t = 0; t < N; ++t)
            for (int64_t i = 0; i < m; ++i) AT(A, i, s + t, lda) = AT(tmp, i, t, m);
        for (int64_t t = 0; t < N; ++t) Jt[t] = J[s + Jsk[t]];
        for (int64_t t = 0; t < N; ++t) J[s + t] = Jt[t];

        /* early exit: the first permuted working column is all zero */
        {
            int allzero = 1;
            for (int64_t i = s; i < m; ++i) if (AT(A, i, s, lda) != 0.0) { allzero = 0; break; }
            if (allzero) { ell = s; break; }
        }
        if (k == 0) { ell = s; break; }

        int64_t rows = m - s;
        double* Mp = &AT(A, s, s, lda);                /* panel, rows x w */
        double* Y = Pre;                               /* rows x k, ld m */

        if (panel_kind == 0) {
            /* ---- Alg. 3: preconditioned Cholesky QR + reconstruction ---- */
            int64_t kc = ref_cholqr_panel(rows, w, k, Mp, lda, Ssk, d, Pre, m, G, Rc, T, D, R11, b);
            if (kc < k) {
                /* Cholesky breakdown: the block is numerically rank kc; redo the
                 * panel on its leading kc columns (same Gram block). */
                k = kc;
                if (trace && it < trace_iters) trace[4 * it + 0] = (double)k;
                if (k == 0) { ell = s; break; }
                ref_cholqr_panel(rows, w, k, Mp, lda, Ssk, d, Pre, m, G, Rc, T, D, R11, b);
            }
            for (int64_t j = 0; j < k; ++j) tau[s + j] = AT(T, j, j, b);
        } else {
            /* ---- Householder panel (GEQRF on all w panel columns) ---- */
            for (int64_t j = 0; j < w; ++j)
                for (int64_t i = 0; i < rows; ++i) AT(Pre, i, j, m) = AT(Mp, i, j, lda);
            double* ptau = D;   /* reuse: w <= b scalars */
            bqrrp_ref_geqrf(rows, w, Pre, m, ptau);
            for (int64_t j = 0; j < w; ++j)
                for (int64_t i = 0; i < k; ++i) AT(R11, i, j, b) = (i <= j) ? AT(Pre, i, j, m) : 0.0;
            for (int64_t j = 0; j < k; ++j) {
                tau[s + j] = ptau[j];
                for (int64_t i = 0; i <= j; ++i) AT(Pre, i, j, m) = (i == j) ? 1.0 : 0.0;
            }
        }

        /* ---- apply Q_curr^T to the trailing columns (Alg. 1 apply steps) ---- */
        int64_t keep = (k == w) ? rows : k;
        apply_qt(rows, k, Y, m, &tau[s], &AT(A, s, c, lda), lda, n - c, keep, scratch);
        if (k < w) {
            /* panel columns k..w-1 keep only their R11 rows; the rows below are
             * outside the rank-k factorization and are left unreduced. */
        }
        /* write R11 (rows s..s+k of columns s..c) and the reflectors below */
        for (int64_t j = 0; j < w; ++j)
            for (int64_t i = 0; i < k; ++i)
                if (i <= j) AT(Mp, i, j, lda) = AT(R11, i, j, b);
        for (int64_t j = 0; j < k; ++j)
            for (int64_t i = j + 1; i < rows; ++i) AT(Mp, i, j, lda) = AT(Y, i, j, m);

        if (c == n || k < w) { ell = s + k; break; }

        /* ---- sketch update (Alg. 1, Duersch-Gu): Msk(:, c:) =
         *      [Rsk12 - Rsk11 R11^{-1} R12 ; Rsk22] ---- */
        for (int64_t j = 0; j < w; ++j)                      /* Z = Rsk11 */
            for (int64_t i = 0; i < w; ++i) AT(Z, i, j, b) = (i <= j) ? AT(Ssk, i, j, d) : 0.0;
        trsm_right_upper(w, w, R11, b, Z, b);                 /* Z = Rsk11 R11^{-1} */
        PAR_FOR
        for (int64_t t = 0; t < n - c; ++t)                   /* Rsk12 -= Z * R12 */
            for (int64_t i = 0; i < w; ++i) {
                double acc = 0.0;
                for (int64_t l = 0; l < w; ++l) acc += AT(Z, i, l, b) * AT(A, s + l, c + t, lda);
                AT(Ssk, i, w + t, d) -= acc;
            }
        /* Rsk22 = Ssk(w:d, w:) is already upper trapezoidal with zeros below. */
        if (max_iters > 0 && it + 1 >= max_iters) { ell = c; break; }
    }
    *rank = ell;
    for (int64_t j = 0; j < n; ++j) jpvt[j] = J[j] + 1;
    if (sketch_out)
        for (int64_t j = 0; j < n; ++j)
            for (int64_t r = 0; r < d; ++r) AT(sketch_out, r, j, d) = AT(Msk, r, j, d);

done:
    free(S); free(Msk); free(X); free(tmp); free(ipiv); free(Jsk); free(J); free(Jt);
    free(Pre); free(G); free(Rc); free(T); free(D); free(R11); free(Z); free(scratch); free(sktau);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Rank-revealing truncation (the error measure of Sec. 6 used as a rule).    */
/* ------------------------------------------------------------------------ */

/* Smallest i in [0, rank] with ||R(i:rank, i:n)||_F <= tol * anorm, where R is
 * the upper trapezoid of the factored A (rows 0 .. rank-1; rows at and below
 * the rank are counted as zero).  Since R(r, c) = 0 for c < r, the block norm
 * is the sum over rows r >= i of ||R(r, r:n)||^2, accumulated here from the
 * last row upwards. */
int64_t bqrrp_ref_trunc_rank(int64_t m, int64_t n, const double* A, int64_t lda, int64_t rank,
                             double anorm, double tol)
{
    (void)m;
    double thr = tol * anorm;
    double thr2 = thr * thr;
    double tail = 0.0;          /* ||R(i:rank, i:n)||_F^2 for the current i */
    int64_t best = rank;
    for (int64_t i = rank - 1; i >= 0; --i) {
        double row = 0.0;
        for (int64_t c = i; c < n; ++c) row += AT(A, i, c, lda) * AT(A, i, c, lda);
        tail += row;
        if (tail <= thr2) best = i;
        else break;
    }
    return best;
}

/* Frobenius norm by a plain sum of squares in column order. */
double bqrrp_ref_fro_norm(int64_t m, int64_t n, const double* A, int64_t lda)
{
    double acc = 0.0;
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < m; ++i) acc += AT(A, i, j, lda) * AT(A, i, j, lda);
    return sqrt(acc);
}
