/*
 * bqrrp.h -- C ABI of the B300 (sm_103a) BQRRP library.
 *
 * BQRRP is the blocked randomized column-pivoted QR of arXiv 2507.00976
 * ("Anatomy of High-Performance Column-Pivoted QR Decomposition"), Alg. 1:
 * sketch A once, then per block of b columns pick pivots by LU with partial
 * pivoting on the small d x (n-s) sketch (Alg. 2), permute A's columns
 * (Alg. 5), factor the panel by preconditioned Cholesky QR plus Householder
 * reconstruction (Alg. 3), apply the block reflector to the trailing matrix and
 * update the sketch (Duersch-Gu update, last step of Alg. 1).
 *
 * Common conventions
 *  - Matrices are FP64, column-major: element (i,j) of X lives at
 *    X[i + j*ldx].  All matrix and vector pointers are DEVICE pointers unless
 *    the name ends in _host.
 *  - Every call is asynchronous on `stream` (a cudaStream_t; NULL = legacy
 *    default stream) unless stated otherwise, and allocates no device memory:
 *    scratch space comes from the caller's `workspace`.
 *  - Return value: 0 on success; -i when argument i is invalid (LAPACK "info"
 *    convention, arguments counted from 1); a positive BQRRP_E* code
 *    otherwise.  The message of the last failure on the calling thread is
 *    returned by bqrrp_last_error().  No call aborts the process.
 */
#ifndef BQRRP_H
#define BQRRP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define BQRRP_OK 0
#define BQRRP_ENOMEM 1      /* workspace smaller than bqrrp_workspace_query() */
#define BQRRP_ECUDA 2       /* a CUDA runtime call failed                      */
#define BQRRP_ENUMERIC 3    /* A holds NaN or Inf                              */
#define BQRRP_ETIMEOUT 4    /* a bounded cross-CTA wait gave up                */
#define BQRRP_EUNSUPPORTED 5 /* shape outside the supported range             */

/* Sketching operator kinds (Alg. 1 sample step, Sec. 3.2). */
#define BQRRP_SKETCH_DENSE 0   /* d x m, entries +-1 from Philox4x32-10          */
#define BQRRP_SKETCH_SPARSE 1  /* d x m, nnz entries +-1 per column              */

/* Panel factorizations for qr_tall (Sec. 2.3 / Sec. 3.5). */
#define BQRRP_PANEL_CHOLQR 0   /* Alg. 3: preconditioned CholQR + reconstruction */
#define BQRRP_PANEL_HQR 1      /* Householder QR of the panel                    */

/* Arithmetic of the dense products (sketch S*A and the trailing update). */
#define BQRRP_PRECISION_FP64 0   /* FP64 SIMT throughout                            */
#define BQRRP_PRECISION_MIXED 1  /* sketch and trailing-update products on the bf16
                                    tensor cores through exact balanced 8-bit slices
                                    (see bqrrp_dgemm_ozaki); LU, sketch QR, panel,
                                    tau, R in FP64                                   */
#define BQRRP_PRECISION_MIXED_SKETCH32 2 /* as _MIXED, and Alg. 2 on the sketch in
                                    FP32 arithmetic: the LU panels' pivot search and
                                    eliminations (the sketch stays FP64 in memory,
                                    the updates between panels are FP64 products)
                                    and the QR that forms R^sk from the LU factor.
                                    The pivots are FP32 decisions; R^sk, which
                                    preconditions the panel and becomes the next
                                    sketch, is accurate to FP32 relative to the
                                    current block's sketch; the panel, tau and R
                                    stay FP64                                       */

/* Order of the steps of consecutive blocks (the results are the same bit for bit). */
#define BQRRP_SCHEDULE_OVERLAP 0 /* the sketch update and Alg. 2 of block i+1 run on a
                                    high-priority side stream (created per call)
                                    while rows k.. of block i's trailing update run
                                    on `stream`; FP64 with the CholQR panel only
                                    (the other forms run serially)                  */
#define BQRRP_SCHEDULE_SERIAL 1  /* every step on `stream`, one after the other     */

typedef struct bqrrp_opts {
    int sketch_kind;     /* BQRRP_SKETCH_DENSE (default) or BQRRP_SKETCH_SPARSE */
    int64_t sketch_nnz;  /* nonzeros per column of a sparse sketch (default 8)  */
    int panel_kind;      /* BQRRP_PANEL_CHOLQR (default) or BQRRP_PANEL_HQR    */
    int64_t precision;   /* BQRRP_PRECISION_FP64 (default), _MIXED or _MIXED_SKETCH32 */
    int64_t schedule;    /* BQRRP_SCHEDULE_OVERLAP (default) or _SERIAL         */
    int64_t panel_tc;    /* 0 (default): the CholQR panel in FP64.  1 (only with
                            a _MIXED precision): the panel's Gram matrix and the
                            block updates of its two tall triangular solves
                            (the preconditioner and the reconstruction's) as
                            FP64-accurate slice products on the tensor cores;
                            the Cholesky factor, the reconstruction's LU, tau
                            and R stay in FP64                                  */
    int64_t reserved[2]; /* must be zero                                        */
} bqrrp_opts;

/*
 * bqrrp_factor -- column-pivoted QR  A*P = Q*R  by BQRRP (Alg. 1 with Alg. 2
 * as qrcp_wide and Alg. 3 as qr_tall; Sec. 3 for the storage layout).
 *
 *  m, n      rows and columns of A; 0 <= n <= m (m < n returns -1).
 *  A         device, m x n, column-major, leading dimension lda >= max(1,m).
 *            In: the matrix.  Out (GEQP3 format, Sec. 1.3): rows 0..rank-1 of
 *            the upper trapezoid hold R; below the diagonal of columns
 *            0..rank-1 the Householder vectors v_i (v_i(i) = 1 implicit).
 *            When rank < n the rows rank..m-1 of columns rank..n-1 are
 *            unspecified.
 *  b         block size, b >= 1 (b > n factors in one block).
 *  d         sketch rows, d >= b (the paper's d = ceil(gamma*b)).
 *  seed      64-bit key of the sketching operator (see bqrrp_sketch_operator).
 *  jpvt      device, n int64, out: 1-based permutation, column j of A*P is
 *            column jpvt[j]-1 of A.
 *  tau       device, n doubles, out: tau[0..rank-1] are the reflector scalars,
 *            the rest are zero.
 *  rank      HOST, out: the numerical rank l (Sec. 2.2).  Written before the
 *            call returns: the call synchronizes `stream` a few times per
 *            block (the block rank k decides the control flow).
 *  opts      nullable (defaults above).  With the default overlap schedule
 *            the call also creates a private high-priority stream, orders it
 *            against `stream` with events, and synchronizes and destroys it
 *            before returning (on error paths too).
 *  workspace device scratch of at least bqrrp_workspace_query() bytes,
 *            256-byte aligned; owned by the caller, contents undefined on exit.
 *
 * Errors: -1 m, -2 n, -3 A, -4 lda, -5 b, -6 d, -8 jpvt, -9 tau, -10 rank,
 * -11 opts, -12 workspace, BQRRP_ENOMEM when workspace_bytes is too small,
 * BQRRP_ENUMERIC for NaN/Inf in A (A is then left unchanged), BQRRP_ETIMEOUT,
 * BQRRP_ECUDA.  On any error rank is set to -1 when rank is non-null.
 */
int bqrrp_factor(int64_t m, int64_t n, double* A, int64_t lda, int64_t b, int64_t d,
                 uint64_t seed, int64_t* jpvt, double* tau, int64_t* rank,
                 const bqrrp_opts* opts, void* workspace, size_t workspace_bytes,
                 void* stream);

/* Bytes of device workspace bqrrp_factor needs for this shape (0 on invalid
 * arguments).  Dominant terms: 2*d*n + 2*b*n + m*b + max(m,d)*min(n, 2d) doubles. */
size_t bqrrp_workspace_query(int64_t m, int64_t n, int64_t b, int64_t d, const bqrrp_opts* opts);

/*
 * bqrrp_factor_host -- the same factorization for HOST buffers: A_host
 * (m x n, ld lda, in/out), jpvt_host (n) and tau_host (n) live in host memory
 * (pinned memory gives full PCIe/C2C bandwidth).  The call copies A to the
 * device on `stream`, factors it as bqrrp_factor does, copies A, jpvt and tau
 * back and synchronizes `stream` before returning; the results are bit for bit
 * those of bqrrp_factor.  When A_host is pinned, the copies run on a private
 * copy stream (created and destroyed inside the call, synchronized before it
 * returns): with the dense FP64 sketch A comes in by column halves, each
 * sketched as soon as it has arrived, and each finished column block of R and
 * the reflectors goes back while the later blocks are factored.  Pageable
 * A_host is copied in before the factorization and back after it.
 * workspace is device memory of at least bqrrp_workspace_query_host() bytes
 * (A, jpvt and tau on the device, then bqrrp_factor's workspace).
 * Errors: those of bqrrp_factor.  On BQRRP_ENUMERIC A_host is unchanged; on
 * BQRRP_ETIMEOUT or BQRRP_ECUDA its contents are unspecified.
 */
int bqrrp_factor_host(int64_t m, int64_t n, double* A_host, int64_t lda, int64_t b, int64_t d,
                      uint64_t seed, int64_t* jpvt_host, double* tau_host, int64_t* rank,
                      const bqrrp_opts* opts, void* workspace, size_t workspace_bytes,
                      void* stream);
size_t bqrrp_workspace_query_host(int64_t m, int64_t n, int64_t b, int64_t d, const bqrrp_opts* opts);

/*
 * bqrrp_sketch_operator -- write the d x m sketching operator S explicitly
 * (Alg. 1 sample step; the paper samples Gaussian entries, this library uses
 * +-1 entries, whose scale is immaterial per the paper's footnote to Alg. 1).
 * Dense: key = (seed low word, seed high word); for column j and row r the
 * Philox4x32-10 counter is (j, r/128, 0, 0) and bit r%128 of the 128-bit output
 * (word (r%128)/32, bit r%32) set means -1.  Sparse: column j holds exactly nnz
 * entries at distinct rows; draw t = 0,1,... uses counter (j, 1+t, 0, 0), each
 * output word w proposes row ((w>>1)*d)>>31 with sign -1 iff w&1, repeats are
 * skipped.  S: device, d x m, ld lds >= d.  Test hook; the factorization never
 * stores S.  Errors: -1 d, -2 m, -4 kind, -5 nnz, -6 S, -7 lds.
 */
int bqrrp_sketch_operator(int64_t d, int64_t m, uint64_t seed, int kind, int64_t nnz,
                          double* S, int64_t lds, void* stream);

/*
 * bqrrp_sketch_apply -- Msk = S*A (Alg. 1 sketching step) with S generated on
 * the fly from (seed, kind, nnz) as above.  A: device m x n (ld lda);
 * Msk: device d x n (ld ldsk >= d), overwritten.  The sparse kind needs
 * bqrrp_sketch_apply_workspace() bytes of workspace (the dense kind none).
 */
int bqrrp_sketch_apply(int64_t d, int64_t m, int64_t n, const double* A, int64_t lda,
                       uint64_t seed, int kind, int64_t nnz, double* Msk, int64_t ldsk,
                       void* workspace, size_t workspace_bytes, void* stream);
size_t bqrrp_sketch_apply_workspace(int64_t d, int64_t m, int kind, int64_t nnz);

/*
 * bqrrp_sketch_apply_sparse_noalloc -- the sparse-sign form of
 * bqrrp_sketch_apply (same operator, same result) for callers that cannot
 * allocate device memory or hand over a workspace: code whose device memory is
 * entirely owned by another allocator, plug-ins that get device pointers but
 * no allocator, loops that must never enter an allocator.  The operator's index
 * lists live in a fixed array inside the library's device image (about
 * 12.6 MB, held on every GPU that loads the library until process exit); the
 * call allocates nothing.  The paper has no counterpart: this is a deployment
 * convenience, not part of the method.
 *  Limits: d <= 4096 and m*nnz <= 524288 (2^19); larger shapes return
 *  BQRRP_EUNSUPPORTED with a message in bqrrp_last_error().
 *  The first call on each device looks up the array's device address (with
 *  that device current); make that first call before any stream capture.
 *  All calls share the one array, which keeps the previous call's contents
 *  (the call clears what must start at zero): calls that can overlap on the
 *  GPU -- concurrent streams, other host threads -- race and must be
 *  serialized by the caller.
 *  Arguments as bqrrp_sketch_apply with kind = sparse: -1 d, -2 m, -3 n, -4 A,
 *  -5 lda, -7 nnz, -8 Msk, -9 ldsk.
 */
int bqrrp_sketch_apply_sparse_noalloc(int64_t d, int64_t m, int64_t n, const double* A, int64_t lda,
                                      uint64_t seed, int64_t nnz, double* Msk, int64_t ldsk, void* stream);

/*
 * bqrrp_qrcp_wide -- Alg. 2 on a d x N sketch: row-pivoted LU of Msk^T (all
 * min(N,d) steps, first-maximum pivot rule), piv_transform, column gather and
 * unpivoted Householder QR.  Msk: device d x N (ld ldsk), in: the sketch;
 * out: R^sk (upper trapezoid, zeros below the diagonal).  Jsk: device, N int64,
 * out: 0-based permutation (column t of the permuted sketch was column
 * Jsk[t]).  ipiv: device, min(N,d) int64, out: the LU swap sequence (0-based).
 * If the sketch holds NaN/Inf, Jsk is the identity (Sec. 2.2).
 */
int bqrrp_qrcp_wide(int64_t d, int64_t N, double* Msk, int64_t ldsk, int64_t* Jsk, int64_t* ipiv,
                    void* workspace, size_t workspace_bytes, void* stream);
size_t bqrrp_qrcp_wide_workspace(int64_t d, int64_t N);

/* bqrrp_selftest_lu_wait_timeout -- failure-detection self-test of the pivot
 * exchange of Alg. 2's LU (the cross-CTA waits of bqrrp_qrcp_wide and
 * bqrrp_factor).  Two runs on a copy of Msk (d x N, column-major, ld ldsk,
 * device, read only): first, one CTA of the first LU panel withholds its
 * step-0 candidate, so every bounded wait of that launch runs out (2^12 polls,
 * a few milliseconds) and the status word must report the timeout; then the
 * same LU runs normally in the same CUDA context.  ipiv (device, min(N, d)
 * int64) receives the second run's 0-based swap sequence.  workspace: at
 * least bqrrp_qrcp_wide_workspace(d, N) device bytes.  Returns 0 when the
 * forced wait was reported and the second run completed; BQRRP_ECUDA if the
 * forced wait was not reported; the second run's status otherwise; -i for a
 * bad argument i.  No kernel faults or hangs: every wait is bounded. */
int bqrrp_selftest_lu_wait_timeout(int64_t d, int64_t N, const double* Msk, int64_t ldsk, int64_t* ipiv,
                                   void* workspace, size_t workspace_bytes, void* stream);

/*
 * bqrrp_col_perm -- column permutation of Alg. 5 in place: afterwards column t
 * of M (m x N, ld ldm) is the former column J[t] (0-based J, a permutation of
 * 0..N-1).  Only columns with J[t] != t move; they are staged through the
 * workspace (bqrrp_col_perm_workspace(m, moved) bytes, moved = an upper bound
 * on the number of such columns, e.g. N or 2*min(N,d) after Alg. 2).
 */
int bqrrp_col_perm(int64_t m, int64_t N, double* M, int64_t ldm, const int64_t* J, int64_t max_moved,
                   void* workspace, size_t workspace_bytes, void* stream);
size_t bqrrp_col_perm_workspace(int64_t m, int64_t N, int64_t max_moved);

/*
 * bqrrp_cholqr_panel -- Alg. 3 on one panel: Pre = M(:,0:k) * Rsk(0:k,0:k)^-1,
 * Cholesky QR of Pre, Householder reconstruction (modified LU), and
 * R11 = diag(D) * Rchol * Rsk(0:k, 0:w).  M: device rows x w (ld ldm), in: the
 * permuted panel, out: R11 in rows 0..k-1 of the upper trapezoid and the
 * reflectors below the diagonal of columns 0..k-1.  Rsk: device, upper
 * triangle of a k x w block (ld ldr).  T: device k x k (ld ldt), out: the
 * compact-WY factor (upper).  tau: device, k doubles, out: diag(T).
 * kout: HOST, out: k, lowered if the Cholesky factorization breaks down.
 */
int bqrrp_cholqr_panel(int64_t rows, int64_t w, int64_t k, double* M, int64_t ldm,
                       const double* Rsk, int64_t ldr, double* T, int64_t ldt, double* tau,
                       int64_t* kout, void* workspace, size_t workspace_bytes, void* stream);
size_t bqrrp_cholqr_panel_workspace(int64_t rows, int64_t w);

/*
 * bqrrp_geqrf -- the library's own unpivoted blocked Householder QR (GEQRF
 * semantics, the denominator of the paper's canonical comparison, Sec. 7):
 * A (m x n, ld lda, m >= n) is overwritten with R and the reflectors,
 * tau (n) receives the scalars.  nb: outer block (0 = default 64).
 */
int bqrrp_geqrf(int64_t m, int64_t n, double* A, int64_t lda, double* tau, int64_t nb,
                void* workspace, size_t workspace_bytes, void* stream);
size_t bqrrp_geqrf_workspace(int64_t m, int64_t n, int64_t nb);

/* The same unpivoted QR with the trailing-update products on the bf16 tensor
 * cores (exact slices, FP64 accuracy; see bqrrp_dgemm_ozaki): the baseline the
 * mixed-precision BQRRP is compared with. */
int bqrrp_geqrf_mixed(int64_t m, int64_t n, double* A, int64_t lda, double* tau,
                      void* workspace, size_t workspace_bytes, void* stream);
size_t bqrrp_geqrf_mixed_workspace(int64_t m, int64_t n);

/*
 * bqrrp_dgemm -- C = alpha*op(A)*op(B) + beta*C with the library's FP64 SIMT
 * GEMM (the kernel behind the trailing update of Alg. 1).  transa/transb:
 * 'N' or 'T'.  C is M x N, op(A) M x K, op(B) K x N.  beta == 0 never reads C.
 * Uses up to bqrrp_dgemm_workspace() bytes of workspace for split-K partials
 * (pass NULL/0 to disable splitting).
 */
int bqrrp_dgemm(char transa, char transb, int64_t M, int64_t N, int64_t K, double alpha,
                const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                double* C, int64_t ldc, void* workspace, size_t workspace_bytes, void* stream);
size_t bqrrp_dgemm_workspace(int64_t M, int64_t N, int64_t K);

/*
 * bqrrp_dgemm_ozaki -- the same product as bqrrp_dgemm formed on the bf16
 * tensor cores: each row of op(A) and column of op(B) is scaled by a power of
 * two and cut into seven balanced 8-bit integer slices in [-128, 127] (exact
 * in bf16); the 28 slice products with p + q <= 6 are summed exactly in FP32
 * within K chunks of 128, combined exactly in 64-bit integers and rounded
 * once to FP64.  The error is a few units of 2^-53 times
 * max|op(A)(i,:)| * max|op(B)(:,j)| per term -- FP64 accuracy in the normwise
 * sense; integer data within 2^53 come out exact.  A product of fewer tiles
 * (128 x 64) than half the SMs splits K over more CTAs and adds their
 * integer sums exactly (same bound; the result is deterministic).  This is
 * the "Ozaki-split" trailing update of the mixed-precision form (the paper's
 * apply_trans_q, Sec. 2.4, computed differently; the splitting itself has no
 * counterpart in the paper).  Needs bqrrp_dgemm_ozaki_workspace() bytes of
 * workspace; synchronizes the stream once to read the kernel's wait status.
 */
int bqrrp_dgemm_ozaki(char transa, char transb, int64_t M, int64_t N, int64_t K, double alpha,
                      const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                      double* C, int64_t ldc, void* workspace, size_t workspace_bytes, void* stream);
size_t bqrrp_dgemm_ozaki_workspace(int64_t M, int64_t N, int64_t K);

/*
 * bqrrp_sketch_apply_tc -- Msk = S*A with the dense +-1 operator (as
 * bqrrp_sketch_apply, kind dense) on the bf16 tensor cores: S is one exact
 * slice and A is cut into seven balanced 8-bit slices per column, so the
 * seven products S*A_q give S*A to FP64 accuracy (Alg. 1 sketching step).
 * Needs bqrrp_sketch_apply_tc_workspace() bytes.
 */
int bqrrp_sketch_apply_tc(int64_t d, int64_t m, int64_t n, const double* A, int64_t lda, uint64_t seed,
                          double* Msk, int64_t ldsk, void* workspace, size_t workspace_bytes,
                          void* stream);
size_t bqrrp_sketch_apply_tc_workspace(int64_t d, int64_t m, int64_t n);

/*
 * bqrrp_probe_fp64_peak -- measurement helper: runs an FP64 fused-multiply-add
 * loop on every SM for about `iters` x 32 DFMA per thread and returns the
 * achieved FP64 rate in TFLOP/s (timed with CUDA events; synchronizes).
 * Returns a negative value on failure.
 */
double bqrrp_probe_fp64_peak(int iters, void* stream);

/*
 * Phase profile (measurement helper, off by default).  When enabled,
 * bqrrp_factor records CUDA events on its stream around each step of Alg. 1
 * and, after its final synchronization, adds the device time (ms) and the
 * algorithmic FLOP count of each phase to a process-wide accumulator.
 * Phases: 0 sketch S*A, 1 LU with partial pivoting + piv_transform,
 * 2 sketch gather + Householder QR + tri_rank, 3 permutation of A and J,
 * 4 panel (Alg. 3), 5 trailing update (three GEMMs), 6 sketch update,
 * 7 other (checks, setup, rank read-backs).
 */
#define BQRRP_NPHASES 8
typedef struct bqrrp_profile {
    double ms[BQRRP_NPHASES];     /* accumulated device time per phase          */
    double flops[BQRRP_NPHASES];  /* accumulated algorithmic FLOPs per phase    */
    int64_t calls;                /* profiled bqrrp_factor calls                */
} bqrrp_profile;
void bqrrp_profile_enable(int on);
void bqrrp_profile_reset(void);
int bqrrp_profile_read(bqrrp_profile* out);

/* ------------------------------------------------------------------------
 * Batched BQRRP: many independent FP64 matrices factored together.
 *
 * Each matrix i (m_i x n_i, m_i >= n_i) is factored exactly as bqrrp_factor
 * does with the dense Philox +-1 sketch and the Alg. 3 CholQR panel, with its
 * own block size b_i, sketch size d_i and seed_i; the paper (Alg. 1) treats one
 * matrix, and the batch adds no arithmetic.  The matrices advance block by
 * block in lock step: each phase of a block iteration is one persistent kernel
 * over the whole batch, whose thread blocks take work items (a matrix or a
 * tile of one) from a queue ordered largest first.  A matrix that finishes
 * early (Sec. 3.7) is skipped by the later launches.
 *
 * Packed layout (both the caller and the library use it):
 *  - A: matrix i starts at element offA_i = sum_{j<i} m_j n_j, column-major,
 *    lda = m_i.  On exit it holds R and the reflectors (GEQP3 format).
 *  - jpvt (int64), tau (double): matrix i starts at offJ_i = sum_{j<i} n_j;
 *    n_i entries each; jpvt is 1-based on exit, tau beyond the rank is 0.
 *  - rank, trunc_rank (int64), info (int32): one entry per matrix.
 *
 * Truncation (not in the paper; the residual measure of Sec. 6 used as a
 * rule): trunc_rank_i = the smallest t in [0, rank_i] with
 * ||R(t:rank_i, t:n_i)||_F <= trunc_tol * ||A_i||_F.
 *
 * Limits: n_i <= 4096, m_i <= 2^24, 1 <= b_i <= 128, b_i <= d_i <= 256;
 * otherwise bqrrp_batch_plan_create returns -5 / -6 (b, d) or
 * BQRRP_EUNSUPPORTED.  A matrix holding NaN/Inf is left untouched with
 * info_i = BQRRP_ENUMERIC, rank_i = 0, identity jpvt and tau = 0.
 * ------------------------------------------------------------------------ */
typedef struct bqrrp_batch_plan_s* bqrrp_batch_plan;

/* Build a plan on the host for the current device: the per-matrix records,
 * the work queues of every launch and the workspace layout.  m, n, b, d,
 * seed: HOST arrays of `batch` entries.  *plan receives a handle owned by the
 * caller (free with bqrrp_batch_plan_destroy).  Synchronous; no device
 * memory is touched. */
int bqrrp_batch_plan_create(bqrrp_batch_plan* plan, int64_t batch, const int64_t* m, const int64_t* n,
                            const int64_t* b, const int64_t* d, const uint64_t* seed, double trunc_tol);

/* The same with a tile shape per matrix: tile_cols[i] (HOST, 32 or 64) is the
 * column width of matrix i's trailing-update and sketch-update tiles (one
 * work item each); bqrrp_batch_plan_create uses 64.  Narrow tiles waste fewer
 * threads on narrow trailing blocks and give a matrix's update more parallel
 * items; wide tiles reread Y fewer times.  The arithmetic of a tile differs
 * only in the order of the partial sums of W = Y^T C, so results agree with
 * the 64-column form to rounding, not bit for bit.  Errors as
 * bqrrp_batch_plan_create, and -10 for a tile width other than 32 or 64. */
int bqrrp_batch_plan_create_tiles(bqrrp_batch_plan* plan, int64_t batch, const int64_t* m, const int64_t* n,
                                  const int64_t* b, const int64_t* d, const int64_t* tile_cols, const uint64_t* seed,
                                  double trunc_tol);

/* Device workspace bytes the plan needs (256-byte aligned workspace). */
size_t bqrrp_batch_workspace_bytes(bqrrp_batch_plan plan);

/* Factor the whole batch (device pointers; trunc_rank and info may be NULL).
 * The first call with a given workspace uploads the plan into it
 * (copies queued on `stream` ahead of the launches); later calls reuse it, so the workspace must not be
 * modified between calls.  use_graph != 0 captures the launch sequence into a
 * CUDA graph on the first call (on a private stream of the plan) and replays it
 * on `stream` while (A, jpvt, tau, rank, trunc_rank, info, workspace) stay the
 * same.  Asynchronous on
 * `stream` otherwise; allocates nothing.  Errors: -1 bad plan, -2 null output,
 * BQRRP_ENOMEM short workspace, BQRRP_ECUDA. */
int bqrrp_batch_factor(bqrrp_batch_plan plan, double* A, int64_t* jpvt, double* tau, int64_t* rank,
                       int64_t* trunc_rank, int32_t* info, void* workspace, size_t workspace_bytes, void* stream,
                       int use_graph);

/* Release a plan (and its captured graph).  NULL is ignored. */
void bqrrp_batch_plan_destroy(bqrrp_batch_plan plan);

/* Launch form of a plan (the arithmetic, and so every result, is the same bit
 * for bit in both forms):
 *  BQRRP_BATCH_PERSISTENT (default): one persistent kernel whose thread blocks
 *    take tasks from device queues, each matrix advancing phase by phase as
 *    soon as its previous phase is done;
 *  BQRRP_BATCH_LOCKSTEP: one short kernel per phase and block iteration over
 *    the whole batch (leaves SMs to concurrent work between launches; the
 *    serving loop's small lane uses it).
 * Changing the form drops a captured graph.  Errors: -1 null plan, -2 form. */
#define BQRRP_BATCH_PERSISTENT 0
#define BQRRP_BATCH_LOCKSTEP 1
int bqrrp_batch_plan_set_form(bqrrp_batch_plan plan, int form);

/* Number of kernel launches one bqrrp_batch_factor call issues. */
int bqrrp_batch_launches(bqrrp_batch_plan plan);

/* Algorithmic FLOPs of one bqrrp_batch_factor call in profiler phase `phase`
 * (-1: all phases), counted as if every block kept all its columns.  With the
 * profiler on (bqrrp_profile_enable), a call without graph capture records
 * each launch's device time and adds per-phase times and these FLOPs to the
 * profile, synchronizing `stream`; phase 1 then covers all of Alg. 2 (LU,
 * piv_transform, gather, Householder QR, tri_rank), which runs as one kernel. */
double bqrrp_batch_flops(bqrrp_batch_plan plan, int phase);

/* Autotuner: choose b_i = min(beta_c, n_i) with beta_c from {16, 32, 64, 128}
 * per size class c of n_i
 * ([0,64), [64,128), ..., [1024, inf)) by timing each class alone on the
 * device, then d_i = ceil(gamma * b_i) with gamma from {1.25, 1.5} by timing
 * the whole batch.  A (device, packed as above) is read only: every trial
 * factors a copy held in the workspace.  m, n, seed, b_out, d_out: HOST
 * arrays; best_ms (host, nullable) receives the best whole-batch time.
 * Synchronizes `stream`.  workspace: bqrrp_batch_autotune_workspace_bytes(). */
size_t bqrrp_batch_autotune_workspace_bytes(int64_t batch, const int64_t* m, const int64_t* n);
int bqrrp_batch_autotune(int64_t batch, const int64_t* m, const int64_t* n, const uint64_t* seed, const double* A,
                         double trunc_tol, void* workspace, size_t workspace_bytes, void* stream, int64_t* b_out,
                         int64_t* d_out, double* best_ms);

/* The autotuner with tile shapes: after each size class's b, the class's
 * trailing tile width (32 or 64 columns) is chosen by timing the class alone
 * with that b; gamma is then chosen over the whole batch with those tiles.
 * tile_out (HOST, `batch` entries) receives the widths, for
 * bqrrp_batch_plan_create_tiles.  Same workspace, arguments and errors as
 * bqrrp_batch_autotune, and -12 for a null tile_out. */
int bqrrp_batch_autotune_tiles(int64_t batch, const int64_t* m, const int64_t* n, const uint64_t* seed,
                               const double* A, double trunc_tol, void* workspace, size_t workspace_bytes,
                               void* stream, int64_t* b_out, int64_t* d_out, int64_t* tile_out, double* best_ms);

/* ------------------------------------------------------------------------
 * Request loop (serving layer; the paper factors one matrix per call).
 *
 * A server owns one device pool of hbm_budget_bytes, allocated once at
 * creation: a request arena (hbm_budget_bytes - workspace_bytes) that holds
 * every admitted request's state (its matrix, factored in place, jpvt, tau)
 * from admission until its results are copied back, and a workspace arena
 * (workspace_bytes) for the job that is running.  A worker thread admits
 * submitted requests first-come-first-served whenever their state fits, then
 * alternates between two lanes on one CUDA stream:
 *  - small requests (m*n <= small_max_elems) are factored together in one
 *    batched call (bqrrp_batch_* kernels, each request addressed in place);
 *    requests arriving meanwhile join the next batch;
 *  - larger requests run one at a time through the single-matrix path.
 * Each completed request reports its rank and its truncation rank (smallest t
 * with ||R(t:rank, t:n)||_F <= trunc_tol * ||A||_F) and four timestamps in
 * seconds on the server's clock (bqrrp_server_clock).
 * flags: BQRRP_SERVER_DRYRUN replaces all GPU work by a sleep of
 * (2mn^2 - 2n^3/3) / (dry_gflops * 1e9) seconds and allocates no device
 * memory (host-side tests of admission and batching).
 * ------------------------------------------------------------------------ */
#define BQRRP_SERVER_DRYRUN 1
/* flags: BQRRP_SERVER_MIXED factors the large lane's requests with
 * opts.precision = BQRRP_PRECISION_MIXED (FP64-accurate products on the
 * tensor cores; the same 1e-12 bar as FP64); the small lane is unchanged.
 * Other flag bits: -6. */
#define BQRRP_SERVER_MIXED 2

typedef struct bqrrp_request {
    uint64_t id;              /* caller's tag, echoed in the completion                  */
    int64_t m, n, b, d;       /* shape (m >= n >= 1), block size, sketch rows            */
    uint64_t seed;            /* sketch seed                                              */
    const double* A_host;     /* m x n column-major (lda = m), HOST; read at admission   */
    double* A_out_host;       /* nullable HOST m x n: R above the diagonal, reflectors below */
    int64_t* jpvt_out_host;   /* nullable HOST n: 1-based column permutation              */
    double* tau_out_host;     /* nullable HOST n: reflector scalars                       */
} bqrrp_request;

typedef struct bqrrp_completion {
    uint64_t id;
    int32_t status;           /* 0, or a BQRRP_E* code (BQRRP_ENUMERIC: NaN/Inf input)    */
    int32_t lane;             /* 0 small (batched), 1 large (single-matrix)               */
    int64_t rank, trunc_rank;
    double t_submit, t_admit, t_start, t_done;
} bqrrp_completion;

typedef struct bqrrp_server_stats {
    int64_t submitted, completed, batches, max_batch, large_runs;
    int64_t peak_request_bytes;   /* most request-arena bytes ever held at once            */
    int64_t request_arena_bytes;
    int64_t in_use_bytes;
} bqrrp_server_stats;

typedef struct bqrrp_server_s* bqrrp_server;

/* Create a server on the current device (hbm_budget_bytes >= workspace_bytes
 * + 1 MiB).  Errors: -1 null out, -2 sizes, -4 tolerance, BQRRP_ENOMEM when the
 * pool cannot be allocated. */
int bqrrp_server_create(bqrrp_server* out, size_t hbm_budget_bytes, size_t workspace_bytes, double trunc_tol,
                        int64_t small_max_elems, int flags, double dry_gflops);
/* Queue a request (the descriptor is copied; the host buffers must stay valid
 * until its completion is returned).  Small-lane requests need b <= 128,
 * d <= 256, n <= 4096.  Returns -2 on a bad request, BQRRP_ENOMEM when its
 * state can never fit in the request arena. */
int bqrrp_server_submit(bqrrp_server srv, const bqrrp_request* req);
/* Move up to max_out completions into out (waiting up to wait_s seconds for
 * the first one); returns how many. */
int bqrrp_server_poll(bqrrp_server srv, bqrrp_completion* out, int max_out, double wait_s);
/* Block until every submitted request has completed. */
int bqrrp_server_drain(bqrrp_server srv);
/* Seconds since the server was created (the clock of the timestamps). */
double bqrrp_server_clock(bqrrp_server srv);
/* Message of the last job that failed on the server's worker ("" if none). */
const char* bqrrp_server_last_error(bqrrp_server srv);
int bqrrp_server_get_stats(bqrrp_server srv, bqrrp_server_stats* out);
/* Stop the worker after the queued work, release the pool. */
void bqrrp_server_destroy(bqrrp_server srv);

/* Number of kernel launches the library has issued since it was loaded. */
int64_t bqrrp_launch_counter(void);

/* Message describing the last error on the calling thread ("" if none). */
const char* bqrrp_last_error(void);

/* Library version string. */
const char* bqrrp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BQRRP_H */
