// api_steps.cu -- C-ABI entry points for single steps of BQRRP (used by the
// per-kernel parity tests) and the FP64 peak probe used by the benchmark.
#include <algorithm>
#include <climits>

#include "common.cuh"

namespace bq {
namespace {

__global__ void init_status_small(DevStatus* st) {
    st->err_timeout = 0;
    st->potrf_info = INT_MAX;
    st->sk_nonfinite = 0;
    st->a_nonfinite = 0;
    st->zero_col = 0;
    st->k = 0;
    st->moved = 0;
    st->r00 = 0.0;
    st->blk00 = 0.0;
    st->bar.count = 0;
    st->bar.gen = 0;
}

constexpr size_t kSplitElems = (size_t)1 << 21;

// split-K partials for a blocked QR of n columns: the W = V^T C products have
// one 64-row tile band, so their split count needs s * 64 * n partials
inline size_t qr_split_elems(i64 n) { return std::max(kSplitElems, (size_t)8 * 64 * (size_t)imax(n, 1)); }

// status block, split-K partials and cooperative scratch at the head of a workspace
void carve_common(Arena& ar, Ctx* c, size_t split_elems) {
    c->st = ar.take<DevStatus>(1);
    c->splitk_elems = split_elems;
    c->splitk = ar.take<double>(split_elems);
    coop_scratch_elems(64, 148, &c->coop_elems);
    c->coop = ar.take<double>(c->coop_elems);
}

int begin(void* ws, size_t bytes, void* stream, Arena* ar, Ctx* c, bool dry, size_t split_elems = kSplitElems) {
    ar->dry = dry;
    if (!dry) {
        ar->base = (char*)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
        ar->cap = bytes > (size_t)(ar->base - (char*)ws) ? bytes - (size_t)(ar->base - (char*)ws) : 0;
        BQ_TRY(current_device(&c->dev));
    }
    c->stream = (cudaStream_t)stream;
    carve_common(*ar, c, split_elems);
    return 0;
}

int finish(const Ctx& c) {
    DevStatus hs{};
    BQ_CUDA(cudaMemcpyAsync(&hs, c.st, sizeof(hs), cudaMemcpyDeviceToHost, c.stream));
    BQ_CUDA(cudaStreamSynchronize(c.stream));
    if (hs.err_timeout) { set_error("a bounded cross-CTA wait timed out"); return BQRRP_ETIMEOUT; }
    return 0;
}

struct QrcpWs {
    double *X, *Ub, *stage, *V, *T, *W, *W2, *tau;
    i64 *pos, *src, *cnt;
};

void carve_qrcp(Arena& ar, i64 d, i64 N, QrcpWs* q) {
    const i64 mm = imax(1, imin(N, 2 * imin(d, N)));
    q->X = ar.take<double>((size_t)d * N);
    q->Ub = ar.take<double>((size_t)d * imin(d, N));
    q->stage = ar.take<double>((size_t)d * mm);
    q->V = ar.take<double>((size_t)d * 64);
    q->T = ar.take<double>(64 * 64);
    q->W = ar.take<double>((size_t)64 * N);
    q->W2 = ar.take<double>((size_t)64 * N);
    q->tau = ar.take<double>((size_t)imax(d, N));
    q->pos = ar.take<i64>((size_t)mm);
    q->src = ar.take<i64>((size_t)mm);
    q->cnt = ar.take<i64>(4);
}

__global__ void probe_dfma_kernel(double* out, int iters, double a, double b) {
    double x0 = threadIdx.x * 1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
    double x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
            x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
        }
    }
    const double s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
    if (s == 12345.678) out[0] = s;   // keeps the chains live
}

// Vo = the reflectors stored below the diagonal of A (rows x w, ld lda) with
// a unit diagonal and zeros above it.
__global__ void unit_lower_kernel(i64 rows, i64 w, const double* A, i64 lda, double* V, i64 ldv) {
    const i64 total = rows * w;
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (i64)gridDim.x * blockDim.x) {
        const i64 i = e % rows, j = e / rows;
        V[i + j * ldv] = i > j ? A[i + j * lda] : (i == j ? 1.0 : 0.0);
    }
}

// Copy a k x k upper triangle (zeros below) from T (ld ldt) into To (ld ldo).
__global__ void copy_upper_kernel(i64 k, const double* T, i64 ldt, double* To, i64 ldo) {
    const i64 total = k * k;
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (i64)gridDim.x * blockDim.x) {
        const i64 i = e % k, j = e / k;
        To[i + j * ldo] = i <= j ? T[i + j * ldt] : 0.0;
    }
}

constexpr i64 kOuterQr = 256;   // outer block of the two-level QR

struct TwoLevelWs {
    double *V, *T, *W, *W2;         // inner panels (rows x 64, 64 x 64, 64 x n, 64 x n)
    double *Vo, *To, *G, *X;        // outer block: rows x 256, 256 x 256, 256 x 256, 256 x 64
    double *Wo, *Wo2;               // 256 x n each
};

void carve_two_level(Arena& ar, i64 m, i64 n, TwoLevelWs* w) {
    w->V = ar.take<double>((size_t)imax(m, 1) * 64);
    w->T = ar.take<double>(64 * 64);
    w->W = ar.take<double>((size_t)64 * imax(n, 1));
    w->W2 = ar.take<double>((size_t)64 * imax(n, 1));
    w->Vo = ar.take<double>((size_t)imax(m, 1) * kOuterQr);
    w->To = ar.take<double>((size_t)kOuterQr * kOuterQr);
    w->G = ar.take<double>((size_t)kOuterQr * kOuterQr);
    w->X = ar.take<double>((size_t)kOuterQr * 64);
    w->Wo = ar.take<double>((size_t)kOuterQr * imax(n, 1));
    w->Wo2 = ar.take<double>((size_t)kOuterQr * imax(n, 1));
}

// Two-level blocked Householder QR (GEQRF semantics): outer blocks of 256
// columns, each factored by 64-wide panels whose updates stay inside the
// block; the columns right of the block are updated once per block with the
// block reflector I - Vo To Vo^T of all its reflectors, so that those products
// have K = 256.  To is built from the panels' T factors by the compact-WY
// recurrence [[T1, -T1 (V1^T V2) T2], [0, T2]], with G = Vo^T Vo.
int geqrf_two_level(const Ctx& c, i64 rows, i64 cols, double* A, i64 lda, double* tau, const TwoLevelWs& w) {
    const i64 kk = imin(rows, cols);
    const unsigned gb = (unsigned)imax(1, imin(cdiv(rows * kOuterQr, 256), 16LL * c.dev.sms));
    for (i64 jb = 0; jb < kk; jb += kOuterQr) {
        const i64 bw = imin(kOuterQr, kk - jb), prow = rows - jb, nc = cols - jb - bw;
        double* Ab = A + jb + jb * lda;
        if (nc > 0) BQ_CUDA(cudaMemsetAsync(w.To, 0, sizeof(double) * kOuterQr * kOuterQr, c.stream));
        // the block's panels; after each, its T goes to the diagonal of To
        for (i64 p0 = 0; p0 < bw; p0 += 64) {
            const i64 pw = imin(64, bw - p0);
            BQ_TRY(geqrf_blocked(c, prow - p0, bw - p0, Ab + p0 + p0 * lda, lda, tau + jb + p0, w.V, w.T, w.W, w.W2,
                                 64, pw));
            if (nc > 0) {
                copy_upper_kernel<<<(unsigned)cdiv(pw * pw, 256), 256, 0, c.stream>>>(pw, w.T, 64,
                                                                                     w.To + p0 + p0 * kOuterQr,
                                                                                     kOuterQr);
                BQ_LAUNCH_CHECK();
            }
        }
        if (nc <= 0) continue;
        unit_lower_kernel<<<gb, 256, 0, c.stream>>>(prow, bw, Ab, lda, w.Vo, rows);
        BQ_LAUNCH_CHECK();
        BQ_TRY(pgemm(c, true, false, bw, bw, prow, 1.0, w.Vo, rows, w.Vo, rows, 0.0, w.G, kOuterQr, kGemmCUpper));
        for (i64 p0 = 64; p0 < bw; p0 += 64) {
            const i64 pw = imin(64, bw - p0);
            // X = G(0:p0, p0:p0+pw) T_p ; To(0:p0, p0:p0+pw) = -To(0:p0, 0:p0) X
            BQ_TRY(dgemm(c, false, false, p0, pw, pw, 1.0, w.G + p0 * kOuterQr, kOuterQr, w.To + p0 + p0 * kOuterQr,
                         kOuterQr, 0.0, w.X, kOuterQr));
            BQ_TRY(dgemm(c, false, false, p0, pw, p0, -1.0, w.To, kOuterQr, w.X, kOuterQr, 0.0,
                         w.To + p0 * kOuterQr, kOuterQr, kGemmAUpper));
        }
        double* C = A + jb + (jb + bw) * lda;
        BQ_TRY(pgemm(c, true, false, bw, nc, prow, 1.0, w.Vo, rows, C, lda, 0.0, w.Wo, kOuterQr));
        BQ_TRY(pgemm(c, true, false, bw, nc, bw, 1.0, w.To, kOuterQr, w.Wo, kOuterQr, 0.0, w.Wo2, kOuterQr));
        BQ_TRY(pgemm(c, false, false, prow, nc, bw, -1.0, w.Vo, rows, w.Wo2, kOuterQr, 1.0, C, lda));
    }
    return 0;
}

}  // namespace
}  // namespace bq

using namespace bq;

extern "C" {

size_t bqrrp_qrcp_wide_workspace(int64_t d, int64_t N) {
    if (d < 1 || N < 0) return 0;
    Arena ar;
    Ctx c{};
    begin(nullptr, 0, nullptr, &ar, &c, true);
    QrcpWs q{};
    carve_qrcp(ar, d, imax(N, 1), &q);
    return ar.off + 256;
}

int bqrrp_qrcp_wide(int64_t d, int64_t N, double* Msk, int64_t ldsk, int64_t* Jsk, int64_t* ipiv, void* workspace,
                    size_t workspace_bytes, void* stream) {
    set_error("");
    if (d < 1) return -1;
    if (N < 0) return -2;
    if (ldsk < d) return -4;
    if (N == 0) return 0;
    if (!Msk) return -3;
    if (!Jsk) return -5;
    if (!ipiv) return -6;
    if (workspace_bytes < bqrrp_qrcp_wide_workspace(d, N)) { set_error("workspace too small"); return BQRRP_ENOMEM; }
    Arena ar;
    Ctx c{};
    BQ_TRY(begin(workspace, workspace_bytes, stream, &ar, &c, false));
    QrcpWs q{};
    carve_qrcp(ar, d, N, &q);
    init_status_small<<<1, 1, 0, c.stream>>>(c.st);
    BQ_LAUNCH_CHECK();
    BQ_TRY(any_nonfinite(c, d, N, Msk, ldsk, &c.st->sk_nonfinite));
    BQ_CUDA(cudaMemcpy2DAsync(q.X, sizeof(double) * d, Msk, sizeof(double) * ldsk, sizeof(double) * d, N,
                              cudaMemcpyDeviceToDevice, c.stream));
    const i64 steps = imin(N, d);
    BQ_TRY(getrf_pivots(c, N, d, q.X, d, ipiv));
    BQ_TRY(piv_transform_moved(c, N, steps, ipiv, Jsk, &c.st->sk_nonfinite, q.pos, q.src, q.cnt));
    BQ_TRY(rsk_from_lu(c, d, N, q.X, d, Msk, ldsk, q.Ub, q.tau, q.V, q.T, q.W, q.W2));
    return finish(c);
}

// Failure-detection self-test of the pivot exchange (see the header).
int bqrrp_selftest_lu_wait_timeout(int64_t d, int64_t N, const double* Msk, int64_t ldsk, int64_t* ipiv,
                                   void* workspace, size_t workspace_bytes, void* stream) {
    set_error("");
    if (d < 1) return -1;
    if (N < 1) return -2;
    if (!Msk) return -3;
    if (ldsk < d) return -4;
    if (!ipiv) return -5;
    if (workspace_bytes < bqrrp_qrcp_wide_workspace(d, N)) { set_error("workspace too small"); return BQRRP_ENOMEM; }
    Arena ar;
    Ctx c{};
    BQ_TRY(begin(workspace, workspace_bytes, stream, &ar, &c, false));
    QrcpWs q{};
    carve_qrcp(ar, d, N, &q);
    if (!ar.ok()) { set_error("workspace too small"); return BQRRP_ENOMEM; }
    // 1: CTA 0 of the first panel withholds its step-0 candidate; every wait is
    // bounded by 2^12 polls (a few ms), so the launch ends with the timeout flag set
    init_status_small<<<1, 1, 0, c.stream>>>(c.st);
    BQ_LAUNCH_CHECK();
    BQ_CUDA(cudaMemcpy2DAsync(q.X, sizeof(double) * d, Msk, sizeof(double) * ldsk, sizeof(double) * d, N,
                              cudaMemcpyDeviceToDevice, c.stream));
    BQ_TRY(getrf_pivots_ex(c, N, d, q.X, d, ipiv, 1ull << 12, 0));
    const int forced = finish(c);
    if (forced != BQRRP_ETIMEOUT) {
        set_error("the withheld candidate did not make the exchange time out (status %d)", forced);
        return BQRRP_ECUDA;
    }
    // 2: the same LU without the stall, in the same context, must complete
    init_status_small<<<1, 1, 0, c.stream>>>(c.st);
    BQ_LAUNCH_CHECK();
    BQ_CUDA(cudaMemcpy2DAsync(q.X, sizeof(double) * d, Msk, sizeof(double) * ldsk, sizeof(double) * d, N,
                              cudaMemcpyDeviceToDevice, c.stream));
    BQ_TRY(getrf_pivots(c, N, d, q.X, d, ipiv));
    return finish(c);
}

size_t bqrrp_col_perm_workspace(int64_t m, int64_t N, int64_t max_moved) {
    if (m < 0 || N < 0) return 0;
    const i64 mm = imax(1, imin(N, max_moved));
    Arena ar;
    Ctx c{};
    begin(nullptr, 0, nullptr, &ar, &c, true);
    ar.take<double>((size_t)imax(m, 1) * mm);
    ar.take<i64>((size_t)mm);
    ar.take<i64>((size_t)mm);
    ar.take<i64>(4);
    ar.take<i64>((size_t)imax(N, 1));
    return ar.off + 256;
}

int bqrrp_col_perm(int64_t m, int64_t N, double* M, int64_t ldm, const int64_t* J, int64_t max_moved, void* workspace,
                   size_t workspace_bytes, void* stream) {
    set_error("");
    if (m < 0) return -1;
    if (N < 0) return -2;
    if (ldm < imax(1, m)) return -4;
    if (max_moved < 0) return -6;
    if (N == 0 || m == 0) return 0;
    if (!M) return -3;
    if (!J) return -5;
    if (workspace_bytes < bqrrp_col_perm_workspace(m, N, max_moved)) { set_error("workspace too small"); return BQRRP_ENOMEM; }
    Arena ar;
    Ctx c{};
    BQ_TRY(begin(workspace, workspace_bytes, stream, &ar, &c, false));
    const i64 mm = imax(1, imin(N, max_moved));
    double* stage = ar.take<double>((size_t)m * mm);
    i64* pos = ar.take<i64>((size_t)mm);
    i64* src = ar.take<i64>((size_t)mm);
    i64* cnt = ar.take<i64>(4);
    i64* Jcopy = ar.take<i64>((size_t)N);
    init_status_small<<<1, 1, 0, c.stream>>>(c.st);
    BQ_LAUNCH_CHECK();
    BQ_CUDA(cudaMemcpyAsync(Jcopy, J, sizeof(i64) * N, cudaMemcpyDeviceToDevice, c.stream));
    // compaction of the given permutation (no swaps: steps = 0 keeps J as is)
    BQ_TRY(moved_list_given(c, N, Jcopy, pos, src, cnt, mm));
    i64 moved = 0;
    BQ_CUDA(cudaMemcpyAsync(&moved, cnt, sizeof(i64), cudaMemcpyDeviceToHost, c.stream));
    BQ_CUDA(cudaStreamSynchronize(c.stream));
    if (moved > mm) {
        set_error("col_perm: %lld columns move, more than max_moved = %lld", (long long)moved, (long long)mm);
        return -6;
    }
    BQ_TRY(gather_cols(c, m, M, ldm, pos, src, cnt, mm, stage, m));
    return finish(c);
}

size_t bqrrp_cholqr_panel_workspace(int64_t rows, int64_t w) {
    if (rows < 0 || w < 0) return 0;
    const i64 k = imax(w, 1);
    Arena ar;
    Ctx c{};
    begin(nullptr, 0, nullptr, &ar, &c, true);
    ar.take<double>((size_t)imax(rows, 1) * k);   // Y
    for (int i = 0; i < 5; ++i) ar.take<double>((size_t)k * k);
    ar.take<double>((size_t)k);
    return ar.off + 256;
}

int bqrrp_cholqr_panel(int64_t rows, int64_t w, int64_t k, double* M, int64_t ldm, const double* Rsk, int64_t ldr,
                       double* T, int64_t ldt, double* tau, int64_t* kout, void* workspace, size_t workspace_bytes,
                       void* stream) {
    set_error("");
    if (rows < 0) return -1;
    if (w < 0 || w > rows) return -2;
    if (k < 0 || k > w) return -3;
    if (ldm < imax(1, rows)) return -5;
    if (ldr < imax(1, k)) return -7;
    if (ldt < imax(1, k)) return -9;
    if (!kout) return -11;
    *kout = 0;
    if (k == 0) return 0;
    if (!M) return -4;
    if (!Rsk) return -6;
    if (!T) return -8;
    if (!tau) return -10;
    if (workspace_bytes < bqrrp_cholqr_panel_workspace(rows, w)) { set_error("workspace too small"); return BQRRP_ENOMEM; }
    Arena ar;
    Ctx c{};
    BQ_TRY(begin(workspace, workspace_bytes, stream, &ar, &c, false));
    const i64 kb = imax(w, 1);
    double* Y = ar.take<double>((size_t)rows * kb);
    double* G = ar.take<double>((size_t)kb * kb);
    double* U = ar.take<double>((size_t)kb * kb);
    double* Tb = ar.take<double>((size_t)kb * kb);
    double* R11 = ar.take<double>((size_t)kb * kb);
    ar.take<double>((size_t)kb * kb);
    double* D = ar.take<double>((size_t)kb);
    init_status_small<<<1, 1, 0, c.stream>>>(c.st);
    BQ_LAUNCH_CHECK();
    i64 kk = k;
    BQ_TRY(cholqr_panel_steps(c, rows, w, &kk, M, ldm, Rsk, ldr, Y, rows, G, U, Tb, R11, D, kb, tau));
    if (kk > 0) BQ_TRY(copy_mat(c, kk, kk, Tb, kb, T, ldt));
    *kout = kk;
    return finish(c);
}

size_t bqrrp_geqrf_workspace(int64_t m, int64_t n, int64_t nb) {
    if (m < 0 || n < 0) return 0;
    Arena ar;
    Ctx c{};
    begin(nullptr, 0, nullptr, &ar, &c, true, qr_split_elems(n));
    ar.take<double>((size_t)imax(m, 1) * 64);
    ar.take<double>(64 * 64);
    ar.take<double>((size_t)64 * imax(n, 1));
    ar.take<double>((size_t)64 * imax(n, 1));
    (void)nb;
    return ar.off + 256;
}

int bqrrp_geqrf(int64_t m, int64_t n, double* A, int64_t lda, double* tau, int64_t nb, void* workspace,
                size_t workspace_bytes, void* stream) {
    set_error("");
    if (m < 0) return -1;
    if (n < 0) return -2;
    if (lda < imax(1, m)) return -4;
    if (nb < 0) return -6;
    if (m == 0 || n == 0) return 0;
    if (!A) return -3;
    if (!tau) return -5;
    if (workspace_bytes < bqrrp_geqrf_workspace(m, n, nb)) { set_error("workspace too small"); return BQRRP_ENOMEM; }
    Arena ar;
    Ctx c{};
    BQ_TRY(begin(workspace, workspace_bytes, stream, &ar, &c, false, qr_split_elems(n)));
    double* V = ar.take<double>((size_t)m * 64);
    double* T = ar.take<double>(64 * 64);
    double* W = ar.take<double>((size_t)64 * n);
    double* W2 = ar.take<double>((size_t)64 * n);
    init_status_small<<<1, 1, 0, c.stream>>>(c.st);
    BQ_LAUNCH_CHECK();
    BQ_TRY(geqrf_blocked(c, m, n, A, lda, tau, V, T, W, W2, nb == 0 ? 64 : imin(nb, 64)));
    return finish(c);
}

size_t bqrrp_geqrf_mixed_workspace(int64_t m, int64_t n) {
    if (m < 0 || n < 0) return 0;
    Arena ar;
    Ctx c{};
    begin(nullptr, 0, nullptr, &ar, &c, true, qr_split_elems(n));
    TwoLevelWs w{};
    carve_two_level(ar, m, n, &w);
    const i64 mm = imax(m, 1), nn = imax(n, 1);
    size_t oz = ozaki_ws_bytes(kOuterQr, nn, mm, kOzPlanes);             // Vo^T C, Vo^T Vo
    oz = std::max(oz, ozaki_ws_bytes(mm, nn, kOuterQr, kOzPlanes));      // C -= Vo Wo2
    oz = std::max(oz, ozaki_ws_bytes(64, nn, mm, kOzPlanes));            // the panels' own updates
    oz += ozaki_split_reserve();
    ar.take<char>(oz);
    return ar.off + 256;
}

int bqrrp_geqrf_mixed(int64_t m, int64_t n, double* A, int64_t lda, double* tau, void* workspace,
                      size_t workspace_bytes, void* stream) {
    set_error("");
    if (m < 0) return -1;
    if (n < 0) return -2;
    if (lda < imax(1, m)) return -4;
    if (m == 0 || n == 0) return 0;
    if (!A) return -3;
    if (!tau) return -5;
    if (workspace_bytes < bqrrp_geqrf_mixed_workspace(m, n)) { set_error("workspace too small"); return BQRRP_ENOMEM; }
    Arena ar;
    Ctx c{};
    BQ_TRY(begin(workspace, workspace_bytes, stream, &ar, &c, false, qr_split_elems(n)));
    TwoLevelWs w{};
    carve_two_level(ar, m, n, &w);
    size_t oz = ozaki_ws_bytes(kOuterQr, n, m, kOzPlanes);
    oz = std::max(oz, ozaki_ws_bytes(m, n, kOuterQr, kOzPlanes));
    oz = std::max(oz, ozaki_ws_bytes(64, n, m, kOzPlanes));
    oz += ozaki_split_reserve();
    c.oz_ws = ar.take<char>(oz);
    c.oz_bytes = oz;
    c.mixed = true;
    if (!ar.ok()) { set_error("workspace too small"); return BQRRP_ENOMEM; }
    init_status_small<<<1, 1, 0, c.stream>>>(c.st);
    BQ_LAUNCH_CHECK();
    BQ_TRY(geqrf_two_level(c, m, n, A, lda, tau, w));
    return finish(c);
}

size_t bqrrp_dgemm_workspace(int64_t M, int64_t N, int64_t K) {
    (void)M; (void)N; (void)K;
    Arena ar;
    Ctx c{};
    begin(nullptr, 0, nullptr, &ar, &c, true);
    return ar.off + 256;
}

int bqrrp_dgemm(char transa, char transb, int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t lda,
                const double* B, int64_t ldb, double beta, double* C, int64_t ldc, void* workspace,
                size_t workspace_bytes, void* stream) {
    set_error("");
    const bool ta = (transa == 'T' || transa == 't'), tb = (transb == 'T' || transb == 't');
    if (!ta && transa != 'N' && transa != 'n') return -1;
    if (!tb && transb != 'N' && transb != 'n') return -2;
    if (M < 0) return -3;
    if (N < 0) return -4;
    if (K < 0) return -5;
    if (lda < imax(1, ta ? K : M)) return -8;
    if (ldb < imax(1, tb ? N : K)) return -10;
    if (ldc < imax(1, M)) return -13;
    Ctx c{};
    BQ_TRY(current_device(&c.dev));
    c.stream = (cudaStream_t)stream;
    if (workspace && workspace_bytes >= bqrrp_dgemm_workspace(M, N, K)) {
        Arena ar;
        BQ_TRY(begin(workspace, workspace_bytes, stream, &ar, &c, false));
    }
    return dgemm(c, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
}

size_t bqrrp_dgemm_ozaki_workspace(int64_t M, int64_t N, int64_t K) {
    if (M < 0 || N < 0 || K < 0) return 0;
    return ozaki_ws_bytes(M, N, K, kOzPlanes) + 256;
}

int bqrrp_dgemm_ozaki(char transa, char transb, int64_t M, int64_t N, int64_t K, double alpha, const double* A,
                      int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc, void* workspace,
                      size_t workspace_bytes, void* stream) {
    set_error("");
    const bool ta = (transa == 'T' || transa == 't'), tb = (transb == 'T' || transb == 't');
    if (!ta && transa != 'N' && transa != 'n') return -1;
    if (!tb && transb != 'N' && transb != 'n') return -2;
    if (M < 0) return -3;
    if (N < 0) return -4;
    if (K < 0) return -5;
    if (lda < imax(1, ta ? K : M)) return -8;
    if (ldb < imax(1, tb ? N : K)) return -10;
    if (ldc < imax(1, M)) return -13;
    if (M == 0 || N == 0) return 0;
    if (workspace_bytes < bqrrp_dgemm_ozaki_workspace(M, N, K)) { set_error("workspace too small"); return BQRRP_ENOMEM; }
    Ctx c{};
    BQ_TRY(current_device(&c.dev));
    c.stream = (cudaStream_t)stream;
    char* base = (char*)(((uintptr_t)workspace + 255) & ~(uintptr_t)255);
    return ozaki_gemm(c, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, base,
                      workspace_bytes - (size_t)(base - (char*)workspace));
}

size_t bqrrp_sketch_apply_tc_workspace(int64_t d, int64_t m, int64_t n) {
    if (d < 0 || m < 0 || n < 0) return 0;
    return ozaki_sketch_ws_bytes(d, m, n) + 256;
}

int bqrrp_sketch_apply_tc(int64_t d, int64_t m, int64_t n, const double* A, int64_t lda, uint64_t seed, double* Msk,
                          int64_t ldsk, void* workspace, size_t workspace_bytes, void* stream) {
    set_error("");
    if (d < 0) return -1;
    if (m < 0) return -2;
    if (n < 0) return -3;
    if (lda < imax(1, m)) return -5;
    if (ldsk < imax(1, d)) return -8;
    if (d == 0 || n == 0) return 0;
    if (workspace_bytes < bqrrp_sketch_apply_tc_workspace(d, m, n)) { set_error("workspace too small"); return BQRRP_ENOMEM; }
    Ctx c{};
    BQ_TRY(current_device(&c.dev));
    c.stream = (cudaStream_t)stream;
    char* base = (char*)(((uintptr_t)workspace + 255) & ~(uintptr_t)255);
    return ozaki_sketch(c, d, m, n, seed, A, lda, Msk, ldsk, base, workspace_bytes - (size_t)(base - (char*)workspace));
}

double bqrrp_probe_fp64_peak(int iters, void* stream) {
    set_error("");
    Device dev;
    if (current_device(&dev)) return -1.0;
    cudaStream_t st = (cudaStream_t)stream;
    double* out = nullptr;
    // a one-double sink; this measurement helper is not part of the factorization
    if (cudaMallocAsync(&out, sizeof(double), st) != cudaSuccess) return -1.0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int blocks = dev.sms * 4, thr = 256;
    probe_dfma_kernel<<<blocks, thr, 0, st>>>(out, 16, 1.0000001, 1e-9);
    cudaEventRecord(e0, st);
    probe_dfma_kernel<<<blocks, thr, 0, st>>>(out, iters, 1.0000001, 1e-9);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(out, st);
    cudaStreamSynchronize(st);
    if (cudaGetLastError() != cudaSuccess || ms <= 0.f) return -1.0;
    const double flops = 2.0 * 32.0 * (double)iters * (double)blocks * (double)thr;
    return flops / ((double)ms * 1e-3) / 1e12;
}

}  // extern "C"
