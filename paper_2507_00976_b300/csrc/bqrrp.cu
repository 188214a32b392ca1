// bqrrp.cu -- host orchestrator of BQRRP (Alg. 1) and the C ABI.
//
// Per block (iteration i, s = i*b, c = min(n, s+b), w = c-s, N = n-s):
//   Alg. 2  : LU with partial pivoting of the sketch's transpose (lu panels +
//             GEMM), piv_transform, gather of the moved sketch columns,
//             Householder QR of the d x N sketch -> R^sk
//   tri_rank: k from diag(R^sk11) (device), permutation of A(:, s:) and J(s:)
//   host    : one read-back (k, zero-column flag, barrier status)
//   Alg. 3  : Pre = M Rsk11^-1, G = Pre^T Pre, Rchol = chol(G)
//   host    : one read-back (Cholesky breakdown lowers k)
//             Qc = Pre Rchol^-1, modified LU -> Y, U, D; T = -U D Y1^-T;
//             R11 = D Rchol Rsk(0:k, 0:w)
//   trailing: A(s:, c:) -= Y (T^T (Y^T A(s:, c:)))   (first k rows if k < w)
//   sketch  : Msk(0:w, c:) -= (Rsk11 R11^-1) R12      (Duersch-Gu update)
// All arithmetic runs in the library's kernels; the host only sequences
// launches and reads k.
#include <algorithm>
#include <atomic>
#include <climits>
#include <cstdarg>
#include <cstring>
#include <mutex>
#include <utility>
#include <vector>

#include "common.cuh"

namespace bq {

// ------------------------------------------------------------------ errors
namespace {
thread_local char g_err[512] = "";
}
void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}
const char* get_error() { return g_err; }

namespace {
std::atomic<long long> g_launches{0};

// Phase profiler: event pairs recorded on the factorization's stream,
// resolved after the call's final synchronization.
struct Profiler {
    std::mutex mu;
    bool on = false;
    double ms[BQRRP_NPHASES] = {0};
    double flops[BQRRP_NPHASES] = {0};
    long long calls = 0;
};
Profiler g_prof;
}  // namespace

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

bool profile_on() {
    std::lock_guard<std::mutex> lk(g_prof.mu);
    return g_prof.on;
}

void profile_add(const double* ms, const double* flops) {
    std::lock_guard<std::mutex> lk(g_prof.mu);
    for (int i = 0; i < BQRRP_NPHASES; ++i) {
        g_prof.ms[i] += ms[i];
        g_prof.flops[i] += flops[i];
    }
    g_prof.calls += 1;
}

// Per-call phase timer (active when the profiler is on): CUDA events around
// each phase, resolved after the call.  With the overlap schedule the phases
// of the side stream (LU, sketch QR, sketch update: lane 1) are timed on that
// stream, the others (lane 0) on the caller's stream, and the two lanes'
// spans overlap in time.
struct PhaseRec {
    bool on = false;
    bool split = false;                       // two lanes (overlap schedule)
    cudaStream_t st[2] = {nullptr, nullptr};
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> spans;
    double fl[BQRRP_NPHASES] = {0};
    int cur[2] = {-1, -1};
    cudaEvent_t cur_ev[2] = {nullptr, nullptr};
    std::vector<cudaEvent_t> events;   // created per call, destroyed in resolve()
    cudaEvent_t take() {
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        events.push_back(e);
        return e;
    }
    static int side_phase(int phase) { return phase == 1 || phase == 2 || phase == 6; }   // LUPP, SKQR, SKUPD
    void begin(int phase) {
        if (!on) return;
        const int l = split ? side_phase(phase) : 0;
        end_lane(l);
        cur[l] = phase;
        cur_ev[l] = take();
        cudaEventRecord(cur_ev[l], st[l]);
    }
    void end_lane(int l) {
        if (!on || cur[l] < 0) return;
        cudaEvent_t e = take();
        cudaEventRecord(e, st[l]);
        spans.push_back({cur[l], {cur_ev[l], e}});
        cur[l] = -1;
    }
    void end() {
        end_lane(0);
        end_lane(1);
    }
    void flops(int phase, double f) { if (on) fl[phase] += f; }
    void resolve() {   // after the streams have been synchronized
        if (!on) return;
        end();
        std::lock_guard<std::mutex> lk(g_prof.mu);
        for (auto& sp : spans) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, sp.second.first, sp.second.second) == cudaSuccess) g_prof.ms[sp.first] += t;
        }
        for (int i = 0; i < BQRRP_NPHASES; ++i) g_prof.flops[i] += fl[i];
        g_prof.calls += 1;
        for (cudaEvent_t e : events) cudaEventDestroy(e);
        events.clear();
    }
    ~PhaseRec() {
        for (cudaEvent_t e : events) cudaEventDestroy(e);
    }
};

int kernel_attrs(const void* fn, int smem_bytes, bool nonportable_cluster) {
    struct Rec {
        int dev;
        const void* fn;
        int smem;
        bool cluster;
    };
    static std::mutex mu;
    static std::vector<Rec> done;
    int id = 0;
    BQ_CUDA(cudaGetDevice(&id));
    std::lock_guard<std::mutex> lk(mu);
    for (const Rec& r : done)
        if (r.dev == id && r.fn == fn && r.smem >= smem_bytes && (r.cluster || !nonportable_cluster)) return 0;
    if (nonportable_cluster) BQ_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    BQ_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes));
    done.push_back(Rec{id, fn, smem_bytes, nonportable_cluster});
    return 0;
}

int current_device(Device* dev) {
    static std::mutex mu;
    static int cached_sms[64] = {0};
    int id = 0;
    BQ_CUDA(cudaGetDevice(&id));
    std::lock_guard<std::mutex> lk(mu);
    if (id < 0 || id >= 64) { set_error("device id out of range"); return BQRRP_ECUDA; }
    if (cached_sms[id] == 0) {
        int sms = 0;
        BQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, id));
        cached_sms[id] = sms;
    }
    dev->id = id;
    dev->sms = cached_sms[id];
    return 0;
}


namespace {

constexpr double kUnitRoundoff = 1.1102230246251565e-16;   // 2^-53

// ------------------------------------------------------------------ small kernels
__global__ void init_status_kernel(DevStatus* st) {
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

__global__ void iota_kernel(i64 n, i64* J) {
    const i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) J[i] = i;
}

__global__ void plus_one_kernel(i64 n, const i64* J, i64* jpvt) {
    const i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) jpvt[i] = J[i] + 1;
}

// tri_rank (Sec. 2.2, reading): k = largest j <= w with |Rsk(t,t)| > 10 d u r00
// for all t < j, r00 = |Rsk(0,0)| of the first iteration.
// With the FP32 sketch QRCP (fp32 != 0), R^sk carries FP32 rounding of the
// current block's own scale, so two more cuts apply, both at 10 d 2^-24:
// a diagonal entry that small relative to the block's |Rsk(0,0)| (a rank gap
// inside the block), and a whole block whose |Rsk(0,0)| is that small
// relative to the previous block's (a gap at a block boundary).  Below those
// ratios the FP32 factor cannot tell a column from rounding noise.
constexpr double kUnitRoundoff32 = 5.9604644775390625e-08;   // 2^-24
__global__ void __launch_bounds__(1024) tri_rank_kernel(DevStatus* st, const double* Rsk, i64 ldr, i64 w, i64 d,
                                                        int first, int fp32) {
    __shared__ double r00s, thr32s;
    __shared__ int firstbad, cross_bad;
    if (threadIdx.x == 0) {
        const double a00 = fabs(Rsk[0]);
        if (first) st->r00 = a00;
        r00s = st->r00;
        firstbad = INT_MAX;
        const double floor32 = 10.0 * (double)d * kUnitRoundoff32;
        thr32s = fp32 ? floor32 * a00 : 0.0;
        cross_bad = (fp32 && !first && !(a00 > floor32 * st->blk00)) ? 1 : 0;
        st->blk00 = a00;
    }
    __syncthreads();
    const double r00 = r00s;
    const double thr = fmax(10.0 * (double)d * kUnitRoundoff * r00, thr32s);
    const bool scale_ok = r00 > 0.0 && isfinite(r00);
    for (i64 t = threadIdx.x; t < w; t += blockDim.x) {
        const double v = Rsk[t + t * ldr];
        if (!isfinite(v) || !(fabs(v) > thr)) atomicMin(&firstbad, (int)t);
    }
    __syncthreads();
    if (threadIdx.x == 0) st->k = (scale_ok && !cross_bad) ? (firstbad < w ? (i64)firstbad : w) : 0;
}

// st->zero_col <- 1 if any entry of the column is nonzero (early-exit test)
__global__ void col_nonzero_kernel(i64 rows, const double* col, int* flag) {
    int nz = 0;
    for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += (i64)gridDim.x * blockDim.x)
        nz |= (col[i] != 0.0);
    nz = __syncthreads_or(nz);
    if (nz && threadIdx.x == 0) atomicOr(flag, 1);
}

// From the modified LU result in Y's top k x k block: U = triu, Tb = -U diag(D),
// and Y's top block becomes unit lower triangular.
__global__ void recon_split_kernel(i64 k, double* Y, i64 ldy, const double* D, double* U, double* Tb, i64 ldb) {
    const i64 total = k * k;
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (i64)gridDim.x * blockDim.x) {
        const i64 i = e % k, j = e / k;
        const double y = Y[i + j * ldy];
        if (i <= j) {
            U[i + j * ldb] = y;
            Tb[i + j * ldb] = -y * D[j];
            Y[i + j * ldy] = (i == j) ? 1.0 : 0.0;
        } else {
            U[i + j * ldb] = 0.0;
            Tb[i + j * ldb] = 0.0;
        }
    }
}

// Write the panel back into A (GEQP3 layout): rows 0..k-1 of the upper
// trapezoid get diag(D) * R11, column j < k below the diagonal gets Y(:, j);
// tau[j] = T(j, j).
__global__ void panel_writeback_kernel(i64 rows, i64 w, i64 k, double* A, i64 lda, const double* Y, i64 ldy,
                                       const double* R11, const double* D, const double* Tb, i64 ldb, double* tau) {
    const i64 total = rows * w;
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (i64)gridDim.x * blockDim.x) {
        const i64 i = e % rows, j = e / rows;
        if (i < k && i <= j) A[i + j * lda] = D[i] * R11[i + j * ldb];
        else if (j < k && i > j) A[i + j * lda] = Y[i + j * ldy];
    }
    const i64 t = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < k) tau[t] = Tb[t + t * ldb];
}

__global__ void zero_tail_kernel(i64 from, i64 to, double* tau) {
    const i64 i = from + (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < to) tau[i] = 0.0;
}

inline unsigned gblocks(const Ctx& c, i64 total) { return (unsigned)imax(1, imin(cdiv(total, 256), 8LL * c.dev.sms)); }

// The products of both mixed forms run on the tensor cores.
inline bool is_mixed(const bqrrp_opts& o) {
    return o.precision == BQRRP_PRECISION_MIXED || o.precision == BQRRP_PRECISION_MIXED_SKETCH32;
}

// ------------------------------------------------------------------ workspace plan
struct Bufs {
    DevStatus* st;
    double *Msk, *Xlu, *Ub, *stage, *Ypan, *Vqr, *Tqr, *W, *W2, *G, *U, *Tb, *R11, *Z, *D, *sktau, *splitk, *coop;
    i64 *ipiv, *Jsk, *pos, *src, *cnt, *J, *Jstage;
    char* sparse_ws;
    char* oz_ws;
    size_t sparse_bytes, splitk_elems, coop_elems, oz_bytes;
    i64 max_moved, ldst, bb, wrows;
};

void carve(Arena& ar, i64 m, i64 n, i64 b, i64 d, const bqrrp_opts& o, Bufs* B) {
    const i64 bb = imax(1, imin(b, n));
    B->bb = bb;
    B->max_moved = imax(1, imin(n, 2 * imin(d, n)));
    B->ldst = imax(m, d);
    B->wrows = imax(bb, 64);
    B->st = ar.take<DevStatus>(1);
    B->Msk = ar.take<double>((size_t)d * n);
    B->Xlu = ar.take<double>((size_t)d * n);
    B->Ub = ar.take<double>((size_t)d * imin(d, n));
    B->stage = ar.take<double>((size_t)B->ldst * B->max_moved);
    B->Ypan = ar.take<double>((size_t)m * bb);
    B->Vqr = ar.take<double>((size_t)imax(m, d) * 64);
    B->Tqr = ar.take<double>(64 * 64);
    B->W = ar.take<double>((size_t)B->wrows * n);
    B->W2 = ar.take<double>((size_t)B->wrows * n);
    B->G = ar.take<double>((size_t)bb * bb);
    B->U = ar.take<double>((size_t)bb * bb);
    B->Tb = ar.take<double>((size_t)bb * bb);
    B->R11 = ar.take<double>((size_t)bb * bb);
    B->Z = ar.take<double>((size_t)bb * bb);
    B->D = ar.take<double>((size_t)bb);
    B->sktau = ar.take<double>((size_t)imax(d, n));
    // split-K partials: the trailing product W = Y^T C has only b/64 tile rows,
    // so balancing it over the SMs takes a few splits of b x n partials (2048 n
    // doubles: 8 splits at b = 256; larger b has enough tiles to need fewer)
    B->splitk_elems = (size_t)imax(imax(16 * bb * bb, (i64)1 << 22), 2048 * n);
    B->splitk = ar.take<double>(B->splitk_elems);
    coop_scratch_elems(64, 148, &B->coop_elems);
    B->coop = ar.take<double>(B->coop_elems);
    B->ipiv = ar.take<i64>((size_t)d);
    B->Jsk = ar.take<i64>((size_t)n);
    B->pos = ar.take<i64>((size_t)B->max_moved);
    B->src = ar.take<i64>((size_t)B->max_moved);
    B->cnt = ar.take<i64>(4);
    B->J = ar.take<i64>((size_t)n);
    B->Jstage = ar.take<i64>((size_t)B->max_moved);
    B->oz_bytes = 0;
    B->oz_ws = nullptr;
    if (is_mixed(o)) {
        size_t z = ozaki_ws_bytes(bb, n, m, kOzPlanes);         // W = Y^T C
        z = std::max(z, ozaki_ws_bytes(m, n, bb, kOzPlanes));   // C -= Y W2
        z = std::max(z, ozaki_ws_bytes(bb, n, bb, kOzPlanes));  // W2 = T^T W
        if (o.sketch_kind == BQRRP_SKETCH_DENSE) z = std::max(z, ozaki_sketch_ws_bytes(d, m, n));   // S A
        z = std::max(z, ozaki_ws_bytes(d, n, 64, kOzPlanes));   // LU trailing updates
        z = std::max(z, ozaki_ws_bytes(d, n, d, kOzPlanes));    // R^sk = R1 L^T
        z = std::max(z, ozaki_ws_bytes(64, n, m, kOzPlanes));           // Householder panel updates (HQR panel)
        z += ozaki_split_reserve();   // the split-K sums of any smaller product (the panel's Gram among them)
        B->oz_bytes = z;
        B->oz_ws = ar.take<char>(z);
    } else if (o.sketch_kind == BQRRP_SKETCH_DENSE) {
        // the FP64 form's dense sketch also runs as exact slice products (S*A
        // to FP64 accuracy on the tensor cores)
        B->oz_bytes = ozaki_sketch_ws_bytes(d, m, n);
        B->oz_ws = ar.take<char>(B->oz_bytes);
    }
    B->sparse_bytes = 0;
    B->sparse_ws = nullptr;
    if (o.sketch_kind == BQRRP_SKETCH_SPARSE) {
        B->sparse_bytes = sketch_sparse_ws(d, m, o.sketch_nnz);
        B->sparse_ws = ar.take<char>(B->sparse_bytes);
    }
}

bqrrp_opts defaults(const bqrrp_opts* o) {
    bqrrp_opts r{};
    r.sketch_kind = BQRRP_SKETCH_DENSE;
    r.sketch_nnz = 8;
    r.panel_kind = BQRRP_PANEL_CHOLQR;
    if (o) {
        r.sketch_kind = o->sketch_kind;
        r.sketch_nnz = o->sketch_nnz > 0 ? o->sketch_nnz : 8;
        r.panel_kind = o->panel_kind;
        r.precision = o->precision;
        r.schedule = o->schedule;
        r.panel_tc = o->panel_tc;
    }
    return r;
}

int check_opts(const bqrrp_opts* o, i64 d) {
    if (!o) return 0;
    if (o->sketch_kind != BQRRP_SKETCH_DENSE && o->sketch_kind != BQRRP_SKETCH_SPARSE) return 1;
    if (o->panel_kind != BQRRP_PANEL_CHOLQR && o->panel_kind != BQRRP_PANEL_HQR) return 1;
    if (o->sketch_kind == BQRRP_SKETCH_SPARSE) {
        const i64 nnz = o->sketch_nnz > 0 ? o->sketch_nnz : 8;
        if (nnz > d || nnz > 64) return 1;
    }
    if (o->precision != BQRRP_PRECISION_FP64 && o->precision != BQRRP_PRECISION_MIXED &&
        o->precision != BQRRP_PRECISION_MIXED_SKETCH32)
        return 1;
    if (o->schedule != BQRRP_SCHEDULE_OVERLAP && o->schedule != BQRRP_SCHEDULE_SERIAL) return 1;
    if (o->panel_tc != 0 && o->panel_tc != 1) return 1;
    if (o->panel_tc == 1 && o->precision == BQRRP_PRECISION_FP64) return 1;   // slice products need a mixed form
    for (int i = 0; i < 2; ++i)
        if (o->reserved[i] != 0) return 1;
    return 0;
}

int read_status(const Ctx& c, DevStatus* host) {
    BQ_CUDA(cudaMemcpyAsync(host, c.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, c.stream));
    BQ_CUDA(cudaStreamSynchronize(c.stream));
    if (host->err_timeout) {
        set_error("a bounded cross-CTA wait timed out");
        return BQRRP_ETIMEOUT;
    }
    return 0;
}

}  // namespace

// Alg. 3 on one panel Mp (rows x w, ld ldm) with preconditioner Rsk (upper
// triangle, ld ldr): Pre = Mp(:, 0:k) Rsk11^-1 in Y, G = Pre^T Pre, Rchol =
// chol(G) (a breakdown lowers *k), Qc = Pre Rchol^-1, modified LU of Qc (Y
// unit lower trapezoidal, U, D; only the top k rows of Qc are formed, the
// rows below come from one solve with U Rchol), T = -U D Y1^-T in Tb, R11 = D Rchol
// Rsk(0:k, 0:w); R11 and the reflectors are written into Mp and diag(T) into
// tau.  Y and Tb stay valid for the trailing update.  Synchronizes the stream
// once (to read the Cholesky status).
int cholqr_panel_steps(const Ctx& c, i64 rows, i64 w, i64* kio, double* Mp, i64 ldm, const double* Rsk, i64 ldr,
                       double* Y, i64 ldy, double* G, double* U, double* Tb, double* R11, double* D, i64 ldb,
                       double* tau) {
    i64 k = *kio;
    View Yv = colmajor(Y, ldy);
    BQ_TRY(copy_mat(c, rows, k, Mp, ldm, Y, ldy));
    BQ_TRY(trsm_ru_tall(c, rows, k, Rsk, ldr, Y, ldy));                                 // Pre = M Rsk11^-1
    BQ_TRY(pgemm(c, true, false, k, k, rows, 1.0, Y, ldy, Y, ldy, 0.0, G, ldb, kGemmCUpper));   // G = Pre^T Pre
    BQ_CUDA(cudaMemsetAsync(&c.st->potrf_info, 0x7f, sizeof(int), c.stream));         // "no failure"
    BQ_TRY(potrf_u(c, k, G, ldb));                                                     // Rchol
    DevStatus hs{};
    BQ_TRY(read_status(c, &hs));
    if (hs.potrf_info < k) {
        k = hs.potrf_info;   // Cholesky breakdown: the block's numerical rank is lower
        *kio = k;
        if (k <= 0) return 0;
    }
    // The modified LU of Qc = Pre Rchol^-1 factors its top k x k block,
    // Qc1 - S = Y1 U; the rows below follow from Qc2 = Y2 U, so
    // Y2 = Pre2 Rchol^-1 U^-1 = Pre2 (U Rchol)^-1: one tall solve with the
    // k x k upper triangle U Rchol instead of two (Rchol^-1, then U^-1)
    BQ_TRY(trsm_ru(c, k, k, colmajor(G, ldb), Yv, false));                            // Qc1 = Pre1 Rchol^-1
    BQ_TRY(modlu(c, k, k, Y, ldy, D));                                                 // Qc1 - S = Y1 U
    recon_split_kernel<<<gblocks(c, k * k), 256, 0, c.stream>>>(k, Y, ldy, D, U, Tb, ldb);
    BQ_LAUNCH_CHECK();
    if (rows > k) {
        BQ_TRY(dgemm(c, false, false, k, k, k, 1.0, U, ldb, G, ldb, 0.0, R11, ldb, kGemmAUpper));   // U Rchol
        BQ_TRY(trsm_ru_tall(c, rows - k, k, R11, ldb, Y + k, ldy));                             // Y2
    }
    BQ_TRY(trsm_ru(c, k, k, Yv.t(), colmajor(Tb, ldb), true));                        // T = -U S Y1^-T
    BQ_TRY(dgemm(c, false, false, k, w, k, 1.0, G, ldb, Rsk, ldr, 0.0, R11, ldb));     // Rchol Rsk(0:k, 0:w)
    panel_writeback_kernel<<<gblocks(c, rows * w), 256, 0, c.stream>>>(rows, w, k, Mp, ldm, Y, ldy, R11, D, Tb, ldb,
                                                                       tau);
    BQ_LAUNCH_CHECK();
    *kio = k;
    return 0;
}

namespace {

// ------------------------------------------------------------------ the factorization
inline double geqrf_flops(double r, double c) {   // LAWN 41 count of GEQRF on r x c
    return r >= c ? 2.0 * r * c * c - 2.0 * c * c * c / 3.0 : 2.0 * c * r * r - 2.0 * r * r * r / 3.0;
}

inline double lupp_flops(double N, double d) {      // GETRF on N x d: sum_j (N-j-1)(1 + 2(d-j-1))
    const double s = N < d ? N : d;
    double f = 0.0;
    for (double j = 0; j < s; j += 1.0) f += (N - j - 1.0) * (1.0 + 2.0 * (d - j - 1.0));
    return f;
}

// Pinned host buffers of the host entry point.  A comes in on the copy
// stream; with the dense FP64 sketch it comes in two column halves, the
// second copied while the first is sketched.  Every column block goes back
// on the copy stream as soon as its iteration has finished it, so the copy
// back overlaps the rest of the factorization: after the iteration on
// columns [s, c), later iterations permute, update and read only columns >= c.
struct HostIO {
    double* A_host;     // in: A; out: R and the reflectors (ld lda_host); pinned
    i64 lda_host;
    cudaStream_t cs;    // copy stream
    std::vector<cudaEvent_t>* events;
    i64 copied = 0;     // columns [0, copied) queued for the copy back
    int record(cudaStream_t st, cudaEvent_t* ev) {
        BQ_CUDA(cudaEventCreateWithFlags(ev, cudaEventDisableTiming));
        events->push_back(*ev);
        BQ_CUDA(cudaEventRecord(*ev, st));
        return 0;
    }
    // copy columns [c0, c0 + nc) of A in; the compute stream waits for them
    int bring_in(const Ctx& c, double* A, i64 m, i64 lda, i64 c0, i64 nc) {
        BQ_CUDA(cudaMemcpy2DAsync(A + c0 * lda, sizeof(double) * lda, A_host + c0 * lda_host,
                                  sizeof(double) * lda_host, sizeof(double) * m, nc, cudaMemcpyHostToDevice, cs));
        cudaEvent_t ev;
        BQ_TRY(record(cs, &ev));
        BQ_CUDA(cudaStreamWaitEvent(c.stream, ev, 0));
        return 0;
    }
    // queue the copy back of columns [copied, upto) once the compute stream is past this point
    int send_back(const Ctx& c, const double* A, i64 m, i64 lda, i64 upto) {
        if (upto <= copied) return 0;
        cudaEvent_t ev;
        BQ_TRY(record(c.stream, &ev));
        BQ_CUDA(cudaStreamWaitEvent(cs, ev, 0));
        BQ_CUDA(cudaMemcpy2DAsync(A_host + copied * lda_host, sizeof(double) * lda_host, A + copied * lda,
                                  sizeof(double) * lda, sizeof(double) * m, upto - copied, cudaMemcpyDeviceToHost, cs));
        copied = upto;
        return 0;
    }
};

// The side stream of the overlap schedule: highest priority, non-blocking,
// created and synchronized per call.
struct SideStream {
    cudaStream_t st = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int open() {
        int least = 0, greatest = 0;
        BQ_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        BQ_CUDA(cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, greatest));
        BQ_CUDA(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
        BQ_CUDA(cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming));
        return 0;
    }
    ~SideStream() {
        if (st) {
            cudaStreamSynchronize(st);
            cudaStreamDestroy(st);
        }
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
    }
};

int factor_impl(i64 m, i64 n, double* A, i64 lda, i64 b, i64 d, uint64_t seed, i64* jpvt, double* tau, i64* rank,
                const bqrrp_opts& o, const Bufs& B, Ctx& c, PhaseRec& pr, HostIO* io) {
    enum { P_SKETCH = 0, P_LUPP, P_SKQR, P_PERM, P_PANEL, P_TRAIL, P_SKUPD, P_OTHER };
    DevStatus hs{};
    pr.begin(P_OTHER);
    init_status_kernel<<<1, 1, 0, c.stream>>>(B.st);
    BQ_LAUNCH_CHECK();
    const bool dense_in = o.sketch_kind == BQRRP_SKETCH_DENSE;   // A may come in by halves (see below)
    if (io && !dense_in) BQ_TRY(io->bring_in(c, A, m, lda, 0, n));
    if (!io || !dense_in) {
        // NaN/Inf in A -> BQRRP_ENUMERIC before anything is written
        BQ_TRY(any_nonfinite(c, m, n, A, lda, &B.st->a_nonfinite));
        BQ_TRY(read_status(c, &hs));
        if (hs.a_nonfinite) {
            set_error("A contains NaN or Inf");
            return BQRRP_ENUMERIC;
        }
    }
    BQ_CUDA(cudaMemsetAsync(tau, 0, sizeof(double) * (size_t)n, c.stream));
    iota_kernel<<<(unsigned)cdiv(n, 256), 256, 0, c.stream>>>(n, B.J);
    BQ_LAUNCH_CHECK();

    // Alg. 1: sketch Msk = S * A (d x n)
    pr.begin(P_SKETCH);
    if (io && dense_in) {
        // A from the host in two column halves; each half is checked and
        // sketched once it has arrived (every sketch column depends only on
        // its own column of A, so the bits are those of one call).  The
        // sketch writes only Msk, so the NaN/Inf result, read after it, still
        // comes before anything of A is written.
        const i64 half = n >= 1024 ? cdiv(cdiv(n, 2), 64) * 64 : n;
        for (i64 c0 = 0; c0 < n; c0 += half) {
            const i64 nc0 = imin(half, n - c0);
            BQ_TRY(io->bring_in(c, A, m, lda, c0, nc0));
            BQ_TRY(any_nonfinite(c, m, nc0, A + c0 * lda, lda, &B.st->a_nonfinite));
            BQ_TRY(ozaki_sketch(c, d, m, nc0, seed, A + c0 * lda, lda, B.Msk + c0 * d, d, B.oz_ws, B.oz_bytes));
        }
        pr.flops(P_SKETCH, 2.0 * d * m * n);
        pr.begin(P_OTHER);
        BQ_TRY(read_status(c, &hs));
        if (hs.a_nonfinite) {
            set_error("A contains NaN or Inf");
            return BQRRP_ENUMERIC;
        }
    } else if (o.sketch_kind == BQRRP_SKETCH_DENSE) {
        BQ_TRY(ozaki_sketch(c, d, m, n, seed, A, lda, B.Msk, d, B.oz_ws, B.oz_bytes));
        pr.flops(P_SKETCH, 2.0 * d * m * n);
    } else {
        BQ_TRY(sketch_sparse_apply(c, d, m, n, seed, o.sketch_nnz, A, lda, B.Msk, d, B.sparse_ws, B.sparse_bytes));
        pr.flops(P_SKETCH, 2.0 * (double)o.sketch_nnz * m * n);
    }

    // Schedule: a reordering of independent steps of Alg. 1.  Alg. 2 of the
    // next block needs only the sketch update, and that needs only R11 and
    // the first k rows of the updated trailing block (R12).  So the trailing
    // update forms those rows first; with the overlap schedule the sketch
    // update and the next block's Alg. 2 then run on a high-priority side
    // stream while the rest of the trailing update (rows k.. of C -= Y W2)
    // runs on the caller's stream, and the latency-bound LU and small QR of
    // the sketch take the FP64 cycles the trailing GEMM leaves.  Both
    // schedules launch the same kernels on the same data, so their results
    // are identical bit for bit.  The mixed form and the Householder panel use
    // the serial schedule.
    SideStream side;
    const bool overlap = o.schedule == BQRRP_SCHEDULE_OVERLAP && o.precision == BQRRP_PRECISION_FP64 &&
                         o.panel_kind == BQRRP_PANEL_CHOLQR;
    Ctx cs = c;   // Alg. 2 and the sketch update
    if (overlap) {
        BQ_TRY(side.open());
        cs.stream = side.st;
        pr.end();
        pr.split = true;
        pr.st[1] = side.st;
    }
    auto fork = [&]() -> int {   // side stream after the caller's stream's work so far
        if (!overlap) return 0;
        BQ_CUDA(cudaEventRecord(side.ev_fork, c.stream));
        BQ_CUDA(cudaStreamWaitEvent(cs.stream, side.ev_fork, 0));
        return 0;
    };
    auto join = [&]() -> int {   // caller's stream after the side stream's work so far
        if (!overlap) return 0;
        pr.end_lane(0);   // the wait is no phase of the caller's stream
        BQ_CUDA(cudaEventRecord(side.ev_join, cs.stream));
        BQ_CUDA(cudaStreamWaitEvent(c.stream, side.ev_join, 0));
        return 0;
    };
    // Alg. 2 on the sketch columns it*b..n-1: LUPP of Ssk^T, piv_transform,
    // R^sk from the LU factors (Householder QR of U^T, then R1 L^T), tri_rank
    auto alg2 = [&](i64 it) -> int {
        const i64 s = it * b, N = n - s, w = imin(n, s + b) - s;
        double* Ssk = B.Msk + s * d;
        pr.begin(P_LUPP);
        BQ_CUDA(cudaMemsetAsync(&B.st->sk_nonfinite, 0, sizeof(int), cs.stream));
        BQ_CUDA(cudaMemsetAsync(&B.st->zero_col, 0, sizeof(int), cs.stream));
        BQ_TRY(any_nonfinite(cs, d, N, Ssk, d, &B.st->sk_nonfinite));
        BQ_CUDA(cudaMemcpy2DAsync(B.Xlu, sizeof(double) * d, Ssk, sizeof(double) * d, sizeof(double) * d, N,
                                  cudaMemcpyDeviceToDevice, cs.stream));
        const i64 steps = imin(N, d);
        BQ_TRY(getrf_pivots(cs, N, d, B.Xlu, d, B.ipiv));
        BQ_TRY(piv_transform_moved(cs, N, steps, B.ipiv, B.Jsk, &B.st->sk_nonfinite, B.pos, B.src, B.cnt));
        pr.flops(P_LUPP, lupp_flops((double)N, (double)d));
        pr.begin(P_SKQR);
        // scratch of the blocked-QR fallback: W and the column stage, which the
        // rest of the trailing update (Y, W2, C) does not touch
        BQ_TRY(rsk_from_lu(cs, d, N, B.Xlu, d, Ssk, d, B.Ub, B.sktau, B.Vqr, B.Tqr, B.W, B.stage));
        tri_rank_kernel<<<1, 1024, 0, cs.stream>>>(B.st, Ssk, d, w, d, it == 0 ? 1 : 0, cs.sketch32 ? 1 : 0);
        BQ_LAUNCH_CHECK();
        pr.flops(P_SKQR, geqrf_flops((double)d, (double)N));
        if (overlap) pr.end_lane(1);
        return 0;
    };

    BQ_TRY(fork());
    BQ_TRY(alg2(0));
    i64 ell = 0;
    for (i64 it = 0;; ++it) {
        const i64 s = it * b;
        const i64 cend = imin(n, s + b);
        const i64 w = cend - s;
        const i64 N = n - s;
        const i64 rows = m - s;
        double* Ssk = B.Msk + s * d;
        const i64 mm = imin(N, 2 * imin(N, d));

        // ---- permute A(:, s:) (all m rows: R rows and working rows, merged) and J(s:)
        BQ_TRY(join());
        pr.begin(P_PERM);
        BQ_TRY(gather_cols(c, m, A + s * lda, lda, B.pos, B.src, B.cnt, mm, B.stage, B.ldst));
        BQ_TRY(gather_idx(c, B.J + s, B.pos, B.src, B.cnt, mm, B.Jstage));
        col_nonzero_kernel<<<gblocks(c, rows), 256, 0, c.stream>>>(rows, A + s + s * lda, &B.st->zero_col);
        BQ_LAUNCH_CHECK();
        pr.begin(P_OTHER);
        BQ_TRY(read_status(c, &hs));
        if (!hs.zero_col) { ell = s; break; }   // first permuted working column is zero
        i64 k = hs.k;
        if (k <= 0) { ell = s; break; }

        double* Ap = A + s + s * lda;   // panel / working block origin
        const i64 nc = n - cend;
        // ---- sketch update, Msk(0:w, c:) = Rsk12 - (Rsk11 R11^-1) R12 (Rsk22 stays),
        // then Alg. 2 of the next block
        auto next_block = [&]() -> int {
            BQ_TRY(fork());
            pr.begin(P_SKUPD);
            BQ_TRY(copy_triu(cs, w, w, Ssk, d, B.Z, B.bb));
            BQ_TRY(trsm_ru(cs, w, w, colmajor(Ap, lda), colmajor(B.Z, B.bb), false));
            BQ_TRY(pgemm(cs, false, false, w, nc, w, -1.0, B.Z, B.bb, A + s + cend * lda, lda, 1.0,
                         B.Msk + cend * d, d));
            pr.flops(P_SKUPD, (double)w * w * w + 2.0 * (double)w * w * nc);
            return alg2(it + 1);
        };
        bool more = false;
        if (o.panel_kind == BQRRP_PANEL_HQR) {
            // Householder QR of all w panel columns, reflectors applied to the
            // whole trailing block; only the first k are kept (Sec. 3.5).
            pr.begin(P_PANEL);
            BQ_TRY(geqrf_blocked(c, rows, N, Ap, lda, tau + s, B.Vqr, B.Tqr, B.W, B.W2, 64, w));
            if (k < w) {
                zero_tail_kernel<<<(unsigned)cdiv(w, 256), 256, 0, c.stream>>>(s + k, s + w, tau);
                BQ_LAUNCH_CHECK();
            }
            pr.flops(P_PANEL, geqrf_flops((double)rows, (double)w) + 4.0 * rows * w * nc);
            more = cend < n && k == w;
            if (more) BQ_TRY(next_block());
        } else {
            // ---- Alg. 3: precondition, Cholesky QR, reconstruction, R11 (written back)
            pr.begin(P_PANEL);
            // With the FP32 sketch QRCP, R11's columns k.. (when the block keeps
            // k < w columns) would come from the FP32 R^sk; they are formed
            // instead from the panel's own columns, saved here, as Q^T A.
            if (c.sketch32)
                BQ_CUDA(cudaMemcpy2DAsync(B.stage, sizeof(double) * B.ldst, Ap, sizeof(double) * lda,
                                          sizeof(double) * rows, w, cudaMemcpyDeviceToDevice, c.stream));
            {
                // The panel stays in FP64 unless opts.panel_tc asks for its Gram
                // and its tall solves' block updates as FP64-accurate slice
                // products (the Cholesky factor, the reconstruction's LU, tau and
                // R stay in FP64 either way).
                Ctx cp = c;
                cp.mixed = c.mixed && o.panel_tc == 1;
                BQ_TRY(cholqr_panel_steps(cp, rows, w, &k, Ap, lda, Ssk, d, B.Ypan, m, B.G, B.U, B.Tb, B.R11, B.D,
                                          B.bb, tau + s));
            }
            if (c.sketch32 && k > 0 && k < w) {
                // R(0:k, k:w) = the first k rows of (I - Y T Y^T)^T A(:, k:w), in FP64
                double* Sk0 = B.stage + k * B.ldst;
                BQ_TRY(dgemm(c, true, false, k, w - k, rows, 1.0, B.Ypan, m, Sk0, B.ldst, 0.0, B.W, B.wrows));
                BQ_TRY(dgemm(c, true, false, k, w - k, k, 1.0, B.Tb, B.bb, B.W, B.wrows, 0.0, B.W2, B.wrows));
                BQ_TRY(dgemm(c, false, false, k, w - k, k, -1.0, B.Ypan, m, B.W2, B.wrows, 1.0, Sk0, B.ldst));
                BQ_CUDA(cudaMemcpy2DAsync(Ap + k * lda, sizeof(double) * lda, Sk0, sizeof(double) * B.ldst,
                                          sizeof(double) * k, w - k, cudaMemcpyDeviceToDevice, c.stream));
            }
            {
                const double r = (double)rows, kk = (double)k;
                // the method's count: preconditioner TRSM, Gram (SYRK), TRSM, reconstruction:
                // rows*k^2 FLOPs each (summed over the loop, 2 b n^2; the last two are one
                // solve here); + Cholesky, T (k^3/3 each) and R11 (2 k^2 w)
                pr.flops(P_PANEL, 4.0 * r * kk * kk + kk * kk * kk * (1.0 / 3.0 + 1.0 / 3.0) + 2.0 * kk * kk * w);
            }
            if (k <= 0) { ell = s; break; }
            more = cend < n && k == w;
            // ---- trailing update with the block reflector (I - Y T Y^T)^T
            double* C = A + s + cend * lda;
            const i64 keep = (k == w) ? rows : k;
            if (nc > 0 && is_mixed(o)) {
                pr.begin(P_TRAIL);
                BQ_TRY(ozaki_gemm(c, true, false, k, nc, rows, 1.0, B.Ypan, m, C, lda, 0.0, B.W, B.wrows,
                                  B.oz_ws, B.oz_bytes));
                BQ_TRY(ozaki_gemm(c, true, false, k, nc, k, 1.0, B.Tb, B.bb, B.W, B.wrows, 0.0, B.W2, B.wrows,
                                  B.oz_ws, B.oz_bytes));
                BQ_TRY(ozaki_gemm(c, false, false, keep, nc, k, -1.0, B.Ypan, m, B.W2, B.wrows, 1.0, C, lda,
                                  B.oz_ws, B.oz_bytes));
                if (more) BQ_TRY(next_block());
            } else if (nc > 0) {
                pr.begin(P_TRAIL);
                BQ_TRY(dgemm(c, true, false, k, nc, rows, 1.0, B.Ypan, m, C, lda, 0.0, B.W, B.wrows));
                BQ_TRY(dgemm(c, true, false, k, nc, k, 1.0, B.Tb, B.bb, B.W, B.wrows, 0.0, B.W2, B.wrows));
                // R12 rows first: the sketch update reads only these
                BQ_TRY(dgemm(c, false, false, k, nc, k, -1.0, B.Ypan, m, B.W2, B.wrows, 1.0, C, lda));
                if (more) BQ_TRY(next_block());
                if (keep > k) {
                    // rows k.. with no split-K, so that it shares no scratch with Alg. 2 on the side stream
                    pr.begin(P_TRAIL);
                    Ctx c3 = c;
                    c3.splitk = nullptr;
                    BQ_TRY(dgemm(c3, false, false, keep - k, nc, k, -1.0, B.Ypan + k, m, B.W2, B.wrows, 1.0, C + k,
                                 lda));
                }
            }
            if (nc > 0)
                pr.flops(P_TRAIL, 2.0 * (double)k * nc * (double)rows + 2.0 * (double)k * k * nc +
                                      2.0 * (double)keep * nc * k);
        }
        if (!more) { ell = s + k; break; }
        if (io) BQ_TRY(io->send_back(c, A, m, lda, cend));   // block [s, cend) is final
    }
    pr.begin(P_OTHER);
    if (io) BQ_TRY(io->send_back(c, A, m, lda, n));          // the rest, after the last iteration
    plus_one_kernel<<<(unsigned)cdiv(n, 256), 256, 0, c.stream>>>(n, B.J, jpvt);
    BQ_LAUNCH_CHECK();
    BQ_TRY(read_status(c, &hs));
    pr.end();
    *rank = ell;
    return 0;
}

int make_ctx(void* stream, Ctx* c) {
    BQ_TRY(current_device(&c->dev));
    c->stream = (cudaStream_t)stream;
    return 0;
}

}  // namespace
}  // namespace bq

using namespace bq;

extern "C" {

const char* bqrrp_last_error(void) { return get_error(); }

void bqrrp_profile_enable(int on) {
    std::lock_guard<std::mutex> lk(g_prof.mu);
    g_prof.on = on != 0;
}

void bqrrp_profile_reset(void) {
    std::lock_guard<std::mutex> lk(g_prof.mu);
    for (int i = 0; i < BQRRP_NPHASES; ++i) { g_prof.ms[i] = 0.0; g_prof.flops[i] = 0.0; }
    g_prof.calls = 0;
}

int bqrrp_profile_read(bqrrp_profile* out) {
    if (!out) return -1;
    std::lock_guard<std::mutex> lk(g_prof.mu);
    for (int i = 0; i < BQRRP_NPHASES; ++i) { out->ms[i] = g_prof.ms[i]; out->flops[i] = g_prof.flops[i]; }
    out->calls = g_prof.calls;
    return 0;
}

int64_t bqrrp_launch_counter(void) { return g_launches.load(); }

const char* bqrrp_version(void) { return "bqrrp-b300 0.1 (sm_103a, FP64 SIMT)"; }

size_t bqrrp_workspace_query(int64_t m, int64_t n, int64_t b, int64_t d, const bqrrp_opts* opts) {
    if (m < 0 || n < 0 || m < n || b < 1 || d < b || check_opts(opts, d)) return 0;
    bqrrp_opts o = defaults(opts);
    Arena ar;
    ar.dry = true;
    Bufs B{};
    carve(ar, m, imax(n, 1), b, d, o, &B);
    return ar.off + 256;
}

}  // extern "C"

namespace bq {
namespace {

int factor_entry(int64_t m, int64_t n, double* A, int64_t lda, int64_t b, int64_t d, uint64_t seed, int64_t* jpvt,
                 double* tau, int64_t* rank, const bqrrp_opts* opts, void* workspace, size_t workspace_bytes,
                 void* stream, HostIO* io) {
    if (rank) *rank = -1;
    if (m < 0 || m < n) { set_error("m must satisfy m >= n >= 0"); return -1; }
    if (n < 0) return -2;
    if (lda < imax(1, m)) { set_error("lda < max(1, m)"); return -4; }
    if (b < 1) { set_error("b < 1"); return -5; }
    if (d < b) { set_error("d < b"); return -6; }
    if (!rank) return -10;
    if (check_opts(opts, d)) { set_error("invalid opts"); return -11; }
    if (n == 0) { *rank = 0; return 0; }
    if (!A) return -3;
    if (!jpvt) return -8;
    if (!tau) return -9;
    if (!workspace) return -12;
    const size_t need = bqrrp_workspace_query(m, n, b, d, opts);
    if (workspace_bytes < need) {
        set_error("workspace has %zu bytes, needs %zu", workspace_bytes, need);
        return BQRRP_ENOMEM;
    }
    bqrrp_opts o = defaults(opts);
    Arena ar;
    ar.base = (char*)(((uintptr_t)workspace + 255) & ~(uintptr_t)255);
    ar.cap = workspace_bytes - (size_t)(ar.base - (char*)workspace);
    Bufs B{};
    carve(ar, m, n, b, d, o, &B);
    if (!ar.ok()) { set_error("workspace too small after alignment"); return BQRRP_ENOMEM; }
    Ctx c{};
    BQ_TRY(make_ctx(stream, &c));
    c.st = B.st;
    c.splitk = B.splitk;
    c.splitk_elems = B.splitk_elems;
    c.coop = B.coop;
    c.coop_elems = B.coop_elems;
    c.mixed = is_mixed(o);
    c.sketch32 = (o.precision == BQRRP_PRECISION_MIXED_SKETCH32);
    c.oz_ws = B.oz_ws;
    c.oz_bytes = B.oz_bytes;
    i64 r = 0;
    PhaseRec pr;
    {
        std::lock_guard<std::mutex> lk(g_prof.mu);
        pr.on = g_prof.on;
    }
    pr.st[0] = pr.st[1] = c.stream;
    const int rc = factor_impl(m, n, A, lda, b, d, seed, jpvt, tau, &r, o, B, c, pr, io);
    if (rc == 0) {
        *rank = r;
        pr.resolve();
    }
    return rc;
}

}  // namespace
}  // namespace bq

extern "C" {

int bqrrp_factor(int64_t m, int64_t n, double* A, int64_t lda, int64_t b, int64_t d, uint64_t seed, int64_t* jpvt,
                 double* tau, int64_t* rank, const bqrrp_opts* opts, void* workspace, size_t workspace_bytes,
                 void* stream) {
    set_error("");
    return factor_entry(m, n, A, lda, b, d, seed, jpvt, tau, rank, opts, workspace, workspace_bytes, stream, nullptr);
}

size_t bqrrp_workspace_query_host(int64_t m, int64_t n, int64_t b, int64_t d, const bqrrp_opts* opts) {
    const size_t base = bqrrp_workspace_query(m, n, b, d, opts);
    if (!base) return 0;
    const size_t am = ((size_t)m * (size_t)n * 8 + 255) & ~(size_t)255;
    const size_t jv = ((size_t)n * 8 + 255) & ~(size_t)255;
    return base + am + 2 * jv + 512;
}

int bqrrp_factor_host(int64_t m, int64_t n, double* A_host, int64_t lda, int64_t b, int64_t d, uint64_t seed,
                      int64_t* jpvt_host, double* tau_host, int64_t* rank, const bqrrp_opts* opts, void* workspace,
                      size_t workspace_bytes, void* stream) {
    set_error("");
    if (rank) *rank = -1;
    if (m < 0 || m < n) return -1;
    if (n < 0) return -2;
    if (lda < imax(1, m)) return -4;
    if (!rank) return -10;
    if (n == 0) { *rank = 0; return 0; }
    if (!A_host) return -3;
    if (!jpvt_host) return -8;
    if (!tau_host) return -9;
    if (!workspace) return -12;
    const size_t need = bqrrp_workspace_query_host(m, n, b, d, opts);
    if (!need) { set_error("invalid arguments"); return b < 1 ? -5 : (d < b ? -6 : -11); }
    if (workspace_bytes < need) { set_error("workspace too small"); return BQRRP_ENOMEM; }
    cudaStream_t st = (cudaStream_t)stream;
    char* base = (char*)(((uintptr_t)workspace + 255) & ~(uintptr_t)255);
    double* dA = (double*)base;
    const size_t am = ((size_t)m * (size_t)n * 8 + 255) & ~(size_t)255;
    const size_t jv = ((size_t)n * 8 + 255) & ~(size_t)255;
    int64_t* dj = (int64_t*)(base + am);
    double* dt = (double*)(base + am + jv);
    char* rest = base + am + 2 * jv;
    const size_t rest_bytes = workspace_bytes - (size_t)(rest - (char*)workspace);
    // Pinned A_host is copied in and back on a copy stream, overlapped with
    // the factorization; pageable memory (where an asynchronous copy may
    // synchronize the stream or block this thread) is copied in before it
    // and back after it.
    cudaPointerAttributes pa{};
    const bool pinned = cudaPointerGetAttributes(&pa, A_host) == cudaSuccess && pa.type == cudaMemoryTypeHost;
    (void)cudaGetLastError();
    std::vector<cudaEvent_t> events;
    HostIO io{A_host, lda, nullptr, &events};
    if (pinned) {
        BQ_CUDA(cudaStreamCreateWithFlags(&io.cs, cudaStreamNonBlocking));
        // the copy stream starts after the work queued on `stream` so far
        cudaEvent_t ev;
        const int e = io.record(st, &ev);
        if (e != 0 || cudaStreamWaitEvent(io.cs, ev, 0) != cudaSuccess) {
            cudaStreamDestroy(io.cs);
            for (cudaEvent_t x : events) cudaEventDestroy(x);
            set_error("bqrrp_factor_host: copy stream setup failed");
            return BQRRP_ECUDA;
        }
    } else {
        BQ_CUDA(cudaMemcpy2DAsync(dA, sizeof(double) * m, A_host, sizeof(double) * lda, sizeof(double) * m, n,
                                  cudaMemcpyHostToDevice, st));
    }
    int rc = factor_entry(m, n, dA, m, b, d, seed, dj, dt, rank, opts, rest, rest_bytes, stream,
                          pinned ? &io : nullptr);
    cudaError_t ce = cudaSuccess;   // of the copies back and the final synchronizations
    if (rc == 0) {
        if (!pinned)
            ce = cudaMemcpy2DAsync(A_host, sizeof(double) * lda, dA, sizeof(double) * m, sizeof(double) * m, n,
                                   cudaMemcpyDeviceToHost, st);
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(jpvt_host, dj, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, st);
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(tau_host, dt, sizeof(double) * n, cudaMemcpyDeviceToHost, st);
    }
    // both streams finish before the events, the copy stream and the call go
    const cudaError_t se = cudaStreamSynchronize(st);
    if (ce == cudaSuccess) ce = se;
    if (io.cs) {
        const cudaError_t ss = cudaStreamSynchronize(io.cs);
        if (ce == cudaSuccess) ce = ss;
        cudaStreamDestroy(io.cs);
    }
    for (cudaEvent_t ev : events) cudaEventDestroy(ev);
    if (rc == 0 && ce != cudaSuccess) {
        set_error("bqrrp_factor_host: %s", cudaGetErrorString(ce));
        rc = BQRRP_ECUDA;
    }
    if (rc != 0 && rank) *rank = -1;
    return rc;
}

int bqrrp_sketch_operator(int64_t d, int64_t m, uint64_t seed, int kind, int64_t nnz, double* S, int64_t lds,
                          void* stream) {
    set_error("");
    if (d < 0) return -1;
    if (m < 0) return -2;
    if (kind != BQRRP_SKETCH_DENSE && kind != BQRRP_SKETCH_SPARSE) return -4;
    if (kind == BQRRP_SKETCH_SPARSE && (nnz < 1 || nnz > d || nnz > 64)) return -5;
    if (d * m > 0 && !S) return -6;
    if (lds < imax(1, d)) return -7;
    Ctx c{};
    BQ_TRY(make_ctx(stream, &c));
    c.st = nullptr;
    return sketch_write(c, d, m, seed, kind, nnz, S, lds);
}

size_t bqrrp_sketch_apply_workspace(int64_t d, int64_t m, int kind, int64_t nnz) {
    if (kind == BQRRP_SKETCH_SPARSE) return sketch_sparse_ws(d, m, nnz) + 256;
    return 0;
}

int bqrrp_sketch_apply(int64_t d, int64_t m, int64_t n, const double* A, int64_t lda, uint64_t seed, int kind,
                       int64_t nnz, double* Msk, int64_t ldsk, void* workspace, size_t workspace_bytes,
                       void* stream) {
    set_error("");
    if (d < 0) return -1;
    if (m < 0) return -2;
    if (n < 0) return -3;
    if (lda < imax(1, m)) return -5;
    if (kind != BQRRP_SKETCH_DENSE && kind != BQRRP_SKETCH_SPARSE) return -7;
    if (kind == BQRRP_SKETCH_SPARSE && (nnz < 1 || nnz > d || nnz > 64)) return -8;
    if (ldsk < imax(1, d)) return -10;
    Ctx c{};
    BQ_TRY(make_ctx(stream, &c));
    if (kind == BQRRP_SKETCH_DENSE) return sketch_dense_gemm(c, d, m, n, seed, A, lda, Msk, ldsk);
    if (workspace_bytes < sketch_sparse_ws(d, m, nnz)) { set_error("workspace too small"); return BQRRP_ENOMEM; }
    return sketch_sparse_apply(c, d, m, n, seed, nnz, A, lda, Msk, ldsk, workspace, workspace_bytes);
}

}  // extern "C"
