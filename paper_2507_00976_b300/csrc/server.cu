// server.cu -- a request loop for BQRRP factorization / low-rank compression
// requests of mixed shapes (the paper treats one matrix per call; this is the
// serving layer around it).
//
// Design.  One worker thread owns one CUDA stream and a device pool of
// `hbm_budget` bytes allocated once.  The pool has two arenas:
//  - the request arena holds each admitted request's state (its matrix, then
//    R and the reflectors in place, jpvt, tau) from admission until its results
//    are copied back;
//  - the workspace arena holds the scratch of the job currently running.
// Requests are admitted first-come-first-served whenever their state fits in
// the request arena (a coalescing first-fit free list).
//
// Three workers run concurrently, each with its own thread, CUDA stream and
// third of the workspace arena:
//  - small lane (m*n <= small_max_elems), one worker: every admitted small
//    request is factored in one batched call (the lock-step batched kernels,
//    whose short launches interleave with the large lane, addressing each
//    request's state in place through per-matrix offsets).  Requests that
//    arrive meanwhile join the next batch (continuous batching);
//  - large lane, two workers: each admits one large request at a time (first
//    come, first served) and runs it through the single-matrix path, so two
//    large factorizations overlap and fill each other's latency-bound steps
//    (the sketch's LU and QR, the small panel kernels).
// The batched kernels never wait on other work, and every cross-CTA wait of the
// single-matrix path is bounded, so the lanes can share the GPU.
//
// Every request also gets its truncation rank: the smallest t with
// ||R(t:rank, t:n)||_F <= tol ||A||_F.  Timestamps (submit, admit, start, done)
// come from one steady clock, in seconds since the server was created.
// A dry-run mode replaces the GPU work by a modelled service time (FLOPs over a
// given rate) so that the admission and batching logic can run without a GPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "common.cuh"

namespace bq {
namespace {

constexpr size_t kAlign = 256;
size_t up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

double canonical(i64 m, i64 n) { return 2.0 * m * (double)n * n - 2.0 * (double)n * n * n / 3.0; }

// First-fit free list over [0, cap) with coalescing of neighbours.
class FreeList {
   public:
    explicit FreeList(size_t cap) : cap_(cap) {
        if (cap) free_[0] = cap;
    }
    bool alloc(size_t bytes, size_t* off) {
        bytes = up(bytes ? bytes : 1);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t at = it->first + bytes;
                free_.erase(it);
                if (rest) free_[at] = rest;
                used_ += bytes;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = up(bytes ? bytes : 1);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }
    size_t cap() const { return cap_; }

   private:
    size_t cap_ = 0, used_ = 0;
    std::map<size_t, size_t> free_;
};

struct Req {
    bqrrp_request r;
    bqrrp_completion c;
    bool small = false;
    size_t bytes = 0;       // request-arena bytes
    size_t offA = 0, offJ = 0, offT = 0;
};

__global__ void norm_partial_kernel(const double* A, i64 count, double* part) {
    __shared__ double red[256];
    const i64 per = (count + gridDim.x - 1) / gridDim.x;
    const i64 lo = (i64)blockIdx.x * per, hi = min(count, lo + per);
    double acc = 0.0;
    for (i64 e = lo + threadIdx.x; e < hi; e += blockDim.x) acc += A[e] * A[e];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// rn[r] = ||R(r, r:n)||^2 for r < ell
__global__ void rownorm_kernel(const double* A, i64 m, i64 n, i64 ell, double* rn) {
    const i64 r = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= ell) return;
    double acc = 0.0;
    for (i64 c = r; c < n; ++c) acc += A[r + c * m] * A[r + c * m];
    rn[r] = acc;
}

// anorm^2 = sum of the partials in order; the truncation rank by a suffix scan
__global__ void trunc_final_kernel(const double* part, int nparts, const double* rn, i64 ell, double tol,
                                   int64_t* out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double a2 = 0.0;
    for (int q = 0; q < nparts; ++q) a2 += part[q];
    const double thr = tol * sqrt(a2);
    const double thr2 = thr * thr;
    double tail = 0.0;
    i64 best = ell;
    for (i64 i = ell - 1; i >= 0; --i) {
        tail += rn[i];
        if (tail <= thr2) best = i;
        else break;
    }
    *out = best;
}

constexpr int kNormParts = 256;

}  // namespace

struct Server {
    size_t budget = 0, ws_bytes = 0;
    double tol = 1e-8;
    i64 small_max = 1 << 20;
    int flags = 0;
    double dry_gflops = 1000.0;
    bool dry = false;
    bool mixed = false;                           // large lane in BQRRP_PRECISION_MIXED
    int device = 0;
    static constexpr int kWorkers = 3;          // 0: small lane; 1, 2: large lane
    char* base = nullptr;                         // request arena, then workspace arena
    char* wsbase[kWorkers] = {nullptr, nullptr, nullptr};   // per worker: a third of the workspace arena
    size_t lane_ws = 0;
    FreeList arena{0};
    cudaStream_t st[kWorkers] = {nullptr, nullptr, nullptr};
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv, cv_done;
    std::deque<Req*> pending;       // submitted, waiting for admission
    std::vector<Req*> ready_small;  // admitted
    std::deque<bqrrp_completion> done;
    std::atomic<bool> stop{false};
    i64 submitted = 0, completed = 0, batches = 0, max_batch = 0, larges = 0;
    char last_err[512] = {0};       // message of the last failed job (worker thread)
    size_t peak = 0;
    std::thread worker[kWorkers];

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    void run_small();
    void run_large(int wk);
    int admit_locked(int lane, std::vector<Req*>& newly, size_t max_new);
    int do_small(std::vector<Req*>& batch);
    int do_large(Req* q, int wk);
    void finish(std::vector<Req*>& reqs, int status);
};

size_t request_state_bytes(i64 m, i64 n) { return up((size_t)m * n * 8) + up((size_t)n * 8) * 2; }

// Admit, in submission order, up to max_new of this lane's pending requests
// that fit.
int Server::admit_locked(int lane, std::vector<Req*>& newly, size_t max_new) {
    for (auto it = pending.begin(); it != pending.end() && newly.size() < max_new;) {
        Req* q = *it;
        size_t off;
        if (q->c.lane == lane && arena.alloc(q->bytes, &off)) {
            q->offA = off;
            q->offJ = off + up((size_t)q->r.m * q->r.n * 8);
            q->offT = q->offJ + up((size_t)q->r.n * 8);
            q->c.t_admit = now();
            peak = std::max(peak, arena.used());
            newly.push_back(q);
            it = pending.erase(it);
        } else {
            ++it;
        }
    }
    return 0;
}

void Server::finish(std::vector<Req*>& reqs, int status) {
    std::lock_guard<std::mutex> lk(mu);
    if (status != 0) std::snprintf(last_err, sizeof(last_err), "%s", get_error());
    for (Req* q : reqs) {
        if (q->c.status == 0) q->c.status = status;
        q->c.t_done = now();
        arena.release(q->offA, q->bytes);
        done.push_back(q->c);
        ++completed;
        delete q;
    }
    reqs.clear();
    cv.notify_all();
    cv_done.notify_all();
}

// One batched factorization of the admitted small requests (in place).
int Server::do_small(std::vector<Req*>& batch) {
    const i64 nb = (i64)batch.size();
    const double t_start = now();
    for (Req* q : batch) q->c.t_start = t_start;
    if (dry) {
        double fl = 0.0;
        for (Req* q : batch) {
            fl += canonical(q->r.m, q->r.n);
            q->c.rank = q->r.n;
            q->c.trunc_rank = q->r.n;
        }
        std::this_thread::sleep_for(std::chrono::duration<double>(fl / (dry_gflops * 1e9)));
        return 0;
    }
    std::vector<i64> m(nb), n(nb), b(nb), d(nb), oA(nb), oJ(nb), oT(nb);
    std::vector<uint64_t> sd(nb);
    for (i64 i = 0; i < nb; ++i) {
        const Req* q = batch[i];
        m[i] = q->r.m;
        n[i] = q->r.n;
        b[i] = q->r.b;
        d[i] = q->r.d;
        sd[i] = q->r.seed;
        oA[i] = (i64)(q->offA / 8);          // element offsets from the arena base
        oJ[i] = (i64)(q->offJ / 8);
        oT[i] = (i64)(q->offT / 8);
    }
    BatchPlan* P = nullptr;
    int rc = batch_plan_create_ex(&P, nb, m.data(), n.data(), b.data(), d.data(), sd.data(), tol, oA.data(),
                                  oJ.data(), oT.data(), nullptr);
    if (rc != 0) return rc;
    // short per-phase launches: they interleave with the large lane's
    // grid-wide kernels, where the persistent form would hold the SMs
    batch_plan_set_lockstep(P, true);
    // workspace arena: rank, truncation rank, info, then the plan's workspace
    char* w = wsbase[0];
    int64_t* rk = (int64_t*)w;   w += up(sizeof(int64_t) * nb);
    int64_t* tr = (int64_t*)w;   w += up(sizeof(int64_t) * nb);
    int32_t* inf = (int32_t*)w;  w += up(sizeof(int32_t) * nb);
    const size_t have = lane_ws - (size_t)(w - wsbase[0]);
    if (batch_plan_bytes(P) > have) {
        batch_plan_destroy(P);
        set_error("batch workspace %zu > %zu", batch_plan_bytes(P), have);
        return BQRRP_ENOMEM;
    }
    rc = batch_factor(P, (double*)base, (int64_t*)base, (double*)base, rk, tr, inf, w, have, st[0], 0);
    if (rc == 0) {
        std::vector<int64_t> hrk(nb), htr(nb);
        std::vector<int32_t> hinf(nb);
        cudaMemcpyAsync(hrk.data(), rk, sizeof(int64_t) * nb, cudaMemcpyDeviceToHost, st[0]);
        cudaMemcpyAsync(htr.data(), tr, sizeof(int64_t) * nb, cudaMemcpyDeviceToHost, st[0]);
        cudaMemcpyAsync(hinf.data(), inf, sizeof(int32_t) * nb, cudaMemcpyDeviceToHost, st[0]);
        for (Req* q : batch) {
            if (q->r.A_out_host)
                cudaMemcpyAsync(q->r.A_out_host, base + q->offA, (size_t)q->r.m * q->r.n * 8, cudaMemcpyDeviceToHost, st[0]);
            if (q->r.jpvt_out_host)
                cudaMemcpyAsync(q->r.jpvt_out_host, base + q->offJ, (size_t)q->r.n * 8, cudaMemcpyDeviceToHost, st[0]);
            if (q->r.tau_out_host)
                cudaMemcpyAsync(q->r.tau_out_host, base + q->offT, (size_t)q->r.n * 8, cudaMemcpyDeviceToHost, st[0]);
        }
        if (cudaStreamSynchronize(st[0]) != cudaSuccess) {
            set_error("small lane: %s", cudaGetErrorString(cudaGetLastError()));
            rc = BQRRP_ECUDA;
        } else {
            for (i64 i = 0; i < nb; ++i) {
                batch[i]->c.rank = hrk[i];
                batch[i]->c.trunc_rank = htr[i];
                batch[i]->c.status = hinf[i];
            }
        }
    }
    batch_plan_destroy(P);
    return rc;
}

// One large request through the single-matrix path.
int Server::do_large(Req* q, int wk) {
    q->c.t_start = now();
    const i64 m = q->r.m, n = q->r.n;
    if (dry) {
        std::this_thread::sleep_for(std::chrono::duration<double>(canonical(m, n) / (dry_gflops * 1e9)));
        q->c.rank = n;
        q->c.trunc_rank = n;
        return 0;
    }
    double* A = (double*)(base + q->offA);
    int64_t* J = (int64_t*)(base + q->offJ);
    double* tau = (double*)(base + q->offT);
    char* w = wsbase[wk];
    double* part = (double*)w;   w += up(sizeof(double) * kNormParts);
    double* rn = (double*)w;     w += up(sizeof(double) * (size_t)std::max<i64>(n, 1));
    int64_t* trd = (int64_t*)w;  w += up(sizeof(int64_t));
    const size_t have = lane_ws - (size_t)(w - wsbase[wk]);
    bqrrp_opts o{};
    o.precision = mixed ? BQRRP_PRECISION_MIXED : BQRRP_PRECISION_FP64;
    const size_t need = bqrrp_workspace_query(m, n, q->r.b, q->r.d, &o);
    if (need > have) {
        set_error("large request needs %zu workspace bytes, the arena has %zu", need, have);
        return BQRRP_ENOMEM;
    }
    norm_partial_kernel<<<kNormParts, 256, 0, st[wk]>>>(A, m * n, part);
    BQ_LAUNCH_CHECK();
    int64_t rank = 0;
    int rc = bqrrp_factor(m, n, A, m, q->r.b, q->r.d, q->r.seed, J, tau, &rank, &o, w, have, st[wk]);
    if (rc != 0) return rc;
    if (rank > 0) {
        rownorm_kernel<<<(unsigned)cdiv(rank, 128), 128, 0, st[wk]>>>(A, m, n, rank, rn);
        BQ_LAUNCH_CHECK();
    }
    trunc_final_kernel<<<1, 32, 0, st[wk]>>>(part, kNormParts, rn, rank, tol, trd);
    BQ_LAUNCH_CHECK();
    int64_t htr = 0;
    cudaMemcpyAsync(&htr, trd, sizeof(int64_t), cudaMemcpyDeviceToHost, st[wk]);
    if (q->r.A_out_host) cudaMemcpyAsync(q->r.A_out_host, A, (size_t)m * n * 8, cudaMemcpyDeviceToHost, st[wk]);
    if (q->r.jpvt_out_host) cudaMemcpyAsync(q->r.jpvt_out_host, J, (size_t)n * 8, cudaMemcpyDeviceToHost, st[wk]);
    if (q->r.tau_out_host) cudaMemcpyAsync(q->r.tau_out_host, tau, (size_t)n * 8, cudaMemcpyDeviceToHost, st[wk]);
    BQ_CUDA(cudaStreamSynchronize(st[wk]));
    q->c.rank = rank;
    q->c.trunc_rank = htr;
    return 0;
}

void Server::run_small() {
    if (!dry) cudaSetDevice(device);
    for (;;) {
        std::vector<Req*> newly, work;
        {
            std::unique_lock<std::mutex> lk(mu);
            auto mine = [&] {
                if (!ready_small.empty()) return true;
                for (Req* q : pending)
                    if (q->c.lane == 0) return true;
                return false;
            };
            cv.wait(lk, [&] { return stop.load() || mine(); });
            admit_locked(0, newly, (size_t)-1);
            if (ready_small.empty() && newly.empty()) {
                bool waiting = false;
                for (Req* q : pending)
                    if (q->c.lane == 0) waiting = true;
                if (stop.load() && !waiting) break;
                // this lane's requests do not fit yet: wait for a completion
                cv.wait_for(lk, std::chrono::milliseconds(1));
                continue;
            }
        }
        // copy newly admitted matrices in on this lane's stream
        for (Req* q : newly) {
            if (!dry)
                cudaMemcpyAsync(base + q->offA, q->r.A_host, (size_t)q->r.m * q->r.n * 8, cudaMemcpyHostToDevice,
                                st[0]);
            std::lock_guard<std::mutex> lk(mu);
            ready_small.push_back(q);
        }
        {
            std::lock_guard<std::mutex> lk(mu);
            work.swap(ready_small);
        }
        if (work.empty()) continue;
        const int rc = do_small(work);
        {
            std::lock_guard<std::mutex> lk(mu);
            ++batches;
            max_batch = std::max<i64>(max_batch, (i64)work.size());
        }
        finish(work, rc);
    }
}

// A large-lane worker: admits one large request when it fits, copies it in on
// its own stream and factors it there.
void Server::run_large(int wk) {
    if (!dry) cudaSetDevice(device);
    for (;;) {
        std::vector<Req*> work;
        {
            std::unique_lock<std::mutex> lk(mu);
            auto mine = [&] {
                for (Req* q : pending)
                    if (q->c.lane == 1) return true;
                return false;
            };
            cv.wait(lk, [&] { return stop.load() || mine(); });
            admit_locked(1, work, 1);
            if (work.empty()) {
                if (stop.load() && !mine()) break;
                // no large request fits yet: wait for a completion
                cv.wait_for(lk, std::chrono::milliseconds(1));
                continue;
            }
        }
        Req* q = work[0];
        if (!dry)
            cudaMemcpyAsync(base + q->offA, q->r.A_host, (size_t)q->r.m * q->r.n * 8, cudaMemcpyHostToDevice, st[wk]);
        const int rc = do_large(q, wk);
        {
            std::lock_guard<std::mutex> lk(mu);
            ++larges;
        }
        finish(work, rc);
    }
}

}  // namespace bq

// ================================================================== C ABI
struct bqrrp_server_s {
    bq::Server s;
};

extern "C" {

int bqrrp_server_create(bqrrp_server* out, size_t hbm_budget_bytes, size_t workspace_bytes, double trunc_tol,
                        int64_t small_max_elems, int flags, double dry_gflops) {
    bq::set_error("");
    if (!out) { bq::set_error("out is null"); return -1; }
    *out = nullptr;
    if (workspace_bytes < (1u << 20) || hbm_budget_bytes < workspace_bytes + (1u << 20)) {
        bq::set_error("need hbm_budget >= workspace + 1 MiB and workspace >= 1 MiB");
        return -2;
    }
    if (!(trunc_tol >= 0.0)) { bq::set_error("trunc_tol < 0"); return -4; }
    if (flags & ~(BQRRP_SERVER_DRYRUN | BQRRP_SERVER_MIXED)) { bq::set_error("unknown flags"); return -6; }
    auto* h = new bqrrp_server_s();
    bq::Server& S = h->s;
    S.budget = hbm_budget_bytes & ~(bq::kAlign - 1);
    S.ws_bytes = bq::up(workspace_bytes);
    S.lane_ws = (S.ws_bytes / bq::Server::kWorkers) & ~(bq::kAlign - 1);
    S.tol = trunc_tol;
    S.small_max = small_max_elems;
    S.flags = flags;
    S.dry = (flags & BQRRP_SERVER_DRYRUN) != 0;
    S.mixed = (flags & BQRRP_SERVER_MIXED) != 0;
    S.dry_gflops = dry_gflops > 0.0 ? dry_gflops : 1000.0;
    S.arena = bq::FreeList(S.budget - S.ws_bytes);
    S.t0 = std::chrono::steady_clock::now();
    if (!S.dry) {
        bq::Device dev;
        int rc = bq::current_device(&dev);
        if (rc != 0) { delete h; return rc; }
        S.device = dev.id;
        cudaError_t e = cudaMalloc(&S.base, S.budget);
        if (e != cudaSuccess) {
            bq::set_error("cudaMalloc(%zu): %s", S.budget, cudaGetErrorString(e));
            delete h;
            return BQRRP_ENOMEM;
        }
        S.wsbase[0] = S.base + (S.budget - S.ws_bytes);
        for (int k = 1; k < bq::Server::kWorkers; ++k) S.wsbase[k] = S.wsbase[k - 1] + S.lane_ws;
        e = cudaSuccess;
        for (int k = 0; k < bq::Server::kWorkers && e == cudaSuccess; ++k)
            e = cudaStreamCreateWithFlags(&S.st[k], cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            cudaFree(S.base);
            bq::set_error("cudaStreamCreate: %s", cudaGetErrorString(e));
            delete h;
            return BQRRP_ECUDA;
        }
    }
    S.worker[0] = std::thread([&S] { S.run_small(); });
    for (int k = 1; k < bq::Server::kWorkers; ++k) S.worker[k] = std::thread([&S, k] { S.run_large(k); });
    *out = h;
    return 0;
}

int bqrrp_server_submit(bqrrp_server srv, const bqrrp_request* req) {
    if (!srv || !req) return -1;
    bq::Server& S = srv->s;
    const bqrrp_request& r = *req;
    if (r.n < 1 || r.m < r.n) { bq::set_error("request %llu: need m >= n >= 1", (unsigned long long)r.id); return -2; }
    if (!S.dry && !r.A_host) { bq::set_error("request %llu: A_host is null", (unsigned long long)r.id); return -2; }
    const bool small = r.m * r.n <= S.small_max;
    if (r.b < 1 || r.d < r.b || (small && (r.b > 128 || r.d > 256 || r.n > 4096))) {
        bq::set_error("request %llu: block sizes outside the lane's range", (unsigned long long)r.id);
        return -2;
    }
    auto* q = new bq::Req();
    q->r = r;
    q->small = small;
    q->bytes = bq::request_state_bytes(r.m, r.n);
    std::memset(&q->c, 0, sizeof(q->c));
    q->c.id = r.id;
    q->c.lane = small ? 0 : 1;
    {
        std::lock_guard<std::mutex> lk(S.mu);
        if (q->bytes > S.arena.cap()) {
            delete q;
            bq::set_error("request larger than the whole request arena");
            return BQRRP_ENOMEM;
        }
        q->c.t_submit = S.now();
        S.pending.push_back(q);
        ++S.submitted;
    }
    S.cv.notify_all();
    return 0;
}

int bqrrp_server_poll(bqrrp_server srv, bqrrp_completion* out, int max_out, double wait_s) {
    if (!srv || (!out && max_out > 0)) return -1;
    bq::Server& S = srv->s;
    std::unique_lock<std::mutex> lk(S.mu);
    if (S.done.empty() && wait_s > 0.0)
        S.cv_done.wait_for(lk, std::chrono::duration<double>(wait_s), [&] { return !S.done.empty(); });
    int k = 0;
    while (k < max_out && !S.done.empty()) {
        out[k++] = S.done.front();
        S.done.pop_front();
    }
    return k;
}

int bqrrp_server_drain(bqrrp_server srv) {
    if (!srv) return -1;
    bq::Server& S = srv->s;
    std::unique_lock<std::mutex> lk(S.mu);
    S.cv_done.wait(lk, [&] { return S.completed == S.submitted; });
    return 0;
}

double bqrrp_server_clock(bqrrp_server srv) { return srv ? srv->s.now() : 0.0; }

const char* bqrrp_server_last_error(bqrrp_server srv) {
    if (!srv) return "";
    std::lock_guard<std::mutex> lk(srv->s.mu);
    return srv->s.last_err;
}

int bqrrp_server_get_stats(bqrrp_server srv, bqrrp_server_stats* out) {
    if (!srv || !out) return -1;
    bq::Server& S = srv->s;
    std::lock_guard<std::mutex> lk(S.mu);
    out->submitted = S.submitted;
    out->completed = S.completed;
    out->batches = S.batches;
    out->max_batch = S.max_batch;
    out->large_runs = S.larges;
    out->peak_request_bytes = (int64_t)S.peak;
    out->request_arena_bytes = (int64_t)S.arena.cap();
    out->in_use_bytes = (int64_t)S.arena.used();
    return 0;
}

void bqrrp_server_destroy(bqrrp_server srv) {
    if (!srv) return;
    bq::Server& S = srv->s;
    {
        std::lock_guard<std::mutex> lk(S.mu);
        S.stop.store(true);
    }
    S.cv.notify_all();
    for (auto& t : S.worker)
        if (t.joinable()) t.join();
    if (!S.dry) {
        for (auto& st : S.st)
            if (st) cudaStreamDestroy(st);
        if (S.base) cudaFree(S.base);
    }
    for (auto* q : S.pending) delete q;
    for (auto* q : S.ready_small) delete q;
    delete srv;
}

}  // extern "C"
