// batched.cu -- BQRRP (Alg. 1 with the Alg. 2 sketch QRCP and the Alg. 3
// CholQR panel) on many independent small matrices at once.
//
// Design.  The matrices advance in lock step: block iteration i of every
// matrix that still has columns runs in the same set of launches.  Each phase
// of an iteration is ONE persistent kernel over the whole batch; its CTAs pull
// work items (a matrix, or a column / row tile of a matrix) from a queue that
// the host orders by decreasing cost, so the large matrices start first.  A
// matrix that terminates early (rank found, Sec. 3.7) is skipped by the later
// launches through its device-side state, so the launch sequence is fixed and
// is captured once into a CUDA graph.
//
// Per matrix (m x n, lda = m, block b, sketch rows d):
//   init      ||A||_F, NaN/Inf check, J = identity, tau = 0
//   sketch    Msk = S A, S the d x m Philox +-1 operator (Sec. 3.2), generated
//             in shared memory and never stored
//   per iteration i (s = i b, c = min(n, s + b), w = c - s, N = n - s):
//   qrcp      Alg. 2: LU with partial pivoting of Msk(:, s:)^T (first-maximum
//             rule, all min(N, d) steps), piv_transform, gather of the sketch
//             columns, Householder QR -> R^sk, tri_rank -> k; moved-column list
//   perm      the columns of A(:, s:) and J(s:) that the pivots move
//   panel     Alg. 3: Pre = A_p Rsk11^{-1}, G = Pre^T Pre, R_chol = chol(G),
//             Q_c = Pre R_chol^{-1}, modified-LU reconstruction (Y, T, D),
//             R11 = diag(D) R_chol Rsk(0:k, 0:w), Z = Rsk11 R11^{-1}
//   trailing  A(s:, c:) -= Y (T^T (Y^T A(s:, c:)))  (first k rows when k < w)
//   skupdate  Msk(:, c:) = [Rsk12 - Z R12 ; Rsk22]  (Duersch-Gu update)
//   finish    jpvt 1-based, rank, truncation rank (smallest i with
//             ||R(i:rank, i:n)||_F <= tol ||A||_F)
//
// Every CTA has 256 threads.  B300 runs FP64 at 2 DFMA per clock per SM, so a
// single SM's arithmetic, not its memory, bounds these per-matrix loops; they
// are written for coalesced column access and shared-memory reuse, not for
// tensor cores (there is no FP64 tensor path on this part).
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace bq {
namespace {

constexpr int BT = 256;          // threads per CTA, every phase
constexpr int NW = BT / 32;      // warps per CTA
constexpr int kMaxD = 256;       // largest sketch size d
constexpr int kMaxB = 128;       // largest block size b
constexpr int kMaxN = 4096;      // largest column count n
constexpr int CT = 64;           // columns per tile (sketch); the widest trailing tile
constexpr int CT_MIN = 32;       // the narrowest trailing tile (a plan chooses 32 or 64 per matrix)
constexpr int SK_RK = 32;        // rows of A per sketch chunk
constexpr int RCH = 32;          // rows per permutation chunk
constexpr int RG = 32;           // rows per Gram chunk
constexpr int RT = 32;           // rows per trailing-update chunk

// ------------------------------------------------------------------ plan records
struct BatMat {                  // per matrix, written by the host, read-only on the device
    i64 m, n, b, d;
    i64 ct;                      // columns per trailing-update / sketch-update tile: 32 or 64
    i64 offA;                    // element offset of A (column-major, lda = m)
    i64 offJ;                    // element offset of jpvt
    i64 offT;                    // element offset of tau
    i64 offSk;                   // sketch d x n (ld d) in the double workspace
    i64 offW;                    // work d x n (ld d): LU copy, then R^sk
    i64 offY;                    // explicit Y, m x b (ld m)
    i64 offV;                    // V = Y T^T, m x b (ld m)
    i64 offSm;                   // T, P, Z: three b x b blocks (ld b)
    i64 offI;                    // int workspace: Jsk (n), moved list (n)
    uint64_t seed;
};

struct BatState {                // per matrix, device-written
    double anorm;                // ||A||_F of the input
    double r00;                  // |Rsk(0,0)| of the first iteration (tri_rank scale)
    i64 k;                       // panel rank of the current iteration
    i64 nmoved;                  // columns moved by the current permutation
    i64 ell;                     // rank when done
    int done;                    // the factorization has ended
    int upd_iter;                // iteration whose panel was factored (trailing update runs)
    int cont_iter;               // iteration whose sketch update runs
    int info;                    // 0 or BQRRP_ENUMERIC
};

struct Slot {                    // one launch: matrices [first, first + nmats) of the slot lists
    int first, nmats, total;     // total = number of work items
};

struct BatArgs {
    const BatMat* mats;
    BatState* st;
    const int* smat;             // slot matrix lists
    const int* spre;             // slot exclusive prefix sums of items (nmats + 1 per slot)
    unsigned int* ctr;           // one counter per launch
    double* A;
    int64_t* jpvt;
    double* tau;
    double* wsd;
    int* wsi;
    int64_t* rank_out;
    int64_t* trunc_out;
    int32_t* info_out;
    double tol;
};

// Next work item of a launch: returns (matrix, sub-item), or mat = -1 when the
// queue is empty.  Thread 0 takes a ticket and finds its matrix by binary
// search over the slot's prefix sums.
struct Item {
    int mat, sub;
};

__device__ Item next_item(const BatArgs& a, const Slot sl, int slot_id) {
    __shared__ int s_mat, s_sub;
    __syncthreads();
    if (threadIdx.x == 0) {
        const int t = (int)atomicAdd(&a.ctr[slot_id], 1u);
        if (t >= sl.total) {
            s_mat = -1;
            s_sub = 0;
        } else {
            const int* pre = a.spre + sl.first + slot_id;   // nmats + 1 entries
            int lo = 0, hi = sl.nmats;                     // pre[lo] <= t < pre[hi]
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (pre[mid] <= t) lo = mid;
                else hi = mid;
            }
            s_mat = a.smat[sl.first + lo];
            s_sub = t - pre[lo];
        }
    }
    __syncthreads();
    return Item{s_mat, s_sub};
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// First maximum of (value, index) pairs: larger value wins, ties go to the
// smaller index.
__device__ __forceinline__ void argmax_merge(double& v, int& i, double v2, int i2) {
    if (v2 > v || (v2 == v && i2 < i)) {
        v = v2;
        i = i2;
    }
}

// |x| as an ordering key: for non-negative doubles the bit patterns order like
// the values, so pivot searches compare integers (an FP64 compare holds a
// sub-partition's FP64 unit for ~64 cycles on B300, like a DFMA).
__device__ __forceinline__ unsigned long long abs_key(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

// First maximum over (key, index): larger key, then smaller index.
__device__ __forceinline__ void argmax_merge_key(unsigned long long& k, int& i, unsigned long long k2, int i2) {
    if (k2 > k || (k2 == k && i2 < i)) {
        k = k2;
        i = i2;
    }
}

// X(i, 0:k) <- X(i, 0:k) R^{-1} for one row i, R upper triangular in shared
// memory (ld ldr >= k rounded up to 16), rinv[j] = 1 / R(j, j) formed once
// per CTA (an FP64 division holds a sub-partition's FP64 unit for ~640
// cycles on B300).  Left-looking in blocks of 16 columns held in registers;
// the subtractions of each element run in column order, then the scaling by
// the reciprocal, as in row-wise forward substitution.
__device__ void row_trsm_upper(const double* src, i64 lds, double* dst, i64 ldd, i64 i, int k,
                               const double* R, int ldr, const double* rinv) {
    for (int jb = 0; jb < k; jb += 16) {
        const int nb = min(16, k - jb);
        double x[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) x[q] = (q < nb) ? src[i + (i64)(jb + q) * lds] : 0.0;
        for (int t = 0; t < jb; ++t) {
            const double y = dst[i + (i64)t * ldd];
#pragma unroll
            for (int q = 0; q < 16; ++q) x[q] -= y * R[t + (jb + q) * ldr];
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            if (q < nb) {
                x[q] *= rinv[jb + q];
#pragma unroll
                for (int u = q + 1; u < 16; ++u) x[u] -= x[q] * R[(jb + q) + (jb + u) * ldr];
            }
        }
#pragma unroll
        for (int q = 0; q < 16; ++q)
            if (q < nb) dst[i + (i64)(jb + q) * ldd] = x[q];
    }
}

// ------------------------------------------------------------------ init
__device__ void body_init(const BatArgs& a, const int mat, const int sub) {
    __shared__ double red[BT];
    __shared__ int s_bad;
        {
        const BatMat M = a.mats[mat];
        const double* A = a.A + M.offA;
        const i64 tot = M.m * M.n;
        double acc = 0.0;
        int bad = 0;
        for (i64 e = threadIdx.x; e < tot; e += BT) {
            const double v = A[e];
            bad |= !isfinite(v);
            acc += v * v;
        }
        if (threadIdx.x == 0) s_bad = 0;
        red[threadIdx.x] = acc;
        __syncthreads();
        if (bad) s_bad = 1;
        for (int h = BT / 2; h > 0; h >>= 1) {
            if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
            __syncthreads();
        }
        int64_t* J = a.jpvt + M.offJ;
        double* tau = a.tau + M.offT;
        for (i64 j = threadIdx.x; j < M.n; j += BT) {
            J[j] = j;
            tau[j] = 0.0;
        }
        if (threadIdx.x == 0) {
            BatState& S = a.st[mat];
            S.anorm = sqrt(red[0]);
            S.r00 = 0.0;
            S.k = 0;
            S.nmoved = 0;
            S.ell = 0;
            S.upd_iter = -1;
            S.cont_iter = -1;
            S.info = s_bad ? BQRRP_ENUMERIC : 0;
            S.done = (s_bad || M.n == 0) ? 1 : 0;
        }
    }
}

__global__ void __launch_bounds__(BT) bat_init_kernel(BatArgs a, Slot sl, int slot_id) {
    for (;;) {
        const Item it = next_item(a, sl, slot_id);
        if (it.mat < 0) break;
        body_init(a, it.mat, it.sub);
    }
}

// ------------------------------------------------------------------ sketch: Msk = S A
// Item = (matrix, 64-column tile).  The d sketch rows are done in passes of
// 128 (one Philox block each).  Thread (jj = tid % 64, rg = tid / 64)
// accumulates rows i = 128 p + rg + 4q of column jj.  The signs of S(block p,
// rows of the chunk) come from one Philox4x32-10 call per row of A: counter
// (row of A, p, 0, 0), key = seed; bit (i mod 128) of the 128-bit output
// selects -1.
template <int QN>
__device__ void sketch_pass(const double* A, i64 m, i64 j0, int nc, i64 d, int p, uint32_t k0s, uint32_t k1s,
                            double (*As)[CT], uint32_t (*Sw)[4], double* Sk) {
    const int jj = threadIdx.x % CT;
    const int rg = threadIdx.x / CT;
    const int base = 128 * p;
    const int nrows = (int)min((i64)128, d - base);
    double acc[QN];
#pragma unroll
    for (int q = 0; q < QN; ++q) acc[q] = 0.0;
    for (i64 r0 = 0; r0 < m; r0 += SK_RK) {
        const int kr = (int)min((i64)SK_RK, m - r0);
        __syncthreads();
        for (int e = threadIdx.x; e < SK_RK * CT; e += BT) {
            const int r = e % SK_RK, cc = e / SK_RK;
            As[r][cc] = (r < kr && cc < nc) ? A[(r0 + r) + (j0 + cc) * m] : 0.0;
        }
        if (threadIdx.x < SK_RK) {
            uint32_t o[4];
            philox4x32_10((uint32_t)(r0 + threadIdx.x), (uint32_t)p, 0u, 0u, k0s, k1s, o);
#pragma unroll
            for (int q = 0; q < 4; ++q) Sw[threadIdx.x][q] = o[q];
        }
        __syncthreads();
        for (int kk = 0; kk < kr; ++kk) {
            const long long ab = __double_as_longlong(As[kk][jj]);
            uint32_t wd[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) wd[q] = Sw[kk][q];
#pragma unroll
            for (int q = 0; q < QN; ++q) {
                const long long sg = (long long)((wd[q >> 3] >> (4 * (q & 7) + rg)) & 1u) << 63;
                acc[q] += __longlong_as_double(ab ^ sg);
            }
        }
    }
    if (jj < nc) {
        double* out = Sk + (j0 + jj) * d + base;
#pragma unroll
        for (int q = 0; q < QN; ++q)
            if (rg + 4 * q < nrows) out[rg + 4 * q] = acc[q];
    }
}

__device__ void body_sketch(const BatArgs& a, const int mat, const int sub) {
    __shared__ double As[SK_RK][CT];
    __shared__ uint32_t Sw[SK_RK][4];
        {
        if (a.st[mat].done) return;
        const BatMat M = a.mats[mat];
        const i64 j0 = (i64)sub * CT;
        const int nc = (int)min((i64)CT, M.n - j0);
        const double* A = a.A + M.offA;
        double* Sk = a.wsd + M.offSk;
        const uint32_t k0s = (uint32_t)M.seed, k1s = (uint32_t)(M.seed >> 32);
        const int npass = (int)((M.d + 127) / 128);
        for (int p = 0; p < npass; ++p) {
            const int nrows = (int)min((i64)128, M.d - 128 * p);
            if (nrows <= 32) sketch_pass<8>(A, M.m, j0, nc, M.d, p, k0s, k1s, As, Sw, Sk);
            else if (nrows <= 64) sketch_pass<16>(A, M.m, j0, nc, M.d, p, k0s, k1s, As, Sw, Sk);
            else if (nrows <= 96) sketch_pass<24>(A, M.m, j0, nc, M.d, p, k0s, k1s, As, Sw, Sk);
            else sketch_pass<32>(A, M.m, j0, nc, M.d, p, k0s, k1s, As, Sw, Sk);
        }
    }
}

__global__ void __launch_bounds__(BT) bat_sketch_kernel(BatArgs a, Slot sl, int slot_id) {
    for (;;) {
        const Item it = next_item(a, sl, slot_id);
        if (it.mat < 0) break;
        body_sketch(a, it.mat, it.sub);
    }
}

// ------------------------------------------------------------------ Alg. 2 on one matrix per CTA
// First maximum of |W(j, t)| over t in [j, N) (W ld d): the pivot search of
// LU step j on X = W^T.
__device__ int cta_first_argmax(const double* W, i64 d, i64 j, i64 N, unsigned long long* wk, int* wi) {
    __shared__ int s_p;
    unsigned long long bk = 0;
    int bi = INT_MAX;
    for (i64 t = j + threadIdx.x; t < N; t += BT) argmax_merge_key(bk, bi, abs_key(W[j + t * d]), (int)t);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, bk, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
        argmax_merge_key(bk, bi, k2, i2);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        wk[wid] = bk;
        wi[wid] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long k = wk[0];
        int i = wi[0];
        for (int q = 1; q < NW; ++q) argmax_merge_key(k, i, wk[q], wi[q]);
        s_p = (i == INT_MAX) ? (int)j : i;
    }
    __syncthreads();
    return s_p;
}

// Householder QR (LAPACK dlarfg convention) of the d x nc matrix W (ld d) in
// place, one CTA: warp 0 forms each reflector, every warp applies it to its
// columns.  R ends up in the upper trapezoid; below it, the reflectors.
__device__ void cta_house_qr(double* W, i64 d, i64 nc, double* vbuf, double* s_tau) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const i64 kk = min(d, nc);
    for (i64 j = 0; j < kk; ++j) {
        if (wid == 0) {
            double* col = W + j * d;
            double xn2 = 0.0;
            for (i64 rr = j + 1 + lane; rr < d; rr += 32) xn2 += col[rr] * col[rr];
            xn2 = warp_sum(xn2);
            const double alpha = col[j];
            double tau = 0.0, beta = alpha, scal = 1.0;
            if (xn2 != 0.0) {
                const double nrm = sqrt(alpha * alpha + xn2);
                beta = (alpha >= 0.0) ? -nrm : nrm;
                tau = (beta - alpha) / beta;
                scal = 1.0 / (alpha - beta);
            }
            for (i64 rr = j + 1 + lane; rr < d; rr += 32) {
                const double v = (xn2 != 0.0) ? col[rr] * scal : col[rr];
                col[rr] = v;
                vbuf[rr] = v;
            }
            __syncwarp();
            if (lane == 0) {
                col[j] = beta;
                vbuf[j] = 1.0;
                *s_tau = tau;
            }
        }
        __syncthreads();
        const double tau = *s_tau;
        if (tau != 0.0) {
            for (i64 t = j + 1 + wid; t < nc; t += NW) {
                double* col = W + t * d;
                double dot = 0.0;
                for (i64 rr = j + lane; rr < d; rr += 32) dot += vbuf[rr] * col[rr];
                dot = warp_sum(dot) * tau;
                for (i64 rr = j + lane; rr < d; rr += 32) col[rr] -= dot * vbuf[rr];
            }
        }
        __syncthreads();
    }
}

__device__ void body_qrcp(const BatArgs& a, const int mat, const int sub, int iter) {
    __shared__ double pc[kMaxD];
    __shared__ unsigned long long wv[NW];
    __shared__ int wi[NW];
    __shared__ double s_rp;
    __shared__ int ipiv[kMaxD];
    // dynamic shared memory: one L row per warp, then the pivot vector
    extern __shared__ double qdsm[];
    double (*Lw)[kMaxD] = reinterpret_cast<double (*)[kMaxD]>(qdsm);
    int* Js = reinterpret_cast<int*>(qdsm + NW * kMaxD);
    __shared__ int s_flag, s_cnt, s_next;
    __shared__ double s_tau;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        {
        BatState* S = a.st + mat;
        if (S->done) return;
        const BatMat M = a.mats[mat];
        const i64 d = M.d, n = M.n, b = M.b;
        const i64 s = (i64)iter * b;
        const i64 c = min(n, s + b), w = c - s, N = n - s;
        const i64 r = min(N, d);
        double* Sk = a.wsd + M.offSk + s * d;           // working sketch d x N (scratch after the copy)
        double* Wk = a.wsd + M.offW;                     // d x N
        int* Jg = a.wsi + M.offI;
        int* mv = Jg + n;

        // copy the working sketch and look for NaN/Inf (R10: identity pivots)
        if (threadIdx.x == 0) s_flag = 0;
        __syncthreads();
        int bad = 0;
        for (i64 e = threadIdx.x; e < d * N; e += BT) {
            const double v = Sk[e];
            bad |= !isfinite(v);
            Wk[e] = v;
        }
        if (bad) s_flag = 1;
        __syncthreads();
        const bool nonfinite = s_flag != 0;

        // ---- LU with partial pivoting of X = Wk^T (N x d), all r steps, with
        // full row swaps (GETRF).  One thread per column of Wk (row of X); the
        // next step's pivot candidates come out of the Schur update.  At the
        // end Wk(l, t), l < min(t, r), holds L(t, l) and Wk(c, j), c >= j, j < r,
        // holds U(j, c).
        // The multipliers use one reciprocal of the pivot per step, formed by
        // thread 0 as soon as the pivot is known, and one FMA correction that
        // makes l the quotient x / piv of GETRF; |x| is compared as an integer key.
        if (!nonfinite) {
            bool search = true;
            for (i64 j = 0; j < r; ++j) {
                const int p = search ? cta_first_argmax(Wk, d, j, N, wv, wi) : s_next;
                if (p != j)
                    for (i64 e = threadIdx.x; e < d; e += BT) {
                        const double t0 = Wk[e + j * d];
                        Wk[e + j * d] = Wk[e + (i64)p * d];
                        Wk[e + (i64)p * d] = t0;
                    }
                if (threadIdx.x == 0) ipiv[j] = p;
                __syncthreads();
                const double piv = Wk[j + j * d];
                if (abs_key(piv) != 0) {   // exact zero pivot: no elimination, as GETRF
                    // after a search (first step, or after a zero pivot) every thread
                    // forms the reciprocal itself; otherwise thread 0 formed it last step
                    const double rp = search ? 1.0 / piv : s_rp;
                    for (i64 e = j + 1 + threadIdx.x; e < d; e += BT) pc[e] = Wk[e + j * d];
                    __syncthreads();
                    unsigned long long bk = 0;
                    int bi = INT_MAX;
                    for (i64 t = j + 1 + threadIdx.x; t < N; t += BT) {
                        double* col = Wk + t * d;
                        const double x = col[j];
                        double l = x * rp;
                        l = fma(fma(-piv, l, x), rp, l);   // the quotient x / piv (Markstein correction)
                        col[j] = l;
                        if (j + 1 < d) {
                            const double v1 = fma(-l, pc[j + 1], col[j + 1]);
                            col[j + 1] = v1;
                            argmax_merge_key(bk, bi, abs_key(v1), (int)t);
                        }
#pragma unroll 4
                        for (i64 rr = j + 2; rr < d; ++rr) col[rr] = fma(-l, pc[rr], col[rr]);
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, bk, o);
                        const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
                        argmax_merge_key(bk, bi, k2, i2);
                    }
                    if (lane == 0) {
                        wv[wid] = bk;
                        wi[wid] = bi;
                    }
                    __syncthreads();
                    if (threadIdx.x == 0) {
                        unsigned long long k = wv[0];
                        int i = wi[0];
                        for (int q = 1; q < NW; ++q) argmax_merge_key(k, i, wv[q], wi[q]);
                        const int nx = (i == INT_MAX) ? (int)(j + 1) : i;
                        s_next = nx;
                        if (j + 1 < r) {   // next pivot X(nx, j+1), already updated
                            const double pv = Wk[(j + 1) + (i64)nx * d];
                            s_rp = (abs_key(pv) != 0) ? 1.0 / pv : 0.0;
                        }
                    }
                    search = false;
                } else {
                    search = true;
                }
                __syncthreads();
            }
        }

        // ---- piv_transform and the list of columns the permutation moves
        for (i64 t = threadIdx.x; t < N; t += BT) Js[t] = (int)t;
        __syncthreads();
        if (threadIdx.x == 0 && !nonfinite)
            for (i64 j = 0; j < r; ++j) {
                const int p = ipiv[j];
                const int t0 = Js[j];
                Js[j] = Js[p];
                Js[p] = t0;
            }
        if (threadIdx.x == 0) s_cnt = 0;
        __syncthreads();
        for (i64 t = threadIdx.x; t < N; t += BT) {
            const int jt = Js[t];
            Jg[t] = jt;
            if (jt != (int)t) mv[atomicAdd(&s_cnt, 1)] = (int)t;
        }
        __syncthreads();

        if (nonfinite) {
            // identity pivots: R^sk is the Householder R of the sketch itself
            cta_house_qr(Wk, d, N, pc, &s_tau);
            for (i64 t = wid; t < min(d, N); t += NW)
                for (i64 rr = t + 1 + lane; rr < d; rr += 32) Wk[rr + t * d] = 0.0;
            __syncthreads();
        } else {
            // ---- R^sk from the LU factors.  Msk(:, J^sk) = (P X)^T = U^T L^T; with
            // U^T = Q1 R1 (d x r, Householder), Msk(:, J^sk) = Q1 (R1 L^T), so
            // R^sk = R1 L^T: the R factor of the permuted sketch up to the signs
            // of its rows, which cancel in every later use (R^sk11^{-1} in the
            // preconditioner, R^sk11 in R11, R^sk12 and R^sk22 in the update).
            double* Ub = Sk;                               // d x r scratch (ld d)
            for (i64 e = threadIdx.x; e < d * r; e += BT) {
                const i64 cc = e % d, j = e / d;
                Ub[e] = (cc >= j) ? Wk[cc + j * d] : 0.0;
            }
            __syncthreads();
            cta_house_qr(Ub, d, r, pc, &s_tau);
            // column t of R^sk: rows i < min(t + 1, r) are
            //   sum_{l = i}^{lt - 1} R1(i, l) L(t, l) + [t < r] R1(i, t),  lt = min(t, r)
            for (i64 t = wid; t < N; t += NW) {
                double* col = Wk + t * d;
                const i64 lt = min(t, r);
                for (i64 l = lane; l < lt; l += 32) Lw[wid][l] = col[l];
                __syncwarp();
                const i64 top = min(t + 1, r);
                for (i64 i = lane; i < d; i += 32) {
                    double acc = 0.0;
                    if (i < top) {
                        for (i64 l = i; l < lt; ++l) acc = fma(Ub[i + l * d], Lw[wid][l], acc);
                        if (t < r) acc += Ub[i + t * d];
                    }
                    col[i] = acc;
                }
                __syncwarp();
            }
            __syncthreads();
        }

        // ---- tri_rank (Sec. 2.2 reading): |Rsk(t,t)| > 10 d u |Rsk0(0,0)|
        if (threadIdx.x == 0) {
            const double r00 = (iter == 0) ? fabs(Wk[0]) : S->r00;
            if (iter == 0) S->r00 = r00;
            const double thr = 10.0 * (double)d * 1.1102230246251565e-16 * r00;
            i64 k = 0;
            if (r00 > 0.0 && isfinite(r00))
                while (k < w && isfinite(Wk[k + k * d]) && fabs(Wk[k + k * d]) > thr) ++k;
            S->k = k;
            S->nmoved = s_cnt;
        }
    }
}

__global__ void __launch_bounds__(BT) bat_qrcp_kernel(BatArgs a, Slot sl, int slot_id, int iter) {
    for (;;) {
        const Item it = next_item(a, sl, slot_id);
        if (it.mat < 0) break;
        body_qrcp(a, it.mat, it.sub, iter);
    }
}

// ------------------------------------------------------------------ permutation (Alg. 5 on moved columns)
// Item = (matrix, 32-row chunk).  The moved columns are staged in shared
// memory, then written to their new places; chunk 0 also permutes J.
__device__ void body_perm(const BatArgs& a, const int mat, const int sub, int iter) {
    extern __shared__ double stg[];      // [moved][RCH]
    __shared__ int64_t jst[2 * kMaxD];
        {
        const BatState* S = a.st + mat;
        if (S->done) return;
        const int nm = (int)S->nmoved;
        if (nm == 0) return;
        const BatMat M = a.mats[mat];
        const i64 m = M.m, s = (i64)iter * M.b;
        const i64 r0 = (i64)sub * RCH;
        const int nr = (int)min((i64)RCH, m - r0);
        const int* Jg = a.wsi + M.offI;
        const int* mv = Jg + M.n;
        double* A = a.A + M.offA;
        for (int e = threadIdx.x; e < nm * RCH; e += BT) {
            const int q = e / RCH, rr = e % RCH;
            if (rr < nr) stg[e] = A[(r0 + rr) + (s + Jg[mv[q]]) * m];
        }
        __syncthreads();
        for (int e = threadIdx.x; e < nm * RCH; e += BT) {
            const int q = e / RCH, rr = e % RCH;
            if (rr < nr) A[(r0 + rr) + (s + mv[q]) * m] = stg[e];
        }
        if (sub == 0) {
            int64_t* J = a.jpvt + M.offJ;
            for (int q = threadIdx.x; q < nm; q += BT) jst[q] = J[s + Jg[mv[q]]];
            __syncthreads();
            for (int q = threadIdx.x; q < nm; q += BT) J[s + mv[q]] = jst[q];
        }
    }
}

__global__ void __launch_bounds__(BT) bat_perm_kernel(BatArgs a, Slot sl, int slot_id, int iter) {
    for (;;) {
        const Item it = next_item(a, sl, slot_id);
        if (it.mat < 0) break;
        body_perm(a, it.mat, it.sub, iter);
    }
}

// ------------------------------------------------------------------ Alg. 3 panel, one matrix per CTA
// Shared memory: Gs (kb x kb, ld kb) and a Gram chunk (RG x kb, [row][col]).
__device__ void body_panel(const BatArgs& a, const int mat, const int sub, int iter, int kb) {
    extern __shared__ double sm[];
    double* Gs = sm;
    double* Yc = sm + (size_t)kb * kb;
    __shared__ double Dsg[kMaxB];
    __shared__ double Rinv[kMaxB];   // reciprocals of the diagonal of the triangle in Gs
    __shared__ int s_flag, s_kc;
        {
        BatState* S = a.st + mat;
        if (S->done) return;
        const BatMat M = a.mats[mat];
        const i64 m = M.m, n = M.n, b = M.b, d = M.d;
        const i64 s = (i64)iter * b;
        const i64 c = min(n, s + b), w = c - s, rows = m - s;
        int k = (int)S->k;
        double* A = a.A + M.offA;
        double* Ap = A + s + s * m;                 // panel rows x w, ld m
        double* Y = a.wsd + M.offY;                 // rows x b, ld m
        const double* Wk = a.wsd + M.offW;          // R^sk, d x N, ld d
        double* Tb = a.wsd + M.offSm;               // T  (b x b)
        double* Pb = Tb + b * b;                    // P = R_chol Rsk(0:k, 0:w)
        double* Zb = Pb + b * b;                    // Z = Rsk11 R11^{-1}

        // early exit: the first permuted working column is all zero, or k = 0
        if (threadIdx.x == 0) s_flag = 0;
        __syncthreads();
        for (i64 i = threadIdx.x; i < rows; i += BT)
            if (Ap[i] != 0.0) s_flag = 1;
        __syncthreads();
        if (!s_flag || k == 0) {
            if (threadIdx.x == 0) {
                S->ell = s;
                S->done = 1;
            }
            return;
        }

        // ---- Pre = A_p(:, 0:k) Rsk11^{-1}  (Rsk11 staged in Gs)
        for (int e = threadIdx.x; e < k * k; e += BT) {
            const int i = e % k, j = e / k;
            Gs[i + j * kb] = (i <= j) ? Wk[i + (i64)j * d] : 0.0;
        }
        for (int j = threadIdx.x; j < k; j += BT) Rinv[j] = 1.0 / Wk[j + (i64)j * d];
        __syncthreads();
        for (i64 i = threadIdx.x; i < rows; i += BT) row_trsm_upper(Ap, m, Y, m, i, k, Gs, kb, Rinv);
        __syncthreads();

        // ---- G = Pre^T Pre, upper triangle, 4x4 tiles; thread groups split
        // the rows of each chunk and are summed in group order
        {
            const int nt4 = (k + 3) / 4;
            const int T = nt4 * (nt4 + 1) / 2;
            const int groups = (T >= BT) ? 1 : BT / T;
            const int slots = (T + BT - 1) / BT;         // 1..3 when groups == 1
            const int g = (groups == 1) ? 0 : (int)threadIdx.x / T;
            double acc[3][16];
#pragma unroll
            for (int q = 0; q < 3; ++q)
#pragma unroll
                for (int e = 0; e < 16; ++e) acc[q][e] = 0.0;
            int ti[3], tj[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                int e = (groups == 1) ? (int)threadIdx.x + q * BT : (int)threadIdx.x % T;
                if (q >= slots || g >= groups || e >= T) {
                    ti[q] = -1;
                    tj[q] = -1;
                    continue;
                }
                // tile e of the upper triangle in row-major order of tile rows
                int r = 0;
                while (e >= nt4 - r) {
                    e -= nt4 - r;
                    ++r;
                }
                ti[q] = r;
                tj[q] = r + e;
            }
            for (i64 r0 = 0; r0 < rows; r0 += RG) {
                const int nr = (int)min((i64)RG, rows - r0);
                __syncthreads();
                for (int e = threadIdx.x; e < RG * kb; e += BT) {
                    const int rr = e % RG, j = e / RG;
                    Yc[rr * kb + j] = (rr < nr && j < k) ? Y[(r0 + rr) + (i64)j * m] : 0.0;
                }
                __syncthreads();
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    if (ti[q] < 0) continue;
                    for (int rr = g; rr < nr; rr += groups) {
                        double x[4], y[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            x[u] = Yc[rr * kb + 4 * ti[q] + u];
                            y[u] = Yc[rr * kb + 4 * tj[q] + u];
                        }
#pragma unroll
                        for (int u = 0; u < 4; ++u)
#pragma unroll
                            for (int v = 0; v < 4; ++v) acc[q][4 * u + v] += x[u] * y[v];
                    }
                }
            }
            __syncthreads();
            for (int g2 = 0; g2 < groups; ++g2) {
                if (g == g2) {
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        if (ti[q] < 0) continue;
#pragma unroll
                        for (int u = 0; u < 4; ++u)
#pragma unroll
                            for (int v = 0; v < 4; ++v) {
                                const int i = 4 * ti[q] + u, j = 4 * tj[q] + v;
                                if (i <= j && j < k) {
                                    const double prev = (g2 == 0) ? 0.0 : Gs[i + j * kb];
                                    Gs[i + j * kb] = prev + acc[q][4 * u + v];
                                }
                            }
                    }
                }
                __syncthreads();
            }
        }

        // ---- R_chol = chol(G), upper, right-looking; breakdown lowers k (R15)
        if (threadIdx.x == 0) s_kc = k;
        __syncthreads();
        // thread 0 forms r_jj = g_jj * rsqrt(g_jj) and keeps 1 / r_jj for the row
        // scaling and the solve with R_chol (one special function per step)
        for (int j = 0; j < k; ++j) {
            if (threadIdx.x == 0) {
                const double sv = Gs[j + j * kb];
                const long long bits = __double_as_longlong(sv);
                if (!(bits > 0 && bits < 0x7ff0000000000000ll)) s_kc = j;   // not (finite and > 0)
                else {
                    const double ri = rsqrt(sv);
                    Gs[j + j * kb] = sv * ri;
                    Rinv[j] = ri;
                }
            }
            __syncthreads();
            if (s_kc < k) break;
            const double ri = Rinv[j];
            for (int l = j + 1 + threadIdx.x; l < k; l += BT) Gs[j + l * kb] *= ri;
            __syncthreads();
            const int nt = k - j - 1;
            for (int e = threadIdx.x; e < nt * nt; e += BT) {
                const int i = j + 1 + e % nt, l = j + 1 + e / nt;
                if (i <= l) Gs[i + l * kb] -= Gs[j + i * kb] * Gs[j + l * kb];
            }
            __syncthreads();
        }
        if (s_kc < k) {
            k = s_kc;
            if (k == 0) {
                if (threadIdx.x == 0) {
                    S->k = 0;
                    S->ell = s;
                    S->done = 1;
                }
                return;
            }
        }

        // ---- Q_c = Pre R_chol^{-1} (in place in Y); P = R_chol Rsk(0:k, 0:w)
        for (i64 i = threadIdx.x; i < rows; i += BT) row_trsm_upper(Y, m, Y, m, i, k, Gs, kb, Rinv);
        for (int e = threadIdx.x; e < k * (int)w; e += BT) {
            const int i = e % k, j = e / k;
            double acc = 0.0;
            const int tmax = min(j, k - 1);
            for (int t = i; t <= tmax; ++t) acc += Gs[i + t * kb] * Wk[t + (i64)j * d];
            Pb[i + (i64)j * b] = (i <= j) ? acc : 0.0;
        }
        __syncthreads();

        // ---- modified LU (Householder reconstruction): top k x k block in Gs
        for (int e = threadIdx.x; e < k * k; e += BT) {
            const int i = e % k, j = e / k;
            Gs[i + j * kb] = Y[i + (i64)j * m];
        }
        __syncthreads();
        for (int j = 0; j < k; ++j) {
            if (threadIdx.x == 0) {
                const double av = Gs[j + j * kb];
                const long long ab = __double_as_longlong(av);
                const double sg = (ab >= 0 || ab == (long long)0x8000000000000000ull) ? -1.0 : 1.0;   // av >= 0
                Dsg[j] = sg;                                         // s_j = -sign(a), sign(0) = +1
                const double pv = av - sg;
                Gs[j + j * kb] = pv;
                Rinv[j] = 1.0 / pv;
            }
            __syncthreads();
            const double rp = Rinv[j];
            for (int i = j + 1 + threadIdx.x; i < k; i += BT) Gs[i + j * kb] *= rp;
            __syncthreads();
            const int nt = k - j - 1;
            for (int e = threadIdx.x; e < nt * nt; e += BT) {
                const int i = j + 1 + e % nt, cc = j + 1 + e / nt;
                Gs[i + cc * kb] -= Gs[i + j * kb] * Gs[j + cc * kb];
            }
            __syncthreads();
        }
        // rows k .. rows-1: Y(i, :) = Q(i, :) U^{-1}
        for (i64 i = k + threadIdx.x; i < rows; i += BT) row_trsm_upper(Y, m, Y, m, i, k, Gs, kb, Rinv);
        // explicit unit lower top block of Y
        for (int e = threadIdx.x; e < k * k; e += BT) {
            const int i = e % k, j = e / k;
            Y[i + (i64)j * m] = (i > j) ? Gs[i + j * kb] : (i == j ? 1.0 : 0.0);
        }
        // ---- T = -U S L1^{-T}, row by row
        if ((int)threadIdx.x < k) {
            const int i = threadIdx.x;
            for (int j = 0; j < k; ++j) {
                double v = (i <= j) ? -Gs[i + j * kb] * Dsg[j] : 0.0;
                for (int t = 0; t < j; ++t) v -= Tb[i + (i64)t * b] * Gs[j + t * kb];
                Tb[i + (i64)j * b] = v;
            }
        }
        __syncthreads();
        double* tau = a.tau + M.offT + s;
        for (int j = threadIdx.x; j < k; j += BT) tau[j] = Tb[j + (i64)j * b];

        // ---- V = Y T^T (rows x k), so that the trailing update is
        // C -= V (Y^T C); T (upper, zeros below) staged in Gs
        for (int e = threadIdx.x; e < k * k; e += BT) {
            const int i = e % k, j = e / k;
            Gs[i + j * kb] = (i <= j) ? Tb[i + (i64)j * b] : 0.0;
        }
        __syncthreads();
        {
            double* V = a.wsd + M.offV;
            for (i64 i = threadIdx.x; i < rows; i += BT)
                for (int cb = 0; cb < k; cb += 16) {
                    double x[16];
#pragma unroll
                    for (int q = 0; q < 16; ++q) x[q] = 0.0;
                    for (int l = cb; l < k; ++l) {
                        const double y = Y[i + (i64)l * m];
#pragma unroll
                        for (int q = 0; q < 16; ++q) x[q] = fma(y, Gs[(cb + q) + l * kb], x[q]);
                    }
                    const int nb = min(16, k - cb);
#pragma unroll
                    for (int q = 0; q < 16; ++q)
                        if (q < nb) V[i + (i64)(cb + q) * m] = x[q];
                }
        }
        __syncthreads();

        // ---- R11 = diag(D) P into A(s:s+k, s:c) (upper part); reflectors below
        for (int e = threadIdx.x; e < k * (int)w; e += BT) {
            const int i = e % k, j = e / k;
            if (i <= j) Ap[i + (i64)j * m] = Dsg[i] * Pb[i + (i64)j * b];
        }
        for (int j = 0; j < k; ++j)
            for (i64 i = j + 1 + threadIdx.x; i < rows; i += BT) Ap[i + (i64)j * m] = Y[i + (i64)j * m];
        __syncthreads();

        // ---- Z = Rsk11 R11^{-1} for the sketch update (k = w and c < n)
        const bool cont = (k == w) && (c < n);
        if (cont) {
            __syncthreads();   // Rinv (the modified LU's) is read above until here
            for (int e = threadIdx.x; e < k * k; e += BT) {
                const int i = e % k, j = e / k;
                Gs[i + j * kb] = (i <= j) ? Dsg[i] * Pb[i + (i64)j * b] : 0.0;
            }
            for (int j = threadIdx.x; j < k; j += BT) Rinv[j] = 1.0 / (Dsg[j] * Pb[j + (i64)j * b]);
            __syncthreads();
            for (int i = threadIdx.x; i < k; i += BT) row_trsm_upper(Wk, d, Zb, b, i, k, Gs, kb, Rinv);
        }
        if (threadIdx.x == 0) {
            S->k = k;
            S->upd_iter = iter;
            if (!cont) {
                S->ell = s + k;
                S->done = 1;
                S->cont_iter = -1;
            } else {
                S->cont_iter = iter;
            }
        }
    }
}

__global__ void __launch_bounds__(BT, 1) bat_panel_kernel(BatArgs a, Slot sl, int slot_id, int iter, int kb) {
    for (;;) {
        const Item it = next_item(a, sl, slot_id);
        if (it.mat < 0) break;
        body_panel(a, it.mat, it.sub, iter, kb);
    }
}

// ------------------------------------------------------------------ trailing update
// Item = (matrix, ct-column tile of A(:, c:)), ct = 32 or 64 per matrix (the
// plan's tile shape).  W = Y^T C (k x ct), then C(0:keep, :) -= V(0:keep, :) W
// with V = Y T^T from the panel; keep = rows when k = w, else k.  Shared
// memory: Yc (RT2 x kb, [row][col]) holds Y chunks of RT rows, then V chunks of
// RT2 rows; Cc (RT x CT); Ws (kb x CT, [i][j]) (row stride CT for either ct).
// Register blocking:
//  - W: 4 x 4 blocks; the ceil(k/4) x (ct/4) blocks are spread over the
//    threads; when there are fewer blocks than threads, G = 256 / blocks groups
//    split the rows of each chunk (group g takes rows g, g + G, ...) and their
//    partial sums are added in group order (deterministic); with more blocks, a
//    thread takes two;
//  - update: JB = ct/4 column blocks of 4; thread (rb, jb) = (tid / JB, tid % JB)
//    owns RU = JB / 4 rows (4 for ct = 64, 2 for ct = 32) of an RT2-row chunk
//    and columns 4 jb .. 4 jb + 3.
constexpr int RT2 = 64;

// C(r0 .. r0 + nr, 0 .. nc) -= Vc W for one RT2-row chunk (Vc in Yc).
template <int JB>
__device__ __forceinline__ void trail_update_chunk(const double* Yc, const double* Ws, double* C, i64 m, i64 r0,
                                                   int nr, int nc, int k, int kb) {
    constexpr int RU = RT2 * JB / BT;   // rows per thread: 4 (JB = 16) or 2 (JB = 8)
    static_assert(RU * (BT / JB) == RT2, "the threads cover the chunk's rows");
    const int rb = threadIdx.x / JB, jb = threadIdx.x % JB;
    // this thread's block of C, loaded before the k loop so that the
    // global-load latency overlaps the FMAs
    double cpre[RU][4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const int col = 4 * jb + v;
#pragma unroll
        for (int u = 0; u < RU; ++u)
            cpre[u][v] = (col < nc && RU * rb + u < nr) ? C[(r0 + RU * rb + u) + (i64)col * m] : 0.0;
    }
    double u4[RU][4];
#pragma unroll
    for (int u = 0; u < RU; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) u4[u][v] = 0.0;
    for (int i = 0; i < k; ++i) {
        double vv[RU], wv[4];
#pragma unroll
        for (int u = 0; u < RU; ++u) vv[u] = Yc[(RU * rb + u) * kb + i];
#pragma unroll
        for (int v = 0; v < 4; ++v) wv[v] = Ws[i * CT + 4 * jb + v];
#pragma unroll
        for (int u = 0; u < RU; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) u4[u][v] = fma(vv[u], wv[v], u4[u][v]);
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const int col = 4 * jb + v;
        if (col < nc)
#pragma unroll
            for (int u = 0; u < RU; ++u)
                if (RU * rb + u < nr) C[(r0 + RU * rb + u) + (i64)col * m] = cpre[u][v] - u4[u][v];
    }
}

__device__ void body_trailing(const BatArgs& a, const int mat, const int sub, int iter, int kb) {
    extern __shared__ double sm[];
    double* Yc = sm;
    double* Cc = Yc + (size_t)RT2 * kb;
    double* Ws = Cc + (size_t)RT * CT;
        {
        const BatState* S = a.st + mat;
        if (S->upd_iter != iter) return;
        const BatMat M = a.mats[mat];
        const i64 m = M.m, n = M.n, b = M.b;
        const i64 s = (i64)iter * b;
        const i64 c = min(n, s + b), w = c - s, rows = m - s;
        const int k = (int)S->k;
        const i64 keep = (k == w) ? rows : k;
        const int ct = (int)M.ct;
        const i64 j0 = c + (i64)sub * ct;
        const int nc = (int)min((i64)ct, n - j0);
        if (nc <= 0) return;
        const double* Y = a.wsd + M.offY;
        const double* V = a.wsd + M.offV;
        double* C = a.A + M.offA + s + j0 * m;

        // ---- W = Y^T C
        const int jbs = ct / 4;   // column blocks of the tile
        const int nblk = ((k + 3) / 4) * jbs;
        const int G = (nblk >= BT) ? 1 : BT / nblk;
        const int g = (G == 1) ? 0 : (int)threadIdx.x / nblk;
        int bi[2], bj[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int blk = (G == 1) ? (int)threadIdx.x + q * BT : (int)threadIdx.x % nblk;
            const bool on = (q == 0 || G == 1) && g < G && blk < nblk && (G == 1 || q == 0);
            bi[q] = on ? 4 * (blk / jbs) : -1;
            bj[q] = on ? 4 * (blk % jbs) : -1;
        }
        double acc[2][4][4];
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[q][u][v] = 0.0;
        for (i64 r0 = 0; r0 < rows; r0 += RT) {
            const int nr = (int)min((i64)RT, rows - r0);
            __syncthreads();
            for (int e = threadIdx.x; e < RT * kb; e += BT) {
                const int rr = e % RT, i = e / RT;
                Yc[rr * kb + i] = (rr < nr && i < k) ? Y[(r0 + rr) + (i64)i * m] : 0.0;
            }
            for (int e = threadIdx.x; e < RT * ct; e += BT) {
                const int rr = e % RT, j = e / RT;
                Cc[rr * CT + j] = (rr < nr && j < nc) ? C[(r0 + rr) + (i64)j * m] : 0.0;
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                if (bi[q] < 0) continue;
                for (int rr = g; rr < nr; rr += G) {
                    double y[4], cv[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) y[u] = Yc[rr * kb + bi[q] + u];
#pragma unroll
                    for (int v = 0; v < 4; ++v) cv[v] = Cc[rr * CT + bj[q] + v];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int v = 0; v < 4; ++v) acc[q][u][v] = fma(y[u], cv[v], acc[q][u][v]);
                }
            }
        }
        // add the groups' partial sums into Ws in group order
        for (int g2 = 0; g2 < G; ++g2) {
            if (g == g2) {
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    if (bi[q] < 0) continue;
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            const int i = bi[q] + u;
                            if (i < k) {
                                double* wp = Ws + i * CT + bj[q] + v;
                                *wp = (g2 == 0) ? acc[q][u][v] : *wp + acc[q][u][v];
                            }
                        }
                }
            }
            __syncthreads();
        }
        // ---- C(0:keep, :) -= V(0:keep, :) W
        for (i64 r0 = 0; r0 < keep; r0 += RT2) {
            const int nr = (int)min((i64)RT2, keep - r0);
            __syncthreads();
            for (int e = threadIdx.x; e < RT2 * kb; e += BT) {
                const int rr = e % RT2, i = e / RT2;
                Yc[rr * kb + i] = (rr < nr && i < k) ? V[(r0 + rr) + (i64)i * m] : 0.0;
            }
            __syncthreads();
            if (ct == CT)
                trail_update_chunk<CT / 4>(Yc, Ws, C, m, r0, nr, nc, k, kb);
            else
                trail_update_chunk<CT_MIN / 4>(Yc, Ws, C, m, r0, nr, nc, k, kb);
        }
    }
}

__global__ void __launch_bounds__(BT) bat_trailing_kernel(BatArgs a, Slot sl, int slot_id, int iter, int kb) {
    for (;;) {
        const Item it = next_item(a, sl, slot_id);
        if (it.mat < 0) break;
        body_trailing(a, it.mat, it.sub, iter, kb);
    }
}

// ------------------------------------------------------------------ sketch update (Duersch-Gu)
// Item = (matrix, ct-column tile of Msk(:, c:)), the trailing update's tiles.
__device__ void body_skupdate(const BatArgs& a, const int mat, const int sub, int iter) {
        {
        const BatState* S = a.st + mat;
        if (S->cont_iter != iter) return;
        const BatMat M = a.mats[mat];
        const i64 m = M.m, n = M.n, b = M.b, d = M.d;
        const i64 s = (i64)iter * b;
        const i64 c = min(n, s + b), w = c - s;
        const i64 j0 = c + (i64)sub * M.ct;
        const int nc = (int)min(M.ct, n - j0);
        if (nc <= 0) return;
        const double* Wk = a.wsd + M.offW;
        const double* Zb = a.wsd + M.offSm + 2 * b * b;
        const double* A = a.A + M.offA;
        double* Sk = a.wsd + M.offSk;
        for (i64 e = threadIdx.x; e < d * nc; e += BT) {
            const i64 i = e % d, jx = j0 + e / d;
            double v = Wk[i + (jx - s) * d];
            if (i < w) {
                double acc = 0.0;
                for (i64 l = i; l < w; ++l) acc += Zb[i + l * b] * A[(s + l) + jx * m];
                v -= acc;
            }
            Sk[i + jx * d] = v;
        }
    }
}

__global__ void __launch_bounds__(BT) bat_skupdate_kernel(BatArgs a, Slot sl, int slot_id, int iter) {
    for (;;) {
        const Item it = next_item(a, sl, slot_id);
        if (it.mat < 0) break;
        body_skupdate(a, it.mat, it.sub, iter);
    }
}

// ------------------------------------------------------------------ finish
__device__ void body_finish(const BatArgs& a, const int mat, const int sub) {
        {
        const BatMat M = a.mats[mat];
        const BatState* S = a.st + mat;
        const i64 m = M.m, n = M.n;
        int64_t* J = a.jpvt + M.offJ;
        for (i64 j = threadIdx.x; j < n; j += BT) J[j] += 1;
        const i64 ell = S->info ? 0 : S->ell;
        // row norms ||R(r, r:n)||^2 for r < ell, in the Y scratch
        double* rn = a.wsd + M.offY;
        const double* A = a.A + M.offA;
        for (i64 r = threadIdx.x; r < ell; r += BT) {
            double acc = 0.0;
            for (i64 cc = r; cc < n; ++cc) acc += A[r + cc * m] * A[r + cc * m];
            rn[r] = acc;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const double thr = a.tol * S->anorm;
            const double thr2 = thr * thr;
            double tail = 0.0;
            i64 best = ell;
            for (i64 i = ell - 1; i >= 0; --i) {
                tail += rn[i];
                if (tail <= thr2) best = i;
                else break;
            }
            a.rank_out[mat] = ell;
            if (a.trunc_out) a.trunc_out[mat] = best;
            if (a.info_out) a.info_out[mat] = S->info;
        }
    }
}

__global__ void __launch_bounds__(BT) bat_finish_kernel(BatArgs a, Slot sl, int slot_id) {
    for (;;) {
        const Item it = next_item(a, sl, slot_id);
        if (it.mat < 0) break;
        body_finish(a, it.mat, it.sub);
    }
}

// ------------------------------------------------------------------ dependency-driven form
// One persistent kernel runs every phase of every matrix.  Its CTAs take
// tasks from a device queue; a matrix moves to its next phase as soon as the
// last task of its current phase finishes, independently of the others, so no
// SM waits for the slowest matrix of a lock-step iteration.  Per matrix:
//   INIT -> SKETCH (one task per 64-column tile) -> per block iteration
//   QRCP (Alg. 2 plus the column permutation) -> PANEL (Alg. 3) ->
//   TRAIL (one task per 64-column tile, plus that tile's sketch update)
//   -> QRCP of the next block, or FINISH.
// The last finisher of a phase (an atomic count per matrix) pushes the next
// phase's tasks.  There are two queues, each a slot array written once per
// run (a slot holds task + 1 once published by a release store, 0 before):
//  - the hot queue takes every task of the largest matrices, whose chains of
//    phases are the critical path;
//  - the normal queue takes the rest.
// A worker reserves the next normal slot; while that slot is unpublished it
// claims published hot tasks (compare-and-swap on the hot head) and runs
// them, keeping its reservation.  Polls are bounded; a worker that gives up
// records a timeout.
enum : int { T_INIT = 0, T_SKETCH = 1, T_QRCP = 2, T_PANEL = 3, T_TRAIL = 4, T_FINISH = 5 };

struct MegaArgs {
    unsigned long long* slots;   // normal queue, cap entries
    unsigned long long* hslots;  // hot queue, hcap entries
    unsigned int* ctl;           // [0] head, [1] tail, [2] matrices done, [3] error, [4] hot head, [5] hot tail
    int* pending;                // per matrix: unfinished tasks of its current phase
    int* finished;               // per matrix: 1 once FINISH has run
    const int* order;            // initial INIT order (largest first); the first nhot are hot
    const int* hot;              // per matrix: 1 if its tasks go to the hot queue
    unsigned int cap, hcap;
    int batch;
    int nhot;
    int kb;
};

__device__ __forceinline__ i64 dcdiv(i64 x, i64 y) { return (x + y - 1) / y; }

__device__ __forceinline__ unsigned long long task_enc(int mat, int type, int iter, int sub) {
    return ((unsigned long long)mat << 44) | ((unsigned long long)type << 40) | ((unsigned long long)iter << 20) |
           (unsigned long long)sub;
}

__device__ __forceinline__ unsigned long long ld_acq_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned int ld_acq_u32(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ void task_push(const MegaArgs& q, unsigned long long t, bool hot) {
    const unsigned int idx = atomicAdd(&q.ctl[hot ? 5 : 1], 1u);
    if (idx >= (hot ? q.hcap : q.cap)) {
        atomicExch(&q.ctl[3], 1u);
        return;
    }
    unsigned long long* slot = (hot ? q.hslots : q.slots) + idx;
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(slot), "l"(t + 1ull) : "memory");
}

// Thread 0, after every thread of the CTA has finished task (mat, type, iter):
// if it was the last task of the matrix's phase, start the next phase.
__device__ void task_done(const BatArgs& a, const MegaArgs& q, int mat, int type, int iter) {
    __threadfence();
    if (atomicSub(&q.pending[mat], 1) != 1) return;
    __threadfence();
    const BatMat M = a.mats[mat];
    const BatState* S = a.st + mat;
    int ntype = T_FINISH, niter = iter, count = 1;
    switch (type) {
        case T_INIT:
            if (!S->done) { ntype = T_SKETCH; count = (int)dcdiv(M.n, CT); }
            break;
        case T_SKETCH: ntype = T_QRCP; niter = 0; break;
        case T_QRCP: ntype = T_PANEL; break;
        case T_PANEL:
            if (S->upd_iter == iter) {
                const i64 c = min(M.n, (i64)iter * M.b + M.b);
                const int nt = (int)dcdiv(M.n - c, M.ct);
                if (nt > 0) { ntype = T_TRAIL; count = nt; }
            }
            break;
        case T_TRAIL:
            if (S->cont_iter == iter) { ntype = T_QRCP; niter = iter + 1; }
            break;
        default:
            q.finished[mat] = 1;
            __threadfence();
            atomicAdd(&q.ctl[2], 1u);
            return;
    }
    q.pending[mat] = count;
    __threadfence();
    const bool hot = q.hot[mat] != 0;
    for (int sub = 0; sub < count; ++sub) task_push(q, task_enc(mat, ntype, niter, sub), hot);
}

constexpr unsigned long long kPollLimit = 1ull << 27;

__global__ void __launch_bounds__(BT, 3) bat_mega_kernel(BatArgs a, MegaArgs q) {
    __shared__ unsigned long long s_task;
    __shared__ int s_stop;
    __shared__ unsigned int s_low;    // reserved normal slot (valid while s_have)
    __shared__ int s_have;
    if (threadIdx.x == 0) s_have = 0;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            s_stop = 0;
            if (!s_have) {
                s_low = atomicAdd(&q.ctl[0], 1u);
                s_have = 1;
            }
            const bool low_ok = s_low < q.cap;
            unsigned long long spins = 0;
            for (;;) {
                // a published hot task, if any
                const unsigned int h = *((volatile unsigned int*)&q.ctl[4]);
                if (h < q.hcap) {
                    const unsigned long long v = ld_acq_u64(q.hslots + h);
                    if (v) {
                        if (atomicCAS(&q.ctl[4], h, h + 1) == h) {
                            s_task = v - 1ull;
                            break;
                        }
                        continue;
                    }
                }
                // the reserved normal slot
                if (low_ok) {
                    const unsigned long long v = ld_acq_u64(q.slots + s_low);
                    if (v) {
                        s_task = v - 1ull;
                        s_have = 0;
                        break;
                    }
                }
                if (ld_acq_u32(&q.ctl[2]) >= (unsigned)q.batch || ld_acq_u32(&q.ctl[3])) {
                    s_stop = 1;
                    break;
                }
                if (++spins > kPollLimit) {
                    atomicExch(&q.ctl[3], 1u);
                    s_stop = 1;
                    break;
                }
            }
        }
        __syncthreads();
        if (s_stop) break;
        const unsigned long long t = s_task;
        const int mat = (int)(t >> 44), type = (int)((t >> 40) & 15ull), iter = (int)((t >> 20) & 0xFFFFFull),
                  sub = (int)(t & 0xFFFFFull);
        switch (type) {
            case T_INIT: body_init(a, mat, 0); break;
            case T_SKETCH: body_sketch(a, mat, sub); break;
            case T_QRCP: {
                body_qrcp(a, mat, 0, iter);
                const i64 nch = dcdiv(a.mats[mat].m, RCH);
                for (i64 ch = 0; ch < nch; ++ch) {
                    __syncthreads();
                    body_perm(a, mat, (int)ch, iter);
                }
                break;
            }
            case T_PANEL: body_panel(a, mat, 0, iter, q.kb); break;
            case T_TRAIL:
                body_trailing(a, mat, sub, iter, q.kb);
                __syncthreads();
                body_skupdate(a, mat, sub, iter);
                break;
            default: body_finish(a, mat, 0); break;
        }
        __syncthreads();
        if (threadIdx.x == 0) task_done(a, q, mat, type, iter);
    }
}

// Reset the queue for a run: slot i < batch holds INIT of order[i], the rest
// are empty; every matrix has one pending task.
__global__ void mega_reset_kernel(MegaArgs q) {
    const unsigned int stride = gridDim.x * blockDim.x;
    const unsigned int nlow = (unsigned)(q.batch - q.nhot);
    for (unsigned int i = blockIdx.x * blockDim.x + threadIdx.x; i < q.cap; i += stride)
        q.slots[i] = (i < nlow) ? task_enc(q.order[q.nhot + i], T_INIT, 0, 0) + 1ull : 0ull;
    for (unsigned int i = blockIdx.x * blockDim.x + threadIdx.x; i < q.hcap; i += stride)
        q.hslots[i] = (i < (unsigned)q.nhot) ? task_enc(q.order[i], T_INIT, 0, 0) + 1ull : 0ull;
    for (unsigned int i = blockIdx.x * blockDim.x + threadIdx.x; i < (unsigned)q.batch; i += stride) {
        q.pending[i] = 1;
        q.finished[i] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        q.ctl[0] = 0;
        q.ctl[1] = nlow;
        q.ctl[2] = 0;
        q.ctl[3] = 0;
        q.ctl[4] = 0;
        q.ctl[5] = (unsigned)q.nhot;
    }
}

// After a run: a matrix the queue did not finish (a worker gave up) reports
// BQRRP_ETIMEOUT and rank 0.
__global__ void mega_check_kernel(BatArgs a, MegaArgs q) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= q.batch || q.finished[i]) return;
    a.rank_out[i] = 0;
    if (a.trunc_out) a.trunc_out[i] = 0;
    if (a.info_out) a.info_out[i] = BQRRP_ETIMEOUT;
}

}  // namespace

// ================================================================== host plan
struct BatchPlan {
    i64 batch = 0;
    double tol = 0.0;
    std::vector<BatMat> mats;
    std::vector<i64> mh, nh, bh, dh;
    std::vector<uint64_t> seeds;
    i64 iters = 0;
    int kb = 16;                     // bmax rounded up to 16
    int maxmoved = 1;
    // launch list
    enum Kind { K_INIT, K_SKETCH, K_QRCP, K_PERM, K_PANEL, K_TRAIL, K_SKUPD, K_FINISH };
    struct Launch {
        Kind kind;
        int iter;
        Slot slot;
        double flops;            // algorithmic FLOPs of the launch if every block is full rank
    };
    std::vector<Launch> launches;
    std::vector<int> smat, spre;
    // dependency-driven form: queue capacity, initial order, launch shape
    bool mega = true;
    unsigned int qcap = 0, hcap = 0;
    int nhot = 0;
    std::vector<int> order, hot;
    size_t dsm_mega = 0;
    int grid_mega = 0;
    int grid_cap = 0;                // > 0: at most this many persistent CTAs (leaves SMs to other work)
    // device image offsets (bytes) in the workspace
    size_t o_mats = 0, o_state = 0, o_smat = 0, o_spre = 0, o_ctr = 0, o_wsd = 0, o_wsi = 0, total = 0;
    size_t o_order = 0, o_slots = 0, o_qctl = 0, o_pend = 0, o_fin = 0, o_hot = 0, o_hslots = 0;
    size_t n_wsd = 0, n_wsi = 0;
    // grid sizes
    int grid[8] = {0};
    size_t dsm_perm = 0, dsm_panel = 0, dsm_trail = 0, dsm_qrcp = 0;
    // device image written where
    void* uploaded_ws = nullptr;
    int device = -1;
    // captured graph and the pointers it was captured with
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t cap = nullptr;      // private stream the graph is captured on
    const void* gkey[7] = {nullptr};
    ~BatchPlan() {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (cap) cudaStreamDestroy(cap);
    }
};

namespace {

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Costs used only to order the work queues (largest first).
double cost_qrcp(const BatMat& M, i64 s) {
    const double N = (double)(M.n - s), d = (double)M.d;
    return N * d * d;
}
double cost_panel(const BatMat& M, i64 s) {
    const double rows = (double)(M.m - s), b = (double)M.b;
    return rows * b * b;
}

void add_slot(BatchPlan& P, BatchPlan::Kind kind, int iter, std::vector<std::pair<double, int>>& order,
              const std::vector<int>& nsub_of) {
    std::stable_sort(order.begin(), order.end(),
                     [](const std::pair<double, int>& x, const std::pair<double, int>& y) { return x.first > y.first; });
    Slot sl;
    sl.first = (int)P.smat.size();
    sl.nmats = 0;
    int tot = 0;
    // spre holds nmats + 1 entries per slot starting at (first + slot index):
    // store the prefix right after this slot's previous entries
    std::vector<int> pre;
    for (auto& o : order) {
        const int ns = nsub_of[o.second];
        if (ns <= 0) continue;
        P.smat.push_back(o.second);
        pre.push_back(tot);
        tot += ns;
        ++sl.nmats;
    }
    pre.push_back(tot);
    sl.total = tot;
    // spre index for slot q is smat.first + q (one extra entry per slot so far)
    const int slot_idx = (int)P.launches.size();
    (void)slot_idx;
    P.spre.insert(P.spre.end(), pre.begin(), pre.end());
    P.launches.push_back(BatchPlan::Launch{kind, iter, sl, 0.0});
}

// Algorithmic FLOPs of one launch for matrix M at iteration it, assuming the
// panel keeps all w columns (the profile's accounting; the kernels do less
// when a matrix ends early).
double launch_flops(BatchPlan::Kind kind, const BatMat& M, i64 it) {
    const double m = (double)M.m, n = (double)M.n, d = (double)M.d;
    const i64 s = it * M.b;
    if (kind == BatchPlan::K_SKETCH) return 2.0 * d * m * n;
    if (s >= M.n) return 0.0;
    const double N = (double)(M.n - s), rows = (double)(M.m - s);
    const double w = (double)(std::min(M.n, s + M.b) - s), nc = N - w;
    switch (kind) {
        case BatchPlan::K_QRCP: {
            double lu = 0.0;
            const i64 r = std::min<i64>(M.n - s, M.d);
            for (i64 j = 0; j < r; ++j) lu += (N - j - 1) * (1.0 + 2.0 * (d - j - 1));
            const double kq = std::min(d, N);
            const double qr = 2.0 * d * N * kq - (d + N) * kq * kq + 2.0 * kq * kq * kq / 3.0;
            return lu + qr;
        }
        case BatchPlan::K_PANEL: return 4.0 * rows * w * w + 2.0 * w * w * w;
        case BatchPlan::K_TRAIL: return 4.0 * rows * w * nc;
        case BatchPlan::K_SKUPD: return (nc > 0.0) ? w * w * nc : 0.0;
        default: return 0.0;
    }
}

}  // namespace

// Plan with caller-chosen element offsets of every matrix in A (lda = m_i),
// jpvt and tau (all three may be null: the packed layout).
int batch_plan_create_ex(BatchPlan** out, i64 batch, const i64* m, const i64* n, const i64* b, const i64* d,
                         const uint64_t* seed, double tol, const i64* offA_in, const i64* offJ_in,
                         const i64* offT_in, const i64* ct_in) {
    if (!out) { set_error("plan pointer is null"); return -1; }
    *out = nullptr;
    if (batch < 0) { set_error("batch < 0"); return -2; }
    if (batch > 0 && (!m || !n || !b || !d || !seed)) { set_error("null size array"); return -3; }
    if (!(tol >= 0.0) || !std::isfinite(tol)) { set_error("trunc_tol must be finite and >= 0"); return -9; }
    for (i64 i = 0; i < batch; ++i) {
        if (n[i] < 0 || m[i] < n[i]) { set_error("matrix %lld: need m >= n >= 0", (long long)i); return -3; }
        if (n[i] > kMaxN) { set_error("matrix %lld: n > %d", (long long)i, kMaxN); return BQRRP_EUNSUPPORTED; }
        if (m[i] > (i64)1 << 24) { set_error("matrix %lld: m > 2^24", (long long)i); return BQRRP_EUNSUPPORTED; }
        if (b[i] < 1 || b[i] > kMaxB) { set_error("matrix %lld: b outside [1, %d]", (long long)i, kMaxB); return -5; }
        if (d[i] < b[i] || d[i] > kMaxD) { set_error("matrix %lld: d outside [b, %d]", (long long)i, kMaxD); return -6; }
        if (ct_in && ct_in[i] != CT && ct_in[i] != CT_MIN) {
            set_error("matrix %lld: tile columns must be %d or %d", (long long)i, CT_MIN, CT);
            return -10;
        }
    }
    Device dev;
    BQ_TRY(current_device(&dev));
    BatchPlan* P = new BatchPlan();
    P->batch = batch;
    P->tol = tol;
    P->device = dev.id;
    P->mh.assign(m, m + batch);
    P->nh.assign(n, n + batch);
    P->bh.assign(b, b + batch);
    P->dh.assign(d, d + batch);
    P->seeds.assign(seed, seed + batch);
    P->mats.resize(batch);
    i64 offA = 0, offJ = 0;
    size_t wd = 0, wi = 0;
    i64 bmax = 1, iters = 0;
    int maxmoved = 1;
    for (i64 i = 0; i < batch; ++i) {
        BatMat& M = P->mats[i];
        M.m = m[i];
        M.n = n[i];
        M.b = b[i];
        M.d = d[i];
        M.ct = ct_in ? ct_in[i] : CT;
        M.seed = seed[i];
        M.offA = offA_in ? offA_in[i] : offA;
        M.offJ = offJ_in ? offJ_in[i] : offJ;
        M.offT = offT_in ? offT_in[i] : offJ;
        offA += m[i] * n[i];
        offJ += n[i];
        const i64 nn = std::max<i64>(n[i], 1);
        M.offSk = (i64)wd; wd += (size_t)(d[i] * nn + 31) / 32 * 32;
        M.offW = (i64)wd;  wd += (size_t)(d[i] * nn + 31) / 32 * 32;
        M.offY = (i64)wd;  wd += (size_t)(std::max<i64>(m[i], 1) * b[i] + 31) / 32 * 32;
        M.offV = (i64)wd;  wd += (size_t)(std::max<i64>(m[i], 1) * b[i] + 31) / 32 * 32;
        M.offSm = (i64)wd; wd += (size_t)(3 * b[i] * b[i] + 31) / 32 * 32;
        M.offI = (i64)wi;  wi += (size_t)(2 * nn + 31) / 32 * 32;
        bmax = std::max(bmax, b[i]);
        if (n[i] > 0) iters = std::max(iters, cdiv(n[i], b[i]));
        maxmoved = std::max<int>(maxmoved, (int)(2 * std::min(n[i], d[i])));
    }
    P->iters = iters;
    P->kb = (int)((bmax + 15) / 16 * 16);
    P->maxmoved = maxmoved;
    P->n_wsd = wd;
    P->n_wsi = wi;

    // dependency-driven form: the initial order (largest first), the hot
    // matrices (the largest tenth, 1 to 512 of them) and every task a run can
    // push into each queue
    {
        std::vector<std::pair<double, int>> ord;
        std::vector<unsigned long long> tasks(batch);
        for (i64 i = 0; i < batch; ++i) {
            const BatMat& M = P->mats[i];
            unsigned long long t = 2;                           // INIT, FINISH
            if (M.n > 0) {
                t += (unsigned long long)cdiv(M.n, CT);         // SKETCH tiles
                for (i64 it = 0; it * M.b < M.n; ++it) {
                    const i64 c = std::min(M.n, it * M.b + M.b);
                    t += 2 + (unsigned long long)cdiv(M.n - c, M.ct);   // QRCP, PANEL, TRAIL tiles
                }
            }
            tasks[i] = t;
            ord.push_back({2.0 * M.m * (double)M.n * M.n, (int)i});
        }
        std::stable_sort(ord.begin(), ord.end(), [](const std::pair<double, int>& x, const std::pair<double, int>& y) {
            return x.first > y.first;
        });
        P->nhot = (int)std::min<i64>(batch, std::min<i64>(512, std::max<i64>(1, batch / 10)));
        if (batch == 0) P->nhot = 0;
        P->hot.assign(batch, 0);
        unsigned long long cap = 0, hcap = 0;
        for (i64 r = 0; r < batch; ++r) {
            const int i = ord[r].second;
            P->order.push_back(i);
            if (r < P->nhot) {
                P->hot[i] = 1;
                hcap += tasks[i];
            } else {
                cap += tasks[i];
            }
        }
        if (cap + hcap >= (1ull << 31)) { set_error("batched: too many tasks"); delete P; return BQRRP_EUNSUPPORTED; }
        P->qcap = (unsigned int)std::max<unsigned long long>(cap, 1);
        P->hcap = (unsigned int)std::max<unsigned long long>(hcap, 1);
        P->mega = true;   // the dependency-driven form; bqrrp_batch_plan_set_form selects the other
    }

    // launch list and work queues
    std::vector<std::pair<double, int>> order;
    std::vector<int> ns(batch);
    auto build = [&](BatchPlan::Kind kind, int iter, auto nsub, auto cost) {
        order.clear();
        for (i64 i = 0; i < batch; ++i) {
            ns[i] = nsub(P->mats[i]);
            if (ns[i] > 0) order.push_back({cost(P->mats[i]), (int)i});
        }
        add_slot(*P, kind, iter, order, ns);
        double fl = 0.0;
        for (auto& o : order) fl += launch_flops(kind, P->mats[o.second], iter);
        P->launches.back().flops = fl;
    };
    build(BatchPlan::K_INIT, 0, [](const BatMat&) { return 1; },
          [](const BatMat& M) { return (double)(M.m * M.n); });
    build(BatchPlan::K_SKETCH, 0, [](const BatMat& M) { return (int)cdiv(M.n, CT); },
          [](const BatMat& M) { return (double)(M.m * M.d); });
    for (i64 it = 0; it < iters; ++it) {
        auto active = [it](const BatMat& M) { return M.n > 0 && it * M.b < M.n; };
        build(BatchPlan::K_QRCP, (int)it, [&](const BatMat& M) { return active(M) ? 1 : 0; },
              [it](const BatMat& M) { return cost_qrcp(M, it * M.b); });
        build(BatchPlan::K_PERM, (int)it, [&](const BatMat& M) { return active(M) ? (int)cdiv(M.m, RCH) : 0; },
              [](const BatMat& M) { return (double)M.d; });
        build(BatchPlan::K_PANEL, (int)it, [&](const BatMat& M) { return active(M) ? 1 : 0; },
              [it](const BatMat& M) { return cost_panel(M, it * M.b); });
        auto ntail = [it](const BatMat& M) {
            const i64 c = std::min(M.n, it * M.b + M.b);
            return (M.n > 0 && it * M.b < M.n) ? (int)cdiv(M.n - c, M.ct) : 0;
        };
        build(BatchPlan::K_TRAIL, (int)it, ntail,
              [it](const BatMat& M) { return (double)(M.m - it * M.b) * (double)M.b; });
        build(BatchPlan::K_SKUPD, (int)it, ntail, [](const BatMat& M) { return (double)M.d * (double)M.b; });
    }
    build(BatchPlan::K_FINISH, 0, [](const BatMat&) { return 1; },
          [](const BatMat& M) { return (double)M.n; });

    // spre entries: slot q's prefix starts at smat-first + q
    // (add_slot appended nmats + 1 entries per slot in order, so the running
    // offset of slot q is sum over earlier slots of (nmats + 1) = first + q)
    const size_t nl = P->launches.size();
    size_t off = 0;
    P->o_mats = off;  off = align256(off + sizeof(BatMat) * std::max<i64>(batch, 1));
    P->o_state = off; off = align256(off + sizeof(BatState) * std::max<i64>(batch, 1));
    P->o_smat = off;  off = align256(off + sizeof(int) * std::max<size_t>(P->smat.size(), 1));
    P->o_spre = off;  off = align256(off + sizeof(int) * std::max<size_t>(P->spre.size(), 1));
    P->o_ctr = off;   off = align256(off + sizeof(unsigned int) * std::max<size_t>(nl, 1));
    P->o_order = off; off = align256(off + sizeof(int) * std::max<i64>(batch, 1));
    P->o_slots = off; off = align256(off + sizeof(unsigned long long) * (size_t)P->qcap);
    P->o_hslots = off; off = align256(off + sizeof(unsigned long long) * (size_t)P->hcap);
    P->o_hot = off;   off = align256(off + sizeof(int) * std::max<i64>(batch, 1));
    P->o_qctl = off;  off = align256(off + sizeof(unsigned int) * 8);
    P->o_pend = off;  off = align256(off + sizeof(int) * std::max<i64>(batch, 1));
    P->o_fin = off;   off = align256(off + sizeof(int) * std::max<i64>(batch, 1));
    P->o_wsd = off;   off = align256(off + sizeof(double) * std::max<size_t>(P->n_wsd, 1));
    P->o_wsi = off;   off = align256(off + sizeof(int) * std::max<size_t>(P->n_wsi, 1));
    P->total = off;

    // dynamic shared memory and grid sizes
    const int kb = P->kb;
    P->dsm_perm = sizeof(double) * (size_t)maxmoved * RCH;
    P->dsm_panel = sizeof(double) * ((size_t)kb * kb + (size_t)RG * kb);
    P->dsm_trail = sizeof(double) * ((size_t)RT2 * kb + (size_t)RT * CT + (size_t)kb * CT);
    P->dsm_qrcp = sizeof(double) * NW * kMaxD + sizeof(int) * kMaxN;
    struct KInfo { const void* fn; size_t dsm; };
    const KInfo ki[8] = {
        {(const void*)bat_init_kernel, 0},        {(const void*)bat_sketch_kernel, 0},
        {(const void*)bat_qrcp_kernel, P->dsm_qrcp}, {(const void*)bat_perm_kernel, P->dsm_perm},
        {(const void*)bat_panel_kernel, P->dsm_panel}, {(const void*)bat_trailing_kernel, P->dsm_trail},
        {(const void*)bat_skupdate_kernel, 0},    {(const void*)bat_finish_kernel, 0}};
    for (int q = 0; q < 8; ++q) {
        if (ki[q].dsm > 0) {
            // always set: dynamic plus static shared memory may exceed the 48 KiB
            // default even when the dynamic part alone does not
            cudaError_t e = cudaFuncSetAttribute(ki[q].fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ki[q].dsm);
            if (e != cudaSuccess) {
                set_error("cudaFuncSetAttribute: %s", cudaGetErrorString(e));
                delete P;
                return BQRRP_ECUDA;
            }
        }
        int occ = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ki[q].fn, BT, ki[q].dsm);
        if (e != cudaSuccess || occ < 1) {
            set_error("kernel %d cannot be resident (%s)", q, cudaGetErrorString(e));
            delete P;
            return BQRRP_ECUDA;
        }
        P->grid[q] = occ * dev.sms;
    }
    P->dsm_mega = std::max(std::max(P->dsm_perm, P->dsm_qrcp), std::max(P->dsm_panel, P->dsm_trail));
    {
        cudaError_t e = cudaFuncSetAttribute((const void*)bat_mega_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)P->dsm_mega);
        int occ = 0;
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void*)bat_mega_kernel, BT, P->dsm_mega);
        if (e != cudaSuccess || occ < 1) {
            set_error("dependency-driven kernel cannot be resident (%s)", cudaGetErrorString(e));
            delete P;
            return BQRRP_ECUDA;
        }
        P->grid_mega = occ * dev.sms;
    }
    *out = P;
    return 0;
}

int batch_plan_create(BatchPlan** out, i64 batch, const i64* m, const i64* n, const i64* b, const i64* d,
                      const uint64_t* seed, double tol) {
    return batch_plan_create_ex(out, batch, m, n, b, d, seed, tol, nullptr, nullptr, nullptr, nullptr);
}

size_t batch_plan_bytes(const BatchPlan* P) { return P ? P->total : 0; }

// Copies on the caller's stream, so they are ordered after its earlier work
// (a previous plan's kernels on the same workspace) and before this call's
// launches.  The sources are host memory the plan owns, or `img`, which is
// pageable: cudaMemcpyAsync stages pageable memory before it returns, so
// `img` may go out of scope afterwards.
static int batch_upload(BatchPlan* P, char* ws, cudaStream_t stream) {
    // records and launch queues up to the counters, then the initial task order
    std::vector<char> img(P->o_ctr);
    if (P->batch > 0) std::memcpy(img.data() + P->o_mats, P->mats.data(), sizeof(BatMat) * P->batch);
    if (!P->smat.empty()) std::memcpy(img.data() + P->o_smat, P->smat.data(), sizeof(int) * P->smat.size());
    if (!P->spre.empty()) std::memcpy(img.data() + P->o_spre, P->spre.data(), sizeof(int) * P->spre.size());
    BQ_CUDA(cudaMemcpyAsync(ws, img.data(), img.size(), cudaMemcpyHostToDevice, stream));
    if (!P->order.empty()) {
        BQ_CUDA(cudaMemcpyAsync(ws + P->o_order, P->order.data(), sizeof(int) * P->order.size(),
                                cudaMemcpyHostToDevice, stream));
        BQ_CUDA(cudaMemcpyAsync(ws + P->o_hot, P->hot.data(), sizeof(int) * P->hot.size(), cudaMemcpyHostToDevice,
                                stream));
    }
    P->uploaded_ws = ws;
    return 0;
}

// Profiler phase of each launch kind (phase 1 covers the whole of Alg. 2 here:
// LU, piv_transform, gather, Householder QR and tri_rank run in one kernel).
constexpr int kPhaseOf[8] = {7, 0, 1, 3, 4, 5, 6, 7};

static MegaArgs mega_args(const BatchPlan* P, char* ws) {
    MegaArgs q;
    q.slots = (unsigned long long*)(ws + P->o_slots);
    q.hslots = (unsigned long long*)(ws + P->o_hslots);
    q.ctl = (unsigned int*)(ws + P->o_qctl);
    q.pending = (int*)(ws + P->o_pend);
    q.finished = (int*)(ws + P->o_fin);
    q.order = (const int*)(ws + P->o_order);
    q.hot = (const int*)(ws + P->o_hot);
    q.cap = P->qcap;
    q.hcap = P->hcap;
    q.batch = (int)P->batch;
    q.nhot = P->nhot;
    q.kb = P->kb;
    return q;
}

// The dependency-driven form: reset the queue, one persistent kernel, then
// mark the matrices a worker gave up on.
static int batch_launch_mega(BatchPlan* P, BatArgs a, cudaStream_t st, char* ws) {
    const MegaArgs q = mega_args(P, ws);
    const unsigned rb = (unsigned)std::min<i64>(1024, std::max<i64>(1, cdiv((i64)std::max(P->qcap, P->hcap), 256)));
    mega_reset_kernel<<<rb, 256, 0, st>>>(q);
    BQ_LAUNCH_CHECK();
    const int grid = (P->grid_cap > 0) ? std::min(P->grid_cap, P->grid_mega) : P->grid_mega;
    bat_mega_kernel<<<grid, BT, P->dsm_mega, st>>>(a, q);
    BQ_LAUNCH_CHECK();
    mega_check_kernel<<<(unsigned)cdiv(P->batch, 256), 256, 0, st>>>(a, q);
    BQ_LAUNCH_CHECK();
    return 0;
}

static int batch_launch_all(BatchPlan* P, BatArgs a, cudaStream_t st, char* ws, std::vector<cudaEvent_t>* ev) {
    if (P->mega && !ev) return batch_launch_mega(P, a, st, ws);
    BQ_CUDA(cudaMemsetAsync(ws + P->o_ctr, 0, sizeof(unsigned int) * std::max<size_t>(P->launches.size(), 1), st));
    for (size_t q = 0; q < P->launches.size(); ++q) {
        const BatchPlan::Launch& L = P->launches[q];
        if (L.slot.total == 0) continue;
        if (ev) BQ_CUDA(cudaEventRecord((*ev)[2 * q], st));
        const int g = std::max(1, std::min(P->grid[L.kind], L.slot.total));
        const int sid = (int)q;
        switch (L.kind) {
            case BatchPlan::K_INIT: bat_init_kernel<<<g, BT, 0, st>>>(a, L.slot, sid); break;
            case BatchPlan::K_SKETCH: bat_sketch_kernel<<<g, BT, 0, st>>>(a, L.slot, sid); break;
            case BatchPlan::K_QRCP: bat_qrcp_kernel<<<g, BT, P->dsm_qrcp, st>>>(a, L.slot, sid, L.iter); break;
            case BatchPlan::K_PERM: bat_perm_kernel<<<g, BT, P->dsm_perm, st>>>(a, L.slot, sid, L.iter); break;
            case BatchPlan::K_PANEL:
                bat_panel_kernel<<<g, BT, P->dsm_panel, st>>>(a, L.slot, sid, L.iter, P->kb);
                break;
            case BatchPlan::K_TRAIL:
                bat_trailing_kernel<<<g, BT, P->dsm_trail, st>>>(a, L.slot, sid, L.iter, P->kb);
                break;
            case BatchPlan::K_SKUPD: bat_skupdate_kernel<<<g, BT, 0, st>>>(a, L.slot, sid, L.iter); break;
            case BatchPlan::K_FINISH: bat_finish_kernel<<<g, BT, 0, st>>>(a, L.slot, sid); break;
        }
        BQ_LAUNCH_CHECK();
        if (ev) BQ_CUDA(cudaEventRecord((*ev)[2 * q + 1], st));
    }
    return 0;
}

// Eager launch with one event pair per launch; waits for the stream and adds
// the per-phase times and FLOPs to the profiler.
static int batch_launch_profiled(BatchPlan* P, BatArgs a, cudaStream_t st, char* ws) {
    std::vector<cudaEvent_t> ev(2 * P->launches.size(), nullptr);
    for (auto& e : ev) cudaEventCreate(&e);
    int rc = batch_launch_all(P, a, st, ws, &ev);
    if (rc == 0 && cudaStreamSynchronize(st) != cudaSuccess) {
        set_error("batched factorization failed: %s", cudaGetErrorString(cudaGetLastError()));
        rc = BQRRP_ECUDA;
    }
    if (rc == 0) {
        double ms[BQRRP_NPHASES] = {0}, fl[BQRRP_NPHASES] = {0};
        for (size_t q = 0; q < P->launches.size(); ++q) {
            const BatchPlan::Launch& L = P->launches[q];
            if (L.slot.total == 0) continue;
            float t = 0.f;
            if (cudaEventElapsedTime(&t, ev[2 * q], ev[2 * q + 1]) == cudaSuccess) ms[kPhaseOf[L.kind]] += t;
            fl[kPhaseOf[L.kind]] += L.flops;
        }
        profile_add(ms, fl);
    }
    for (auto& e : ev) cudaEventDestroy(e);
    return rc;
}

int batch_factor(BatchPlan* P, double* A, int64_t* jpvt, double* tau, int64_t* rank, int64_t* trunc,
                 int32_t* info, void* ws, size_t ws_bytes, cudaStream_t stream, int use_graph) {
    if (!P) { set_error("plan is null"); return -1; }
    if (P->batch == 0) return 0;
    if (!A || !jpvt || !tau || !rank) { set_error("null output pointer"); return -2; }
    if (!ws || ws_bytes < P->total) { set_error("workspace smaller than bqrrp_batch_workspace_bytes()"); return BQRRP_ENOMEM; }
    if (((uintptr_t)ws & 255) != 0) { set_error("workspace must be 256-byte aligned"); return -9; }
    Device dev;
    BQ_TRY(current_device(&dev));
    if (dev.id != P->device) { set_error("plan was made for device %d", P->device); return -1; }
    char* w = (char*)ws;
    if (P->uploaded_ws != ws) {
        if (P->gexec) {
            cudaGraphExecDestroy(P->gexec);
            P->gexec = nullptr;
        }
        BQ_TRY(batch_upload(P, w, stream));
    }
    BatArgs a;
    a.mats = (const BatMat*)(w + P->o_mats);
    a.st = (BatState*)(w + P->o_state);
    a.smat = (const int*)(w + P->o_smat);
    a.spre = (const int*)(w + P->o_spre);
    a.ctr = (unsigned int*)(w + P->o_ctr);
    a.A = A;
    a.jpvt = jpvt;
    a.tau = tau;
    a.wsd = (double*)(w + P->o_wsd);
    a.wsi = (int*)(w + P->o_wsi);
    a.rank_out = rank;
    a.trunc_out = trunc;
    a.info_out = info;
    a.tol = P->tol;
    if (!use_graph) return profile_on() ? batch_launch_profiled(P, a, stream, w) : batch_launch_all(P, a, stream, w, nullptr);

    // The graph is captured on a private stream (the legacy default stream
    // cannot be captured) and launched on the caller's stream; it depends on
    // the buffer addresses only.
    const void* key[7] = {A, jpvt, tau, rank, trunc, info, ws};
    if (P->gexec && std::memcmp(key, P->gkey, sizeof(key)) == 0) {
        BQ_CUDA(cudaGraphLaunch(P->gexec, stream));
        return 0;
    }
    if (P->gexec) {
        cudaGraphExecDestroy(P->gexec);
        P->gexec = nullptr;
    }
    if (!P->cap) BQ_CUDA(cudaStreamCreateWithFlags(&P->cap, cudaStreamNonBlocking));
    BQ_CUDA(cudaStreamBeginCapture(P->cap, cudaStreamCaptureModeThreadLocal));
    int rc = batch_launch_all(P, a, P->cap, w, nullptr);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(P->cap, &g);
    if (rc != 0) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) { set_error("stream capture: %s", cudaGetErrorString(e)); return BQRRP_ECUDA; }
    e = cudaGraphInstantiate(&P->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        P->gexec = nullptr;
        set_error("graph instantiate: %s", cudaGetErrorString(e));
        return BQRRP_ECUDA;
    }
    std::memcpy(P->gkey, key, sizeof(key));
    BQ_CUDA(cudaGraphLaunch(P->gexec, stream));
    return 0;
}

void batch_plan_destroy(BatchPlan* P) { delete P; }

void batch_plan_set_grid_cap(BatchPlan* P, int ctas) {
    if (P) P->grid_cap = ctas;
}

void batch_plan_set_lockstep(BatchPlan* P, bool on) {
    if (!P || P->mega == !on) return;
    P->mega = !on;
    if (P->gexec) {   // a captured graph holds the other form's launches
        cudaGraphExecDestroy(P->gexec);
        P->gexec = nullptr;
    }
}

double batch_plan_flops(const BatchPlan* P, int phase) {
    double f = 0.0;
    if (P)
        for (auto& L : P->launches)
            if (phase < 0 || kPhaseOf[L.kind] == phase) f += L.flops;
    return f;
}

int batch_plan_launches(const BatchPlan* P) {
    if (!P) return 0;
    if (P->mega) return 3;
    int c = 0;
    for (auto& L : P->launches) c += L.slot.total > 0;
    return c;
}

}  // namespace bq

// ================================================================== autotuner
// Picks b per size class (by n: [0,64), [64,128), [128,256), [256,512),
// [512,1024), [1024, ...)) from {16, 32, 64, 128} (capped at n: a block wider
// than the matrix only makes the sketch larger) by timing each class alone,
// refines each class's pick by one step on the whole batch, then picks the
// sketch ratio d/b from {1.25, 1.5} on the whole batch.  Every trial
// factors a fresh copy of the caller's matrices; the caller's A is not
// modified.
namespace bq {
namespace {

int size_class(i64 n) {
    int c = 0;
    while (c < 5 && n >= ((i64)64 << c)) ++c;
    return c;
}

i64 sketch_rows(i64 b, double gamma) {
    i64 d = (i64)std::ceil(gamma * (double)b - 1e-9);
    return std::min<i64>(std::max<i64>(d, b), kMaxD);
}

struct TuneBuffers {
    double* A;
    int64_t* jpvt;
    double* tau;
    int64_t* rank;
    char* ws;
    size_t ws_bytes;
};

// Time one batched factorization of the matrices `idx` (copied from the
// packed source) with block sizes bsel/dsel and trailing tile widths csel;
// returns milliseconds or < 0.
double time_subbatch(const std::vector<int>& idx, const i64* m, const i64* n, const uint64_t* seed,
                     const double* Asrc, const std::vector<i64>& offsrc, const std::vector<i64>& bsel,
                     const std::vector<i64>& dsel, const std::vector<i64>& csel, double tol, const TuneBuffers& tb,
                     cudaStream_t st) {
    const i64 cnt = (i64)idx.size();
    std::vector<i64> mm(cnt), nn(cnt), bb(cnt), dd(cnt), cc(cnt);
    std::vector<uint64_t> ss(cnt);
    for (i64 q = 0; q < cnt; ++q) {
        const int i = idx[q];
        mm[q] = m[i];
        nn[q] = n[i];
        bb[q] = bsel[i];
        dd[q] = dsel[i];
        cc[q] = csel[i];
        ss[q] = seed[i];
    }
    BatchPlan* P = nullptr;
    if (batch_plan_create_ex(&P, cnt, mm.data(), nn.data(), bb.data(), dd.data(), ss.data(), tol, nullptr, nullptr,
                             nullptr, cc.data()) != 0)
        return -1.0;
    double best = -1.0;
    if (P->total <= tb.ws_bytes) {
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        for (int rep = 0; rep < 3; ++rep) {
            i64 off = 0;
            for (i64 q = 0; q < cnt; ++q) {
                const int i = idx[q];
                cudaMemcpyAsync(tb.A + off, Asrc + offsrc[i], sizeof(double) * (size_t)(m[i] * n[i]),
                                cudaMemcpyDeviceToDevice, st);
                off += m[i] * n[i];
            }
            cudaEventRecord(e0, st);
            const int rc = batch_factor(P, tb.A, tb.jpvt, tb.tau, tb.rank, nullptr, nullptr, tb.ws, tb.ws_bytes, st, 1);
            cudaEventRecord(e1, st);
            if (rc != 0 || cudaEventSynchronize(e1) != cudaSuccess) {
                best = -1.0;
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && (best < 0.0 || ms < best)) best = ms;   // the first run captures the graph
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    batch_plan_destroy(P);
    return best;
}

}  // namespace

size_t batch_autotune_bytes(i64 batch, const i64* m, const i64* n) {
    i64 totA = 0, totJ = 0;
    size_t wd = 0, wi = 0;
    for (i64 i = 0; i < batch; ++i) {
        totA += m[i] * n[i];
        totJ += n[i];
        const i64 nn = std::max<i64>(n[i], 1);
        const i64 d = sketch_rows(kMaxB, 1.5);
        auto rnd = [](i64 x) { return (size_t)(x + 31) / 32 * 32; };
        wd += 2 * rnd(d * nn) + 2 * rnd(std::max<i64>(m[i], 1) * kMaxB) + rnd(3 * (i64)kMaxB * kMaxB);
        wi += rnd(2 * nn);
    }
    // plan image: records, queues and counters (generous bound), then the workspaces
    const size_t img = (size_t)batch * (sizeof(BatMat) + sizeof(BatState)) +
                       sizeof(int) * (size_t)(batch + 1) * (size_t)(3 + 5 * (kMaxN / 16 + 1)) * 2 + (1 << 20);
    size_t tot = align256(sizeof(double) * (size_t)std::max<i64>(totA, 1)) +
                 align256(sizeof(int64_t) * (size_t)std::max<i64>(totJ, 1)) +
                 align256(sizeof(double) * (size_t)std::max<i64>(totJ, 1)) +
                 align256(sizeof(int64_t) * (size_t)std::max<i64>(batch, 1));
    tot += align256(img) + align256(sizeof(double) * wd) + align256(sizeof(int) * wi) + 4096;
    return tot;
}

// Per size class of n: the block size b (timing the class alone), then, when
// ct_out is given, the trailing tile width (32 or 64 columns, timing the class
// alone with its b); then one step of b per class (half or double) on the
// whole batch; then the sketch ratio gamma over the whole batch.
int batch_autotune(i64 batch, const i64* m, const i64* n, const uint64_t* seed, const double* A, double tol,
                   void* ws, size_t ws_bytes, cudaStream_t st, i64* b_out, i64* d_out, i64* ct_out,
                   double* best_ms) {
    if (batch < 0) { set_error("batch < 0"); return -1; }
    if (batch == 0) return 0;
    if (!m || !n || !seed || !A || !b_out || !d_out) { set_error("null argument"); return -2; }
    if (!ws || ws_bytes < batch_autotune_bytes(batch, m, n)) {
        set_error("workspace smaller than bqrrp_batch_autotune_workspace_bytes()");
        return BQRRP_ENOMEM;
    }
    if (((uintptr_t)ws & 255) != 0) { set_error("workspace must be 256-byte aligned"); return -7; }
    i64 totA = 0, totJ = 0;
    std::vector<i64> offsrc(batch);
    for (i64 i = 0; i < batch; ++i) {
        if (n[i] < 0 || m[i] < n[i] || n[i] > kMaxN) { set_error("matrix %lld: unsupported shape", (long long)i); return -3; }
        offsrc[i] = totA;
        totA += m[i] * n[i];
        totJ += n[i];
    }
    char* w = (char*)ws;
    TuneBuffers tb;
    tb.A = (double*)w;                 w += align256(sizeof(double) * (size_t)std::max<i64>(totA, 1));
    tb.jpvt = (int64_t*)w;             w += align256(sizeof(int64_t) * (size_t)std::max<i64>(totJ, 1));
    tb.tau = (double*)w;               w += align256(sizeof(double) * (size_t)std::max<i64>(totJ, 1));
    tb.rank = (int64_t*)w;             w += align256(sizeof(int64_t) * (size_t)std::max<i64>(batch, 1));
    tb.ws = w;
    tb.ws_bytes = ws_bytes - (size_t)(w - (char*)ws);

    const i64 cands[4] = {16, 32, 64, 128};
    std::vector<i64> bsel(batch, 32), dsel(batch, sketch_rows(32, 1.25)), csel(batch, CT);
    std::vector<std::vector<int>> cls(6);
    std::vector<i64> cls_b(6, 32);
    for (i64 i = 0; i < batch; ++i) cls[size_class(n[i])].push_back((int)i);
    for (int c = 0; c < 6; ++c) {
        if (cls[c].empty()) continue;
        double bt = -1.0;
        i64 bb = 32;
        for (i64 cb : cands) {
            for (int i : cls[c]) {
                bsel[i] = std::min<i64>(cb, std::max<i64>(n[i], 1));    // a block never exceeds the matrix
                dsel[i] = sketch_rows(bsel[i], 1.25);
            }
            const double t = time_subbatch(cls[c], m, n, seed, A, offsrc, bsel, dsel, csel, tol, tb, st);
            if (t >= 0.0 && (bt < 0.0 || t < bt)) {
                bt = t;
                bb = cb;
            }
        }
        cls_b[c] = bb;
        for (int i : cls[c]) {
            bsel[i] = std::min<i64>(bb, std::max<i64>(n[i], 1));
            dsel[i] = sketch_rows(bsel[i], 1.25);
        }
        if (ct_out && bt >= 0.0) {
            for (int i : cls[c]) csel[i] = CT_MIN;
            const double t = time_subbatch(cls[c], m, n, seed, A, offsrc, bsel, dsel, csel, tol, tb, st);
            const bool narrow = t >= 0.0 && t < bt;
            for (int i : cls[c]) csel[i] = narrow ? CT_MIN : CT;
        }
    }
    std::vector<int> all(batch);
    for (i64 i = 0; i < batch; ++i) all[i] = (int)i;
    // A class timed alone may not fill the GPU, so its pick favours the
    // shorter critical path of a wider block; in the whole batch the classes
    // share the SMs and total work decides.  So each class's neighbouring
    // block sizes (half and double its pick) are retried on the whole batch,
    // widest class first, keeping a change only when the batch gets faster.
    double t_best = time_subbatch(all, m, n, seed, A, offsrc, bsel, dsel, csel, tol, tb, st);
    for (int c = 5; c >= 0 && t_best >= 0.0; --c) {
        if (cls[c].empty()) continue;
        int pick = 0;
        for (int ci = 0; ci < 4; ++ci) {
            if (cands[ci] == cls_b[c]) pick = ci;
        }
        std::vector<i64> bkeep(batch), dkeep(batch);
        for (int i : cls[c]) { bkeep[i] = bsel[i]; dkeep[i] = dsel[i]; }
        for (int ci : {pick - 1, pick + 1}) {
            if (ci < 0 || ci > 3) continue;
            bool changed = false;
            for (int i : cls[c]) {
                bsel[i] = std::min<i64>(cands[ci], std::max<i64>(n[i], 1));
                dsel[i] = sketch_rows(bsel[i], 1.25);
                changed |= bsel[i] != bkeep[i];
            }
            if (!changed) continue;   // every matrix of the class is narrower than both blocks
            const double t = time_subbatch(all, m, n, seed, A, offsrc, bsel, dsel, csel, tol, tb, st);
            if (t >= 0.0 && t < t_best) {
                t_best = t;
                for (int i : cls[c]) { bkeep[i] = bsel[i]; dkeep[i] = dsel[i]; }
            }
        }
        for (int i : cls[c]) { bsel[i] = bkeep[i]; dsel[i] = dkeep[i]; }
    }
    double g_best = 1.25;
    {
        std::vector<i64> dg(batch);
        for (i64 i = 0; i < batch; ++i) dg[i] = sketch_rows(bsel[i], 1.5);
        const double t = time_subbatch(all, m, n, seed, A, offsrc, bsel, dg, csel, tol, tb, st);
        if (t >= 0.0 && (t_best < 0.0 || t < t_best)) {
            t_best = t;
            g_best = 1.5;
        }
    }
    if (t_best < 0.0) {
        set_error("autotune: no candidate ran (%s)", get_error());
        return BQRRP_ECUDA;
    }
    for (i64 i = 0; i < batch; ++i) {
        b_out[i] = bsel[i];
        d_out[i] = sketch_rows(bsel[i], g_best);
        if (ct_out) ct_out[i] = csel[i];
    }
    if (best_ms) *best_ms = t_best;
    return 0;
}

}  // namespace bq

// ================================================================== C ABI
extern "C" {

int bqrrp_batch_plan_create(bqrrp_batch_plan* plan, int64_t batch, const int64_t* m, const int64_t* n,
                            const int64_t* b, const int64_t* d, const uint64_t* seed, double trunc_tol) {
    bq::set_error("");
    bq::BatchPlan* P = nullptr;
    const int rc = bq::batch_plan_create(&P, batch, m, n, b, d, seed, trunc_tol);
    if (plan) *plan = reinterpret_cast<bqrrp_batch_plan>(P);
    return rc;
}

int bqrrp_batch_plan_create_tiles(bqrrp_batch_plan* plan, int64_t batch, const int64_t* m, const int64_t* n,
                                  const int64_t* b, const int64_t* d, const int64_t* tile_cols, const uint64_t* seed,
                                  double trunc_tol) {
    bq::set_error("");
    bq::BatchPlan* P = nullptr;
    const int rc = bq::batch_plan_create_ex(&P, batch, m, n, b, d, seed, trunc_tol, nullptr, nullptr, nullptr,
                                            tile_cols);
    if (plan) *plan = reinterpret_cast<bqrrp_batch_plan>(P);
    return rc;
}

size_t bqrrp_batch_workspace_bytes(bqrrp_batch_plan plan) {
    return bq::batch_plan_bytes(reinterpret_cast<const bq::BatchPlan*>(plan));
}

int bqrrp_batch_factor(bqrrp_batch_plan plan, double* A, int64_t* jpvt, double* tau, int64_t* rank,
                       int64_t* trunc_rank, int32_t* info, void* workspace, size_t workspace_bytes, void* stream,
                       int use_graph) {
    bq::set_error("");
    return bq::batch_factor(reinterpret_cast<bq::BatchPlan*>(plan), A, jpvt, tau, rank, trunc_rank, info,
                            workspace, workspace_bytes, (cudaStream_t)stream, use_graph);
}

void bqrrp_batch_plan_destroy(bqrrp_batch_plan plan) {
    bq::batch_plan_destroy(reinterpret_cast<bq::BatchPlan*>(plan));
}

int bqrrp_batch_plan_set_form(bqrrp_batch_plan plan, int form) {
    bq::set_error("");
    if (!plan) return -1;
    if (form != BQRRP_BATCH_PERSISTENT && form != BQRRP_BATCH_LOCKSTEP) return -2;
    bq::batch_plan_set_lockstep(reinterpret_cast<bq::BatchPlan*>(plan), form == BQRRP_BATCH_LOCKSTEP);
    return 0;
}

int bqrrp_batch_launches(bqrrp_batch_plan plan) {
    return bq::batch_plan_launches(reinterpret_cast<const bq::BatchPlan*>(plan));
}

double bqrrp_batch_flops(bqrrp_batch_plan plan, int phase) {
    return bq::batch_plan_flops(reinterpret_cast<const bq::BatchPlan*>(plan), phase);
}

size_t bqrrp_batch_autotune_workspace_bytes(int64_t batch, const int64_t* m, const int64_t* n) {
    if (batch <= 0 || !m || !n) return 0;
    return bq::batch_autotune_bytes(batch, m, n);
}

int bqrrp_batch_autotune(int64_t batch, const int64_t* m, const int64_t* n, const uint64_t* seed, const double* A,
                         double trunc_tol, void* workspace, size_t workspace_bytes, void* stream, int64_t* b_out,
                         int64_t* d_out, double* best_ms) {
    bq::set_error("");
    return bq::batch_autotune(batch, m, n, seed, A, trunc_tol, workspace, workspace_bytes, (cudaStream_t)stream,
                              b_out, d_out, nullptr, best_ms);
}

int bqrrp_batch_autotune_tiles(int64_t batch, const int64_t* m, const int64_t* n, const uint64_t* seed,
                               const double* A, double trunc_tol, void* workspace, size_t workspace_bytes,
                               void* stream, int64_t* b_out, int64_t* d_out, int64_t* tile_out, double* best_ms) {
    bq::set_error("");
    if (batch > 0 && !tile_out) { bq::set_error("tile_out is null"); return -12; }
    return bq::batch_autotune(batch, m, n, seed, A, trunc_tol, workspace, workspace_bytes, (cudaStream_t)stream,
                              b_out, d_out, tile_out, best_ms);
}

}  // extern "C"
