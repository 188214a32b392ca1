// panels.cu -- cooperative (grid-wide) panel kernels and the blocked LU / QR
// drivers built on them.
//
//  * lu_panel_kernel: one nb-wide panel of the row-pivoted LU that Alg. 2
//    runs on the transposed sketch.  X = Sk^T is never formed: a row of X is a
//    column of the sketch buffer Sk (d x N, column-major), so each CTA keeps a
//    contiguous slab of X rows (= sketch columns) of the panel in shared memory;
//    per pivot step the CTAs exchange their argmax candidates (first maximum,
//    as GETRF/IDAMAX) through published slots, without a grid barrier.
//  * hh_panel_kernel: Householder QR (dlarfg convention) of a tall panel,
//    rows split across CTAs, two grid barriers per column (norm, then the
//    reflector's dot products), then the compact-WY factor T of the panel
//    (LAPACK larft recurrence from V^T V).
//  * small_qr_cluster_kernel: the R factor of the d x d factor of the sketch's
//    LU on one thread-block cluster (distributed shared memory).
//
// The grid-wide kernels are launched cooperatively so that all CTAs are
// co-resident; every cross-CTA wait is bounded (grid_barrier, the LU's slot
// polls).
#include <cooperative_groups.h>

#include <climits>
#include <cstdio>
#include <cstdlib>

#include <atomic>
#include <mutex>

#include "common.cuh"

namespace bq {

namespace {

constexpr int NT = 256;
constexpr int kMaxSmemLu = 210 * 1024;   // dynamic part; static use is ~2 KB
constexpr int kMaxSmemHh = 185 * 1024;   // dynamic part; static use is ~35 KB


// ---------------------------------------------------------------------------
// LU panel.  X(t, c) = Sk[c + t*ldsk]; panel = X rows [jb, N), columns
// [jb, jb+pw); steps pivot steps.  CTA g owns rows [jb + g*R, jb + (g+1)*R).
//
// Pivot exchange without a grid barrier: for every step each CTA publishes
// one slot {candidate value bits, candidate row}, both words all-ones until
// published, and the candidate row itself; every CTA polls the G slots of the
// step, picks the winner (largest |value|, then smallest row) and fetches the
// winner's row.  Slots and rows are triple-buffered by step: once a CTA has
// seen every slot of step j, all CTAs have finished reading step j-1's
// buffer, so the CTA resets its own slot there for step j+2 (the reset is
// ordered before its next publication, which readers of step j+2 have seen).
//
// Lookahead: after the interchange of step j a CTA computes the multipliers,
// updates only column j+1 (the next pivot column), publishes its step-(j+1)
// candidate and the current row j+1 (their other columns updated on the fly),
// and only then runs the bulk update of columns j+2.. while the other CTAs'
// slots arrive.
//
// Cost model on B300: every FP64 instruction holds its SM sub-partition's
// FP64 unit for ~64 cycles whatever the number of active lanes, and a
// division ~640.  The search therefore compares |x| as integers (the bit
// patterns of non-negative doubles order like their values), and the
// multipliers use one reciprocal of the pivot, formed by a single warp while
// the pivot row is in flight, plus one FMA correction (the quotient x/piv).
struct LuArgs {
    i64 N, jb, ldsk;
    int pw, steps, R, Rp;
    double* Sk;
    i64* ipiv;
    DevStatus* st;
    unsigned long long* slot;   // [3][G][2], all-ones before the launch
    double* cand_row;           // [3][G][pw]
    double* cur_row;            // [3][pw]
    unsigned long long poll_limit;   // polls per slot wait before giving up
    int stall_cta;                   // diagnostics: this CTA never publishes step 0 (-1: none)
};

constexpr unsigned long long kSlotEmpty = ~0ull;
constexpr unsigned long long kAbsMask = 0x7fffffffffffffffull;
constexpr long long kNoRow = LLONG_MAX;
constexpr unsigned long long kPollLimit = 1ull << 22;   // slot polls of ~1 us: a few seconds

__device__ inline unsigned long long ld_relaxed_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ inline void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Release / acquire fence at GPU scope: with the relaxed slot stores and loads
// it forms the PTX release and acquire patterns (a sequentially consistent
// fence is not needed for a publish/observe exchange).
__device__ inline void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// A pivot candidate: key = bits of |x|, row t.  "No candidate" is {0, kNoRow},
// which loses to every row.  (A NaN's key exceeds every finite one; the
// sketch's non-finite check reports such input.)
struct Cand {
    unsigned long long key;
    long long t;
};

__device__ inline unsigned long long abs_key(double x) {
    return (unsigned long long)__double_as_longlong(x) & kAbsMask;
}
// The panel's arithmetic type T (double; float for the reduced-precision
// pivot choice): a value's bits as published in a slot, |value| as a key from
// those bits, and the value back.
__device__ inline unsigned long long abs_key(float x) { return (unsigned long long)(__float_as_uint(x) & 0x7fffffffu); }
__device__ inline unsigned long long val_bits(double x) { return (unsigned long long)__double_as_longlong(x); }
__device__ inline unsigned long long val_bits(float x) { return (unsigned long long)__float_as_uint(x); }
template <typename T> __device__ inline unsigned long long abs_of_bits(unsigned long long vb);
template <> __device__ inline unsigned long long abs_of_bits<double>(unsigned long long vb) { return vb & kAbsMask; }
template <> __device__ inline unsigned long long abs_of_bits<float>(unsigned long long vb) { return vb & 0x7fffffffull; }
template <typename T> __device__ inline T from_bits(unsigned long long vb);
template <> __device__ inline double from_bits<double>(unsigned long long vb) { return __longlong_as_double((long long)vb); }
template <> __device__ inline float from_bits<float>(unsigned long long vb) { return __uint_as_float((unsigned)vb); }

// First-maximum rule: the larger |x| wins, equal values go to the smaller row.
__device__ inline Cand better(Cand a, Cand b) { return (b.key > a.key || (b.key == a.key && b.t < a.t)) ? b : a; }

__device__ inline Cand shfl_down_cand(Cand x, int o) {
    return Cand{__shfl_down_sync(0xffffffffu, x.key, o), __shfl_down_sync(0xffffffffu, x.t, o)};
}

// Block-wide first maximum; every thread returns the same result.  wk/wt hold
// one entry per warp and are rewritten only after a later __syncthreads.
template <int NTB>
__device__ inline Cand block_best_all_n(Cand x, unsigned long long* wk, long long* wt) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = better(x, shfl_down_cand(x, o));
    if (lane == 0) { wk[w] = x.key; wt[w] = x.t; }
    __syncthreads();
    Cand r{wk[0], wt[0]};
#pragma unroll
    for (int q = 1; q < NTB / 32; ++q) r = better(r, Cand{wk[q], wt[q]});
    return r;
}
__device__ inline Cand block_best_all(Cand x, unsigned long long* wk, long long* wt) {
    return block_best_all_n<NT>(x, wk, wt);
}

// T: the panel's arithmetic.  The sketch Sk stays FP64 in memory; with float
// the slab holds the rows rounded to FP32, the pivot search, multipliers and
// eliminations run in FP32, and the factors are written back widened.
template <typename T>
__global__ void __launch_bounds__(NT) lu_panel_kernel(LuArgs a) {
    extern __shared__ __align__(16) unsigned char slab_raw[];
    T* slab = (T*)slab_raw;                   // [pw][Rp]
    T* cand_row = (T*)a.cand_row;             // [3][G][pw]
    T* cur_row = (T*)a.cur_row;               // [3][pw]
    __shared__ T prow[64];
    __shared__ unsigned long long wk[NT / 32];
    __shared__ long long wt[NT / 32];
    __shared__ long long s_p;
    __shared__ unsigned long long s_pivbits;
    __shared__ T s_rpiv;
    __shared__ int s_gw, s_ok;
    const int G = gridDim.x, g = blockIdx.x, tid = threadIdx.x;
    const i64 t0 = a.jb + (i64)g * a.R;
    const i64 t1 = (t0 + a.R < a.N) ? t0 + a.R : a.N;
    const int nloc = t1 > t0 ? (int)(t1 - t0) : 0;
    const int pw = a.pw, Rp = a.Rp;

    for (int e = tid; e < nloc * pw; e += NT) {
        const int c = e % pw, rl = e / pw;
        slab[c * Rp + rl] = (T)a.Sk[(a.jb + c) + (t0 + rl) * a.ldsk];
    }
    // identity pivots first: a panel that gives up on the exchange (timeout)
    // leaves in-range, no-op interchanges for the kernels that follow it
    if (g == 0)
        for (int t = tid; t < a.steps; t += NT) a.ipiv[a.jb + t] = a.jb + t;
    __syncthreads();

    // Publish the candidate for pivot step k = j + 1 (j = -1: the first step).
    // Row r's entry in column c: columns <= j+1 are current in the slab; the
    // later ones still lack step j's update, applied here when elim is set.
    auto publish = [&](int j, bool elim, Cand b) {
        const int k = j + 1, buf = k % 3;
        const i64 cur = a.jb + k;
        if (b.t != kNoRow && tid < pw) {
            const int r = (int)(b.t - t0), c = tid;
            const T x = slab[c * Rp + r];
            cand_row[((size_t)buf * G + g) * pw + c] = (elim && c > j + 1) ? fma(-slab[j * Rp + r], prow[c], x) : x;
        }
        if (cur >= t0 && cur < t1 && tid >= 64 && tid < 64 + pw) {
            const int r = (int)(cur - t0), c = tid - 64;
            const T x = slab[c * Rp + r];
            cur_row[(size_t)buf * pw + c] = (elim && c > j + 1) ? fma(-slab[j * Rp + r], prow[c], x) : x;
        }
        __syncthreads();
        if (tid == 0) {
            if (j >= 0) {
                unsigned long long* old = a.slot + ((size_t)((j + 2) % 3) * G + g) * 2;
                st_relaxed_u64(old, kSlotEmpty);
                st_relaxed_u64(old + 1, kSlotEmpty);
            }
            unsigned long long vb = 0;   // signed candidate value (+0 for "no candidate")
            if (b.t != kNoRow) vb = val_bits(slab[k * Rp + (int)(b.t - t0)]);
            if (vb == kSlotEmpty) vb = 0xfff8000000000000ull;   // that NaN pattern marks an empty slot
            fence_acq_rel_gpu();
            unsigned long long* s = a.slot + ((size_t)buf * G + g) * 2;
            st_relaxed_u64(s, vb);
            st_relaxed_u64(s + 1, (unsigned long long)b.t);
        }
    };

    {   // step 0 candidate: first maximum of |X(t, jb)| over the owned rows
        Cand b{0, kNoRow};
        for (int rl = tid; rl < nloc; rl += NT) b = better(b, Cand{abs_key(slab[rl]), t0 + rl});
        b = block_best_all(b, wk, wt);
        if (g != a.stall_cta) publish(-1, false, b);   // a stalled CTA leaves its slot empty
    }

    for (int j = 0; j < a.steps; ++j) {
        const i64 jg = a.jb + j;
        const bool has_next = j + 1 < a.steps;
        // (1) wait for the G slots of step j; winner = largest |value|, then smallest row
        if (tid < 32) {
            const unsigned long long* sl = a.slot + (size_t)(j % 3) * G * 2;
            Cand w{0, kNoRow};
            unsigned long long wvb = 0;
            int wq = -1, ok = 1;
            unsigned long long polls = 0;
            for (;;) {
                bool all = true;
                w = Cand{0, kNoRow};
                wq = -1;
                for (int q = tid; q < G; q += 32) {
                    const unsigned long long vb = ld_relaxed_u64(sl + 2 * q), tb = ld_relaxed_u64(sl + 2 * q + 1);
                    if (vb == kSlotEmpty || tb == kSlotEmpty) { all = false; continue; }
                    const Cand z = better(w, Cand{abs_of_bits<T>(vb), (long long)tb});
                    if (z.t != w.t) { w = z; wq = q; wvb = vb; }
                }
                if (__all_sync(0xffffffffu, all)) break;
                // warp-uniform exit: the poll count is the same in every lane and the
                // error flag is voted on
                ++polls;
                if (polls > a.poll_limit ||
                    ((polls & 1023) == 0 &&
                     __any_sync(0xffffffffu, *((volatile int*)&a.st->err_timeout) != 0))) {
                    ok = 0;
                    break;
                }
            }
            // acquire side of the slots' publication: each lane fences after its own polls
            fence_acq_rel_gpu();
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const Cand y = shfl_down_cand(w, o);
                const int yq = __shfl_down_sync(0xffffffffu, wq, o);
                const unsigned long long yvb = __shfl_down_sync(0xffffffffu, wvb, o);
                const Cand z = better(w, y);
                if (z.t != w.t) { w = z; wq = yq; wvb = yvb; }
            }
            if (tid == 0) {
                if (!ok || wq < 0) atomicExch(&a.st->err_timeout, 1);
                s_ok = ok && wq >= 0;
                s_p = w.t;
                s_gw = wq;
                s_pivbits = wvb;
                if (g == 0 && s_ok) a.ipiv[jg] = w.t;
            }
        }
        __syncthreads();
        if (!s_ok) return;
        const i64 p = s_p;
        const int gw = s_gw, buf = j % 3;
        const bool elim = abs_of_bits<T>(s_pivbits) != 0;   // exact zero pivot: no elimination, as GETRF
        // (2) pivot row into prow and the slab; current row jg to the winner's
        // place; one warp forms 1/piv meanwhile
        if (tid < pw) {
            const T pr = __ldcg(&cand_row[((size_t)buf * G + gw) * pw + tid]);
            prow[tid] = pr;
            if (jg >= t0 && jg < t1) slab[tid * Rp + (jg - t0)] = pr;
            if (p != jg && p >= t0 && p < t1) slab[tid * Rp + (p - t0)] = __ldcg(&cur_row[(size_t)buf * pw + tid]);
        }
        if (tid == 64 && elim) s_rpiv = T(1) / from_bits<T>(s_pivbits);
        __syncthreads();
        // (3) multipliers and column j+1 of the owned rows below jg; next candidate.
        // l = x / piv from the reciprocal with one FMA correction (Markstein's
        // quotient refinement: r = x - piv*l is exact, l + r/piv rounds to x/piv),
        // so equal rows still cancel exactly as in GETRF.
        const T rpiv = s_rpiv, pivv = from_bits<T>(s_pivbits);
        const int r0 = (jg + 1 > t0) ? (int)(jg + 1 - t0) : 0;
        Cand b{0, kNoRow};
        for (int rl = r0 + tid; rl < nloc; rl += NT) {
            T l = T(0);
            if (elim) {
                const T x = slab[j * Rp + rl];
                l = x * rpiv;
                l = fma(fma(-pivv, l, x), rpiv, l);
                slab[j * Rp + rl] = l;
            }
            if (has_next) {
                T x = slab[(j + 1) * Rp + rl];
                if (elim) {
                    x = fma(-l, prow[j + 1], x);
                    slab[(j + 1) * Rp + rl] = x;
                }
                b = better(b, Cand{abs_key(x), t0 + rl});
            }
        }
        if (has_next) {
            b = block_best_all(b, wk, wt);
            publish(j, elim, b);
        } else {
            __syncthreads();
        }
        // (4) bulk update of columns cs.. of the owned rows below jg
        const int nr = nloc - r0, cs = has_next ? j + 2 : j + 1;
        if (elim && nr > 0 && cs < pw) {
            if (nr >= NT) {
                for (int rl = r0 + tid; rl < nloc; rl += NT) {
                    const T l = slab[j * Rp + rl];
                    for (int c = cs; c < pw; ++c) slab[c * Rp + rl] = fma(-l, prow[c], slab[c * Rp + rl]);
                }
            } else {
                const int ng = NT / nr, grp = tid / nr;
                if (grp < ng) {
                    const int rl = r0 + tid - grp * nr;
                    const T l = slab[j * Rp + rl];
                    for (int c = cs + grp; c < pw; c += ng) slab[c * Rp + rl] = fma(-l, prow[c], slab[c * Rp + rl]);
                }
            }
        }
        __syncthreads();
    }
    for (int e = tid; e < nloc * pw; e += NT) {
        const int c = e % pw, rl = e / pw;
        a.Sk[(a.jb + c) + (t0 + rl) * a.ldsk] = (double)slab[c * Rp + rl];
    }
}

// Apply the panel's interchanges to every sketch row outside the panel rows
// [jb, jb+pw): swap columns jb+j and ipiv[jb+j] in order (LAPACK applies them to
// the L part on the left and the trailing part on the right alike).  The
// swaps name at most 2*steps positions; each CTA tracks every named position y
// forward through the sequence to its final place f(y), then gathers its rows
// in one pass (all loads, a barrier, all stores), so a row costs one memory
// round trip instead of a chain of dependent swaps.  Duplicate names carry the
// same (y, f(y)) pair and store the same value.
constexpr int kSwapRows = 32;
__global__ void __launch_bounds__(256) lu_swap_rows_kernel(i64 pw, i64 d, i64 jb, int steps,
                                                           const i64* __restrict__ ipiv, double* Sk, i64 ldsk) {
    __shared__ i64 ip[64];
    __shared__ i64 ys[128], fs[128];
    const int tid = threadIdx.x, ne = 2 * steps;
    if (tid < steps) ip[tid] = ipiv[jb + tid];
    __syncthreads();
    if (tid < ne) {
        const i64 y = tid < steps ? jb + tid : ip[tid - steps];
        i64 cur = y;
        for (int j = 0; j < steps; ++j) {
            const i64 a = jb + j, p = ip[j];
            if (cur == a) cur = p;
            else if (cur == p) cur = a;
        }
        ys[tid] = y;
        fs[tid] = cur;
    }
    __syncthreads();
    const i64 q = (i64)blockIdx.x * kSwapRows + (tid & 31);
    const bool valid = q < d - pw;
    const i64 r = (q < jb) ? q : q + pw;
    double v[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const int i = (tid >> 5) + 8 * k;
        if (valid && i < ne) v[k] = Sk[r + ys[i] * ldsk];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const int i = (tid >> 5) + 8 * k;
        if (valid && i < ne) Sk[r + fs[i] * ldsk] = v[k];
    }
}

// ---------------------------------------------------------------------------
// Householder panel: rows x pw panel A (ld lda).
struct HhArgs {
    i64 rows, lda, ldv, ldt;
    int pw, R, Rp;
    double* A;
    double* tau;
    double* V;
    double* T;
    DevStatus* st;
    double* part1;   // [G]
    double* alpha;   // [1]
    double* part2;   // [G][pw]
    double* gpart;   // [G][pw*pw]
    double* gsum;    // [pw*pw]
};

__global__ void __launch_bounds__(NT) hh_panel_kernel(HhArgs a) {
    extern __shared__ double slab[];   // [pw][Rp]
    __shared__ double red[NT / 32];
    __shared__ double red4[4][64];
    __shared__ double wv[64];
    __shared__ double s_tau, s_beta, s_scal;
    __shared__ double Ts[64][65];
    const int G = gridDim.x, g = blockIdx.x, tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const i64 r0 = (i64)g * a.R;
    const i64 r1 = (r0 + a.R < a.rows) ? r0 + a.R : a.rows;
    const int nloc = r1 > r0 ? (int)(r1 - r0) : 0;
    const int pw = a.pw;

    for (int e = tid; e < nloc * pw; e += NT) {
        const int rl = e % nloc, c = e / nloc;
        slab[c * a.Rp + rl] = a.A[(r0 + rl) + c * a.lda];
    }
    __syncthreads();

    const int jmax = (a.rows < pw) ? (int)a.rows : pw;
    for (int j = 0; j < jmax; ++j) {
        // (1) partial sum of squares below the diagonal; owner publishes alpha
        double s = 0.0;
        const int rb = (j + 1 > r0) ? (int)(j + 1 - r0) : 0;
        for (int rl = rb + tid; rl < nloc; rl += NT) {
            const double x = slab[j * a.Rp + rl];
            s = fma(x, x, s);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) red[warp] = s;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int q = 0; q < NT / 32; ++q) t += red[q];
            a.part1[g] = t;
            if (j >= r0 && j < r1) *a.alpha = slab[j * a.Rp + (j - r0)];
        }
        if (!grid_barrier(a.st, G)) return;
        // (3) reflector (every CTA computes the same numbers in the same order)
        if (warp == 0) {
            double xs = 0.0;
#pragma unroll 5
            for (int q = lane; q < G; q += 32) xs += __ldcg(&a.part1[q]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) xs += __shfl_down_sync(0xffffffffu, xs, o);
            if (lane == 0) red[0] = xs;
        }
        __syncthreads();
        if (tid == 0) {
            const double xn2 = red[0];
            const double al = __ldcg(a.alpha);
            if (xn2 == 0.0) {
                s_tau = 0.0; s_beta = al; s_scal = 1.0;
            } else {
                const double nrm = sqrt(fma(al, al, xn2));
                const double be = (al >= 0.0) ? -nrm : nrm;
                s_tau = (be - al) / be;
                s_beta = be;
                s_scal = 1.0 / (al - be);
            }
            if (g == 0) a.tau[j] = s_tau;
        }
        __syncthreads();
        const double tau = s_tau;
        if (tau != 0.0) {
            const double scal = s_scal;
            for (int rl = rb + tid; rl < nloc; rl += NT) slab[j * a.Rp + rl] *= scal;
            if (tid == 0 && j >= r0 && j < r1) slab[j * a.Rp + (j - r0)] = s_beta;
        }
        __syncthreads();
        if (tau == 0.0 || j + 1 >= pw) continue;   // uniform across CTAs: no barrier skipped unevenly
        // (5) partial dots w_c = v^T A(:, c), c > j, v_j = 1
        const int rv = (j > r0) ? (int)(j - r0) : 0;
        for (int c = j + 1 + warp; c < pw; c += NT / 32) {
            double acc = 0.0;
            for (int rl = rv + lane; rl < nloc; rl += 32) {
                const i64 r = r0 + rl;
                const double v = (r == j) ? 1.0 : slab[j * a.Rp + rl];
                acc = fma(v, slab[c * a.Rp + rl], acc);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
            if (lane == 0) a.part2[(size_t)g * pw + c] = acc;
        }
        if (!grid_barrier(a.st, G)) return;
        // (7) reduce partial dots in a fixed order: thread (group g4, column cl)
        // sums sources q = g4, g4 + 4, ... with many loads in flight, then the
        // four group sums are added in group order.
        {
            const int cl = tid & 63, g4 = tid >> 6;
            const int c = j + 1 + cl;
            double acc = 0.0;
            if (c < pw) {
#pragma unroll 8
                for (int q = g4; q < G; q += 4) acc += __ldcg(&a.part2[(size_t)q * pw + c]);
            }
            red4[g4][cl] = acc;
            __syncthreads();
            if (tid < pw - j - 1) wv[j + 1 + tid] = (((red4[0][tid] + red4[1][tid]) + red4[2][tid]) + red4[3][tid]) * tau;
        }
        __syncthreads();
        for (int e = tid; e < (pw - j - 1) * (nloc - rv > 0 ? nloc - rv : 0); e += NT) {
            const int span = nloc - rv;
            const int rl = rv + e % span, c = j + 1 + e / span;
            const i64 r = r0 + rl;
            const double v = (r == j) ? 1.0 : slab[j * a.Rp + rl];
            slab[c * a.Rp + rl] = fma(-wv[c], v, slab[c * a.Rp + rl]);
        }
        __syncthreads();
    }
    if (g == 0)
        for (int j = jmax + tid; j < pw; j += NT) a.tau[j] = 0.0;

    // write the panel back (R above, v below) and V explicitly
    for (int e = tid; e < nloc * pw; e += NT) {
        const int rl = e % nloc, c = e / nloc;
        const i64 r = r0 + rl;
        const double x = slab[c * a.Rp + rl];
        a.A[r + c * a.lda] = x;
        a.V[r + c * a.ldv] = (c >= jmax) ? 0.0 : (r > c ? x : (r == c ? 1.0 : 0.0));
    }
    // partial Gram V^T V (upper triangle) over owned rows
    for (int e = tid; e < pw * pw; e += NT) {
        const int i = e % pw, j = e / pw;
        double acc = 0.0;
        if (i <= j && j < jmax) {
            const int rs = (j > r0) ? (int)(j - r0) : 0;   // V(r, j) = 0 for r < j
            for (int rl = rs; rl < nloc; ++rl) {
                const i64 r = r0 + rl;
                const double vi = (r > i) ? slab[i * a.Rp + rl] : (r == i ? 1.0 : 0.0);
                const double vj = (r > j) ? slab[j * a.Rp + rl] : (r == j ? 1.0 : 0.0);
                acc = fma(vi, vj, acc);
            }
        }
        a.gpart[(size_t)g * pw * pw + e] = acc;
    }
    if (!grid_barrier(a.st, G)) return;
    // distributed fixed-order reduction of the Gram partials
    for (int e = g * NT + tid; e < pw * pw; e += G * NT) {
        double acc = 0.0;
#pragma unroll 8
        for (int q = 0; q < G; ++q) acc += __ldcg(&a.gpart[(size_t)q * pw * pw + e]);
        a.gsum[e] = acc;
    }
    if (!grid_barrier(a.st, G)) return;
    if (g != 0) return;
    // T by the larft recurrence: T(j,j) = tau_j, T(0:j,j) = -tau_j T(0:j,0:j) G(0:j,j)
    for (int e = tid; e < 64 * 65; e += NT) (&Ts[0][0])[e] = 0.0;
    // Gram into shared memory (the slab is free now when it is large enough)
    double* Gs = slab;
    const bool gsm = (size_t)pw * pw <= (size_t)pw * a.Rp;
    if (gsm)
        for (int e = tid; e < pw * pw; e += NT) Gs[e] = __ldcg(&a.gsum[e]);
    __shared__ double taus[64];
    for (int j = tid; j < pw; j += NT) taus[j] = (j < jmax) ? __ldcg(&a.tau[j]) : 0.0;
    __syncthreads();
    for (int j = 0; j < pw; ++j) {
        const double tj = taus[j];
        for (int i = tid; i < j; i += NT) {
            double z = 0.0;
            if (gsm)
                for (int l = i; l < j; ++l) z = fma(Ts[i][l], Gs[l + j * pw], z);
            else
                for (int l = i; l < j; ++l) z = fma(Ts[i][l], __ldcg(&a.gsum[l + j * pw]), z);
            Ts[i][j] = -tj * z;
        }
        if (tid == 0) Ts[j][j] = tj;
        __syncthreads();
    }
    for (int e = tid; e < pw * pw; e += NT) {
        const int i = e % pw, j = e / pw;
        a.T[i + j * a.ldt] = Ts[i][j];
    }
}

// ---------------------------------------------------------------------------
// Householder panel on one thread-block cluster (short panels, e.g. the d-row
// sketch): same arithmetic and reduction order as hh_panel_kernel, but the
// per-CTA partial sums are read through distributed shared memory and the two
// exchanges per column use the hardware cluster barrier.
namespace cg = cooperative_groups;

__global__ void __launch_bounds__(NT) hh_panel_cluster_kernel(HhArgs a) {
    extern __shared__ double slab[];   // [pw][Rp], then the Gram partial [pw*pw]
    __shared__ double red[NT / 32];
    __shared__ double wv[64];
    __shared__ double part2_s[64];
    __shared__ double part1_s, alpha_s;
    __shared__ double s_tau, s_beta, s_scal;
    __shared__ double Ts[64][65];
    cg::cluster_group cl = cg::this_cluster();
    const int G = (int)cl.num_blocks(), g = (int)cl.block_rank(), tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const i64 r0 = (i64)g * a.R;
    const i64 r1 = (r0 + a.R < a.rows) ? r0 + a.R : a.rows;
    const int nloc = r1 > r0 ? (int)(r1 - r0) : 0;
    const int pw = a.pw;
    double* gram = slab + (size_t)pw * a.Rp;

    for (int e = tid; e < nloc * pw; e += NT) {
        const int rl = e % nloc, c = e / nloc;
        slab[c * a.Rp + rl] = a.A[(r0 + rl) + c * a.lda];
    }
    __syncthreads();
    const int jmax = (a.rows < pw) ? (int)a.rows : pw;
    for (int j = 0; j < jmax; ++j) {
        double s = 0.0;
        const int rb = (j + 1 > r0) ? (int)(j + 1 - r0) : 0;
        for (int rl = rb + tid; rl < nloc; rl += NT) {
            const double x = slab[j * a.Rp + rl];
            s = fma(x, x, s);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) red[warp] = s;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int q = 0; q < NT / 32; ++q) t += red[q];
            part1_s = t;
            if (j >= r0 && j < r1) alpha_s = slab[j * a.Rp + (j - r0)];
        }
        cl.sync();
        if (warp == 0) {
            double xs = 0.0;
            for (int q = lane; q < G; q += 32) xs += *cl.map_shared_rank(&part1_s, q);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) xs += __shfl_down_sync(0xffffffffu, xs, o);
            if (lane == 0) {
                const double al = *cl.map_shared_rank(&alpha_s, (int)(j / a.R));
                if (xs == 0.0) {
                    s_tau = 0.0; s_beta = al; s_scal = 1.0;
                } else {
                    const double nrm = sqrt(fma(al, al, xs));
                    const double be = (al >= 0.0) ? -nrm : nrm;
                    s_tau = (be - al) / be;
                    s_beta = be;
                    s_scal = 1.0 / (al - be);
                }
                if (g == 0) a.tau[j] = s_tau;
            }
        }
        __syncthreads();
        const double tau = s_tau;
        if (tau != 0.0) {
            const double scal = s_scal;
            for (int rl = rb + tid; rl < nloc; rl += NT) slab[j * a.Rp + rl] *= scal;
            if (tid == 0 && j >= r0 && j < r1) slab[j * a.Rp + (j - r0)] = s_beta;
        }
        __syncthreads();
        if (tau == 0.0 || j + 1 >= pw) {
            cl.sync();   // keep the two-exchanges-per-column rhythm on every CTA
            continue;
        }
        const int rv = (j > r0) ? (int)(j - r0) : 0;
        for (int c = j + 1 + warp; c < pw; c += NT / 32) {
            double acc = 0.0;
            for (int rl = rv + lane; rl < nloc; rl += 32) {
                const i64 r = r0 + rl;
                const double v = (r == j) ? 1.0 : slab[j * a.Rp + rl];
                acc = fma(v, slab[c * a.Rp + rl], acc);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
            if (lane == 0) part2_s[c] = acc;
        }
        cl.sync();
        for (int c = j + 1 + warp; c < pw; c += NT / 32) {
            double acc = 0.0;
            for (int q = lane; q < G; q += 32) acc += *cl.map_shared_rank(&part2_s[c], q);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
            if (lane == 0) wv[c] = acc * tau;
        }
        __syncthreads();
        const int span = nloc - rv;
        for (int e = tid; span > 0 && e < (pw - j - 1) * span; e += NT) {
            const int rl = rv + e % span, c = j + 1 + e / span;
            const i64 r = r0 + rl;
            const double v = (r == j) ? 1.0 : slab[j * a.Rp + rl];
            slab[c * a.Rp + rl] = fma(-wv[c], v, slab[c * a.Rp + rl]);
        }
        __syncthreads();
    }
    if (g == 0)
        for (int j = jmax + tid; j < pw; j += NT) a.tau[j] = 0.0;
    for (int e = tid; e < nloc * pw; e += NT) {
        const int rl = e % nloc, c = e / nloc;
        const i64 r = r0 + rl;
        const double x = slab[c * a.Rp + rl];
        a.A[r + c * a.lda] = x;
        a.V[r + c * a.ldv] = (c >= jmax) ? 0.0 : (r > c ? x : (r == c ? 1.0 : 0.0));
    }
    for (int e = tid; e < pw * pw; e += NT) {
        const int i = e % pw, j = e / pw;
        double acc = 0.0;
        if (i <= j && j < jmax) {
            const int rs = (j > r0) ? (int)(j - r0) : 0;
            for (int rl = rs; rl < nloc; ++rl) {
                const i64 r = r0 + rl;
                const double vi = (r > i) ? slab[i * a.Rp + rl] : (r == i ? 1.0 : 0.0);
                const double vj = (r > j) ? slab[j * a.Rp + rl] : (r == j ? 1.0 : 0.0);
                acc = fma(vi, vj, acc);
            }
        }
        gram[e] = acc;
    }
    cl.sync();
    if (g == 0) {
        for (int e = tid; e < 64 * 65; e += NT) (&Ts[0][0])[e] = 0.0;
        // reduce the Gram partials in rank order into this CTA's slab
        for (int e = tid; e < pw * pw; e += NT) {
            double acc = gram[e];
            for (int q = 1; q < G; ++q) acc += *cl.map_shared_rank(&gram[e], q);
            gram[e] = acc;
        }
        __syncthreads();
        for (int j = 0; j < pw; ++j) {
            const double tj = (j < jmax) ? a.tau[j] : 0.0;
            for (int i = tid; i < j; i += NT) {
                double z = 0.0;
                for (int l = i; l < j; ++l) z = fma(Ts[i][l], gram[l + j * pw], z);
                Ts[i][j] = -tj * z;
            }
            if (tid == 0) Ts[j][j] = tj;
            __syncthreads();
        }
        for (int e = tid; e < pw * pw; e += NT) {
            const int i = e % pw, j = e / pw;
            a.T[i + j * a.ldt] = Ts[i][j];
        }
    }
    cl.sync();   // peers' shared memory stays alive until rank 0 has read it
}

// One panel of the row-pivoted LU on a single thread-block cluster, in FP32
// (the reduced-precision Alg. 2 of BQRRP_PRECISION_MIXED_SKETCH32, when the
// panel's rows fit the cluster's shared memory).  The arithmetic is that of
// lu_panel_kernel<float> step for step -- the same first-maximum rule, the
// same quotients and FMA updates of every row -- so the factors and pivots are
// the same bits; only the exchange differs.  Each CTA publishes its candidate
// (|value| key, row, signed value), the candidate's row and, if it owns it,
// the next current row in its own shared memory (double-buffered by step
// parity); one hardware cluster barrier per step (release / acquire) makes
// them visible, and every CTA reads the others' through distributed shared
// memory.  The barrier is split: a CTA arrives as soon as it has published
// (before its bulk elimination, which so overlaps the barrier) and waits at the
// top of the next step.  A buffer is rewritten two steps later, after a wait
// that completes only once every CTA has finished reading it.  No wait can
// hang: the barriers are the cluster's own, reached by every CTA on every step.
constexpr int kLuCluster = 16;
constexpr int NTC = 256;    // threads per CTA (1024 measured slower: the step is bound by its barriers)
__device__ __forceinline__ void cluster_arrive_release() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait_acquire() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }
constexpr int kMaxSmemLuCl = 200 * 1024;

struct LuClArgs {
    i64 N, jb, ldsk;
    int pw, steps, R, Rp;
    double* Sk;
    i64* ipiv;
};

__global__ void __launch_bounds__(NTC) lu_panel_cluster_kernel(LuClArgs a) {
    extern __shared__ __align__(16) unsigned char slab_raw[];
    float* slab = (float*)slab_raw;               // [pw][Rp]
    __shared__ float prow[64];
    __shared__ float cand_row[2][64];             // this CTA's candidate row for a step
    __shared__ float cur_row[2][64];              // the step's current row, if this CTA owns it
    __shared__ float cur_loc[64];                 // the step's current row, fetched from its owner
    __shared__ unsigned long long cand_key[2];    // |value| bits of the candidate (0 with no candidate)
    __shared__ long long cand_t[2];               // its row (kNoRow: none)
    __shared__ unsigned int cand_vb[2];           // its signed value bits
    __shared__ unsigned long long wk[NTC / 32];
    __shared__ long long wt[NTC / 32];
    __shared__ long long s_p;
    __shared__ unsigned int s_pivbits;
    __shared__ int s_gw;
    __shared__ float s_rpiv;
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks(), g = (int)cl.block_rank(), tid = threadIdx.x;
    const i64 t0 = a.jb + (i64)g * a.R;
    const i64 t1 = (t0 + a.R < a.N) ? t0 + a.R : a.N;
    const int nloc = t1 > t0 ? (int)(t1 - t0) : 0;
    const int pw = a.pw, Rp = a.Rp;

    for (int e = tid; e < nloc * pw; e += NTC) {
        const int c = e % pw, rl = e / pw;
        slab[c * Rp + rl] = (float)a.Sk[(a.jb + c) + (t0 + rl) * a.ldsk];
    }
    __syncthreads();

    // Publish the candidate for step k = j + 1 (j = -1: the first step) into
    // buffer k & 1; columns > j + 1 of the rows still lack step j's update,
    // applied here when elim is set (as lu_panel_kernel does).
    auto publish = [&](int j, bool elim, Cand b) {
        const int k = j + 1, buf = k & 1;
        const i64 cur = a.jb + k;
        if (b.t != kNoRow && tid < pw) {
            const int r = (int)(b.t - t0), c = tid;
            const float x = slab[c * Rp + r];
            cand_row[buf][c] = (elim && c > j + 1) ? fmaf(-slab[j * Rp + r], prow[c], x) : x;
        }
        if (cur >= t0 && cur < t1 && tid >= 64 && tid < 64 + pw) {
            const int r = (int)(cur - t0), c = tid - 64;
            const float x = slab[c * Rp + r];
            cur_row[buf][c] = (elim && c > j + 1) ? fmaf(-slab[j * Rp + r], prow[c], x) : x;
        }
        if (tid == 0) {
            cand_key[buf] = b.key;
            cand_t[buf] = b.t;
            cand_vb[buf] = (b.t != kNoRow) ? __float_as_uint(slab[k * Rp + (int)(b.t - t0)]) : 0u;
        }
    };

    {   // step 0 candidate: first maximum of |X(t, jb)| over the owned rows
        Cand b{0, kNoRow};
        for (int rl = tid; rl < nloc; rl += NTC) b = better(b, Cand{abs_key(slab[rl]), t0 + rl});
        b = block_best_all_n<NTC>(b, wk, wt);
        publish(-1, false, b);
        __syncthreads();
        cluster_arrive_release();
    }

    for (int j = 0; j < a.steps; ++j) {
        const i64 jg = a.jb + j;
        const bool has_next = j + 1 < a.steps;
        const int buf = j & 1;
        cluster_wait_acquire();   // every CTA's step-j candidate, candidate row and current row are visible
        // (1) winner: largest |value|, then smallest row, over the C candidates
        // (key, row and signed value read in one round of remote loads); warps
        // 2-3 meanwhile fetch the current row jg from its owner
        if (tid < 32) {
            Cand w{0, kNoRow};
            int wq = -1;
            unsigned int wvb = 0u;
            for (int q = tid; q < C; q += 32) {
                const unsigned long long kq = *cl.map_shared_rank(&cand_key[buf], q);
                const long long tq = *cl.map_shared_rank(&cand_t[buf], q);
                const unsigned int vq = *cl.map_shared_rank(&cand_vb[buf], q);
                if (tq == kNoRow) continue;
                const Cand y = better(w, Cand{kq, tq});
                if (y.t != w.t) { w = y; wq = q; wvb = vq; }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const Cand y = shfl_down_cand(w, o);
                const int yq = __shfl_down_sync(0xffffffffu, wq, o);
                const unsigned int yvb = __shfl_down_sync(0xffffffffu, wvb, o);
                const Cand z = better(w, y);
                if (z.t != w.t) { w = z; wq = yq; wvb = yvb; }
            }
            if (tid == 0) {
                // a row t >= jg always exists, so some CTA has a candidate
                s_p = (wq >= 0) ? w.t : jg;
                s_gw = wq;
                s_pivbits = (wq >= 0) ? wvb : 0u;
                if (g == 0) a.ipiv[jg] = s_p;
            }
        } else if (tid >= 64 && tid < 64 + pw) {
            const int og = (int)((jg - a.jb) / a.R);   // owner of row jg
            cur_loc[tid - 64] = *cl.map_shared_rank(&cur_row[buf][tid - 64], og);
        }
        __syncthreads();
        const i64 p = s_p;
        const int gw = s_gw;
        const bool elim = gw >= 0 && (s_pivbits & 0x7fffffffu) != 0;   // exact zero pivot: no elimination
        // (2) pivot row into prow and the slab; current row jg to the winner's place
        if (gw >= 0 && tid < pw) {
            const float pr = *cl.map_shared_rank(&cand_row[buf][tid], gw);
            prow[tid] = pr;
            if (jg >= t0 && jg < t1) slab[tid * Rp + (jg - t0)] = pr;
            if (p != jg && p >= t0 && p < t1) slab[tid * Rp + (p - t0)] = cur_loc[tid];
        }
        if (tid == 64 && elim) s_rpiv = 1.0f / __uint_as_float(s_pivbits);
        __syncthreads();
        // (3) multipliers (reciprocal plus one FMA correction: the rounded
        // quotient) and column j+1 of the owned rows below jg; next candidate
        const float rpiv = s_rpiv, pivv = __uint_as_float(s_pivbits);
        const int r0 = (jg + 1 > t0) ? (int)(jg + 1 - t0) : 0;
        Cand b{0, kNoRow};
        for (int rl = r0 + tid; rl < nloc; rl += NTC) {
            float l = 0.f;
            if (elim) {
                const float x = slab[j * Rp + rl];
                l = x * rpiv;
                l = fmaf(fmaf(-pivv, l, x), rpiv, l);
                slab[j * Rp + rl] = l;
            }
            if (has_next) {
                float x = slab[(j + 1) * Rp + rl];
                if (elim) {
                    x = fmaf(-l, prow[j + 1], x);
                    slab[(j + 1) * Rp + rl] = x;
                }
                b = better(b, Cand{abs_key(x), t0 + rl});
            }
        }
        if (has_next) {
            b = block_best_all_n<NTC>(b, wk, wt);
            publish(j, elim, b);
        }
        __syncthreads();
        cluster_arrive_release();   // published (or, on the last step, done reading)
        // (4) bulk update of columns cs.. of the owned rows below jg
        const int nr = nloc - r0, cs = has_next ? j + 2 : j + 1;
        if (elim && nr > 0 && cs < pw) {
            if (nr >= NTC) {
                for (int rl = r0 + tid; rl < nloc; rl += NTC) {
                    const float l = slab[j * Rp + rl];
                    for (int c = cs; c < pw; ++c) slab[c * Rp + rl] = fmaf(-l, prow[c], slab[c * Rp + rl]);
                }
            } else {
                const int ng = NTC / nr, grp = tid / nr;
                if (grp < ng) {
                    const int rl = r0 + tid - grp * nr;
                    const float l = slab[j * Rp + rl];
                    for (int c = cs + grp; c < pw; c += ng) slab[c * Rp + rl] = fmaf(-l, prow[c], slab[c * Rp + rl]);
                }
            }
        }
        __syncthreads();
    }
    cluster_wait_acquire();   // no CTA leaves while another may still read its shared memory
    for (int e = tid; e < nloc * pw; e += NTC) {
        const int c = e % pw, rl = e / pw;
        a.Sk[(a.jb + c) + (t0 + rl) * a.ldsk] = (double)slab[c * Rp + rl];
    }
}

// The panel on one cluster if its rows fit (R = ceil(rows / 16) rows per CTA);
// returns -1 when they do not or the cluster cannot be launched.
static int lu_panel_cluster(const Ctx& c, i64 N, i64 jb, int pw, int st, double* Sk, i64 ldsk, i64* ipiv) {
    const i64 rows = N - jb;
    const i64 R = cdiv(rows, kLuCluster);
    const size_t smem = (size_t)pw * (size_t)(R | 1) * sizeof(float);
    if (smem > (size_t)kMaxSmemLuCl) return -1;
    BQ_TRY(kernel_attrs((const void*)lu_panel_cluster_kernel, kMaxSmemLuCl, true));
    LuClArgs a{};
    a.N = N; a.jb = jb; a.ldsk = ldsk; a.pw = pw; a.steps = st; a.R = (int)R; a.Rp = (int)(R | 1);
    a.Sk = Sk; a.ipiv = ipiv;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kLuCluster);
    cfg.blockDim = dim3(NTC);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = c.stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = kLuCluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    count_launch();
    if (cudaLaunchKernelEx(&cfg, lu_panel_cluster_kernel, a) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return 0;
}

int coop_grid(const void* kernel, size_t smem, const Ctx& c, int want) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, NT, smem) != cudaSuccess || per_sm < 1)
        return 0;
    const int cap = per_sm * c.dev.sms;
    return want < cap ? want : cap;
}

}  // namespace

int coop_scratch_elems(i64 nb, int grid, size_t* elems) {
    // LU: 6G (slots) + 3*G*nb (candidate rows) + 3*nb (current rows); HH: G + 1 + G*nb + G*nb*nb + nb*nb
    const size_t G = (size_t)grid;
    const size_t lu = 6 * G + 3 * G * nb + 3 * nb;
    const size_t hh = G + 8 + G * nb + G * nb * nb + nb * nb;
    *elems = (lu > hh ? lu : hh) + 64;
    return 0;
}

static int launch_coop(const Ctx& c, const void* kernel, int grid, size_t smem, void* args) {
    void* kargs[] = {args};
    // the barrier's arrival counter starts from zero in every launch
    if (cudaMemsetAsync(&c.st->bar, 0, sizeof(GridBar), c.stream) != cudaSuccess) {
        set_error("cooperative launch: resetting the barrier failed");
        return BQRRP_ECUDA;
    }
    count_launch();
    cudaError_t e = cudaLaunchCooperativeKernel(kernel, dim3(grid), dim3(NT), kargs, smem, c.stream);
    if (e != cudaSuccess) {
        set_error("cooperative launch (grid %d, smem %zu): %s", grid, smem, cudaGetErrorString(e));
        return BQRRP_ECUDA;
    }
    return 0;
}

// Row-pivoted LU (first-maximum rule) of X = Sk^T, X: N x d, Sk: d x N with ld
// ldsk, all min(N, d) steps; writes the 0-based swap sequence to ipiv.  Sk is
// overwritten by the factors (in transposed layout).
int getrf_pivots(const Ctx& c, i64 N, i64 d, double* Sk, i64 ldsk, i64* ipiv) {
    return getrf_pivots_ex(c, N, d, Sk, ldsk, ipiv, kPollLimit, -1);
}

// poll_limit bounds every slot wait of the pivot exchange; stall_cta >= 0 makes
// that CTA of the first panel withhold its step-0 candidate, so every wait of
// that launch runs out (the failure-detection self-test).
int getrf_pivots_ex(const Ctx& c, i64 N, i64 d, double* Sk, i64 ldsk, i64* ipiv, unsigned long long poll_limit,
                    int stall_cta) {
    const i64 steps = imin(N, d);
    if (steps <= 0) return 0;
    // c.sketch32: the panels' pivot search and eliminations in FP32
    const void* kfn = c.sketch32 ? (const void*)lu_panel_kernel<float> : (const void*)lu_panel_kernel<double>;
    const size_t esz = c.sketch32 ? sizeof(float) : sizeof(double);
    BQ_TRY(kernel_attrs(kfn, kMaxSmemLu));
    const i64 nbmax = 64;
    const int Gmax_all = (int)imin(c.dev.sms, 148);
    size_t need = 0;
    coop_scratch_elems(nbmax, Gmax_all, &need);
    if (need > c.coop_elems) {
        set_error("getrf_pivots: cooperative scratch too small");
        return BQRRP_ENOMEM;
    }
    View Skv = colmajor(Sk, ldsk);
    for (i64 jb = 0; jb < steps; jb += nbmax) {
        const int pw = (int)imin(nbmax, d - jb);
        const int st = (int)imin(nbmax, steps - jb);
        const i64 rows = N - jb;
        // FP32 panels that fit one cluster exchange pivots through distributed
        // shared memory; the others take the grid kernel
        const bool on_cluster = c.sketch32 && lu_panel_cluster(c, N, jb, pw, st, Sk, ldsk, ipiv) == 0;
        if (!on_cluster) {
            // CTAs: one slab of >= 16 rows each, at most one per SM
            int G = (int)imin(cdiv(rows, 16), Gmax_all);
            i64 R = cdiv(rows, G);
            size_t smem = (size_t)pw * (size_t)(R | 1) * esz;
            if (smem > (size_t)kMaxSmemLu) {
                set_error("getrf_pivots: %lld rows exceed the panel capacity", (long long)rows);
                return BQRRP_EUNSUPPORTED;
            }
            const int Gc = coop_grid(kfn, smem, c, G);
            if (Gc < G) {
                G = Gc;
                if (G < 1) { set_error("getrf_pivots: no co-resident grid"); return BQRRP_ECUDA; }
                R = cdiv(rows, G);
                smem = (size_t)pw * (size_t)(R | 1) * esz;
                if (smem > (size_t)kMaxSmemLu) { set_error("getrf_pivots: panel too tall"); return BQRRP_EUNSUPPORTED; }
            }
            G = (int)cdiv(rows, R);   // drop CTAs that would own no rows
            LuArgs a{};
            a.N = N; a.jb = jb; a.ldsk = ldsk; a.pw = pw; a.steps = st; a.R = (int)R; a.Rp = (int)(R | 1);
            a.Sk = Sk; a.ipiv = ipiv; a.st = c.st;
            a.slot = reinterpret_cast<unsigned long long*>(c.coop);
            a.cand_row = c.coop + 6 * (size_t)G;
            a.cur_row = c.coop + 6 * (size_t)G + 3 * (size_t)G * pw;
            a.poll_limit = poll_limit;
            a.stall_cta = (jb == 0 && stall_cta < G) ? stall_cta : -1;
            // every slot starts unpublished (all-ones) in each launch
            BQ_CUDA(cudaMemsetAsync(a.slot, 0xff, 6 * (size_t)G * sizeof(unsigned long long), c.stream));
            BQ_TRY(launch_coop(c, kfn, G, smem, &a));
        }
        const i64 below = d - (jb + pw);
        if (d - pw > 0) {
            lu_swap_rows_kernel<<<(unsigned)cdiv(d - pw, kSwapRows), 256, 0, c.stream>>>(pw, d, jb, st, ipiv, Sk,
                                                                                       ldsk);
            BQ_LAUNCH_CHECK();
        }
        if (below > 0) {
            // U12^T = Sk(jb+pw:d, jb:jb+st) * L11^{-T}; L11^T = unit upper part of Sk(jb:jb+st, jb:jb+st).
            // Needed even after the last pivot step (N < d): R^sk is formed from the complete U.
            BQ_TRY(trsm_ru(c, below, st, Skv.sub(jb, jb), Skv.sub(jb + pw, jb), true));
            // trailing: Sk(jb+pw:d, jb+pw:N) -= U12^T * L21^T
            if (jb + st < steps)
                BQ_TRY(pgemm(c, false, false, below, N - jb - pw, pw, -1.0, Sk + (jb + pw) + jb * ldsk, ldsk,
                             Sk + jb + (jb + pw) * ldsk, ldsk, 1.0, Sk + (jb + pw) + (jb + pw) * ldsk, ldsk));
        }
        if (jb + st >= steps) break;
    }
    return 0;
}

constexpr i64 kClusterRowsMax = 16 * 280;   // 16 CTAs x 280 rows x 64 columns fit shared memory

// Householder panel (prow x pw) on one cluster of up to 16 CTAs.  Returns 0 on
// success, -1 if the cluster cannot be launched (the caller falls back to the
// cooperative grid kernel), or an error code.
static int hh_panel_cluster(const Ctx& c, i64 prow, int pw, double* Ap, i64 lda, double* tau, double* V, i64 ldv,
                            double* T, i64 ldt) {
    BQ_TRY(kernel_attrs((const void*)hh_panel_cluster_kernel, kMaxSmemHh, true));
    int C = (int)imin(16, imax(1, cdiv(prow, 32)));
    i64 R = cdiv(prow, C);
    C = (int)cdiv(prow, R);
    const size_t smem = ((size_t)pw * (size_t)(R | 1) + (size_t)pw * pw) * sizeof(double);
    if (smem > (size_t)kMaxSmemHh) return -1;
    HhArgs a{};
    a.rows = prow; a.lda = lda; a.ldv = ldv; a.ldt = ldt; a.pw = pw; a.R = (int)R; a.Rp = (int)(R | 1);
    a.A = Ap; a.tau = tau; a.V = V; a.T = T; a.st = c.st;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = c.stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    count_launch();
    const cudaError_t e = cudaLaunchKernelEx(&cfg, hh_panel_cluster_kernel, a);
    if (e != cudaSuccess) {
        cudaGetLastError();   // clear the launch error; the grid kernel takes over
        static std::atomic<bool> logged{false};
        if (getenv("BQRRP_LOG") && !logged.exchange(true))
            fprintf(stderr, "bqrrp: cluster launch (%d CTAs, %zu B smem) failed: %s; using the grid kernel\n", C,
                    smem, cudaGetErrorString(e));
        return -1;
    }
    return 0;
}

// Blocked Householder QR (GEQRF semantics) of rows x cols A: panels of nb
// columns by hh_panel_kernel, trailing update C -= V (T^T (V^T C)).
// V: rows x nb, T: nb x nb, W, W2: nb x cols.
int geqrf_blocked(const Ctx& c, i64 rows, i64 cols, double* A, i64 lda, double* tau, double* V, double* T,
                  double* W, double* W2, i64 nb, i64 kstop) {
    i64 kk = imin(rows, cols);
    if (kstop >= 0) kk = imin(kk, kstop);   // factor only the first kstop columns, update all
    if (kk <= 0) return 0;
    if (nb > 64) nb = 64;
    BQ_TRY(kernel_attrs((const void*)hh_panel_kernel, kMaxSmemHh));
    const int Gmax_all = (int)imin(c.dev.sms, 148);
    size_t need = 0;
    coop_scratch_elems(nb, Gmax_all, &need);
    if (need > c.coop_elems) {
        set_error("geqrf_blocked: cooperative scratch too small");
        return BQRRP_ENOMEM;
    }
    for (i64 jb = 0; jb < kk; jb += nb) {
        const int pw = (int)imin(nb, kk - jb);
        const i64 prow = rows - jb;
        if (prow <= kClusterRowsMax) {
            const int rc = hh_panel_cluster(c, prow, pw, A + jb + jb * lda, lda, tau + jb, V, rows, T, nb);
            if (rc == 0) goto trailing;
            if (rc != -1) return rc;   // -1: cluster launch not possible, use the grid kernel
        }
        {
        int G = (int)imin(cdiv(prow, 32), Gmax_all);
        i64 R = cdiv(prow, G);
        size_t smem = (size_t)pw * (size_t)(R | 1) * sizeof(double);
        if (smem > (size_t)kMaxSmemHh) {
            set_error("geqrf_blocked: %lld rows exceed the panel capacity", (long long)prow);
            return BQRRP_EUNSUPPORTED;
        }
        const int Gc = coop_grid((const void*)hh_panel_kernel, smem, c, G);
        if (Gc < G) {
            G = Gc;
            if (G < 1) { set_error("geqrf_blocked: no co-resident grid"); return BQRRP_ECUDA; }
            R = cdiv(prow, G);
            smem = (size_t)pw * (size_t)(R | 1) * sizeof(double);
            if (smem > (size_t)kMaxSmemHh) { set_error("geqrf_blocked: panel too tall"); return BQRRP_EUNSUPPORTED; }
        }
        G = (int)cdiv(prow, R);
        HhArgs a{};
        a.rows = prow; a.lda = lda; a.ldv = rows; a.ldt = nb; a.pw = pw; a.R = (int)R; a.Rp = (int)(R | 1);
        a.A = A + jb + jb * lda; a.tau = tau + jb; a.V = V; a.T = T; a.st = c.st;
        a.part1 = c.coop;
        a.alpha = c.coop + G;
        a.part2 = c.coop + G + 8;
        a.gpart = c.coop + G + 8 + (size_t)G * pw;
        a.gsum = a.gpart + (size_t)G * pw * pw;
        BQ_TRY(launch_coop(c, (const void*)hh_panel_kernel, G, smem, &a));
        }
    trailing:
        const i64 nc = cols - jb - pw;
        if (nc > 0) {
            double* C = A + jb + (jb + pw) * lda;
            BQ_TRY(pgemm(c, true, false, pw, nc, prow, 1.0, V, rows, C, lda, 0.0, W, nb));
            BQ_TRY(dgemm(c, true, false, pw, nc, pw, 1.0, T, nb, W, nb, 0.0, W2, nb));
            BQ_TRY(pgemm(c, false, false, prow, nc, pw, -1.0, V, rows, W2, nb, 1.0, C, lda));
        }
    }
    return 0;
}

namespace {
// From the LU factors held in X (Sk layout, d x N, ld ldx, all interchanges
// applied): U^T (d x s lower trapezoid, s = min(N, d)) into Ub, and X itself
// becomes L^T (s x N unit upper trapezoid).
__global__ void lu_split_kernel(i64 d, i64 s, i64 N, double* X, i64 ldx, double* Ub, i64 ldu) {
    const i64 total = d * N;
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (i64)gridDim.x * blockDim.x) {
        const i64 j = e % d, t = e / d;
        const double x = X[j + t * ldx];
        if (t < s) Ub[j + t * ldu] = (j >= t) ? x : 0.0;
        if (j < s) X[j + t * ldx] = (t > j) ? x : (t == j ? 1.0 : 0.0);
    }
}

__global__ void zero_rows_kernel(i64 r0, i64 r1, i64 N, double* X, i64 ldx) {
    const i64 h = r1 - r0;
    const i64 total = h * N;
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (i64)gridDim.x * blockDim.x)
        X[r0 + e % h + (e / h) * ldx] = 0.0;
}
}  // namespace

// R^sk of Alg. 2 from the LU factors: the permuted sketch is U^T L^T, so with
// U^T = Q1 R1 (Householder QR of a d x s matrix) its R factor is R1 L^T.  This
// is the R of GEQRF on the permuted sketch up to row signs (and rounding); the
// row signs cancel in everything BQRRP derives from R^sk (R11, Y, T) and leave
// the next LU's pivots unchanged.  Writes R^sk (zeros below the diagonal) into
// Sk (d x N, ld ldsk); X (the LU factors) is consumed.
namespace {
// R factor of the Householder QR (dlarfg convention) of a small d x s matrix
// W (ld d, s <= d) held entirely in the distributed shared memory of one
// thread-block cluster.  Column c lives in CTA c mod C at local slot c / C.
// Reflector j is published by the owner of column j in its shared memory
// (double-buffered by step parity).  Step j: every CTA copies reflector j
// through DSMEM and applies it to its own columns; with lookahead, warp 0 of
// the owner of column j+1 first updates that column and forms reflector j+1
// while the other warps update the rest, so one cluster barrier per step
// separates the reflectors and the owner's scalar work (a square root and a
// division, ~650 cycles each on B300's FP64 unit) leaves the critical path.
// Only R (upper triangle, zeros below) is written back to W.
constexpr int kSqrMaxD = 640;

__device__ inline void bar_sync_64() { asm volatile("bar.sync 1, 64;" ::: "memory"); }   // warps 0-1

// T: the arithmetic (double; float for the reduced-precision sketch QR, whose
// loads and stores of W convert).  Sign and zero tests on T's bit pattern.
__device__ __forceinline__ bool sq_nonzero(double x) {
    return ((unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull) != 0;
}
__device__ __forceinline__ bool sq_nonzero(float x) { return ((unsigned)__float_as_uint(x) & 0x7fffffffu) != 0; }
__device__ __forceinline__ bool sq_nonneg(double x) {   // x >= 0.0 (-0.0 counts as non-negative)
    const long long b = __double_as_longlong(x);
    return b >= 0 || b == (long long)0x8000000000000000ull;
}
__device__ __forceinline__ bool sq_nonneg(float x) {
    const int b = __float_as_int(x);
    return b >= 0 || b == (int)0x80000000u;
}

template <typename T, int NTQ>
__global__ void __launch_bounds__(NTQ) small_qr_cluster_kernel(i64 d, i64 s, double* W) {
    extern __shared__ __align__(16) unsigned char loc_raw[];
    T* loc = (T*)loc_raw;                           // [ncl][d] local columns
    __shared__ T vbuf[2][kSqrMaxD];
    __shared__ T vloc[kSqrMaxD];
    __shared__ T s_tau[2], s_scal[2];
    __shared__ T red2[2];
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks(), g = (int)cl.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ncl = (int)((s - g + C - 1) / C);    // columns g, g + C, ... below s
    for (int lc = 0; lc < ncl; ++lc) {
        const i64 gc = (i64)lc * C + g;
        for (i64 r = tid; r < d; r += NTQ) loc[(i64)lc * d + r] = (T)W[r + gc * d];
    }
    __syncthreads();

    // Reflector of column j (owned here), by one warp: v(j) = 1,
    // v(j+1:) = x(j+1:) / (alpha - beta), tau = (beta - alpha) / beta, both
    // from the single quotient q = 1 / (beta (alpha - beta)).  vbuf[par] gets
    // x(j+1:) unscaled and s_scal[par] the scale, which every reader applies
    // as it copies (off the owner's critical path).  The column becomes
    // (beta, 0, ..., 0).
    // Scalars of the reflector of column j (x), given xn2 = ||x(j+1:)||^2;
    // one thread.  Writes beta into x(j) and tau, scale to s_tau/s_scal[par].
    auto reflector_scalars = [&](T* x, i64 j, T xn2, int par) {
        const T alpha = x[j];
        const bool nz = sq_nonzero(xn2);
        T tau = T(0), beta = alpha, scal = T(1);
        if (nz) {
            const bool apos = sq_nonneg(alpha);
            const T nrm = sqrt(alpha * alpha + xn2);
            beta = apos ? -nrm : nrm;
            const T am = alpha - beta;
            const T q = T(1) / (beta * am);
            scal = beta * q;
            tau = -(am * am) * q;
        }
        x[j] = beta;
        s_tau[par] = tau;
        s_scal[par] = scal;
    };
    // The first reflector, by one warp.
    auto reflect = [&](i64 j, int par) {
        T* x = loc + (j / C) * d;
        T xn2 = T(0);
        for (i64 r = j + 1 + lane; r < d; r += 32) xn2 = fma(x[r], x[r], xn2);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) xn2 += __shfl_xor_sync(0xffffffffu, xn2, off);
        __syncwarp();
        if (lane == 0) reflector_scalars(x, j, xn2, par);
        for (i64 r = j + 1 + lane; r < d; r += 32) {
            vbuf[par][r] = x[r];
            x[r] = T(0);                                  // below the diagonal of R
        }
    };
    // col -= tau v (v^T col) over rows [j, d), by one warp
    auto apply = [&](T* col, i64 j, T tau) {
        T dot = T(0);
        for (i64 r = j + lane; r < d; r += 32) dot = fma(vloc[r], col[r], dot);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, off);
        const T w = tau * dot;
        for (i64 r = j + lane; r < d; r += 32) col[r] = fma(-w, vloc[r], col[r]);
    };

    if (g == 0 && warp == 0) reflect(0, 0);
    cl.sync();
    for (i64 j = 0; j < s; ++j) {
        const int o = (int)(j % C), par = (int)(j & 1);
        // reflector j from its owner (the two scalars and the vector in one round of
        // remote loads)
        const T* vsrc = cl.map_shared_rank(&vbuf[par][0], o);
        const T scal = *cl.map_shared_rank(&s_scal[par], o);
        const T tau = *cl.map_shared_rank(&s_tau[par], o);
        for (i64 r = j + tid; r < d; r += NTQ) vloc[r] = (r == j) ? T(1) : vsrc[r] * scal;
        __syncthreads();
        const bool live = sq_nonzero(tau);
        const bool next_here = j + 1 < s && (int)((j + 1) % C) == g;
        if (next_here && warp < 2) {
            // lookahead: warps 0-1 update column j+1 first, then form its reflector
            // (rows split over 64 threads, partial sums combined through shared
            // memory behind named barrier 1)
            const int t = tid;
            T* x = loc + ((j + 1) / C) * d;
            if (live) {
                T dot = T(0);
                for (i64 r = j + t; r < d; r += 64) dot = fma(vloc[r], x[r], dot);
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, off);
                if (lane == 0) red2[warp] = dot;
                bar_sync_64();
                const T w = tau * (red2[0] + red2[1]);
                for (i64 r = j + t; r < d; r += 64) x[r] = fma(-w, vloc[r], x[r]);
                bar_sync_64();
            }
            const i64 jj = j + 1;
            T xn2 = T(0);
            for (i64 r = jj + 1 + t; r < d; r += 64) xn2 = fma(x[r], x[r], xn2);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) xn2 += __shfl_xor_sync(0xffffffffu, xn2, off);
            if (lane == 0) red2[warp] = xn2;
            bar_sync_64();
            if (t == 0) reflector_scalars(x, jj, red2[0] + red2[1], par ^ 1);
            for (i64 r = jj + 1 + t; r < d; r += 64) {   // same rows as this thread's norm terms
                vbuf[par ^ 1][r] = x[r];
                x[r] = T(0);                              // below the diagonal of R
            }
        }
        if (live) {
            const int w0 = next_here ? 2 : 0, nw = NTQ / 32 - w0;
            if (warp >= w0) {
                for (int lc = warp - w0; lc < ncl; lc += nw) {
                    const i64 gc = (i64)lc * C + g;
                    if (gc <= j || (next_here && gc == j + 1)) continue;
                    apply(loc + (i64)lc * d, j, tau);
                }
            }
        }
        cl.sync();   // reflector j+1 published; reflector j no longer read
    }
    for (int lc = 0; lc < ncl; ++lc) {
        const i64 gc = (i64)lc * C + g;
        for (i64 r = tid; r < d; r += NTQ) W[r + gc * d] = (r <= gc) ? (double)loc[(i64)lc * d + r] : 0.0;
    }
    cl.sync();    // no CTA leaves while another may still read its shared memory
}

// Launch on a cluster of up to 16 CTAs; -1 when the shape or the cluster does
// not fit (the caller then uses the blocked QR).
// c.sketch32: the QR in FP32 arithmetic (W converted on load and store).
int small_qr_cluster(const Ctx& c, i64 d, i64 s, double* W) {
    if (d > kSqrMaxD || s < 1 || s > d) return -1;
    int C = 16;
    size_t smem = (size_t)((s + C - 1) / C) * (size_t)d * sizeof(double);
    if (smem > 208 * 1024) return -1;
    // 256 threads in either precision (1024 measured slower for FP32: each
    // step is bound by its cluster barrier and the owner's reflector chain)
    const void* fn = c.sketch32 ? (const void*)small_qr_cluster_kernel<float, NT>
                                : (const void*)small_qr_cluster_kernel<double, NT>;
    if (c.sketch32) smem /= 2;
    BQ_TRY(kernel_attrs(fn, 208 * 1024, true));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = c.stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    count_launch();
    const cudaError_t le = c.sketch32 ? cudaLaunchKernelEx(&cfg, small_qr_cluster_kernel<float, NT>, d, s, W)
                                      : cudaLaunchKernelEx(&cfg, small_qr_cluster_kernel<double, NT>, d, s, W);
    if (le != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return 0;
}
}  // namespace

int rsk_from_lu(const Ctx& c, i64 d, i64 N, double* X, i64 ldx, double* Sk, i64 ldsk, double* Ub, double* tau,
                double* V, double* T, double* W, double* W2) {
    const i64 s = imin(N, d);
    if (s <= 0) return 0;
    const unsigned blocks = (unsigned)imax(1, imin(cdiv(d * N, 256), 8LL * c.dev.sms));
    lu_split_kernel<<<blocks, 256, 0, c.stream>>>(d, s, N, X, ldx, Ub, d);
    BQ_LAUNCH_CHECK();
    // R1 of U^T: on one cluster when the d x s factor fits its shared memory,
    // else by the blocked Householder QR
    if (small_qr_cluster(c, d, s, Ub) != 0) {
        BQ_TRY(geqrf_blocked(c, d, s, Ub, d, tau, V, T, W, W2, 64));
        BQ_TRY(set_zero_below(c, s, s, Ub, d));
    }
    BQ_TRY(pgemm(c, false, false, s, N, s, 1.0, Ub, d, X, ldx, 0.0, Sk, ldsk, kGemmAUpper));
    if (s < d) {
        zero_rows_kernel<<<blocks, 256, 0, c.stream>>>(s, d, N, Sk, ldsk);
        BQ_LAUNCH_CHECK();
    }
    return 0;
}

}  // namespace bq
