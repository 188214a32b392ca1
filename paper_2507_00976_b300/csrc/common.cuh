// common.cuh -- shared internals of the sm_103a BQRRP library (not public).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <cstdio>
#include <string>

#include "../../include/bqrrp.h"

namespace bq {

using i64 = int64_t;

// ------------------------------------------------------------------ errors
void set_error(const char* fmt, ...);
const char* get_error();

#define BQ_CUDA(call)                                                              \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            ::bq::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call,             \
                            cudaGetErrorString(e_));                               \
            return BQRRP_ECUDA;                                                    \
        }                                                                          \
    } while (0)

#define BQ_TRY(expr)                                                               \
    do {                                                                           \
        int rc_ = (expr);                                                          \
        if (rc_ != 0) return rc_;                                                  \
    } while (0)

void count_launch();
// Phase profiler (bqrrp_profile_*): whether it is on, and adding one call's
// per-phase device milliseconds and algorithmic FLOPs to its totals.
bool profile_on();
void profile_add(const double* ms, const double* flops);

#define BQ_LAUNCH_CHECK()                                                          \
    do {                                                                           \
        ::bq::count_launch();                                                      \
        cudaError_t e_ = cudaGetLastError();                                       \
        if (e_ != cudaSuccess) {                                                   \
            ::bq::set_error("%s:%d launch: %s", __FILE__, __LINE__,                \
                            cudaGetErrorString(e_));                               \
            return BQRRP_ECUDA;                                                    \
        }                                                                          \
    } while (0)

// ------------------------------------------------------------------ views
// Strided matrix view: element (i, j) at p[i*rs + j*cs].
struct View {
    double* p;
    i64 rs, cs;
    __host__ __device__ double* at(i64 i, i64 j) const { return p + i * rs + j * cs; }
    View sub(i64 i, i64 j) const { return View{p + i * rs + j * cs, rs, cs}; }
    View t() const { return View{p, cs, rs}; }
};
inline View colmajor(double* p, i64 ld) { return View{p, 1, ld}; }
inline View colmajor(const double* p, i64 ld) { return View{const_cast<double*>(p), 1, ld}; }

// ------------------------------------------------------------------ workspace
struct Arena {
    char* base = nullptr;
    size_t cap = 0;
    size_t off = 0;
    bool dry = false;   // sizing pass: count bytes, hand out nothing usable
    template <class T>
    T* take(size_t count) {
        size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
        size_t at = off;
        off += bytes;
        if (dry || off > cap) return nullptr;
        return reinterpret_cast<T*>(base + at);
    }
    bool ok() const { return dry || off <= cap; }
};

// ------------------------------------------------------------------ device status
// One per call, zeroed at the start; read back by the host at a few points.
struct GridBar {
    unsigned int count;
    unsigned int gen;
};

struct DevStatus {
    int err_timeout;       // a grid barrier gave up
    int potrf_info;        // first failing Cholesky column (INT_MAX if none)
    int sk_nonfinite;      // the sketch held NaN/Inf this iteration
    int a_nonfinite;       // the input held NaN/Inf
    int zero_col;          // first permuted working column is all zero
    int pad0;
    i64 k;                 // tri_rank result
    i64 moved;             // number of columns the permutation moves
    double r00;            // |Rsk(0,0)| of the first iteration (tri_rank scale)
    double blk00;          // |Rsk(0,0)| of the previous iteration (FP32 sketch QRCP: rank floor)
    GridBar bar;
    unsigned int pad1[2];
};

// ------------------------------------------------------------------ helpers
inline i64 cdiv(i64 a, i64 b) { return (a + b - 1) / b; }
inline i64 imin(i64 a, i64 b) { return a < b ? a : b; }
inline i64 imax(i64 a, i64 b) { return a > b ? a : b; }

struct Device {
    int id = 0;
    int sms = 148;
};
int current_device(Device* dev);
// Kernel attributes are per device: raise `fn`'s dynamic shared-memory limit
// to at least smem_bytes (and allow non-portable cluster sizes when asked) on
// the current device, once per (device, kernel); the CUDA result is checked.
int kernel_attrs(const void* fn, int smem_bytes, bool nonportable_cluster = false);

// ------------------------------------------------------------------ Philox4x32-10
// Salmon, Moraes, Dror, Shaw, SC'11: two-word key, four-word counter, ten rounds.
__host__ __device__ inline void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                              uint32_t k0, uint32_t k1, uint32_t out[4]) {
    const uint32_t kM0 = 0xD2511F53u, kM1 = 0xCD9E8D57u;
    const uint32_t kW0 = 0x9E3779B9u, kW1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)kM0 * c0;
        const uint64_t p1 = (uint64_t)kM1 * c2;
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        const uint32_t n1 = (uint32_t)p1;
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        const uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += kW0;
        k1 += kW1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// Dense +-1 sketch entry S(r, j) (see bqrrp_sketch_operator).
__host__ __device__ inline double sketch_dense_entry(uint64_t seed, i64 r, i64 j) {
    uint32_t o[4];
    philox4x32_10((uint32_t)j, (uint32_t)(r >> 7), 0u, 0u, (uint32_t)seed, (uint32_t)(seed >> 32), o);
    const int q = (int)(r & 127);
    return ((o[q >> 5] >> (q & 31)) & 1u) ? -1.0 : 1.0;
}

// ------------------------------------------------------------------ grid barrier
// Barrier for cooperative launches (all CTAs co-resident).  The arrival
// counter only grows within a launch (the host zeroes it before every
// cooperative launch): arrival number a of a grid of n CTAs belongs to epoch
// a / n and waits until the counter reaches (a / n + 1) * n.  Arrival is a
// release, polling an acquire (thread 0 of each CTA, bracketed by
// __syncthreads).  Every wait is bounded: after kSpinLimit polls the CTA
// records a timeout in the status block and the barrier returns false;
// callers then exit.
constexpr unsigned long long kSpinLimit = 1ull << 28;   // polls of ~20 ns: a few seconds

__device__ inline unsigned int ld_acquire_u32(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ inline bool grid_barrier(DevStatus* st, unsigned int nblocks) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned int* cnt = &st->bar.count;
        unsigned int a;
        asm volatile("atom.add.release.gpu.global.u32 %0, [%1], 1;" : "=r"(a) : "l"(cnt) : "memory");
        const unsigned int target = (a / nblocks + 1) * nblocks;
        unsigned long long spins = 0;
        while ((int)(ld_acquire_u32(cnt) - target) < 0) {
            if (++spins > kSpinLimit || ((spins & 1023) == 0 && *((volatile int*)&st->err_timeout))) {
                atomicExch(&st->err_timeout, 1);
                ok = 0;
                break;
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ------------------------------------------------------------------ batched plans (batched.cu)
struct BatchPlan;
// ct: columns per trailing-update tile of each matrix, 32 or 64 (null: 64).
int batch_plan_create_ex(BatchPlan** out, i64 batch, const i64* m, const i64* n, const i64* b, const i64* d,
                         const uint64_t* seed, double tol, const i64* offA, const i64* offJ, const i64* offT,
                         const i64* ct);
size_t batch_plan_bytes(const BatchPlan* P);
int batch_factor(BatchPlan* P, double* A, int64_t* jpvt, double* tau, int64_t* rank, int64_t* trunc,
                 int32_t* info, void* ws, size_t ws_bytes, cudaStream_t stream, int use_graph);
void batch_plan_destroy(BatchPlan* P);
// Cap the dependency-driven kernel's grid (persistent CTAs), leaving SMs to
// concurrent work; 0 removes the cap.
void batch_plan_set_grid_cap(BatchPlan* P, int ctas);
// Run the plan as one kernel per phase and block iteration (short launches
// that interleave with concurrent work) instead of the persistent form.
void batch_plan_set_lockstep(BatchPlan* P, bool on);

// ------------------------------------------------------------------ launchers (internal API)
struct Ctx {
    cudaStream_t stream;
    Device dev;
    DevStatus* st;          // device status block
    double* splitk;         // split-K partials (may be null)
    size_t splitk_elems;
    // cooperative-kernel scratch
    double* coop;           // partial buffers
    size_t coop_elems;
    // mixed precision: large products go to the bf16-slice tensor-core GEMM
    bool mixed = false;
    // reduced-precision Alg. 2: the LU panels and the QR of the d x d LU
    // factor (R^sk) in FP32 arithmetic
    bool sketch32 = false;
    void* oz_ws = nullptr;
    size_t oz_bytes = 0;
};

// gemm.cu
// Structure flags of dgemm/pgemm.  kGemmAUpper: op(A) is upper triangular
// (M == K), so output rows [m0, m0+64) only take K >= m0.  kGemmCUpper: only
// the upper triangle of C is wanted (M == N); output tiles strictly below the
// diagonal are written as beta*C (zero when beta == 0) without a K loop.
constexpr int kGemmAUpper = 1, kGemmCUpper = 2;
int dgemm(const Ctx& c, bool ta, bool tb, i64 M, i64 N, i64 K, double alpha, const double* A, i64 lda,
          const double* B, i64 ldb, double beta, double* C, i64 ldc, int flags = 0);
int gemm_view(const Ctx& c, i64 M, i64 N, i64 K, double alpha, View A, View B, double beta, View C);
// FP64-accurate product: the tensor-core slice GEMM when c.mixed and the
// problem is large enough (and its workspace fits), else the FP64 SIMT GEMM.
int pgemm(const Ctx& c, bool ta, bool tb, i64 M, i64 N, i64 K, double alpha, const double* A, i64 lda,
          const double* B, i64 ldb, double beta, double* C, i64 ldc, int flags = 0);
// Msk = S A with the +-1 operator generated in the tile loader.  splits > 0
// forces the split-K count (sketch_dense_splits(d, m, n) of the whole product
// makes column slices of it give the whole product's bits).
int sketch_dense_gemm(const Ctx& c, i64 d, i64 m, i64 n, uint64_t seed, const double* A, i64 lda, double* Msk,
                      i64 ldsk, int splits = 0);
int sketch_dense_splits(const Ctx& c, i64 d, i64 m, i64 n);

// dense.cu
int trsm_ru(const Ctx& c, i64 rows, i64 k, View R, View X, bool unit);   // X <- X * R^{-1}
// X <- X * R^{-1} for a tall column-major X (R upper, non-unit): with
// c.mixed the updates between 64-column blocks are pgemm products.
int trsm_ru_tall(const Ctx& c, i64 rows, i64 k, const double* R, i64 ldr, double* X, i64 ldx);
int potrf_u(const Ctx& c, i64 k, double* G, i64 ldg);                    // G = R^T R, info -> st
int modlu(const Ctx& c, i64 rows, i64 k, double* Y, i64 ldy, double* D); // Householder reconstruction LU
int copy_mat(const Ctx& c, i64 rows, i64 cols, const double* src, i64 lds, double* dst, i64 ldd);
int copy_triu(const Ctx& c, i64 rows, i64 cols, const double* src, i64 lds, double* dst, i64 ldd);
int set_zero_below(const Ctx& c, i64 rows, i64 cols, double* A, i64 lda);
int any_nonfinite(const Ctx& c, i64 rows, i64 cols, const double* A, i64 lda, int* flag);

// sketch.cu
int sketch_write(const Ctx& c, i64 d, i64 m, uint64_t seed, int kind, i64 nnz, double* S, i64 lds);
int sketch_sparse_apply(const Ctx& c, i64 d, i64 m, i64 n, uint64_t seed, i64 nnz, const double* A, i64 lda,
                        double* Msk, i64 ldsk, void* ws, size_t ws_bytes);
size_t sketch_sparse_ws(i64 d, i64 m, i64 nnz);

// bqrrp.cu
int cholqr_panel_steps(const Ctx& c, i64 rows, i64 w, i64* kio, double* Mp, i64 ldm, const double* Rsk, i64 ldr,
                       double* Y, i64 ldy, double* G, double* U, double* Tb, double* R11, double* D, i64 ldb,
                       double* tau);

// ozaki.cu (FP64-accurate products on the bf16 tensor cores)
constexpr int kOzPlanes = 7;              // balanced 8-bit slices per FP64 operand (54-bit fixed point)
constexpr i64 kOzMaxK = (i64)1 << 17;     // K per slice-GEMM launch (longer K is split)
size_t ozaki_ws_bytes(i64 M, i64 N, i64 K, int sa);
// Bytes to add to a workspace sized as the largest of several ozaki_ws_bytes
// so that every product whose slice planes fit it also has room for its
// split-K integer sums.
size_t ozaki_split_reserve();
int ozaki_gemm(const Ctx& c, bool ta, bool tb, i64 M, i64 N, i64 K, double alpha, const double* A, i64 lda,
               const double* B, i64 ldb, double beta, double* C, i64 ldc, void* ws, size_t ws_bytes);
int ozaki_sketch(const Ctx& c, i64 d, i64 m, i64 n, uint64_t seed, const double* A, i64 lda, double* Msk, i64 ldsk,
                 void* ws, size_t ws_bytes);
size_t ozaki_sketch_ws_bytes(i64 d, i64 m, i64 n);   // workspace of ozaki_sketch

// panels.cu
int getrf_pivots(const Ctx& c, i64 N, i64 d, double* X, i64 ldx, i64* ipiv); // LUPP in Sk layout
int getrf_pivots_ex(const Ctx& c, i64 N, i64 d, double* X, i64 ldx, i64* ipiv, unsigned long long poll_limit,
                    int stall_cta);
int geqrf_blocked(const Ctx& c, i64 rows, i64 cols, double* A, i64 lda, double* tau, double* V,
                  double* T, double* W, double* W2, i64 nb, i64 kstop = -1);
int coop_scratch_elems(i64 nb, int grid, size_t* elems);
int rsk_from_lu(const Ctx& c, i64 d, i64 N, double* X, i64 ldx, double* Sk, i64 ldsk, double* Ub, double* tau,
                double* V, double* T, double* W, double* W2);

// perm.cu
int piv_transform_moved(const Ctx& c, i64 N, i64 steps, const i64* ipiv, i64* Jsk, const int* identity_flag,
                        i64* pos, i64* src, i64* count);
int moved_list_given(const Ctx& c, i64 N, i64* J, i64* pos, i64* src, i64* count, i64 max_moved);
int gather_cols(const Ctx& c, i64 rows, double* M, i64 ldm, const i64* pos, const i64* src, const i64* count,
                i64 max_moved, double* stage, i64 ldst);
int gather_idx(const Ctx& c, i64* J, const i64* pos, const i64* src, const i64* count, i64 max_moved,
               i64* stage);

}  // namespace bq
