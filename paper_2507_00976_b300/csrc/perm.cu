// perm.cu -- pivot-format conversion and the column permutation (Alg. 5).
//
// Alg. 2's LU yields a swap sequence ipiv of s = min(N, d) steps with
// ipiv[j] >= j, so the permutation J^sk it encodes moves at most 2s of the N
// columns.  Instead of the paper's full out-of-place copy of M (Alg. 5 with
// pointer ping-pong, Sec. 4.2), the moved positions are listed once and only
// those columns are staged out (gather) and written back (scatter):
// 2 * 2s * m * 16 bytes per iteration instead of m * N * 16, and no m x n
// second buffer.  The result equals Alg. 5's out(:, t) = in(:, J[t]).
#include <mutex>

#include "common.cuh"

namespace bq {

namespace {

constexpr int PT = 1024;

// piv_transform (Alg. 2): J = identity on N entries, then swap J[j] and
// J[ipiv[j]] for j = 0..steps-1 in order (identity when *identity_flag).
// The swaps run sequentially on one thread over a shared-memory copy; the
// moved list (positions t with J[t] != t, increasing t) is then compacted by
// the whole block.
__global__ void __launch_bounds__(PT) piv_moved_kernel(i64 N, i64 steps, const i64* __restrict__ ipiv, i64* Jsk,
                                                       const int* identity_flag, i64* pos, i64* src, i64* count,
                                                       int use_smem, int given, i64 cap) {
    extern __shared__ int Js[];
    __shared__ int s_ident;
    __shared__ i64 warp_tot[PT / 32];
    const int tid = threadIdx.x;
    if (tid == 0) s_ident = identity_flag ? *identity_flag : 0;
    if (use_smem) {
        for (i64 t = tid; t < N; t += PT) Js[t] = given ? (int)Jsk[t] : (int)t;
    } else if (!given) {
        for (i64 t = tid; t < N; t += PT) Jsk[t] = t;
    }
    __syncthreads();
    int* ip = Js + (use_smem ? N : 0);   // ipiv staged in shared memory
    if (use_smem)
        for (i64 j = tid; j < steps; j += PT) ip[j] = (int)ipiv[j];
    __syncthreads();
    if (tid == 0 && !s_ident && !given) {
        if (use_smem) {
            for (i64 j = 0; j < steps; ++j) {
                const int p = ip[j];
                const int x = Js[j];
                Js[j] = Js[p];
                Js[p] = x;
            }
        } else {
            for (i64 j = 0; j < steps; ++j) {
                const i64 p = ipiv[j];
                const i64 x = Jsk[j];
                Jsk[j] = Jsk[p];
                Jsk[p] = x;
            }
        }
    }
    __syncthreads();
    if (use_smem && !given)
        for (i64 t = tid; t < N; t += PT) Jsk[t] = Js[t];
    __syncthreads();
    // compaction: thread tid scans the contiguous range [lo, hi)
    const i64 chunk = (N + PT - 1) / PT;
    const i64 lo = (i64)tid * chunk;
    const i64 hi = (lo + chunk < N) ? lo + chunk : N;
    i64 cnt = 0;
    for (i64 t = lo; t < hi; ++t) {
        const i64 v = use_smem ? (i64)Js[t] : Jsk[t];
        cnt += (v != t);
    }
    // exclusive scan of cnt over the block
    const int lane = tid & 31, w = tid >> 5;
    i64 x = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const i64 y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
        i64 z = (lane < PT / 32) ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const i64 y = __shfl_up_sync(0xffffffffu, z, o);
            if (lane >= o) z += y;
        }
        if (lane < PT / 32) warp_tot[lane] = z;   // inclusive
    }
    __syncthreads();
    i64 off = x - cnt + (w > 0 ? warp_tot[w - 1] : 0);
    for (i64 t = lo; t < hi; ++t) {
        const i64 v = use_smem ? (i64)Js[t] : Jsk[t];
        if (v != t) {
            if (off < cap) {   // never write past the caller's list capacity
                pos[off] = t;
                src[off] = v;
            }
            ++off;
        }
    }
    if (tid == PT - 1) *count = warp_tot[PT / 32 - 1];
}

// pass 0: stage(:, q) = M(:, src[q]);  pass 1: M(:, pos[q]) = stage(:, q).
// A CTA copies kMoveChunk consecutive rows of one column; with both column
// bases 16-byte aligned (even leading dimensions, aligned buffers) each thread
// moves 8 double2 (128 bytes in flight per thread), else single doubles.
constexpr int kMoveChunk = 4096;
__global__ void __launch_bounds__(256) move_cols_kernel(i64 rows, double* M, i64 ldm, const i64* __restrict__ pos,
                                                        const i64* __restrict__ src, const i64* __restrict__ count,
                                                        double* stage, i64 ldst, int pass, int vec) {
    const i64 q = blockIdx.y;
    if (q >= *count) return;   // q < gridDim.y = the list capacity
    const i64 col = pass == 0 ? src[q] : pos[q];
    const double* from = pass == 0 ? M + col * ldm : stage + q * ldst;
    double* to = pass == 0 ? stage + q * ldst : M + col * ldm;
    const i64 base = (i64)blockIdx.x * kMoveChunk;
    if (vec && base + kMoveChunk <= rows) {
        const double2* f2 = reinterpret_cast<const double2*>(from + base);
        double2* t2 = reinterpret_cast<double2*>(to + base);
        double2 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = f2[threadIdx.x + 256 * u];
#pragma unroll
        for (int u = 0; u < 8; ++u) t2[threadIdx.x + 256 * u] = v[u];
        return;
    }
    double v[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        const i64 i = base + threadIdx.x + 256 * u;
        if (i < rows) v[u] = from[i];
    }
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        const i64 i = base + threadIdx.x + 256 * u;
        if (i < rows) to[i] = v[u];
    }
}

__global__ void move_idx_kernel(i64* J, const i64* __restrict__ pos, const i64* __restrict__ src,
                                const i64* __restrict__ count, i64 max_moved, i64* stage, int pass) {
    const i64 q = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= max_moved || q >= *count) return;
    if (pass == 0) stage[q] = J[src[q]];
    else J[pos[q]] = stage[q];
}

}  // namespace

int piv_transform_moved(const Ctx& c, i64 N, i64 steps, const i64* ipiv, i64* Jsk, const int* identity_flag,
                        i64* pos, i64* src, i64* count) {
    if (N <= 0) return 0;
    const size_t smem = (size_t)(N + steps) * sizeof(int);
    int use_smem = smem <= 200 * 1024 ? 1 : 0;
    BQ_TRY(kernel_attrs((const void*)piv_moved_kernel, 200 * 1024));
    piv_moved_kernel<<<1, PT, use_smem ? smem : 0, c.stream>>>(N, steps, ipiv, Jsk, identity_flag, pos, src, count,
                                                               use_smem, 0, imin(N, 2 * steps));
    BQ_LAUNCH_CHECK();
    return 0;
}

// Moved list of a given permutation J (0-based); fails when more than
// max_moved positions move.
int moved_list_given(const Ctx& c, i64 N, i64* J, i64* pos, i64* src, i64* count, i64 max_moved) {
    if (N <= 0) return 0;
    const size_t smem = (size_t)N * sizeof(int);
    const int use_smem = smem <= 200 * 1024 ? 1 : 0;
    BQ_TRY(kernel_attrs((const void*)piv_moved_kernel, 200 * 1024));
    piv_moved_kernel<<<1, PT, use_smem ? smem : 0, c.stream>>>(N, 0, nullptr, J, nullptr, pos, src, count, use_smem, 1,
                                                               max_moved);
    BQ_LAUNCH_CHECK();
    return 0;
}

int gather_cols(const Ctx& c, i64 rows, double* M, i64 ldm, const i64* pos, const i64* src, const i64* count,
                i64 max_moved, double* stage, i64 ldst) {
    if (rows <= 0 || max_moved <= 0) return 0;
    if (max_moved > 65535) {
        set_error("gather_cols: too many moved columns (%lld)", (long long)max_moved);
        return BQRRP_EUNSUPPORTED;
    }
    dim3 grid((unsigned)cdiv(rows, kMoveChunk), (unsigned)max_moved);
    const int vec = ((ldm | ldst) % 2 == 0) && ((uintptr_t)M % 16 == 0) && ((uintptr_t)stage % 16 == 0);
    move_cols_kernel<<<grid, 256, 0, c.stream>>>(rows, M, ldm, pos, src, count, stage, ldst, 0, vec);
    BQ_LAUNCH_CHECK();
    move_cols_kernel<<<grid, 256, 0, c.stream>>>(rows, M, ldm, pos, src, count, stage, ldst, 1, vec);
    BQ_LAUNCH_CHECK();
    return 0;
}

int gather_idx(const Ctx& c, i64* J, const i64* pos, const i64* src, const i64* count, i64 max_moved,
               i64* stage) {
    if (max_moved <= 0) return 0;
    const unsigned blocks = (unsigned)cdiv(max_moved, 256);
    move_idx_kernel<<<blocks, 256, 0, c.stream>>>(J, pos, src, count, max_moved, stage, 0);
    BQ_LAUNCH_CHECK();
    move_idx_kernel<<<blocks, 256, 0, c.stream>>>(J, pos, src, count, max_moved, stage, 1);
    BQ_LAUNCH_CHECK();
    return 0;
}

}  // namespace bq
