// dense.cu -- blocked FP64 triangular kernels built on the SIMT GEMM.
//
// Every O(b^3) step of the panel (Alg. 3) is cast as a right-looking blocked
// algorithm: a 64-wide diagonal block handled by one CTA in shared memory (or,
// for triangular solves, one warp per matrix row -- four rows per warp for tall
// blocks -- with the block in shared memory, rows spread over all SMs) plus
// GEMM updates.  With B300's slow FP64
// pipe a single SM runs at ~8 GFLOP/s, so nothing of size b^3 may stay on one
// SM.
#include <climits>

#include "common.cuh"

namespace bq {

namespace {

constexpr int NBD = 64;   // diagonal block size

// X <- X * R^{-1} for the nb (<= 64) columns of X; R upper (unit diagonal if
// unit != 0; then only the strictly upper part of R is read).
//
// The kernel factors R = D R' (D = diag(R), R' unit upper with R'(t, j) =
// R(t, j) / R(t, t)), solves y R' = x by forward substitution and returns
// x = y D^{-1}: the dependency chain then holds only FMAs, and the nb
// divisions happen once per CTA instead of once per row and column.  On
// B300 every FP64 instruction is slow (2 DFMA/clk/SM), so rows are spread
// over all SMs.
__device__ inline void load_unit_triangle(int nb, View R, int unit, double (*Rs)[NBD + 1], double* dinv) {
    for (int e = threadIdx.x; e < NBD; e += blockDim.x) dinv[e] = (e < nb && !unit) ? 1.0 / *R.at(e, e) : 1.0;
    __syncthreads();
    for (int e = threadIdx.x; e < NBD * NBD; e += blockDim.x) {
        const int t = e % NBD, j = e / NBD;
        Rs[t][j] = (t < j && j < nb) ? *R.at(t, j) * dinv[t] : 0.0;
    }
    __syncthreads();
}

// One warp per row: lane l holds columns l and l + 32; step j broadcasts y_j
// from its lane and the lanes of the later columns apply it (right-looking),
// so a row costs nb shuffle+FMA steps.  Rows are strided over a grid of at
// most a few CTAs per SM.  (Measured against one thread per row with the row
// in registers: faster at every height, as the warp form keeps many more
// warps in flight per SM.)
constexpr int kTrsmWarps = 4;
constexpr i64 kTrsmTall = 4096;   // rows from which four rows per warp pay (enough warps for every SMSP)
__global__ void __launch_bounds__(32 * kTrsmWarps) trsm_warp_kernel(i64 rows, int nb, View R, View X, int unit) {
    __shared__ double Rs[NBD][NBD + 1];
    __shared__ double dinv[NBD];
    load_unit_triangle(nb, R, unit, Rs, dinv);
    const int lane = threadIdx.x & 31;
    const i64 stride = (i64)gridDim.x * kTrsmWarps;
    for (i64 i = (i64)blockIdx.x * kTrsmWarps + (threadIdx.x >> 5); i < rows; i += stride) {
        double x0 = (lane < nb) ? *X.at(i, lane) : 0.0;
        double x1 = (lane + 32 < nb) ? *X.at(i, lane + 32) : 0.0;
        const int n0 = nb < 32 ? nb : 32;
        for (int j = 0; j < n0; ++j) {
            const double y = __shfl_sync(0xffffffffu, x0, j);
            if (lane > j) x0 = fma(-y, Rs[j][lane], x0);
            x1 = fma(-y, Rs[j][lane + 32], x1);
        }
        for (int j = 32; j < nb; ++j) {
            const double y = __shfl_sync(0xffffffffu, x1, j - 32);
            if (lane + 32 > j) x1 = fma(-y, Rs[j][lane + 32], x1);
        }
        if (lane < nb) *X.at(i, lane) = x0 * dinv[lane];
        if (lane + 32 < nb) *X.at(i, lane + 32) = x1 * dinv[lane + 32];
    }
}

// Four rows per warp for tall X, where throughput rather than latency
// bounds the solve: lane l serves row l / 8 and columns l % 8 + 8q (q < 8).
// Step j issues one FMA per column group still ahead of j, 8 - j/8 of them,
// 72 FP64 instructions per row against 96 for one row per warp.
__global__ void __launch_bounds__(32 * kTrsmWarps) trsm_warp4_kernel(i64 rows, int nb, View R, View X, int unit) {
    __shared__ double Rs[NBD][NBD + 1];
    __shared__ double dinv[NBD];
    load_unit_triangle(nb, R, unit, Rs, dinv);
    const int lane = threadIdx.x & 31, l8 = lane & 7, sub = lane >> 3;
    const i64 stride = (i64)gridDim.x * kTrsmWarps * 4;
    for (i64 i0 = ((i64)blockIdx.x * kTrsmWarps + (threadIdx.x >> 5)) * 4; i0 < rows; i0 += stride) {
        const i64 i = i0 + sub;
        const bool live = i < rows;
        double x[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) x[q] = (live && l8 + 8 * q < nb) ? *X.at(i, l8 + 8 * q) : 0.0;
#pragma unroll
        for (int j = 0; j < NBD; ++j) {
            if (j < nb) {
                const double y = __shfl_sync(0xffffffffu, x[j / 8], (lane & ~7) | (j & 7));
                if (l8 > (j & 7)) x[j / 8] = fma(-y, Rs[j][l8 + 8 * (j / 8)], x[j / 8]);
#pragma unroll
                for (int q = j / 8 + 1; q < 8; ++q) x[q] = fma(-y, Rs[j][l8 + 8 * q], x[q]);
            }
        }
        if (live) {
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (l8 + 8 * q < nb) *X.at(i, l8 + 8 * q) = x[q] * dinv[l8 + 8 * q];
        }
    }
}

// Element e of the upper triangle (c1 <= c2) of a w x w block, folded so
// that rows i and w-1-i share one row of length w+1: consecutive e cover
// consecutive c2, and no lane is masked off in the middle of the range.
__device__ inline bool upper_pair(int e, int w, int* c1, int* c2) {
    const int i = e / (w + 1), k = e - i * (w + 1);
    if (k < w - i) { *c1 = i; *c2 = i + k; return true; }
    const int i2 = w - 1 - i;
    if (i2 == i) return false;   // middle row of an odd w: already covered
    *c1 = i2;
    *c2 = i2 + (k - (w - i));
    return true;
}

// Upper Cholesky of one nb x nb diagonal block in place (G = R^T R), reading
// and writing only the upper triangle; zeroes the strict lower triangle.  A
// non-positive or non-finite pivot at local column j records jg0 + j in
// st->potrf_info (atomicMin) and stops.
//
// B300 cost model: an FP64 instruction holds an SM sub-partition's FP64 unit
// for ~64 cycles whatever the active lanes, a square root or a division
// ~650.  So the pivot test is an integer test on the bits, r_jj = d_jj *
// rsqrt(d_jj) and the row is scaled by that reciprocal (one special function
// per step instead of a square root plus a division), and the symmetric
// update touches only the upper triangle through the folded enumeration.
__global__ void __launch_bounds__(256) potrf_small_kernel(int nb, double* G, i64 ldg, int jg0, DevStatus* st) {
    __shared__ double A[NBD][NBD + 1];
    __shared__ double s_rinv;
    __shared__ int fail;
    for (int e = threadIdx.x; e < NBD * NBD; e += blockDim.x) {
        const int i = e % NBD, j = e / NBD;
        A[i][j] = (i < nb && j < nb && i <= j) ? G[i + (i64)j * ldg] : 0.0;
    }
    if (threadIdx.x == 0) fail = (st->potrf_info < jg0) ? 1 : 0;   // an earlier block failed
    __syncthreads();
    if (fail) return;
    for (int j = 0; j < nb; ++j) {
        if (threadIdx.x == 0) {
            const double dj = A[j][j];
            const long long bits = __double_as_longlong(dj);
            if (!(bits > 0 && bits < 0x7ff0000000000000ll)) {   // not (finite and > 0)
                fail = 1;
                atomicMin(&st->potrf_info, jg0 + j);
            } else {
                const double ri = rsqrt(dj);
                A[j][j] = dj * ri;
                s_rinv = ri;
            }
        }
        __syncthreads();
        if (fail) break;
        const double ri = s_rinv;
        for (int c = j + 1 + threadIdx.x; c < nb; c += blockDim.x) A[j][c] *= ri;
        __syncthreads();
        const int w = nb - j - 1, np = (w + 1) / 2 * (w + 1);
        for (int e = threadIdx.x; e < np; e += blockDim.x) {
            int c1, c2;
            if (upper_pair(e, w, &c1, &c2)) {
                c1 += j + 1;
                c2 += j + 1;
                A[c1][c2] = fma(-A[j][c1], A[j][c2], A[c1][c2]);
            }
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        const int i = e % nb, j = e / nb;
        G[i + (i64)j * ldg] = (i <= j) ? A[i][j] : 0.0;
    }
}

// Modified LU (Householder reconstruction, BD2015 Alg. 5 as cited in Sec. 2.3)
// of one nb x nb diagonal block in place: for each column j the sign
// s_j = -sign(a_jj) (sign(0) = +1) is recorded in D[j], a_jj -= s_j, then the
// column below is scaled by 1/a_jj and the block's trailing part gets the
// rank-1 update.  No pivoting.  Lookahead: thread 0 forms the next pivot
// (its one entry of the update, the sign and the reciprocal, ~700 cycles of
// FP64 latency) while warps 1.. update the rest of the block.
__global__ void __launch_bounds__(256) modlu_small_kernel(int nb, double* Y, i64 ldy, double* D) {
    __shared__ double A[NBD][NBD + 1];
    __shared__ double s_rp;
    for (int e = threadIdx.x; e < NBD * NBD; e += blockDim.x) {
        const int i = e % NBD, j = e / NBD;
        A[i][j] = (i < nb && j < nb) ? Y[i + (i64)j * ldy] : 0.0;
    }
    __syncthreads();
    // pivot of column jj from its (fully updated) diagonal entry: sign, shift, reciprocal
    auto pivot = [&](int jj) {
        const double a = A[jj][jj];
        const long long bits = __double_as_longlong(a);
        const double s = (bits >= 0 || bits == (long long)0x8000000000000000ull) ? -1.0 : 1.0;   // a >= 0
        D[jj] = s;
        const double piv = a - s;
        A[jj][jj] = piv;
        s_rp = 1.0 / piv;
    };
    if (threadIdx.x == 0 && nb > 0) pivot(0);
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        const double rp = s_rp;
        for (int i = j + 1 + threadIdx.x; i < nb; i += blockDim.x) A[i][j] *= rp;
        __syncthreads();
        const int w = nb - j - 1;
        if (threadIdx.x < 32) {
            // warp 0 does only the pivot (its other lanes idle): a lane of a warp
            // that also ran update FMAs would serialize with them
            if (threadIdx.x == 0 && w > 0) {
                A[j + 1][j + 1] = fma(-A[j + 1][j], A[j][j + 1], A[j + 1][j + 1]);
                pivot(j + 1);
            }
        } else {
            for (int e = threadIdx.x - 32; e < w * w; e += blockDim.x - 32) {
                if (e == 0) continue;   // (j+1, j+1): the pivot warp's
                const int i = j + 1 + e % w, c = j + 1 + e / w;
                A[i][c] = fma(-A[i][j], A[j][c], A[i][c]);
            }
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        const int i = e % nb, j = e / nb;
        Y[i + (i64)j * ldy] = A[i][j];
    }
}

__global__ void copy_kernel(i64 rows, i64 cols, const double* __restrict__ s, i64 lds, double* __restrict__ d,
                            i64 ldd, int triu) {
    const i64 total = rows * cols;
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (i64)gridDim.x * blockDim.x) {
        const i64 i = e % rows, j = e / rows;
        d[i + j * ldd] = (triu && i > j) ? 0.0 : s[i + j * lds];
    }
}

__global__ void zero_below_kernel(i64 rows, i64 cols, double* A, i64 lda) {
    const i64 total = rows * cols;
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (i64)gridDim.x * blockDim.x) {
        const i64 i = e % rows, j = e / rows;
        if (i > j) A[i + j * lda] = 0.0;
    }
}

__global__ void nonfinite_kernel(i64 rows, i64 cols, const double* __restrict__ A, i64 lda, int* flag) {
    const i64 total = rows * cols;
    int bad = 0;
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (i64)gridDim.x * blockDim.x) {
        const i64 i = e % rows, j = e / rows;
        if (!isfinite(A[i + j * lda])) bad = 1;
    }
    bad = __syncthreads_or(bad);
    if (bad && threadIdx.x == 0) atomicOr(flag, 1);
}

inline int grid_for(const Ctx& c, i64 total) {
    return (int)imax(1, imin(cdiv(total, 256), 16LL * c.dev.sms));
}

}  // namespace

int trsm_ru(const Ctx& c, i64 rows, i64 k, View R, View X, bool unit) {
    if (rows <= 0 || k <= 0) return 0;
    for (i64 jb = 0; jb < k; jb += NBD) {
        const int nb = (int)imin(NBD, k - jb);
        if (rows >= kTrsmTall) {
            const i64 grid = imin(cdiv(rows, 4 * kTrsmWarps), 6LL * c.dev.sms);
            trsm_warp4_kernel<<<(unsigned)grid, 32 * kTrsmWarps, 0, c.stream>>>(rows, nb, R.sub(jb, jb),
                                                                              X.sub(0, jb), unit ? 1 : 0);
        } else {
            const i64 grid = imin(cdiv(rows, kTrsmWarps), 6LL * c.dev.sms);
            trsm_warp_kernel<<<(unsigned)grid, 32 * kTrsmWarps, 0, c.stream>>>(rows, nb, R.sub(jb, jb),
                                                                             X.sub(0, jb), unit ? 1 : 0);
        }
        BQ_LAUNCH_CHECK();
        if (jb + nb < k) {
            // X(:, jb+nb:k) -= X(:, jb:jb+nb) * R(jb:jb+nb, jb+nb:k)
            BQ_TRY(gemm_view(c, rows, k - jb - nb, nb, -1.0, X.sub(0, jb), R.sub(jb, jb + nb), 1.0,
                             X.sub(0, jb + nb)));
        }
    }
    return 0;
}

int potrf_u(const Ctx& c, i64 k, double* G, i64 ldg) {
    View Gv = colmajor(G, ldg);
    for (i64 jb = 0; jb < k; jb += NBD) {
        const int nb = (int)imin(NBD, k - jb);
        potrf_small_kernel<<<1, 256, 0, c.stream>>>(nb, G + jb + jb * ldg, ldg, (int)jb, c.st);
        BQ_LAUNCH_CHECK();
        const i64 rest = k - jb - nb;
        if (rest > 0) {
            // R12 = R11^{-T} G12  <=>  R12^T = G12^T R11^{-1}
            BQ_TRY(trsm_ru(c, rest, nb, Gv.sub(jb, jb), Gv.sub(jb, jb + nb).t(), false));
            // G22 -= R12^T R12
            BQ_TRY(dgemm(c, true, false, rest, rest, nb, -1.0, G + jb + (jb + nb) * ldg, ldg,
                         G + jb + (jb + nb) * ldg, ldg, 1.0, G + (jb + nb) + (jb + nb) * ldg, ldg));
        }
    }
    return set_zero_below(c, k, k, G, ldg);
}

int modlu(const Ctx& c, i64 rows, i64 k, double* Y, i64 ldy, double* D) {
    View Yv = colmajor(Y, ldy);
    for (i64 jb = 0; jb < k; jb += NBD) {
        const int nb = (int)imin(NBD, k - jb);
        modlu_small_kernel<<<1, 256, 0, c.stream>>>(nb, Y + jb + jb * ldy, ldy, D + jb);
        BQ_LAUNCH_CHECK();
        const i64 below = rows - jb - nb;
        if (below > 0)   // L21 = A21 U11^{-1}
            BQ_TRY(trsm_ru(c, below, nb, Yv.sub(jb, jb), Yv.sub(jb + nb, jb), false));
        const i64 right = k - jb - nb;
        if (right > 0) {
            // U12 = L11^{-1} A12  <=>  U12^T = A12^T L11^{-T}, L11^T unit upper
            BQ_TRY(trsm_ru(c, right, nb, Yv.sub(jb, jb).t(), Yv.sub(jb, jb + nb).t(), true));
            if (below > 0)   // A22 -= L21 U12
                BQ_TRY(dgemm(c, false, false, below, right, nb, -1.0, Y + (jb + nb) + jb * ldy, ldy,
                             Y + jb + (jb + nb) * ldy, ldy, 1.0, Y + (jb + nb) + (jb + nb) * ldy, ldy));
        }
    }
    return 0;
}

int copy_mat(const Ctx& c, i64 rows, i64 cols, const double* src, i64 lds, double* dst, i64 ldd) {
    if (rows <= 0 || cols <= 0) return 0;
    copy_kernel<<<grid_for(c, rows * cols), 256, 0, c.stream>>>(rows, cols, src, lds, dst, ldd, 0);
    BQ_LAUNCH_CHECK();
    return 0;
}

int copy_triu(const Ctx& c, i64 rows, i64 cols, const double* src, i64 lds, double* dst, i64 ldd) {
    if (rows <= 0 || cols <= 0) return 0;
    copy_kernel<<<grid_for(c, rows * cols), 256, 0, c.stream>>>(rows, cols, src, lds, dst, ldd, 1);
    BQ_LAUNCH_CHECK();
    return 0;
}

int set_zero_below(const Ctx& c, i64 rows, i64 cols, double* A, i64 lda) {
    if (rows <= 1 || cols <= 0) return 0;
    zero_below_kernel<<<grid_for(c, rows * cols), 256, 0, c.stream>>>(rows, cols, A, lda);
    BQ_LAUNCH_CHECK();
    return 0;
}

int any_nonfinite(const Ctx& c, i64 rows, i64 cols, const double* A, i64 lda, int* flag) {
    if (rows <= 0 || cols <= 0) return 0;
    nonfinite_kernel<<<grid_for(c, rows * cols), 256, 0, c.stream>>>(rows, cols, A, lda, flag);
    BQ_LAUNCH_CHECK();
    return 0;
}

}  // namespace bq
