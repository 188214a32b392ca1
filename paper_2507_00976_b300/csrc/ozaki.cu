// ozaki.cu -- FP64-accurate GEMM on the bf16 tensor cores (error-free
// splitting, in the manner of the Ozaki scheme).
//
// B300 executes FP64 at ~1.2 TFLOP/s while its bf16 tensor cores run at
// ~1.4 PFLOP/s (tcgen05, sustained).  A product of FP64 matrices can be formed
// exactly from integer slices:
//   * every row i of op(A) is scaled by 2^-ea_i and every column j of op(B) by
//     2^-eb_j (ea_i, eb_j = exponent just above the row / column maximum);
//   * the scaled value x is truncated to a 54-bit fixed-point integer X with
//     integer bit operations, and X is written in seven balanced base-256
//     digits q_0 .. q_6 in [-128, 127] (exact in bf16):
//     x ~ 2^(e - 54) sum_p q_p 2^(8 (6 - p));
//   * op(A) op(B) ~ 2^(ea_i + eb_j - 60) sum_{t <= 6} 2^(8 (6 - t)) G_t with
//     G_t = sum_{p + q = t} A_p B_q: the 28 slice products with p + q <= 6; the
//     dropped pairs and the truncation together stay below about 2^-53 of
//     max|row| * max|column| per term (FP64's own unit roundoff is 2^-53);
//   * the products of one group t are summed on the tensor cores in FP32.
//     Every partial sum is an integer of magnitude at most 7 * Kc * 128^2 <
//     2^24 for a K chunk Kc = 128, so FP32 holds it exactly; after each chunk
//     the seven group sums are combined exactly, rounded to a multiple of
//     2^dsh (dsh = max(ceil(log2 K) - 2, 8)) and added into one 64-bit integer per
//     element (ozaki_tc.cu), which is rounded once to FP64 at the end.
// Balanced digits halve the largest slice magnitude of unsigned 8-bit ones,
// which is what lets eight bits per slice keep a 128-deep exact chunk.  The
// result matches an FP64 GEMM to a few units of roundoff (normwise).  A sketch
// with +-1 entries is exact in one slice, so S*A needs only the seven products
// S A_q.
#include <cuda_bf16.h>

#include "common.cuh"

namespace bq {

namespace {

constexpr int kSlices = kOzPlanes;   // balanced 8-bit slices per FP64 operand (54-bit fixed point)
constexpr int OBM = 64, OBN = 32, OBK = 32;   // padding of the slice planes (rows, rows, k)

__device__ __forceinline__ int exp_above(double m) {
    // smallest e with m < 2^e (m >= 0); 0 for m == 0
    if (!(m > 0.0)) return 0;
    int e;
    frexp(m, &e);
    return e;
}

// x (|x| < 2^e) -> 54-bit fixed point X = trunc(x 2^(54-e)) using integer ops.
__device__ __forceinline__ long long fixed54(double x, int e) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)((bits >> 52) & 0x7FF);
    if (ex == 0) return 0;   // zero (subnormals are far below every slice)
    const long long mant = (long long)((bits & 0xFFFFFFFFFFFFFull) | (1ull << 52));
    const int sh = ex - 1075 + 54 - e;   // <= 1 because |x| < 2^e
    long long X;
    if (sh >= 0) X = mant << sh;
    else if (sh > -63) X = mant >> (-sh);
    else X = 0;
    return (bits >> 63) ? -X : X;
}

// |v| as its bit pattern, which orders like the value for non-negative
// doubles; NaN counts as 0 (as fmax would ignore it).  The maxima are taken
// on these integers: FP64 min/max runs at the FP64 pipe's rate on this part,
// integer compares at the full ALU rate.
__device__ __forceinline__ unsigned long long abs_bits(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
    return b > 0x7FF0000000000000ull ? 0ull : b;
}

// Row maxima exponents of op(A) (M rows, K columns).  trans: op(A)(i,k) =
// A[k + i*lda], a row is contiguous and one warp takes it; else op(A)(i,k) =
// A[i + k*lda], 32 consecutive rows per block (one per lane, so every warp
// load is 32 consecutive doubles) with the eight warps splitting K.  Four
// independent maxima per thread keep several loads in flight.
constexpr int kRowExpThreads = 256;
__global__ void __launch_bounds__(kRowExpThreads) row_exp_kernel(i64 M, i64 K, const double* __restrict__ A,
                                                                 i64 lda, int trans, int* __restrict__ e) {
    typedef unsigned long long u64;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    u64 m0 = 0, m1 = 0, m2 = 0, m3 = 0;
    if (trans) {
        const i64 i = (i64)blockIdx.x * 8 + warp;
        if (i >= M) return;
        const double* row = A + i * lda;
        i64 k = lane;
        for (; k + 96 < K; k += 128) {
            m0 = max(m0, abs_bits(row[k]));
            m1 = max(m1, abs_bits(row[k + 32]));
            m2 = max(m2, abs_bits(row[k + 64]));
            m3 = max(m3, abs_bits(row[k + 96]));
        }
        for (; k < K; k += 32) m0 = max(m0, abs_bits(row[k]));
        u64 mx = max(max(m0, m1), max(m2, m3));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_down_sync(0xffffffffu, mx, o));
        if (lane == 0) e[i] = exp_above(__longlong_as_double((long long)mx));
        return;
    }
    __shared__ u64 part[8][32];
    const i64 i = (i64)blockIdx.x * 32 + lane;
    if (i < M) {
        const double* col = A + i;
        i64 k = warp;
        for (; k + 24 < K; k += 32) {
            m0 = max(m0, abs_bits(col[k * lda]));
            m1 = max(m1, abs_bits(col[(k + 8) * lda]));
            m2 = max(m2, abs_bits(col[(k + 16) * lda]));
            m3 = max(m3, abs_bits(col[(k + 24) * lda]));
        }
        for (; k < K; k += 8) m0 = max(m0, abs_bits(col[k * lda]));
    }
    part[warp][lane] = max(max(m0, m1), max(m2, m3));
    __syncthreads();
    if (warp == 0 && i < M) {
        u64 mx = part[0][lane];
#pragma unroll
        for (int w = 1; w < 8; ++w) mx = max(mx, part[w][lane]);
        e[i] = exp_above(__longlong_as_double((long long)mx));
    }
}

// Blocks of row_exp_kernel for M rows.
inline unsigned row_exp_blocks(i64 M, int trans) { return (unsigned)(trans ? (M + 7) / 8 : (M + 31) / 32); }

// Bias that turns balanced base-256 digits into bytes: for |X| < 2^54 the
// seven digits q_p in [-128, 127] (X = sum_p q_p 2^(8 (6 - p))) are the bytes
// of X + sum_p 128 2^(8p), each minus 128 (the sum of digits plus 128 is the
// plain base-256 representation of the biased value, which lies in
// (2^54, 2^56)).
constexpr long long kDigitBias = 0x80808080808080LL;

// FP32 bit pattern of the integer b - 128, b = byte j (0..3) of w: one byte
// permute forms 0x4B000000 | b, the FP32 pattern of 2^23 + b (exact), and the
// subtraction of 2^23 + 128 is exact.  Its upper 16 bits are the bf16 of
// b - 128 (8 significant bits).
__device__ __forceinline__ uint32_t digit_f32(uint32_t w, int j) {
    return __float_as_uint(__uint_as_float(__byte_perm(w, 0x4Bu, 0x4650u | (uint32_t)j)) - 8388736.0f);
}

// Split op(X) (R rows x K columns, row r scaled by 2^-e[r]) into kSlices bf16
// slices S[p][r][k] (row length ldk >= K, rows padded to Rp with zeros, k
// padded to ldk with zeros).  trans: op(X)(r,k) = X[k + r*ldx] (k contiguous),
// else op(X)(r,k) = X[r + k*ldx] (r contiguous; staged through shared memory).
// Each thread writes two adjacent k of one row as one 32-bit word per plane.
__global__ void __launch_bounds__(256) split_kernel(i64 R, i64 K, i64 Rp, i64 ldk, const double* X, i64 ldx,
                                                    int trans, const int* e, __nv_bfloat16* S) {
    __shared__ double tile[32][33];
    const i64 r0 = (i64)blockIdx.y * 32, k0 = (i64)blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
    if (!trans) {
        // load a 32 x 32 tile of op(X) as tile[r][k] (r contiguous in memory)
        for (int q = ty; q < 32; q += 8) {
            const i64 r = r0 + tx, k = k0 + q;
            tile[tx][q] = (r < R && k < K) ? X[r + k * ldx] : 0.0;
        }
        __syncthreads();
    }
    const size_t slice = (size_t)Rp * (size_t)ldk;
    const int kp = 2 * (threadIdx.x & 15);   // k pair within the tile
    for (int q = threadIdx.x >> 4; q < 32; q += 16) {
        const i64 r = r0 + q, k = k0 + kp;
        if (r >= Rp || k >= ldk) continue;   // ldk is even, so k + 1 < ldk too
        const int er = r < R ? e[r] : 0;
        // k contiguous in memory: the two values straight from global memory
        // (16 lanes read 32 consecutive doubles), no staging
        const double x0 = trans ? ((r < R && k < K) ? X[k + r * ldx] : 0.0) : tile[q][kp];
        const double x1 = trans ? ((r < R && k + 1 < K) ? X[k + 1 + r * ldx] : 0.0) : tile[q][kp + 1];
        const long long X0 = (r < R && k < K) ? fixed54(x0, er) : 0;
        const long long X1 = (r < R && k + 1 < K) ? fixed54(x1, er) : 0;
        const unsigned long long Z0 = (unsigned long long)(X0 + kDigitBias);
        const unsigned long long Z1 = (unsigned long long)(X1 + kDigitBias);
        const uint32_t w0[2] = {(uint32_t)Z0, (uint32_t)(Z0 >> 32)}, w1[2] = {(uint32_t)Z1, (uint32_t)(Z1 >> 32)};
        uint32_t* out = reinterpret_cast<uint32_t*>(S + (size_t)r * ldk + k);
#pragma unroll
        for (int p = 0; p < kSlices; ++p) {
            const int j = kSlices - 1 - p;   // byte of Z: plane 0 holds the most significant digit
            // low half: the bf16 of element k, high half: of element k + 1
            out[(size_t)p * (slice / 2)] =
                __byte_perm(digit_f32(w0[j >> 2], j & 3), digit_f32(w1[j >> 2], j & 3), 0x7632);
        }
    }
}

// The dense +-1 sketch operator as one exact bf16 slice, rows padded.
__global__ void sketch_slice_kernel(i64 d, i64 m, i64 Rp, i64 ldk, uint64_t seed, __nv_bfloat16* S) {
    const i64 total = Rp * ldk;
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (i64)gridDim.x * blockDim.x) {
        const i64 r = e / ldk, k = e % ldk;
        float v = 0.f;
        if (r < d && k < m) v = (float)sketch_dense_entry(seed, r, k);
        S[e] = __float2bfloat16_rn(v);
    }
}

inline i64 rup(i64 x, i64 m) { return (x + m - 1) / m * m; }

__global__ void fill_int_kernel(int* x, i64 n, int v) {
    const i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = v;
}

// After a launch on a context without a status block: read the kernel's
// timeout flag (one synchronization) and report it.
int check_flag(const Ctx& c, int* flag) {
    if (c.st) return 0;
    int h = 0;
    BQ_CUDA(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    BQ_CUDA(cudaStreamSynchronize(c.stream));
    if (h) { set_error("tensor-core slice GEMM: a pipeline wait timed out"); return BQRRP_ETIMEOUT; }
    return 0;
}

}  // namespace

int ozaki_tc_gemm(const Ctx& c, const __nv_bfloat16* As, i64 Mp, const __nv_bfloat16* Bs, i64 Np, i64 ldk, i64 M,
                  i64 N, const int* ea, const int* eb, double alpha, double beta, double* C, i64 ldc, int* err,
                  unsigned long long* acc64);
int ozaki_tc_sketch(const Ctx& c, const __nv_bfloat16* Ss, i64 Mp, const __nv_bfloat16* Bs, i64 Np, i64 ldk, i64 M,
                    i64 N, const int* ea, const int* eb, double* C, i64 ldc, int* err);

// Products of at most this many 128 x 64 tiles may split K over the SMs
// (half of B300's 148; a GPU with more SMs splits only when the workspace
// holds the integer sums).
constexpr i64 kSplitMaxTiles = 74;

bool ozaki_may_split(i64 M, i64 N) { return cdiv(imax(M, 1), 128) * cdiv(imax(N, 1), 64) <= kSplitMaxTiles; }

size_t ozaki_split_reserve() { return sizeof(unsigned long long) * (size_t)(kSplitMaxTiles * 128 * 64) + 256; }

// Workspace (bytes) for ozaki_gemm / ozaki_sketch on these sizes: the slice
// planes, the exponents, and for a product that may split K its M x N
// integer sums.
size_t ozaki_ws_bytes(i64 M, i64 N, i64 K, int sa) {
    const i64 Mp = rup(imax(M, 1), OBM), Np = rup(imax(N, 1), OBN), Kp = rup(imax(K, 1), OBK);
    size_t z = ((size_t)sa * Mp * Kp + (size_t)kSlices * Np * Kp) * sizeof(__nv_bfloat16) +
               (size_t)(Mp + Np) * sizeof(int) + 2048;
    if (sa == kSlices && ozaki_may_split(M, N)) z += sizeof(unsigned long long) * (size_t)(imax(M, 1) * imax(N, 1)) + 256;
    return z;
}

// C = alpha op(A) op(B) + beta C, FP64 in and out, products on the bf16 tensor cores.
int ozaki_gemm(const Ctx& c, bool ta, bool tb, i64 M, i64 N, i64 K, double alpha, const double* A, i64 lda,
               const double* B, i64 ldb, double beta, double* C, i64 ldc, void* ws, size_t ws_bytes) {
    if (M <= 0 || N <= 0) return 0;
    if (K <= 0) return dgemm(c, ta, tb, M, N, 0, alpha, A, lda, B, ldb, beta, C, ldc);
    const i64 Mp = rup(M, OBM), Np = rup(N, OBN), Kp = rup(K, OBK);
    if (ws_bytes < ozaki_ws_bytes(M, N, K, kSlices)) { set_error("ozaki_gemm: workspace too small"); return BQRRP_ENOMEM; }
    Arena ar;
    ar.base = (char*)ws;
    ar.cap = ws_bytes;
    __nv_bfloat16* As = ar.take<__nv_bfloat16>((size_t)kSlices * Mp * Kp);
    __nv_bfloat16* Bs = ar.take<__nv_bfloat16>((size_t)kSlices * Np * Kp);
    int* ea = ar.take<int>((size_t)Mp);
    int* eb = ar.take<int>((size_t)Np);
    int* flag = ar.take<int>(1);
    unsigned long long* acc64 = nullptr;
    if (ozaki_may_split(M, N) || ar.off + sizeof(unsigned long long) * (size_t)(M * N) + 256 <= ar.cap)
        acc64 = ar.take<unsigned long long>((size_t)(M * N));
    if (!ar.ok()) { set_error("ozaki_gemm: workspace too small"); return BQRRP_ENOMEM; }
    // exponents: rows of op(A), columns of op(B) (= rows of op(B)^T)
    row_exp_kernel<<<row_exp_blocks(M, ta ? 1 : 0), kRowExpThreads, 0, c.stream>>>(M, K, A, lda, ta ? 1 : 0, ea);
    BQ_LAUNCH_CHECK();
    row_exp_kernel<<<row_exp_blocks(N, tb ? 0 : 1), kRowExpThreads, 0, c.stream>>>(N, K, B, ldb, tb ? 0 : 1, eb);
    BQ_LAUNCH_CHECK();
    // slices: op(A) rows x K, op(B)^T rows (= N) x K
    split_kernel<<<dim3((unsigned)(Kp / 32), (unsigned)(Mp / 32)), 256, 0, c.stream>>>(M, K, Mp, Kp, A, lda,
                                                                                      ta ? 1 : 0, ea, As);
    BQ_LAUNCH_CHECK();
    split_kernel<<<dim3((unsigned)(Kp / 32), (unsigned)(Np / 32)), 256, 0, c.stream>>>(N, K, Np, Kp, B, ldb,
                                                                                      tb ? 0 : 1, eb, Bs);
    BQ_LAUNCH_CHECK();
    int* err = c.st ? &c.st->err_timeout : flag;
    if (!c.st) BQ_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), c.stream));
    BQ_TRY(ozaki_tc_gemm(c, As, Mp, Bs, Np, Kp, M, N, ea, eb, alpha, beta, C, ldc, err, acc64));
    return check_flag(c, flag);
}

int pgemm(const Ctx& c, bool ta, bool tb, i64 M, i64 N, i64 K, double alpha, const double* A, i64 lda,
          const double* B, i64 ldb, double beta, double* C, i64 ldc, int flags) {
    if (c.mixed && c.oz_ws && M > 0 && N > 0 && K >= 32 && (double)M * N * K >= 16.0 * 1024 * 1024 &&
        ozaki_ws_bytes(M, N, K, kSlices) <= c.oz_bytes)
        return ozaki_gemm(c, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, c.oz_ws, c.oz_bytes);
    return dgemm(c, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, flags);
}

// Right-looking blocked solve: each 64-column block of X is solved against
// its diagonal block of R in FP64 (trsm_ru), then removed from the columns to
// its right with one product.  In the mixed form those products (three
// quarters of the solve's work for k = 256) run on the tensor cores; with the
// FP64 form, or when X is short, this is trsm_ru itself.
int trsm_ru_tall(const Ctx& c, i64 rows, i64 k, const double* R, i64 ldr, double* X, i64 ldx) {
    constexpr i64 kBlk = 64;
    if (!c.mixed || !c.oz_ws || rows < 2048 || k <= kBlk)
        return trsm_ru(c, rows, k, colmajor(R, ldr), colmajor(X, ldx), false);
    for (i64 jb = 0; jb < k; jb += kBlk) {
        const i64 nb = imin(kBlk, k - jb);
        BQ_TRY(trsm_ru(c, rows, nb, colmajor(R + jb + jb * ldr, ldr), colmajor(X + jb * ldx, ldx), false));
        if (jb + nb < k)   // X(:, jb+nb:k) -= X(:, jb:jb+nb) R(jb:jb+nb, jb+nb:k)
            BQ_TRY(pgemm(c, false, false, rows, k - jb - nb, nb, -1.0, X + jb * ldx, ldx, R + jb + (jb + nb) * ldr,
                         ldr, 1.0, X + (jb + nb) * ldx, ldx));
    }
    return 0;
}

// Columns of A sliced at a time by ozaki_sketch (the slice planes of a block
// take 16 bytes per element; 8192 columns give the sketch GEMM enough tiles).
constexpr i64 kSketchCols = 8192;

size_t ozaki_sketch_ws_bytes(i64 d, i64 m, i64 n) { return ozaki_ws_bytes(d, imin(imax(n, 1), kSketchCols), m, 1); }

// Msk = S A with the dense +-1 operator S (d x m) as one exact slice:
// seven tensor-core products S A_q; FP32 sums of |+-1 * q| <= 128 over 2^17
// columns stay below 2^24, so one exact flush per 2^17 columns suffices.  A
// is sliced and multiplied kSketchCols columns at a time (every column of Msk
// depends only on its own column of A, so the blocking changes no bit).
int ozaki_sketch(const Ctx& c, i64 d, i64 m, i64 n, uint64_t seed, const double* A, i64 lda, double* Msk, i64 ldsk,
                 void* ws, size_t ws_bytes) {
    if (d <= 0 || n <= 0) return 0;
    const i64 nb = imin(n, kSketchCols);
    const i64 Mp = rup(d, OBM), Np = rup(nb, OBN), Kp = rup(imax(m, 1), OBK);
    if (ws_bytes < ozaki_sketch_ws_bytes(d, m, n)) { set_error("ozaki_sketch: workspace too small"); return BQRRP_ENOMEM; }
    Arena ar;
    ar.base = (char*)ws;
    ar.cap = ws_bytes;
    __nv_bfloat16* Ss = ar.take<__nv_bfloat16>((size_t)Mp * Kp);
    __nv_bfloat16* Bs = ar.take<__nv_bfloat16>((size_t)kSlices * Np * Kp);
    int* ea = ar.take<int>((size_t)Mp);
    int* eb = ar.take<int>((size_t)Np);
    int* flag = ar.take<int>(1);
    if (!ar.ok()) { set_error("ozaki_sketch: workspace too small"); return BQRRP_ENOMEM; }
    const unsigned blocks = (unsigned)imax(1, imin(cdiv(Mp * Kp, 256), 16LL * c.dev.sms));
    sketch_slice_kernel<<<blocks, 256, 0, c.stream>>>(d, m, Mp, Kp, seed, Ss);
    BQ_LAUNCH_CHECK();
    // S has one slice q_0 = +-1 with weight 2^(ea - 54 + 48) = 1: ea = 6 on every row
    fill_int_kernel<<<(unsigned)cdiv(Mp, 256), 256, 0, c.stream>>>(ea, Mp, 6);
    BQ_LAUNCH_CHECK();
    int* err = c.st ? &c.st->err_timeout : flag;
    if (!c.st) BQ_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), c.stream));
    for (i64 j0 = 0; j0 < n; j0 += nb) {
        const i64 nj = imin(nb, n - j0), Npj = rup(nj, OBN);
        const double* Aj = A + j0 * lda;
        row_exp_kernel<<<row_exp_blocks(nj, 1), kRowExpThreads, 0, c.stream>>>(nj, m, Aj, lda, 1, eb);
        BQ_LAUNCH_CHECK();
        split_kernel<<<dim3((unsigned)(Kp / 32), (unsigned)(Npj / 32)), 256, 0, c.stream>>>(nj, m, Npj, Kp, Aj, lda, 1,
                                                                                           eb, Bs);
        BQ_LAUNCH_CHECK();
        BQ_TRY(ozaki_tc_sketch(c, Ss, Mp, Bs, Npj, Kp, d, nj, ea, eb, Msk + j0 * ldsk, ldsk, err));
    }
    return check_flag(c, flag);
}

}  // namespace bq
