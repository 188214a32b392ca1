// ozaki.cu -- FP64-accurate GEMM on the bf16 tensor cores (error-free
// splitting, in the manner of the Ozaki scheme).
//
// B300 executes FP64 at ~1.2 TFLOP/s while its bf16 tensor cores run
// mma.sync at ~570 TFLOP/s.  A product of FP64 matrices can be formed exactly
// from integer slices:
//   * every row i of op(A) is scaled by 2^-ea_i and every column j of op(B) by
//     2^-eb_j (ea_i, eb_j = exponent just above the row / column maximum);
//   * the scaled value x is truncated to a 54-bit fixed-point integer X with
//     integer bit operations, and X is cut into nine signed 6-bit slices
//     q_0 .. q_8 (|q| <= 63, exact in bf16):  x ~ sum_p q_p 2^(e - 6 - 6p);
//   * op(A) op(B) ~ sum_{p+q <= 9} 2^(ea_i + eb_j - 12 - 6(p+q)) (A_p B_q):
//     the 53 slice products with p + q <= 9 keep everything above 2^-54 of
//     max|row| * max|column| per term (FP64's own unit roundoff is 2^-53);
//   * the products of one group t = p + q are summed on the tensor cores in
//     FP32.  Every partial sum is an integer of magnitude below
//     (t+1) * Kc * 63^2 < 2^24 for a K chunk Kc = 256, so FP32 holds it
//     exactly; after each chunk the ten group sums are added into FP64 with
//     weights 2^-6t.
// The result matches an FP64 GEMM to a few units of roundoff (normwise).  A
// sketch with +-1 entries is exact in one slice, so S*A needs only the nine
// products S A_q.
#include <cuda_bf16.h>

#include <cstdlib>

#include <mutex>

#include "common.cuh"

namespace bq {

namespace {

constexpr int kSlices = 9;     // 6-bit slices per FP64 operand (54 bits)
constexpr int kTmax = 9;       // keep slice pairs with p + q <= kTmax
constexpr int OBM = 64, OBN = 32, OBK = 32;
constexpr int OPAD = 40;       // smem row length (bf16) of a 32-deep k tile: 80 bytes
constexpr int ONT = 256;

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

// Row maxima exponents of op(A) (M rows, K columns); trans: op(A)(i,k) = A[k + i*lda].
__global__ void row_exp_kernel(i64 M, i64 K, const double* A, i64 lda, int trans, int* e) {
    const i64 i = (i64)blockIdx.x;
    double mx = 0.0;
    for (i64 k = threadIdx.x; k < K; k += blockDim.x) {
        const double v = trans ? A[k + i * lda] : A[i + k * lda];
        mx = fmax(mx, fabs(v));
    }
    __shared__ double red[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x < 32) {
        mx = (threadIdx.x < blockDim.x / 32) ? red[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
        if (threadIdx.x == 0) e[i] = exp_above(mx);
    }
}

// Split op(X) (R rows x K columns, row r scaled by 2^-e[r]) into kSlices bf16
// slices S[p][r][k] (row length ldk >= K, rows padded to Rp with zeros, k
// padded to ldk with zeros).  trans: op(X)(r,k) = X[k + r*ldx] (k contiguous),
// else op(X)(r,k) = X[r + k*ldx] (r contiguous; staged through shared memory).
__global__ void __launch_bounds__(256) split_kernel(i64 R, i64 K, i64 Rp, i64 ldk, const double* X, i64 ldx,
                                                    int trans, const int* e, __nv_bfloat16* S) {
    __shared__ double tile[32][33];
    const i64 r0 = (i64)blockIdx.y * 32, k0 = (i64)blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
    // load a 32 x 32 tile of op(X) as tile[r][k]
    for (int q = ty; q < 32; q += 8) {
        if (trans) {
            const i64 r = r0 + q, k = k0 + tx;
            tile[q][tx] = (r < R && k < K) ? X[k + r * ldx] : 0.0;
        } else {
            const i64 r = r0 + tx, k = k0 + q;
            tile[tx][q] = (r < R && k < K) ? X[r + k * ldx] : 0.0;
        }
    }
    __syncthreads();
    const size_t slice = (size_t)Rp * (size_t)ldk;
    for (int q = ty; q < 32; q += 8) {
        const i64 r = r0 + q, k = k0 + tx;
        if (r >= Rp || k >= ldk) continue;
        const long long Xi = (r < R && k < K) ? fixed54(tile[q][tx], e[r]) : 0;
        const unsigned long long a = (unsigned long long)(Xi < 0 ? -Xi : Xi);
        const bool neg = Xi < 0;
#pragma unroll
        for (int p = 0; p < kSlices; ++p) {
            const int v = (int)((a >> (48 - 6 * p)) & 63ull);
            S[(size_t)p * slice + (size_t)r * ldk + k] = __int2bfloat16_rn(neg ? -v : v);
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

__global__ void fill_int_kernel(int* x, i64 n, int v) {
    const i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = v;
}

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem)), "l"(gmem));
}

__device__ __forceinline__ void ldsm_x4(unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3, const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(smem_u32(p)));
}

__device__ __forceinline__ void mma_bf16(float* c, unsigned a0, unsigned a1, unsigned a2, unsigned a3, unsigned b0,
                                         unsigned b1) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};\n"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

struct OzArgs {
    i64 M, N, K;          // logical sizes
    i64 ldk;              // padded K (row length of the slices), multiple of OBK
    i64 sa_stride, sb_stride;   // elements between consecutive slices
    const __nv_bfloat16* As;    // [SA][Mp][ldk]
    const __nv_bfloat16* Bs;    // [SB][Np][ldk]
    const int* ea;        // row exponents of op(A)
    const int* eb;        // column exponents of op(B)
    double alpha, beta;
    double* C;
    i64 ldc;
    i64 kc;               // K chunk between FP64 flushes (multiple of OBK)
};

// C tile 64 x 32 per CTA; 8 warps as 4 (M) x 2 (N), each 16 x 16 (one m16,
// two n8).  Per k16 step a warp keeps the fragments of all SA slices of its A
// rows in registers and loads each B slice once; the products of group
// t = p + q accumulate in acc[t] (FP32, exact), flushed to FP64 every p.kc.
template <int SA, int SB, int TMAX>
__global__ void __launch_bounds__(ONT, 1) ozaki_mma_kernel(OzArgs p) {
    constexpr int NG = TMAX + 1;                       // groups t = 0..TMAX
    extern __shared__ __align__(16) unsigned char smraw[];
    __nv_bfloat16* sm = reinterpret_cast<__nv_bfloat16*>(smraw);
    constexpr int A_ELEMS = SA * OBM * OPAD, B_ELEMS = SB * OBN * OPAD;
    constexpr int STAGE = A_ELEMS + B_ELEMS;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 3, wn = warp >> 2;
    const i64 m0 = (i64)blockIdx.x * OBM, n0 = (i64)blockIdx.y * OBN;

    double acc64[2][4];
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc64[j][r] = 0.0;

    auto load_stage = [&](int buf, i64 k0) {
        __nv_bfloat16* sa = sm + buf * STAGE;
        __nv_bfloat16* sb = sa + A_ELEMS;
        constexpr int CH_A = SA * OBM * (OBK / 8), CH_B = SB * OBN * (OBK / 8);
        for (int c = tid; c < CH_A + CH_B; c += ONT) {
            if (c < CH_A) {
                const int s = c / (OBM * 4), rem = c % (OBM * 4), row = rem / 4, kk = (rem % 4) * 8;
                cp_async16(sa + (s * OBM + row) * OPAD + kk,
                           p.As + (size_t)s * p.sa_stride + (size_t)(m0 + row) * p.ldk + k0 + kk);
            } else {
                const int cc = c - CH_A;
                const int s = cc / (OBN * 4), rem = cc % (OBN * 4), row = rem / 4, kk = (rem % 4) * 8;
                cp_async16(sb + (s * OBN + row) * OPAD + kk,
                           p.Bs + (size_t)s * p.sb_stride + (size_t)(n0 + row) * p.ldk + k0 + kk);
            }
        }
        asm volatile("cp.async.commit_group;\n" ::);
    };

    const i64 K = p.ldk;
    int buf = 0;
    load_stage(0, 0);
    for (i64 kc0 = 0; kc0 < K; kc0 += p.kc) {
        const i64 kc1 = (kc0 + p.kc < K) ? kc0 + p.kc : K;
        float acc[NG][2][4];
#pragma unroll
        for (int t = 0; t < NG; ++t)
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int r = 0; r < 4; ++r) acc[t][j][r] = 0.f;
        for (i64 k0 = kc0; k0 < kc1; k0 += OBK) {
            const i64 kn = k0 + OBK;
            if (kn < K) {
                load_stage(buf ^ 1, kn);
                asm volatile("cp.async.wait_group 1;\n" ::);
            } else {
                asm volatile("cp.async.wait_group 0;\n" ::);
            }
            __syncthreads();
            const __nv_bfloat16* sa = sm + buf * STAGE;
            const __nv_bfloat16* sb = sa + A_ELEMS;
#pragma unroll
            for (int kk = 0; kk < OBK; kk += 16) {
                unsigned a[SA][4];
                const int arow = wm * 16 + (lane & 15);
                const int akof = kk + ((lane >> 4) << 3);
#pragma unroll
                for (int pa = 0; pa < SA; ++pa)
                    ldsm_x4(a[pa][0], a[pa][1], a[pa][2], a[pa][3], sa + (pa * OBM + arow) * OPAD + akof);
                const int nrow = wn * 16 + ((lane >> 4) << 3) + (lane & 7);
                const int bkof = kk + (((lane >> 3) & 1) << 3);
#pragma unroll
                for (int q = 0; q < SB; ++q) {
                    unsigned b00, b01, b10, b11;
                    ldsm_x4(b00, b01, b10, b11, sb + (q * OBN + nrow) * OPAD + bkof);
#pragma unroll
                    for (int pa = 0; pa < SA; ++pa) {
                        if (pa + q > TMAX) continue;
                        mma_bf16(acc[pa + q][0], a[pa][0], a[pa][1], a[pa][2], a[pa][3], b00, b01);
                        mma_bf16(acc[pa + q][1], a[pa][0], a[pa][1], a[pa][2], a[pa][3], b10, b11);
                    }
                }
            }
            __syncthreads();
            buf ^= 1;
        }
        // flush the exact group sums (integers below 2^24) into FP64 with weights
        // 2^-6t.  Groups t <= 4 and t >= 5 are first combined exactly in 64-bit
        // integers by Horner steps of 2^6 (each below 2^53), so the FP64 pipe
        // sees two conversions and two FMAs per element instead of one per group.
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                long long hi = 0, lo = 0;
#pragma unroll
                for (int t = 0; t < NG && t <= 4; ++t) hi = hi * 64 + (long long)__float2int_rz(acc[t][j][r]);
#pragma unroll
                for (int t = 5; t < NG; ++t) lo = lo * 64 + (long long)__float2int_rz(acc[t][j][r]);
                const int nhi = (NG < 5) ? NG : 5;
                acc64[j][r] = fma((double)hi, ldexp(1.0, -6 * (nhi - 1)), acc64[j][r]);
                if (NG > 5) acc64[j][r] = fma((double)lo, ldexp(1.0, -6 * (NG - 1)), acc64[j][r]);
            }
    }
    // epilogue: C = alpha 2^(ea_i + eb_j - 12) acc + beta C
    const int g = lane >> 2, tq = lane & 3;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const i64 row = m0 + wm * 16 + g + ((r >> 1) << 3);
            const i64 col = n0 + wn * 16 + j * 8 + 2 * tq + (r & 1);
            if (row < p.M && col < p.N) {
                const double v = p.alpha * ldexp(acc64[j][r], p.ea[row] + p.eb[col] - 12);
                double* cp = p.C + row + col * p.ldc;
                *cp = (p.beta == 0.0) ? v : fma(p.beta, *cp, v);
            }
        }
    }
}

inline i64 rup(i64 x, i64 m) { return (x + m - 1) / m * m; }

template <int SA, int SB, int TMAX>
int launch_mma(const Ctx& c, OzArgs a, i64 Mp, i64 Np) {
    const size_t smem = 2ull * (size_t)(SA * OBM + SB * OBN) * OPAD * sizeof(__nv_bfloat16);
    static std::once_flag attr_once;
    std::call_once(attr_once, [&] {
        cudaFuncSetAttribute(ozaki_mma_kernel<SA, SB, TMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    });
    if (Np / OBN > 65535) { set_error("ozaki: N too large"); return BQRRP_EUNSUPPORTED; }
    dim3 grid((unsigned)(Mp / OBM), (unsigned)(Np / OBN));
    ozaki_mma_kernel<SA, SB, TMAX><<<grid, ONT, smem, c.stream>>>(a);
    BQ_LAUNCH_CHECK();
    return 0;
}

// The tcgen05 kernel (ozaki_tc.cu) runs the slice products unless
// BQRRP_OZAKI_MMA is set in the environment, which selects the mma.sync
// kernel above (kept for side-by-side timing).
bool use_tcgen05() {
    static const bool tc = (getenv("BQRRP_OZAKI_MMA") == nullptr);
    return tc;
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
                  i64 N, const int* ea, const int* eb, double alpha, double beta, double* C, i64 ldc, int* err);
int ozaki_tc_sketch(const Ctx& c, const __nv_bfloat16* Ss, i64 Mp, const __nv_bfloat16* Bs, i64 Np, i64 ldk, i64 M,
                    i64 N, const int* ea, const int* eb, double* C, i64 ldc, int* err);

// Workspace (bytes) for ozaki_gemm / ozaki_sketch on these sizes.
size_t ozaki_ws_bytes(i64 M, i64 N, i64 K, int sa) {
    const i64 Mp = rup(imax(M, 1), OBM), Np = rup(imax(N, 1), OBN), Kp = rup(imax(K, 1), OBK);
    return ((size_t)sa * Mp * Kp + (size_t)kSlices * Np * Kp) * sizeof(__nv_bfloat16) +
           (size_t)(Mp + Np) * sizeof(int) + 2048;
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
    if (!ar.ok()) { set_error("ozaki_gemm: workspace too small"); return BQRRP_ENOMEM; }
    // exponents: rows of op(A), columns of op(B) (= rows of op(B)^T)
    row_exp_kernel<<<(unsigned)M, 256, 0, c.stream>>>(M, K, A, lda, ta ? 1 : 0, ea);
    BQ_LAUNCH_CHECK();
    row_exp_kernel<<<(unsigned)N, 256, 0, c.stream>>>(N, K, B, ldb, tb ? 0 : 1, eb);
    BQ_LAUNCH_CHECK();
    // slices: op(A) rows x K, op(B)^T rows (= N) x K
    split_kernel<<<dim3((unsigned)(Kp / 32), (unsigned)(Mp / 32)), 256, 0, c.stream>>>(M, K, Mp, Kp, A, lda,
                                                                                      ta ? 1 : 0, ea, As);
    BQ_LAUNCH_CHECK();
    split_kernel<<<dim3((unsigned)(Kp / 32), (unsigned)(Np / 32)), 256, 0, c.stream>>>(N, K, Np, Kp, B, ldb,
                                                                                      tb ? 0 : 1, eb, Bs);
    BQ_LAUNCH_CHECK();
    OzArgs a{};
    a.M = M; a.N = N; a.K = K; a.ldk = Kp;
    a.sa_stride = Mp * Kp; a.sb_stride = Np * Kp;
    a.As = As; a.Bs = Bs; a.ea = ea; a.eb = eb;
    a.alpha = alpha; a.beta = beta; a.C = C; a.ldc = ldc;
    a.kc = 256;
    if (!use_tcgen05()) return launch_mma<kSlices, kSlices, kTmax>(c, a, Mp, Np);
    int* err = c.st ? &c.st->err_timeout : flag;
    if (!c.st) BQ_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), c.stream));
    BQ_TRY(ozaki_tc_gemm(c, As, Mp, Bs, Np, Kp, M, N, ea, eb, alpha, beta, C, ldc, err));
    return check_flag(c, flag);
}

int pgemm(const Ctx& c, bool ta, bool tb, i64 M, i64 N, i64 K, double alpha, const double* A, i64 lda,
          const double* B, i64 ldb, double beta, double* C, i64 ldc, int flags) {
    if (c.mixed && c.oz_ws && M > 0 && N > 0 && K >= 32 && (double)M * N * K >= 16.0 * 1024 * 1024 &&
        ozaki_ws_bytes(M, N, K, kSlices) <= c.oz_bytes)
        return ozaki_gemm(c, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, c.oz_ws, c.oz_bytes);
    return dgemm(c, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, flags);
}

// Msk = S A with the dense +-1 operator S (d x m) as one exact slice:
// nine tensor-core products S A_q; FP32 sums of |+-1 * q| over K = m stay
// below 2^24 for m < 2^18, so one FP64 flush per 2^17 columns suffices.
int ozaki_sketch(const Ctx& c, i64 d, i64 m, i64 n, uint64_t seed, const double* A, i64 lda, double* Msk, i64 ldsk,
                 void* ws, size_t ws_bytes) {
    if (d <= 0 || n <= 0) return 0;
    const i64 Mp = rup(d, OBM), Np = rup(n, OBN), Kp = rup(imax(m, 1), OBK);
    if (ws_bytes < ozaki_ws_bytes(d, n, m, 1)) { set_error("ozaki_sketch: workspace too small"); return BQRRP_ENOMEM; }
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
    // S has one slice q_0 = +-1 with weight 2^(ea - 6) = 1: ea = 6 on every row
    fill_int_kernel<<<(unsigned)cdiv(Mp, 256), 256, 0, c.stream>>>(ea, Mp, 6);
    BQ_LAUNCH_CHECK();
    row_exp_kernel<<<(unsigned)n, 256, 0, c.stream>>>(n, m, A, lda, 1, eb);
    BQ_LAUNCH_CHECK();
    split_kernel<<<dim3((unsigned)(Kp / 32), (unsigned)(Np / 32)), 256, 0, c.stream>>>(n, m, Np, Kp, A, lda, 1, eb, Bs);
    BQ_LAUNCH_CHECK();
    OzArgs a{};
    a.M = d; a.N = n; a.K = m; a.ldk = Kp;
    a.sa_stride = Mp * Kp; a.sb_stride = Np * Kp;
    a.As = Ss; a.Bs = Bs; a.ea = ea; a.eb = eb;
    a.alpha = 1.0; a.beta = 0.0; a.C = Msk; a.ldc = ldsk;
    a.kc = (i64)1 << 17;
    if (!use_tcgen05()) return launch_mma<1, kSlices, kSlices - 1>(c, a, Mp, Np);
    int* err = c.st ? &c.st->err_timeout : flag;
    if (!c.st) BQ_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), c.stream));
    BQ_TRY(ozaki_tc_sketch(c, Ss, Mp, Bs, Np, Kp, d, n, ea, eb, Msk, ldsk, err));
    return check_flag(c, flag);
}

}  // namespace bq
