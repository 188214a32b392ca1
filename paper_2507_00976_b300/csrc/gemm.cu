// gemm.cu -- FP64 SIMT GEMM for sm_103a.
//
// On B300 the FP64 pipe (about 2 DFMA/clk/SM; tcgen05 has no f64 kind and the
// f64 mma.sync path measured slower than plain DFMA) is the bound of every
// dense contraction in BQRRP, so this kernel only has to keep that pipe fed:
// 64x64 output tiles, 16-deep K slabs staged through shared memory with a
// register double buffer, 4x4 outputs per thread.  Operand traffic per DFMA is
// tiny, so occupancy and load balance across the 148 SMs are what matter:
// products whose tiles would load the SMs unevenly use a deterministic split-K
// (partials in the workspace, reduced in a fixed order), with the split count
// chosen to even out the FP64 work per SM.
//
// The same kernel, with the A operand generated from Philox4x32-10 instead of
// loaded, forms the sketch S*A of Alg. 1 without ever storing S.
#include "common.cuh"

namespace bq {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

struct GemmArgs {
    i64 M, N, K;
    double alpha, beta;
    const double* A;
    i64 lda;
    const double* B;
    i64 ldb;
    double* C;
    i64 ldc;
    i64 kchunk;        // K range per split
    double* partial;   // non-null when gridDim.z > 1
    uint64_t seed;     // sketch generator
    int flags;         // kGemmAUpper / kGemmCUpper
};

// AMODE: 0 = load A, 1 = load A^T, 2 = generate the dense +-1 sketch S (M x K).
template <int AMODE, bool TB>
__global__ void __launch_bounds__(NT) dgemm_kernel(GemmArgs p) {
    __shared__ double As[2][BK][BM + 1];
    __shared__ double Bs[2][BK][BN + 1];

    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const i64 m0 = (i64)blockIdx.x * BM;
    const i64 n0 = (i64)blockIdx.y * BN;
    const i64 kz = (i64)blockIdx.z * p.kchunk;
    const i64 kend = ((p.flags & kGemmCUpper) && m0 >= n0 + BN) ? kz            // tile below the diagonal
                     : (kz + p.kchunk < p.K) ? kz + p.kchunk : p.K;
    const i64 kbeg = ((p.flags & kGemmAUpper) && m0 > kz) ? m0 : kz;   // m0 is a multiple of BK

    double ra[4], rb[4];
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

    auto load_a = [&](i64 k0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int idx = tid + NT * q;
            int mm, kk;
            if (AMODE == 1) { kk = idx & 15; mm = idx >> 4; }
            else            { mm = idx & 63; kk = idx >> 6; }
            const i64 gm = m0 + mm, gk = k0 + kk;
            double v = 0.0;
            if (gm < p.M && gk < kend) {
                if (AMODE == 0) v = p.A[gm + gk * p.lda];
                else if (AMODE == 1) v = p.A[gk + gm * p.lda];
                else v = sketch_dense_entry(p.seed, gm, gk);
            }
            ra[q] = v;
        }
    };
    auto load_b = [&](i64 k0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int idx = tid + NT * q;
            int nn, kk;
            if (TB) { nn = idx & 63; kk = idx >> 6; }
            else    { kk = idx & 15; nn = idx >> 4; }
            const i64 gn = n0 + nn, gk = k0 + kk;
            double v = 0.0;
            if (gn < p.N && gk < kend) v = TB ? p.B[gn + gk * p.ldb] : p.B[gk + gn * p.ldb];
            rb[q] = v;
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int idx = tid + NT * q;
            if (AMODE == 1) As[buf][idx & 15][idx >> 4] = ra[q];
            else            As[buf][idx >> 6][idx & 63] = ra[q];
            if (TB) Bs[buf][idx >> 6][idx & 63] = rb[q];
            else    Bs[buf][idx & 15][idx >> 4] = rb[q];
        }
    };

    int cur = 0;
    if (kbeg < kend) {
        load_a(kbeg);
        load_b(kbeg);
        store(0);
    }
    for (i64 k0 = kbeg; k0 < kend; k0 += BK) {
        __syncthreads();
        const bool more = k0 + BK < kend;
        if (more) {
            load_a(k0 + BK);
            load_b(k0 + BK);
        }
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[cur][kk][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[cur][kk][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        if (more) store(cur ^ 1);
        cur ^= 1;
    }

    if (p.partial) {
        double* P = p.partial + (size_t)blockIdx.z * (size_t)p.M * (size_t)p.N;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const i64 gn = n0 + ty + 16 * j;
            if (gn >= p.N) continue;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const i64 gm = m0 + tx + 16 * i;
                if (gm < p.M) P[gm + gn * p.M] = acc[i][j];
            }
        }
        return;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const i64 gn = n0 + ty + 16 * j;
        if (gn >= p.N) continue;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const i64 gm = m0 + tx + 16 * i;
            if (gm >= p.M) continue;
            double* c = p.C + gm + gn * p.ldc;
            const double v = p.alpha * acc[i][j];
            *c = (p.beta == 0.0) ? v : fma(p.beta, *c, v);
        }
    }
}

__global__ void splitk_reduce_kernel(i64 M, i64 N, int splits, const double* __restrict__ P, double alpha,
                                     double beta, double* C, i64 ldc) {
    const i64 total = M * N;
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (i64)gridDim.x * blockDim.x) {
        const i64 i = e % M, j = e / M;
        double s = 0.0;
        for (int z = 0; z < splits; ++z) s += P[(size_t)z * (size_t)total + e];
        double* c = C + i + j * ldc;
        const double v = alpha * s;
        *c = (beta == 0.0) ? v : fma(beta, *c, v);
    }
}

// Split count along K for an M x N x K product (1 = no split).
int pick_splits(const Ctx& c, i64 M, i64 N, i64 K, int flags) {
    const i64 tm = cdiv(M, BM), tn = cdiv(N, BN);
    // split-K balances the FP64 work over the SMs: one 64x64 tile with K = 64
    // is ~65 us on a single SM, and the tile count of a product is rarely a
    // multiple of the SM count (W = V^T C of a 256-wide block, 4 x nc/64 tiles,
    // lost ~10 % to its last partial wave).  FP64 throughput is per SM, so the
    // time of a split GEMM goes with the CTAs on the busiest SM over the split
    // count, ceil(work_tiles * s / SMs) / s; s minimizes that, down to one
    // 16-deep slab per CTA, taking a larger s only for a gain above 1 % (large
    // products stay unsplit).  Tiles below the diagonal of an
    // upper-triangle-only C do no work.
    int splits = 1;
    const i64 tiles = tm * tn;
    const i64 work_tiles = (flags & kGemmCUpper) ? imin(tm, tn) * (imin(tm, tn) + 1) / 2 + imax(0, tn - tm) * tm
                                                 : tiles;
    const i64 sms = c.dev.sms;
    if (K >= 2 * BK && c.splitk != nullptr) {
        const i64 fit = (i64)(c.splitk_elems / (size_t)(M * N));
        const i64 smax = imin(imin(K / BK, 64), fit);
        double best = 1e30;
        i64 bs = 1;
        for (i64 sc = 1; sc <= smax; ++sc) {
            const double cost = (double)cdiv(work_tiles * sc, sms) / (double)sc;
            if (cost < best * 0.99) { best = cost; bs = sc; }
        }
        splits = (int)bs;
    }
    if (K <= 0) return 1;
    const i64 kchunk = cdiv(cdiv(K, splits), BK) * BK;
    return (int)imax(1, cdiv(K, kchunk));
}

// force_splits > 0 launches with that split count (whose partials must fit
// the split-K scratch); otherwise pick_splits decides.
template <int AMODE, bool TB>
int launch(const Ctx& c, GemmArgs a, int force_splits = 0) {
    const i64 tm = cdiv(a.M, BM), tn = cdiv(a.N, BN);
    if (tm > 2147483647 || tn > 65535) {
        set_error("dgemm: grid too large (%lld x %lld tiles)", (long long)tm, (long long)tn);
        return BQRRP_EUNSUPPORTED;
    }
    int splits = force_splits > 0 ? force_splits : pick_splits(c, a.M, a.N, a.K, a.flags);
    if (splits > 1 && (c.splitk == nullptr || (size_t)splits * (size_t)(a.M * a.N) > c.splitk_elems)) {
        set_error("dgemm: %d splits do not fit the split-K scratch", splits);
        return BQRRP_EUNSUPPORTED;
    }
    a.kchunk = cdiv(cdiv(a.K, splits), BK) * BK;
    splits = (int)cdiv(a.K, a.kchunk);
    if (splits < 1) splits = 1;
    a.partial = splits > 1 ? c.splitk : nullptr;
    dim3 grid((unsigned)tm, (unsigned)tn, (unsigned)splits);
    dgemm_kernel<AMODE, TB><<<grid, NT, 0, c.stream>>>(a);
    BQ_LAUNCH_CHECK();
    if (splits > 1) {
        const i64 total = a.M * a.N;
        const int blocks = (int)imin(cdiv(total, 256), 8LL * c.dev.sms);
        splitk_reduce_kernel<<<blocks, 256, 0, c.stream>>>(a.M, a.N, splits, c.splitk, a.alpha, a.beta, a.C, a.ldc);
        BQ_LAUNCH_CHECK();
    }
    return 0;
}

}  // namespace

int dgemm(const Ctx& c, bool ta, bool tb, i64 M, i64 N, i64 K, double alpha, const double* A, i64 lda,
          const double* B, i64 ldb, double beta, double* C, i64 ldc, int flags) {
    if (M <= 0 || N <= 0) return 0;
    GemmArgs a{};
    a.M = M; a.N = N; a.K = K < 0 ? 0 : K; a.alpha = alpha; a.beta = beta;
    a.A = A; a.lda = lda; a.B = B; a.ldb = ldb; a.C = C; a.ldc = ldc;
    a.flags = flags;
    if (a.K == 0) {
        // C = beta*C: run the kernel with an empty K range (writes alpha*0 + beta*C)
        a.kchunk = BK;
        dim3 grid((unsigned)cdiv(M, BM), (unsigned)cdiv(N, BN), 1);
        dgemm_kernel<0, false><<<grid, NT, 0, c.stream>>>(a);
        BQ_LAUNCH_CHECK();
        return 0;
    }
    if (!ta && !tb) return launch<0, false>(c, a);
    if (!ta && tb) return launch<0, true>(c, a);
    if (ta && !tb) return launch<1, false>(c, a);
    return launch<1, true>(c, a);
}

// C (M x N) = alpha * A (M x K) * B (K x N) + beta * C on strided views; each
// view must be column-major (rs == 1) or row-major (cs == 1).
int gemm_view(const Ctx& c, i64 M, i64 N, i64 K, double alpha, View A, View B, double beta, View C) {
    if (M <= 0 || N <= 0) return 0;
    auto as_op = [](View v, i64 rows, i64 cols, bool* trans, i64* ld) -> bool {
        if (v.rs == 1 && (v.cs >= rows || cols == 1)) { *trans = false; *ld = v.cs > 0 ? v.cs : 1; return true; }
        if (v.cs == 1 && (v.rs >= cols || rows == 1)) { *trans = true; *ld = v.rs > 0 ? v.rs : 1; return true; }
        if (v.rs == 1) { *trans = false; *ld = v.cs; return true; }
        if (v.cs == 1) { *trans = true; *ld = v.rs; return true; }
        return false;
    };
    bool tA, tB, tC;
    i64 la, lb, lc;
    if (!as_op(C, M, N, &tC, &lc)) { set_error("gemm_view: bad C view"); return BQRRP_EUNSUPPORTED; }
    if (!tC) {
        if (!as_op(A, M, K, &tA, &la) || !as_op(B, K, N, &tB, &lb)) {
            set_error("gemm_view: bad operand view");
            return BQRRP_EUNSUPPORTED;
        }
        return dgemm(c, tA, tB, M, N, K, alpha, A.p, la, B.p, lb, beta, C.p, lc);
    }
    // C^T = B^T A^T with C^T column-major
    View At = A.t(), Bt = B.t();
    if (!as_op(Bt, N, K, &tB, &lb) || !as_op(At, K, M, &tA, &la)) {
        set_error("gemm_view: bad operand view");
        return BQRRP_EUNSUPPORTED;
    }
    return dgemm(c, tB, tA, N, M, K, alpha, Bt.p, lb, At.p, la, beta, C.p, lc);
}

int sketch_dense_splits(const Ctx& c, i64 d, i64 m, i64 n) { return pick_splits(c, d, n, m, 0); }

int sketch_dense_gemm(const Ctx& c, i64 d, i64 m, i64 n, uint64_t seed, const double* A, i64 lda, double* Msk,
                      i64 ldsk, int splits) {
    if (d <= 0 || n <= 0) return 0;
    GemmArgs a{};
    a.M = d; a.N = n; a.K = m; a.alpha = 1.0; a.beta = 0.0;
    a.A = nullptr; a.lda = 0; a.B = A; a.ldb = lda; a.C = Msk; a.ldc = ldsk; a.seed = seed;
    if (m == 0) {
        a.kchunk = BK;
        a.K = 0;
        dim3 grid((unsigned)cdiv(d, BM), (unsigned)cdiv(n, BN), 1);
        dgemm_kernel<2, false><<<grid, NT, 0, c.stream>>>(a);
        BQ_LAUNCH_CHECK();
        return 0;
    }
    return launch<2, false>(c, a, splits);
}

}  // namespace bq
