// ozaki_tc.cu -- the slice products of the FP64-accurate GEMM (ozaki.cu) on
// the 5th-generation tensor cores: tcgen05.mma with operands staged in shared
// memory by TMA and FP32 accumulators in tensor memory (TMEM).
//
// Each tile of C = alpha op(A) op(B) + beta C is 128 x 32; one persistent CTA
// per SM walks the tiles.  The operands are the
// bf16 slice planes As[p][row][k] (p < SA) and Bs[q][col][k] (q < SB), both
// K-contiguous.  Warp roles (320 threads):
//   warp 0      TMA producer: per 64-deep k block, one 3-D load of all SB
//               B planes (32 x 64 each) and SA loads of A planes (128 x 64),
//               128-byte swizzled, into rings of shared-memory stages;
//   warp 1      allocates 512 TMEM columns; one thread issues the MMAs.
//               The B planes q = 0..7 of a stage lie back to back, so one
//               tcgen05.mma.kind::f16 with M = 128, N = 256, K = 16 whose
//               accumulator starts at TMEM column 32 p multiplies A plane p by
//               all eight at once and lands block q in columns 32 (p + q):
//               the accumulator of group t = p + q.  The MMA for plane p
//               takes only the planes with p + q <= TMAX (N = 32 per plane,
//               at most eight); plane q = 8 adds one N = 32 MMA where
//               p + 8 <= TMAX.  Exactly the 53 products are formed;
//   warps 2-9   epilogue (two warps per 32-lane TMEM quarter, 16 columns
//               each): zeroes the group accumulators before every K chunk
//               (all MMAs accumulate) and after each chunk (Kc deep, every group sum an
//               integer below 2^24, so exact in FP32) it reads the ten
//               group accumulators with tcgen05.ld and adds them into two
//               64-bit integers per element, exactly:
//                 HI += sum_{t <= 4} acc_t 2^(6(4-t)),
//                 LO += sum_{t >= 5} acc_t 2^(6(TMAX-t));
//               at the end C = alpha 2^(ea+eb-12) (HI 2^-24 + LO 2^-6TMAX)
//               + beta C, one FP64 rounding per term.
// Every wait on an mbarrier is bounded; a wait that gives up sets an error
// flag, the roles stop issuing work, in-flight copies and MMAs are waited for
// (bounded), TMEM is freed and the CTA returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <mutex>

#include "common.cuh"

namespace bq {
namespace {

constexpr int TC_M = 128, TC_N = 32, TC_KB = 64;   // tile rows, tile columns, k block
constexpr int TC_THREADS = 320;
constexpr int TC_NA = 4, TC_NB = 2;                // A and B ring stages
constexpr int TC_ABYTES = TC_M * TC_KB * 2;        // 16 KiB per A stage
constexpr int TC_BPLANE = TC_N * TC_KB * 2;        // 4 KiB per B plane
constexpr unsigned long long kTcSpin = 1ull << 26;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(b), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(b) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint32_t b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred P1;\nmbarrier.test_wait.parity.shared::cta.b64 P1, [%1], %2;\nselp.b32 %0, 1, 0, P1;\n}\n"
        : "=r"(ok)
        : "r"(b), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase with this parity; false (and *err set) on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t b, uint32_t parity, int* err) {
    for (unsigned long long i = 0; i < kTcSpin; ++i) {
        if (mbar_test(b, parity)) return true;
        if ((i & 4095) == 4095 && *((volatile int*)err)) return false;
    }
    atomicExch(err, 1);
    return false;
}

// Bounded wait that ignores the error flag: used to drain in-flight copies and
// MMAs before the CTA releases its shared memory and TMEM.
__device__ __forceinline__ void mbar_drain(uint32_t b, uint32_t parity) {
    for (unsigned long long i = 0; i < kTcSpin; ++i)
        if (mbar_test(b, parity)) return;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* tm, int x, int y, int z, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"((uint64_t)tm), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes in 8-row (1024-byte) atoms: start address >> 4, leading offset 1
// (unused for this layout), stride between 8-row groups 1024 B, version 1,
// layout 2 = SWIZZLE_128B.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFF) >> 4) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) |
           (2ull << 61);
}

// Instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16
// (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_f16(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}
constexpr uint32_t kIdesc32 = idesc_f16(TC_N);

// D (TMEM) += A (smem) B (smem)
__device__ __forceinline__ void mma_f16_acc(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, 1, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            dtmem),
        "l"(ad), "l"(bd), "r"(idesc));
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Zero 16 consecutive 32-bit TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_zero16(uint32_t taddr) {
    const uint32_t z = 0;
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr),
        "r"(z)
        : "memory");
}

// 16 consecutive 32-bit TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

struct TcArgs {
    i64 M, N;
    int KB;            // 64-deep k blocks
    int kbpc;          // k blocks per exact chunk
    int mt, ntiles;    // row tiles, all tiles (tile = row tile + mt * column tile)
    const int* ea;
    const int* eb;
    double alpha, beta;
    double* C;
    i64 ldc;
    int* err;
};

// Planes of B multiplied by A plane pa in one MMA: q = 0 .. nq-1 with
// pa + q <= TMAX, at most eight (the ninth plane gets its own MMA).
template <int TMAX>
__device__ __forceinline__ int stacked_planes(int pa) {
    const int nq = TMAX - pa + 1;
    return nq < 8 ? nq : 8;
}

// Persistent: CTA b handles tiles b, b + gridDim.x, ...  The accumulators of a
// tile are released as soon as the epilogue has read its last chunk, so the
// final FP64 conversion and the stores of C overlap the next tile's MMAs.
template <int SA, int SB, int TMAX>
__global__ void __launch_bounds__(TC_THREADS, 1)
    ozaki_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TcArgs p) {
    constexpr int NG = TMAX + 1;
    static_assert(NG * TC_N <= 512, "group accumulators exceed TMEM");
    static_assert(SB == 9 && SA <= 9, "the stacked-B MMA covers B planes 0..7 plus plane 8");
    constexpr int BBYTES = SB * TC_BPLANE;
    extern __shared__ unsigned char smraw[];
    // 1024-byte aligned stage buffers (the 128-byte swizzle atom)
    unsigned char* sm = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    unsigned char* sA = sm;                              // TC_NA x 16 KiB
    unsigned char* sB = sA + TC_NA * TC_ABYTES;          // TC_NB x BBYTES
    uint64_t* bars = (uint64_t*)(sB + TC_NB * BBYTES);   // full_a, empty_a, full_b, empty_b, acc_full, acc_empty, drain
    uint32_t* tslot = (uint32_t*)(bars + 2 * TC_NA + 2 * TC_NB + 3);
    const uint32_t bfa = su32(bars), bea = bfa + 8 * TC_NA, bfb = bea + 8 * TC_NA, beb = bfb + 8 * TC_NB;
    const uint32_t bacc_full = beb + 8 * TC_NB, bacc_empty = bacc_full + 8, bdrain = bacc_empty + 8;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nchunks = (p.KB + p.kbpc - 1) / p.kbpc;

    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_NA; ++s) {
            mbar_init(bfa + 8 * s, 1);
            mbar_init(bea + 8 * s, 1);
        }
        for (int s = 0; s < TC_NB; ++s) {
            mbar_init(bfb + 8 * s, 1);
            mbar_init(beb + 8 * s, 1);
        }
        mbar_init(bacc_full, 1);
        mbar_init(bacc_empty, 8);
        mbar_init(bdrain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)), "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == 0) {
        // ---------------- TMA producer
        if (lane == 0) {
            int sa = 0, sb = 0;
            uint32_t pha = 0, phb = 0;
            // stages loaded at least once (bit s) and the parity of their last load
            uint32_t used_a = 0, par_a = 0, used_b = 0, par_b = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < p.ntiles && ok; tile += gridDim.x) {
                const int m0 = (tile % p.mt) * TC_M, n0 = (tile / p.mt) * TC_N;
                for (int kb = 0; kb < p.KB && ok; ++kb) {
                    if (!(ok = mbar_wait(beb + 8 * sb, phb ^ 1, p.err))) break;
                    mbar_expect_tx(bfb + 8 * sb, BBYTES);
                    tma_load_3d(su32(sB + sb * BBYTES), &tmB, kb * TC_KB, n0, 0, bfb + 8 * sb);
                    used_b |= 1u << sb;
                    par_b = (par_b & ~(1u << sb)) | (phb << sb);
                    for (int pa = 0; pa < SA; ++pa) {
                        if (!(ok = mbar_wait(bea + 8 * sa, pha ^ 1, p.err))) break;
                        mbar_expect_tx(bfa + 8 * sa, TC_ABYTES);
                        tma_load_3d(su32(sA + sa * TC_ABYTES), &tmA, kb * TC_KB, m0, pa, bfa + 8 * sa);
                        used_a |= 1u << sa;
                        par_a = (par_a & ~(1u << sa)) | (pha << sa);
                        if (++sa == TC_NA) {
                            sa = 0;
                            pha ^= 1;
                        }
                    }
                    if (++sb == TC_NB) {
                        sb = 0;
                        phb ^= 1;
                    }
                }
            }
            // every issued copy has landed before the CTA may exit (the phase a
            // stage was last loaded in completes when its bytes arrive)
            for (int s = 0; s < TC_NA; ++s)
                if (used_a >> s & 1u) mbar_drain(bfa + 8 * s, (par_a >> s) & 1u);
            for (int s = 0; s < TC_NB; ++s)
                if (used_b >> s & 1u) mbar_drain(bfb + 8 * s, (par_b >> s) & 1u);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            int sa = 0, sb = 0;
            uint32_t pha = 0, phb = 0;
            unsigned g = 0;                              // chunks issued so far (all tiles)
            bool ok = true;
            for (int tile = blockIdx.x; tile < p.ntiles && ok; tile += gridDim.x) {
                for (int c = 0; c < nchunks && ok; ++c, ++g) {
                    // the epilogue has zeroed the accumulators (initially, and
                    // right after reading every chunk)
                    if (!(ok = mbar_wait(bacc_empty, g & 1u, p.err))) break;
                    tc_fence_after();
                    const int kb0 = c * p.kbpc, kb1 = min(p.KB, kb0 + p.kbpc);
                    for (int kb = kb0; kb < kb1 && ok; ++kb) {
                        if (!(ok = mbar_wait(bfb + 8 * sb, phb, p.err))) break;
                        tc_fence_after();
                        const uint32_t bbase = su32(sB + sb * BBYTES);
                        const uint64_t b8 = sdesc(bbase);                    // planes 0..7 stacked along N
                        const uint64_t b1 = sdesc(bbase + 8 * TC_BPLANE);    // plane 8
                        for (int pa = 0; pa < SA; ++pa) {
                            if (!(ok = mbar_wait(bfa + 8 * sa, pha, p.err))) break;
                            tc_fence_after();
                            const uint64_t ad = sdesc(su32(sA + sa * TC_ABYTES));
                            const int nq = stacked_planes<TMAX>(pa);
                            const uint32_t idn = idesc_f16(nq * TC_N);
#pragma unroll
                            for (int ks = 0; ks < TC_KB / 16; ++ks) {
                                // +32 bytes per 16-deep k step inside the swizzled 128-byte rows
                                mma_f16_acc(tmem + (uint32_t)(pa * TC_N), ad + (uint64_t)(ks * 2),
                                            b8 + (uint64_t)(ks * 2), idn);
                                if (pa + 8 <= TMAX)
                                    mma_f16_acc(tmem + (uint32_t)((pa + 8) * TC_N), ad + (uint64_t)(ks * 2),
                                                b1 + (uint64_t)(ks * 2), kIdesc32);
                            }
                            mma_commit(bea + 8 * sa);
                            if (++sa == TC_NA) {
                                sa = 0;
                                pha ^= 1;
                            }
                        }
                        mma_commit(beb + 8 * sb);
                        if (++sb == TC_NB) {
                            sb = 0;
                            phb ^= 1;
                        }
                    }
                    if (ok) mma_commit(bacc_full);
                }
            }
            // wait for every issued MMA before TMEM is released
            mma_commit(bdrain);
            mbar_drain(bdrain, 0);
        }
    } else {
        // ---------------- epilogue: warp w owns TMEM lanes 32 (w % 4) .. + 31 and
        // columns 16 h .. 16 h + 15 of every group, h = (w - 2) / 4
        constexpr int HN = TC_N / 2;
        const int wq = warp & 3, h = (warp - 2) >> 2;
        const uint32_t tl = tmem + ((uint32_t)(32 * wq) << 16) + (uint32_t)(HN * h);
        // zero this warp's share of the group accumulators for the first chunk
#pragma unroll
        for (int t = 0; t < NG; ++t) tmem_zero16(tl + (uint32_t)(t * TC_N));
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(bacc_empty);
        unsigned g = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < p.ntiles && ok; tile += gridDim.x) {
            const int m0 = (tile % p.mt) * TC_M, n0 = (tile / p.mt) * TC_N;
            long long HI[HN], LO[HN];
#pragma unroll
            for (int j = 0; j < HN; ++j) {
                HI[j] = 0;
                LO[j] = 0;
            }
            for (int c = 0; c < nchunks && ok; ++c, ++g) {
                // lane 0 waits; the outcome is shared so that the warp-collective
                // tcgen05.ld below always runs with the whole warp
                int got = 0;
                if (lane == 0) got = mbar_wait(bacc_full, g & 1u, p.err) ? 1 : 0;
                ok = __shfl_sync(0xffffffffu, got, 0) != 0;
                if (!ok) break;
                tc_fence_after();
#pragma unroll
                for (int t = 0; t < NG; ++t) {
                    uint32_t v[HN];
                    tmem_ld16(tl + (uint32_t)(t * TC_N), v);
#pragma unroll
                    for (int j = 0; j < HN; ++j) {
                        const long long x = (long long)__float2int_rz(__uint_as_float(v[j]));
                        if (t <= 4) HI[j] += x * (1ll << (6 * (4 - t)));
                        else LO[j] += x * (1ll << (6 * (TMAX - t)));
                    }
                    tmem_zero16(tl + (uint32_t)(t * TC_N));
                }
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(bacc_empty);
            }
            // the accumulators are free again: convert and store while the next
            // tile's MMAs run
            const i64 row = m0 + 32 * wq + lane;
            if (ok && row < p.M) {
                const int er = p.ea[row];
#pragma unroll
                for (int j = 0; j < HN; ++j) {
                    const i64 col = n0 + HN * h + j;
                    if (col < p.N) {
                        double v = ldexp((double)HI[j], -24);
                        if (TMAX >= 5) v += ldexp((double)LO[j], -6 * TMAX);
                        const double out = p.alpha * ldexp(v, er + p.eb[col] - 12);
                        double* cp = p.C + row + col * p.ldc;
                        *cp = (p.beta == 0.0) ? out : fma(p.beta, *cp, out);
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)f;
    });
    return fn;
}

// 3-D map over slice planes S[plane][row][k] (k contiguous, ldk elements per
// row, rows_p rows per plane), box {64, box_rows, box_planes}, 128-byte swizzle.
int make_plane_map(CUtensorMap* tm, const void* base, i64 ldk, i64 rows_p, int planes, int box_rows, int box_planes) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) { set_error("cuTensorMapEncodeTiled is unavailable"); return BQRRP_ECUDA; }
    cuuint64_t dims[3] = {(cuuint64_t)ldk, (cuuint64_t)rows_p, (cuuint64_t)planes};
    cuuint64_t strides[2] = {(cuuint64_t)ldk * 2, (cuuint64_t)ldk * 2 * (cuuint64_t)rows_p};
    cuuint32_t box[3] = {(cuuint32_t)TC_KB, (cuuint32_t)box_rows, (cuuint32_t)box_planes};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) { set_error("cuTensorMapEncodeTiled failed (%d)", (int)r); return BQRRP_ECUDA; }
    return 0;
}

template <int SA, int SB, int TMAX>
int launch_tc(const Ctx& c, const __nv_bfloat16* As, i64 Mp, const __nv_bfloat16* Bs, i64 Np, i64 ldk, i64 M, i64 N,
              i64 kc, const int* ea, const int* eb, double alpha, double beta, double* C, i64 ldc, int* err) {
    CUtensorMap tmA, tmB;
    BQ_TRY(make_plane_map(&tmA, As, ldk, Mp, SA, TC_M, 1));
    BQ_TRY(make_plane_map(&tmB, Bs, ldk, Np, SB, TC_N, SB));
    const size_t smem = 1024 + (size_t)TC_NA * TC_ABYTES + (size_t)TC_NB * SB * TC_BPLANE + 8 * (2 * TC_NA + 2 * TC_NB + 3) + 16;
    BQ_TRY(kernel_attrs((const void*)ozaki_tc_kernel<SA, SB, TMAX>, (int)smem));
    TcArgs a;
    a.M = M;
    a.N = N;
    a.KB = (int)cdiv(ldk, TC_KB);
    a.kbpc = (int)imax(1, kc / TC_KB);
    a.ea = ea;
    a.eb = eb;
    a.alpha = alpha;
    a.beta = beta;
    a.C = C;
    a.ldc = ldc;
    a.err = err;
    const i64 mt = cdiv(M, TC_M), tiles = mt * cdiv(N, TC_N);
    if (tiles > (i64)1 << 30) { set_error("ozaki_tc: too many tiles"); return BQRRP_EUNSUPPORTED; }
    a.mt = (int)mt;
    a.ntiles = (int)tiles;
    const unsigned grid = (unsigned)imin(tiles, (i64)c.dev.sms);   // one CTA per SM (TMEM, shared memory)
    ozaki_tc_kernel<SA, SB, TMAX><<<grid, TC_THREADS, smem, c.stream>>>(tmA, tmB, a);
    BQ_LAUNCH_CHECK();
    return 0;
}

}  // namespace

// Slice products on tcgen05: the 9 x 9 FP64 split (53 pairs) and the +-1
// sketch (one A plane, nine B planes).
int ozaki_tc_gemm(const Ctx& c, const __nv_bfloat16* As, i64 Mp, const __nv_bfloat16* Bs, i64 Np, i64 ldk, i64 M,
                  i64 N, const int* ea, const int* eb, double alpha, double beta, double* C, i64 ldc, int* err) {
    return launch_tc<9, 9, 9>(c, As, Mp, Bs, Np, ldk, M, N, 256, ea, eb, alpha, beta, C, ldc, err);
}

int ozaki_tc_sketch(const Ctx& c, const __nv_bfloat16* Ss, i64 Mp, const __nv_bfloat16* Bs, i64 Np, i64 ldk, i64 M,
                    i64 N, const int* ea, const int* eb, double* C, i64 ldc, int* err) {
    return launch_tc<1, 9, 8>(c, Ss, Mp, Bs, Np, ldk, M, N, (i64)1 << 17, ea, eb, 1.0, 0.0, C, ldc, err);
}

}  // namespace bq
