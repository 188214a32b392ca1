// ozaki_tc.cu -- the slice products of the FP64-accurate GEMM (ozaki.cu) on
// the 5th-generation tensor cores: tcgen05.mma with operands staged in shared
// memory by TMA and FP32 accumulators in tensor memory (TMEM).
//
// Operands are bf16 slice planes, K-contiguous: As[p][row][k] (p < SA; SA = 7
// for an FP64 operand, 1 for the +-1 sketch) and Bs[q][col][k] (q < 7).  Every
// slice is an integer in [-128, 127].  The product of planes p and q has
// weight 2^-8(p+q); the pairs with p + q <= 6 are formed (28 of them for
// SA = 7, 7 for the sketch) and the products of one group t = p + q are summed
// in one FP32 accumulator, exactly: within a K chunk of CL k blocks every
// partial sum is an integer of magnitude at most 7 * 128 * 128^2 < 2^24
// (SA = 7, CL = 2) or 2^17 * 128 = 2^24 (sketch, CL = 2048).
//
// Tile: 128 rows x 64 columns; one persistent CTA per SM walks the tiles in
// the grouped raster of tc_schedule.cuh.  TMEM (512 columns of 32 bits) holds
// the tile's accumulators: column half h (C columns 32h .. 32h+31) owns TMEM
// columns [256 h, 256 h + 256), group t of it [256 h + 32 t, + 32) (t < 7).
//
// Shared memory (213 KiB): eight A slots of one 128 x 64 plane tile (16 KiB,
// 128-byte swizzled) and three B slots of one half-stage (the 7 planes of 32
// columns x 64 k, 28 KiB), with full/empty mbarriers.
//
// Warp roles (576 threads); the order of their work is tc_schedule.cuh's:
//   warp 0      TMA producer (one thread): per 64-deep k block the B half of
//               the first segment, the SA A planes, the B half of the second;
//   warp 1      allocates the 512 TMEM columns; one thread issues the MMAs.
//               Segment (k block, half h), A plane p: the B planes q = 0..6-p of
//               the half lie back to back in its B slot, so one
//               tcgen05.mma.kind::f16 (M = 128, N = 32 (7 - p), K = 16) whose
//               accumulator starts at TMEM column 256 h + 32 p lands plane q in
//               group p + q; four such MMAs cover the k block.  The half whose
//               chunk ends in a k block goes first, so the epilogue of one half
//               overlaps the other half's MMAs;
//   warps 2-17  epilogue, eight warps per half (warp w reads TMEM lanes
//               32 (w % 4) ..; two warps share a lane quarter, 16 columns
//               each).  After each chunk a warp reads the seven groups with
//               tcgen05.ld, zeroes them with tcgen05.st, releases the half and
//               forms the chunk's exact value per element,
//                 W = (sum_{t <= 2} G_t 2^(8(2-t))) 2^32 + sum_{t >= 3} G_t 2^(8(6-t)),
//               rounded to a multiple of 2^dsh and added into one 64-bit
//               integer; after a tile's last chunk (the half is already
//               released for the next tile) C = alpha acc 2^(ea+eb-60+dsh) + beta C,
//               the integer rounded once to FP64 with integer operations.
// Split K: a product of fewer tiles than half the SMs runs each tile as
// several CTAs over consecutive ranges of k blocks; each adds its 64-bit sums
// into an integer buffer with atomics (exact in any order) and a second kernel
// converts them (TcArgs).
// Every wait on an mbarrier is bounded; a wait that gives up sets an error
// flag, the roles stop issuing work, in-flight copies and MMAs are waited for
// (bounded), TMEM is freed and the CTA returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <mutex>

#include "common.cuh"
#include "tc_schedule.cuh"

namespace bq {
namespace {

constexpr int TC_M = 128, TC_N = 64, TC_HN = 32, TC_KB = 64;   // tile rows, columns, half columns, k block
constexpr int TC_NP = kOzPlanes;                                // planes of op(B)
constexpr int TC_NG = kOzPlanes;                                // groups t = 0..6
constexpr int TC_EPI = 16;                                      // epilogue warps
constexpr int TC_THREADS = 64 + 32 * TC_EPI;
constexpr int TC_APLANE = TC_M * TC_KB * 2;                     // 16 KiB per A slot
constexpr int TC_BHALF = TC_NP * TC_HN * TC_KB * 2;             // 28 KiB per B slot
static_assert(TC_BHALF % 1024 == 0, "B slots keep the 1024-byte swizzle alignment");
constexpr int TC_NBAR = 2 * tcs::kNAS + 2 * tcs::kNBS + 2 + 2 + 1;
constexpr size_t TC_SMEM =
    1024 + (size_t)tcs::kNAS * TC_APLANE + (size_t)tcs::kNBS * TC_BHALF + 8 * TC_NBAR + 16;
constexpr unsigned long long kTcSpin = 1ull << 26;   // test_wait polls: a few seconds
static_assert(TC_SMEM <= 232448, "shared memory of the slice GEMM exceeds the per-CTA limit");

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
// Bounded wait for the phase with this parity; false (and *err set) on
// timeout, or when another role has set it.  (Polling with test_wait measured
// faster here than try_wait with a suspend-time hint.)
__device__ __forceinline__ bool mbar_wait(uint32_t b, uint32_t parity, int* err) {
    for (unsigned long long i = 0; i < kTcSpin; ++i) {
        if (mbar_test(b, parity)) return true;
        if ((i & 4095) == 4095 && *((volatile int*)err)) return false;
    }
    atomicExch(err, 1);
    return false;
}
// The same wait with a back-off of about 100 ns between polls, for the
// epilogue warps: their waits are long, and spinning at full rate would take
// issue slots from the MMA-issuing thread that shares their sub-partition.
__device__ __forceinline__ bool mbar_wait_backoff(uint32_t b, uint32_t parity, int* err) {
    for (unsigned long long i = 0; i < (kTcSpin >> 4); ++i) {
        if (mbar_test(b, parity)) return true;
        if ((i & 255) == 255 && *((volatile int*)err)) return false;
        __nanosleep(100);
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

// D (TMEM) += A (smem) B (smem) for the four 16-deep k steps of a 64-deep k
// block: the descriptors advance by 32 bytes (2 in 16-byte units) per step
// inside the 128-byte swizzled rows.
__device__ __forceinline__ void mma_f16_kblock(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc) {
    asm volatile(
        "{\n.reg .pred p;\n.reg .b64 a1, a2, a3, b1, b2, b3;\nsetp.ne.b32 p, 1, 0;\n"
        "add.s64 a1, %1, 2;\nadd.s64 a2, %1, 4;\nadd.s64 a3, %1, 6;\n"
        "add.s64 b1, %2, 2;\nadd.s64 b2, %2, 4;\nadd.s64 b3, %2, 6;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], a1, b1, %3, p;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], a2, b2, %3, p;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], a3, b3, %3, p;\n}\n" ::"r"(dtmem),
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

// 4 consecutive 32-bit TMEM columns of this thread's lane (no wait: the
// caller issues tcgen05.wait::ld before using them).
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t& v0, uint32_t& v1, uint32_t& v2, uint32_t& v3) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v0), "=r"(v1), "=r"(v2), "=r"(v3)
                 : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Integer-valued FP32 (|v| < 2^24) to int32: exact.
__device__ __forceinline__ int f2i(uint32_t v) { return __float2int_rz(__uint_as_float(v)); }

// The out-of-range case of i64_scaled (kept out of line so that its FP64
// instructions are not executed speculatively on the common path).
__device__ __noinline__ double i64_scaled_slow(unsigned long long a, bool neg, int e) {
    const double v = ldexp((double)a, e);
    return neg ? -v : v;
}

// w * 2^e rounded to the nearest double (ties to even), w a 64-bit integer,
// with integer operations only.  Results outside the normal range (never met
// by the products of this library's inputs) take a plain conversion.
__device__ __forceinline__ double i64_scaled(long long w, int e) {
    if (w == 0) return 0.0;
    const bool neg = w < 0;
    const unsigned long long a = neg ? 0ull - (unsigned long long)w : (unsigned long long)w;
    const int nb = 64 - __clzll((long long)a);   // bit length of a
    unsigned long long mant;
    int ex = nb - 1 + e;   // exponent of the leading bit
    if (nb <= 53) {
        mant = a << (53 - nb);
    } else {
        const int s = nb - 53;
        const unsigned long long rem = a & ((1ull << s) - 1), half = 1ull << (s - 1);
        mant = a >> s;
        if (rem > half || (rem == half && (mant & 1ull))) {
            ++mant;
            if (mant == (1ull << 53)) {
                mant >>= 1;
                ++ex;
            }
        }
    }
    const int be = ex + 1023;
    if (be <= 0 || be >= 2047) return i64_scaled_slow(a, neg, e);
    const unsigned long long bits =
        ((unsigned long long)neg << 63) | ((unsigned long long)be << 52) | (mant & ((1ull << 52) - 1));
    return __longlong_as_double((long long)bits);
}

struct TcArgs {
    tcs::Plan plan;
    int dsh;   // bits dropped (rounded) from each chunk's sum: ceil(log2 K) - 2, at least 8
    i64 M, N;
    const int* ea;
    const int* eb;
    double alpha, beta;
    double* C;
    i64 ldc;
    int* err;
    // Split K: plan.ntiles = tiles x nsplit, tile index = split * tiles + tile,
    // split s covering k blocks [s KB, (s + 1) KB).  Each split adds its 64-bit
    // integers into acc64 (M x N, column-major, zeroed before the launch); a
    // second kernel converts the sums.  nsplit = 1: acc64 is unused.
    int nsplit;
    unsigned long long* acc64;
};

// Split and tile (within the split) of a tile index.
__device__ __forceinline__ int split_of(const TcArgs* p, int tile, int* t) {
    const int per = p->plan.mt * p->plan.nct;
    const int s = tile / per;
    *t = tile - s * per;
    return s;
}

// Barrier addresses: full_a[8], empty_a[8], full_b[3], empty_b[3], acc_full[2], acc_empty[2], drain.
struct Bars {
    uint32_t base;
    __device__ uint32_t full_a(int s) const { return base + 8 * s; }
    __device__ uint32_t empty_a(int s) const { return base + 8 * (tcs::kNAS + s); }
    __device__ uint32_t full_b(int s) const { return base + 8 * (2 * tcs::kNAS + s); }
    __device__ uint32_t empty_b(int s) const { return base + 8 * (2 * tcs::kNAS + tcs::kNBS + s); }
    __device__ uint32_t acc_full(int h) const { return base + 8 * (2 * tcs::kNAS + 2 * tcs::kNBS + h); }
    __device__ uint32_t acc_empty(int h) const { return base + 8 * (2 * tcs::kNAS + 2 * tcs::kNBS + 2 + h); }
    __device__ uint32_t drain() const { return base + 8 * (2 * tcs::kNAS + 2 * tcs::kNBS + 4); }
};

// ---------------------------------------------------------------- role visitors
struct ProducerV {
    const TcArgs* p;
    Bars bar;
    uint32_t sA, sB;
    const CUtensorMap* tmA;
    const CUtensorMap* tmB;
    int m0, n0, kb0;               // origin of the current tile; its split's first k block
    long long last_a[tcs::kNAS];   // last fill issued per slot (-1: none)
    long long last_b[tcs::kNBS];
    __device__ __forceinline__ void tile_begin(int tile) {
        int rt, ct, t;
        kb0 = split_of(p, tile, &t) * p->plan.KB;
        tcs::tile_coords(p->plan, t, &rt, &ct);
        m0 = rt * TC_M;
        n0 = ct * TC_N;
    }
    __device__ __forceinline__ bool load_a(int, int kb, int pl, int slot, long long fill) {
        if (!mbar_wait(bar.empty_a(slot), (uint32_t)((fill & 1) ^ 1), p->err)) return false;
        mbar_expect_tx(bar.full_a(slot), TC_APLANE);
        tma_load_3d(sA + slot * TC_APLANE, tmA, (kb0 + kb) * TC_KB, m0, pl, bar.full_a(slot));
        last_a[slot] = fill;
        return true;
    }
    __device__ __forceinline__ bool load_b(int, int kb, int h, int slot, long long fill) {
        if (!mbar_wait(bar.empty_b(slot), (uint32_t)((fill & 1) ^ 1), p->err)) return false;
        mbar_expect_tx(bar.full_b(slot), TC_BHALF);
        tma_load_3d(sB + slot * TC_BHALF, tmB, (kb0 + kb) * TC_KB, n0 + h * TC_HN, 0, bar.full_b(slot));
        last_b[slot] = fill;
        return true;
    }
};

struct MmaV {
    const TcArgs* p;
    Bars bar;
    uint64_t ad0, bd0;   // descriptors of A slot 0 and B slot 0
    uint32_t tmem;
    __device__ __forceinline__ bool wait_acc_empty(int h, long long chunk) {
        if (!mbar_wait(bar.acc_empty(h), (uint32_t)(chunk & 1), p->err)) return false;
        tc_fence_after();
        return true;
    }
    __device__ __forceinline__ bool wait_full_b(int sb, long long fill) {
        if (!mbar_wait(bar.full_b(sb), (uint32_t)(fill & 1), p->err)) return false;
        tc_fence_after();
        return true;
    }
    __device__ __forceinline__ bool wait_full_a(int sa, long long fill) {
        if (!mbar_wait(bar.full_a(sa), (uint32_t)(fill & 1), p->err)) return false;
        tc_fence_after();
        return true;
    }
    // slot offsets go straight into the descriptors' start-address field (16-byte
    // units; every slot address stays below 2^18)
    __device__ __forceinline__ void mma(int, int, int h, int pl, int sa, int sb) {
        const uint64_t ad = ad0 + (uint64_t)(sa * (TC_APLANE >> 4));
        const uint64_t bd = bd0 + (uint64_t)(sb * (TC_BHALF >> 4));   // planes 0 .. 6 - pl stacked along N
        mma_f16_kblock(tmem + (uint32_t)(256 * h + TC_HN * pl), ad, bd, idesc_f16(TC_HN * (TC_NG - pl)));
    }
    __device__ __forceinline__ void release_a(int sa) { mma_commit(bar.empty_a(sa)); }
    __device__ __forceinline__ void release_b(int sb) { mma_commit(bar.empty_b(sb)); }
    __device__ __forceinline__ void acc_ready(int h) { mma_commit(bar.acc_full(h)); }
};

// Per element the epilogue keeps one 64-bit integer: the sum over chunks of
// the chunk's exact value W (in units of 2^(ea+eb-60)) rounded to a multiple
// of 2^dsh.  One k term is at most 2^54 2^54 / 2^48 = 2^60 units, so |sum|
// stays below K 2^60 / 2^dsh <= 2^62; the rounding adds at most
// K/128 * 2^(dsh-1) units, about K^2 2^-70 of max|A(i,:)| max|B(:,j)|, below
// K 2^-53 of it for K <= 2^17 (the launcher's limit): the normwise error of
// an FP64 GEMM.
struct EpilogueV {
    const TcArgs* p;
    Bars bar;
    uint32_t tl;   // this warp's TMEM address: lane quarter, half, 16-column sub-block
    int lane, lq, sub;
    long long acc[16];
    __device__ __forceinline__ void zero_all() {
#pragma unroll
        for (int t = 0; t < TC_NG; ++t) tmem_zero16(tl + (uint32_t)(TC_HN * t));
    }
    __device__ __forceinline__ void release_acc(int h) {
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(bar.acc_empty(h));
    }
    __device__ __forceinline__ bool wait_acc_full(int h, long long chunk) {
        // lane 0 waits; the outcome is shared so that the warp-collective
        // tcgen05.ld always runs with the whole warp
        int got = 0;
        if (lane == 0) got = mbar_wait_backoff(bar.acc_full(h), (uint32_t)(chunk & 1), p->err) ? 1 : 0;
        if (__shfl_sync(0xffffffffu, got, 0) == 0) return false;
        tc_fence_after();
        return true;
    }
    __device__ __forceinline__ void tile_begin() {
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[j] = 0;
    }
    // W = HI 2^32 + LO with HI = G_0 2^16 + G_1 2^8 + G_2 and
    // LO = G_3 2^24 + G_4 2^16 + G_5 2^8 + G_6, exact in 64 bits: the group
    // sums obey |G_t| <= (t + 1) 128^3 = (t + 1) 2^21 (or 2^24 for the sketch's
    // 2^17-deep chunks), so |HI| < 2^41 and |LO| < 2^49.  Four columns at a
    // time; HI 2^32 is a multiple of 2^dsh (dsh <= 15), so only LO is rounded.
    __device__ __forceinline__ void read_chunk(int) {
        const int dsh = p->dsh, sh = 32 - dsh;
        const long long half = 1ll << (dsh - 1);
#pragma unroll
        for (int cb = 0; cb < 4; ++cb) {
            uint32_t v[TC_NG][4];
#pragma unroll
            for (int t = 0; t < TC_NG; ++t)
                tmem_ld4(tl + (uint32_t)(TC_HN * t + 4 * cb), v[t][0], v[t][1], v[t][2], v[t][3]);
            tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const long long hi =
                    ((long long)f2i(v[0][j]) << 16) + ((long long)f2i(v[1][j]) << 8) + (long long)f2i(v[2][j]);
                const long long lo = ((long long)f2i(v[3][j]) << 24) + ((long long)f2i(v[4][j]) << 16) +
                                     ((long long)f2i(v[5][j]) << 8) + (long long)f2i(v[6][j]);
                acc[4 * cb + j] += (hi << sh) + ((lo + half) >> dsh);
            }
        }
#pragma unroll
        for (int t = 0; t < TC_NG; ++t) tmem_zero16(tl + (uint32_t)(TC_HN * t));
    }
    __device__ __forceinline__ void tile_end(int tile, int h) {
        int rt, ct, t;
        split_of(p, tile, &t);
        tcs::tile_coords(p->plan, t, &rt, &ct);
        const i64 row = (i64)rt * TC_M + 32 * lq + lane;
        if (row >= p->M) return;
        const i64 col0 = (i64)ct * TC_N + TC_HN * h + 16 * sub;
        const int ncol = (int)(p->N - col0 < 16 ? p->N - col0 : 16);
        if (p->nsplit > 1) {
            // integer sums add exactly in any order (|total| < 2^62, see above)
            unsigned long long* ap = p->acc64 + row + col0 * p->M;
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (j < ncol) atomicAdd(ap + j * p->M, (unsigned long long)acc[j]);
            return;
        }
        const int er = p->ea[row] - 60 + p->dsh;
        const double alpha = p->alpha, beta = p->beta;
        double* cp = p->C + row + col0 * p->ldc;
        // alpha = +-1 (a negation of the integer) and beta = 0 or 1 (the
        // library's products) take loops of their own, so that the only FP64
        // instruction is the addition into C; anything else takes the general
        // loop.  (A select between the forms inside one loop would execute the
        // FP64 multiply and FMA of every form.)
        if ((alpha == 1.0 || alpha == -1.0) && beta == 0.0) {
            const bool neg = alpha == -1.0;
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (j < ncol) cp[j * p->ldc] = i64_scaled(neg ? -acc[j] : acc[j], er + p->eb[col0 + j]);
        } else if ((alpha == 1.0 || alpha == -1.0) && beta == 1.0) {
            const bool neg = alpha == -1.0;
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (j < ncol) {
                    double* cj = cp + j * p->ldc;
                    *cj = *cj + i64_scaled(neg ? -acc[j] : acc[j], er + p->eb[col0 + j]);
                }
        } else {
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (j < ncol) {
                    double* cj = cp + j * p->ldc;
                    const double out = alpha * i64_scaled(acc[j], er + p->eb[col0 + j]);
                    *cj = (beta == 0.0) ? out : fma(beta, *cj, out);
                }
        }
    }
};

template <int SA>
__global__ void __launch_bounds__(TC_THREADS, 1)
    ozaki_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                    const __grid_constant__ TcArgs p) {
    extern __shared__ unsigned char smraw[];
    // 1024-byte aligned slots (the 128-byte swizzle atom)
    unsigned char* sm = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    unsigned char* sA = sm;
    unsigned char* sB = sA + tcs::kNAS * TC_APLANE;
    uint64_t* bars = (uint64_t*)(sB + tcs::kNBS * TC_BHALF);
    uint32_t* tslot = (uint32_t*)(bars + TC_NBAR);
    const Bars bar{su32(bars)};
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < tcs::kNAS; ++s) {
            mbar_init(bar.full_a(s), 1);
            mbar_init(bar.empty_a(s), 1);
        }
        for (int s = 0; s < tcs::kNBS; ++s) {
            mbar_init(bar.full_b(s), 1);
            mbar_init(bar.empty_b(s), 1);
        }
        for (int h = 0; h < 2; ++h) {
            mbar_init(bar.acc_full(h), 1);
            mbar_init(bar.acc_empty(h), TC_EPI / 2);
        }
        mbar_init(bar.drain(), 1);
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
        if (lane == 0) {
            ProducerV v{&p, bar, su32(sA), su32(sB), &tmA, &tmB, 0, 0, 0, {}, {}};
            for (int s = 0; s < tcs::kNAS; ++s) v.last_a[s] = -1;
            for (int s = 0; s < tcs::kNBS; ++s) v.last_b[s] = -1;
            tcs::producer<SA>(p.plan, blockIdx.x, v);
            // every issued copy lands before the CTA may exit (fill n of a slot
            // completes phase n of its full barrier)
            for (int s = 0; s < tcs::kNAS; ++s)
                if (v.last_a[s] >= 0) mbar_drain(bar.full_a(s), (uint32_t)(v.last_a[s] & 1));
            for (int s = 0; s < tcs::kNBS; ++s)
                if (v.last_b[s] >= 0) mbar_drain(bar.full_b(s), (uint32_t)(v.last_b[s] & 1));
        }
    } else if (warp == 1) {
        if (lane == 0) {
            MmaV v{&p, bar, sdesc(su32(sA)), sdesc(su32(sB)), tmem};
            tcs::mma_issuer<SA>(p.plan, blockIdx.x, v);
            // every issued MMA completes before TMEM is released
            mma_commit(bar.drain());
            mbar_drain(bar.drain(), 0);
        }
    } else {
        const int e = warp - 2;                 // epilogue warp 0..15
        const int h = e / 8, sub = (e / 4) % 2, lq = warp % 4;
        EpilogueV v;
        v.p = &p;
        v.bar = bar;
        v.lane = lane;
        v.lq = lq;
        v.sub = sub;
        v.tl = tmem + ((uint32_t)(32 * lq) << 16) + (uint32_t)(256 * h + 16 * sub);
        tcs::epilogue(p.plan, blockIdx.x, h, v);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
    }
}

// The end of a split-K product: C = alpha acc64 2^(ea+eb-60+dsh) + beta C per
// element, with the epilogue's rounding and its alpha / beta forms.
__global__ void tc_splitk_finish_kernel(i64 M, i64 N, const unsigned long long* __restrict__ acc64,
                                        const int* __restrict__ ea, const int* __restrict__ eb, int dsh, double alpha,
                                        double beta, double* C, i64 ldc) {
    const i64 total = M * N;
    for (i64 idx = (i64)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (i64)gridDim.x * blockDim.x) {
        const i64 i = idx % M, j = idx / M;
        const long long w = (long long)acc64[idx];
        const int e = ea[i] - 60 + dsh + eb[j];
        double* cj = C + i + j * ldc;
        if ((alpha == 1.0 || alpha == -1.0) && beta == 0.0) {
            *cj = i64_scaled(alpha == -1.0 ? -w : w, e);
        } else if ((alpha == 1.0 || alpha == -1.0) && beta == 1.0) {
            *cj = *cj + i64_scaled(alpha == -1.0 ? -w : w, e);
        } else {
            const double out = alpha * i64_scaled(w, e);
            *cj = (beta == 0.0) ? out : fma(beta, *cj, out);
        }
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
// row, rows_p rows per plane; the map covers k < kext from `base`), box
// {64, box_rows, box_planes}, 128-byte swizzle.  Rows and k beyond the
// extent read as zeros.
int make_plane_map(CUtensorMap* tm, const void* base, i64 ldk, i64 kext, i64 rows_p, int planes, int box_rows,
                   int box_planes) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) { set_error("cuTensorMapEncodeTiled is unavailable"); return BQRRP_ECUDA; }
    cuuint64_t dims[3] = {(cuuint64_t)kext, (cuuint64_t)rows_p, (cuuint64_t)planes};
    cuuint64_t strides[2] = {(cuuint64_t)ldk * 2, (cuuint64_t)ldk * 2 * (cuuint64_t)rows_p};
    cuuint32_t box[3] = {(cuuint32_t)TC_KB, (cuuint32_t)box_rows, (cuuint32_t)box_planes};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) { set_error("cuTensorMapEncodeTiled failed (%d)", (int)r); return BQRRP_ECUDA; }
    return 0;
}

// One launch over k in [0, kext) of the planes starting at As, Bs (row
// stride ldk): C = alpha (sum over those k) + beta C.  With acc64 (M x N
// 64-bit integers) a product of fewer than half as many tiles as SMs splits
// its k blocks over up to SMs / tiles CTAs per tile (at least 4 k blocks
// each); the splits' integer sums are exact, so the result has the unsplit
// product's error bound.
int launch_tc(const Ctx& c, int SA, int CL, const __nv_bfloat16* As, i64 Mp, const __nv_bfloat16* Bs, i64 Np,
              i64 ldk, i64 kext, i64 M, i64 N, const int* ea, const int* eb, double alpha, double beta, double* C,
              i64 ldc, int* err, unsigned long long* acc64) {
    if (ldk % 8 != 0) { set_error("ozaki_tc: slice rows must be a multiple of 8 elements"); return BQRRP_EUNSUPPORTED; }
    if (kext > kOzMaxK) { set_error("ozaki_tc: K above %lld per launch", (long long)kOzMaxK); return BQRRP_EUNSUPPORTED; }
    if (CL < 2 || (CL & (CL - 1)) != 0) { set_error("ozaki_tc: chunk must be a power of two"); return BQRRP_EUNSUPPORTED; }
    CUtensorMap tmA, tmB;
    BQ_TRY(make_plane_map(&tmA, As, ldk, kext, Mp, SA, TC_M, 1));
    BQ_TRY(make_plane_map(&tmB, Bs, ldk, kext, Np, TC_NP, TC_HN, TC_NP));
    const void* fn = SA == 1 ? (const void*)ozaki_tc_kernel<1> : (const void*)ozaki_tc_kernel<kOzPlanes>;
    BQ_TRY(kernel_attrs(fn, (int)TC_SMEM));
    TcArgs a;
    a.M = M;
    a.N = N;
    a.ea = ea;
    a.eb = eb;
    a.alpha = alpha;
    a.beta = beta;
    a.C = C;
    a.ldc = ldc;
    a.err = err;
    i64 KB = cdiv(kext, TC_KB);
    const i64 mt = cdiv(M, TC_M), nct = cdiv(N, TC_N);
    if (mt * nct > (i64)1 << 30 || KB > (i64)1 << 30) { set_error("ozaki_tc: too many tiles"); return BQRRP_EUNSUPPORTED; }
    i64 nsplit = 1;
    if (acc64 && 2 * mt * nct <= (i64)c.dev.sms) {
        const i64 want = imin((i64)c.dev.sms / (mt * nct), KB / 4);
        if (want >= 2) {
            KB = cdiv(KB, want);           // k blocks per split; the last split may run past kext (zero fill)
            nsplit = cdiv(cdiv(kext, TC_KB), KB);
        }
    }
    a.nsplit = (int)nsplit;
    a.acc64 = nsplit > 1 ? acc64 : nullptr;
    a.plan.SA = SA;
    a.plan.KB = (int)KB;
    a.plan.CL = CL;
    a.plan.mt = (int)mt;
    a.plan.nct = (int)nct;
    a.plan.ntiles = (int)(mt * nct * nsplit);
    a.plan.grid = (int)imin(mt * nct * nsplit, (i64)c.dev.sms);   // one CTA per SM (TMEM, shared memory)
    // dsh follows the whole K, so that the splits' sum stays below 2^62
    int lg = 0;
    while (((i64)1 << lg) < kext) ++lg;
    a.dsh = lg - 2 < 8 ? 8 : lg - 2;
    if (nsplit > 1) BQ_CUDA(cudaMemsetAsync(acc64, 0, sizeof(unsigned long long) * (size_t)(M * N), c.stream));
    if (SA == 1)
        ozaki_tc_kernel<1><<<(unsigned)a.plan.grid, TC_THREADS, TC_SMEM, c.stream>>>(tmA, tmB, a);
    else
        ozaki_tc_kernel<kOzPlanes><<<(unsigned)a.plan.grid, TC_THREADS, TC_SMEM, c.stream>>>(tmA, tmB, a);
    BQ_LAUNCH_CHECK();
    if (nsplit > 1) {
        tc_splitk_finish_kernel<<<(unsigned)imin(cdiv(M * N, 256), 4LL * c.dev.sms), 256, 0, c.stream>>>(
            M, N, acc64, ea, eb, a.dsh, alpha, beta, C, ldc);
        BQ_LAUNCH_CHECK();
    }
    return 0;
}

}  // namespace

// Slice products on tcgen05: the 7 x 7 FP64 split (the 28 pairs with
// p + q <= 6, exact in chunks of two k blocks) and the +-1 sketch (one A
// plane, seven B planes, exact in chunks of 2048 k blocks).
// K beyond kOzMaxK runs as consecutive launches over K pieces, each adding
// its FP64-rounded part into C.
int ozaki_tc_gemm(const Ctx& c, const __nv_bfloat16* As, i64 Mp, const __nv_bfloat16* Bs, i64 Np, i64 ldk, i64 M,
                  i64 N, const int* ea, const int* eb, double alpha, double beta, double* C, i64 ldc, int* err,
                  unsigned long long* acc64) {
    for (i64 k0 = 0; k0 < ldk; k0 += kOzMaxK)
        BQ_TRY(launch_tc(c, kOzPlanes, 2, As + k0, Mp, Bs + k0, Np, ldk, imin(kOzMaxK, ldk - k0), M, N, ea, eb,
                         alpha, k0 == 0 ? beta : 1.0, C, ldc, err, acc64));
    return 0;
}

int ozaki_tc_sketch(const Ctx& c, const __nv_bfloat16* Ss, i64 Mp, const __nv_bfloat16* Bs, i64 Np, i64 ldk, i64 M,
                    i64 N, const int* ea, const int* eb, double* C, i64 ldc, int* err) {
    for (i64 k0 = 0; k0 < ldk; k0 += kOzMaxK)
        BQ_TRY(launch_tc(c, 1, (int)(kOzMaxK / TC_KB), Ss + k0, Mp, Bs + k0, Np, ldk, imin(kOzMaxK, ldk - k0), M, N,
                         ea, eb, 1.0, k0 == 0 ? 0.0 : 1.0, C, ldc, err, nullptr));
    return 0;
}

}  // namespace bq
