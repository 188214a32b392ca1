// tc_schedule.cuh -- the order of work of the tensor-core slice GEMM
// (ozaki_tc.cu): which tile, k block, plane and accumulator half each role
// handles next, and which shared-memory slot and barrier phase it uses.
//
// The three roles of ozaki_tc_kernel (TMA producer, MMA issuer, epilogue)
// walk the same sequence; each role's loop is written once here, over a
// visitor that performs the actual operations (PTX on the device, a recording
// simulator in the CPU test tests/test_tc_schedule_cpu.py, which checks that
// every wait is eventually satisfied, that every MMA reads the operands it
// expects and that every accumulator chunk is read exactly once).
//
// Layout recap (ozaki_tc.cu has the full description): a C tile is 128 x 64;
// its two 32-column halves h = 0, 1 own TMEM columns [256 h, 256 h + 256),
// seven groups of 32 used.  A k block is 64 deep.  Per k block and half there is one
// "segment": the MMAs of that half over all A planes.  A half's accumulators
// are read by the epilogue every CL k blocks (a chunk); the two halves' chunk
// ends are staggered by CL/2 k blocks, and in each k block the half whose
// chunk ends goes first, so the epilogue of one half overlaps the other
// half's MMAs.
#pragma once

#ifdef __CUDACC__
#define TC_HD __host__ __device__ __forceinline__
#else
#define TC_HD inline
#endif

namespace tcs {

constexpr int kNAS = 8;    // A slots (one plane tile each)
constexpr int kNBS = 3;    // B slots (one half-stage each: 7 planes x 32 rows)
constexpr int kGroupRows = 64;   // row tiles per raster group

struct Plan {
    int SA;       // planes of op(A): 7 (FP64 split) or 1 (the +-1 sketch)
    int KB;       // 64-deep k blocks per tile
    int CL;       // k blocks per exact chunk, a power of two (2, or 2048 for the sketch)
    int mt, nct;  // row tiles, column tiles
    int ntiles;   // mt * nct
    int grid;     // persistent CTAs; CTA c takes tiles c, c + grid, ...
};

// Grouped raster: tiles run in groups of up to kGroupRows row tiles, row tile
// fastest, so that a group's A rows stay in L2 while its column tiles stream.
TC_HD void tile_coords(const Plan& P, int tile, int* rt, int* ct) {
    const int GR = P.mt < kGroupRows ? P.mt : kGroupRows;
    const int per_group = GR * P.nct;
    const int g = tile / per_group, r = tile % per_group;
    const int rows = (P.mt - g * GR) < GR ? (P.mt - g * GR) : GR;
    *rt = g * GR + r % rows;
    *ct = r / rows;
}

// The half whose chunks end first in the it-th tile of a CTA.  With CL = 2
// and an even number of k blocks the roles alternate, so that the half read
// first at the end of a tile is the one that starts the next tile.
TC_HD int early_half(const Plan& P, int it) { return (P.CL == 2 && (P.KB % 2) == 0) ? (it & 1) : 0; }

TC_HD bool natural_end(const Plan& P, int E, int h, int kb) {
    const int shift = (h == E) ? (P.CL >> 1) : 0;
    return ((kb + 1 + shift) & (P.CL - 1)) == 0;
}

// Does the chunk of half h end with k block kb (its accumulators are read)?
TC_HD bool chunk_end(const Plan& P, int E, int h, int kb) { return natural_end(P, E, h, kb) || kb == P.KB - 1; }

// The half whose segment comes first in k block kb.
TC_HD int first_half(const Plan& P, int E, int kb) {
    for (int h = 0; h < 2; ++h)
        if (natural_end(P, E, h, kb)) return h;
    if (kb > 0)
        for (int h = 0; h < 2; ++h)
            if (natural_end(P, E, h, kb - 1)) return 1 - h;
    return E;
}

// Plane order of segment seg (global count): ascending or descending.  The two
// segments of a k block use opposite orders and the next k block continues in
// the order of the last segment, so the plane whose slot frees first (its last
// use comes first) is the first one loaded and needed again.
TC_HD bool ascending(long long seg) {
    const bool asc0 = ((seg >> 1) & 1) == 0;
    return (seg & 1) ? !asc0 : asc0;
}

// Slot and fill count of A plane p in global k block G.  With 7 planes each
// plane has a slot of its own (refilled once per k block); with one plane the
// slots form a ring over k blocks.
TC_HD int a_slot(const Plan& P, long long G, int p) { return P.SA == 1 ? (int)(G & (kNAS - 1)) : p; }
TC_HD long long a_fill(const Plan& P, long long G) { return P.SA == 1 ? (G >> 3) : G; }
static_assert(kNAS == 8, "a_slot and a_fill assume eight A slots");

// Position in the B ring: slot and fill count, advanced without divisions.
struct BRing {
    int slot = 0;
    long long fill = 0;
    TC_HD void next() {
        if (++slot == kNBS) {
            slot = 0;
            ++fill;
        }
    }
};

// ---------------------------------------------------------------- roles
// Visitor methods return false when a bounded wait gave up; the role stops.

// TMA producer: per k block the first segment's B half, the A planes in the
// order the MMAs need them, then the second segment's B half.  SA (the number
// of A planes, P.SA) is a compile-time constant so that the plane loops unroll.
template <int SA, class V>
TC_HD void producer(const Plan& P, int cta, V& v) {
    long long G = 0;
    BRing br;
    int it = 0;
    for (int tile = cta; tile < P.ntiles; tile += P.grid, ++it) {
        const int E = early_half(P, it);
        v.tile_begin(tile);
        for (int kb = 0; kb < P.KB; ++kb, ++G) {
            const int h1 = first_half(P, E, kb);
            if (!v.load_b(tile, kb, h1, br.slot, br.fill)) return;
            br.next();
            const long long fill = a_fill(P, G);
            const bool asc = ascending(2 * G);
#pragma unroll 1
            for (int j = 0; j < SA; ++j) {
                const int p = asc ? j : SA - 1 - j;
                if (!v.load_a(tile, kb, p, a_slot(P, G, p), fill)) return;
            }
            if (!v.load_b(tile, kb, 1 - h1, br.slot, br.fill)) return;
            br.next();
        }
    }
}

// MMA issuer: per k block two segments; a half waits for its accumulators to
// be free at the start of each of its chunks and signals them full at the end.
// The plane loops are not unrolled: the single issuing thread's code stays
// small (unrolling them measured slower, the kernel's code being large).

template <int SA, class V>
TC_HD void mma_issuer(const Plan& P, int cta, V& v) {
    long long G = 0;
    BRing br;
    long long chunks[2] = {0, 0};
    int it = 0;
    for (int tile = cta; tile < P.ntiles; tile += P.grid, ++it) {
        const int E = early_half(P, it);
        for (int kb = 0; kb < P.KB; ++kb, ++G) {
            const int h1 = first_half(P, E, kb);
            for (int j = 0; j < 2; ++j) {
                const int h = j ? 1 - h1 : h1;
                if (kb == 0 || chunk_end(P, E, h, kb - 1))
                    if (!v.wait_acc_empty(h, chunks[h])) return;
                const int sb = br.slot;
                if (!v.wait_full_b(sb, br.fill)) return;
                const bool asc = ascending(2 * G + j);
                const long long fill = a_fill(P, G);
#pragma unroll 1
                for (int jj = 0; jj < SA; ++jj) {
                    const int p = asc ? jj : SA - 1 - jj;
                    const int sa = a_slot(P, G, p);
                    if (j == 0 && !v.wait_full_a(sa, fill)) return;
                    v.mma(tile, kb, h, p, sa, sb);
                    if (j == 1) v.release_a(sa);
                }
                v.release_b(sb);
                br.next();
                if (chunk_end(P, E, h, kb)) {
                    v.acc_ready(h);
                    ++chunks[h];
                }
            }
        }
    }
}

// Epilogue of half h: zero its accumulators once, then per chunk wait, read
// (and zero) them and release them; at the end of a tile convert and store.
template <class V>
TC_HD void epilogue(const Plan& P, int cta, int h, V& v) {
    long long chunks = 0;
    int it = 0;
    v.zero_all();
    v.release_acc(h);
    for (int tile = cta; tile < P.ntiles; tile += P.grid, ++it) {
        const int E = early_half(P, it);
        v.tile_begin();
        for (int kb = 0; kb < P.KB; ++kb) {
            if (!chunk_end(P, E, h, kb)) continue;
            if (!v.wait_acc_full(h, chunks)) return;
            v.read_chunk(h);
            v.release_acc(h);
            ++chunks;
        }
        v.tile_end(tile, h);
    }
}

}  // namespace tcs
