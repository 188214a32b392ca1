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
// eight groups of 32.  A k block is 64 deep.  Each half has an MMA-issuing
// thread of its own; per k block it runs one "segment": the MMAs of its half
// over all A planes.  The A planes of a k block are shared by both halves (a
// slot is refilled once both have used it); the B half-stages form one ring in
// the order (k block, half 0), (k block, half 1), ...  A half's accumulators
// are read by the epilogue every CL k blocks (a chunk); the two halves' chunk
// ends are staggered by CL/2 k blocks, so that while one half waits for its
// epilogue the other half's MMAs keep the tensor core busy.
#pragma once

#ifdef __CUDACC__
#define TC_HD __host__ __device__ __forceinline__
#else
#define TC_HD inline
#endif

namespace tcs {

constexpr int kNAS = 8;    // A slots (one plane tile each)
constexpr int kNBS = 3;    // B slots (one half-stage each: 8 planes x 32 rows)
constexpr int kGroupRows = 64;   // row tiles per raster group

struct Plan {
    int SA;       // planes of op(A): 8 (FP64 split) or 1 (the +-1 sketch)
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

// Does the chunk of half h end with k block kb (its accumulators are read)?
// Half 1's chunks end CL/2 k blocks before half 0's; both end at the tile's
// last k block.
TC_HD bool chunk_end(const Plan& P, int h, int kb) {
    const int shift = h ? (P.CL >> 1) : 0;
    return ((kb + 1 + shift) & (P.CL - 1)) == 0 || kb == P.KB - 1;
}

// Slot and fill count of A plane p in global k block G.  With 8 planes each
// plane has a slot of its own (refilled once per k block); with one plane the
// slots form a ring over k blocks.
TC_HD int a_slot(const Plan& P, long long G, int p) { return P.SA == 1 ? (int)(G & (kNAS - 1)) : p; }
TC_HD long long a_fill(const Plan& P, long long G) { return P.SA == 1 ? (G >> 3) : G; }
static_assert(kNAS == 8, "a_slot and a_fill assume eight A slots");

// Position in the B ring (slot and fill count) of segment s = 2 G + h,
// advanced without divisions.
struct BRing {
    int slot = 0;
    long long fill = 0;
    TC_HD void advance(int by) {   // by = 1 or 2
        slot += by;
        if (slot >= kNBS) {
            slot -= kNBS;
            ++fill;
        }
    }
};

// ---------------------------------------------------------------- roles
// Visitor methods return false when a bounded wait gave up; the role stops.

// TMA producer: per k block the B half of half 0, the A planes, the B half of
// half 1 (the order in which the two issuers need them).
template <int SA, class V>
TC_HD void producer(const Plan& P, int cta, V& v) {
    long long G = 0;
    BRing br;
    for (int tile = cta; tile < P.ntiles; tile += P.grid) {
        v.tile_begin(tile);
        for (int kb = 0; kb < P.KB; ++kb, ++G) {
            if (!v.load_b(tile, kb, 0, br.slot, br.fill)) return;
            br.advance(1);
            const long long fill = a_fill(P, G);
            for (int p = 0; p < SA; ++p)
                if (!v.load_a(tile, kb, p, a_slot(P, G, p), fill)) return;
            if (!v.load_b(tile, kb, 1, br.slot, br.fill)) return;
            br.advance(1);
        }
    }
}

// MMA issuer of half h: per k block one segment; it waits for its
// accumulators to be free at the start of each of its chunks and signals them
// full at the end.  Every A plane is released by both issuers (the slot's
// empty barrier counts two arrivals).
template <int SA, class V>
TC_HD void mma_issuer(const Plan& P, int cta, int h, V& v) {
    long long G = 0, chunks = 0;
    BRing br;
    br.advance(h);   // segment 2 G + h
    for (int tile = cta; tile < P.ntiles; tile += P.grid) {
        for (int kb = 0; kb < P.KB; ++kb, ++G) {
            if (kb == 0 || chunk_end(P, h, kb - 1))
                if (!v.wait_acc_empty(h, chunks)) return;
            const int sb = br.slot;
            if (!v.wait_full_b(sb, br.fill)) return;
            const long long fill = a_fill(P, G);
            for (int p = 0; p < SA; ++p) {
                const int sa = a_slot(P, G, p);
                if (!v.wait_full_a(sa, fill)) return;
                v.mma(tile, kb, h, p, sa, sb);
                v.release_a(sa);
            }
            v.release_b(sb);
            br.advance(2);
            if (chunk_end(P, h, kb)) {
                v.acc_ready(h);
                ++chunks;
            }
        }
    }
}

// Epilogue of half h: zero its accumulators once, then per chunk wait, read
// (and zero) them and release them; at the end of a tile convert and store.
template <class V>
TC_HD void epilogue(const Plan& P, int cta, int h, V& v) {
    long long chunks = 0;
    v.zero_all();
    v.release_acc(h);
    for (int tile = cta; tile < P.ntiles; tile += P.grid) {
        v.tile_begin();
        for (int kb = 0; kb < P.KB; ++kb) {
            if (!chunk_end(P, h, kb)) continue;
            if (!v.wait_acc_full(h, chunks)) return;
            v.read_chunk(h);
            v.release_acc(h);
            ++chunks;
        }
        v.tile_end(tile, h);
    }
}

}  // namespace tcs
