// CPU simulation of the tensor-core slice GEMM's schedule (tc_schedule.cuh):
// the producer, MMA-issuer and epilogue roles of one CTA run as interleaved
// processes over simulated mbarriers with the hardware's parity-wait rule.
// Checks: every role runs to completion (no wait is left unsatisfied), no
// wait could confuse two phases of a barrier, every MMA reads the A plane and
// B half it expects, no slot is refilled before its uses are released, MMAs
// only accumulate into a free half, and each accumulator read sees exactly
// the k blocks of its chunk.  Usage: tc_schedule_sim SA KB CL mt nct grid seed
#include <cstdio>
#include <cstdlib>
#include <functional>
#include <map>
#include <random>
#include <set>
#include <tuple>
#include <vector>

#include "../../paper_2507_00976_b300/csrc/tc_schedule.cuh"

static void fail(const char* what) {
    std::fprintf(stderr, "FAIL: %s\n", what);
    std::exit(1);
}

struct Bar {
    int count = 1, arrived = 0;
    long long tx = 0, completed = 0;
    std::function<void()> on_complete;
    void check() {
        if (arrived == count && tx == 0) {
            arrived = 0;
            ++completed;
            if (on_complete) on_complete();
        }
    }
    void arrive() {
        ++arrived;
        if (arrived > count) fail("too many arrivals");
        check();
    }
    // does a wait for phase n (parity n & 1) pass?  Aliasing is an error.
    bool passes(long long n) const {
        const bool hw = (completed & 1) != (n & 1);
        if (hw && completed != n + 1) fail("parity wait would confuse two phases");
        return hw;
    }
};

// A role as a list of steps; each step is a predicate (may it run now?) and an action.
struct Step {
    std::function<bool()> ready;
    std::function<void()> run;
};

struct Sim {
    tcs::Plan P;
    int cta;
    Bar full_a[tcs::kNAS], empty_a[tcs::kNAS], full_b[tcs::kNBS], empty_b[tcs::kNBS], acc_full[2], acc_empty[2];
    // slot contents and their uses
    std::tuple<int, int, int> a_content[tcs::kNAS];
    int a_uses[tcs::kNAS], a_filled[tcs::kNAS];
    std::tuple<int, int, int> b_content[tcs::kNBS];
    int b_uses[tcs::kNBS], b_filled[tcs::kNBS];
    // accumulators: open for MMAs, and the (tile, kb) -> MMA count since the last read
    bool acc_open[2] = {false, false};
    std::map<std::pair<int, int>, int> acc[2];
    int readers[2] = {0, 0};   // epilogue warps that read the current chunk
    std::set<std::tuple<int, int, int>> covered;   // (tile, kb, h) read by an epilogue
    std::vector<int> tiles_seen;

    Sim(tcs::Plan p, int c) : P(p), cta(c) {
        for (int h = 0; h < 2; ++h) {
            acc_empty[h].count = 8;
            acc_empty[h].on_complete = [this, h] {
                acc_open[h] = true;
                acc[h].clear();
                readers[h] = 0;
            };
        }
        for (int s = 0; s < tcs::kNAS; ++s) a_uses[s] = a_filled[s] = 0;
        for (int s = 0; s < tcs::kNBS; ++s) b_uses[s] = b_filled[s] = 0;
    }
};

// ---- visitors that record steps
struct ProdRec {
    Sim& S;
    std::vector<Step>& out;
    void tile_begin(int) {}
    bool load_a(int tile, int kb, int p, int slot, long long fill) {
        out.push_back({[this, slot, fill] { return S.empty_a[slot].passes(fill - 1); },
                       [this, tile, kb, p, slot] {
                           if (S.a_filled[slot] && S.a_uses[slot] != 2) fail("A slot refilled before both uses");
                           S.a_content[slot] = {tile, kb, p};
                           S.a_uses[slot] = 0;
                           S.a_filled[slot] = 1;
                           S.full_a[slot].tx += 1;   // expect_tx (arrival) then the copy lands
                           S.full_a[slot].arrive();
                           S.full_a[slot].tx -= 1;
                           S.full_a[slot].check();
                       }});
        return true;
    }
    bool load_b(int tile, int kb, int h, int slot, long long fill) {
        out.push_back({[this, slot, fill] { return S.empty_b[slot].passes(fill - 1); },
                       [this, tile, kb, h, slot] {
                           if (S.b_filled[slot] && S.b_uses[slot] != S.P.SA) fail("B slot refilled before its uses");
                           S.b_content[slot] = {tile, kb, h};
                           S.b_uses[slot] = 0;
                           S.b_filled[slot] = 1;
                           S.full_b[slot].tx += 1;
                           S.full_b[slot].arrive();
                           S.full_b[slot].tx -= 1;
                           S.full_b[slot].check();
                       }});
        return true;
    }
};

struct MmaRec {
    Sim& S;
    std::vector<Step>& out;
    bool wait_acc_empty(int h, long long chunk) {
        out.push_back({[this, h, chunk] { return S.acc_empty[h].passes(chunk); }, [] {}});
        return true;
    }
    bool wait_full_b(int sb, long long fill) {
        out.push_back({[this, sb, fill] { return S.full_b[sb].passes(fill); }, [] {}});
        return true;
    }
    bool wait_full_a(int sa, long long fill) {
        out.push_back({[this, sa, fill] { return S.full_a[sa].passes(fill); }, [] {}});
        return true;
    }
    void mma(int tile, int kb, int h, int p, int sa, int sb) {
        out.push_back({[] { return true; }, [this, tile, kb, h, p, sa, sb] {
                           if (S.a_content[sa] != std::make_tuple(tile, kb, p)) fail("MMA reads the wrong A plane");
                           if (S.b_content[sb] != std::make_tuple(tile, kb, h)) fail("MMA reads the wrong B half");
                           if (!S.acc_open[h]) fail("MMA into accumulators that are not free");
                           ++S.a_uses[sa];
                           ++S.b_uses[sb];
                           ++S.acc[h][{tile, kb}];
                       }});
    }
    void release_a(int sa) {
        out.push_back({[] { return true; }, [this, sa] {
                           if (S.a_uses[sa] != 2) fail("A slot released early");
                           S.empty_a[sa].arrive();
                       }});
    }
    void release_b(int sb) {
        out.push_back({[] { return true; }, [this, sb] { S.empty_b[sb].arrive(); }});
    }
    void acc_ready(int h) {
        out.push_back({[] { return true; }, [this, h] {
                           S.acc_open[h] = false;
                           S.acc_full[h].arrive();
                       }});
    }
};

struct EpiRec {
    Sim& S;
    std::vector<Step>& out;
    int warp;
    int tile_cur = -1;
    void zero_all() {}
    void release_acc(int h) {
        out.push_back({[] { return true; }, [this, h] { S.acc_empty[h].arrive(); }});
    }
    bool wait_acc_full(int h, long long chunk) {
        out.push_back({[this, h, chunk] { return S.acc_full[h].passes(chunk); }, [] {}});
        return true;
    }
    void read_chunk(int h) {
        out.push_back({[] { return true; }, [this, h] {
                           if (S.acc_open[h]) fail("accumulators read while open");
                           if (S.acc[h].empty()) fail("empty chunk read");
                           // every k block of the chunk has its SA MMAs, all of one tile, contiguous
                           int tile = -1, lo = 1 << 30, hi = -1;
                           for (auto& kv : S.acc[h]) {
                               if (kv.second != S.P.SA) fail("k block with a wrong MMA count");
                               if (tile >= 0 && kv.first.first != tile) fail("chunk spans two tiles");
                               tile = kv.first.first;
                               lo = std::min(lo, kv.first.second);
                               hi = std::max(hi, kv.first.second);
                           }
                           if ((int)S.acc[h].size() != hi - lo + 1) fail("chunk k blocks not contiguous");
                           if (S.readers[h]++ == 0)
                               for (int kb = lo; kb <= hi; ++kb)
                                   if (!S.covered.insert({tile, kb, h}).second) fail("k block read twice");
                       }});
    }
    void tile_begin() {}
    void tile_end(int tile, int h) {
        out.push_back({[] { return true; }, [this, tile, h] {
                           for (int kb = 0; kb < S.P.KB; ++kb)
                               if (!S.covered.count({tile, kb, h})) fail("tile ended with a k block never read");
                       }});
    }
};

int main(int argc, char** argv) {
    if (argc < 8) return 2;
    tcs::Plan P;
    P.SA = std::atoi(argv[1]);
    P.KB = std::atoi(argv[2]);
    P.CL = std::atoi(argv[3]);
    P.mt = std::atoi(argv[4]);
    P.nct = std::atoi(argv[5]);
    P.ntiles = P.mt * P.nct;
    P.grid = std::atoi(argv[6]);
    const unsigned seed = (unsigned)std::atoi(argv[7]);

    // the raster is a bijection onto (row tile, column tile)
    std::set<std::pair<int, int>> cells;
    for (int t = 0; t < P.ntiles; ++t) {
        int rt, ct;
        tcs::tile_coords(P, t, &rt, &ct);
        if (rt < 0 || rt >= P.mt || ct < 0 || ct >= P.nct) fail("raster out of range");
        cells.insert({rt, ct});
    }
    if ((int)cells.size() != P.ntiles) fail("raster is not a bijection");

    std::mt19937 rng(seed);
    for (int cta = 0; cta < std::min(P.grid, P.ntiles); ++cta) {
        Sim S(P, cta);
        std::vector<std::vector<Step>> roles(18);
        ProdRec pr{S, roles[0]};
        MmaRec mr{S, roles[1]};
        if (P.SA == 7) {
            tcs::producer<7>(P, cta, pr);
            tcs::mma_issuer<7>(P, cta, mr);
        } else if (P.SA == 1) {
            tcs::producer<1>(P, cta, pr);
            tcs::mma_issuer<1>(P, cta, mr);
        } else {
            fail("SA must be 7 or 1");
        }
        std::vector<EpiRec> ep;
        ep.reserve(16);
        for (int w = 0; w < 16; ++w) ep.push_back(EpiRec{S, roles[2 + w], w});
        for (int w = 0; w < 16; ++w) tcs::epilogue(P, cta, w / 8, ep[w]);
        std::vector<size_t> pc(roles.size(), 0);
        while (true) {
            std::vector<int> can;
            bool done = true;
            for (size_t r = 0; r < roles.size(); ++r) {
                if (pc[r] < roles[r].size()) {
                    done = false;
                    if (roles[r][pc[r]].ready()) can.push_back((int)r);
                }
            }
            if (done) break;
            if (can.empty()) {
                for (size_t r = 0; r < roles.size(); ++r)
                    std::fprintf(stderr, "role %zu at step %zu of %zu\n", r, pc[r], roles[r].size());
                fail("deadlock");
            }
            const int r = can[rng() % can.size()];
            roles[r][pc[r]].run();
            ++pc[r];
        }
        for (int t = cta; t < P.ntiles; t += P.grid)
            for (int kb = 0; kb < P.KB; ++kb)
                for (int h = 0; h < 2; ++h)
                    if (!S.covered.count({t, kb, h})) fail("a k block was never accumulated and read");
    }
    std::printf("ok\n");
    return 0;
}
