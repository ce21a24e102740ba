// Host check of the serving loop's pool allocator (pool_map.h) against a
// brute-force model: one owner flag per 256-byte granule.  After every step
// the allocator's free ranges must be exactly the model's maximal free runs
// (so returned ranges have merged with their neighbours), its used bytes the
// model's, and take() must succeed exactly when some free run holds the
// request, at the lowest such offset (first fit).  Prints "ok <steps>" or the
// first mismatch.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "pool_map.h"

namespace {

constexpr uint64_t kG = 256;

struct Model {
    std::vector<int> owner;   // 0 free, else the block id
    explicit Model(uint64_t granules) : owner(granules, 0) {}
    // maximal free runs as (offset, size) in bytes
    std::vector<std::pair<uint64_t, uint64_t>> runs() const {
        std::vector<std::pair<uint64_t, uint64_t>> r;
        for (uint64_t i = 0; i < owner.size();) {
            if (owner[i]) { ++i; continue; }
            uint64_t j = i;
            while (j < owner.size() && !owner[j]) ++j;
            r.push_back({i * kG, (j - i) * kG});
            i = j;
        }
        return r;
    }
};

int fail(const char* what, long step) {
    std::printf("mismatch at step %ld: %s\n", step, what);
    return 1;
}

}  // namespace

int main(int argc, char** argv) {
    const long steps = argc > 1 ? std::atol(argv[1]) : 20000;
    const uint64_t granules = 97;   // an odd pool: 24,832 bytes
    hicops::PoolMap pm;
    pm.init(granules * kG);
    Model m(granules);
    struct Block { uint64_t off, bytes; int id; };
    std::vector<Block> live;
    std::mt19937_64 rng(12345);
    uint64_t peak = 0, used = 0;
    int next_id = 1;
    // hand case first: three blocks, free the middle then the first: one
    // merged range in front, then the last block, then the tail
    {
        uint64_t a, b, c;
        if (!pm.take(2 * kG, &a) || !pm.take(3 * kG, &b) || !pm.take(kG, &c)) return fail("hand take", -1);
        if (a != 0 || b != 2 * kG || c != 5 * kG) return fail("hand offsets", -1);
        pm.give(b, 3 * kG);
        pm.give(a, 2 * kG);
        if (pm.free_ranges.size() != 2 || pm.free_ranges.begin()->second != 5 * kG) return fail("hand merge", -1);
        pm.give(c, kG);
        if (pm.free_ranges.size() != 1 || pm.largest() != granules * kG || pm.used != 0)
            return fail("hand whole", -1);
        pm.init(granules * kG);
    }
    for (long s = 0; s < steps; ++s) {
        const bool do_take = live.empty() || (rng() % 100) < 55;
        if (do_take) {
            const uint64_t want = (1 + rng() % 24) * kG;
            // the model's first free run that holds the request
            uint64_t expect = UINT64_MAX;
            for (auto& r : m.runs())
                if (r.second >= want) { expect = r.first; break; }
            uint64_t off = 0;
            const bool ok = pm.take(want, &off);
            if (ok != (expect != UINT64_MAX)) return fail("take success differs from the model", s);
            if (ok) {
                if (off != expect) return fail("not first fit", s);
                if (off % kG) return fail("unaligned offset", s);
                for (uint64_t g = off / kG; g < (off + want) / kG; ++g) {
                    if (g >= granules) return fail("range leaves the pool", s);
                    if (m.owner[g]) return fail("range overlaps a live block", s);
                    m.owner[g] = next_id;
                }
                live.push_back({off, want, next_id++});
                used += want;
            }
        } else {
            const size_t i = rng() % live.size();
            const Block b = live[i];
            live[i] = live.back();
            live.pop_back();
            pm.give(b.off, b.bytes);
            for (uint64_t g = b.off / kG; g < (b.off + b.bytes) / kG; ++g) m.owner[g] = 0;
            used -= b.bytes;
        }
        if (used > peak) peak = used;
        const auto runs = m.runs();
        if (runs.size() != pm.free_ranges.size()) return fail("free range count", s);
        size_t j = 0;
        uint64_t largest = 0;
        for (auto& f : pm.free_ranges) {
            if (f.first != runs[j].first || f.second != runs[j].second) return fail("free ranges differ", s);
            if (f.second > largest) largest = f.second;
            ++j;
        }
        if (pm.largest() != largest) return fail("largest", s);
        if (pm.used != used || pm.peak != peak) return fail("used or peak", s);
    }
    std::printf("ok %ld\n", steps);
    return 0;
}
