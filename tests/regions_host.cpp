// The serving loop's pool allocator (orbg_regions.h) driven by a seeded random
// sequence of placements and returns, checked against a granule-by-granule
// model of the pool.  Built for the host by tests/test_regions_host.py.
#include <cstdint>
#include <vector>

#include "orbg_regions.h"

namespace {

// xorshift64*: the sequence's own random source
struct Rng {
    uint64_t s;
    uint64_t next()
    {
        s ^= s >> 12;
        s ^= s << 25;
        s ^= s >> 27;
        return s * 2685821657736338717ull;
    }
};

}  // namespace

// Returns 0 when every check held, else the number of the failed check.
extern "C" int regions_run(uint64_t seed, uint64_t pool_granules, int steps, uint64_t *placed_out)
{
    const size_t G = orbg_host::Regions::kGranule;
    orbg_host::Regions r(pool_granules * G);
    std::vector<char> used(pool_granules, 0);
    struct Live {
        size_t off, bytes;
    };
    std::vector<Live> live;
    Rng rng{seed * 0x9E3779B97F4A7C15ull + 1};
    uint64_t placed = 0;
    for (int step = 0; step < steps; step++) {
        const bool give_back = !live.empty() && (rng.next() % 100) < 45;
        if (give_back) {
            const size_t i = rng.next() % live.size();
            const Live l = live[i];
            r.release(l.off, l.bytes);
            const size_t g0 = l.off / G, g1 = (l.off + l.bytes + G - 1) / G;
            for (size_t g = g0; g < g1; g++)
                used[g] = 0;
            live[i] = live.back();
            live.pop_back();
        } else {
            // sizes from one byte to a quarter of the pool, granule-ragged
            const size_t bytes = 1 + rng.next() % (pool_granules * G / 4);
            const size_t need = (bytes + G - 1) / G;
            // first fit in the model: the lowest run of `need` free granules
            size_t want = SIZE_MAX, run = 0;
            for (size_t g = 0; g < pool_granules; g++) {
                run = used[g] ? 0 : run + 1;
                if (run == need) {
                    want = g + 1 - need;
                    break;
                }
            }
            size_t off = 0;
            const bool ok = r.alloc(bytes, &off);
            if (ok != (want != SIZE_MAX))
                return 1;  // placed exactly when the model has room
            if (!ok)
                continue;
            if (off != want * G)
                return 2;  // at the lowest offset that fits
            for (size_t g = want; g < want + need; g++) {
                if (used[g])
                    return 3;  // never over a live range
                used[g] = 1;
            }
            live.push_back({off, bytes});
            placed++;
        }
        // the free list is the complement of the live ranges, merged
        size_t prev_end = 0;
        bool first = true;
        size_t free_granules = 0;
        for (const auto &kv : r.free_ranges()) {
            if (kv.first % G || kv.second % G || kv.second == 0)
                return 4;
            if (!first && kv.first <= prev_end)
                return 5;  // sorted, disjoint and not touching: merged
            for (size_t g = kv.first / G; g < (kv.first + kv.second) / G; g++)
                if (g >= pool_granules || used[g])
                    return 6;
            free_granules += kv.second / G;
            prev_end = kv.first + kv.second;
            first = false;
        }
        size_t used_granules = 0;
        for (char u : used)
            used_granules += u != 0;
        if (free_granules + used_granules != pool_granules)
            return 7;
    }
    // returning everything leaves one range: the whole pool
    for (const Live &l : live)
        r.release(l.off, l.bytes);
    const auto &f = r.free_ranges();
    if (f.size() != 1 || f.begin()->first != 0 || f.begin()->second != pool_granules * G)
        return 8;
    *placed_out = placed;
    return 0;
}
