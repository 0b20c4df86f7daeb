/*
 * orbg_regions.h -- the serving loop's pool allocator (host code only):
 * first fit over the byte range [0, size) of one pool, in 256-byte granules,
 * with freed ranges merged with their free neighbours.  The server keeps
 * one for its device pool and one for its pinned host pool, and admits a
 * batch only when both can place its footprint.  Kept in its own header so
 * the host test suite can exercise it without CUDA.
 */
#pragma once
#include <cstddef>
#include <iterator>
#include <map>

namespace orbg_host {

class Regions {
  public:
    static constexpr size_t kGranule = 256;

    explicit Regions(size_t size)
    {
        if (size)
            free_[0] = size;
    }

    /* Places `bytes` (rounded up to whole granules) at the lowest free
     * offset that fits; false, with nothing changed, if none does. */
    bool alloc(size_t bytes, size_t *off)
    {
        bytes = round_up(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t start = it->first + bytes;
                free_.erase(it);
                if (rest)
                    free_[start] = rest;
                return true;
            }
        }
        return false;
    }

    /* Returns a range alloc placed (same offset and byte count). */
    void release(size_t off, size_t bytes)
    {
        bytes = round_up(bytes);
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }

    /* Free ranges, offset -> length (for tests). */
    const std::map<size_t, size_t> &free_ranges() const { return free_; }

  private:
    static size_t round_up(size_t x) { return (x + kGranule - 1) / kGranule * kGranule; }
    std::map<size_t, size_t> free_;
};

}  // namespace orbg_host
