// First-fit allocator over the byte offsets of the serving loop's device
// pool (host bookkeeping only; server.cu owns the device memory).  Header-only
// so that a host test can exercise it without CUDA.
#pragma once

#include <algorithm>
#include <cstdint>
#include <iterator>
#include <map>

namespace hicops {

// Free ranges are kept by offset and are never adjacent: a returned range
// merges with its free neighbours.  The server asks for multiples of 256
// bytes, so every offset stays 256-byte aligned.  take() fails (false) when
// no free range holds the bytes; give() takes back exactly a range take()
// handed out.
struct PoolMap {
    std::map<uint64_t, uint64_t> free_ranges;   // offset -> size
    uint64_t size = 0, used = 0, peak = 0;
    void init(uint64_t bytes) {
        size = bytes;
        free_ranges.clear();
        if (bytes) free_ranges[0] = bytes;
    }
    uint64_t largest() const {
        uint64_t m = 0;
        for (const auto& f : free_ranges) m = std::max(m, f.second);
        return m;
    }
    bool take(uint64_t bytes, uint64_t* off) {
        for (auto it = free_ranges.begin(); it != free_ranges.end(); ++it) {
            if (it->second < bytes) continue;
            *off = it->first;
            const uint64_t rest = it->second - bytes;
            free_ranges.erase(it);
            if (rest) free_ranges[*off + bytes] = rest;
            used += bytes;
            peak = std::max(peak, used);
            return true;
        }
        return false;
    }
    void give(uint64_t off, uint64_t bytes) {
        used -= bytes;
        auto next = free_ranges.lower_bound(off);
        if (next != free_ranges.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                off = prev->first;
                bytes += prev->second;
                free_ranges.erase(prev);
            }
        }
        if (next != free_ranges.end() && off + bytes == next->first) {
            bytes += next->second;
            free_ranges.erase(next);
        }
        free_ranges[off] = bytes;
    }
};

}  // namespace hicops
