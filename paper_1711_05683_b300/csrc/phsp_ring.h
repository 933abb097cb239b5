// phsp_ring.h -- the byte ring of the serving loop (host only): blocks handed out in arrival
// order, 256-byte aligned, released in any order; a block is only handed out where it overlaps
// no live one.  Header-only so that a CPU test can build it on its own.
#pragma once

#include <cstdint>
#include <deque>
#include <utility>

namespace hydra {

struct Ring {
    uint64_t size = 0, head = 0;
    std::deque<std::pair<uint64_t, uint64_t>> live;  // [start, end) of every live block
    // A block of nbytes (rounded up to 256) at the head, or at 0 when it would run past the end;
    // false when that place overlaps a live block or the ring is too small.
    bool alloc(uint64_t nbytes, uint64_t* start) {
        nbytes = (nbytes + 255) / 256 * 256;
        if (nbytes == 0 || nbytes > size) return false;
        const uint64_t s = head + nbytes <= size ? head : 0;
        const uint64_t e = s + nbytes;
        for (const auto& b : live)
            if (b.first < e && s < b.second) return false;
        head = e;
        live.emplace_back(s, e);
        *start = s;
        return true;
    }
    void release(uint64_t start) {
        for (auto it = live.begin(); it != live.end(); ++it)
            if (it->first == start) {
                live.erase(it);
                return;
            }
    }
};

}  // namespace hydra
