// Host-only test build of the C++ serving loop's ring (phsp_ring.h), loaded by
// tests/test_serve_ring.py through ctypes.
#include <cstdint>

#include "phsp_ring.h"

extern "C" {

void* ring_new(uint64_t size) {
    hydra::Ring* r = new hydra::Ring();
    r->size = size;
    return r;
}

int ring_alloc(void* h, uint64_t nbytes, uint64_t* start) { return static_cast<hydra::Ring*>(h)->alloc(nbytes, start); }

void ring_release(void* h, uint64_t start) { static_cast<hydra::Ring*>(h)->release(start); }

void ring_free(void* h) { delete static_cast<hydra::Ring*>(h); }

}
