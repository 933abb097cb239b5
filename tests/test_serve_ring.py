"""Host logic of the server's ring allocator (pinned host and device arenas): blocks are
256-byte aligned, never overlap a live block, wrap around, and may be released in any order."""
import random

import pytest

torch = pytest.importorskip("torch")

from paper_1711_05683_b300.serve import Ring  # noqa: E402


def test_ring_blocks_are_aligned_disjoint_and_reused():
    ring = Ring(torch.empty(1 << 16, dtype=torch.uint8))
    rng = random.Random(7)
    live = {}
    allocated = 0
    for step in range(5000):
        if live and (rng.random() < 0.45 or len(live) > 40):
            start = rng.choice(list(live))
            ring.free(start)
            del live[start]
            continue
        n = rng.randint(1, 6000)
        start = ring.alloc(n)
        if start is None:
            continue
        allocated += 1
        end = start + (n + 255) // 256 * 256
        assert start % 256 == 0 and end <= ring.size
        for s, e in live.items():
            assert end <= s or e <= start, (start, end, s, e)
        live[start] = end
    assert allocated > 1000
    for start in list(live):
        ring.free(start)
    assert ring.alloc(1 << 16) is not None  # everything released: the whole buffer fits again


def test_ring_refuses_oversized_and_views_typed_slices():
    ring = Ring(torch.empty(4096, dtype=torch.uint8))
    assert ring.alloc(4097) is None
    a = ring.alloc(1024)
    v = ring.view(a, 1024, torch.float32)
    assert v.numel() == 256 and v.dtype == torch.float32
    b = ring.alloc(3072)
    assert b == 1024 and ring.alloc(1) is None  # full
    ring.free(a)
    assert ring.alloc(1000) == 0  # wraps to the freed front
