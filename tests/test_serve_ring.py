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


# ----------------------------------------------------------------------------- the C++ ring
class _NativeRing:
    """The C++ loop's ring (csrc/phsp_ring.h) built for the host with g++ and driven through ctypes."""

    def __init__(self, lib, size):
        import ctypes
        self.lib, self.size, self.c = lib, size, ctypes
        self.h = lib.ring_new(size)

    def alloc(self, n):
        out = self.c.c_uint64()
        return out.value if self.lib.ring_alloc(self.h, n, self.c.byref(out)) else None

    def free(self, start):
        self.lib.ring_release(self.h, start)

    def close(self):
        self.lib.ring_free(self.h)


@pytest.fixture(scope="module")
def native_ring_lib(tmp_path_factory):
    import ctypes
    import os
    import shutil
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if not shutil.which("g++"):
        pytest.skip("g++ not available")
    so = str(tmp_path_factory.mktemp("ring") / "ring_probe.so")
    subprocess.check_call(["g++", "-std=c++17", "-O2", "-shared", "-fPIC", "-I",
                           os.path.join(root, "paper_1711_05683_b300", "csrc"),
                           os.path.join(root, "tests", "native", "ring_probe.cpp"), "-o", so])
    lib = ctypes.CDLL(so)
    u64, vp = ctypes.c_uint64, ctypes.c_void_p
    lib.ring_new.restype, lib.ring_new.argtypes = vp, [u64]
    lib.ring_alloc.restype, lib.ring_alloc.argtypes = ctypes.c_int, [vp, u64, ctypes.POINTER(u64)]
    lib.ring_release.argtypes = [vp, u64]
    lib.ring_free.argtypes = [vp]
    return lib


def test_native_ring_blocks_are_aligned_disjoint_and_reused(native_ring_lib):
    """The same randomized invariants as the Python ring: aligned, within the ring, disjoint
    from every live block, released in any order, and the whole ring free again at the end."""
    ring = _NativeRing(native_ring_lib, 1 << 16)
    rng = random.Random(7)
    live = {}
    allocated = 0
    for step in range(20000):
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
    assert allocated > 4000
    for start in list(live):
        ring.free(start)
    assert ring.alloc(1 << 16) is not None
    ring.close()


def test_native_ring_refuses_oversized_and_wraps(native_ring_lib):
    ring = _NativeRing(native_ring_lib, 4096)
    assert ring.alloc(4097) is None and ring.alloc(0) is None
    a = ring.alloc(1024)
    b = ring.alloc(3072)
    assert (a, b) == (0, 1024) and ring.alloc(1) is None  # full
    ring.free(a)
    assert ring.alloc(1000) == 0  # wraps to the freed front
    ring.close()
