"""Unit tier for the generator's sorting network (the pruned Batcher odd-even merge network that
sorts the n - 2 intermediate-mass draws, K = n - 2 = 1..8), run by a test probe on the GPU and
compared with numpy's sort: every 0/1 input of K values (by the 0-1 principle a comparator
network that sorts all of them sorts every input), every permutation of K distinct values, and
random rows with ties and the uint32 extremes."""
import ctypes
import itertools
import os
import subprocess

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    so = tmp_path_factory.mktemp("probe") / "sort_probe.so"
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-fmad=false",
                           "-std=c++17", "-Xcompiler", "-fPIC", "-shared", "-cudart", "shared",
                           "-I", os.path.join(ROOT, "paper_1711_05683_b300", "csrc"),
                           "-I", os.path.join(ROOT, "include"), "-o", str(so),
                           os.path.join(ROOT, "tests", "gpu_probes", "sort_probe.cu")])
    lib = ctypes.CDLL(str(so))
    lib.probe_sort.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]
    return lib


def _sorted_on_gpu(probe, rows):
    rows = np.ascontiguousarray(rows, dtype=np.uint32)
    out = np.empty_like(rows)
    assert probe.probe_sort(rows.shape[1], rows.ctypes.data, rows.shape[0], out.ctypes.data) == 0
    return out


@pytest.mark.parametrize("k", range(1, 9))
def test_sort_network(probe, k):
    binary = np.array(list(itertools.product((0, 1), repeat=k)), dtype=np.uint32)
    perms = np.array(list(itertools.permutations(range(k))), dtype=np.uint32) * 977 + 3
    rng = np.random.default_rng(k)
    rand = rng.integers(0, 1 << 32, size=(20000, k), dtype=np.uint64).astype(np.uint32)
    ties = rng.integers(0, 3, size=(5000, k)).astype(np.uint32) * np.uint32(0x7FFFFFFF)  # 0, 2^31 - 1, 2^32 - 2
    ext = rng.choice(np.array([0, 1, 0xFFFFFFFE, 0xFFFFFFFF], dtype=np.uint32), size=(2000, k))
    for rows in (binary, perms, rand, ties, ext):
        assert np.array_equal(_sorted_on_gpu(probe, rows), np.sort(rows, axis=1))
