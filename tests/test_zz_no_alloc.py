"""The allocation-free kNN entry point (for callers that cannot allocate
device memory, e.g. hosts that own every device buffer or cannot afford a
synchronising cudaMalloc) must produce exactly the neighbour table of the
regular ngs_build_graph call, at every size up to its limit, without touching
the library's memory pool or the device's free memory.  Collected last on
purpose."""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import knn_agreement
from paper_2603_16103_gb300 import synth

pytestmark = pytest.mark.gpu

NOALLOC_MAX_N = 65536


def call_noalloc(lib, xyz, n, k, out):
    stream = torch.cuda.current_stream().cuda_stream
    return lib.ngs_knn_noalloc(ctypes.c_void_p(xyz.data_ptr()), n, k,
                               ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))


def pool_usage(lib):
    used, reserved = ctypes.c_int64(-1), ctypes.c_int64(-1)
    assert lib.ngs_pool_usage(torch.cuda.current_device(), ctypes.byref(used),
                              ctypes.byref(reserved)) == 0
    return used.value, reserved.value


def reference_table(ngs, ds, k):
    c = ngs.Context(k=k)
    try:
        g, ref, lo, hi = c.build_graph(ds)
        return ref.clone()
    finally:
        c.close()


def test_knn_noalloc_matches_build_graph_twice(ngs):
    lib = ngs.load()
    for seed, n, k in ((21, 20000, 16), (22, 3001, 8)):   # two calls in a row
        scene = synth.surfaces_unit_cube(n, seed=seed)
        ds = ngs.DeviceSplats.from_numpy(scene)
        ref = reference_table(ngs, ds, k)
        out = torch.full((n, k), -7, dtype=torch.int32, device="cuda")
        assert call_noalloc(lib, ds.xyz, n, k, out) == 0, ngs.ngs_last_error()
        torch.cuda.synchronize()
        assert torch.equal(out, ref)


@pytest.mark.parametrize("n,k", [(NOALLOC_MAX_N, 32), (2, 1)])
def test_knn_noalloc_extremes(ngs, n, k):
    """The largest accepted input (the fixed cell table, sort histograms and
    scan partials exactly at their bound) and the smallest with a neighbour."""
    lib = ngs.load()
    scene = synth.patches_cube(n, seed=23, frac_degenerate=0.05, frac_duplicate=0.01) \
        if n > 100 else synth.surfaces_unit_cube(n, seed=23)
    ds = ngs.DeviceSplats.from_numpy(scene)
    ref = reference_table(ngs, ds, k)
    ke = min(k, n - 1)
    out = torch.full((n, ke), -7, dtype=torch.int32, device="cuda")
    assert call_noalloc(lib, ds.xyz, n, k, out) == 0, ngs.ngs_last_error()
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    got = out.cpu().numpy()
    orc = O.knn(scene.xyz, k, "grid")
    assert knn_agreement(scene.xyz, got, orc) <= max(2, n // 2000)


def test_knn_noalloc_allocates_nothing(ngs):
    """After one call (kernels loaded), a second call leaves the library's
    pool and the device's free memory exactly as they were."""
    lib = ngs.load()
    n, k = 50000, 16
    scene = synth.surfaces_unit_cube(n, seed=24)
    ds = ngs.DeviceSplats.from_numpy(scene)
    out = torch.zeros((n, k), dtype=torch.int32, device="cuda")
    assert call_noalloc(lib, ds.xyz, n, k, out) == 0, ngs.ngs_last_error()
    torch.cuda.synchronize()
    first = out.clone()
    pool0 = pool_usage(lib)
    free0 = torch.cuda.mem_get_info()[0]
    out.fill_(-7)
    assert call_noalloc(lib, ds.xyz, n, k, out) == 0, ngs.ngs_last_error()
    torch.cuda.synchronize()
    assert pool_usage(lib) == pool0
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.equal(out, first)


def test_knn_noalloc_limits(ngs):
    lib = ngs.load()
    n = NOALLOC_MAX_N + 1
    xyz = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    out = torch.zeros((n, 16), dtype=torch.int32, device="cuda")
    assert call_noalloc(lib, xyz, n, 16, out) == ngs.NGS_ERR_INVALID_ARG
    assert str(NOALLOC_MAX_N) in ngs.ngs_last_error()
    assert call_noalloc(lib, xyz, 1, 16, out) == 0       # nothing to do
    bad = torch.tensor([[0.0, 0.0, 0.0], [float("nan"), 1.0, 2.0]], device="cuda")
    assert call_noalloc(lib, bad, 2, 1, out) == ngs.NGS_ERR_INVALID_ARG
