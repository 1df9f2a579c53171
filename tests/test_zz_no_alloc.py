"""The allocation-free kNN entry point (for callers that cannot allocate
device memory, e.g. hosts that own every device buffer or cannot afford a
synchronising cudaMalloc) must produce exactly the neighbour table of the
regular ngs_build_graph call.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2603_16103_gb300 import synth

pytestmark = pytest.mark.gpu


def call_noalloc(lib, xyz, n, k, out):
    stream = torch.cuda.current_stream().cuda_stream
    return lib.ngs_knn_noalloc(ctypes.c_void_p(xyz.data_ptr()), n, k,
                               ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))


def test_knn_noalloc_matches_build_graph_twice(ngs):
    lib = ngs.load()
    ctx = ngs.Context()
    try:
        for seed, n, k in ((21, 20000, 16), (22, 3001, 8)):   # two calls in a row
            scene = synth.surfaces_unit_cube(n, seed=seed)
            ds = ngs.DeviceSplats.from_numpy(scene)
            c = ngs.Context(k=k)
            try:
                g, ref, lo, hi = c.build_graph(ds)
            finally:
                c.close()
            out = torch.full((n, k), -7, dtype=torch.int32, device="cuda")
            assert call_noalloc(lib, ds.xyz, n, k, out) == 0, ngs.ngs_last_error()
            torch.cuda.synchronize()
            assert torch.equal(out, ref)
    finally:
        ctx.close()


def test_knn_noalloc_limits(ngs):
    lib = ngs.load()
    n = 65537
    xyz = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    out = torch.zeros((n, 16), dtype=torch.int32, device="cuda")
    assert call_noalloc(lib, xyz, n, 16, out) == ngs.NGS_ERR_INVALID_ARG
    assert "65536" in ngs.ngs_last_error()
    assert call_noalloc(lib, xyz, 1, 16, out) == 0       # nothing to do
    bad = torch.tensor([[0.0, 0.0, 0.0], [float("nan"), 1.0, 2.0]], device="cuda")
    assert call_noalloc(lib, bad, 2, 1, out) == ngs.NGS_ERR_INVALID_ARG
