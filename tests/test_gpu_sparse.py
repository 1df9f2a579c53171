"""Parity on sparse scenes: the patch recipe with 100 k and 400 k splats in the
20 m cube (the batched workload's small scenes), where neighbour offsets are
an order of magnitude larger than the splats and about 2 % of the edges fail
the FP32 error estimate (against 0.2 % on the dense 6M scene).

First pass through the per-step C-ABI calls:
* every edge cost within the accuracy contract of the FP64 oracle;
* the pair set equal to the oracle's greedy on the GPU's costs, and certified
  as the greedy matching of the oracle's FP64 costs (zero violations beyond
  1e-6 relative);
* the extended-precision costs in float-float (default) within one FP32
  spacing of the same costs evaluated in FP64 (fp64_policy 3)."""
import numpy as np
import pytest

import oracle as O
from gpu_util import cost_excess, greedy_certificate_np
from paper_2603_16103_gb300 import synth

pytestmark = pytest.mark.gpu


def _pass0(ngs, scene, ratio, **params):
    target = O.target_count(scene.n, ratio)
    with ngs.Context(**params) as c:
        ds = ngs.DeviceSplats.from_numpy(scene)
        c.prefilter(ds)
        cur = synth.Scene(*ds.numpy())
        g, nbr, lo, hi = c.build_graph(ds)
        cost = c.edge_costs(ds, g, 0)
        pairs = c.select_pairs(g, cost, cur.n - target)
        return dict(cur=cur, lo=lo.cpu().numpy(), hi=hi.cpu().numpy(), cost=cost.cpu().numpy(),
                    pairs=pairs.cpu().numpy(), P=cur.n - target)


@pytest.fixture(scope="module", params=[(100_000, 0.0), (400_000, 0.05)],
                ids=["sparse100k", "sparse400k_degenerate"])
def sparse(ngs, request):
    n, frac = request.param
    scene = synth.patches_cube(n, seed=1003, frac_degenerate=frac)
    r0 = _pass0(ngs, scene, 0.1)
    r3 = _pass0(ngs, scene, 0.1, fp64_policy=3)
    z, u = O.mc_draws(0, 0, 1)
    c64 = O.edge_costs(r0["cur"], r0["lo"], r0["hi"], z, u)
    return r0, r3, c64


def test_sparse_costs_within_contract(sparse):
    r0, _, c64 = sparse
    assert cost_excess(r0["cost"], c64) <= 1.0


def test_sparse_pairs_exact_and_certified(sparse):
    r0, _, c64 = sparse
    cur, lo, hi = r0["cur"], r0["lo"], r0["hi"]
    rlo, rhi = O.greedy(cur.n, lo, hi, r0["cost"].astype(np.float64), r0["P"])
    ref = np.stack([rlo, rhi], 1)
    assert np.array_equal(r0["pairs"], ref[np.argsort(ref[:, 0])])
    if len(r0["pairs"]) < r0["P"]:  # uncapped: the whole matching is certified
        assert greedy_certificate_np(cur.n, lo, hi, c64, r0["pairs"], rel=1e-6) == 0


def test_sparse_float_float_matches_fp64(sparse):
    r0, r3, c64 = sparse
    assert np.array_equal(r0["lo"], r3["lo"]) and np.array_equal(r0["hi"], r3["hi"])
    a, b = r0["cost"], r3["cost"]
    fin = np.isfinite(b)
    assert np.array_equal(np.isfinite(a), fin)
    sp = np.spacing(np.abs(b[fin]).astype(np.float32))
    assert np.all(np.abs(a[fin] - b[fin]) <= sp)
    assert cost_excess(b, c64) <= 1.0
