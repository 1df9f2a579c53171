"""Parity at the full sizes of the workloads, in the launch configuration the
benchmark times (default parameters and tuning):

* the 1M-splat patch scene: every neighbour list against the FP64 oracle's
  grid search, and the pair set of the first pass against the oracle's greedy
  matching fed the GPU's costs (exact) and against FP64 costs (certificate);
* the 6M-splat benchmark scene (5 % near-degenerate splats, 1 % duplicated
  centres): sampled neighbour lists, every edge cost of the first pass against
  the FP64 oracle, the whole first-pass pair set against the oracle's greedy on
  the GPU's costs (exact) and on FP64 costs (certificate), sampled merged
  rows, and the one-call loop (the engine) equal bit for bit to the per-step
  calls down to 10 % and to 1 %.
"""
import numpy as np
import pytest

import oracle as O
from gpu_util import check_merge_rows, cost_excess, greedy_certificate_np as certificate, knn_agreement, stepwise
from paper_2603_16103_gb300 import synth

pytestmark = pytest.mark.gpu


def _pass0(ngs, scene, ratio):
    """Pre-filter, graph, costs, pairs and merge of the first pass through the
    per-step C-ABI calls; host copies of everything."""
    target = O.target_count(scene.n, ratio)
    with ngs.Context() as c:
        ds = ngs.DeviceSplats.from_numpy(scene)
        c.prefilter(ds)
        cur = synth.Scene(*ds.numpy())
        g, nbr, lo, hi = c.build_graph(ds)
        cost = c.edge_costs(ds, g, 0)
        pairs = c.select_pairs(g, cost, cur.n - target)
        out = dict(cur=cur, nbr=nbr.cpu().numpy(), lo=lo.cpu().numpy(), hi=hi.cpu().numpy(),
                   cost=cost.cpu().numpy(), pairs=pairs.cpu().numpy(), P=cur.n - target)
        c.merge_compact(ds, pairs)
        out["merged"] = ds.numpy()
    return out


@pytest.fixture(scope="module")
def run1m(ngs):
    return _pass0(ngs, synth.workload("patches1m"), 0.1)


@pytest.fixture(scope="module")
def scene6m():
    return synth.workload("patches6m")


@pytest.fixture(scope="module")
def run6m(ngs, scene6m):
    return _pass0(ngs, scene6m, 0.1)


def test_1m_all_neighbour_lists(run1m):
    cur = run1m["cur"]
    ref = O.knn(cur.xyz, 16, "grid")
    assert run1m["nbr"].shape == ref.shape
    differ = knn_agreement(cur.xyz, run1m["nbr"], ref)
    assert differ <= cur.n // 2000


def test_1m_pairs_exact_on_gpu_costs_and_certified_on_fp64(run1m):
    cur, lo, hi = run1m["cur"], run1m["lo"], run1m["hi"]
    rlo, rhi = O.greedy(cur.n, lo, hi, run1m["cost"].astype(np.float64), run1m["P"])
    ref = np.stack([rlo, rhi], 1)
    assert np.array_equal(run1m["pairs"], ref[np.argsort(ref[:, 0])])
    z, u = O.mc_draws(0, 0, 1)
    c64 = O.edge_costs(cur, lo, hi, z, u)
    assert cost_excess(run1m["cost"], c64) <= 1.0
    assert len(run1m["pairs"]) < run1m["P"]      # uncapped: the whole matching is certified
    # the FP64 greedy order wherever FP64 costs differ by more than 1e-6
    assert certificate(cur.n, lo, hi, c64, run1m["pairs"], rel=1e-6) == 0


def test_6m_sampled_neighbour_lists(run6m):
    cur = run6m["cur"]
    rows = np.random.default_rng(61).choice(cur.n, 300, replace=False)
    ref = O.knn(cur.xyz, 16, queries=rows)
    assert knn_agreement(cur.xyz, run6m["nbr"][rows], ref, rows=rows) <= 1


def test_6m_edges_are_the_union_of_the_lists(run6m):
    rlo, rhi = O.union_edges(run6m["nbr"])
    assert np.array_equal(run6m["lo"], rlo) and np.array_equal(run6m["hi"], rhi)


@pytest.fixture(scope="module")
def c64_6m(run6m):
    z, u = O.mc_draws(0, 0, 1)
    return O.edge_costs(run6m["cur"], run6m["lo"], run6m["hi"], z, u)


def test_6m_all_edge_costs(run6m, c64_6m):
    """All 54.6 M first-pass costs against the FP64 oracle, elementwise."""
    print("cost error / contract: max %.3g" % cost_excess(run6m["cost"], c64_6m))
    assert cost_excess(run6m["cost"], c64_6m) <= 1.0


def test_6m_pairs_certified_on_fp64_costs(run6m, c64_6m):
    """The whole first-pass pair set is the greedy matching of the FP64 costs
    wherever they differ by more than 1e-6 (uncapped pass)."""
    cur, lo, hi = run6m["cur"], run6m["lo"], run6m["hi"]
    assert len(run6m["pairs"]) < run6m["P"]
    assert certificate(cur.n, lo, hi, c64_6m, run6m["pairs"], rel=1e-6) == 0


def test_6m_pairs_exact_on_gpu_costs(run6m):
    cur, lo, hi = run6m["cur"], run6m["lo"], run6m["hi"]
    rlo, rhi = O.greedy(cur.n, lo, hi, run6m["cost"].astype(np.float64), run6m["P"])
    ref = np.stack([rlo, rhi], 1)
    assert np.array_equal(run6m["pairs"], ref[np.argsort(ref[:, 0])])


def test_6m_merged_rows(run6m):
    cur, pairs = run6m["cur"], run6m["pairs"]
    keep = np.random.default_rng(63).choice(len(pairs), 20000, replace=False)
    keep.sort()
    sub = pairs[keep]
    # the sampled pairs merged alone: rows of the other pairs stay as they are
    got_rows = _merged_rows(cur, pairs, run6m["merged"], sub)
    ref = O.merge_compact(cur, sub[:, 0], sub[:, 1])
    ref_rows = _merged_rows(cur, sub, ref, sub)
    check_merge_rows(cur, sub, got_rows, ref_rows)


def _merged_rows(cur, pairs_all, out, sub):
    """Rows of `out` (the result of merging `pairs_all`) that hold the pairs of
    `sub`: the merged splat sits at the lower row, shifted down by the removed
    higher rows before it."""
    removed = np.zeros(cur.n + 1, np.int64)
    removed[pairs_all[:, 1] + 1] = 1
    shift = np.cumsum(removed)[:-1]
    idx = sub[:, 0] - shift[sub[:, 0]]
    return tuple(a[idx] for a in out)


@pytest.mark.parametrize("ratio", [0.1, 0.01])
def test_6m_engine_equals_stepwise(ngs, scene6m, ratio):
    """Both targets of the benchmark scene: 600 k (4 passes) and 60 k."""
    scene = scene6m
    target = O.target_count(scene.n, ratio)
    with ngs.Context() as c:
        ds = ngs.DeviceSplats.from_numpy(scene)
        st = c.simplify(ds, target)
        ref, passes = stepwise(ngs, c, scene, target)
    assert st["passes"] == passes and ds.n == ref.n == target
    for a, b in zip(ds.numpy(), ref.numpy()):
        assert np.array_equal(a, b)
