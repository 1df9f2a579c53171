"""Local neighbourhood refresh (Sec. 3.4) on the GPU against the oracle's
refresh step, in lockstep: pass 0 through the per-step C-ABI calls, then the
graph of pass 1 by ngs_build_graph_refresh from pass 0's lists and pairs,
compared with oracle.refresh_lists on the GPU's own pass-1 input; and the
one-call loop with a refresh period equal bit for bit to the per-step calls."""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import knn_agreement, small_scene
from paper_2603_16103_gb300 import synth

pytestmark = pytest.mark.gpu


def _pass0(ngs, c, scene, target):
    ds = ngs.DeviceSplats.from_numpy(scene)
    c.prefilter(ds)
    g, nbr, lo, hi = c.build_graph(ds)
    cost = c.edge_costs(ds, g, 0)
    pairs = c.select_pairs(g, cost, ds.n - target)
    c.merge_compact(ds, pairs)
    return ds, nbr, pairs


@pytest.mark.parametrize("n,kind,k,ratio", [(20000, "unit", 16, 0.5), (9001, "patch", 16, 0.1),
                                            (3000, "unit", 8, 0.3), (2500, "patch", 5, 0.5)])
def test_refresh_graph_matches_oracle(ngs, n, kind, k, ratio):
    scene = small_scene(n, seed=n + 1, kind=kind)
    c = ngs.Context(k=k)
    try:
        target = O.target_count(scene.n, ratio)
        ds, nbr0, pairs = _pass0(ngs, c, scene, target)
        g, nbr1, lo, hi, nq = c.build_graph_refresh(ds, nbr0, pairs)
        cur = ds.numpy()
        p = pairs.cpu().numpy()
        ref, rq = O.refresh_lists(nbr0.cpu().numpy(), p[:, 0], p[:, 1], cur[0], k)
        got = nbr1.cpu().numpy()
        assert nq == int(rq.sum())
        print(f"n={ds.n}: {nq} of {ds.n} rows queried anew ({nq / ds.n:.1%})")
        # carried rows: the same neighbours (the order by distance may differ
        # only where FP64 distances are within 1e-6)
        keep = ~rq
        assert np.array_equal(np.sort(got[keep], 1), np.sort(ref[keep], 1))
        rows = np.nonzero(keep)[0]
        assert knn_agreement(cur[0], got[keep], ref[keep], rows=rows) <= max(2, len(rows) // 2000)
        # queried rows: the exact kNN
        qr = np.nonzero(rq)[0]
        assert knn_agreement(cur[0], got[rq], ref[rq], rows=qr) <= max(2, len(qr) // 2000)
        # the edges are the union of the GPU's lists
        rlo, rhi = O.union_edges(got)
        assert np.array_equal(lo.cpu().numpy(), rlo) and np.array_equal(hi.cpu().numpy(), rhi)
    finally:
        c.close()


def test_refresh_rejects_bad_input(ngs):
    scene = small_scene(2000, seed=5)
    c = ngs.Context()
    try:
        ds, nbr0, pairs = _pass0(ngs, c, scene, 1000)
        bad = nbr0.clone()
        bad[3, 2] = nbr0.shape[0] + 7            # outside [0, n_old)
        with pytest.raises(ngs.NgsError):
            c.build_graph_refresh(ds, bad, pairs)
        with pytest.raises(ngs.NgsError):        # pairs that do not match the sizes
            c.build_graph_refresh(ds, nbr0, pairs[:-1])
    finally:
        c.close()


def _stepwise_refresh(ngs, c, scene, target, period, max_passes=64):
    ds = ngs.DeviceSplats.from_numpy(scene)
    c.prefilter(ds)
    p, prev, pairs, queried = 0, None, None, 0
    while ds.n > target and ds.n > 1 and p < max_passes:
        if period > 1 and p % period != 0 and prev is not None:
            g, nbr, lo, hi, nq = c.build_graph_refresh(ds, prev, pairs)
        else:
            g, nbr, lo, hi = c.build_graph(ds)
            nq = ds.n
        queried += nq
        cost = c.edge_costs(ds, g, p)
        pairs = c.select_pairs(g, cost, ds.n - target)
        p += 1
        if pairs.shape[0] == 0:
            break
        prev = nbr
        c.merge_compact(ds, pairs)
    return ds, p, queried


@pytest.mark.parametrize("n,kind,ratio,period", [(20000, "unit", 0.1, 2), (9001, "patch", 0.05, 3),
                                                 (6000, "unit", 0.2, 64)])
def test_engine_refresh_equals_stepwise(ngs, n, kind, ratio, period):
    scene = small_scene(n, seed=n + 3, kind=kind)
    target = O.target_count(scene.n, ratio)
    c = ngs.Context(refresh_period=period)
    try:
        ds = ngs.DeviceSplats.from_numpy(scene)
        st = c.simplify(ds, target)
        ref, passes, queried = _stepwise_refresh(ngs, c, scene, target, period)
    finally:
        c.close()
    assert st["passes"] == passes and ds.n == ref.n == target
    assert st["requeried_rows"] == queried <= sum(st["pass_n"])
    for a, b in zip(ds.numpy(), ref.numpy()):
        assert np.array_equal(a, b)


def test_refresh_period_one_is_the_rebuild(ngs):
    scene = small_scene(8000, seed=11)
    target = O.target_count(scene.n, 0.1)
    outs = []
    for period in (1, None):
        c = ngs.Context() if period is None else ngs.Context(refresh_period=period)
        try:
            ds = ngs.DeviceSplats.from_numpy(scene)
            st = c.simplify(ds, target)
            outs.append((ds.numpy(), st))
        finally:
            c.close()
    assert outs[0][1]["requeried_rows"] == sum(outs[0][1]["pass_n"])
    for a, b in zip(outs[0][0], outs[1][0]):
        assert np.array_equal(a, b)
