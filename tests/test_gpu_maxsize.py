"""The largest scene one call accepts: NGS_MAX_N = 2^26 splats at k = 16, so
n * k = 2^30 list slots, the limit of the library's int32 slot indices.

The scene is the patches recipe drawn on the device (5 % near-degenerate
splats, 1 % duplicated centres).  Checked at that size:

* the one-call loop (the engine) equal bit for bit to the per-step calls
  down to 10 %, reaching the target exactly;
* first pass: sampled neighbour lists against the oracle's brute force; the
  edge set equal to the union of all lists (an independent torch sort of all
  2^30 directed pairs); sampled edge costs and merged rows against the FP64
  oracle; the whole pair set certified as the greedy matching of the GPU's
  costs under (cost, lo, hi).
"""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import check_merge_rows, cost_excess, knn_agreement
from paper_2603_16103_gb300 import synth

pytestmark = pytest.mark.gpu

RATIO = 0.1


@pytest.fixture(scope="module")
def pristine(ngs):
    arrays = synth.patches_cube_device(ngs.NGS_MAX_N, 5, frac_degenerate=0.05, frac_duplicate=0.01)
    return ngs.DeviceSplats(*arrays)


def test_max_engine_equals_stepwise(ngs, pristine):
    target = O.target_count(pristine.n, RATIO)
    with ngs.Context() as c:
        ds = pristine.clone()
        st = c.simplify(ds, target)
        ref = pristine.clone()
        c.prefilter(ref)
        p = 0
        while ref.n > target and p < 64:
            g, _, _, _ = c.build_graph(ref)
            cost = c.edge_costs(ref, g, p)
            pairs = c.select_pairs(g, cost, ref.n - target)
            p += 1
            if pairs.shape[0] == 0:
                break
            c.merge_compact(ref, pairs)
            del g, cost, pairs
    assert st["passes"] == p and ds.n == ref.n == target
    for a, b in zip(ds.tensors(), ref.tensors()):
        assert torch.equal(a[:ds.n], b[:ref.n])
    del ds, ref
    torch.cuda.empty_cache()


@pytest.fixture(scope="module")
def pass0(ngs, pristine):
    target = O.target_count(pristine.n, RATIO)
    with ngs.Context() as c:
        ds = pristine.clone()
        c.prefilter(ds)
        pre = ds.clone()
        g, nbr, lo, hi = c.build_graph(ds)
        cost = c.edge_costs(ds, g, 0)
        P = ds.n - target
        pairs = c.select_pairs(g, cost, P)
        c.merge_compact(ds, pairs)
    torch.cuda.synchronize()
    return dict(pre=pre, n=pre.n, nbr=nbr, lo=lo, hi=hi, cost=cost, pairs=pairs, P=P, merged=ds)


def _sub_scene(pre, rows):
    """Rows of the device splats `pre` as a host scene."""
    r = rows.long()
    return synth.Scene(*(a[r].cpu().numpy() for a in pre.tensors()))


def test_max_sampled_neighbour_lists(pass0):
    n = pass0["n"]
    xyz = pass0["pre"].xyz[:n].cpu().numpy()
    rows = np.random.default_rng(71).choice(n, 48, replace=False)
    ref = O.knn(xyz, 16, queries=rows)
    got = pass0["nbr"][torch.as_tensor(rows, device="cuda")].cpu().numpy()
    assert knn_agreement(xyz, got, ref, rows=rows) <= 1


def test_max_edges_are_the_union_of_the_lists(pass0):
    n, nbr = pass0["n"], pass0["nbr"]
    u = nbr.long()
    v = torch.arange(n, device=u.device).unsqueeze(1)
    keys = torch.minimum(u, v).mul_(n).add_(torch.maximum(u, v)).view(-1)
    del u
    union = torch.unique(keys)
    del keys
    got = pass0["lo"].long().mul_(n).add_(pass0["hi"].long())
    assert torch.equal(union, got)
    del union, got
    torch.cuda.empty_cache()


def test_max_sampled_edge_costs(pass0):
    lo, hi = pass0["lo"], pass0["hi"]
    m = 20000
    e = torch.as_tensor(np.random.default_rng(72).choice(lo.numel(), m, replace=False), device="cuda")
    sub = _sub_scene(pass0["pre"], torch.stack([lo[e], hi[e]], 1).view(-1))
    z, u = O.mc_draws(0, 0, 1)
    ref = O.edge_costs(sub, np.arange(0, 2 * m, 2), np.arange(1, 2 * m, 2), z, u)
    got = pass0["cost"][e].cpu().numpy().astype(np.float64)
    assert cost_excess(got, ref) <= 1.0


def _order_key(cost):
    """Cost as an orderable unsigned key (NaN ranked as +inf, -0 as +0)."""
    c = torch.where(torch.isnan(cost), torch.full_like(cost, float("inf")), cost)
    c = torch.where(c == 0, torch.zeros_like(c), c)
    b = c.view(torch.int32).long() & 0xFFFFFFFF
    return torch.where(b >= 0x80000000, (~b) & 0xFFFFFFFF, b | 0x80000000)


def test_max_pairs_greedy_certificate(pass0):
    """The pair set is the greedy matching of the GPU's costs under the strict
    order (cost, lo, hi): a matching, each pair an edge, and every other edge
    touching a pair that precedes it (which also makes it maximal)."""
    n, lo, hi, pairs = pass0["n"], pass0["lo"], pass0["hi"], pass0["pairs"]
    assert 0 < pairs.shape[0] < pass0["P"]          # uncapped: the whole matching
    a, b = pairs[:, 0].long(), pairs[:, 1].long()
    assert bool((a < b).all())
    assert torch.unique(pairs.view(-1)).numel() == 2 * pairs.shape[0]
    ekey = lo.long() * n + hi.long()
    pkey = a * n + b
    at = torch.searchsorted(ekey, pkey)
    assert bool((at < ekey.numel()).all()) and torch.equal(ekey[at], pkey)
    ck = _order_key(pass0["cost"])
    big = torch.iinfo(torch.int64).max
    pc = torch.full((n,), big, dtype=torch.int64, device="cuda")
    pl = torch.zeros(n, dtype=torch.int64, device="cuda")
    mate = torch.full((n,), -1, dtype=torch.int64, device="cuda")
    pc[a] = pc[b] = ck[at]
    pl[a] = pl[b] = pkey
    mate[a], mate[b] = b, a
    del at
    bad = 0
    step = 1 << 27
    for s in range(0, ekey.numel(), step):
        el, eh = lo[s:s + step].long(), hi[s:s + step].long()
        ec, ek = ck[s:s + step], ekey[s:s + step]
        member = mate[el] == eh
        before = torch.zeros_like(member)
        for v in (el, eh):
            c1, l1 = pc[v], pl[v]
            before |= (c1 < ec) | ((c1 == ec) & (l1 < ek))
        bad += int((~member & ~before).sum())
    assert bad == 0


def test_max_merged_rows(pass0):
    n, pairs, pre, merged = pass0["n"], pass0["pairs"], pass0["pre"], pass0["merged"]
    m = 20000
    sel = np.sort(np.random.default_rng(73).choice(pairs.shape[0], m, replace=False))
    sub = pairs[torch.as_tensor(sel, device="cuda")].long()
    # the merged splat sits at the lower row, shifted down by the removed
    # higher rows before it
    removed = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    removed[pairs[:, 1].long() + 1] = 1
    shift = torch.cumsum(removed, 0)[:-1]
    idx = sub[:, 0] - shift[sub[:, 0]]
    got = tuple(t[idx].cpu().numpy() for t in merged.tensors())
    cur = _sub_scene(pre, sub.reshape(-1))
    local = np.stack([np.arange(0, 2 * m, 2), np.arange(1, 2 * m, 2)], 1)
    ref = O.merge_compact(cur, local[:, 0], local[:, 1])
    check_merge_rows(cur, local, got, ref)
