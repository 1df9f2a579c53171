"""CUDA path vs the FP64 oracle, stage by stage, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import (ATTR_RTOL, COST_TOL, cost_excess, greedy_certificate, knn_agreement, sigma_of,
                      small_scene, stepwise)
from paper_2603_16103_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture
def ctx(ngs):
    c = ngs.Context()
    yield c
    c.close()


def dev(ngs, scene):
    return ngs.DeviceSplats.from_numpy(scene)


@pytest.mark.parametrize("n,kind,k", [(20000, "unit", 16), (9001, "patch", 16), (4000, "unit", 5),
                                      (2000, "patch", 32), (3000, "unit", 4), (3500, "patch", 8),
                                      (40, "unit", 16), (17, "unit", 16), (2, "unit", 16),
                                      (3, "unit", 16), (6, "unit", 2)])
def test_knn_and_edges(ngs, n, kind, k):
    scene = small_scene(n, seed=n, kind=kind)
    c = ngs.Context(k=k)
    try:
        ds = dev(ngs, scene)
        g, nbr, lo, hi = c.build_graph(ds)
        ref = O.knn(scene.xyz, k)
        nbr = nbr.cpu().numpy()
        assert nbr.shape == ref.shape
        differ = knn_agreement(scene.xyz, nbr, ref)
        assert differ <= max(2, n // 2000)
        rlo, rhi = O.union_edges(nbr)       # union of the GPU's own lists: exact
        assert np.array_equal(lo.cpu().numpy(), rlo) and np.array_equal(hi.cpu().numpy(), rhi)
        assert g.n_edges == len(rlo)
    finally:
        c.close()


def test_knn_duplicates_and_ties(ngs, ctx):
    rng = np.random.default_rng(3)
    base = synth.surfaces_unit_cube(600, seed=3)
    idx = np.concatenate([np.arange(600), rng.integers(0, 600, 300), rng.integers(0, 600, 100)])
    scene = base.subset(idx)
    scene.xyz[600:700] = scene.xyz[0]        # a 101-fold stack at one point
    g, nbr, lo, hi = ctx.build_graph(dev(ngs, scene))
    ref = O.knn(scene.xyz, 16)
    assert np.array_equal(nbr.cpu().numpy(), ref)   # exact ties break by index on both sides


def test_edge_costs(ngs, ctx):
    scene = small_scene(20000, seed=0)
    ds = dev(ngs, scene)
    g, nbr, lo, hi = ctx.build_graph(ds)
    for p in (0, 3):
        cost = ctx.edge_costs(ds, g, p).cpu().numpy().astype(np.float64)
        z, u = O.mc_draws(0, p, 1)
        ref = O.edge_costs(scene, lo.cpu().numpy(), hi.cpu().numpy(), z, u)
        print("cost error / contract: max %.3g" % cost_excess(cost, ref))
        assert np.all(np.isfinite(cost))
        assert cost_excess(cost, ref) <= 1.0


def test_edge_costs_degenerate_and_modes(ngs):
    scene = small_scene(9001, seed=7, kind="patch")
    for mode, S in ((0, 1), (0, 4), (1, 1), (1, 3), (2, 1), (2, 8), (3, 1), (0, 128)):
        c = ngs.Context(cost_mode=mode, mc_samples=S, seed=11)
        try:
            ds = dev(ngs, scene)
            g, nbr, lo, hi = c.build_graph(ds)
            cost = c.edge_costs(ds, g, 2).cpu().numpy().astype(np.float64)
            z, u = O.mc_draws(11, 2, S)
            ref = O.edge_costs(scene, lo.cpu().numpy(), hi.cpu().numpy(), z, u, mode=mode)
            print(mode, S, "cost error / contract: max %.3g" % cost_excess(cost, ref))
            # every edge, every mode: the FP32 costs kept are within the
            # contract, the others extended precision, float-float by default
            # (mode 1 included: a draw u_s within FP32 reach of pi goes there)
            assert cost_excess(cost, ref) <= 1.0
        finally:
            c.close()


def test_refined_costs_match_fp64(ngs):
    """Edges whose cost differs between cost_tol = 0 (FP32 as computed; the
    extended path only for near-degenerate merged covariances) and the default
    contract were evaluated in extended precision (float-float by default;
    error estimate or near tie): they equal the oracle's FP64 cost rounded to
    FP32, within one FP32 spacing."""
    scene = small_scene(9001, seed=7, kind="patch")
    costs = {}
    for tol in (0.0, COST_TOL):
        c = ngs.Context(cost_tol=tol, seed=11)
        try:
            ds = dev(ngs, scene)
            g, nbr, lo, hi = c.build_graph(ds)
            costs[tol] = c.edge_costs(ds, g, 2).cpu().numpy()
        finally:
            c.close()
    z, u = O.mc_draws(11, 2, 1)
    ref = O.edge_costs(scene, lo.cpu().numpy(), hi.cpu().numpy(), z, u)
    changed = costs[0.0] != costs[COST_TOL]
    print("edges evaluated in extended precision beyond the pivot rule:", int(changed.sum()), "of", len(ref))
    assert changed.any()
    got = costs[COST_TOL][changed].astype(np.float64)
    r = ref[changed]
    assert np.all(np.abs(got - r) <= np.spacing(np.abs(r).astype(np.float32)).astype(np.float64))


@pytest.mark.parametrize("cap_frac", [None, 0.3, 0.05])
def test_select_pairs_equals_greedy_on_gpu_costs(ngs, ctx, cap_frac):
    scene = small_scene(20000, seed=1)
    ds = dev(ngs, scene)
    g, nbr, lo, hi = ctx.build_graph(ds)
    cost = ctx.edge_costs(ds, g, 0)
    n = scene.n
    P = n if cap_frac is None else int(cap_frac * n)
    pairs = ctx.select_pairs(g, cost, P).cpu().numpy()
    rlo, rhi = O.greedy(n, lo.cpu().numpy(), hi.cpu().numpy(),
                        cost.cpu().numpy().astype(np.float64), P)
    ref = np.stack([rlo, rhi], 1)
    ref = ref[np.argsort(ref[:, 0])]
    assert np.array_equal(pairs, ref)


def test_select_pairs_certificate_against_fp64_costs(ngs, ctx):
    scene = small_scene(20000, seed=2)
    ds = dev(ngs, scene)
    g, nbr, lo, hi = ctx.build_graph(ds)
    pairs = ctx.select_pairs(g, ctx.edge_costs(ds, g, 0), scene.n).cpu().numpy()
    z, u = O.mc_draws(0, 0, 1)
    ref = O.edge_costs(scene, lo.cpu().numpy(), hi.cpu().numpy(), z, u)
    bad = greedy_certificate(scene.n, lo.cpu().numpy(), hi.cpu().numpy(), ref, pairs, rel=1e-6)
    assert bad == 0


def test_select_pairs_ties_and_nan(ngs, ctx):
    scene = small_scene(3000, seed=4)
    ds = dev(ngs, scene)
    g, nbr, lo, hi = ctx.build_graph(ds)
    rng = np.random.default_rng(0)
    c = rng.integers(0, 4, g.n_edges).astype(np.float32)     # massive exact ties
    c[rng.integers(0, g.n_edges, 50)] = np.nan
    c[rng.integers(0, g.n_edges, 50)] = -0.0
    ct = torch.from_numpy(c).cuda()
    pairs = ctx.select_pairs(g, ct, scene.n).cpu().numpy()
    rlo, rhi = O.greedy(scene.n, lo.cpu().numpy(), hi.cpu().numpy(), c.astype(np.float64), scene.n)
    ref = np.stack([rlo, rhi], 1)
    assert np.array_equal(pairs, ref[np.argsort(ref[:, 0])])


def check_merge(scene, pairs, got):
    ref = O.merge_compact(scene, pairs[:, 0], pairs[:, 1])
    assert got[0].shape[0] == ref[0].shape[0]
    merged = np.zeros(scene.n, bool)
    merged[pairs[:, 0]] = True
    keep = np.ones(scene.n, bool)
    keep[pairs[:, 1]] = False
    m = merged[keep]           # rows of the output that are merges
    # unmerged rows: exact copies
    for a, b in zip(got, ref):
        assert np.array_equal(a[~m].astype(np.float64), b[~m])
    xyz, ls, rot, logit, sh = got
    rxyz, rls, rrot, rlogit, rsh = ref
    i, j = pairs[:, 0], pairs[:, 1]
    span = np.linalg.norm(scene.xyz[i].astype(np.float64) - scene.xyz[j], axis=1) + \
        np.exp(scene.log_scale[i].astype(np.float64)).max(1)
    # relative to the pair's extent, plus the FP32 spacing of the coordinate itself
    eps32 = np.finfo(np.float32).eps
    assert np.all(np.linalg.norm(xyz[m] - rxyz[m], axis=1) <=
                  ATTR_RTOL * span + 4 * eps32 * np.linalg.norm(rxyz[m], axis=1))
    S, RS = sigma_of(ls[m], rot[m]), sigma_of(rls[m], rrot[m])
    nrm = np.linalg.norm(RS, axis=(1, 2))
    assert np.all(np.linalg.norm(S - RS, axis=(1, 2)) <= ATTR_RTOL * nrm)
    fs = np.abs(scene.sh[i].astype(np.float64)) + np.abs(scene.sh[j])
    assert np.all(np.abs(sh[m] - rsh[m]) <= ATTR_RTOL * fs + 1e-7)
    a, ra = 1 / (1 + np.exp(-logit[m].astype(np.float64))), 1 / (1 + np.exp(-rlogit[m]))
    assert np.all(np.abs(a - ra) <= ATTR_RTOL * ra)


def test_merge_compact_oracle_pairs(ngs, ctx):
    scene = small_scene(20000, seed=0, kind="patch")
    nbr = O.knn(scene.xyz, 16, "grid")
    lo, hi = O.union_edges(nbr)
    z, u = O.mc_draws(0, 0, 1)
    c = O.edge_costs(scene, lo, hi, z, u)
    plo, phi = O.greedy(scene.n, lo, hi, c, scene.n)
    pairs = np.stack([plo, phi], 1).astype(np.int32)
    pairs = pairs[np.argsort(pairs[:, 0])]
    ds = dev(ngs, scene)
    nn = ctx.merge_compact(ds, torch.from_numpy(pairs).cuda())
    assert nn == scene.n - len(pairs)
    check_merge(scene, pairs, ds.numpy())


def test_merge_compact_rejects_bad_pairs(ngs, ctx):
    scene = small_scene(100, seed=0)
    ds = dev(ngs, scene)
    before = [a.clone() for a in ds.tensors()]
    for bad in ([[5, 5]], [[7, 3]], [[1, 2], [2, 9]], [[0, 100]], [[-1, 4]]):
        with pytest.raises(ngs.NgsError):
            ctx.merge_compact(ds, torch.tensor(bad, dtype=torch.int32).cuda())
        assert ds.n == 100
        for a, b in zip(before, ds.tensors()):
            assert torch.equal(a, b)


def test_prefilter(ngs, ctx):
    for n, shift in ((20000, 0.0), (1001, -9.0), (2, -9.0), (1, 0.0)):
        scene = small_scene(max(n, 3), seed=n).subset(np.arange(n))
        scene.logit = (scene.logit + shift).astype(np.float32)
        ds = dev(ngs, scene)
        kept = ctx.prefilter(ds)
        keep, cnt = O.prefilter(scene.logit)
        assert kept == cnt
        assert np.array_equal(ds.numpy()[0], scene.xyz[keep])
        assert np.array_equal(ds.numpy()[4], scene.sh[keep])


@pytest.mark.parametrize("n,ratio,kind", [(20000, 0.5, "unit"), (9001, 0.1, "patch"),
                                          (500, 0.01, "unit"), (64, 0.5, "patch")])
def test_simplify_equals_stepwise(ngs, ctx, n, ratio, kind):
    scene = small_scene(n, seed=n, kind=kind)
    target = O.target_count(n, ratio)
    ds = dev(ngs, scene)
    st = ctx.simplify(ds, target)
    ref, passes = stepwise(ngs, ctx, scene, target)
    assert st["passes"] == passes
    assert ds.n == ref.n
    for a, b in zip(ds.numpy(), ref.numpy()):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("k", [4, 8, 32, 5])
def test_simplify_equals_stepwise_other_k(ngs, k):
    """Every k the graph builder specialises (whole rows per warp for 4, 8, 32)
    and one it does not (5)."""
    scene = small_scene(6000, seed=60 + k, kind="patch")
    target = O.target_count(scene.n, 0.25)
    with ngs.Context(k=k) as c:
        ds = dev(ngs, scene)
        st = c.simplify(ds, target)
        ref, passes = stepwise(ngs, c, scene, target)
    assert st["passes"] == passes and ds.n == ref.n
    for a, b in zip(ds.numpy(), ref.numpy()):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("mode,S", [(2, 1), (3, 1), (2, 8)])
def test_simplify_equals_stepwise_cost_modes(ngs, mode, S):
    """The closed-form cross-entropy and MSE-surrogate costs through the whole
    loop: the one-call path equals the per-step C-ABI calls."""
    scene = small_scene(8000, seed=70 + mode, kind="patch")
    target = O.target_count(scene.n, 0.1)
    with ngs.Context(cost_mode=mode, mc_samples=S) as c:
        ds = dev(ngs, scene)
        st = c.simplify(ds, target)
        ref, passes = stepwise(ngs, c, scene, target)
    assert st["passes"] == passes and ds.n == ref.n
    for a, b in zip(ds.numpy(), ref.numpy()):
        assert np.array_equal(a, b)


def test_simplify_counts_vs_oracle(ngs, ctx):
    scene = small_scene(20000, seed=0)
    target = O.target_count(scene.n, 0.5)
    ds = dev(ngs, scene)
    st = ctx.simplify(ds, target)
    ref, rst = O.simplify(scene, target)
    assert st["n_filtered"] == rst["n"][0]
    assert ds.n == target == ref[0].shape[0]
    assert st["pass_n"][0] == rst["n"][0]


def test_simplify_pass0_lockstep(ngs, ctx):
    """First pass on the same input: pair set bit-identical to the oracle when
    the oracle's matcher gets the GPU's costs, and merged rows within tolerance."""
    scene = small_scene(20000, seed=6, kind="patch")
    ds = dev(ngs, scene)
    ctx.prefilter(ds)
    cur = synth.Scene(*ds.numpy())
    g, nbr, lo, hi = ctx.build_graph(ds)
    cost = ctx.edge_costs(ds, g, 0)
    pairs = ctx.select_pairs(g, cost, cur.n // 2)
    rlo, rhi = O.greedy(cur.n, lo.cpu().numpy(), hi.cpu().numpy(),
                        cost.cpu().numpy().astype(np.float64), cur.n // 2)
    ref = np.stack([rlo, rhi], 1)
    assert np.array_equal(pairs.cpu().numpy(), ref[np.argsort(ref[:, 0])])
    p = pairs.cpu().numpy()
    ctx.merge_compact(ds, pairs)
    check_merge(cur, p, ds.numpy())


def test_edge_cases(ngs, ctx):
    scene = small_scene(50, seed=9)
    for n in (0, 1, 2):
        s = scene.subset(np.arange(n))
        ds = dev(ngs, s) if n else ngs.DeviceSplats(*(torch.zeros((0,) + a.shape[1:], dtype=torch.float32, device="cuda")
                                                        for a in scene.arrays()))
        st = ctx.simplify(ds, 1)
        assert ds.n == min(n, 1) or (n == 2 and ds.n in (1, 2))
    ds = dev(ngs, scene)
    st = ctx.simplify(ds, 1000)            # target above n: prefilter only
    assert st["passes"] == 0 and ds.n == O.prefilter(scene.logit)[1]
    ds = dev(ngs, scene)
    st = ctx.simplify(ds, 1)               # down to one splat
    assert ds.n == 1
    with pytest.raises(ngs.NgsError):
        ctx.simplify(dev(ngs, scene), 0)
    bad = scene.copy()
    bad.xyz[3, 1] = np.nan
    with pytest.raises(ngs.NgsError):
        ctx.simplify(dev(ngs, bad), 10)


def test_simplify_host_api(ngs, ctx):
    scene = small_scene(5000, seed=12)
    target = O.target_count(scene.n, 0.25)
    hs = ngs.DeviceSplats.from_numpy(scene, device="cpu", pin=True)
    st = ctx.simplify_host(hs, target)
    ds = dev(ngs, scene)
    ctx.simplify(ds, target)
    assert hs.n == ds.n == target
    for a, b in zip(hs.numpy(), ds.numpy()):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("F", [48, 12, 5, 3])
def test_simplify_host_equals_device(ngs, F):
    """Host buffers, uploaded in pieces on two streams (opacities and centres,
    then scales and rotations, then SH), give the device path's result, for SH
    widths whose rows the engine gathers late (48, 12) and at once (5, 3)."""
    scene = small_scene(300000, seed=13, kind="patch")
    rng = np.random.default_rng(F)
    scene.sh = rng.normal(0, 0.3, (scene.n, F)).astype(np.float32)
    target = O.target_count(scene.n, 0.1)
    with ngs.Context() as c:
        hs = ngs.DeviceSplats.from_numpy(scene, device="cpu", pin=True)
        for _ in range(2):   # a second call reuses the staging buffers
            hs = ngs.DeviceSplats.from_numpy(scene, device="cpu", pin=True)
            c.simplify_host(hs, target)
        ds = dev(ngs, scene)
        c.simplify(ds, target)
    assert hs.n == ds.n
    for a, b in zip(hs.numpy(), ds.numpy()):
        assert np.array_equal(a, b)


def test_scan_wait_budget_runs_out_and_ctx_stays_usable(ngs):
    """The single-pass scan's look-back waits are bounded: with one tile made
    to publish 4 budgets late, its successor gives up, completes the prefix
    from the inputs, and the call returns NGS_ERR_TIMEOUT without a hang; the
    same ctx then runs normally and matches a fresh one bit for bit."""
    scene = small_scene(200000, seed=12)
    target = O.target_count(scene.n, 0.5)
    c = ngs.Context()
    try:
        c.set_tuning(scan_method=1, wait_budget_cycles=2000, wait_test_tile=1)
        with pytest.raises(ngs.NgsError) as e:
            c.simplify(ngs.DeviceSplats.from_numpy(scene), target)
        assert e.value.code == ngs.NGS_ERR_TIMEOUT
        d = ngs.ngs_default_tuning()
        c.set_tuning(wait_budget_cycles=d.wait_budget_cycles, wait_test_tile=-1)   # scan_method stays 1
        ds = ngs.DeviceSplats.from_numpy(scene)
        c.simplify(ds, target)
        got = ds.numpy()
    finally:
        c.close()
    with ngs.Context() as f:
        ref = ngs.DeviceSplats.from_numpy(scene)
        f.simplify(ref, target)
        for a, b in zip(got, ref.numpy()):
            assert np.array_equal(a, b)


def test_scan_methods_give_identical_results(ngs):
    """The single-pass scan (decoupled look-back) and the three-kernel scan
    are exact: the whole loop gives the same splats with either."""
    scene = small_scene(150000, seed=14, kind="patch")
    target = O.target_count(scene.n, 0.1)
    outs = []
    for method in (0, 1):
        with ngs.Context() as c:
            c.set_tuning(scan_method=method)
            ds = ngs.DeviceSplats.from_numpy(scene)
            c.simplify(ds, target)
            outs.append(ds.numpy())
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
