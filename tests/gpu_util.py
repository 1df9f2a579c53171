"""Shared checks for the GPU parity tests (compare CUDA results with the oracle)."""
import math

import numpy as np

from paper_2603_16103_gb300 import synth


def d2_fp64(xyz, i, js):
    x = xyz.astype(np.float64)
    return np.sum((x[js] - x[i]) ** 2, axis=1)


def knn_agreement(xyz, got, ref, rel=1e-6, rows=None):
    """Neighbour lists must be identical except where FP64 squared distances
    are within `rel` of each other (near ties may reorder or swap the last
    member).  Row r of `got` and `ref` is the list of point rows[r] (of point
    r when rows is None).  Returns the number of rows that differ (all
    explained)."""
    differ = 0
    for r in np.nonzero(np.any(got != ref, axis=1))[0]:
        differ += 1
        i = r if rows is None else int(rows[r])
        dg = d2_fp64(xyz, i, got[r])
        dr = d2_fp64(xyz, i, ref[r])
        assert len(set(got[r].tolist())) == got.shape[1], f"row {i}: duplicate neighbours"
        assert i not in set(got[r].tolist()), f"row {i}: self in list"
        scale = max(dr.max(), 1e-300)
        assert np.all(np.abs(np.sort(dg) - np.sort(dr)) <= rel * scale), \
            f"row {i}: neighbour distances differ beyond near-ties"
        assert np.all(np.diff(dg) >= -rel * scale), f"row {i}: order not by distance"
    return differ


def sigma_of(ls, rot):
    q = rot.astype(np.float64)
    q = q / np.linalg.norm(q, axis=-1, keepdims=True)
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    R = np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], -2)
    s2 = np.exp(2 * ls.astype(np.float64))
    return np.einsum("...ik,...k,...jk->...ij", R, s2, R)


def greedy_certificate(n, lo, hi, cost64, pairs, rel=1e-6):
    """`pairs` is a matching, and every non-member edge touches a member edge
    whose FP64 cost is not larger beyond `rel` -- i.e. `pairs` is the greedy
    matching for some order consistent with the FP64 costs up to near-ties.
    Also maximal: no edge has two free endpoints."""
    mate = -np.ones(n, dtype=np.int64)
    for a, b in pairs:
        assert mate[a] < 0 and mate[b] < 0, "not a matching"
        mate[a], mate[b] = b, a
    pc = {}
    key = {(int(a), int(b)): float(c) for a, b, c in zip(lo, hi, cost64)}
    for a, b in pairs:
        pc[int(a)] = pc[int(b)] = key[(int(min(a, b)), int(max(a, b)))]
    bad = 0
    for a, b, c in zip(lo.tolist(), hi.tolist(), cost64.tolist()):
        if mate[a] == b:
            continue
        assert mate[a] >= 0 or mate[b] >= 0, f"edge ({a},{b}) has two free endpoints"
        best = min(pc.get(a, math.inf), pc.get(b, math.inf))
        if not (best <= c + rel * max(abs(c), 1.0)):
            bad += 1
    return bad


def check_merge_rows(cur, sub, got, ref):
    """Merged rows `got` (GPU) against `ref` (FP64 oracle) for the pairs `sub`
    of rows of `cur`: centre relative to the pair's span, covariance relative
    to its Frobenius norm, SH relative to |f_i| + |f_j|, opacity on alpha."""
    i, j = sub[:, 0], sub[:, 1]
    xyz, ls, rot, logit, sh = (a.astype(np.float64) for a in got)
    rxyz, rls, rrot, rlogit, rsh = ref
    span = np.linalg.norm(cur.xyz[i].astype(np.float64) - cur.xyz[j], axis=1) + \
        np.exp(cur.log_scale[i].astype(np.float64)).max(1)
    eps32 = np.finfo(np.float32).eps
    assert np.all(np.linalg.norm(xyz - rxyz, axis=1) <=
                  ATTR_RTOL * span + 4 * eps32 * np.linalg.norm(rxyz, axis=1))
    S, RS = sigma_of(ls, rot), sigma_of(rls, rrot)
    assert np.all(np.linalg.norm(S - RS, axis=(1, 2)) <= ATTR_RTOL * np.linalg.norm(RS, axis=(1, 2)))
    fs = np.abs(cur.sh[i].astype(np.float64)) + np.abs(cur.sh[j])
    assert np.all(np.abs(sh - rsh) <= ATTR_RTOL * fs + 1e-7)
    a, ra = 1 / (1 + np.exp(-logit)), 1 / (1 + np.exp(-rlogit))
    assert np.all(np.abs(a - ra) <= ATTR_RTOL * ra)


def small_scene(n, seed=0, kind="unit"):
    if kind == "unit":
        return synth.surfaces_unit_cube(n, seed=seed)
    return synth.patches_cube(n, seed=seed, frac_degenerate=0.05, frac_duplicate=0.01)


COST_TOL = 3e-5      # |C_gpu - C_fp64| <= COST_TOL * max(|C|, 1) for every edge
ATTR_RTOL = 1e-5     # merged attributes vs FP64


def cost_excess(cost, ref, tol=None):
    """Largest |C_gpu - C_fp64| / max(|C_fp64|, 1) over all edges, divided by
    the accuracy contract (<= 1 passes)."""
    tol = COST_TOL if tol is None else tol
    err = np.abs(np.asarray(cost, np.float64) - ref) / np.maximum(np.abs(ref), 1.0)
    return float(err.max() / tol) if len(err) else 0.0


def stepwise(ngs, ctx, scene, target, max_passes=64):
    """Algorithm 1 through the per-step C-ABI calls."""
    ds = ngs.DeviceSplats.from_numpy(scene)
    ctx.prefilter(ds)
    p = 0
    while ds.n > target and ds.n > 1 and p < max_passes:
        g, nbr, lo, hi = ctx.build_graph(ds)
        cost = ctx.edge_costs(ds, g, p)
        pairs = ctx.select_pairs(g, cost, ds.n - target)
        p += 1
        if pairs.shape[0] == 0:
            break
        ctx.merge_compact(ds, pairs)
    return ds, p


def greedy_certificate_np(n, lo, hi, cost64, pairs, rel=1e-6):
    """Vectorised form of the greedy certificate: `pairs` is a matching, no
    edge has two free endpoints, and every other edge touches a pair whose FP64
    cost is not larger beyond `rel`.  Returns the number of violating edges."""
    mate = np.full(n, -1, np.int64)
    assert len(np.unique(pairs.reshape(-1))) == 2 * len(pairs), "not a matching"
    mate[pairs[:, 0]], mate[pairs[:, 1]] = pairs[:, 1], pairs[:, 0]
    keys = lo.astype(np.int64) * n + hi
    pk = pairs[:, 0].astype(np.int64) * n + pairs[:, 1]
    at = np.searchsorted(keys, pk)               # lo, hi are in lexicographic order
    assert np.array_equal(keys[at], pk), "a pair is not an edge"
    pc = np.full(n, np.inf)
    pc[pairs[:, 0]] = pc[pairs[:, 1]] = cost64[at]
    member = mate[lo] == hi
    assert not np.any((mate[lo] < 0) & (mate[hi] < 0)), "an edge has two free endpoints"
    best = np.minimum(pc[lo], pc[hi])
    ok = best <= cost64 + rel * np.maximum(np.abs(cost64), 1.0)
    return int(np.sum(~ok & ~member))
