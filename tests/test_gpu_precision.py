"""Precision report: error of every output attribute against the FP64 oracle
on the 200,000-splat scene with 5% near-degenerate splats and 1% duplicated
centres, for each FP64 policy.  One pass in lockstep (the oracle runs on the
GPU's own pass input); the report is printed as one JSON line per policy
(3: the eigendecomposition finished in FP64 instead of float-float)."""
import json

import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import sigma_of
from paper_2603_16103_gb300 import synth

pytestmark = pytest.mark.gpu


def attr_errors(cur, pairs, got):
    ref = O.merge_compact(cur, pairs[:, 0], pairs[:, 1])
    merged = np.zeros(cur.n, bool)
    merged[pairs[:, 0]] = True
    keep = np.ones(cur.n, bool)
    keep[pairs[:, 1]] = False
    m = merged[keep]
    xyz, ls, rot, logit, sh = (a[m].astype(np.float64) for a in got)
    rxyz, rls, rrot, rlogit, rsh = (a[m] for a in ref)
    i, j = pairs[:, 0], pairs[:, 1]
    S, RS = sigma_of(ls, rot), sigma_of(rls, rrot)
    lam = np.linalg.eigvalsh(RS)
    well = (np.diff(lam, axis=1).min(1) > 1e-6 * lam[:, -1:].ravel())
    sig_err = np.linalg.norm(S - RS, axis=(1, 2)) / np.linalg.norm(RS, axis=(1, 2))
    fs = np.abs(cur.sh[i].astype(np.float64)) + np.abs(cur.sh[j]) + 1e-30
    a, ra = 1 / (1 + np.exp(-logit)), 1 / (1 + np.exp(-rlogit))
    lse = np.abs(np.sort(ls, 1) - np.sort(rls, 1))
    qd = np.minimum(np.linalg.norm(rot - rrot, axis=1), np.linalg.norm(rot + rrot, axis=1))
    out = {
        "merges": int(m.sum()),
        "mu_rel": np.linalg.norm(xyz - rxyz, axis=1) / np.linalg.norm(rxyz, axis=1),
        "mu_err_over_fp32_spacing": np.linalg.norm(xyz - rxyz, axis=1) /
        (np.finfo(np.float32).eps * np.linalg.norm(rxyz, axis=1)),
        "Sigma_rel_fro": sig_err,
        "log_scale_abs": lse.max(1),
        "rot_quat_dist_well_conditioned": qd[well],
        "opacity_rel": np.abs(a - ra) / ra,
        "sh_rel": (np.abs(sh - rsh) / fs).max(1),
    }
    return {k: (v if k == "merges" else {"max": float(np.max(v)), "mean": float(np.mean(v))})
            for k, v in out.items()}


@pytest.mark.parametrize("policy", [0, 1, 2, 3])
def test_precision_report(ngs, policy):
    scene = synth.workload("patches200k")
    c = ngs.Context(fp64_policy=policy)
    try:
        ds = ngs.DeviceSplats.from_numpy(scene)
        c.prefilter(ds)
        cur = synth.Scene(*ds.numpy())
        g, nbr, lo, hi = c.build_graph(ds)
        cost = c.edge_costs(ds, g, 0)
        z, u = O.mc_draws(0, 0, 1)
        rc = O.edge_costs(cur, lo.cpu().numpy(), hi.cpu().numpy(), z, u)
        cerr = np.abs(cost.cpu().numpy().astype(np.float64) - rc) / np.maximum(np.abs(rc), 1)
        pairs = c.select_pairs(g, cost, cur.n // 2)
        rlo, rhi = O.greedy(cur.n, lo.cpu().numpy(), hi.cpu().numpy(),
                            cost.cpu().numpy().astype(np.float64), cur.n // 2)
        ref = np.stack([rlo, rhi], 1)
        assert np.array_equal(pairs.cpu().numpy(), ref[np.argsort(ref[:, 0])])
        p = pairs.cpu().numpy()
        c.merge_compact(ds, pairs)
        rep = attr_errors(cur, p, ds.numpy())
        rep["edge_cost_rel_max1"] = {"max": float(cerr.max()), "mean": float(cerr.mean()),
                                "p99.9": float(np.quantile(cerr, 0.999))}
        w = int(np.argmax(cerr))
        lw, hw = int(lo[w]), int(hi[w])
        rep["worst_edge"] = {"lo": lw, "hi": hw, "gpu": float(cost[w]), "fp64": float(rc[w]),
                             "log_scale_lo": cur.log_scale[lw].tolist(),
                             "log_scale_hi": cur.log_scale[hw].tolist(),
                             "dist": float(np.linalg.norm(cur.xyz[lw].astype(np.float64) - cur.xyz[hw]))}
        rep["policy"] = policy
        rep["scene"] = "patches200k (5% degenerate, 1% duplicate centres), pass 0"
        print("PRECISION " + json.dumps(rep))
        assert rep["Sigma_rel_fro"]["max"] <= 1e-5
        assert rep["sh_rel"]["max"] <= 1e-5
        assert rep["opacity_rel"]["max"] <= 1e-5
        assert rep["mu_rel"]["max"] <= 1e-5
        assert rep["mu_err_over_fp32_spacing"]["max"] <= 4
        # the extended-precision eigen finish keeps small eigenvalues accurate
        # (sorted log-scales); policy 2 skips it for well-conditioned merges
        assert rep["log_scale_abs"]["max"] <= (1e-5 if policy != 2 else 1e-4)
        assert cerr.max() <= c.params.cost_tol
    finally:
        c.close()
