"""Serving form on the GPU: every job's result is the same alone and in the
mix (bit for bit), whether it ran alone on a slot, concurrently with other
slots, or grouped into one batched run with other small jobs."""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import small_scene

pytestmark = pytest.mark.gpu


def _alone(ngs, scene, target):
    with ngs.Context() as c:
        ds = ngs.DeviceSplats.from_numpy(scene)
        c.simplify(ds, target)
        return [a.copy() for a in ds.numpy()]


def _mix(sizes, seed0=300):
    scenes, targets = [], []
    ratios = [0.5, 0.1, 0.25, 0.01]
    for i, n in enumerate(sizes):
        s = small_scene(n, seed=seed0 + i, kind="patch" if i % 2 else "unit")
        scenes.append(s)
        targets.append(O.target_count(n, ratios[i % len(ratios)]))
    return scenes, targets


def _check_mix(ngs, scenes, targets, **cfg):
    ref = [_alone(ngs, s, t) for s, t in zip(scenes, targets)]
    dev = [ngs.DeviceSplats.from_numpy(s) for s in scenes]
    torch.cuda.synchronize()
    with ngs.Server(**cfg) as srv:
        ids = [srv.submit(d.struct(), t) for d, t in zip(dev, targets)]
        outs = [srv.wait(j, 300) for j in ids]
        infos = [srv.info(j) for j in ids]
        st = srv.stats()
    for i, (d, n, r) in enumerate(zip(dev, outs, ref)):
        d.n = n
        got = d.numpy()
        assert n == r[0].shape[0], f"job {i}: {n} rows, alone {r[0].shape[0]}"
        for a, b in zip(got, r):
            assert np.array_equal(a, b), f"job {i} differs from its run alone"
    assert st["finished"] == len(scenes) and st["failed"] == 0
    assert st["gpu_launches"] > 0
    return infos, st


def test_serve_isolation_concurrent_and_grouped(ngs):
    sizes = [30000, 4000, 2500, 6000, 50000, 3000, 1200, 9000, 800, 20000]
    scenes, targets = _mix(sizes)
    infos, st = _check_mix(ngs, scenes, targets, slots=3, group_small=1, small_rows=10000,
                           group_rows=40000)
    assert max(i["group_size"] for i in infos) >= 1
    assert st["peak_workspace_bytes"] > 0


def test_serve_isolation_plain(ngs):
    scenes, targets = _mix([8000, 3000, 12000])
    infos, _ = _check_mix(ngs, scenes, targets, slots=1, group_small=0)
    starts = sorted(i["start_s"] for i in infos)
    assert starts == [i["start_s"] for i in infos]


def test_serve_forced_grouping_and_release(ngs):
    """One slot, queue filled before the worker frees up: the small jobs run
    as one batch; then a budget that forces idle workers to give back their
    workspace."""
    scenes, targets = _mix([40000, 3000, 2000, 5000, 4000])
    infos, _ = _check_mix(ngs, scenes, targets, slots=1, group_small=1, small_rows=6000,
                          group_rows=100000)
    assert any(i["group_size"] > 1 for i in infos)
    # budget = 1.2 x the largest estimate: jobs run one at a time and idle
    # workers release their workspace before the next admission
    bps = 1536
    budget = int(1.2 * bps * max(s.n for s in scenes))
    _check_mix(ngs, scenes, targets, slots=3, group_small=0, hbm_budget_bytes=budget,
               bytes_per_splat=bps)


def test_serve_replay_latencies(ngs):
    scenes, targets = _mix([5000, 20000, 3000, 8000, 1500, 12000])
    dev = [ngs.DeviceSplats.from_numpy(s) for s in scenes]
    torch.cuda.synchronize()
    arrivals = [0.0, 0.01, 0.015, 0.05, 0.06, 0.1]
    with ngs.Server(slots=2) as srv:
        ids = srv.replay([d.struct() for d in dev], targets, arrivals)
        lat = [srv.info(j)["finish_s"] - srv.info(j)["submit_s"] for j in ids]
        assert all(srv.info(j)["status"] == ngs.NGS_JOB_DONE for j in ids)
    assert all(x > 0 for x in lat)


def test_serve_bad_job_fails_alone(ngs):
    """A job with a non-finite centre fails; the jobs grouped with it still
    finish with the right result."""
    scenes, targets = _mix([3000, 2000, 2500])
    bad = scenes[1].copy()
    bad.xyz[7, 2] = np.nan
    ref0 = _alone(ngs, scenes[0], targets[0])
    dev = [ngs.DeviceSplats.from_numpy(s) for s in (scenes[0], bad, scenes[2])]
    torch.cuda.synchronize()
    with ngs.Server(slots=1, group_small=1, small_rows=10000, dry_run_ns_per_splat=0.0) as srv:
        ids = [srv.submit(d.struct(), t) for d, t in zip(dev, targets)]
        with pytest.raises(ngs.NgsError):
            srv.wait(ids[1], 300)
        n0 = srv.wait(ids[0], 300)
        srv.wait(ids[2], 300)
    dev[0].n = n0
    for a, b in zip(dev[0].numpy(), ref0):
        assert np.array_equal(a, b)
