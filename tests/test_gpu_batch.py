"""Batched form: ngs_batch_simplify over many scenes gives, for every scene,
exactly (bit for bit) what ngs_simplify gives on that scene alone, and the
per-scene counts the FP64 oracle gives."""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import small_scene

pytestmark = pytest.mark.gpu


def _dev(ngs, scene):
    return ngs.DeviceSplats.from_numpy(scene)


def _empty(ngs, like):
    return ngs.DeviceSplats(*(torch.zeros((0,) + a.shape[1:], dtype=torch.float32, device="cuda")
                              for a in like.arrays()))


def _alone(ngs, scene, target, **params):
    with ngs.Context(**params) as c:
        ds = _dev(ngs, scene)
        st = c.simplify(ds, target)
        return ds, st


def _check_batch(ngs, scenes, targets, **params):
    alone = [_alone(ngs, s, t, **params) if s.n else None for s, t in zip(scenes, targets)]
    with ngs.Context(**params) as c:
        batch = [_dev(ngs, s) if s.n else _empty(ngs, scenes[0]) for s in scenes]
        st = c.batch_simplify(batch, targets)
    for i, (ds, ref) in enumerate(zip(batch, alone)):
        if ref is None:
            assert ds.n == 0
            continue
        assert ds.n == ref[0].n, f"scene {i}: {ds.n} rows, alone {ref[0].n}"
        for a, b in zip(ds.numpy(), ref[0].numpy()):
            assert np.array_equal(a, b), f"scene {i} differs from its single-scene run"
    used = [r for r in alone if r is not None]
    assert st["n_output"] == sum(r[0].n for r in used)
    assert st["n_filtered"] == sum(r[1]["n_filtered"] for r in used)
    assert st["passes"] == max([r[1]["passes"] for r in used] + [0])
    return batch, st


def test_batch_mixed_scenes_equal_alone(ngs):
    """Sizes, ratios and kinds mixed; one scene below k (runs alone inside the
    call), one whose target is above its size (pre-filter only), one empty."""
    spec = [(20000, 0.5, "unit", 1), (9001, 0.1, "patch", 2), (500, 0.25, "unit", 3),
            (64, 0.5, "patch", 4), (40, 0.25, "unit", 5), (3000, 2.0, "patch", 6),
            (0, 0.5, "unit", 7), (7000, 0.01, "unit", 8)]
    scenes, targets = [], []
    for n, ratio, kind, seed in spec:
        s = small_scene(max(n, 1), seed=seed, kind=kind)
        if n == 0:
            s = s.subset(np.arange(0))
        scenes.append(s)
        targets.append(max(1, int(n * ratio)) if ratio <= 1 else 10 * n)
    _check_batch(ngs, scenes, targets)


def test_batch_log_uniform_sizes(ngs):
    """Sixteen patch scenes, sizes log-uniform in [5k, 60k], ratios 0.5/0.25/0.1."""
    rng = np.random.default_rng(11)
    sizes = np.exp(rng.uniform(np.log(5000), np.log(60000), 16)).astype(int)
    ratios = [0.5, 0.25, 0.1]
    scenes = [small_scene(int(n), seed=100 + i, kind="patch" if i % 2 else "unit")
              for i, n in enumerate(sizes)]
    targets = [O.target_count(s.n, ratios[i % 3]) for i, s in enumerate(scenes)]
    batch, _ = _check_batch(ngs, scenes, targets)
    for ds, t in zip(batch, targets):
        assert ds.n >= t


@pytest.mark.parametrize("params", [dict(prefilter=0), dict(fp64_policy=2, k=8),
                                    dict(cost_mode=1, mc_samples=4), dict(cost_mode=2, mc_samples=2),
                                    dict(cost_mode=3)])
def test_batch_params(ngs, params):
    scenes = [small_scene(n, seed=20 + n % 7, kind=kind)
              for n, kind in [(6000, "patch"), (2500, "unit"), (12000, "patch")]]
    targets = [O.target_count(s.n, 0.25) for s in scenes]
    _check_batch(ngs, scenes, targets, **params)


def test_batch_counts_vs_oracle(ngs):
    scenes = [small_scene(4000, seed=31, kind="patch"), small_scene(2500, seed=32)]
    targets = [O.target_count(s.n, 0.5) for s in scenes]
    with ngs.Context() as c:
        batch = [_dev(ngs, s) for s in scenes]
        c.batch_simplify(batch, targets)
    for s, t, ds in zip(scenes, targets, batch):
        ref, rst = O.simplify(s, t)
        assert ds.n == ref[0].shape[0]


def test_batch_errors(ngs):
    a, b = small_scene(3000, seed=41), small_scene(2000, seed=42)
    with ngs.Context() as c:
        with pytest.raises(ngs.NgsError):
            c.batch_simplify([_dev(ngs, a), _dev(ngs, b)], [100, 0])
        short = _dev(ngs, b)
        short.sh = short.sh[:, :12].contiguous()
        with pytest.raises(ngs.NgsError):
            c.batch_simplify([_dev(ngs, a), short], [100, 100])
        bad = b.copy()
        bad.xyz[5, 0] = np.inf
        with pytest.raises(ngs.NgsError):
            c.batch_simplify([_dev(ngs, a), _dev(ngs, bad)], [100, 100])
        st = c.batch_simplify([], [])
        assert st["n_output"] == 0
        # the context still works after the errors
        ds = _dev(ngs, a)
        c.batch_simplify([ds], [1000])
        assert ds.n >= 1000


@pytest.mark.parametrize("sh_dim", [5, 3])
def test_batch_sh_dim_not_multiple_of_4(ngs, sh_dim):
    scenes = [small_scene(n, seed=50 + n % 5) for n in (3000, 1800)]
    for s in scenes:
        s.sh = np.ascontiguousarray(s.sh[:, :sh_dim])
    targets = [O.target_count(s.n, 0.25) for s in scenes]
    _check_batch(ngs, scenes, targets)


def test_batch_many_small_scenes(ngs):
    """450 scenes of 120-400 splats: the per-scene tables no longer fit a
    kernel parameter and go up by a copy; every scene still equals its run
    alone."""
    rng = np.random.default_rng(77)
    sizes = rng.integers(120, 400, 450)
    scenes = [small_scene(int(n), seed=500 + i, kind="patch" if i % 3 else "unit")
              for i, n in enumerate(sizes)]
    targets = [O.target_count(s.n, 0.25) for s in scenes]
    _check_batch(ngs, scenes, targets)
