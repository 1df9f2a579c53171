"""Tuning changes speed, never results: the autotuner picks from its
candidate sets, and simplification under any tuning is bit-identical."""
import numpy as np
import pytest

import oracle as O
from gpu_util import small_scene

pytestmark = pytest.mark.gpu


def test_autotune_picks_a_candidate_and_keeps_results(ngs):
    scene = small_scene(30000, seed=71, kind="patch")
    target = O.target_count(scene.n, 0.25)
    with ngs.Context() as c:
        ref = ngs.DeviceSplats.from_numpy(scene)
        c.simplify(ref, target)
        sample = ngs.DeviceSplats.from_numpy(scene)
        before = [a.copy() for a in sample.numpy()]
        t, ms = c.autotune(sample)
        assert ms > 0
        assert t["knn_block_min"] in (48, 64, 96) and t["cells_per_point"] in (2, 4, 8)
        assert t["cost_blocks_per_sm"] in (4, 8, 12)
        assert c.tuning() == t
        for a, b in zip(sample.numpy(), before):   # the sample is not modified
            assert np.array_equal(a, b)
        ds = ngs.DeviceSplats.from_numpy(scene)
        c.simplify(ds, target)
    assert ds.n == ref.n
    for a, b in zip(ds.numpy(), ref.numpy()):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("tuning", [dict(knn_block_min=16, cells_per_point=1, cost_blocks_per_sm=1),
                                    dict(knn_block_min=1024, cells_per_point=8, cost_blocks_per_sm=64),
                                    dict(match_method=0), dict(match_method=1),
                                    dict(match_max_steps=1)])   # proposals fall back to rounds
def test_extreme_tunings_give_identical_results(ngs, tuning):
    scene = small_scene(12000, seed=72)
    target = O.target_count(scene.n, 0.1)
    with ngs.Context() as c:
        ref = ngs.DeviceSplats.from_numpy(scene)
        c.simplify(ref, target)
        c.set_tuning(**tuning)
        ds = ngs.DeviceSplats.from_numpy(scene)
        c.simplify(ds, target)
        with pytest.raises(ngs.NgsError):
            c.set_tuning(cells_per_point=3)
    for a, b in zip(ds.numpy(), ref.numpy()):
        assert np.array_equal(a, b)
