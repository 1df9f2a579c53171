"""Local neighbourhood refresh (Sec. 3.4) measured on the oracle.

The refresh would re-run kNN queries only around the splats a pass formed,
and keep the other rows' lists with their entries carried through the merge.
A kept row can keep its list only when no two of its neighbours merged into
one splat (else the carried list holds a repeated entry and needs a query).
Algorithm 1 merges a maximal disjoint matching each pass (P = N - N_tgt
rarely binds), so nearly every splat is merged: the rows that need a query
are practically all rows, and the refresh would do the same kNN work as the
full rebuild that the pass already performs.  This test pins that count.
"""
import numpy as np
import pytest

import oracle as O
from paper_2603_16103_gb300 import synth


@pytest.mark.parametrize("kind", ["unit", "patch"])
def test_refresh_would_requery_nearly_every_row(kind):
    k = 16
    if kind == "unit":
        scene = synth.surfaces_unit_cube(20000, seed=3)
    else:
        scene = synth.patches_cube(20000, seed=3)
    n = scene.n
    nbr = O.knn(scene.xyz, k)
    lo, hi = O.union_edges(nbr)
    z, u = O.mc_draws(0, 0, 1)
    plo, phi = O.greedy(n, lo, hi, O.edge_costs(scene, lo, hi, z, u), n - O.target_count(n, 0.1))
    partner = np.full(n, -1, np.int64)
    partner[plo], partner[phi] = phi, plo
    rows = np.arange(n)
    survive = (partner < 0) | (rows < partner)          # the merged splat takes row min(i, j)
    new_row = np.cumsum(survive) - 1
    carried = new_row[np.where(partner >= 0, np.minimum(rows, partner), rows)]
    kept = partner < 0
    lists = np.sort(carried[nbr[kept]], axis=1)
    repeated = np.any(lists[:, 1:] == lists[:, :-1], axis=1)
    n_new = int(survive.sum())
    formed = len(plo) / n_new
    need_query = (len(plo) + int(repeated.sum())) / n_new
    print(f"{kind}: {len(plo)} pairs, formed {formed:.3f}, rows needing a query {need_query:.4f}")
    assert formed > 0.85
    assert need_query > 0.98
