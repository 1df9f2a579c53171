"""The two matching schemes of the CUDA pair selection, modelled in Python on
the host, against the oracle's greedy (sort, then scan): both reach the
greedy matching under the strict order (cost, lo, hi), whatever order the
vertices are processed in.  The models mirror the kernels' rules, not their
code: proposals with displacement (k_suitor) and locally-dominant rounds
(k_match_scan / k_match_pair)."""
import numpy as np
import pytest

import oracle as O
from gpu_util import small_scene


def _graph(seed, ties):
    sc = small_scene(600, seed=seed, kind="patch" if seed % 2 else "unit")
    lo, hi = O.union_edges(O.knn(sc.xyz, 16, "brute"))
    z, u = O.mc_draws(0, 0, 1)
    cost = O.edge_costs(sc, lo, hi, z, u).astype(np.float32).astype(np.float64)
    if ties:
        cost = np.round(cost * 3) / 3      # massive exact ties
    return sc.n, lo, hi, cost


def _adjacency(n, lo, hi, cost):
    adj = [[] for _ in range(n)]
    for a, b, c in zip(lo.tolist(), hi.tolist(), cost.tolist()):
        adj[a].append((c, b))
        adj[b].append((c, a))
    return adj


def proposals(n, lo, hi, cost, rng):
    """Each vertex proposes along its best edge (cost, other id) among those
    whose other endpoint holds a worse offer (cost, proposer id); a beaten
    holder proposes again.  Steps of the active vertices interleave at random."""
    adj = _adjacency(n, lo, hi, cost)
    offer = [(np.inf, n)] * n
    holder = [-1] * n
    active = list(range(n))
    while active:
        t = int(rng.integers(len(active)))
        u = active[t]
        best = min(((c, v) for c, v in adj[u] if (c, u) < offer[v]), default=None)
        if best is None:
            active.pop(t)
            continue
        c, v = best
        offer[v], prev, holder[v] = (c, u), holder[v], u
        if prev >= 0:
            active[t] = prev
        else:
            active.pop(t)
    return sorted((v, holder[v]) for v in range(n)
                  if holder[v] > v and holder[holder[v]] == v)


def rounds(n, lo, hi, cost, rng):
    """Free vertices point at their best free neighbour; mutual pointers match;
    repeat until a round matches nothing.  Vertices are visited in a random
    order each round (the result must not depend on it)."""
    adj = _adjacency(n, lo, hi, cost)
    mate = [-1] * n
    while True:
        cand = [-1] * n
        for v in rng.permutation(n).tolist():
            if mate[v] < 0:
                free = [(c, u) for c, u in adj[v] if mate[u] < 0]
                cand[v] = min(free)[1] if free else -1
        new = [(v, cand[v]) for v in range(n) if cand[v] > v and cand[cand[v]] == v]
        if not new:
            break
        for a, b in new:
            mate[a], mate[b] = b, a
    return sorted((v, mate[v]) for v in range(n) if mate[v] > v)


@pytest.mark.parametrize("seed,ties", [(0, False), (1, False), (2, True), (3, True)])
@pytest.mark.parametrize("scheme", [proposals, rounds])
def test_scheme_equals_greedy(seed, ties, scheme):
    n, lo, hi, cost = _graph(seed, ties)
    glo, ghi = O.greedy(n, lo, hi, cost, n)
    greedy = sorted(zip(glo.tolist(), ghi.tolist()))
    for rep in range(2):
        assert scheme(n, lo, hi, cost, np.random.default_rng(10 * seed + rep)) == greedy


def test_planted_wrong_order_is_caught():
    """A model that breaks cost ties by the wrong endpoint differs from greedy
    on the tied graph, so the tie-break is what the equality checks."""
    n, lo, hi, cost = _graph(2, True)
    glo, ghi = O.greedy(n, lo, hi, cost, n)
    greedy = sorted(zip(glo.tolist(), ghi.tolist()))
    m = n - 1    # relabel v -> m - v: the same graph with the id order reversed
    flipped = proposals(n, m - hi, m - lo, cost, np.random.default_rng(0))
    back = sorted((min(m - a, m - b), max(m - a, m - b)) for a, b in flipped)
    assert back != greedy
