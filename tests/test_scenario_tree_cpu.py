"""Pins of the scenario-tree oracle (fast forward selection, Heitsch and
Römisch; forward tree construction): brute force on tiny bundles, a
library distance routine, well-separated clusters, and the invariants of a
scenario tree."""
import itertools

import numpy as np
import pytest

from oracle.scenario_tree import (build_tree, fast_forward_selection, kantorovich,
                                  tail_distances)


def paths(S=40, N=5, dim=2, seed=0):
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.standard_normal((S, N, dim)), axis=1)


def test_tail_distances_equal_cdist():
    scipy_dist = pytest.importorskip("scipy.spatial.distance")
    P = paths()
    idx = np.array([3, 7, 1, 20, 33, 5])
    for t in (0, 2, 4):
        X = P[idx, t:, :].reshape(len(idx), -1)
        np.testing.assert_allclose(tail_distances(P, idx, t), scipy_dist.cdist(X, X),
                                   rtol=1e-13, atol=1e-13)


def test_first_choice_is_the_weighted_median_and_greedy_bounds_optimum():
    rng = np.random.default_rng(1)
    P = paths(S=9, seed=2)
    D = tail_distances(P, np.arange(9), 0)
    p = rng.dirichlet(np.ones(9))
    med = int(np.argmin([np.sum(p * D[:, u]) for u in range(9)]))
    assert fast_forward_selection(D, p, 1) == [med]
    for K in (2, 3, 4):
        g = fast_forward_selection(D, p, K)
        assert len(set(g)) == K
        opt = min(kantorovich(D, p, c) for c in itertools.combinations(range(9), K))
        assert kantorovich(D, p, g) >= opt - 1e-12
    assert kantorovich(D, p, fast_forward_selection(D, p, 9)) == 0.0


def test_separated_clusters_get_one_representative_each():
    rng = np.random.default_rng(3)
    centers = np.array([[0.0, 0.0], [100.0, 0.0], [0.0, 100.0]])
    X = np.concatenate([c + 0.1 * rng.standard_normal((5, 2)) for c in centers])
    P = X[:, None, :]
    D = tail_distances(P, np.arange(15), 0)
    p = np.full(15, 1 / 15)
    g = fast_forward_selection(D, p, 3)
    assert sorted(i // 5 for i in g) == [0, 1, 2]
    # every path lies within its cluster's diameter of its representative
    diam = max(D[5 * c:5 * c + 5, 5 * c:5 * c + 5].max() for c in range(3))
    opt = min(kantorovich(D, p, c) for c in itertools.combinations(range(15), 3))
    assert opt - 1e-12 <= kantorovich(D, p, g) <= diam


@pytest.mark.parametrize("branching", [[3, 2, 1, 1, 1], [1, 4, 2, 1, 1], [2, 2, 2, 2, 2]])
def test_tree_invariants(branching):
    S = 60
    P = paths(S=S, seed=4)
    prob = np.random.default_rng(5).dirichlet(np.ones(S))
    T = build_tree(P, prob, branching)
    n = len(T.anc)
    assert T.stage_ptr[-1] == n and T.stage_ptr[0] == 0 and T.stage_ptr[1] == 1
    # children's probabilities add up to the parent's; leaves add up to one
    for v in range(1, n):
        assert T.anc[v] < v
    for v in range(T.stage_ptr[-2]):
        kids = np.where(T.anc == v)[0]
        assert len(kids) >= 1
        assert np.isclose(T.prob[kids].sum(), T.prob[v])
    assert np.isclose(T.prob[T.stage_ptr[-2]:].sum(), 1.0)
    # at most the branching's node count per stage
    cap = 1
    for t, b in enumerate(branching):
        cap *= b
        assert T.stage_ptr[t + 2] - T.stage_ptr[t + 1] <= cap
    # every path's leaf; a node's value is its representative path's value,
    # and the representative belongs to the node's bundle
    assert np.all(T.leaf_of >= T.stage_ptr[-2])
    for s in range(S):
        v, t = T.leaf_of[s], len(branching)
        while v > 0:
            assert np.array_equal(T.value[v], P[T.rep[v], t - 1])
            v, t = T.anc[v], t - 1
    for v in range(1, n):
        assert T.leaf_of[T.rep[v]] >= 0


def test_ties_go_to_the_lowest_index():
    """In one dimension the median of an even number of equally likely paths
    is an interval: both middle paths give the same z (up to rounding), and
    the lower index is chosen; a path midway between two representatives
    goes to the one chosen first."""
    from oracle.scenario_tree import first_within_tie
    x = np.array([0.0, 1.0, 2.0, 3.0])
    P = x[:, None, None]
    D = tail_distances(P, np.arange(4), 0)
    p = np.full(4, 0.25)
    assert fast_forward_selection(D, p, 1) == [1]
    assert first_within_tie([3.0, 1.0 + 1e-15, 1.0, 2.0]) == 1
    assert first_within_tie([3.0, 1.0 + 1e-9, 1.0, 2.0]) == 2
