"""Scenario tree from Monte-Carlo paths (paper §2.3 and §6.2: sampled
scenarios reduced into a tree with the method of Heitsch and Römisch).

TEST INFRASTRUCTURE: this module is the oracle of the GPU scenario-tree
construction; only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline may import it.

Reading (the paper only cites the method): the tree is built forward,
stage by stage.  Every node of stage t holds a bundle of the sampled paths
(the root holds all of them).  Its children are b_t representatives of
its bundle, chosen by fast forward selection on the distance between the
remaining parts of the paths (stages t+1 .. N, Euclidean); every path of
the bundle goes to the nearest representative, and a child carries the
representative's value at stage t+1 and the total probability of its
paths.  Fast forward selection (Heitsch and Römisch 2003) picks the
representatives one at a time, each the candidate that minimises the
probability-weighted distance of the bundle's paths to the nearest chosen
one:
    z(u) = sum_j p_j min(m_j, d(j, u)),   m_j = min over chosen c of d(j, c)
(m_j = +inf before the first choice), ties to the lowest path index.  A
tie is a value within TIE (relative) of the smallest: such ties are real
(in one dimension the weighted median of an even number of paths is an
interval, and near the end of the horizon the remaining parts are short),
and two sides that add the same terms in different orders must take the
same decision on them.  The assignment of paths to representatives breaks
ties the same way.  Everything here is FP64 and follows those definitions
literally.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class ReducedTree:
    N: int
    stage_ptr: np.ndarray   # (N + 2,) breadth-first stage boundaries
    anc: np.ndarray         # (n_nodes,) ancestor, anc[0] = -1
    prob: np.ndarray        # (n_nodes,)
    value: np.ndarray       # (n_nodes, dim): the node's value (root row zero)
    leaf_of: np.ndarray     # (S,) leaf node of every path
    rep: np.ndarray         # (n_nodes,) the path a node represents (root: -1)


def tail_distances(paths: np.ndarray, idx: np.ndarray, t: int) -> np.ndarray:
    """d(i, j) = || paths[i, t:] - paths[j, t:] || (Euclidean over the
    remaining stages and dimensions) for the paths idx."""
    X = paths[idx, t:, :].reshape(len(idx), -1)
    d2 = np.zeros((len(idx), len(idx)))
    for c in range(X.shape[1]):
        diff = X[:, c][:, None] - X[:, c][None, :]
        d2 += diff * diff
    return np.sqrt(d2)


TIE = 1e-12  # values within TIE (relative) of the smallest count as ties


def first_within_tie(values) -> int:
    """Lowest index whose value is within TIE of the smallest value."""
    v = np.asarray(values, float)
    lo = v.min()
    return int(np.flatnonzero(v <= lo + TIE * abs(lo))[0])


def fast_forward_selection(D: np.ndarray, p: np.ndarray, K: int) -> list:
    """Indices (into D's rows) of K representatives chosen greedily."""
    M = D.shape[0]
    K = min(K, M)
    m = np.full(M, np.inf)
    chosen: list = []
    for _ in range(K):
        z = np.full(M, np.inf)
        for u in range(M):
            if u not in chosen:
                z[u] = float(np.sum(p * np.minimum(m, D[:, u])))
        best = first_within_tie(z)
        chosen.append(best)
        m = np.minimum(m, D[:, best])
    return chosen


def build_tree(paths: np.ndarray, prob: np.ndarray, branching) -> ReducedTree:
    """paths (S, N, dim): sampled values at stages 1 .. N; prob (S,);
    branching[t] (t = 0 .. N-1): children of every node of stage t."""
    paths = np.asarray(paths, float)
    S, N, dim = paths.shape
    prob = np.asarray(prob, float)
    assert len(branching) == N
    anc, pr, val, rep = [-1], [1.0], [np.zeros(dim)], [-1]
    stage_ptr = [0, 1]
    bundles = [np.arange(S)]
    leaf_of = np.full(S, -1)
    for t in range(N):
        new_bundles = []
        for off, idx in enumerate(bundles):
            parent = stage_ptr[t] + off
            D = tail_distances(paths, idx, t)
            sel = fast_forward_selection(D, prob[idx], branching[t])
            # every path to its nearest representative (first chosen on ties)
            owner = np.array([first_within_tie(D[a, sel]) for a in range(len(idx))])
            for c, s in enumerate(sel):
                members = idx[owner == c]
                anc.append(parent)
                pr.append(float(prob[members].sum()))
                val.append(paths[idx[s], t, :].copy())
                rep.append(int(idx[s]))
                new_bundles.append(members)
        bundles = new_bundles
        stage_ptr.append(len(anc))
    for off, idx in enumerate(bundles):
        leaf_of[idx] = stage_ptr[N] + off
    return ReducedTree(N=N, stage_ptr=np.asarray(stage_ptr), anc=np.asarray(anc),
                       prob=np.asarray(pr), value=np.asarray(val), leaf_of=leaf_of,
                       rep=np.asarray(rep))


def kantorovich(D: np.ndarray, p: np.ndarray, chosen) -> float:
    """sum_j p_j min over chosen c of d(j, c): the transport cost of moving
    every path of the bundle to its nearest representative."""
    return float(np.sum(p * D[:, list(chosen)].min(axis=1)))
