"""Synthetic scenario trees (paper §2.3, Fig. "tree").

Nodes are numbered breadth first, stage by stage: node 0 is the root
(stage 0) and the nodes of stage t occupy [stage_ptr[t], stage_ptr[t+1]).
The children of a node are contiguous and appear in the order of their
parents.  anc[nu] is the ancestor of node nu (anc[0] = -1) and prob[nu]
the probability of reaching nu from the root; the probabilities of a
node's children are its own probability split by a Dirichlet(5, ..., 5)
draw (scenario reduction yields unequal probabilities).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Tree:
    N: int                 # horizon = number of stages after the root
    n_nodes: int
    stage_ptr: np.ndarray  # (N + 2,) int64
    anc: np.ndarray        # (n_nodes,) int64, anc[0] = -1
    prob: np.ndarray       # (n_nodes,) float64
    stage: np.ndarray      # (n_nodes,) int64

    @property
    def n_scenarios(self) -> int:
        return int(self.stage_ptr[self.N + 1] - self.stage_ptr[self.N])


def _build(children_per_stage, seed: int, dirichlet: float = 5.0,
           uniform: bool = False) -> Tree:
    """children_per_stage[t] lists the child count of each stage-t node."""
    rng = np.random.default_rng(seed)
    N = len(children_per_stage)
    anc = [-1]
    prob = [1.0]
    stage = [0]
    stage_ptr = [0, 1]
    for t in range(N):
        first, last = stage_ptr[t], stage_ptr[t + 1]
        counts = children_per_stage[t]
        if len(counts) != last - first:
            raise ValueError(f"stage {t}: {len(counts)} counts for {last - first} nodes")
        for off, nc in enumerate(counts):
            parent = first + off
            if nc < 1:
                raise ValueError("every node before the last stage needs a child")
            if nc == 1 or uniform:
                w = np.full(nc, 1.0 / nc)
            else:
                w = rng.dirichlet(np.full(nc, dirichlet))
            for c in range(nc):
                anc.append(parent)
                prob.append(prob[parent] * float(w[c]))
                stage.append(t + 1)
        stage_ptr.append(len(anc))
    return Tree(N=N, n_nodes=len(anc), stage_ptr=np.asarray(stage_ptr, dtype=np.int64),
                anc=np.asarray(anc, dtype=np.int64), prob=np.asarray(prob),
                stage=np.asarray(stage, dtype=np.int64))


def make_tree(branching, seed: int = 2, uniform: bool = False) -> Tree:
    """Tree in which every stage-t node has branching[t] children."""
    counts = []
    width = 1
    for b in branching:
        counts.append([int(b)] * width)
        width *= int(b)
    return _build(counts, seed, uniform=uniform)


def random_branching(N: int, seed: int, s_min: int = 16, s_max: int = 512,
                     branch_stages: int = 6) -> Tree:
    """Uneven tree: nodes of the first stages draw 1-4 children each, so
    sibling subtrees differ in size; the scenario count lies in
    [s_min, s_max] (target drawn log-uniformly)."""
    rng = np.random.default_rng(seed)
    target = int(round(np.exp(rng.uniform(np.log(s_min), np.log(s_max)))))
    counts = []
    width = 1
    for t in range(N):
        if width < target and (t < branch_stages or width < s_min):
            c = rng.integers(1, 5, size=width)
            # keep the total within the target by trimming from the end
            excess = int(c.sum()) - target
            i = width - 1
            while excess > 0 and i >= 0:
                cut = min(excess, int(c[i]) - 1)
                c[i] -= cut
                excess -= cut
                i -= 1
        else:
            c = np.ones(width, dtype=np.int64)
        counts.append([int(v) for v in c])
        width = int(c.sum())
    return _build(counts, seed + 7)
