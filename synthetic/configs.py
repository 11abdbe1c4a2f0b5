"""Named workloads.

* tiny: nx=4, nu=6, nd=3, ne=2; N=6; branching [2,2,1,1,1,1] (22 decision
  nodes);
* barcelona32: Barcelona-sized network (63 tanks, 114 flows, 88 demand
  sectors, 17 mixing nodes, §6); N=24; branching [4,2,2,2,1,...]
  (32 scenarios, 700 decision nodes);
* barcelona512: same network; branching [8,4,4,2,2,1,...] (512 scenarios,
  10,664 decision nodes).

Seeds: network 1, tree 2, data 3.
"""
from __future__ import annotations

from dataclasses import dataclass

from .data import SolveData, make_data
from .network import Cost, Network, make_cost, make_network
from .tree import Tree, make_tree


def _pad(b, N):
    return list(b) + [1] * (N - len(b))


CONFIGS = {
    "tiny": dict(dims=(4, 6, 3, 2), branching=[2, 2, 1, 1, 1, 1]),
    "barcelona32": dict(dims=(63, 114, 88, 17), branching=_pad([4, 2, 2, 2], 24)),
    "barcelona512": dict(dims=(63, 114, 88, 17), branching=_pad([8, 4, 4, 2, 2], 24)),
}


@dataclass
class Problem:
    net: Network
    cost: Cost
    tree: Tree
    data: SolveData


def make_problem(name: str, net_seed: int = 1, tree_seed: int = 2,
                 data_seed: int = 3, **cost_kw) -> Problem:
    cfg = CONFIGS[name]
    nx, nu, nd, ne = cfg["dims"]
    net = make_network(nx, nu, nd, ne, seed=net_seed)
    cost = make_cost(net, seed=net_seed, **cost_kw)
    tree = make_tree(cfg["branching"], seed=tree_seed)
    data = make_data(net, tree, seed=data_seed)
    return Problem(net=net, cost=cost, tree=tree, data=data)
