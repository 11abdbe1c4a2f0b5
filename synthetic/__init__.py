"""Seeded synthetic inputs for the scenario-tree stochastic MPC problem.

This module builds plain arrays only: a flow-based water network
(tanks, pumps/valves, mixing nodes, demand sectors; paper §2.1), a
scenario tree (§2.3, Fig. "tree") and the per-node demand/price data
that the tree carries (§2.2-§2.3).  It contains none of the solver's
arithmetic: no costs are evaluated, no dual or primal quantity is
formed.  Both the CPU oracle and the CUDA path take their inputs from
here, so the two sides see identical data.

The paper's own data (the Barcelona network, its demand history and the
EXAA price series) is not available; these generators stand in for it
with the same dimensions and structure:

* network: A = I (exact discretisation of the tank mass balance, §2.1),
  B / E incidence in {-1,0,1}, Gd / Ed demand draws in {0,-1}, umin = 0;
* tree: a branching vector per stage, Dirichlet splits of probability;
* demand: positive daily sinusoid times (1 + 0.1 N(0,1)) per node;
* price: lognormal(log 0.1, 0.3) per node and hour, multiplied by a
  per-pump energy coefficient (valves cost nothing to operate);
* sampled price paths (AR(1) log-price deviations with a daily profile)
  for the scenario-tree construction.
"""
from .network import Cost, Network, make_cost, make_network
from .tree import Tree, make_tree, random_branching
from .data import SolveData, make_data
from .configs import CONFIGS, Problem, make_problem
from .paths import make_price_paths

__all__ = [
    "Cost", "Network", "make_cost", "make_network", "Tree", "make_tree", "random_branching",
    "SolveData", "make_data", "CONFIGS", "Problem", "make_problem", "make_price_paths",
]
