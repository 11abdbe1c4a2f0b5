"""Per-solve data on the tree: initial state, previous input, demands
and prices at every node (paper §2.2-§2.3, eq. prediction-error).

The forecasts of the paper (SVM demand model, ARIMA price model) are
replaced by a seeded generator with the shape the paper describes:
demand follows a positive daily sinusoid per sector with 10 % Gaussian
noise per node; the hourly day-ahead price is lognormal(log 0.1, 0.3)
per node.  alpha at a node is the price times the per-flow energy
coefficient (zero on valves).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .network import NOISE_CLIP, NOISE_SIGMA, SIN_AMPLITUDE, Network
from .tree import Tree


@dataclass
class SolveData:
    x0: np.ndarray       # (nx,) current tank levels p
    q: np.ndarray        # (nu,) previous input u_{k-1}
    demand: np.ndarray   # (n_nodes, nd); row 0 unused
    alpha: np.ndarray    # (n_nodes, nu); row 0 unused


def make_data(net: Network, tree: Tree, seed: int = 3, hour0: int = 0) -> SolveData:
    rng = np.random.default_rng(seed)
    x0 = rng.uniform(0.4, 0.8, size=net.nx) * net.xmax
    q = rng.uniform(0.1, 0.4, size=net.nu) * net.umax
    hours = (hour0 + tree.stage).astype(np.float64)[:, None]
    base = net.dbar[None, :] * (1.0 + SIN_AMPLITUDE *
                                np.sin(2.0 * np.pi * (hours + net.phase[None, :]) / 24.0))
    base = np.maximum(base, 1e-3)
    noise = np.clip(rng.standard_normal((tree.n_nodes, net.nd)), -NOISE_CLIP, NOISE_CLIP)
    demand = base * (1.0 + NOISE_SIGMA * noise)
    price = rng.lognormal(mean=np.log(0.1), sigma=0.3, size=tree.n_nodes)
    alpha = price[:, None] * net.e_pump[None, :]
    return SolveData(x0=x0, q=q, demand=demand, alpha=alpha)
