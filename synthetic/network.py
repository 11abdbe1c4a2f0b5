"""Synthetic flow-based drinking-water network (paper §2.1).

Elements follow the paper's hydraulic model: tanks with a mass balance
(eq. tank-dynamics), mixing nodes with an algebraic balance, pumps and
valves whose flows are the inputs u (eq. flow-constraints, u >= 0), and
demand sectors that draw the exogenous demand d.  Discretising the tank
balance exactly gives A = I; B, Gd, E, Ed are incidence matrices
(eq. dynamics and eq. input-disturbance-coupling).

Feasibility of E u + Ed d = 0 inside the input box is guaranteed by
construction: each mixing node owns one dedicated inflow whose upper
bound exceeds the largest demand that can be drawn at that node (the
demand generator clips its noise so that this bound holds).  The same
dedicated inflows make E full row rank.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Network:
    """Dynamics x+ = A x + B u + Gd d, coupling E u + Ed d = 0, boxes."""
    nx: int
    nu: int
    nd: int
    ne: int
    A: np.ndarray
    B: np.ndarray
    Gd: np.ndarray
    E: np.ndarray
    Ed: np.ndarray
    xmin: np.ndarray
    xmax: np.ndarray
    xs: np.ndarray
    umin: np.ndarray
    umax: np.ndarray
    # demand-sector description used by the data generator (not by the solver)
    dbar: np.ndarray = field(repr=False, default=None)
    phase: np.ndarray = field(repr=False, default=None)
    dmax: np.ndarray = field(repr=False, default=None)
    # energy coefficient per flow: > 0 on pumps, 0 on valves
    e_pump: np.ndarray = field(repr=False, default=None)


@dataclass
class Cost:
    """Weights of the stage cost (§3.1): W_alpha, alpha0, W_u, W_s, W_x."""
    W_alpha: float
    alpha0: np.ndarray
    Wu: np.ndarray
    Ws: float
    Wx: float


# demand noise is clipped to +-NOISE_CLIP standard deviations so that the
# dedicated inflow bounds below are never exceeded
NOISE_SIGMA = 0.1
NOISE_CLIP = 4.0
SIN_AMPLITUDE = 0.5


def _demand_upper_bound(dbar: np.ndarray) -> np.ndarray:
    return dbar * (1.0 + SIN_AMPLITUDE) * (1.0 + NOISE_SIGMA * NOISE_CLIP)


def make_network(nx: int, nu: int, nd: int, ne: int, seed: int = 1,
                 pump_fraction: float = 75.0 / 114.0) -> Network:
    """Seeded random network with the requested dimensions.

    Flow j has a source (external source, tank or mixing node) and a
    destination (tank or mixing node).  B[i, j] = +1 if flow j enters
    tank i and -1 if it leaves tank i; E[k, j] likewise for mixing node
    k.  Demand m is drawn from a tank (Gd[i, m] = -1, about 80 % of
    sectors) or from a mixing node (Ed[k, m] = -1).
    """
    if not (nx >= 1 and ne >= 0 and nu >= ne + 1 and nd >= 1):
        raise ValueError("need nx >= 1, nd >= 1, nu >= ne + 1")
    rng = np.random.default_rng(seed)
    SRC, TANK, MIX = 0, 1, 2
    src = np.zeros((nu, 2), dtype=np.int64)   # (kind, index)
    dst = np.zeros((nu, 2), dtype=np.int64)
    j = 0
    # dedicated inflow of each mixing node
    for k in range(ne):
        if rng.random() < 0.5:
            src[j] = (TANK, rng.integers(nx))
        else:
            src[j] = (SRC, 0)
        dst[j] = (MIX, k)
        j += 1
    # one refill flow per tank while flows last
    for i in range(nx):
        if j >= nu:
            break
        r = rng.random()
        if r < 0.5 or nx == 1:
            src[j] = (SRC, 0)
        elif r < 0.8 or ne == 0:
            other = int(rng.integers(nx - 1))
            src[j] = (TANK, other if other < i else other + 1)
        else:
            src[j] = (MIX, rng.integers(ne))
        dst[j] = (TANK, i)
        j += 1
    # remaining flows: random types
    while j < nu:
        r = rng.random()
        if r < 0.25 or (nx == 1 and ne == 0):
            src[j] = (SRC, 0)
            dst[j] = (TANK, rng.integers(nx))
        elif r < 0.55 and nx >= 2:
            a, b = rng.choice(nx, size=2, replace=False)
            src[j] = (TANK, a)
            dst[j] = (TANK, b)
        elif r < 0.75 and ne >= 1:
            src[j] = (TANK, rng.integers(nx))
            dst[j] = (MIX, rng.integers(ne))
        elif ne >= 1:
            src[j] = (MIX, rng.integers(ne))
            dst[j] = (TANK, rng.integers(nx))
        else:
            src[j] = (SRC, 0)
            dst[j] = (TANK, rng.integers(nx))
        j += 1

    B = np.zeros((nx, nu))
    E = np.zeros((ne, nu))
    for j in range(nu):
        kind, idx = src[j]
        if kind == TANK:
            B[idx, j] -= 1.0
        elif kind == MIX:
            E[idx, j] -= 1.0
        kind, idx = dst[j]
        if kind == TANK:
            B[idx, j] += 1.0
        else:
            E[idx, j] += 1.0

    Gd = np.zeros((nx, nd))
    Ed = np.zeros((ne, nd))
    at_mix = np.full(nd, -1, dtype=np.int64)
    for m in range(nd):
        if ne >= 1 and rng.random() < 0.2:
            k = int(rng.integers(ne))
            Ed[k, m] = -1.0
            at_mix[m] = k
        else:
            Gd[rng.integers(nx), m] = -1.0

    dbar = rng.uniform(0.2, 1.0, size=nd)
    phase = rng.uniform(0.0, 24.0, size=nd)
    dmax = _demand_upper_bound(dbar)

    umin = np.zeros(nu)
    scale = max(dmax.sum() / nx, 0.5) * 2.0
    umax = rng.uniform(1.0, 2.0, size=nu) * 1.5 * scale
    for k in range(ne):
        need = dmax[at_mix == k].sum()
        umax[k] = rng.uniform(1.0, 2.0) * 1.5 * max(need, 0.1)

    xmax = rng.uniform(50.0, 150.0, size=nx)
    xmin = np.zeros(nx)
    xs = 0.3 * xmax

    n_pump = int(round(pump_fraction * nu))
    pumps = rng.choice(nu, size=n_pump, replace=False)
    e_pump = np.zeros(nu)
    e_pump[pumps] = rng.uniform(0.5, 1.5, size=n_pump)

    return Network(nx=nx, nu=nu, nd=nd, ne=ne, A=np.eye(nx), B=B, Gd=Gd,
                   E=E, Ed=Ed, xmin=xmin, xmax=xmax, xs=xs, umin=umin,
                   umax=umax, dbar=dbar, phase=phase, dmax=dmax,
                   e_pump=e_pump)


def make_cost(net: Network, seed: int = 1, W_alpha: float = 1.0,
              wu: float = 13.0, Ws: float = 0.1, Wx: float = 100.0,
              dense_wu: bool = False) -> Cost:
    """Weights with the paper's ratios (§6.3: W_u / W_alpha = 13,
    W_s / W_alpha = 0.1, W_x / W_alpha = 100) and alpha0 ~ U[0, 0.02].

    ``dense_wu`` gives a dense symmetric positive definite W_u with the
    same diagonal scale instead of wu * I.
    """
    rng = np.random.default_rng(seed + 1000)
    alpha0 = rng.uniform(0.0, 0.02, size=net.nu)
    if dense_wu:
        M = rng.standard_normal((net.nu, net.nu)) / np.sqrt(net.nu)
        Wu = wu * (np.eye(net.nu) + 0.3 * (M @ M.T) / max(1.0, np.linalg.norm(M @ M.T, 2)))
        Wu = 0.5 * (Wu + Wu.T)
    else:
        Wu = wu * np.eye(net.nu)
    return Cost(W_alpha=float(W_alpha), alpha0=alpha0, Wu=Wu, Ws=float(Ws),
                Wx=float(Wx))
