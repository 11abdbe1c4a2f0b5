"""Closed-loop operation of the stochastic MPC (the experiment shape of
paper §6.3): at every hour the controller solves the problem on the
scenario tree from the current tank levels, applies the first move, and
the network moves on by one hour.

The scenario tree must have a single stage-1 node (branching 1 at the
root), so that the first move is one input vector: u at that node.  The
solves run on the GPU through the C ABI (``Factor.solve``); what this
module adds is bookkeeping on the host:
  * the plant update x_{k+1} = x_k + B u_k + Gd d_k (A = I, eq. dynamics
    of §2.1) with the realised demand of the hour, taken equal to the
    forecast at the stage-1 node (the current hour's demand is known);
  * warm starts: each solve starts from the previous solve's dual;
  * the three indices of §6.3:
      KPI_E   = (1/Hs) sum_k (alpha0 + alpha_k)' u_k      (average hourly cost)
      KPI_S   = sum_k || max(x_s - x_k, 0) ||_1           (safety violation)
      KPI_tau = max_k tau_k                               (worst solve time)
    with tau_k the wall time of the solve call (host to host) and, beside
    it, the device time of its APG iterations.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np


@dataclass
class ClosedLoopResult:
    x: np.ndarray            # (steps + 1, nx) tank levels, x[0] the initial state
    u: np.ndarray            # (steps, nu) applied first moves
    demand: np.ndarray       # (steps, nd) realised demands
    alpha: np.ndarray        # (steps, nu) prices times energy coefficients of the hour
    tau_s: np.ndarray        # (steps,) wall time of each solve call
    apg_ms: np.ndarray       # (steps,) device time of each solve's iterations
    iters: np.ndarray        # (steps,) iterations of each solve
    residual: np.ndarray     # (steps,) final residual of each solve
    status: list = field(default_factory=list)
    kpi_e: float = 0.0
    kpi_s: float = 0.0
    kpi_tau: float = 0.0
    kpi_tau_device: float = 0.0


def kpis(alpha0, alpha, u, xs, x) -> tuple:
    """KPI_E and KPI_S of §6.3 for applied moves u (steps, nu) with prices
    alpha (steps, nu) and the states x_1 .. x_Hs (steps, nx)."""
    steps = u.shape[0]
    kpi_e = float(np.sum((alpha0[None, :] + alpha) * u)) / max(steps, 1)
    kpi_s = float(np.sum(np.maximum(xs[None, :] - x, 0.0)))
    return kpi_e, kpi_s


def simulate(fac, net, cost, forecast: Callable[[int], tuple], x0, u_prev, steps: int = 168,
             max_iters: int = 2000, tol: float = 0.0, warm: bool = True,
             stage1_node: int = 1, solve: Optional[Callable] = None) -> ClosedLoopResult:
    """Run `steps` hours of closed-loop operation.

    fac: a Factor of the network, cost and a tree with one stage-1 node
    (node 1).  forecast(k) -> (demand, alpha): the per-node forecasts of
    hour k on that tree (rows as for Factor.solve).  solve: replaces
    fac.solve (same signature and result keys), for tests of the host
    logic without a device.
    """
    solve = solve or fac.solve
    nx, nu, nd = net.nx, net.nu, net.nd
    B = np.asarray(net.B, float).reshape(nx, nu)
    Gd = np.asarray(net.Gd, float).reshape(nx, nd)
    x = np.empty((steps + 1, nx))
    x[0] = np.asarray(x0, float)
    U = np.empty((steps, nu))
    D = np.empty((steps, nd))
    AL = np.empty((steps, nu))
    tau = np.empty(steps)
    apg = np.empty(steps)
    its = np.empty(steps, dtype=np.int64)
    res = np.empty(steps)
    status = []
    q = np.asarray(u_prev, float)
    y = None
    for k in range(steps):
        demand, alpha = forecast(k)
        t0 = time.perf_counter()
        r = solve(x[k], q, demand, alpha, max_iters=max_iters, tol=tol,
                  y_warm=y if warm else None)
        tau[k] = time.perf_counter() - t0
        apg[k] = r["apg_ms"]
        its[k] = r["iters"]
        res[k] = r["primal_res"]
        status.append(r["status"])
        y = r["y"]
        U[k] = r["u"][stage1_node]
        D[k] = demand[stage1_node]
        AL[k] = alpha[stage1_node]
        x[k + 1] = x[k] + B @ U[k] + Gd @ D[k]
        q = U[k]
    out = ClosedLoopResult(x=x, u=U, demand=D, alpha=AL, tau_s=tau, apg_ms=apg, iters=its,
                           residual=res, status=status)
    out.kpi_e, out.kpi_s = kpis(np.asarray(cost.alpha0, float), AL, U,
                                np.asarray(net.xs, float), x[1:])
    out.kpi_tau = float(tau.max()) if steps else 0.0
    out.kpi_tau_device = float(apg.max()) / 1e3 if steps else 0.0
    return out
