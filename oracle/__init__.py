"""Plain FP64 CPU oracle of the dual accelerated proximal gradient method
for scenario-based stochastic MPC (paper §3-§4).

TEST INFRASTRUCTURE ONLY.  This package is the slow, obviously correct
reference that the CUDA path is checked against.  Only the test suite,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it; the product library never does, and shares no code with it.

Every function follows the paper's steps in its order and notation:

* ``factor``: the data-independent part of the dynamic-programming
  (Riccati-type) recursion that gives the dual gradient (§4.4), done in
  its general per-node form (a Cholesky factor of the reduced Hessian at
  every node), without the structural simplifications the GPU uses;
* ``dual_gradient``: x*(w) = grad f*(-H'w), eq. dual-gradient, by the
  backward/forward recursion over the tree (§4.4);
* ``prox_g``: the proximal operator of g/gamma (§4.3, distance-to-set
  prox and box projection) and the Moreau decomposition (§4.2);
* ``apg``: Nesterov's accelerated proximal gradient on the Fenchel dual,
  eqs. apg:1 / apg:2, with the theta rule that meets the requirement
  with equality (§4.3), or theta_nu = 2/(nu+2), and optionally the
  averaged primal iterate (the averaging of the cited accelerated dual
  method; the paper does not print it);
* ``power_iteration``: the Lipschitz constant of the dual gradient used
  to pick the step gamma (the paper does not state its step size).

Parity: pinned against a dense KKT solve of the tree QP, constraint
residuals, brute-force prox minimisation, the Moreau identity, the theta
identity, a scipy QP solve of the input-box-only problem, a scipy NLP of
the full problem with active soft terms (epigraph form, no duality) and a
vanishing duality gap (tests/test_oracle_*.py).
"""
from .smpc import (
    OracleProblem, Factor, SolveConsts, factor, solve_consts, dual_gradient,
    apply_H, prox_dist, prox_g, theta_beta, apg, power_iteration, splitmix64_unit,
    primal_cost, dual_value, ubox_violation, ApgResult, step_size, prox_gstar,
)

__all__ = [
    "OracleProblem", "Factor", "SolveConsts", "factor", "solve_consts",
    "dual_gradient", "apply_H", "prox_dist", "prox_g", "theta_beta", "apg",
    "power_iteration", "splitmix64_unit", "primal_cost", "dual_value",
    "ubox_violation", "ApgResult", "step_size", "prox_gstar",
]
