"""FP64 oracle of the dual APG for scenario-based stochastic MPC.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain numpy in
float64; stage loops follow the tree from the leaves to the root and
back.  Operations over the nodes of one stage are batched with numpy,
which is the paper's own observation that the nodes of a stage are
independent (§4.4); nothing is fused or reordered beyond that.

Notation (paper §2-§4):
  node nu, ancestor a(nu), probability p_nu, stage t = 0..N (N = H_p);
  every non-root node carries an input u_nu (n_u), a state x_nu (n_x) and
  a dual block y_nu = (y1, y2, y3) in R^{2 n_x + n_u} (eq. H);
  the root carries the fixed x_0 = p and u_{-1} = q (eq. SMPC initial
  conditions).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


# ----------------------------------------------------------------------------
# problem data
# ----------------------------------------------------------------------------
@dataclass
class OracleProblem:
    """Network (§2.1 eq. dynamics / input-disturbance-coupling, boxes
    eq. state-constraints / input-constraints), cost weights (§3.1) and the
    scenario tree (§2.3)."""
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
    W_alpha: float
    alpha0: np.ndarray
    Wu: np.ndarray
    Ws: float
    Wx: float
    N: int
    stage_ptr: np.ndarray
    anc: np.ndarray
    prob: np.ndarray

    @classmethod
    def from_parts(cls, net, cost, tree) -> "OracleProblem":
        return cls(A=np.array(net.A, float), B=np.array(net.B, float),
                   Gd=np.array(net.Gd, float), E=np.array(net.E, float).reshape(-1, net.nu),
                   Ed=np.array(net.Ed, float).reshape(-1, net.nd),
                   xmin=np.array(net.xmin, float), xmax=np.array(net.xmax, float),
                   xs=np.array(net.xs, float), umin=np.array(net.umin, float),
                   umax=np.array(net.umax, float), W_alpha=float(cost.W_alpha),
                   alpha0=np.array(cost.alpha0, float), Wu=np.array(cost.Wu, float),
                   Ws=float(cost.Ws), Wx=float(cost.Wx), N=int(tree.N),
                   stage_ptr=np.array(tree.stage_ptr, np.int64),
                   anc=np.array(tree.anc, np.int64), prob=np.array(tree.prob, float))

    @property
    def nx(self) -> int:
        return self.B.shape[0]

    @property
    def nu(self) -> int:
        return self.B.shape[1]

    @property
    def nd(self) -> int:
        return self.Gd.shape[1]

    @property
    def ne(self) -> int:
        return self.E.shape[0]

    @property
    def n_nodes(self) -> int:
        return int(self.stage_ptr[self.N + 1])

    @property
    def ny(self) -> int:
        return 2 * self.nx + self.nu

    def stage(self, t: int) -> slice:
        return slice(int(self.stage_ptr[t]), int(self.stage_ptr[t + 1]))


def _child_sum(P: OracleProblem, t: int, vals: np.ndarray) -> np.ndarray:
    """Sum over child(nu) of the stage-(t+1) values, for every stage-t node
    nu; children are added in ascending node order."""
    s = P.stage(t)
    c = P.stage(t + 1)
    out = np.zeros((s.stop - s.start,) + vals.shape[1:])
    np.add.at(out, P.anc[c] - s.start, vals)
    return out


# ----------------------------------------------------------------------------
# factor step (§4.4 "Riccati-type recursion"; Table 2 Engine::factorStep)
# ----------------------------------------------------------------------------
@dataclass
class Factor:
    L: np.ndarray       # (n_u, n_v) orthonormal basis of ker E
    Epinv: np.ndarray   # (n_u, n_e) Moore-Penrose inverse of E
    Phi: np.ndarray     # (n_nodes, n_u, n_u)  L (L'Q L)^{-1} L'
    K: np.ndarray       # (n_nodes, n_u, n_u)  2 p Phi W_u
    Nm: np.ndarray      # (n_nodes, n_u, n_u)  I - Phi Q
    Pm: np.ndarray = field(repr=False, default=None)  # (n_nodes, n_u, n_u)


def factor(P: OracleProblem, keep_P: bool = False) -> Factor:
    """Data-independent part of the dynamic programme that evaluates
    grad f* (eq. dual-gradient) on the tree.

    The cost-to-go of node nu, as a function of its ancestor's state and
    input (x_a, u_a), is  ell_nu' x_a + 1/2 u_a' P_nu u_a + r_nu' u_a + c
    (x has no quadratic cost, so the cost-to-go is linear in x).  Going
    from stage N down to stage 1:

        Q_nu   = 2 p_nu W_u + sum_{c in child(nu)} P_c
        Phi_nu = L (L' Q_nu L)^{-1} L'        (L spans ker E, eq. Phi_1)
        K_nu   = 2 p_nu Phi_nu W_u
        P_nu   = 2 p_nu W_u - (2 p_nu W_u) Phi_nu (2 p_nu W_u)

    L' Q_nu L is factored by Cholesky at every node; a failure means W_u is
    not positive definite on ker E.
    """
    nu, ne = P.nu, P.ne
    if ne > 0:
        if np.linalg.matrix_rank(P.E) < ne:
            raise np.linalg.LinAlgError("E does not have full row rank")
        # ker E from the SVD of E
        _, sv, Vt = np.linalg.svd(P.E)
        L = Vt[ne:].T.copy()
        Epinv = np.linalg.pinv(P.E)
    else:
        L = np.eye(nu)
        Epinv = np.zeros((nu, 0))
    np.linalg.cholesky(P.Wu)  # raises unless W_u is positive definite
    n = P.n_nodes
    Phi = np.zeros((n, nu, nu))
    K = np.zeros((n, nu, nu))
    Nm = np.zeros((n, nu, nu))
    Pm = np.zeros((n, nu, nu))
    I = np.eye(nu)
    for t in range(P.N, 0, -1):
        s = P.stage(t)
        p = P.prob[s]
        W2 = 2.0 * p[:, None, None] * P.Wu[None, :, :]
        Q = W2.copy()
        if t < P.N:
            Q += _child_sum(P, t, Pm[P.stage(t + 1)])
        LQL = L.T[None] @ Q @ L[None]
        np.linalg.cholesky(LQL)  # positive definiteness of the reduced Hessian
        Phi_t = L[None] @ np.linalg.solve(LQL, np.broadcast_to(L.T, LQL.shape[:1] + L.T.shape))
        Phi[s] = Phi_t
        K[s] = Phi_t @ W2
        Nm[s] = I[None] - Phi_t @ Q
        Pm[s] = W2 - W2 @ Phi_t @ W2
    return Factor(L=L, Epinv=Epinv, Phi=Phi, K=K, Nm=Nm, Pm=Pm if keep_P else None)


# ----------------------------------------------------------------------------
# per-solve constants
# ----------------------------------------------------------------------------
@dataclass
class SolveConsts:
    x0: np.ndarray   # (n_x,)  x_{k|k} = p
    q: np.ndarray    # (n_u,)  u_{k-1|k} = q
    d: np.ndarray    # (n_nodes, n_d)
    alpha: np.ndarray  # (n_nodes, n_u)
    c0: np.ndarray   # (n_nodes, n_u)  p_nu W_alpha (alpha0 + alpha_nu)
    ud: np.ndarray   # (n_nodes, n_u)  particular solution of E u + Ed d = 0
    mc: np.ndarray   # (n_nodes, n_u)  (I - Phi Q) ud
    gd: np.ndarray   # (n_nodes, n_x)  Gd d_nu


def solve_consts(P: OracleProblem, F: Factor, x0, q, demand, alpha) -> SolveConsts:
    """Linear cost c0 = p W_alpha (alpha0 + alpha) (eq. cost:linear inside
    the expectation of eq. SMPC), a particular solution ud = -E^+ Ed d of
    the coupling eq. input-disturbance-coupling, and Gd d (eq. dynamics)."""
    n = P.n_nodes
    d = np.array(demand, float).reshape(n, P.nd)
    al = np.array(alpha, float).reshape(n, P.nu)
    c0 = P.prob[:, None] * P.W_alpha * (P.alpha0[None, :] + al)
    ud = -(d @ P.Ed.T) @ F.Epinv.T
    mc = np.einsum("nij,nj->ni", F.Nm, ud)
    gd = d @ P.Gd.T
    c0[0] = 0.0
    ud[0] = 0.0
    mc[0] = 0.0
    gd[0] = 0.0
    return SolveConsts(x0=np.array(x0, float), q=np.array(q, float), d=d, alpha=al,
                       c0=c0, ud=ud, mc=mc, gd=gd)


# ----------------------------------------------------------------------------
# dual gradient: x*(w) = argmin_x f(x) + <w, H x>   (eq. dual-gradient)
# ----------------------------------------------------------------------------
def dual_gradient(P: OracleProblem, F: Factor, S: SolveConsts, w: np.ndarray,
                  constants: bool = True):
    """Solve step of §4.4: the minimiser of f(x) + <w, Hx> over the tree
    dynamics (eq. dynamics:tree) and couplings (eq. Phi_1, Phi_2).

    Backward (stage N to 1), with w_nu = (w1, w2, w3):
        lambda_nu = w1 + w2 + A' sum_c lambda_c
        g_nu      = c0_nu + w3 + B' lambda_nu + sum_c r_c
        m_nu      = (I - Phi_nu Q_nu) ud_nu - Phi_nu g_nu
        r_nu      = -2 p_nu W_u m_nu
    Forward (stage 1 to N):
        u_nu = m_nu + K_nu u_a(nu),  x_nu = A x_a(nu) + B u_nu + Gd d_nu,
    from u_root = q, x_root = x0.  With constants=False every data term
    (c0, d, x0, q) is zero, which gives the linear part of w -> x*(w).
    Returns (u, x) with the root rows holding (q, x0).
    """
    n, nx, nu = P.n_nodes, P.nx, P.nu
    w = np.asarray(w, float).reshape(n, P.ny)
    w1, w2, w3 = w[:, :nx], w[:, nx:2 * nx], w[:, 2 * nx:]
    lam = np.zeros((n, nx))
    m = np.zeros((n, nu))
    r = np.zeros((n, nu))
    for t in range(P.N, 0, -1):
        s = P.stage(t)
        lam_t = w1[s] + w2[s]
        g_t = w3[s].copy()
        if constants:
            g_t = g_t + S.c0[s]
        if t < P.N:
            c = P.stage(t + 1)
            lam_t = lam_t + _child_sum(P, t, lam[c]) @ P.A
            g_t = g_t + _child_sum(P, t, r[c])
        g_t = g_t + lam_t @ P.B
        m_t = -np.einsum("nij,nj->ni", F.Phi[s], g_t)
        if constants:
            m_t = m_t + S.mc[s]
        lam[s] = lam_t
        m[s] = m_t
        r[s] = -2.0 * P.prob[s][:, None] * (m_t @ P.Wu.T)
    u = np.zeros((n, nu))
    x = np.zeros((n, nx))
    if constants:
        u[0] = S.q
        x[0] = S.x0
    for t in range(1, P.N + 1):
        s = P.stage(t)
        a = P.anc[s]
        u[s] = m[s] + np.einsum("nij,nj->ni", F.K[s], u[a])
        x_t = x[a] @ P.A.T + u[s] @ P.B.T
        if constants:
            x_t = x_t + S.gd[s]
        x[s] = x_t
    return u, x


def apply_H(P: OracleProblem, u: np.ndarray, x: np.ndarray) -> np.ndarray:
    """H maps (x_nu, u_nu) to (x_nu, x_nu, u_nu) at every non-root node
    (eq. H); the root row is zero."""
    Hx = np.concatenate([x, x, u], axis=1)
    Hx[0] = 0.0
    return Hx


# ----------------------------------------------------------------------------
# proximal operators (§4.2-§4.3)
# ----------------------------------------------------------------------------
def proj_box(v, lo, hi):
    return np.minimum(np.maximum(v, lo), hi)


def prox_dist(v: np.ndarray, lam: float, proj) -> np.ndarray:
    """prox of lam * dist(. | C), row by row (§4.3):
        v + lam (proj_C(v) - v) / dist(v | C)   if dist(v | C) > lam,
        proj_C(v)                               otherwise.
    (The paper prints the first branch without the factor lam; the
    minimiser of lam dist(x|C) + 1/2 |x - v|^2 carries it.)"""
    pv = proj(v)
    dist = np.linalg.norm(v - pv, axis=-1, keepdims=True)
    far = dist > lam
    safe = np.where(far, dist, 1.0)
    return np.where(far, v + lam * (pv - v) / safe, pv)


def prox_g(P: OracleProblem, v: np.ndarray, scale: float) -> np.ndarray:
    """prox of scale * g (eq. g), block by block: W_x dist(. | [xmin, xmax])
    on y1, W_s dist(. | [x_s, inf)) on y2, the indicator of U on y3; the
    root row is left at zero."""
    nx = P.nx
    v = np.asarray(v, float)
    t = np.zeros_like(v)
    sl = slice(1, None)
    t[sl, :nx] = prox_dist(v[sl, :nx], scale * P.Wx,
                           lambda z: proj_box(z, P.xmin, P.xmax))
    t[sl, nx:2 * nx] = prox_dist(v[sl, nx:2 * nx], scale * P.Ws,
                                 lambda z: np.maximum(z, P.xs))
    t[sl, 2 * nx:] = proj_box(v[sl, 2 * nx:], P.umin, P.umax)
    return t


def prox_gstar(P: OracleProblem, z: np.ndarray, gamma: float):
    """prox_{gamma g*}(z) by the Moreau decomposition (eq.
    moreau-decomposition): prox_{gamma g*}(z) = z - gamma prox_{g/gamma}(z/gamma).
    Returns (prox, t) with t = prox_{g/gamma}(z/gamma)."""
    t = prox_g(P, z / gamma, 1.0 / gamma)
    return z - gamma * t, t


# ----------------------------------------------------------------------------
# accelerated proximal gradient on the dual (§4.3)
# ----------------------------------------------------------------------------
def theta_beta(n: int, rule: str = "equality"):
    """theta_{-1} = theta_0 = 1 and beta_nu = theta_nu (1/theta_{nu-1} - 1)
    (§4.3), with theta_{nu+1} = (sqrt(theta^4 + 4 theta^2) - theta^2) / 2
    (rule "equality", the paper's choice, which meets the requirement
    1 - theta_{nu+1} <= theta_{nu+1}^2 / theta_nu^2 with equality) or
    theta_nu = 2 / (nu + 2) (rule "simple", the other choice §4.3 names).
    Returns (beta[0..n-1], theta[0..n])."""
    if rule not in ("equality", "simple"):
        raise ValueError("rule must be 'equality' or 'simple'")
    theta = np.empty(n + 1)
    theta[0] = 1.0
    beta = np.empty(n)
    prev = 1.0
    for k in range(n):
        beta[k] = theta[k] * (1.0 / prev - 1.0)
        th = theta[k]
        if rule == "equality":
            theta[k + 1] = 0.5 * (np.sqrt(th ** 4 + 4.0 * th ** 2) - th ** 2)
        else:
            theta[k + 1] = 2.0 / (k + 3)
        prev = th
    return beta, theta


@dataclass
class ApgResult:
    y: np.ndarray          # final dual iterate (n_nodes, 2 n_x + n_u)
    u: np.ndarray          # x*(w) of the last iteration: inputs
    x: np.ndarray          # ... and states
    iters: int
    residual: float        # |H x*(w) - t|_inf of the last iteration
    res_hist: np.ndarray
    gamma: float
    converged: bool
    u_avg: np.ndarray = None  # averaged primal iterate (average=True): inputs
    x_avg: np.ndarray = None  # ... and states


def apg(P: OracleProblem, F: Factor, S: SolveConsts, iters: int, gamma: float,
        tol: float = 0.0, check_every: int = 1, y0=None, y_prev0=None,
        theta_rule: str = "equality", average: bool = False) -> ApgResult:
    """Eqs. apg:1 / apg:2 from y^0 = y^{-1} = 0 (or a warm start):
        w^nu     = y^nu + beta_nu (y^nu - y^{nu-1})
        y^{nu+1} = prox_{gamma g*}(w^nu + gamma H grad f*(-H' w^nu)).
    The residual of iteration nu is |H x*(w^nu) - t^nu|_inf where t^nu is
    the prox of g/gamma inside the Moreau decomposition; it is compared
    with tol at every check_every-th iteration and at the last one.
    theta_rule picks the extrapolation sequence (theta_beta).  average
    also returns the averaged primal iterate that §4.3 credits with the
    O(1/nu^2) rate; the paper does not print it, and the reading taken is
    the averaging of the accelerated dual method it cites,
        xbar^nu = (1 - theta_nu) xbar^{nu-1} + theta_nu x*(w^nu),
    which with theta_0 = 1 starts at xbar^0 = x*(w^0).
    """
    n = P.n_nodes
    y = np.zeros((n, P.ny)) if y0 is None else np.array(y0, float).reshape(n, P.ny)
    y_prev = y.copy() if y_prev0 is None else np.array(y_prev0, float).reshape(n, P.ny)
    y[0] = 0.0
    y_prev[0] = 0.0
    beta, theta = theta_beta(max(iters, 1), theta_rule)
    hist = np.zeros(iters)
    u = x = None
    u_avg = x_avg = None
    res = np.inf
    done = 0
    converged = False
    for k in range(iters):
        w = y + beta[k] * (y - y_prev)
        u, x = dual_gradient(P, F, S, w)
        if average:
            if u_avg is None:
                u_avg, x_avg = u.copy(), x.copy()
            else:
                u_avg = (1.0 - theta[k]) * u_avg + theta[k] * u
                x_avg = (1.0 - theta[k]) * x_avg + theta[k] * x
        Hx = apply_H(P, u, x)
        y_new, t = prox_gstar(P, w + gamma * Hx, gamma)
        y_new[0] = 0.0
        res = float(np.max(np.abs((Hx - t)[1:])))
        hist[k] = res
        y_prev, y = y, y_new
        done = k + 1
        if tol > 0.0 and (done % check_every == 0 or done == iters) and res <= tol:
            converged = True
            break
    return ApgResult(y=y, u=u, x=x, iters=done, residual=res, res_hist=hist[:done],
                     gamma=gamma, converged=converged, u_avg=u_avg, x_avg=x_avg)


# ----------------------------------------------------------------------------
# step size: Lipschitz constant of the dual gradient
# ----------------------------------------------------------------------------
_SM_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_SM_M1 = np.uint64(0xBF58476D1CE4E5B9)
_SM_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64_unit(index: np.ndarray, seed: int = 0) -> np.ndarray:
    """Output number index+1 of the SplitMix64 generator (Steele, Lea and
    Flood, OOPSLA 2014) started from `seed`, as a double in [0, 1) from its
    top 53 bits."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (np.asarray(index, np.uint64) + np.uint64(1)) * _SM_GAMMA
        z = (z ^ (z >> np.uint64(30))) * _SM_M1
        z = (z ^ (z >> np.uint64(27))) * _SM_M2
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def power_iteration(P: OracleProblem, F: Factor, n_iter: int = 200, seed: int = 0):
    """Largest eigenvalue of the symmetric positive semidefinite map
    M v = -H x_lin(v), where x_lin is the linear part of the dual gradient
    (constants set to zero); M is the Hessian of f*(-H' .), so its largest
    eigenvalue is the Lipschitz constant of the dual gradient.  Start
    vector: 1 + SplitMix64 numbers over the non-root dual entries in node
    order.  Returns the last |M v| with |v| = 1."""
    n, ny = P.n_nodes, P.ny
    v = np.zeros((n, ny))
    v[1:] = 1.0 + splitmix64_unit(np.arange((n - 1) * ny), seed).reshape(n - 1, ny)
    v /= np.linalg.norm(v)
    est = 0.0
    for _ in range(n_iter):
        u, x = dual_gradient(P, F, None, v, constants=False)
        Mv = -apply_H(P, u, x)
        est = float(np.linalg.norm(Mv))
        v = Mv / est
    return est


def step_size(L: float, margin: float = 1.01) -> float:
    return 1.0 / (margin * L)


# ----------------------------------------------------------------------------
# objective values
# ----------------------------------------------------------------------------
def _smooth_cost(P: OracleProblem, S: SolveConsts, u: np.ndarray) -> float:
    """f on the dynamics/coupling set: sum_nu p_nu [W_alpha (alpha0 +
    alpha_nu)' u_nu + du' W_u du], du = u_nu - u_a(nu) (eqs. cost:linear,
    cost:smooth, f)."""
    du = u[1:] - u[P.anc[1:]]
    lin = float(np.sum(S.c0[1:] * u[1:]))
    quad = float(np.sum(P.prob[1:] * np.einsum("ni,ij,nj->n", du, P.Wu, du)))
    return lin + quad


def _soft_cost(P: OracleProblem, x: np.ndarray) -> float:
    """V_s: W_x dist(x | [xmin, xmax]) + W_s dist(x | [x_s, inf)) per node,
    Euclidean distance, summed over the non-root nodes (eqs. cost:non-smooth,
    g); not probability weighted."""
    xx = x[1:]
    dx = np.linalg.norm(xx - proj_box(xx, P.xmin, P.xmax), axis=1)
    ds = np.linalg.norm(xx - np.maximum(xx, P.xs), axis=1)
    return float(P.Wx * dx.sum() + P.Ws * ds.sum())


def primal_cost(P: OracleProblem, S: SolveConsts, u: np.ndarray, x: np.ndarray) -> float:
    """Objective of eq. SMPC at (u, x), without the indicator of U (the
    input-box violation is reported separately by ubox_violation)."""
    return _smooth_cost(P, S, u) + _soft_cost(P, x)


def ubox_violation(P: OracleProblem, u: np.ndarray) -> float:
    uu = u[1:]
    return float(max(0.0, np.max(P.umin - uu), np.max(uu - P.umax)))


def dual_value(P: OracleProblem, F: Factor, S: SolveConsts, y: np.ndarray,
               rtol: float = 1e-9) -> float:
    """-f*(-H'y) - g*(y) = f(x*(y)) + <y, H x*(y)> - g*(y) (eq. fenchel-dual,
    with f* through eq. dual-gradient).  g* per node: the support function
    of [xmin, xmax] on y1 with |y1| <= W_x, <y2, x_s> with y2 <= 0 and
    |y2| <= W_s, the support function of U on y3.  Returns -inf outside
    dom g* (relative slack rtol)."""
    nx = P.nx
    y = np.asarray(y, float).reshape(P.n_nodes, P.ny)
    u, x = dual_gradient(P, F, S, y)
    Hx = apply_H(P, u, x)
    yy = y[1:]
    y1, y2, y3 = yy[:, :nx], yy[:, nx:2 * nx], yy[:, 2 * nx:]
    if np.any(np.linalg.norm(y1, axis=1) > P.Wx * (1 + rtol) + 1e-300):
        return -np.inf
    if np.any(np.linalg.norm(y2, axis=1) > P.Ws * (1 + rtol) + 1e-300):
        return -np.inf
    if np.any(y2 > rtol * max(P.Ws, 1e-300)):
        return -np.inf
    sig_x = np.sum(np.maximum(y1 * P.xmax, y1 * P.xmin))
    sig_s = np.sum(y2 * P.xs)
    sig_u = np.sum(np.maximum(y3 * P.umax, y3 * P.umin))
    gstar = float(sig_x + sig_s + sig_u)
    return _smooth_cost(P, S, u) + float(np.sum(y[1:] * Hx[1:])) - gstar
