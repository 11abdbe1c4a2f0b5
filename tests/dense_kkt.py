"""Dense KKT solve of the scenario-tree QP that defines the dual gradient.

An independent formulation of x*(w) = argmin f(x) + <w, Hx> (paper eq.
dual-gradient with f of eq. f): all inputs and states of the non-root
nodes are stacked into one vector, the smooth cost becomes one dense
Hessian, the tree dynamics (eq. dynamics:tree) and the couplings
(eq. input-disturbance-coupling) become one dense constraint matrix, and
the optimality system is solved with numpy.linalg.solve.  No recursion
over the tree is used.  Only for small trees (a few hundred nodes).
"""
import numpy as np


def kkt_dual_gradient(P, w, x0, q, demand, alpha, constants=True):
    n, nx, nu, ne = P.n_nodes, P.nx, P.nu, P.ne
    m = n - 1
    nz = m * (nu + nx)
    iu = lambda k: slice((k - 1) * nu, k * nu)            # u of node k >= 1
    ix = lambda k: slice(m * nu + (k - 1) * nx, m * nu + k * nx)
    if not constants:
        x0 = np.zeros(nx); q = np.zeros(nu)
        demand = np.zeros((n, P.nd)); alpha = np.zeros((n, nu))
    w = np.asarray(w, float).reshape(n, 2 * nx + nu)
    Hq = np.zeros((nz, nz))
    h = np.zeros(nz)
    for k in range(1, n):
        a = int(P.anc[k])
        W2 = 2.0 * P.prob[k] * P.Wu
        Hq[iu(k), iu(k)] += W2
        lin = w[k, 2 * nx:].copy()
        if constants:
            lin += P.prob[k] * P.W_alpha * (P.alpha0 + alpha[k])
        if a == 0:
            lin -= W2 @ q
        else:
            Hq[iu(a), iu(a)] += W2
            Hq[iu(k), iu(a)] -= W2
            Hq[iu(a), iu(k)] -= W2
        h[iu(k)] += lin
        h[ix(k)] += w[k, :nx] + w[k, nx:2 * nx]
    nc = m * (nx + ne)
    C = np.zeros((nc, nz))
    b = np.zeros(nc)
    for k in range(1, n):
        a = int(P.anc[k])
        r = slice((k - 1) * (nx + ne), (k - 1) * (nx + ne) + nx)
        C[r, ix(k)] = np.eye(nx)
        C[r, iu(k)] = -P.B
        rhs = P.Gd @ demand[k]
        if a == 0:
            rhs = rhs + P.A @ x0
        else:
            C[r, ix(a)] = -P.A
        b[r] = rhs
        if ne:
            r2 = slice((k - 1) * (nx + ne) + nx, k * (nx + ne))
            C[r2, iu(k)] = P.E
            b[r2] = -P.Ed @ demand[k]
    KKT = np.block([[Hq, C.T], [C, np.zeros((nc, nc))]])
    sol = np.linalg.solve(KKT, np.concatenate([-h, b]))
    z = sol[:nz]
    u = np.zeros((n, nu)); x = np.zeros((n, nx))
    u[0] = q; x[0] = x0
    for k in range(1, n):
        u[k] = z[iu(k)]
        x[k] = z[ix(k)]
    return u, x
