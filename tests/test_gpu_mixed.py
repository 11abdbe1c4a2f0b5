"""Mixed precision (FP32 iteration around an FP64 reference) against the FP64
oracle at the same iteration count.

Bar (the accuracy statement of the mixed-precision mode): cost within
1e-3 relative of the oracle's; the returned (u, x) satisfy the dynamics
and couplings (they come from an FP64 evaluation of the dual gradient at
the last w) to 1e-9 of their scale, i.e. primal infeasibility far below
1e-4; the input-box violation within 1e-4 of the oracle's.  The relative
errors of u, x and y are reported in the assertion messages.
"""
import numpy as np
import pytest

import oracle as O
import paper_1904_10548_gb300 as rn
from paper_1904_10548_gb300 import _binding as B
from tests.test_gpu_parity import oracle_for, problem, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()


def infeasibility(pb, u, x):
    net, tree, d = pb.net, pb.tree, pb.data
    a = tree.anc[1:]
    dyn = x[1:] - x[a] - u[1:] @ net.B.T - d.demand[1:] @ net.Gd.T
    cpl = u[1:] @ net.E.T + d.demand[1:] @ net.Ed.T if net.ne else np.zeros(1)
    return float(max(np.abs(dyn).max(), np.abs(cpl).max()))


@pytest.mark.parametrize("kind,iters", [("tiny", 500), ("barcelona32", 300), ("uneven1", 400),
                                        ("uneven2", 300), ("tight", 500), ("single", 400),
                                        ("ne0", 400), ("stage1_chains", 400)])
def test_mixed_matches_oracle(kind, iters):
    pb = problem(kind)
    P, F, S = oracle_for(kind, pb)
    gamma = O.step_size(O.power_iteration(P, F, 100))
    ref = O.apg(P, F, S, iters, gamma)
    fac = rn.Factor(pb.net, pb.cost, pb.tree, gamma=gamma, precision=rn.RN_PREC_MIXED)
    out = fac.solve(pb.data.x0, pb.data.q, pb.data.demand, pb.data.alpha, max_iters=iters,
                    res_hist_len=1000)
    fac.close()
    assert out["status"] == B.RN_OK and out["iters"] == iters
    cost = O.primal_cost(P, S, ref.u, ref.x)
    msg = (f"{kind}: cost rel {abs(out['cost'] - cost) / abs(cost):.2e}, u {rel_err(out['u'], ref.u):.2e},"
           f" x {rel_err(out['x'], ref.x):.2e}, y {rel_err(out['y'], ref.y):.2e},"
           f" res {out['primal_res']:.3e} vs {ref.residual:.3e}")
    assert abs(out["cost"] - cost) <= 1e-3 * abs(cost), msg
    scale = max(np.abs(out["x"]).max(), np.abs(out["u"]).max())
    assert infeasibility(pb, out["u"], out["x"]) <= 1e-9 * scale, msg
    assert abs(out["ubox_viol"] - O.ubox_violation(P, ref.u)) <= 1e-4, msg
    assert rel_err(out["u"], ref.u) <= 1e-3, msg
    assert rel_err(out["y"], ref.y) <= 1e-3, msg


def test_mixed_tolerance_stop():
    pb = problem("tiny")
    P, F, S = oracle_for("tiny", pb)
    gamma = O.step_size(O.power_iteration(P, F, 100))
    fac = rn.Factor(pb.net, pb.cost, pb.tree, gamma=gamma, precision=rn.RN_PREC_MIXED)
    out = fac.solve(pb.data.x0, pb.data.q, pb.data.demand, pb.data.alpha, max_iters=20000,
                    tol=1e-3)
    fac.close()
    ref = O.apg(P, F, S, 20000, gamma, tol=1e-3, check_every=10)
    assert out["status"] == B.RN_OK and out["primal_res"] <= 1e-3
    assert abs(out["iters"] - ref.iters) <= 50, (out["iters"], ref.iters)


def spread(a, b):
    return dict(cost=abs(a["cost"] - b["cost"]) / abs(b["cost"]), u=rel_err(a["u"], b["u"]),
                y=rel_err(a["y"], b["y"]))


@pytest.mark.slow
@pytest.mark.parametrize("iters", [500, 2000])
def test_mixed_full_size_against_fp64_gpu(iters):
    """512-scenario tree, bench configuration, against the FP64 path at the
    same iteration count.  Far from convergence the accelerated iteration
    carries any perturbation forward and amplifies it (an FP64 run whose step
    size differs by one FP32 ulp drifts from the unperturbed one by a growing
    amount), so the bar is the larger of 1e-3 and twenty times that FP64
    spread, for the cost, u and y.  The returned primal satisfies the
    dynamics and couplings, and the mixed path's residual and input-box
    violation (the primal infeasibility of the reading of the paper's
    tolerance) are within 10 % of the FP64 path's."""
    pb = problem("barcelona512")
    d = pb.data
    f64 = rn.Factor(pb.net, pb.cost, pb.tree)
    gamma = f64.info()["gamma"]
    a = f64.solve(d.x0, d.q, d.demand, d.alpha, max_iters=iters)
    f64.close()
    f64b = rn.Factor(pb.net, pb.cost, pb.tree, gamma=gamma * (1.0 + 2.0 ** -23))
    e = f64b.solve(d.x0, d.q, d.demand, d.alpha, max_iters=iters)
    f64b.close()
    mx = rn.Factor(pb.net, pb.cost, pb.tree, gamma=gamma, precision=rn.RN_PREC_MIXED)
    b = mx.solve(d.x0, d.q, d.demand, d.alpha, max_iters=iters)
    mx.close()
    env, got = spread(e, a), spread(b, a)
    msg = f"mixed vs FP64 {got}; FP64 one-ulp spread {env}; res {a['primal_res']:.4g} vs {b['primal_res']:.4g}"
    for k in ("cost", "u", "y"):
        assert got[k] <= max(1e-3, 20.0 * env[k]), msg
    scale = max(np.abs(b["x"]).max(), np.abs(b["u"]).max())
    assert infeasibility(pb, b["u"], b["x"]) <= 1e-9 * scale, msg
    assert abs(b["primal_res"] - a["primal_res"]) <= 0.1 * a["primal_res"], msg
    assert abs(b["ubox_viol"] - a["ubox_viol"]) <= 0.1 * max(a["ubox_viol"], 1e-6), msg
