"""Parity of the per-node factor form (general recursion of §4.4, one
matrix pair per node streamed from device memory) with the FP64 oracle,
through the C ABI.

Bars: FP64 dual gradient 1e-9 relative (the two sides add in different
orders; nothing else differs), FP64 APG iterates 1e-6 (the parity bar of
the FP64 path); FP32 iteration against the oracle 2e-4 relative on one
dual-gradient evaluation (FP32 arithmetic, unit roundoff 6e-8, through
the matrix products and sums of a 24-stage recursion).  A != I throughout
except where the test compares with the shared-operator form.
"""
import numpy as np
import pytest

import oracle as O
import paper_1904_10548_gb300 as rn
from paper_1904_10548_gb300 import _binding as B
from synthetic import make_cost, make_data, make_network, make_problem, make_tree, random_branching
from synthetic.configs import Problem

pytestmark = pytest.mark.gpu

PN = rn.RN_FACTOR_PER_NODE


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    assert torch.cuda.is_available()


def rel_err(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300))


def general_A(nx, seed):
    rng = np.random.default_rng(seed)
    A = np.eye(nx) * (1.0 - 0.01 * rng.random(nx))
    mask = rng.random((nx, nx)) < 0.1
    return A + 0.03 * rng.standard_normal((nx, nx)) * mask


def problem(kind):
    """kind[:-2] == '_A': the same workload with a general A."""
    base = kind[:-2] if kind.endswith("_A") else kind
    if base in ("tiny", "barcelona32", "barcelona512"):
        pb = make_problem(base)
    elif base.startswith("uneven"):
        seed = int(base[6:] or 0)
        net = make_network(16, 29, 22, 4, seed=10 + seed)
        tree = random_branching(12, seed=20 + seed, s_min=6, s_max=40, branch_stages=5)
        pb = Problem(net=net, cost=make_cost(net, seed=10 + seed), tree=tree,
                     data=make_data(net, tree, seed=30 + seed))
    elif base == "single":
        net = make_network(8, 14, 10, 3, seed=5)
        tree = make_tree([1] * 20, seed=6)
        pb = Problem(net=net, cost=make_cost(net, seed=5), tree=tree, data=make_data(net, tree, 7))
    elif base in ("horizon1", "horizon1s"):
        # a one-stage horizon: the root and five leaves, or the root and one
        net = make_network(8, 14, 10, 3, seed=5)
        tree = make_tree([5] if base == "horizon1" else [1], seed=3)
        pb = Problem(net=net, cost=make_cost(net, seed=5), tree=tree, data=make_data(net, tree, 8))
    elif base == "ne0":
        net = make_network(6, 9, 5, 0, seed=8)
        tree = make_tree([3, 2, 1, 2, 1, 1, 1], seed=9)
        pb = Problem(net=net, cost=make_cost(net, seed=8), tree=tree, data=make_data(net, tree, 10))
    elif base == "bushy":
        # branching at every stage: top nodes at all but the last stage, chains of one node
        net = make_network(10, 18, 12, 3, seed=14)
        tree = make_tree([2, 2, 2, 2, 2, 3], seed=15)
        pb = Problem(net=net, cost=make_cost(net, seed=14), tree=tree, data=make_data(net, tree, 16))
    elif base == "dense":
        net = make_network(16, 29, 22, 4, seed=43)
        tree = random_branching(12, seed=44, s_min=6, s_max=40, branch_stages=5)
        pb = Problem(net=net, cost=make_cost(net, seed=43, dense_wu=True), tree=tree,
                     data=make_data(net, tree, seed=45))
    elif base == "wide":
        # nu above the shared form's limit of 256
        net = make_network(160, 300, 200, 40, seed=17)
        tree = make_tree([3, 2, 1, 1, 1, 1], seed=18)
        pb = Problem(net=net, cost=make_cost(net, seed=17), tree=tree, data=make_data(net, tree, 19))
    elif base == "widest":
        # six to eight rows per thread; one team per block (its vectors fill the shared memory)
        net = make_network(400, 720, 500, 100, seed=20)
        tree = make_tree([2, 2, 1, 1], seed=21)
        pb = Problem(net=net, cost=make_cost(net, seed=20), tree=tree, data=make_data(net, tree, 22))
    else:
        raise KeyError(kind)
    if kind.endswith("_A"):
        pb.net.A = general_A(pb.net.nx, 3)
    return pb


_ORACLE = {}


def oracle_for(kind, pb):
    if kind not in _ORACLE:
        P = O.OracleProblem.from_parts(pb.net, pb.cost, pb.tree)
        F = O.factor(P)
        S = O.solve_consts(P, F, pb.data.x0, pb.data.q, pb.data.demand, pb.data.alpha)
        _ORACLE[kind] = (P, F, S)
    return _ORACLE[kind]


def dev(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def dual_gradient(fac, pb, w, data=True):
    import torch
    n = pb.tree.stage_ptr[-1]
    u = torch.empty((n, pb.net.nu), dtype=torch.float64, device="cuda")
    x = torch.empty((n, pb.net.nx), dtype=torch.float64, device="cuda")
    if data:
        d = pb.data
        fac.dual_gradient_device(dev(w), u, x, dev(d.x0), dev(d.q), dev(d.demand), dev(d.alpha))
    else:
        fac.dual_gradient_device(dev(w), u, x)
    torch.cuda.synchronize()
    return u.cpu().numpy(), x.cpu().numpy()


DG_KINDS = ["tiny_A", "barcelona32_A", "uneven0_A", "uneven1_A", "single_A", "ne0_A", "bushy_A",
            "dense_A", "tiny", "wide_A", "widest_A", "horizon1_A", "horizon1s_A"]


@pytest.mark.parametrize("kind", DG_KINDS)
def test_dual_gradient_matches_oracle(kind):
    pb = problem(kind)
    P, F, S = oracle_for(kind, pb)
    rng = np.random.default_rng(1)
    w = rng.standard_normal((P.n_nodes, P.ny)) * 3.0
    w[0] = 0.0
    u_o, x_o = O.dual_gradient(P, F, S, w)
    fac = rn.Factor(pb.net, pb.cost, pb.tree, gamma=1.0, factor_form=PN)
    assert fac.info()["factor_form"] == PN
    u, x = dual_gradient(fac, pb, w)
    assert rel_err(u, u_o) <= 1e-9
    assert rel_err(x, x_o) <= 1e-9
    # a second evaluation on the prepared data
    u_o2, x_o2 = O.dual_gradient(P, F, S, -0.5 * w)
    u, x = dual_gradient(fac, pb, -0.5 * w, data=False)
    assert rel_err(u, u_o2) <= 1e-9
    assert rel_err(x, x_o2) <= 1e-9
    fac.close()


@pytest.mark.parametrize("kind", ["tiny_A", "barcelona32_A", "dense_A", "widest_A"])
def test_fp32_dual_gradient_matches_oracle(kind):
    pb = problem(kind)
    P, F, S = oracle_for(kind, pb)
    rng = np.random.default_rng(2)
    w = rng.standard_normal((P.n_nodes, P.ny)) * 3.0
    w[0] = 0.0
    u_o, x_o = O.dual_gradient(P, F, S, w)
    fac = rn.Factor(pb.net, pb.cost, pb.tree, gamma=1.0, factor_form=PN,
                    precision=rn.RN_PREC_FP32)
    u, x = dual_gradient(fac, pb, w)
    fac.close()
    assert rel_err(u, u_o) <= 2e-4
    assert rel_err(x, x_o) <= 2e-4


@pytest.mark.parametrize("kind", ["tiny_A", "uneven1_A", "barcelona32_A"])
def test_step_size_matches_oracle_power_iteration(kind):
    pb = problem(kind)
    P, F, S = oracle_for(kind, pb)
    L_o = O.power_iteration(P, F, 200)
    fac = rn.Factor(pb.net, pb.cost, pb.tree, factor_form=PN)
    info = fac.info()
    fac.close()
    assert abs(info["L"] - L_o) <= 1e-9 * L_o
    assert abs(info["gamma"] - O.step_size(L_o)) <= 1e-9 * O.step_size(L_o)


@pytest.mark.parametrize("kind,iters", [("tiny_A", 500), ("barcelona32_A", 300),
                                        ("uneven0_A", 400), ("uneven2_A", 300), ("single_A", 400),
                                        ("ne0_A", 400), ("bushy_A", 300), ("dense_A", 300),
                                        ("horizon1_A", 300), ("horizon1s_A", 300)])
def test_apg_matches_oracle(kind, iters):
    pb = problem(kind)
    P, F, S = oracle_for(kind, pb)
    gamma = O.step_size(O.power_iteration(P, F, 100))
    ref = O.apg(P, F, S, iters, gamma)
    fac = rn.Factor(pb.net, pb.cost, pb.tree, gamma=gamma, factor_form=PN)
    out = fac.solve(pb.data.x0, pb.data.q, pb.data.demand, pb.data.alpha, max_iters=iters,
                    res_hist_len=1000)
    fac.close()
    assert out["status"] == B.RN_OK
    assert out["iters"] == iters
    for k in "uxy":
        assert rel_err(out[k], getattr(ref, k)) <= 1e-6, k
    assert abs(out["primal_res"] - ref.residual) <= 1e-6 * max(ref.residual, 1e-12) + 1e-12
    cost = O.primal_cost(P, S, ref.u, ref.x)
    assert abs(out["cost"] - cost) <= 1e-6 * abs(cost)
    assert abs(out["ubox_viol"] - O.ubox_violation(P, ref.u)) <= 1e-6 * np.abs(ref.u).max()
    # one residual per check of every 10 iterations (and the last)
    hist = out["res_hist"]
    assert len(hist) == out["n_checks"] == iters // 10
    np.testing.assert_allclose(hist, ref.res_hist[9::10][:len(hist)], rtol=1e-6, atol=1e-12)


def test_warm_start_simple_rule_and_averaged_primal():
    kind = "uneven1_A"
    pb = problem(kind)
    P, F, S = oracle_for(kind, pb)
    gamma = O.step_size(O.power_iteration(P, F, 100))
    rng = np.random.default_rng(5)
    y0 = rng.standard_normal((P.n_nodes, P.ny)) * 0.1
    y0[0] = 0.0
    ref = O.apg(P, F, S, 250, gamma, y0=y0, theta_rule="simple", average=True)
    fac = rn.Factor(pb.net, pb.cost, pb.tree, gamma=gamma, factor_form=PN,
                    theta_rule=B.RN_THETA_SIMPLE)
    out = fac.solve(pb.data.x0, pb.data.q, pb.data.demand, pb.data.alpha, max_iters=250,
                    y_warm=y0, average=True)
    fac.close()
    for k in "uxy":
        assert rel_err(out[k], getattr(ref, k)) <= 1e-6, k
    assert rel_err(out["u_avg"], ref.u_avg) <= 1e-6
    assert rel_err(out["x_avg"], ref.x_avg) <= 1e-6


def test_stops_at_the_first_check_below_tol():
    kind = "tiny_A"
    pb = problem(kind)
    P, F, S = oracle_for(kind, pb)
    gamma = O.step_size(O.power_iteration(P, F, 100))
    full = O.apg(P, F, S, 3000, gamma)
    checks = full.res_hist[9::10]
    # a tolerance met first at some check with a clear margin on both sides
    tol, at = None, None
    for c in range(5, len(checks)):
        lo = checks[:c].min()
        if checks[c] < lo * 0.99:
            tol, at = checks[c] * 1.001, c
            if c > 20:
                break
    assert tol is not None
    ref = O.apg(P, F, S, 3000, gamma, tol=tol, check_every=10)
    assert ref.converged and ref.iters == 10 * (at + 1)
    fac = rn.Factor(pb.net, pb.cost, pb.tree, gamma=gamma, factor_form=PN)
    out = fac.solve(pb.data.x0, pb.data.q, pb.data.demand, pb.data.alpha, max_iters=3000,
                    tol=tol)
    fac.close()
    assert out["status"] == B.RN_OK
    assert out["iters"] == ref.iters
    for k in "uxy":
        assert rel_err(out[k], getattr(ref, k)) <= 1e-6, k


@pytest.mark.parametrize("name,iters", [("barcelona32", 300)])
def test_per_node_form_equals_shared_form(name, iters):
    """With A = I both forms compute the same iterates (FP64)."""
    pb = make_problem(name)
    shared = rn.Factor(pb.net, pb.cost, pb.tree, factor_form=rn.RN_FACTOR_SHARED)
    gamma = shared.info()["gamma"]
    pn = rn.Factor(pb.net, pb.cost, pb.tree, gamma=gamma, factor_form=PN)
    d = pb.data
    a = shared.solve(d.x0, d.q, d.demand, d.alpha, max_iters=iters)
    b = pn.solve(d.x0, d.q, d.demand, d.alpha, max_iters=iters)
    L_pn = rn.Factor(pb.net, pb.cost, pb.tree, factor_form=PN)
    assert abs(L_pn.info()["L"] - shared.info()["L"]) <= 1e-9 * shared.info()["L"]
    L_pn.close()
    shared.close()
    pn.close()
    for k in "uxy":
        assert rel_err(b[k], a[k]) <= 1e-8, k
    assert abs(a["cost"] - b["cost"]) <= 1e-8 * abs(a["cost"])


def test_full_size_512_scenarios():
    """barcelona512 (10,664 nodes) in the launch configuration the bench
    times: the FP64 per-node dual gradient equals the shared form's, its
    outputs satisfy the dynamics and the coupling exactly up to rounding,
    and the FP32 per-node evaluation stays within the FP32 bar."""
    pb = make_problem("barcelona512")
    n = pb.tree.stage_ptr[-1]
    rng = np.random.default_rng(9)
    w = rng.standard_normal((n, 2 * pb.net.nx + pb.net.nu))
    w[0] = 0.0
    shared = rn.Factor(pb.net, pb.cost, pb.tree, gamma=1.0, factor_form=rn.RN_FACTOR_SHARED)
    u_s, x_s = dual_gradient(shared, pb, w)
    shared.close()
    f64 = rn.Factor(pb.net, pb.cost, pb.tree, gamma=1.0, factor_form=PN)
    u, x = dual_gradient(f64, pb, w)
    f64.close()
    assert rel_err(u, u_s) <= 1e-9 and rel_err(x, x_s) <= 1e-9
    net, d, anc = pb.net, pb.data, np.asarray(pb.tree.anc)
    A = np.asarray(net.A).reshape(net.nx, net.nx)
    Bm = np.asarray(net.B).reshape(net.nx, net.nu)
    Gd = np.asarray(net.Gd).reshape(net.nx, net.nd)
    E = np.asarray(net.E).reshape(net.ne, net.nu)
    Ed = np.asarray(net.Ed).reshape(net.ne, net.nd)
    dyn = x[1:] - (x[anc[1:]] @ A.T + u[1:] @ Bm.T + np.asarray(d.demand)[1:] @ Gd.T)
    cpl = u[1:] @ E.T + np.asarray(d.demand)[1:] @ Ed.T
    assert np.abs(dyn).max() <= 1e-9 * np.abs(x).max()
    assert np.abs(cpl).max() <= 1e-9 * np.abs(u).max()
    f32 = rn.Factor(pb.net, pb.cost, pb.tree, gamma=1.0, factor_form=PN,
                    precision=rn.RN_PREC_FP32)
    u32, x32 = dual_gradient(f32, pb, w)
    f32.close()
    assert rel_err(u32, u) <= 2e-4 and rel_err(x32, x) <= 2e-4


def test_refusals_of_the_per_node_form():
    pb = problem("tiny_A")
    fac = rn.Factor(pb.net, pb.cost, pb.tree, gamma=1.0)  # A != I: per-node by default
    assert fac.info()["factor_form"] == PN
    d = pb.data
    with pytest.raises(B.RapidNetError) as ei:
        fac.solve(d.x0, d.q, d.demand, d.alpha, max_iters=10, compute_gap=True)
    assert ei.value.status == B.RN_ERR_UNSUPPORTED
    fac.solve(d.x0, d.q, d.demand, d.alpha, max_iters=10)
    import torch
    n = pb.tree.stage_ptr[-1]
    w = torch.zeros((n, 2 * pb.net.nx + pb.net.nu), dtype=torch.float64, device="cuda")
    u = torch.empty((n, pb.net.nu), dtype=torch.float64, device="cuda")
    x = torch.empty((n, pb.net.nx), dtype=torch.float64, device="cuda")
    with pytest.raises(B.RapidNetError) as ei:
        fac.dual_gradient_noalloc(w, u, x)
    assert ei.value.status == B.RN_ERR_UNSUPPORTED
    fac.close()


def test_flag_wait_that_runs_out_reports_timeout_and_the_handle_recovers():
    """A top node waits for its children's flags, which other teams set
    only after their whole chain: with a 1 us bound the wait runs out, the
    error word ends the launch at the next residual check, and the call
    returns RN_ERR_TIMEOUT.  Nothing is withheld or faulted; a handle with
    the default bound then solves normally."""
    kind = "barcelona32_A"
    pb = problem(kind)
    P, F, S = oracle_for(kind, pb)
    gamma = O.step_size(O.power_iteration(P, F, 100))
    d = pb.data
    bad = rn.Factor(pb.net, pb.cost, pb.tree, gamma=gamma, factor_form=PN, wait_us=1)
    for _ in range(2):
        with pytest.raises(B.RapidNetError) as ei:
            bad.solve(d.x0, d.q, d.demand, d.alpha, max_iters=50)
        assert ei.value.status == B.RN_ERR_TIMEOUT
        assert "gave up" in str(ei.value)
    bad.close()
    ref = O.apg(P, F, S, 100, gamma)
    good = rn.Factor(pb.net, pb.cost, pb.tree, gamma=gamma, factor_form=PN)
    out = good.solve(d.x0, d.q, d.demand, d.alpha, max_iters=100)
    good.close()
    for k in "uxy":
        assert rel_err(out[k], getattr(ref, k)) <= 1e-6, k


@pytest.mark.parametrize("kind,iters,refresh", [("tiny_A", 500, 20), ("barcelona32_A", 300, 20),
                                                ("uneven1_A", 300, 7), ("dense_A", 300, 20)])
def test_mixed_precision_matches_oracle(kind, iters, refresh):
    """RN_PREC_MIXED on the per-node form: FP32 iterations on the delta from
    an FP64 base refreshed every `refresh` iterations (7: the refreshes fall
    between the residual checks), the final primal in FP64.  Cost, u, y and
    the averaged u against the FP64 oracle at the same iteration count,
    within the larger of 1e-3 and twice the spread of two FP64 per-node
    solves whose step sizes differ by one FP32 ulp: some of these problems
    amplify any perturbation (barcelona32 with this A: 6e-3 in y after 300
    iterations for that one-ulp change, the mixed solve 3e-3; on the others
    the mixed solve lands near 1e-5 and plain FP32 near 1e-4).  The primal
    satisfies the dynamics to FP64 rounding."""
    pb = problem(kind)
    P, F, S = oracle_for(kind, pb)
    gamma = O.step_size(O.power_iteration(P, F, 100))
    ref = O.apg(P, F, S, iters, gamma, average=True)
    fac = rn.Factor(pb.net, pb.cost, pb.tree, gamma=gamma, factor_form=PN,
                    precision=rn.RN_PREC_MIXED, refresh_every=refresh)
    assert fac.info()["factor_form"] == PN
    out = fac.solve(pb.data.x0, pb.data.q, pb.data.demand, pb.data.alpha, max_iters=iters,
                    res_hist_len=1000, average=True)
    fac.close()
    f64 = rn.Factor(pb.net, pb.cost, pb.tree, gamma=gamma * (1.0 + 2.0 ** -23), factor_form=PN)
    e = f64.solve(pb.data.x0, pb.data.q, pb.data.demand, pb.data.alpha, max_iters=iters)
    f64.close()
    assert out["status"] == B.RN_OK and out["iters"] == iters
    assert out["n_checks"] == iters // 10
    cost = O.primal_cost(P, S, ref.u, ref.x)
    bar = {k: max(1e-3, 2 * rel_err(e[k], getattr(ref, k))) for k in "uy"}
    bar["cost"] = max(1e-3, 2 * abs(e["cost"] - cost) / abs(cost))
    for k in "uy":
        assert rel_err(out[k], getattr(ref, k)) <= bar[k], (k, bar)
    assert abs(out["cost"] - cost) <= bar["cost"] * abs(cost)
    net, d, anc = pb.net, pb.data, np.asarray(pb.tree.anc)
    A = np.asarray(net.A).reshape(net.nx, net.nx)
    Bm = np.asarray(net.B).reshape(net.nx, net.nu)
    Gd = np.asarray(net.Gd).reshape(net.nx, net.nd)
    x, u = out["x"], out["u"]
    dyn = x[1:] - (x[anc[1:]] @ A.T + u[1:] @ Bm.T + np.asarray(d.demand)[1:] @ Gd.T)
    assert np.abs(dyn).max() <= 1e-9 * np.abs(x).max()
    assert rel_err(out["u_avg"], ref.u_avg) <= bar["u"]


def test_mixed_precision_full_size_against_fp64():
    """barcelona512 (A = I): the per-node mixed solve after 200 iterations
    against the per-node FP64 solve.  As for the shared form, the bar is the
    larger of 1e-3 and twenty times the spread between two FP64 solves whose
    step sizes differ by one FP32 ulp (far from convergence the accelerated
    iteration amplifies any perturbation), for the cost, u and y."""
    pb = make_problem("barcelona512")
    d = pb.data
    runs = []
    for prec, scale in ((rn.RN_PREC_FP64, 1.0), (rn.RN_PREC_FP64, 1.0 + 2.0 ** -23),
                        (rn.RN_PREC_MIXED, 1.0)):
        if not runs:
            f = rn.Factor(pb.net, pb.cost, pb.tree, factor_form=PN)
            gamma = f.info()["gamma"]
        else:
            f = rn.Factor(pb.net, pb.cost, pb.tree, gamma=gamma * scale, factor_form=PN,
                          precision=prec)
        runs.append(f.solve(d.x0, d.q, d.demand, d.alpha, max_iters=200))
        f.close()
    a, e, b = runs
    assert b["status"] == B.RN_OK and b["iters"] == 200
    spread = {k: rel_err(e[k], a[k]) for k in "uy"}
    spread["cost"] = abs(e["cost"] - a["cost"]) / abs(a["cost"])
    for k in "uy":
        assert rel_err(b[k], a[k]) <= max(1e-3, 20 * spread[k]), (k, spread)
    assert abs(b["cost"] - a["cost"]) <= max(1e-3, 20 * spread["cost"]) * abs(a["cost"])


def test_mixed_precision_tolerance_stop():
    """RN_PREC_MIXED on the per-node form stops at a residual check inside a
    launch of refresh_every iterations (tol 1e-3 on tiny with A != I; the
    oracle stops at 720 iterations): the returned residual is at or below
    the tolerance, the primal is the FP64 evaluation at that iteration (the
    dynamics hold to FP64 rounding), and the iteration count is within 50
    of the oracle's (the FP32 iterates reach the tolerance at a neighbouring
    check)."""
    kind = "tiny_A"
    pb = problem(kind)
    P, F, S = oracle_for(kind, pb)
    gamma = O.step_size(O.power_iteration(P, F, 100))
    ref = O.apg(P, F, S, 20000, gamma, tol=1e-3, check_every=10)
    assert ref.converged
    fac = rn.Factor(pb.net, pb.cost, pb.tree, gamma=gamma, factor_form=PN,
                    precision=rn.RN_PREC_MIXED)
    out = fac.solve(pb.data.x0, pb.data.q, pb.data.demand, pb.data.alpha, max_iters=20000,
                    tol=1e-3)
    fac.close()
    assert out["status"] == B.RN_OK and out["primal_res"] <= 1e-3
    assert out["iters"] % 10 == 0 and out["iters"] < 20000
    assert abs(out["iters"] - ref.iters) <= 50, (out["iters"], ref.iters)
    net, d, anc = pb.net, pb.data, np.asarray(pb.tree.anc)
    A = np.asarray(net.A).reshape(net.nx, net.nx)
    Bm = np.asarray(net.B).reshape(net.nx, net.nu)
    Gd = np.asarray(net.Gd).reshape(net.nx, net.nd)
    x, u = out["x"], out["u"]
    dyn = x[1:] - (x[anc[1:]] @ A.T + u[1:] @ Bm.T + np.asarray(d.demand)[1:] @ Gd.T)
    assert np.abs(dyn).max() <= 1e-9 * np.abs(x).max()


def test_mixed_precision_warm_start_simple_rule():
    """RN_PREC_MIXED on the per-node form from a warm start (the base starts
    at y_warm: an APG iterate, as in a receding-horizon solve) with the
    second theta rule and the averaged primal, against the oracle at the
    mixed bar (1e-3; measured near 3e-6).  A random dual point of the size
    of y as the start puts FP32 iterations of either form near 5e-3 after
    250 iterations (FP64 1e-9), so the start is an iterate."""
    kind = "uneven1_A"
    pb = problem(kind)
    P, F, S = oracle_for(kind, pb)
    gamma = O.step_size(O.power_iteration(P, F, 100))
    y0 = O.apg(P, F, S, 60, gamma, theta_rule="simple").y
    ref = O.apg(P, F, S, 250, gamma, y0=y0, theta_rule="simple", average=True)
    fac = rn.Factor(pb.net, pb.cost, pb.tree, gamma=gamma, factor_form=PN,
                    precision=rn.RN_PREC_MIXED, theta_rule=B.RN_THETA_SIMPLE)
    out = fac.solve(pb.data.x0, pb.data.q, pb.data.demand, pb.data.alpha, max_iters=250,
                    y_warm=y0, average=True)
    fac.close()
    assert out["status"] == B.RN_OK and out["iters"] == 250
    for k in "uxy":
        assert rel_err(out[k], getattr(ref, k)) <= 1e-3, k
    assert rel_err(out["u_avg"], ref.u_avg) <= 1e-3
    assert rel_err(out["x_avg"], ref.x_avg) <= 1e-3


@pytest.mark.parametrize("precision", [rn.RN_PREC_MIXED, rn.RN_PREC_FP64])
def test_auto_form_falls_back_to_per_node(precision):
    """A network the shared form cannot lay out (A = I, nu = 540 above its
    256): in FP64, RN_FACTOR_AUTO takes the per-node form; in the mixed
    precision it keeps the shared form's refusal (RN_ERR_UNSUPPORTED: the
    problem is outside solve_batch) and the per-node form is asked for by
    name.  The solve matches the oracle (FP64 1e-6; mixed 1e-3)."""
    net = make_network(300, 540, 420, 81, seed=3)
    tree = make_tree([2, 2] + [1] * 4, seed=2)
    pb = Problem(net=net, cost=make_cost(net, seed=3), tree=tree,
                 data=make_data(net, tree, seed=4))
    P, F, S = oracle_for("wide540", pb)
    gamma = O.step_size(O.power_iteration(P, F, 100))
    ref = O.apg(P, F, S, 300, gamma)
    if precision == rn.RN_PREC_MIXED:
        with pytest.raises(B.RapidNetError) as ei:
            rn.Factor(pb.net, pb.cost, pb.tree, gamma=gamma, precision=precision)
        assert ei.value.status == B.RN_ERR_UNSUPPORTED
        fac = rn.Factor(pb.net, pb.cost, pb.tree, gamma=gamma, precision=precision,
                        factor_form=PN)
    else:
        fac = rn.Factor(pb.net, pb.cost, pb.tree, gamma=gamma, precision=precision)
    assert fac.info()["factor_form"] == PN
    out = fac.solve(pb.data.x0, pb.data.q, pb.data.demand, pb.data.alpha, max_iters=300)
    fac.close()
    bar = 1e-6 if precision == rn.RN_PREC_FP64 else 1e-3
    assert out["status"] == B.RN_OK and out["iters"] == 300
    for k in "uy":
        assert rel_err(out[k], getattr(ref, k)) <= bar, k
    cost = O.primal_cost(P, S, ref.u, ref.x)
    assert abs(out["cost"] - cost) <= bar * abs(cost)


def test_largest_dimensions():
    """nx = nu = 1024, the largest the per-node form validates: in FP32 one
    team per block with eight rows per thread, the dual gradient against the
    oracle at the FP32 bar (2e-4); in FP64, and so for the FP64 set of the
    mixed precision, one team's vectors exceed a block's shared memory (the
    square limit is nx = nu = 800) and factor creation refuses the handle
    with RN_ERR_UNSUPPORTED before the factor step."""
    net = make_network(1024, 1024, 700, 120, seed=23)
    tree = make_tree([2, 1, 1], seed=24)
    pb = Problem(net=net, cost=make_cost(net, seed=23), tree=tree, data=make_data(net, tree, 25))
    P, F, S = oracle_for("largest", pb)
    rng = np.random.default_rng(1)
    w = rng.standard_normal((P.n_nodes, P.ny))
    w[0] = 0.0
    u_o, x_o = O.dual_gradient(P, F, S, w)
    fac = rn.Factor(pb.net, pb.cost, pb.tree, gamma=1.0, factor_form=PN,
                    precision=rn.RN_PREC_FP32)
    assert fac.info()["block_threads"] == 128
    u, x = dual_gradient(fac, pb, w)
    fac.close()
    assert rel_err(u, u_o) <= 2e-4 and rel_err(x, x_o) <= 2e-4
    for prec in (rn.RN_PREC_FP64, rn.RN_PREC_MIXED):
        with pytest.raises(B.RapidNetError) as ei:
            rn.Factor(pb.net, pb.cost, pb.tree, gamma=1.0, factor_form=PN, precision=prec)
        assert ei.value.status == B.RN_ERR_UNSUPPORTED
        assert "shared memory" in rn.rapidnet_last_error()
