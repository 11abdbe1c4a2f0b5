"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

FP64 tolerance: max |gpu - oracle| <= 1e-6 max |oracle| for every output
(u, x, y, dual gradient), at a fixed iteration count; the two sides sum
in different orders, nothing else differs.  Inputs are the seeded
synthetic workloads; the step size is the oracle's own estimate (passed
to both sides) unless the test is about the step size itself.
"""
import numpy as np
import pytest

import oracle as O
import paper_1904_10548_gb300 as rn
from paper_1904_10548_gb300 import _binding as B
from synthetic import make_cost, make_data, make_network, make_problem, make_tree, random_branching
from synthetic.configs import Problem

pytestmark = pytest.mark.gpu

RTOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    assert torch.cuda.is_available()


def rel_err(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300))


def problem(kind):
    if kind in ("tiny", "barcelona32", "barcelona512"):
        return make_problem(kind)
    if kind == "tight":
        pb = make_problem("tiny", Ws=20.0)
        pb.net.xs = 0.75 * pb.net.xmax
        return pb
    if kind.startswith("uneven"):
        seed = int(kind[6:] or 0)
        net = make_network(16, 29, 22, 4, seed=10 + seed)
        tree = random_branching(12, seed=20 + seed, s_min=6, s_max=40, branch_stages=5)
        return Problem(net=net, cost=make_cost(net, seed=10 + seed), tree=tree,
                       data=make_data(net, tree, seed=30 + seed))
    if kind == "single":
        net = make_network(8, 14, 10, 3, seed=5)
        tree = make_tree([1] * 20, seed=6)
        return Problem(net=net, cost=make_cost(net, seed=5), tree=tree, data=make_data(net, tree, 7))
    if kind in ("horizon1", "horizon1s"):
        # a one-stage horizon: the root and five leaves, or the root and one
        net = make_network(8, 14, 10, 3, seed=5)
        tree = make_tree([5] if kind == "horizon1" else [1], seed=3)
        return Problem(net=net, cost=make_cost(net, seed=5), tree=tree, data=make_data(net, tree, 8))
    if kind == "ne0":
        net = make_network(6, 9, 5, 0, seed=8)
        tree = make_tree([3, 2, 1, 2, 1, 1, 1], seed=9)
        return Problem(net=net, cost=make_cost(net, seed=8), tree=tree, data=make_data(net, tree, 10))
    if kind.startswith("dense_"):
        # a dense symmetric positive definite W_u: the shared operator F is
        # applied as a dense product (tensor cores in the FP32 steps)
        base = kind[6:]
        if base in ("tiny", "barcelona32"):
            pb = make_problem(base)
            pb.cost.Wu = make_cost(pb.net, seed=41, dense_wu=True).Wu
            return pb
        net = make_network(16, 29, 22, 4, seed=43)
        tree = random_branching(12, seed=44, s_min=6, s_max=40, branch_stages=5)
        return Problem(net=net, cost=make_cost(net, seed=43, dense_wu=True), tree=tree,
                       data=make_data(net, tree, seed=45))
    if kind == "stage1_chains":
        # stage-1 nodes with one leaf next to stage-1 nodes that branch later
        net = make_network(10, 18, 12, 3, seed=11)
        counts = [[4], [1, 2, 1, 3], [1, 1, 2, 1, 1, 1, 1], [1] * 8, [1] * 8, [1] * 8]
        tree = O_build(counts, 12)
        return Problem(net=net, cost=make_cost(net, seed=11), tree=tree, data=make_data(net, tree, 13))
    raise KeyError(kind)


def O_build(counts, seed):
    from synthetic.tree import _build
    return _build(counts, seed)


_ORACLE = {}


def oracle_for(kind, pb):
    if kind not in _ORACLE:
        P = O.OracleProblem.from_parts(pb.net, pb.cost, pb.tree)
        F = O.factor(P)
        S = O.solve_consts(P, F, pb.data.x0, pb.data.q, pb.data.demand, pb.data.alpha)
        _ORACLE[kind] = (P, F, S)
    return _ORACLE[kind]


def gpu_factor(pb, gamma=0.0, **kw):
    return rn.Factor(pb.net, pb.cost, pb.tree, gamma=gamma, **kw)


KINDS = ["tiny", "barcelona32", "uneven0", "uneven1", "uneven2", "single", "ne0",
         "stage1_chains", "tight", "horizon1", "horizon1s"]


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kind", KINDS)
def test_dual_gradient_matches_oracle(kind):
    import torch
    pb = problem(kind)
    P, F, S = oracle_for(kind, pb)
    rng = np.random.default_rng(1)
    w = rng.standard_normal((P.n_nodes, P.ny)) * 3.0
    w[0] = 0.0
    u_o, x_o = O.dual_gradient(P, F, S, w)
    fac = gpu_factor(pb, gamma=1.0)
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    u = torch.empty((P.n_nodes, P.nu), dtype=torch.float64, device="cuda")
    x = torch.empty((P.n_nodes, P.nx), dtype=torch.float64, device="cuda")
    fac.dual_gradient_device(dev(w), u, x, dev(pb.data.x0), dev(pb.data.q), dev(pb.data.demand),
                             dev(pb.data.alpha))
    torch.cuda.synchronize()
    assert rel_err(u.cpu().numpy(), u_o) <= 1e-9
    assert rel_err(x.cpu().numpy(), x_o) <= 1e-9
    # a second evaluation reuses the prepared data
    w2 = -0.5 * w
    u_o2, x_o2 = O.dual_gradient(P, F, S, w2)
    fac.dual_gradient_device(dev(w2), u, x)
    torch.cuda.synchronize()
    assert rel_err(u.cpu().numpy(), u_o2) <= 1e-9
    assert rel_err(x.cpu().numpy(), x_o2) <= 1e-9
    fac.close()


@pytest.mark.parametrize("kind", ["tiny", "barcelona32", "uneven1"])
def test_step_size_matches_oracle_power_iteration(kind):
    pb = problem(kind)
    P, F, S = oracle_for(kind, pb)
    L_o = O.power_iteration(P, F, 200)
    fac = gpu_factor(pb)
    info = fac.info()
    fac.close()
    assert abs(info["L"] - L_o) <= 1e-9 * L_o
    assert abs(info["gamma"] - O.step_size(L_o)) <= 1e-9 * O.step_size(L_o)


@pytest.mark.parametrize("kind,iters", [("tiny", 500), ("barcelona32", 300), ("uneven0", 400),
                                        ("uneven1", 400), ("uneven2", 300), ("single", 400),
                                        ("ne0", 400), ("stage1_chains", 400), ("tight", 500),
                                        ("horizon1", 300), ("horizon1s", 300)])
def test_apg_matches_oracle(kind, iters):
    pb = problem(kind)
    P, F, S = oracle_for(kind, pb)
    gamma = O.step_size(O.power_iteration(P, F, 100))
    ref = O.apg(P, F, S, iters, gamma)
    fac = gpu_factor(pb, gamma=gamma)
    out = fac.solve(pb.data.x0, pb.data.q, pb.data.demand, pb.data.alpha, max_iters=iters,
                    compute_gap=True, res_hist_len=1000)
    fac.close()
    assert out["status"] == B.RN_OK
    assert out["iters"] == iters
    assert rel_err(out["u"], ref.u) <= RTOL
    assert rel_err(out["x"], ref.x) <= RTOL
    assert rel_err(out["y"], ref.y) <= RTOL
    assert abs(out["primal_res"] - ref.residual) <= RTOL * max(ref.residual, 1e-12) + 1e-12
    # reported scalars
    cost = O.primal_cost(P, S, ref.u, ref.x)
    assert abs(out["cost"] - cost) <= RTOL * abs(cost)
    assert abs(out["ubox_viol"] - O.ubox_violation(P, ref.u)) <= RTOL * np.abs(ref.u).max()
    uy, xy = O.dual_gradient(P, F, S, ref.y)
    gap = O.primal_cost(P, S, uy, xy) - O.dual_value(P, F, S, ref.y)
    assert abs(out["gap"] - gap) <= 1e-6 * max(abs(cost), 1.0)


@pytest.mark.parametrize("kind,precision", [("uneven1", rn.RN_PREC_FP64),
                                             ("barcelona32", rn.RN_PREC_FP64),
                                             ("uneven1", rn.RN_PREC_MIXED)])
def test_simple_theta_rule_matches_oracle(kind, precision):
    """The second extrapolation sequence of §4.3, theta_nu = 2 / (nu + 2),
    against the oracle's APG with the same rule (FP64: 1e-6; mixed: the
    mixed-precision bar of 1e-3)."""
    pb = problem(kind)
    P, F, S = oracle_for(kind, pb)
    gamma = O.step_size(O.power_iteration(P, F, 100))
    iters = 300
    ref = O.apg(P, F, S, iters, gamma, theta_rule="simple")
    fac = gpu_factor(pb, gamma=gamma, precision=precision, theta_rule=B.RN_THETA_SIMPLE)
    out = fac.solve(pb.data.x0, pb.data.q, pb.data.demand, pb.data.alpha, max_iters=iters)
    fac.close()
    tol = RTOL if precision == rn.RN_PREC_FP64 else 1e-3
    assert out["status"] == B.RN_OK and out["iters"] == iters
    for k in "uxy":
        assert rel_err(out[k], getattr(ref, k)) <= tol, k
    # the rule matters: the equality rule's iterate is elsewhere
    other = O.apg(P, F, S, iters, gamma)
    assert rel_err(other.y, ref.y) > 100 * RTOL


@pytest.mark.parametrize("kind,precision,rule", [("tiny", rn.RN_PREC_FP64, "equality"),
                                                  ("barcelona32", rn.RN_PREC_FP64, "simple"),
                                                  ("uneven2", rn.RN_PREC_FP64, "equality"),
                                                  ("uneven1", rn.RN_PREC_MIXED, "simple"),
                                                  ("tight", rn.RN_PREC_MIXED, "equality")])
def test_averaged_primal_matches_oracle(kind, precision, rule):
    """The averaged primal iterate of §4.3, xbar^nu = (1 - theta_nu)
    xbar^{nu-1} + theta_nu x*(w^nu), against the oracle's (FP64: 1e-6;
    mixed: 1e-3).  Being an average of primal points that satisfy the
    dynamics and couplings, it satisfies them too."""
    pb = problem(kind)
    P, F, S = oracle_for(kind, pb)
    gamma = O.step_size(O.power_iteration(P, F, 100))
    iters = 250
    ref = O.apg(P, F, S, iters, gamma, theta_rule=rule, average=True)
    fac = gpu_factor(pb, gamma=gamma, precision=precision,
                     theta_rule=B.RN_THETA_SIMPLE if rule == "simple" else B.RN_THETA_EQUALITY)
    out = fac.solve(pb.data.x0, pb.data.q, pb.data.demand, pb.data.alpha, max_iters=iters,
                    average=True)
    plain = fac.solve(pb.data.x0, pb.data.q, pb.data.demand, pb.data.alpha, max_iters=iters)
    fac.close()
    tol = RTOL if precision == rn.RN_PREC_FP64 else 1e-3
    assert rel_err(out["u_avg"], ref.u_avg) <= tol
    assert rel_err(out["x_avg"], ref.x_avg) <= tol
    # averaging changes nothing else
    for k in "uxy":
        assert np.array_equal(out[k], plain[k]), k
    net, tree, d = pb.net, pb.tree, pb.data
    u, x = out["u_avg"], out["x_avg"]
    a = tree.anc[1:]
    dyn = x[1:] - x[a] - u[1:] @ net.B.T - d.demand[1:] @ net.Gd.T
    assert np.abs(dyn).max() <= (1e-9 if precision == rn.RN_PREC_FP64 else 1e-5) * np.abs(x).max()
    if net.ne:
        cpl = u[1:] @ net.E.T + d.demand[1:] @ net.Ed.T
        assert np.abs(cpl).max() <= (1e-9 if precision == rn.RN_PREC_FP64 else 1e-5) * np.abs(u).max()


@pytest.mark.parametrize("kind", ["tiny", "barcelona32", "tight"])
def test_first_ten_iterates_match_oracle(kind):
    """Iterate by iterate: the GPU solve stopped after k = 1 .. 10
    iterations against the oracle's k-th APG iterate (eqs. apg:1 / apg:2),
    all ten on the scale of the whole trajectory."""
    pb = problem(kind)
    P, F, S = oracle_for(kind, pb)
    gamma = O.step_size(O.power_iteration(P, F, 100))
    fac = gpu_factor(pb, gamma=gamma)
    got, ref = {k: [] for k in "uxy"}, {k: [] for k in "uxy"}
    for it in range(1, 11):
        out = fac.solve(pb.data.x0, pb.data.q, pb.data.demand, pb.data.alpha, max_iters=it)
        r = O.apg(P, F, S, it, gamma)
        assert out["iters"] == it
        for k in "uxy":
            got[k].append(out[k])
            ref[k].append(getattr(r, k))
    fac.close()
    for k in "uxy":
        assert rel_err(np.stack(got[k]), np.stack(ref[k])) <= RTOL, k


def test_tolerance_stop_and_residual_history():
    pb = problem("tiny")
    P, F, S = oracle_for("tiny", pb)
    gamma = O.step_size(O.power_iteration(P, F, 100))
    tol = 1e-3
    ref = O.apg(P, F, S, 5000, gamma, tol=tol, check_every=10)
    assert ref.converged
    fac = gpu_factor(pb, gamma=gamma, check_every=10)
    out = fac.solve(pb.data.x0, pb.data.q, pb.data.demand, pb.data.alpha, max_iters=5000,
                    tol=tol, res_hist_len=1000)
    assert out["status"] == B.RN_OK
    assert out["iters"] == ref.iters and out["iters"] % 10 == 0
    assert out["primal_res"] <= tol
    hist_o = ref.res_hist[9::10]
    assert np.allclose(out["res_hist"], hist_o, rtol=1e-6, atol=1e-12)
    # not reaching the tolerance: RN_NOT_CONVERGED with valid outputs
    out2 = fac.solve(pb.data.x0, pb.data.q, pb.data.demand, pb.data.alpha, max_iters=25, tol=1e-12)
    assert out2["status"] == B.RN_NOT_CONVERGED and out2["iters"] == 25
    ref2 = O.apg(P, F, S, 25, gamma)
    assert rel_err(out2["y"], ref2.y) <= RTOL
    fac.close()


def test_warm_start_matches_oracle():
    pb = problem("barcelona32")
    P, F, S = oracle_for("barcelona32", pb)
    gamma = O.step_size(O.power_iteration(P, F, 50))
    first = O.apg(P, F, S, 60, gamma)
    ref = O.apg(P, F, S, 80, gamma, y0=first.y, y_prev0=first.y)
    fac = gpu_factor(pb, gamma=gamma)
    out = fac.solve(pb.data.x0, pb.data.q, pb.data.demand, pb.data.alpha, max_iters=80,
                    y_warm=first.y)
    fac.close()
    assert rel_err(out["y"], ref.y) <= RTOL
    assert rel_err(out["u"], ref.u) <= RTOL


def test_device_entry_point_equals_host_entry_point():
    import torch
    pb = problem("uneven1")
    fac = gpu_factor(pb, gamma=0.0)
    host = fac.solve(pb.data.x0, pb.data.q, pb.data.demand, pb.data.alpha, max_iters=120)
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    n = pb.tree.n_nodes
    u = torch.empty((n, pb.net.nu), dtype=torch.float64, device="cuda")
    x = torch.empty((n, pb.net.nx), dtype=torch.float64, device="cuda")
    y = torch.empty((n, 2 * pb.net.nx + pb.net.nu), dtype=torch.float64, device="cuda")
    d = fac.solve_device(dev(pb.data.x0), dev(pb.data.q), dev(pb.data.demand), dev(pb.data.alpha),
                         120, 0.0, u, x, y)
    torch.cuda.synchronize()
    fac.close()
    assert d["iters"] == host["iters"]
    assert np.array_equal(u.cpu().numpy(), host["u"])
    assert np.array_equal(x.cpu().numpy(), host["x"])
    assert np.array_equal(y.cpu().numpy(), host["y"])


def test_repeat_solves_are_bitwise_reproducible():
    pb = problem("barcelona32")
    fac = gpu_factor(pb)
    a = fac.solve(pb.data.x0, pb.data.q, pb.data.demand, pb.data.alpha, max_iters=50)
    b = fac.solve(pb.data.x0, pb.data.q, pb.data.demand, pb.data.alpha, max_iters=50)
    fac.close()
    for k in ("u", "x", "y"):
        assert np.array_equal(a[k], b[k])


@pytest.mark.parametrize("kind", ["tiny", "barcelona32", "ne0"])
def test_factor_check_of_the_shared_operator(kind):
    """The factor step's check of the general per-node recursion (§4.4)
    against the shared F: rounding-level on well-conditioned networks."""
    fac = gpu_factor(problem(kind), gamma=1.0)
    dev = fac.info()["collapse_dev"]
    fac.close()
    assert 0.0 <= dev < 1e-12


def test_rank_deficient_coupling_is_rejected():
    pb = problem("tiny")
    pb.net.E = np.vstack([pb.net.E[:1], pb.net.E[:1]])
    with pytest.raises(B.RapidNetError) as ei:
        gpu_factor(pb, gamma=1.0)
    assert ei.value.status == B.RN_ERR_RANK


def test_invalid_solve_arguments():
    pb = problem("tiny")
    fac = gpu_factor(pb, gamma=1.0)
    with pytest.raises(B.RapidNetError) as ei:
        fac.solve(pb.data.x0, pb.data.q, pb.data.demand, pb.data.alpha, max_iters=0)
    assert ei.value.status == B.RN_ERR_INVAL
    fac.close()


# ---------------------------------------------------------------------------
# full size: 512-scenario Barcelona-sized tree, in the launch configuration
# of the benchmark
# ---------------------------------------------------------------------------
@pytest.mark.slow
def test_full_size_iterates_match_oracle():
    pb = problem("barcelona512")
    P, F, S = oracle_for("barcelona512", pb)
    gamma = O.step_size(O.power_iteration(P, F, 5))
    ref = O.apg(P, F, S, 3, gamma)
    fac = gpu_factor(pb, gamma=gamma)
    out = fac.solve(pb.data.x0, pb.data.q, pb.data.demand, pb.data.alpha, max_iters=3)
    info = fac.info()
    fac.close()
    assert info["n_chains"] == 512 and info["n_nodes"] == 10665
    assert rel_err(out["u"], ref.u) <= RTOL
    assert rel_err(out["x"], ref.x) <= RTOL
    assert rel_err(out["y"], ref.y) <= RTOL


@pytest.mark.slow
def test_full_size_properties_after_many_iterations():
    """At any size the outputs satisfy the dynamics and the couplings, the
    duals lie in dom g*, and the gap is consistent with weak duality."""
    pb = problem("barcelona512")
    fac = gpu_factor(pb)
    out = fac.solve(pb.data.x0, pb.data.q, pb.data.demand, pb.data.alpha, max_iters=2000,
                    compute_gap=True)
    fac.close()
    net, tree, d = pb.net, pb.tree, pb.data
    u, x, y = out["u"], out["x"], out["y"]
    a = tree.anc[1:]
    dyn = x[1:] - x[a] - u[1:] @ net.B.T - d.demand[1:] @ net.Gd.T
    cpl = u[1:] @ net.E.T + d.demand[1:] @ net.Ed.T
    assert np.abs(dyn).max() <= 1e-9 * np.abs(x).max()
    assert np.abs(cpl).max() <= 1e-9 * np.abs(u).max()
    nx = net.nx
    assert np.all(np.linalg.norm(y[1:, :nx], axis=1) <= pb.cost.Wx * (1 + 1e-9))
    assert np.all(y[1:, nx:2 * nx] <= 0.0)
    assert np.all(np.linalg.norm(y[1:, nx:2 * nx], axis=1) <= pb.cost.Ws * (1 + 1e-9))
    assert np.isfinite(out["gap"]) and np.isfinite(out["cost"])
    assert np.array_equal(u[0], d.q) and np.array_equal(x[0], d.x0)


# ---------------------------------------------------------------------------
# dense W_u: F as a dense product (FP64 FMAs; TF32 tensor cores with a
# head/tail split in the FP32 steps of the mixed path)
# ---------------------------------------------------------------------------
DENSE = ["dense_tiny", "dense_uneven", "dense_barcelona32"]


@pytest.mark.parametrize("kind", DENSE)
def test_dense_wu_dual_gradient_matches_oracle(kind):
    import torch
    pb = problem(kind)
    assert np.count_nonzero(pb.cost.Wu - np.diag(np.diag(pb.cost.Wu))) > 0
    P, F, S = oracle_for(kind, pb)
    rng = np.random.default_rng(2)
    w = rng.standard_normal((P.n_nodes, P.ny)) * 3.0
    w[0] = 0.0
    u_o, x_o = O.dual_gradient(P, F, S, w)
    fac = gpu_factor(pb, gamma=1.0)
    assert 0.0 <= fac.info()["collapse_dev"] < 1e-12
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    u = torch.empty((P.n_nodes, P.nu), dtype=torch.float64, device="cuda")
    x = torch.empty((P.n_nodes, P.nx), dtype=torch.float64, device="cuda")
    fac.dual_gradient_device(dev(w), u, x, dev(pb.data.x0), dev(pb.data.q), dev(pb.data.demand),
                             dev(pb.data.alpha))
    torch.cuda.synchronize()
    fac.close()
    assert rel_err(u.cpu().numpy(), u_o) <= 1e-9
    assert rel_err(x.cpu().numpy(), x_o) <= 1e-9


@pytest.mark.parametrize("kind,iters", [("dense_tiny", 400), ("dense_uneven", 300),
                                        ("dense_barcelona32", 200)])
def test_dense_wu_apg_matches_oracle(kind, iters):
    pb = problem(kind)
    P, F, S = oracle_for(kind, pb)
    L_o = O.power_iteration(P, F, 100)
    gamma = O.step_size(L_o)
    ref = O.apg(P, F, S, iters, gamma)
    cost = O.primal_cost(P, S, ref.u, ref.x)
    fac = gpu_factor(pb, gamma=gamma)
    out = fac.solve(pb.data.x0, pb.data.q, pb.data.demand, pb.data.alpha, max_iters=iters)
    fac.close()
    for k in "uxy":
        assert rel_err(out[k], getattr(ref, k)) <= RTOL, k
    assert abs(out["cost"] - cost) <= RTOL * abs(cost)
    # step size by the library's own power iteration
    auto = gpu_factor(pb, power_iters=100)
    assert abs(auto.info()["L"] - L_o) <= 1e-9 * L_o
    auto.close()


@pytest.mark.parametrize("kind,iters", [("dense_tiny", 400), ("dense_uneven", 300),
                                        ("dense_barcelona32", 200)])
def test_dense_wu_mixed_matches_oracle(kind, iters):
    """The FP32 steps apply F on the tensor cores (TF32 head/tail split):
    the mixed-precision bar of 1e-3 against the FP64 oracle."""
    pb = problem(kind)
    P, F, S = oracle_for(kind, pb)
    gamma = O.step_size(O.power_iteration(P, F, 100))
    ref = O.apg(P, F, S, iters, gamma)
    cost = O.primal_cost(P, S, ref.u, ref.x)
    fac = gpu_factor(pb, gamma=gamma, precision=rn.RN_PREC_MIXED)
    out = fac.solve(pb.data.x0, pb.data.q, pb.data.demand, pb.data.alpha, max_iters=iters)
    fac.close()
    msg = (f"{kind}: cost {abs(out['cost'] - cost) / abs(cost):.2e} u {rel_err(out['u'], ref.u):.2e}"
           f" y {rel_err(out['y'], ref.y):.2e}")
    assert abs(out["cost"] - cost) <= 1e-3 * abs(cost), msg
    assert rel_err(out["u"], ref.u) <= 1e-3, msg
    assert rel_err(out["y"], ref.y) <= 1e-3, msg
