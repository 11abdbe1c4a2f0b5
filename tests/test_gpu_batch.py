"""Batched mode (one persistent launch over many problems) against solo
solves and against the FP64 oracle.

Each problem of a batch must give the same result as its solo
mixed-precision solve (same kernels, same arithmetic order per problem:
the batch shares only the launch, barriers and the stop decision
schedule) and meet the mixed-precision bar against the FP64 oracle.
Problems have different networks (nx 6, 16, 63) and uneven trees.
"""
import numpy as np
import pytest

import oracle as O
import paper_1904_10548_gb300 as rn
from paper_1904_10548_gb300 import _binding as B
from synthetic import make_cost, make_data, make_network, make_tree, random_branching
from synthetic.configs import Problem
from tests.test_gpu_parity import rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()


def batch_problem(i):
    dims = [(6, 11, 8, 2), (16, 29, 22, 4), (63, 114, 88, 17)][i % 3]
    net = make_network(*dims, seed=100 + i)
    tree = random_branching(10 if dims[0] > 16 else 12, seed=200 + i, s_min=4, s_max=24,
                            branch_stages=4)
    return Problem(net=net, cost=make_cost(net, seed=100 + i), tree=tree,
                   data=make_data(net, tree, seed=300 + i))


def dev(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def tensors(pb):
    return (dev(pb.data.x0), dev(pb.data.q), dev(pb.data.demand), dev(pb.data.alpha))


def work_items(pb, gamma):
    """Work items of a problem's own kernels: the grid of a handle without a cap."""
    f = rn.Factor(pb.net, pb.cost, pb.tree, gamma=gamma, precision=rn.RN_PREC_MIXED)
    n = f.info()["grid_ctas"]
    f.close()
    return n


@pytest.mark.parametrize("capped", [False, True])
def test_batch_equals_solo_and_oracle(capped):
    """capped: the batch's grid is capped at the largest problem's work-item
    count, far below the batch's total, so that blocks take several items
    of several problems."""
    pbs = [batch_problem(i) for i in range(9)]
    gammas = []
    for pb in pbs:
        P = O.OracleProblem.from_parts(pb.net, pb.cost, pb.tree)
        gammas.append(O.step_size(O.power_iteration(P, O.factor(P), 60)))
    items = [work_items(pb, g) for pb, g in zip(pbs, gammas)]
    max_ctas = max(items) if capped else 0
    assert not capped or max_ctas < sum(items)
    facs = [rn.Factor(pb.net, pb.cost, pb.tree, gamma=g, precision=rn.RN_PREC_MIXED,
                      max_ctas=max_ctas) for pb, g in zip(pbs, gammas)]
    iters = 150
    outs = rn.solve_batch(facs, [tensors(pb) for pb in pbs], iters)
    for i, (pb, f, o) in enumerate(zip(pbs, facs, outs)):
        assert o["status"] == B.RN_OK and o["iters"] == iters
        solo = f.solve(pb.data.x0, pb.data.q, pb.data.demand, pb.data.alpha, max_iters=iters)
        for k in ("u", "x", "y"):
            assert np.array_equal(o[k].cpu().numpy(), solo[k]), (i, k)
        assert o["cost"] == solo["cost"]
        P = O.OracleProblem.from_parts(pb.net, pb.cost, pb.tree)
        F = O.factor(P)
        S = O.solve_consts(P, F, pb.data.x0, pb.data.q, pb.data.demand, pb.data.alpha)
        ref = O.apg(P, F, S, iters, gammas[i])
        cost = O.primal_cost(P, S, ref.u, ref.x)
        assert abs(o["cost"] - cost) <= 1e-3 * abs(cost), i
        assert rel_err(solo["y"], ref.y) <= 1e-3, i
    for f in facs:
        f.close()


def test_batch_per_problem_stopping():
    """Problems stop at their own first converged check; the others go on."""
    pbs = [batch_problem(i) for i in (0, 1, 3, 4)]
    facs = [rn.Factor(pb.net, pb.cost, pb.tree, precision=rn.RN_PREC_MIXED) for pb in pbs]
    tol = 5e-2
    outs = rn.solve_batch(facs, [tensors(pb) for pb in pbs], 3000, tol)
    for pb, f, o in zip(pbs, facs, outs):
        solo = f.solve(pb.data.x0, pb.data.q, pb.data.demand, pb.data.alpha, max_iters=3000,
                       tol=tol)
        assert o["iters"] == solo["iters"]
        assert np.array_equal(o["y"].cpu().numpy(), solo["y"])
        if o["iters"] < 3000:
            assert o["primal_res"] <= tol
    for f in facs:
        f.close()


def test_batch_rejects_fp64_handles():
    pb = batch_problem(0)
    f = rn.Factor(pb.net, pb.cost, pb.tree, gamma=1e-3)
    with pytest.raises(B.RapidNetError) as ei:
        rn.solve_batch([f], [tensors(pb)], 10)
    assert ei.value.status == B.RN_ERR_INVAL
    f.close()


def test_cap_below_the_work_items_is_refused():
    """A handle's own kernels need one resident block per work item: a
    smaller cap is refused at factor creation, before any launch."""
    pb = batch_problem(2)
    n = work_items(pb, 1e-3)
    assert n > 1
    with pytest.raises(B.RapidNetError) as ei:
        rn.Factor(pb.net, pb.cost, pb.tree, gamma=1e-3, precision=rn.RN_PREC_MIXED,
                  max_ctas=n - 1)
    assert ei.value.status == B.RN_ERR_UNSUPPORTED
    assert "work items" in str(ei.value)


def test_batch_refuses_dense_wu():
    """The batched kernel applies F in its sparse form: a handle with a
    dense W_u is refused before any launch."""
    from synthetic import make_cost
    pb = batch_problem(1)
    dense = make_cost(pb.net, seed=5, dense_wu=True)
    f = rn.Factor(pb.net, dense, pb.tree, gamma=1e-3, precision=rn.RN_PREC_MIXED)
    with pytest.raises(B.RapidNetError) as ei:
        rn.solve_batch([f], [tensors(pb)], 10)
    assert ei.value.status == B.RN_ERR_UNSUPPORTED
    f.close()


def test_batch_layouts_and_graph_replay_agree():
    """The layout chosen by timing candidates (batch_tune 0), the rule-based
    layout launched as a graph (1) and directly (2), and a replay of the
    captured graph all give the same results bit for bit: the per-component
    arithmetic does not depend on the team width or the work distribution."""
    pbs = [batch_problem(i) for i in range(6)]
    outs = {}
    for tune in (2, 1, 0):
        facs = [rn.Factor(pb.net, pb.cost, pb.tree, power_iters=50,
                          precision=rn.RN_PREC_MIXED, batch_tune=tune) for pb in pbs]
        data = [tensors(pb) for pb in pbs]
        first = rn.solve_batch(facs, data, 80)
        again = rn.solve_batch(facs, data, 80)  # same arguments: the graph replays
        for a, b in zip(first, again):
            for k in ("u", "x", "y"):
                assert np.array_equal(a[k].cpu().numpy(), b[k].cpu().numpy()), (tune, k)
            assert a["cost"] == b["cost"] and a["iters"] == b["iters"] == 80
        outs[tune] = [{k: o[k].cpu().numpy() for k in ("u", "x", "y")} for o in first]
        for f in facs:
            f.close()
    for tune in (1, 0):
        for a, b in zip(outs[tune], outs[2]):
            for k in ("u", "x", "y"):
                assert np.array_equal(a[k], b[k]), (tune, k)


def test_batch_with_split_subtrees_in_shared_blocks():
    """A tree whose stage-1 subtrees are split into parts (85 top nodes
    each), batched with small problems on a grid capped so that blocks
    hold several work items, parts of one root among them: the batched
    kernel runs the parts in two halves (no part waits for a part its own
    block has not started) and still equals the solo solve, which runs them
    in one."""
    net = make_network(10, 18, 12, 3, seed=61)
    tree = make_tree([2, 4, 4, 4, 2] + [1] * 4, seed=62)
    split = Problem(net=net, cost=make_cost(net, seed=61), tree=tree,
                    data=make_data(net, tree, seed=63))
    pbs = [batch_problem(0), split, batch_problem(1)]
    facs = [rn.Factor(pb.net, pb.cost, pb.tree, power_iters=50, precision=rn.RN_PREC_MIXED)
            for pb in pbs]
    items = [f.info()["grid_ctas"] for f in facs]
    assert facs[1].info()["n_top"] > 2 * 24  # the stage-1 subtrees are split
    for f in facs:
        f.close()
    # the batch takes the first handle's cap (which must cover that handle's
    # own work items); about four items to a block
    cap = max(items[0], sum(items) // 4)
    assert cap < sum(items) // 2
    facs = [rn.Factor(pb.net, pb.cost, pb.tree, power_iters=50, precision=rn.RN_PREC_MIXED,
                      max_ctas=cap if i == 0 else 0) for i, pb in enumerate(pbs)]
    outs = rn.solve_batch(facs, [tensors(pb) for pb in pbs], 60)
    for pb, f, o in zip(pbs, facs, outs):
        assert o["iters"] == 60
        solo = f.solve(pb.data.x0, pb.data.q, pb.data.demand, pb.data.alpha, max_iters=60)
        for k in ("u", "x", "y"):
            assert np.array_equal(o[k].cpu().numpy(), solo[k]), k
    for f in facs:
        f.close()
