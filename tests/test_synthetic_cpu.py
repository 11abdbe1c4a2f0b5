"""The seeded synthetic workloads that stand in for the paper's Barcelona
network, demand forecasts and prices (§6): determinism, the structure the
method assumes (A = I, incidence matrices, full row rank of E, a tree
whose children's probabilities add up to their parent's and whose leaves
all sit at stage N), and per-node feasibility of the coupling within the
input box (checked by linear programs), without which the dual APG
diverges."""
import numpy as np
import pytest
from scipy.optimize import linprog

from synthetic import make_cost, make_network, make_problem, make_tree, random_branching


def _equal(a, b):
    for k in ("A", "B", "Gd", "E", "Ed", "xmin", "xmax", "xs", "umin", "umax"):
        if not np.array_equal(getattr(a.net, k), getattr(b.net, k)):
            return False
    return (np.array_equal(a.tree.prob, b.tree.prob) and np.array_equal(a.tree.anc, b.tree.anc)
            and np.array_equal(a.data.demand, b.data.demand)
            and np.array_equal(a.data.alpha, b.data.alpha) and np.array_equal(a.data.x0, b.data.x0))


def test_seeded_workloads_are_deterministic():
    assert _equal(make_problem("barcelona32"), make_problem("barcelona32"))
    assert not _equal(make_problem("barcelona32"), make_problem("barcelona32", net_seed=5))
    assert not _equal(make_problem("tiny"), make_problem("tiny", tree_seed=7))


@pytest.mark.parametrize("dims", [(4, 6, 3, 2), (63, 114, 88, 17), (128, 230, 179, 35),
                                  (8, 12, 6, 0)])
def test_network_structure(dims):
    net = make_network(*dims, seed=1)
    nx, nu, nd, ne = dims
    assert np.array_equal(net.A, np.eye(nx))
    for M in (net.B, net.E):
        assert set(np.unique(M)) <= {-1.0, 0.0, 1.0}
    # every flow has at most one tank or mixing node at each end
    col = np.abs(net.B).sum(0) + np.abs(net.E).sum(0)
    assert col.min() >= 1 and col.max() <= 2
    if ne > 0:
        assert np.linalg.matrix_rank(net.E) == ne
    # each demand is drawn from exactly one tank or one mixing node
    for M in (net.Gd, net.Ed):
        assert set(np.unique(M)) <= {-1.0, 0.0}
    assert np.array_equal(np.abs(net.Gd).sum(0) + np.abs(net.Ed).sum(0), np.ones(nd))
    assert np.all(net.umin == 0.0) and np.all(net.umax > 0.0)
    assert np.all(net.xmin == 0.0) and np.all((50.0 <= net.xmax) & (net.xmax <= 150.0))
    assert np.allclose(net.xs, 0.3 * net.xmax)


@pytest.mark.parametrize("tree", [
    make_tree([2, 2, 1, 1, 1, 1], seed=2),
    make_tree([4, 2, 2, 2] + [1] * 20, seed=2),
    make_tree([8, 4, 4, 2, 2] + [1] * 19, seed=2),
    random_branching(24, seed=5, s_min=16, s_max=512),
])
def test_tree_structure(tree):
    n, N = tree.n_nodes, tree.N
    assert tree.anc[0] == -1 and tree.prob[0] == 1.0
    assert np.all(np.diff(tree.stage_ptr) >= 1)
    # breadth-first: parents in the previous stage, children contiguous and
    # in parent order
    for v in range(1, n):
        assert tree.stage[tree.anc[v]] == tree.stage[v] - 1
    assert np.all(np.diff(tree.anc[1:]) >= 0)
    kids = np.zeros(n)
    np.add.at(kids, tree.anc[1:], tree.prob[1:])
    inner = np.bincount(tree.anc[1:], minlength=n) > 0
    assert np.allclose(kids[inner], tree.prob[inner], rtol=1e-12, atol=0)
    # every leaf at stage N, leaf probabilities sum to one
    assert np.all(tree.stage[~inner] == N)
    assert abs(tree.prob[tree.stage == N].sum() - 1.0) < 1e-12


def test_node_counts_of_the_named_workloads():
    assert make_problem("tiny").tree.n_nodes - 1 == 22
    assert make_problem("barcelona32").tree.n_nodes - 1 == 700
    assert make_problem("barcelona512").tree.n_nodes - 1 == 10664


def test_data_ranges():
    pb = make_problem("barcelona32")
    d, net = pb.data, pb.net
    assert np.all(d.demand[1:] > 0.0)
    assert np.all((0.4 * net.xmax <= d.x0) & (d.x0 <= 0.8 * net.xmax))
    assert np.all(d.alpha[1:] >= 0.0)
    cost = pb.cost
    assert np.allclose(cost.Wu, 13.0 * np.eye(net.nu))
    assert (cost.W_alpha, cost.Ws, cost.Wx) == (1.0, 0.1, 100.0)


@pytest.mark.parametrize("name,stride", [("tiny", 1), ("barcelona32", 7)])
def test_coupling_is_feasible_in_the_input_box_at_every_node(name, stride):
    """E u + Ed d = 0 with umin <= u <= umax has a solution at each node
    (sampled with the given stride), by a feasibility LP."""
    pb = make_problem(name)
    net = pb.net
    for v in range(1, pb.tree.n_nodes, stride):
        res = linprog(np.zeros(net.nu), A_eq=net.E, b_eq=-net.Ed @ pb.data.demand[v],
                      bounds=list(zip(net.umin, net.umax)), method="highs")
        assert res.status == 0, (v, res.message)


def test_batched_networks_are_feasible():
    """The widest network of the batched set, on the largest demands its
    generator draws (one LP per node of a 32-scenario tree, sampled)."""
    net = make_network(128, 230, 179, 35, seed=1000)
    from synthetic import make_data
    tree = make_tree([4, 2, 2, 2] + [1] * 20, seed=3)
    data = make_data(net, tree, seed=4)
    worst = int(np.argmax(data.demand[1:].sum(1))) + 1
    for v in sorted({worst, *range(1, tree.n_nodes, 31)}):
        res = linprog(np.zeros(net.nu), A_eq=net.E, b_eq=-net.Ed @ data.demand[v],
                      bounds=list(zip(net.umin, net.umax)), method="highs")
        assert res.status == 0, (v, res.message)
    assert make_cost(net, seed=1000).Wu.shape == (230, 230)
