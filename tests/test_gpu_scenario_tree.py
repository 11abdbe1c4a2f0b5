"""Scenario-tree construction on the GPU (rapidnet_scenario_tree) against
the oracle (oracle/scenario_tree.py, fast forward selection of Heitsch and
Römisch, pinned in tests/test_scenario_tree_cpu.py).

The selections are decisions taken on FP64 sums that the two sides add in
different orders; on continuous random paths no two candidates come within
rounding of each other, so the trees must agree exactly in structure and
representatives, probabilities to 1e-12 and values bit for bit."""
import numpy as np
import pytest

import paper_1904_10548_gb300 as rn
from oracle.scenario_tree import build_tree
from paper_1904_10548_gb300 import _binding as B
from synthetic import make_price_paths

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("S,N,dim,branching,uniform", [
    (300, 8, 2, [3, 2, 2, 1, 1, 1, 1, 1], False),
    (1000, 24, 1, [8, 4, 2] + [1] * 21, True),
    (50, 6, 3, [4, 4, 4, 4, 1, 1], False),   # bundles smaller than the branching
])
def test_tree_matches_oracle(S, N, dim, branching, uniform):
    paths = make_price_paths(S, N, dim, seed=S + N)
    prob = None if uniform else np.random.default_rng(1).dirichlet(np.ones(S))
    got = rn.scenario_tree(paths, branching, prob)
    ref = build_tree(paths, np.full(S, 1.0 / S) if uniform else prob, branching)
    n = len(ref.anc)
    assert got["n_nodes"] == n
    np.testing.assert_array_equal(got["stage_ptr"], ref.stage_ptr)
    np.testing.assert_array_equal(got["anc"], ref.anc)
    np.testing.assert_array_equal(got["rep"], ref.rep)
    np.testing.assert_array_equal(got["leaf_of"], ref.leaf_of)
    np.testing.assert_allclose(got["prob"], ref.prob, rtol=1e-12, atol=1e-15)
    np.testing.assert_array_equal(got["value"], ref.value)


def test_tree_feeds_the_solver():
    """A reduced price tree is a valid scenario tree for rapidnet_factor."""
    from synthetic import make_cost, make_data, make_network
    from synthetic.tree import Tree
    paths = make_price_paths(400, 12, 1, seed=3)
    t = rn.scenario_tree(paths, [4, 2, 2] + [1] * 9)
    stage = np.repeat(np.arange(13), np.diff(t["stage_ptr"]))
    tree = Tree(N=12, n_nodes=t["n_nodes"], stage_ptr=t["stage_ptr"].astype(np.int64),
                anc=t["anc"].astype(np.int64), prob=t["prob"], stage=stage)
    net = make_network(6, 11, 8, 2, seed=4)
    f = rn.Factor(net, make_cost(net, seed=4), tree, precision=rn.RN_PREC_MIXED)
    d = make_data(net, tree, seed=5)
    out = f.solve(d.x0, d.q, d.demand, d.alpha, max_iters=50)
    f.close()
    assert out["status"] == B.RN_OK and np.isfinite(out["cost"])


def test_invalid_arguments():
    paths = make_price_paths(20, 4, 1, seed=1)
    with pytest.raises(B.RapidNetError) as ei:
        rn.scenario_tree(paths, [2, 0, 1, 1])
    assert ei.value.status == B.RN_ERR_INVAL
    with pytest.raises(B.RapidNetError) as ei:
        rn.scenario_tree(paths, [2, 1, 1, 1], prob=np.full(20, 0.1))
    assert ei.value.status == B.RN_ERR_INVAL
