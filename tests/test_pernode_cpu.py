"""The per-node form's factor step on the host (no device work): the
matrices of the general recursion of §4.4 against the oracle's factor and
against identities that fix them independently, and the validation that
runs before any CUDA call."""
import numpy as np
import pytest

import oracle as O
import paper_1904_10548_gb300 as rn
from paper_1904_10548_gb300 import _binding as B
from synthetic import make_cost, make_problem


@pytest.fixture(scope="module", autouse=True)
def lib():
    import __graft_entry__
    __graft_entry__.build()


def general_A(nx, seed):
    """A state matrix other than I: a little leakage on the diagonal and
    sparse couplings between tanks."""
    rng = np.random.default_rng(seed)
    A = np.eye(nx) * (1.0 - 0.01 * rng.random(nx))
    mask = rng.random((nx, nx)) < 0.1
    return A + 0.03 * rng.standard_normal((nx, nx)) * mask


def case(name, dense):
    pb = make_problem(name)
    pb.net.A = general_A(pb.net.nx, 7)
    if dense:
        pb.cost.Wu = make_cost(pb.net, seed=41, dense_wu=True).Wu
    return pb


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("name,dense", [("tiny", False), ("tiny", True), ("barcelona32", False),
                                        ("barcelona32", True)])
def test_matrices_match_oracle_factor(name, dense):
    pb = case(name, dense)
    M = rn.pernode_matrices(pb.net, pb.cost, pb.tree)
    P = O.OracleProblem.from_parts(pb.net, pb.cost, pb.tree)
    F = O.factor(P)
    E = np.asarray(pb.net.E, float).reshape(pb.net.ne, pb.net.nu)
    assert rel(M["Phi"][1:], F.Phi[1:]) <= 1e-12
    assert rel(M["K"][1:], F.K[1:]) <= 1e-12
    assert rel(M["Mc"][1:], (F.Nm @ E.T[None])[1:]) <= 1e-12
    assert np.all(M["Phi"][0] == 0.0) and np.all(M["K"][0] == 0.0)


@pytest.mark.parametrize("dense", [False, True])
def test_matrices_satisfy_the_identities_of_the_recursion(dense):
    """Fixed without the oracle: Phi_nu maps into ker E (E Phi = 0), the
    recursion collapses onto 2 p Phi_nu = F = W^-1 - W^-1 E'(E W^-1 E')^-1
    E W^-1 at every node, K_nu = F W_u is a projector, and E Mc_nu = E E'
    (Mc = (I - Phi Q) E' and E Phi = 0)."""
    pb = case("barcelona32", dense)
    M = rn.pernode_matrices(pb.net, pb.cost, pb.tree)
    E = np.asarray(pb.net.E, float).reshape(pb.net.ne, pb.net.nu)
    W = np.asarray(pb.cost.Wu, float)
    Wi = np.linalg.inv(W)
    Fs = Wi - Wi @ E.T @ np.linalg.solve(E @ Wi @ E.T, E @ Wi)
    p = np.asarray(pb.tree.prob)
    Phi, K, Mc = M["Phi"][1:], M["K"][1:], M["Mc"][1:]
    assert np.abs(E[None] @ Phi).max() <= 1e-12 * np.abs(Phi).max()
    assert rel(2.0 * p[1:, None, None] * Phi, np.broadcast_to(Fs, Phi.shape)) <= 1e-10
    assert rel(K, np.broadcast_to(Fs @ W, K.shape)) <= 1e-10
    assert rel(K @ K, K) <= 1e-10
    assert rel(E[None] @ Mc, np.broadcast_to(E @ E.T, (len(Mc),) + (E.shape[0],) * 2)) <= 1e-10


def test_rank_deficient_E_is_refused():
    pb = make_problem("tiny")
    E = np.asarray(pb.net.E, float).reshape(pb.net.ne, pb.net.nu).copy()
    E[1] = 2.0 * E[0]
    pb.net.E = E
    with pytest.raises(B.RapidNetError) as ei:
        rn.pernode_matrices(pb.net, pb.cost, pb.tree)
    assert ei.value.status == B.RN_ERR_RANK


def _status(pb, **kw):
    try:
        f = rn.Factor(pb.net, pb.cost, pb.tree, gamma=1.0, **kw)
        f.close()
        return B.RN_OK
    except B.RapidNetError as e:
        return e.status


def test_form_selection_before_any_device_work():
    pb = case("tiny", False)
    # the shared-operator form needs A = I
    assert _status(pb, factor_form=rn.RN_FACTOR_SHARED) == B.RN_ERR_UNSUPPORTED
    assert "A = I" in rn.rapidnet_last_error()
    # every precision on the per-node form (the next step needs a device)
    for prec in (rn.RN_PREC_MIXED, rn.RN_PREC_FP32, rn.RN_PREC_FP64):
        assert _status(pb, factor_form=rn.RN_FACTOR_PER_NODE, precision=prec) in (
            B.RN_OK, B.RN_ERR_CUDA)
    # RN_PREC_FP32 on the shared form is not a precision it has
    pb_i = make_problem("tiny")
    assert _status(pb_i, factor_form=rn.RN_FACTOR_SHARED,
                   precision=rn.RN_PREC_FP32) == B.RN_ERR_INVAL
    assert _status(pb_i, factor_form=7) == B.RN_ERR_INVAL
    # with A != I the default form is the per-node one: on a machine
    # without a GPU that fails at the first CUDA call, after validation
    assert _status(pb) in (B.RN_OK, B.RN_ERR_CUDA)
