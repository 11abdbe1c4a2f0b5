"""Closed loop on the GPU (paper §6.3 experiment shape): 24 hourly steps of
the stochastic MPC on a tree with one stage-1 node, warm-started duals.

Every applied move comes from an FP64 evaluation of the dual gradient, so
it meets the couplings E u + Ed d = 0 of its hour exactly; the plant obeys
the tank dynamics; the first hour's move equals a direct solve's; and the
indices are finite and consistent with the trajectory."""
import numpy as np
import pytest

import paper_1904_10548_gb300 as rn
from paper_1904_10548_gb300 import _binding as B
from paper_1904_10548_gb300.closed_loop import kpis, simulate
from synthetic import make_cost, make_data, make_network, make_tree

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("precision", [rn.RN_PREC_FP64, rn.RN_PREC_MIXED])
def test_closed_loop_24_hours(precision):
    net = make_network(16, 29, 22, 4, seed=21)
    cost = make_cost(net, seed=21)
    tree = make_tree([1, 3, 2, 2] + [1] * 8, seed=22)
    fac = rn.Factor(net, cost, tree, precision=precision)
    fc = [make_data(net, tree, seed=100 + k, hour0=k) for k in range(24)]
    start = make_data(net, tree, seed=99)
    out = simulate(fac, net, cost, lambda k: (fc[k].demand, fc[k].alpha), start.x0, start.q,
                   steps=24, max_iters=400)
    first = fac.solve(start.x0, start.q, fc[0].demand, fc[0].alpha, max_iters=400)
    fac.close()
    assert all(s in (B.RN_OK, B.RN_NOT_CONVERGED) for s in out.status)
    np.testing.assert_array_equal(out.u[0], first["u"][1])
    for k in range(24):
        d = fc[k].demand[1]
        cpl = net.E @ out.u[k] + net.Ed @ d
        assert np.abs(cpl).max() <= 1e-9 * max(1.0, np.abs(out.u[k]).max()), k
        np.testing.assert_allclose(out.x[k + 1], out.x[k] + net.B @ out.u[k] + net.Gd @ d,
                                   rtol=0, atol=1e-12 * np.abs(out.x).max())
    e, s = kpis(cost.alpha0, out.alpha, out.u, net.xs, out.x[1:])
    assert np.isfinite(out.kpi_e) and out.kpi_e == e and out.kpi_s == s
    assert 0 < out.kpi_tau_device <= out.kpi_tau
    assert np.all(out.iters == 400)
