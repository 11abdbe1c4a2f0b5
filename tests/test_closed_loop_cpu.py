"""Host logic of the closed loop (paper §6.3): plant update, warm starts and
the three indices, with a stand-in for the GPU solve (no device needed)."""
import numpy as np

from paper_1904_10548_gb300.closed_loop import kpis, simulate
from synthetic import make_cost, make_data, make_network, make_tree


def setup():
    net = make_network(4, 6, 3, 2, seed=1)
    cost = make_cost(net, seed=1)
    tree = make_tree([1, 2, 2, 1, 1, 1], seed=2)
    return net, cost, tree


def test_plant_update_warm_start_and_kpis():
    net, cost, tree = setup()
    n = tree.n_nodes
    calls = []

    def fake_solve(x0, q, demand, alpha, max_iters, tol, y_warm):
        k = len(calls)
        calls.append((np.array(x0), np.array(q), None if y_warm is None else np.array(y_warm)))
        u = np.tile(0.5 * (net.umin + net.umax) * (1 + 0.01 * k), (n, 1))
        return dict(u=u, y=np.full((n, 2 * net.nx + net.nu), float(k)), apg_ms=1.0 + k,
                    iters=10, primal_res=0.5, status=0)

    forecasts = [make_data(net, tree, seed=10 + k, hour0=k) for k in range(6)]
    x0 = 0.6 * net.xmax
    out = simulate(None, net, cost, lambda k: (forecasts[k].demand, forecasts[k].alpha), x0,
                   np.zeros(net.nu), steps=6, solve=fake_solve)
    # plant: x_{k+1} = x_k + B u_k + Gd d_k with the stage-1 forecast as the demand
    for k in range(6):
        d = forecasts[k].demand[1]
        np.testing.assert_allclose(out.x[k + 1], out.x[k] + net.B @ out.u[k] + net.Gd @ d)
        np.testing.assert_array_equal(calls[k][0], out.x[k])
        np.testing.assert_array_equal(calls[k][1], out.u[k - 1] if k else np.zeros(net.nu))
        # warm start: the previous solve's dual
        assert (calls[k][2] is None) == (k == 0)
        if k:
            assert np.all(calls[k][2] == k - 1)
    # indices by their definitions
    e = np.mean([(cost.alpha0 + forecasts[k].alpha[1]) @ out.u[k] for k in range(6)])
    s = sum(np.abs(np.maximum(net.xs - out.x[k], 0)).sum() for k in range(1, 7))
    assert np.isclose(out.kpi_e, e) and np.isclose(out.kpi_s, s)
    assert out.kpi_tau == out.tau_s.max() and np.isclose(out.kpi_tau_device, 6e-3)


def test_kpi_safety_counts_only_violations():
    xs = np.array([1.0, 2.0])
    x = np.array([[0.5, 3.0], [2.0, 1.0]])
    e, s = kpis(np.zeros(1), np.ones((2, 1)), np.ones((2, 1)), xs, x)
    assert s == 0.5 + 1.0 and e == 1.0
