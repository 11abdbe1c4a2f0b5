"""The allocation-free dual gradient (rapidnet_dual_gradient_noalloc).

Callers in a no-allocation phase (a real-time control loop, a host that
owns the memory pool) set up a factor handle once and then evaluate the
dual gradient with the library's fixed scratch array.  Its result must
equal that of the allocating entry point for the same data, on two calls
in a row (the array keeps the previous call's contents), and trees larger
than the array must be rejected.  This file is collected last so that a
failure here leaves every other test already run; it passes alone in a
fresh process and after the other tests.
"""
import numpy as np
import pytest

import paper_1904_10548_gb300 as rn
from paper_1904_10548_gb300 import _binding as B
from synthetic import make_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    assert torch.cuda.is_available()


def rel_err(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("name", ["tiny", "barcelona32"])
def test_noalloc_matches_allocating_entry_point_twice(name):
    import torch
    pb = make_problem(name)
    n, nx, nu = pb.tree.n_nodes, pb.net.nx, pb.net.nu
    ny = 2 * nx + nu
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    fac = rn.Factor(pb.net, pb.cost, pb.tree, gamma=1e-3)
    assert fac.info()["noalloc_bytes"] <= B.RN_NOALLOC_SCRATCH_BYTES
    rng = np.random.default_rng(4)
    u_ref = torch.empty((n, nu), dtype=torch.float64, device="cuda")
    x_ref = torch.empty((n, nx), dtype=torch.float64, device="cuda")
    u = torch.full((n, nu), np.nan, dtype=torch.float64, device="cuda")
    x = torch.full((n, nx), np.nan, dtype=torch.float64, device="cuda")
    # set-up: the allocating call with data prepares the handle
    w0 = dev(rng.standard_normal((n, ny)))
    fac.dual_gradient_device(w0, u_ref, x_ref, dev(pb.data.x0), dev(pb.data.q),
                             dev(pb.data.demand), dev(pb.data.alpha))
    for call in range(2):
        w = dev(rng.standard_normal((n, ny)) * (3.0 if call else 0.5))
        fac.dual_gradient_device(w, u_ref, x_ref)
        fac.dual_gradient_noalloc(w, u, x)
        torch.cuda.synchronize()
        assert rel_err(u.cpu().numpy(), u_ref.cpu().numpy()) <= 1e-9, call
        assert rel_err(x.cpu().numpy(), x_ref.cpu().numpy()) <= 1e-9, call
    fac.close()


def test_noalloc_rejects_trees_beyond_the_static_scratch():
    pb = make_problem("barcelona512")
    fac = rn.Factor(pb.net, pb.cost, pb.tree, gamma=1e-3)
    assert fac.info()["noalloc_bytes"] > B.RN_NOALLOC_SCRATCH_BYTES
    import torch
    n, nx, nu = pb.tree.n_nodes, pb.net.nx, pb.net.nu
    fac.solve(pb.data.x0, pb.data.q, pb.data.demand, pb.data.alpha, max_iters=1)
    w = torch.zeros((n, 2 * nx + nu), dtype=torch.float64, device="cuda")
    u = torch.empty((n, nu), dtype=torch.float64, device="cuda")
    x = torch.empty((n, nx), dtype=torch.float64, device="cuda")
    with pytest.raises(B.RapidNetError) as ei:
        fac.dual_gradient_noalloc(w, u, x)
    assert ei.value.status == B.RN_ERR_INVAL
    assert "static" in str(ei.value)
    fac.close()
