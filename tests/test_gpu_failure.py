"""Failure detection on the GPU without a fault: a device-side wait that runs out.

Every wait of the persistent kernels (a group block waiting for its
chains' arrivals, a chain team waiting for its group's flag, a part
waiting for its root, every block at the grid barrier) is a spin bounded
on the device clock.  With the bound set to one microsecond the group
blocks give up before their chains arrive: the launch must end with
RN_ERR_TIMEOUT naming the wait that gave up, leave the device usable, and
the next solve of a handle with the default bound must give the normal
result.  No flag is withheld and nothing faults: the waits simply run out
of time and every block leaves at its next check.
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


@pytest.mark.parametrize("precision", [rn.RN_PREC_FP64, rn.RN_PREC_MIXED])
def test_wait_limit_gives_timeout_and_device_stays_usable(precision):
    pb = make_problem("barcelona32")
    d = pb.data
    good = rn.Factor(pb.net, pb.cost, pb.tree, precision=precision)
    gamma = good.info()["gamma"]
    before = good.solve(d.x0, d.q, d.demand, d.alpha, max_iters=60)
    # a step size is given, so factor creation runs no kernel that waits
    short = rn.Factor(pb.net, pb.cost, pb.tree, precision=precision, gamma=gamma, wait_us=1)
    for _ in range(2):  # twice: the handle stays usable after a timeout
        with pytest.raises(B.RapidNetError) as ei:
            short.solve(d.x0, d.q, d.demand, d.alpha, max_iters=60)
        assert ei.value.status == B.RN_ERR_TIMEOUT
        assert "site" in str(ei.value) and "gave up after 1e-06 s" in str(ei.value)
    short.close()
    after = good.solve(d.x0, d.q, d.demand, d.alpha, max_iters=60)
    good.close()
    assert before["status"] == after["status"] == B.RN_OK
    for k in ("u", "x", "y"):
        assert np.array_equal(before[k], after[k]), k


def test_negative_wait_limit_is_invalid():
    pb = make_problem("tiny")
    with pytest.raises(B.RapidNetError) as ei:
        rn.Factor(pb.net, pb.cost, pb.tree, gamma=1e-3, wait_us=-1)
    assert ei.value.status == B.RN_ERR_INVAL
