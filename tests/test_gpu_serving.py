"""Serving (continuous batching): results are the same alone and in the mix.

Requests for three models (different networks and trees) are first run
one at a time, then all submitted at once; concurrent requests run on
separate slots (resident factor handles, one stream each) and overlap on
the device.  Each result must equal its alone result bit for bit and the
direct solve with the same step size; a small memory budget limits the
slots, a short queue rejects the surplus with RN_ERR_NOMEM.
"""
import time

import numpy as np
import pytest

import paper_1904_10548_gb300 as rn
from paper_1904_10548_gb300 import _binding as B
from synthetic import make_problem
from tests.test_gpu_batch import batch_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()


def models():
    return [make_problem("barcelona32"), make_problem("tiny"), batch_problem(1)]


def perturbed(pb, k):
    rng = np.random.default_rng(50 + k)
    d = pb.data
    return (d.x0 * (1 + 0.01 * rng.standard_normal(d.x0.shape)), d.q,
            d.demand * (1 + 0.02 * rng.standard_normal(d.demand.shape)), d.alpha)


def test_alone_equals_in_the_mix():
    pbs = models()
    srv = rn.Server(workers=6, slots_per_model=2)
    keys = [srv.add_model(pb.net, pb.cost, pb.tree) for pb in pbs]
    reqs = [(i % 3, perturbed(pbs[i % 3], i)) for i in range(12)]
    iters = 400
    alone, t_alone = [], 0.0
    for key, data in reqs:
        t0 = time.perf_counter()
        alone.append(srv.wait(key, srv.submit(key, *data, max_iters=iters)))
        t_alone += time.perf_counter() - t0
    for rep in range(3):  # early passes may still open slots
        t0 = time.perf_counter()
        tickets = [srv.submit(key, *data, max_iters=iters) for key, data in reqs]
        mixed = [srv.wait(key, t) for (key, _), t in zip(reqs, tickets)]
        t_mix = time.perf_counter() - t0
    st = srv.stats()
    for a, b in zip(alone, mixed):
        assert a["status"] == b["status"] == B.RN_OK
        for k in ("u", "x", "y"):
            assert np.array_equal(a[k], b[k])
        assert a["cost"] == b["cost"]
    assert st["completed"] == 48 and st["slots"] > 3  # concurrent requests use several slots
    # they overlapped on the device: the persistent launches of two requests
    # ran at the same time (device-clock stamps taken inside the kernels)
    spans = sorted((b["t_begin_ns"], b["t_end_ns"]) for b in mixed)
    assert all(0 < t0 < t1 for t0, t1 in spans), spans
    overlap = max(min(spans[i][1], spans[j][1]) - max(spans[i][0], spans[j][0])
                  for i in range(len(spans)) for j in range(i + 1, len(spans)))
    assert overlap > 0, (spans, t_mix, t_alone)
    # the same as a direct solve with the model's step size
    for (key, data), a in zip(reqs[:3], alone[:3]):
        pb = pbs[key]
        f = rn.Factor(pb.net, pb.cost, pb.tree, precision=rn.RN_PREC_MIXED)
        d = f.solve(*data, max_iters=iters)
        f.close()
        assert np.array_equal(d["y"], a["y"])
    srv.close()


def test_budget_and_queue_admission():
    pb = make_problem("tiny")
    srv = rn.Server(workers=4, budget_bytes=1, max_queue=3)
    key = srv.add_model(pb.net, pb.cost, pb.tree)
    tickets, rejected = [], 0
    for k in range(40):
        try:
            tickets.append(srv.submit(key, *perturbed(pb, k), max_iters=2000))
        except B.RapidNetError as e:
            assert e.status == B.RN_ERR_NOMEM
            rejected += 1
    outs = [srv.wait(key, t) for t in tickets]
    st = srv.stats()
    assert rejected > 0 and st["rejected"] == rejected
    assert st["slots"] == 1   # the budget admits no second slot
    assert all(o["status"] == B.RN_OK for o in outs)
    with pytest.raises(B.RapidNetError):
        srv.wait(key, tickets[0])  # a ticket is returned once
    srv.close()


def test_warm_start_uses_the_slot_dual():
    pb = make_problem("tiny")
    srv = rn.Server(workers=1)
    key = srv.add_model(pb.net, pb.cost, pb.tree)
    data = perturbed(pb, 0)
    first = srv.wait(key, srv.submit(key, *data, max_iters=200))
    warm = srv.wait(key, srv.submit(key, *data, max_iters=200, warm=True))
    f = rn.Factor(pb.net, pb.cost, pb.tree, precision=rn.RN_PREC_MIXED)
    ref = f.solve(*data, max_iters=200, y_warm=first["y"])
    f.close()
    assert np.array_equal(warm["y"], ref["y"])
    srv.close()


@pytest.mark.parametrize("precision", [rn.RN_PREC_MIXED, rn.RN_PREC_FP64])
def test_per_node_model_is_served(precision):
    """A model with A != I takes the per-node form (RN_FACTOR_AUTO, as in
    rapidnet_factor) and is served beside a shared-form model: its requests,
    alone and in the mix, equal a direct per-node solve of the same request
    bit for bit, and so do the shared-form model's."""
    from tests.test_gpu_pernode import problem as pn_problem
    pbs = [pn_problem("tiny_A"), make_problem("tiny")]
    srv = rn.Server(workers=4, slots_per_model=2)
    keys = [srv.add_model(pb.net, pb.cost, pb.tree, precision=precision) for pb in pbs]
    reqs = [(i % 2, perturbed(pbs[i % 2], i)) for i in range(8)]
    iters = 300
    alone = [srv.wait(keys[k], srv.submit(keys[k], *data, max_iters=iters)) for k, data in reqs]
    tickets = [srv.submit(keys[k], *data, max_iters=iters) for k, data in reqs]
    mixed = [srv.wait(keys[k], t) for (k, _), t in zip(reqs, tickets)]
    srv.close()
    for a, b in zip(alone, mixed):
        assert a["status"] == b["status"] == B.RN_OK
        for k in ("u", "x", "y"):
            assert np.array_equal(a[k], b[k])
    for (k, data), a in zip(reqs[:2], alone[:2]):
        pb = pbs[k]
        f = rn.Factor(pb.net, pb.cost, pb.tree, precision=precision)
        assert f.info()["factor_form"] == (rn.RN_FACTOR_PER_NODE if k == 0 else
                                           rn.RN_FACTOR_SHARED)
        d = f.solve(*data, max_iters=iters)
        f.close()
        for key in ("u", "x", "y"):
            assert np.array_equal(d[key], a[key])
