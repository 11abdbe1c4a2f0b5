"""CPU checks of the C ABI: the library loads, exports every function that
include/rapidnet.h declares, the ctypes structures match the C layouts,
and host-side validation rejects malformed input before any CUDA call."""
import ctypes
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

import paper_1904_10548_gb300 as rn
from paper_1904_10548_gb300 import _binding as B
from synthetic import make_problem, make_tree

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rapidnet.h")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(B.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return B.load()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"\b(rapidnet_\w+)\s*\(", text)))


def test_every_declared_function_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 7
    for name in names:
        assert hasattr(lib, name), name
        assert name in B.EXPORTS, name
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB_PATH], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\bT (rapidnet_\w+)", out))
    assert exported == set(names)


def test_ctypes_layouts_match_header(tmp_path):
    """Compile a C program against the header and compare sizeof/offsetof."""
    structs = {"rn_network": B.rn_network, "rn_tree": B.rn_tree, "rn_cost": B.rn_cost,
               "rn_opts": B.rn_opts, "rn_result": B.rn_result,
               "rn_factor_info": B.rn_factor_info, "rn_tree_out": B.rn_tree_out}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rapidnet.h"',
             'int main(void) {']
    for s, cls in structs.items():
        lines.append(f'printf("{s} %zu\\n", sizeof({s}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{s}.{f} %zu\\n", offsetof({s}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    for s, cls in structs.items():
        assert int(got[s]) == ctypes.sizeof(cls), s
        for f, _ in cls._fields_:
            assert int(got[f"{s}.{f}"]) == getattr(cls, f).offset, f"{s}.{f}"


def _args(pb, **over):
    net, cost, tree = pb.net, pb.cost, pb.tree
    for k, v in over.items():
        obj, attr = k.split("__")
        setattr({"net": net, "cost": cost, "tree": tree}[obj], attr, v)
    return net, cost, tree


def _factor_status(net, cost, tree, **kw):
    try:
        f = rn.Factor(net, cost, tree, gamma=1.0, **kw)
        f.close()
        return B.RN_OK
    except B.RapidNetError as e:
        return e.status


def test_validation_errors_before_cuda(lib):
    pb = make_problem("tiny")
    # A != I is outside what the shared-operator form handles (the default
    # form then is the per-node one, tests/test_pernode_cpu.py)
    net = make_problem("tiny").net
    net.A = np.eye(net.nx) * 1.01
    try:
        rn.Factor(net, pb.cost, pb.tree, gamma=1.0, factor_form=rn.RN_FACTOR_SHARED).close()
        status = B.RN_OK
    except B.RapidNetError as e:
        status = e.status
    assert status == B.RN_ERR_UNSUPPORTED
    assert "A = I" in rn.rapidnet_last_error()
    # a dense symmetric positive definite Wu passes validation (the next step
    # needs a device: RN_ERR_CUDA without one); an indefinite or
    # non-positive one is invalid
    pb2 = make_problem("tiny")
    pb2.cost.Wu = pb2.cost.Wu + 0.1
    assert _factor_status(pb2.net, pb2.cost, pb2.tree) in (B.RN_OK, B.RN_ERR_CUDA)
    pb3 = make_problem("tiny")
    pb3.cost.Wu = -pb3.cost.Wu
    assert _factor_status(pb3.net, pb3.cost, pb3.tree) == B.RN_ERR_INVAL
    pb3b = make_problem("tiny")
    # positive diagonal (8) but indefinite: -12 I + 20 (all ones)
    pb3b.cost.Wu = pb3b.cost.Wu + 20.0 - 25.0 * np.eye(pb3b.net.nu)
    assert _factor_status(pb3b.net, pb3b.cost, pb3b.tree) == B.RN_ERR_INVAL
    assert "positive definite" in rn.rapidnet_last_error()
    # box with xmin > xmax
    pb4 = make_problem("tiny")
    pb4.net.xmin = pb4.net.xmax + 1
    assert _factor_status(pb4.net, pb4.cost, pb4.tree) == B.RN_ERR_INVAL
    # tree: children probabilities that do not add up
    pb5 = make_problem("tiny")
    pb5.tree.prob = pb5.tree.prob.copy()
    pb5.tree.prob[3] *= 1.5
    assert _factor_status(pb5.net, pb5.cost, pb5.tree) == B.RN_ERR_INVAL
    assert "probability" in rn.rapidnet_last_error()
    # tree: a leaf before the last stage
    pb6 = make_problem("tiny")
    t = pb6.tree
    t.anc = t.anc.copy()
    last = t.stage_ptr[t.N + 1] - 1
    t.anc[last] = t.anc[last - 1]  # node of stage N-1 left without a child
    assert _factor_status(pb6.net, pb6.cost, t) == B.RN_ERR_INVAL
    # NaN in the data
    pb7 = make_problem("tiny")
    pb7.net.B = pb7.net.B.copy()
    pb7.net.B[0, 0] = np.nan
    assert _factor_status(pb7.net, pb7.cost, pb7.tree) == B.RN_ERR_INVAL


def test_empty_horizon_is_refused_by_both_forms(lib):
    """A tree of the root alone (N = 0: no decision after the current one)
    has nothing to iterate over: both factor forms refuse it with
    RN_ERR_INVAL before any CUDA call."""
    pb = make_problem("tiny")
    tree = make_tree([], seed=3)
    assert tree.N == 0 and tree.n_nodes == 1
    for form in (rn.RN_FACTOR_SHARED, rn.RN_FACTOR_PER_NODE, rn.RN_FACTOR_AUTO):
        assert _factor_status(pb.net, pb.cost, tree, factor_form=form) == B.RN_ERR_INVAL
        assert "N >= 1" in rn.rapidnet_last_error()


def test_valid_input_reaches_cuda_or_succeeds(lib):
    """Without a GPU a valid problem passes validation and fails at the first
    CUDA call with RN_ERR_CUDA; with a GPU it succeeds."""
    pb = make_problem("tiny")
    st = _factor_status(pb.net, pb.cost, pb.tree)
    assert st in (B.RN_OK, B.RN_ERR_CUDA, B.RN_ERR_NOMEM)


def test_server_argument_validation(lib):
    """The serving calls reject NULL or malformed arguments with
    RN_ERR_INVAL before touching a device; creation without a GPU fails in
    its CUDA call (RN_ERR_CUDA) and hands out no handle."""
    null = ctypes.c_void_p()
    assert lib.rapidnet_server_create(None, None) == B.RN_ERR_INVAL
    h = ctypes.c_void_p()
    st = lib.rapidnet_server_create(None, ctypes.byref(h))
    if st != B.RN_OK:
        assert st == B.RN_ERR_CUDA and not h.value
    else:
        lib.rapidnet_server_destroy(h)
    key = ctypes.c_int()
    assert lib.rapidnet_server_add_model(null, None, None, None, None, ctypes.byref(key)) == \
        B.RN_ERR_INVAL
    ticket = ctypes.c_longlong()
    v = np.zeros(8)
    pv = v.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert lib.rapidnet_server_submit(null, 0, pv, pv, pv, pv, 10, 0.0, 0,
                                      ctypes.byref(ticket)) == B.RN_ERR_INVAL
    assert lib.rapidnet_server_wait(null, 0, 0.0, None, None) == B.RN_ERR_INVAL
    assert lib.rapidnet_server_stats(null, None) == B.RN_ERR_INVAL
    lib.rapidnet_server_destroy(null)  # a NULL handle is ignored
    assert "NULL" in lib.rapidnet_last_error().decode()
