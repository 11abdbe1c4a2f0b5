"""Host-side arithmetic of bench.py's roofline line (no GPU): the
algorithmic values per decision node and iteration, and the traffic record
that the line reports only while the kernel sources are the captured ones."""
import json
import os

import bench
from synthetic import make_problem

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_values_per_node_on_the_barcelona_network():
    """w read twice, y read, y+ and w+ written: 5 (2 nx + nu) values; the
    data terms c0, ubar and Gd d: 2 nu + nx.  For nx = 63, nu = 114 that is
    1,491 values, 5,964 bytes in FP32 and 63.6 MB per iteration over the
    10,664 decision nodes of the 512-scenario tree."""
    pb = make_problem("barcelona512")
    values, flops = bench.node_counts(pb.net)
    assert (pb.net.nx, pb.net.nu) == (63, 114)
    assert values == 1491
    n = int(pb.tree.stage_ptr[-1]) - 1
    assert n == 10664
    assert values * 4 * n == 63_600_096
    assert flops > 0


def test_per_node_bytes_of_the_matrix_stream():
    """The per-node form adds Phi_nu and K_nu (nu x nu each) per node:
    (1,491 + 2 * 114^2) values, 1.172 GB per iteration in FP32."""
    assert (1491 + 2 * 114 * 114) * 4 * 10664 == 1_172_314_848


def test_traffic_record_is_tied_to_the_sources():
    """Every record names its capture and a source hash; a kind that has
    none, or whose hash is not the current one, reports no traffic."""
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)
    for kind, d in rec.items():
        assert d["dram_bytes_per_iter"] > 0 and d["capture"] and len(d["source_hash"]) == 16
        sources = bench.PERNODE_SOURCES if kind.startswith("k_pn") else None
        got = bench.measured_traffic(kind, sources)
        if d["source_hash"] == bench.kernel_source_hash(sources):
            assert got == d["dram_bytes_per_iter"]
        else:
            assert got is None
    assert bench.measured_traffic("no_such_kernel") is None
