"""CPU checks of the shared-memory layout rules (layout.cpp): team width and
teams per block, the split of a block's shared memory into work buffers,
and the layouts that factor creation refuses before any launch.

layout.cpp and plan.cpp are compiled with g++ against a small driver that
replays factor creation's layout decision for given device attributes
(team_bytes_for gets the attributes that the library queries from the
device; the grid is the blocks per SM times the SMs, as the occupancy
query gives for these kernels).  The attributes below are
those of a GB300 (sm_103): 152 SMs, 227 KB of shared memory per block
(opt-in), 228 KB per SM, 1 KB reserved per block."""
import json
import os
import subprocess

import numpy as np
import pytest

from synthetic import make_network, make_tree

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1904_10548_gb300", "csrc")
CUDA_INC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
GB300 = dict(sms=152, optin=232448, per_sm=233472, reserved=1024)
RN_ERR_UNSUPPORTED = -6

DRIVER = r"""
#include <algorithm>
#include <cstdio>
#include <vector>
#include "kernels.cuh"
#include "rn_internal.h"
using namespace rn;
static int ceil4(int v) { return (v + 3) & ~3; }
// per-team bytes for `net` bytes of network data (0 if none are left)
static int budget(int n_items, int tpb, int block, int net, int sms, int optin, int per_sm,
                  int reserved, int *bpsm_out) {
  int tb = 0;
  if (team_bytes_for(sms, optin, per_sm, reserved, n_items, tpb, block, net, 0, &tb, bpsm_out))
    return 0;
  return tb;
}
static void dump(const char *k, const Sizes &z) {
  std::printf("\"%s\": {\"buf\": %d, \"gbuf\": %d, \"segb\": %d, \"gcap\": %d, \"hchunk\": %d,"
              " \"fslots\": %d, \"fbrows\": %d, \"team_bytes\": %d},\n", k, z.buf, z.gbuf, z.segb,
              z.gcap, z.hchunk, z.fslots, z.fbrows, z.team_bytes);
}
int main() {
  int N = 0, n = 0, nx, nu, ne, nnzB, nnzE, mixed, sms, optin, per_sm, reserved;
  if (std::scanf("%d %d", &N, &n) != 2) return 2;
  std::vector<int> sp(N + 2), anc(n);
  std::vector<double> prob(n);
  for (auto &x : sp) if (std::scanf("%d", &x) != 1) return 2;
  for (auto &x : anc) if (std::scanf("%d", &x) != 1) return 2;
  for (auto &x : prob) if (std::scanf("%lf", &x) != 1) return 2;
  if (std::scanf("%d %d %d %d %d %d %d %d %d %d", &nx, &nu, &ne, &nnzB, &nnzE, &mixed, &sms,
                 &optin, &per_sm, &reserved) != 10) return 2;
  rn_tree t{N, n, sp.data(), anc.data(), prob.data()};
  int tw = 0, tpb = 0, maxc = 0;
  int rc = team_layout(0, nx, nu, &tw, &tpb, &maxc);
  if (rc) { std::printf("{\"rc\": %d, \"stage\": \"team_layout\"}\n", rc); return 0; }
  Plan p0, p;
  if (build_plan(&t, p0) != RN_OK) return 3;
  const int chain_blocks = (p0.n_chains + tpb - 1) / tpb;
  if (build_plan(&t, p, std::max(1, sms - chain_blocks)) != RN_OK) return 3;
  const RowDims d{ceil4(nx), ceil4(nu), 2 * ceil4(nx) + ceil4(nu), ceil4(nx) + ceil4(nu),
                  std::max(1, ne)};
  const int block = tpb * tw, n_items = p.n_groups + (p.n_chains + tpb - 1) / tpb;
  const int net_d = (int)net_smem_bytes(nx, nu, ne, nnzB, nnzE, 8);
  const int net_f = (int)net_smem_bytes(nx, nu, ne, nnzB, nnzE, 4);
  std::printf("{\"tw\": %d, \"tpb\": %d, \"maxc\": %d, \"n_items\": %d, \"n_groups\": %d,"
              " \"n_roots\": %d, \"max_group\": %d, \"max_group_chains\": %d,\n", tw, tpb, maxc,
              n_items, p.n_groups, p.n_roots, p.max_group, p.max_group_chains);
  // the FP64 kernel's layout (every factor), then the mixed kernel's
  Sizes a, b, c;
  int bpsm = 1, grid = 0, smem = 0;
  {
    const int tb = budget(n_items, tpb, block, net_d, sms, optin, per_sm, reserved, &bpsm);
    grid = std::min(n_items, bpsm * sms);
    rc = tb <= 0 ? RN_ERR_UNSUPPORTED : layout_sizes(p, d, 8, tb, net_d, tw, tpb, 1, &c);
    if (!rc) rc = check_layout(p, c, n_items, grid, "fp64");
    smem = kHdrBytes + net_d + tpb * c.team_bytes;
    dump("fp64", c);
  }
  if (mixed && !rc) {
    const int net_m = net_f + (int)round16(sizeof(NetDev<double>));
    const int tb = budget(n_items, tpb, block, net_m, sms, optin, per_sm, reserved, &bpsm);
    grid = std::min(n_items, bpsm * sms);
    rc = tb <= 0 ? RN_ERR_UNSUPPORTED : layout_sizes(p, d, 4, tb, net_m, tw, tpb, 2, &a);
    if (!rc) rc = layout_sizes(p, d, 8, tb, net_f, tw, tpb, 0, &b);
    if (!rc) rc = check_layout(p, a, n_items, grid, "mixed");
    if (!rc) rc = check_layout(p, b, n_items, grid, "mixed fp64 steps");
    smem = std::max(smem, kHdrBytes + net_m + tpb * a.team_bytes);
    dump("f32", a);
    dump("f64", b);
  }
  std::printf("\"grid\": %d, \"bpsm\": %d, \"smem_per_block\": %d, \"rc\": %d}\n", grid, bpsm,
              smem, rc);
  return 0;
}
"""


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    d = tmp_path_factory.mktemp("layout")
    src = d / "driver.cpp"
    src.write_text(DRIVER)
    exe = d / "driver"
    r = subprocess.run(["g++", "-std=c++17", "-O1", f"-I{CSRC}", f"-I{os.path.join(ROOT, 'include')}",
                        f"-I{CUDA_INC}", str(src), os.path.join(CSRC, "layout.cpp"),
                        os.path.join(CSRC, "plan.cpp"), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return str(exe)


def layout(driver, net, tree, mixed=True, dev=GB300):
    nnzB = int(np.count_nonzero(net.B))
    nnzE = int(np.count_nonzero(net.E))
    text = f"{tree.N} {tree.n_nodes}\n" + " ".join(map(str, tree.stage_ptr)) + "\n"
    text += " ".join(map(str, tree.anc)) + "\n" + " ".join(repr(float(p)) for p in tree.prob) + "\n"
    text += (f"{net.nx} {net.nu} {net.ne} {nnzB} {nnzE} {int(mixed)} {dev['sms']} {dev['optin']} "
             f"{dev['per_sm']} {dev['reserved']}\n")
    r = subprocess.run([driver], input=text, capture_output=True, text=True)
    assert r.returncode == 0, (r.returncode, r.stderr)
    return json.loads(r.stdout)


BARCELONA = (63, 114, 88, 17)


@pytest.mark.parametrize("mixed", [True, False])
def test_benchmark_tree_fits_one_block_per_sm(driver, mixed):
    """512 scenarios on the Barcelona-sized network: 128 blocks of four
    chains and 24 group blocks, one 512-thread block per SM, every group in
    shared memory with all its heads staged at once."""
    net = make_network(*BARCELONA, seed=1)
    L = layout(driver, net, make_tree([8, 4, 4, 2, 2] + [1] * 19, seed=2), mixed)
    assert L["rc"] == 0
    assert (L["tw"], L["tpb"], L["maxc"]) == (128, 4, 2)
    assert L["n_items"] == L["grid"] == 152 and L["bpsm"] == 1
    assert L["n_groups"] == 24
    assert L["smem_per_block"] <= GB300["optin"]
    for k in ("fp64", "f32", "f64") if mixed else ("fp64",):
        z = L[k]
        assert z["gcap"] >= L["max_group"] and z["hchunk"] >= L["max_group_chains"]
        assert z["fslots"] >= 1 and z["segb"] >= 1


def test_small_networks_use_narrow_teams(driver):
    net = make_network(16, 29, 22, 4, seed=11)
    L = layout(driver, net, make_tree([4, 2, 2, 2] + [1] * 20, seed=2))
    assert L["rc"] == 0 and (L["tw"], L["tpb"], L["maxc"]) == (64, 4, 1)


def test_wide_networks_use_two_teams_of_256(driver):
    net = make_network(128, 230, 179, 35, seed=7)
    L = layout(driver, net, make_tree([4, 2, 2, 2] + [1] * 20, seed=2))
    assert (L["tw"], L["tpb"], L["maxc"]) == (256, 2, 4)
    assert L["rc"] == 0


def test_too_many_work_items_are_refused(driver):
    """More chain sets and groups than resident blocks (several items per
    block is not a validated path)."""
    net = make_network(*BARCELONA, seed=1)
    L = layout(driver, net, make_tree([8, 4, 4, 4, 2] + [1] * 19, seed=2))
    assert L["n_items"] > L["grid"]
    assert L["rc"] == RN_ERR_UNSUPPORTED


def test_oversized_network_is_refused(driver):
    net = make_network(300, 540, 420, 81, seed=3)
    L = layout(driver, net, make_tree([2, 2] + [1] * 4, seed=2))
    assert L["rc"] == RN_ERR_UNSUPPORTED and L.get("stage") == "team_layout"


def test_batched_benchmark_set(driver):
    """The layout rules on the benchmark's 256 batched problems refuse 42,
    all on the widest network (nx = 128), as factor creation did on a
    GB300."""
    import bench
    refused, widths = 0, set()
    for pb in bench.batch_problems(256):
        L = layout(driver, pb.net, pb.tree)
        if L["rc"] != 0:
            refused += 1
            widths.add(pb.net.nx)
    assert refused == 42
    assert widths == {128}


@pytest.mark.parametrize("counts", [[5], [1]])
def test_one_stage_horizons_fit(driver, counts):
    """A one-stage horizon (the root and its leaves): chains of one node
    under the root, one work item per chain set, a layout in both
    precisions."""
    net = make_network(8, 14, 10, 3, seed=5)
    tree = make_tree(counts, seed=3)
    for mixed in (True, False):
        L = layout(driver, net, tree, mixed)
        assert L["rc"] == 0, L
        assert L["n_items"] <= L["grid"]
