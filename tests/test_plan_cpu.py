"""CPU checks of the work schedule over the scenario tree (rn::build_plan):
the host-side logic that decides which thread block sums which top nodes,
which chain owns which top node's per-node step and where every node sits
in the internal order.  plan.cpp is compiled with g++ against a small
driver that prints the schedule; the invariants below are what the
persistent kernels rely on (a violated one would make a kernel read the
wrong rows or wait for arrivals that never come)."""
import json
import os
import subprocess

import numpy as np
import pytest

from synthetic import make_tree
from synthetic.tree import _build, random_branching

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1904_10548_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include <vector>
#include "rn_internal.h"
static void dump(const char *name, const std::vector<int> &v, bool last = false) {
  std::printf("\"%s\": [", name);
  for (size_t i = 0; i < v.size(); ++i) std::printf(i ? ",%d" : "%d", v[i]);
  std::printf("]%s\n", last ? "" : ",");
}
int main() {
  int N = 0, n = 0, max_groups = 1 << 30;
  if (std::scanf("%d %d %d", &N, &n, &max_groups) != 3) return 2;
  std::vector<int> sp(N + 2), anc(n);
  std::vector<double> prob(n);
  for (auto &x : sp) std::scanf("%d", &x);
  for (auto &x : anc) std::scanf("%d", &x);
  for (auto &x : prob) std::scanf("%lf", &x);
  rn_tree t{N, n, sp.data(), anc.data(), prob.data()};
  rn::Plan p;
  if (rn::build_plan(&t, p, max_groups) != RN_OK) return 3;
  std::printf("{\"n_top\": %d, \"n_chains\": %d, \"n_groups\": %d, \"max_group\": %d,"
              " \"max_group_chains\": %d, \"max_chain_len\": %d, \"n_roots\": %d,\n",
              p.n_top, p.n_chains, p.n_groups, p.max_group, p.max_group_chains, p.max_chain_len,
              p.n_roots);
  dump("g_root", p.g_root); dump("r_node", p.r_node); dump("r_part", p.r_part);
  dump("g_hp", p.g_hp); dump("r_hp", p.r_hp);
  dump("perm", p.perm); dump("parent", p.parent); dump("g_node", p.g_node);
  dump("g_chain", p.g_chain); dump("g_lvl", p.g_lvl); dump("lvl", p.lvl);
  dump("g_ccn", p.g_ccn); dump("ccn", p.ccn); dump("tc_ptr", p.tc_ptr); dump("tc", p.tc);
  dump("cc_ptr", p.cc_ptr); dump("cc", p.cc); dump("ch_start", p.ch_start);
  dump("ch_len", p.ch_len); dump("ch_group", p.ch_group); dump("ch_parent", p.ch_parent);
  dump("ch_own_ptr", p.ch_own_ptr); dump("ch_own", p.ch_own, true);
  std::printf("}\n");
  return 0;
}
"""


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    d = tmp_path_factory.mktemp("plan")
    src = d / "driver.cpp"
    src.write_text(DRIVER)
    exe = d / "driver"
    r = subprocess.run(["g++", "-std=c++17", "-O1", f"-I{CSRC}", f"-I{os.path.join(ROOT, 'include')}",
                        str(src), os.path.join(CSRC, "plan.cpp"), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return str(exe)


def plan_of(driver, tree, max_groups=1 << 30):
    text = f"{tree.N} {tree.n_nodes} {max_groups}\n" + " ".join(map(str, tree.stage_ptr)) + "\n"
    text += " ".join(map(str, tree.anc)) + "\n" + " ".join(repr(float(p)) for p in tree.prob)
    r = subprocess.run([driver], input=text, capture_output=True, text=True)
    assert r.returncode == 0, r.returncode
    return json.loads(r.stdout)


TREES = {
    "tiny": lambda: make_tree([2, 2, 1, 1, 1, 1], seed=2),
    "barcelona32": lambda: make_tree([4, 2, 2, 2] + [1] * 20, seed=2),
    "barcelona512": lambda: make_tree([8, 4, 4, 2, 2] + [1] * 19, seed=2),
    "uneven": lambda: random_branching(12, seed=21, s_min=6, s_max=40, branch_stages=5),
    "single": lambda: make_tree([1] * 20, seed=6),
    "ne0": lambda: make_tree([3, 2, 1, 2, 1, 1, 1], seed=9),
    "stage1_chains": lambda: _build([[4], [1, 2, 1, 3], [1, 1, 2, 1, 1, 1, 1], [1] * 8, [1] * 8,
                                     [1] * 8], 12),
    # one-stage horizons: the root with five leaves, the root with one
    "horizon1": lambda: make_tree([5], seed=3),
    "horizon1_single": lambda: make_tree([1], seed=3),
    # three stage-1 subtrees: split, unsplit, split (with room for more groups)
    "mixed_split": lambda: random_branching(24, seed=2006, s_min=16, s_max=512),
}


@pytest.mark.parametrize("name,max_groups", [(t, 1 << 30) for t in sorted(TREES)] +
                         [("barcelona512", 24), ("barcelona512", 16), ("barcelona512", 8),
                          ("mixed_split", 82)])
def test_schedule_invariants(driver, name, max_groups):
    tree = TREES[name]()
    p = plan_of(driver, tree, max_groups)
    n, n_top, K, G = tree.n_nodes, p["n_top"], p["n_chains"], p["n_groups"]
    perm = np.array(p["perm"])
    parent = np.array(p["parent"])
    assert sorted(perm) == list(range(n)) and perm[0] == 0
    # leaves below every original node
    leaves = np.zeros(n, int)
    nchild = np.zeros(n, int)
    for v in range(n - 1, 0, -1):
        nchild[tree.anc[v]] += 1
    for v in range(n - 1, -1, -1):
        if nchild[v] == 0:
            leaves[v] = 1
        if v > 0:
            leaves[tree.anc[v]] += leaves[v]
    # internal 1..n_top are exactly the nodes with two or more leaves
    assert all(leaves[perm[i]] >= 2 for i in range(1, n_top + 1))
    assert all(leaves[perm[i]] == 1 for i in range(n_top + 1, n))
    assert K == tree.n_scenarios
    for i in range(1, n):
        assert perm[parent[i]] == tree.anc[perm[i]]
    # groups: one per stage-1 top node, or (split) one per top child of a
    # stage-1 root; contiguous, levels in breadth-first order; roots last
    stage1_top = [v for v in range(tree.stage_ptr[1], tree.stage_ptr[2]) if leaves[v] >= 2]
    g_node, lvl, g_lvl = p["g_node"], p["lvl"], p["g_lvl"]
    g_root, r_node, r_part, R = p["g_root"], p["r_node"], p["r_part"], p["n_roots"]
    assert len(g_node) == G + 1 and g_node[0] == 1 and g_node[-1] + R == n_top + 1
    assert sorted(r_node) == list(range(g_node[-1], n_top + 1))
    assert sorted(perm[r_node[r]] for r in range(R)) == sorted(
        v for v in stage1_top if v in {perm[x] for x in r_node})
    group_of = {}
    for g in range(G):
        b = lvl[g_lvl[g]:g_lvl[g + 1]]
        assert b[0] == g_node[g] and b[-1] == g_node[g + 1]
        top = g_node[g]
        if g_root[g] < 0:
            assert perm[top] in stage1_top and parent[top] == 0 and b[1] == top + 1
        else:
            r = g_root[g]
            assert r_part[2 * r] <= g < r_part[2 * r + 1]
            # the group's top nodes are consecutive children of the root, and
            # their sums go to the root's hp rows in child order
            kids = sorted(i for i in range(1, n) if parent[i] == r_node[r])
            first = kids.index(top)
            assert p["g_hp"][g] == p["r_hp"][r] + first
            assert kids[first:first + b[1] - b[0]] == list(range(b[0], b[1]))
        for l in range(len(b) - 1):
            assert b[l] < b[l + 1]
            for v in range(b[l], b[l + 1]):
                group_of[v] = g
                if l == 0:
                    assert parent[v] == (0 if g_root[g] < 0 else r_node[g_root[g]])
                else:
                    assert b[l - 1] <= parent[v] < b[l]  # parent one level up
    assert sorted(group_of) == list(range(1, g_node[-1]))
    covered_stage1 = {perm[g_node[g]] for g in range(G) if g_root[g] < 0} | {perm[x] for x in r_node}
    assert covered_stage1 == set(stage1_top)
    for r in range(R):
        kids = [i for i in range(1, n) if parent[i] == r_node[r]]
        tops = [v for g in range(r_part[2 * r], r_part[2 * r + 1])
                for v in range(lvl[g_lvl[g]], lvl[g_lvl[g] + 1])]
        assert sorted(kids) == sorted(tops) and p["r_hp"][r + 1] - p["r_hp"][r] == len(kids)
    assert G <= max(max_groups, len(stage1_top))
    for r in range(R):
        assert [g for g in range(G) if g_root[g] == r] == list(range(r_part[2 * r], r_part[2 * r + 1]))
    if G:
        assert max(g_node[g + 1] - g_node[g] for g in range(G)) == p["max_group"]
    # children lists of the top nodes
    tc_ptr, tc, cc_ptr, cc = p["tc_ptr"], p["tc"], p["cc_ptr"], p["cc"]
    ch_start, ch_len = p["ch_start"], p["ch_len"]
    for v in range(1, n_top + 1):
        kids = sorted(i for i in range(1, n) if parent[i] == v)
        tops = tc[tc_ptr[v]:tc_ptr[v + 1]]
        chains = cc[cc_ptr[v]:cc_ptr[v + 1]]
        assert sorted(tops + [ch_start[k] for k in chains]) == kids
        if v in group_of:
            assert all(t <= n_top and group_of[t] == group_of[v] for t in tops)
        else:
            assert chains == []  # a root has no chain child
    # nodes with chain children, per group
    ccn, g_ccn = p["ccn"], p["g_ccn"]
    for g in range(G):
        want = [v for v in range(g_node[g], g_node[g + 1]) if cc_ptr[v + 1] > cc_ptr[v]]
        assert ccn[g_ccn[g]:g_ccn[g + 1]] == want
    # chains: contiguous rows head to leaf, parent, group, contiguous per group
    covered = []
    for k in range(K):
        rows = list(range(ch_start[k], ch_start[k] + ch_len[k]))
        covered += rows
        assert parent[rows[0]] == p["ch_parent"][k]
        for a, b in zip(rows, rows[1:]):
            assert parent[b] == a
        assert nchild[perm[rows[-1]]] == 0
        par = p["ch_parent"][k]
        assert p["ch_group"][k] == (group_of[par] if par > 0 else -1)
        assert par == 0 or par in group_of
    assert sorted(covered) == list(range(n_top + 1, n))
    g_chain = p["g_chain"]
    for g in range(G):
        ks = [k for k in range(K) if p["ch_group"][k] == g]
        assert ks == list(range(g_chain[2 * g], g_chain[2 * g + 1]))
    assert p["max_chain_len"] == max(ch_len)
    # ownership: every top node exactly once, by the first chain below it
    own = p["ch_own"]
    assert sorted(own) == list(range(1, n_top + 1))
    for k in range(K):
        path = []
        a = p["ch_parent"][k]
        while a > 0:
            path.append(a)
            a = parent[a]
        mine = own[p["ch_own_ptr"][k]:p["ch_own_ptr"][k + 1]]
        assert mine == [v for v in reversed(path) if v in mine]  # path order, stage 1 down
        for v in mine:
            first = min(kk for kk in range(K) if v in _ancestors(parent, ch_start[kk]))
            assert first == k


def _ancestors(parent, v):
    out = set()
    while v > 0:
        v = parent[v]
        if v > 0:
            out.add(v)
    return out


def test_schedule_sizes_of_the_benchmark_tree(driver):
    """Branching [8, 4, 4, 2, 2]: every stage-1 subtree (53 top nodes) is
    split into its 4 stage-2 subtrees, so 32 groups of 13 top nodes with 16
    chains of 20 nodes each, and 8 roots (the stage-1 nodes)."""
    p = plan_of(driver, TREES["barcelona512"]())
    assert p["n_groups"] == 32 and p["n_roots"] == 8 and p["max_group"] == 1 + 4 + 8
    assert p["max_group_chains"] == 16 and p["max_chain_len"] == 20
    assert p["n_chains"] == 512 and p["n_top"] == 8 * 53
    assert p["r_part"] == [x for r in range(8) for x in (4 * r, 4 * r + 4)]


def test_benchmark_tree_within_a_group_budget(driver):
    """With room for 24 groups beside the chain blocks, each stage-1
    subtree is split into 3 parts (bundles of 2, 1 and 1 stage-2 subtrees);
    with 16 into 2; with 8 not at all."""
    for budget, parts, biggest in [(24, 3, 26), (16, 2, 26), (8, 1, 53)]:
        p = plan_of(driver, TREES["barcelona512"](), budget)
        assert p["n_groups"] == 8 * parts and p["max_group"] == biggest
        assert p["n_roots"] == (8 if parts > 1 else 0)


def test_small_subtrees_are_not_split(driver):
    """Branching [4, 2, 2, 2]: 7 top nodes per stage-1 subtree, one group each."""
    p = plan_of(driver, TREES["barcelona32"]())
    assert p["n_groups"] == 4 and p["n_roots"] == 0 and p["max_group"] == 7
