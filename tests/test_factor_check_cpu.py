"""CPU checks of the factor check (rn::collapse_deviation): one step of the
general per-node recursion of the dual gradient (paper §4.4; Q = 2 p W_u +
sum of the children's P, Phi = L (L' Q L)^-1 L') evaluated with the shared
operator F = W^-1 - W^-1 E' S^-1 E W^-1 that the kernels apply.  The
library refuses a factor whose F does not reproduce 2 p Phi.

factor_check.cpp is compiled with g++ against a small driver that builds
S^-1 with the library's own Cholesky helpers, optionally from a planted
wrong W or a scaled S^-1, and prints the deviation."""
import os
import subprocess

import numpy as np
import pytest
from scipy.linalg import null_space

from synthetic import make_network, make_tree

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1904_10548_gb300", "csrc")
TOL = 1e-8  # kCollapseTol

DRIVER = r"""
#include <cstdio>
#include <vector>
#include "rn_internal.h"
int main() {
  int N = 0, n = 0, nu = 0, ne = 0;
  if (std::scanf("%d %d", &N, &n) != 2) return 2;
  std::vector<int> sp(N + 2), anc(n);
  std::vector<double> prob(n);
  for (auto &x : sp) std::scanf("%d", &x);
  for (auto &x : anc) std::scanf("%d", &x);
  for (auto &x : prob) std::scanf("%lf", &x);
  if (std::scanf("%d %d", &nu, &ne) != 2) return 2;
  std::vector<double> E((size_t)ne * nu), wS(nu), w(nu);
  double scale = 1.0;
  for (auto &x : E) std::scanf("%lf", &x);
  for (auto &x : wS) std::scanf("%lf", &x);
  for (auto &x : w) std::scanf("%lf", &x);
  std::scanf("%lf", &scale);
  // S = E W_S^-1 E' and its inverse, scaled by `scale`
  std::vector<double> S((size_t)ne * ne, 0.0), Sinv(ne > 0 ? (size_t)ne * ne : 1, 0.0), winv(nu);
  for (int j = 0; j < nu; ++j) winv[j] = 1.0 / w[j];
  for (int r = 0; r < ne; ++r)
    for (int c = 0; c < ne; ++c)
      for (int j = 0; j < nu; ++j) S[(size_t)r * ne + c] += E[(size_t)r * nu + j] * E[(size_t)c * nu + j] / wS[j];
  if (ne > 0) {
    if (!rn::cholesky(S, ne)) return 4;
    Sinv = rn::chol_inverse(S, ne);
    for (auto &x : Sinv) x *= scale;
  }
  rn_tree t{N, n, sp.data(), anc.data(), prob.data()};
  std::printf("%.17g\n", rn::collapse_deviation(&t, nu, ne, E.data(), winv.data(), Sinv.data()));
  return 0;
}
"""


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    d = tmp_path_factory.mktemp("factor_check")
    src = d / "driver.cpp"
    src.write_text(DRIVER)
    exe = d / "driver"
    r = subprocess.run(["g++", "-std=c++17", "-O2", f"-I{CSRC}", f"-I{os.path.join(ROOT, 'include')}",
                        str(src), os.path.join(CSRC, "factor_check.cpp"), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return str(exe)


def deviation(driver, tree, E, w, wS=None, scale=1.0):
    nu = len(w)
    ne = E.shape[0]
    wS = w if wS is None else wS
    text = f"{tree.N} {tree.n_nodes}\n" + " ".join(map(str, tree.stage_ptr)) + "\n"
    text += " ".join(map(str, tree.anc)) + "\n" + " ".join(repr(float(p)) for p in tree.prob) + "\n"
    text += f"{nu} {ne}\n" + " ".join(repr(float(v)) for v in E.ravel()) + "\n"
    text += " ".join(repr(float(v)) for v in wS) + "\n" + " ".join(repr(float(v)) for v in w)
    text += f"\n{scale!r}\n"
    r = subprocess.run([driver], input=text, capture_output=True, text=True)
    assert r.returncode == 0, r.returncode
    return float(r.stdout)


def sampled_nodes(tree):
    out = []
    for t in (1, (tree.N + 1) // 2, tree.N):
        v = int(tree.stage_ptr[t])
        if v not in out:
            out.append(v)
    return out


def numpy_deviation(tree, E, w, wS, scale):
    """The same quantity from an independent evaluation: L from an SVD
    (scipy null_space), dense numpy algebra."""
    nu, ne = len(w), E.shape[0]
    W, Wi = np.diag(w), np.diag(1.0 / w)
    S = E @ np.diag(1.0 / wS) @ E.T
    Sinv = np.linalg.inv(S) * scale
    F = Wi - Wi @ E.T @ Sinv @ E @ Wi
    L = null_space(E) if ne > 0 else np.eye(nu)
    D = W - W @ F @ W
    stage = np.searchsorted(tree.stage_ptr, np.arange(tree.n_nodes), side="right") - 1
    worst = 0.0
    for v in sampled_nodes(tree):
        pc = sum(tree.prob[c] for c in range(tree.n_nodes) if tree.anc[c] == v and c != v)
        Q = 2 * tree.prob[v] * W + 2 * pc * D
        Phi = L @ np.linalg.inv(L.T @ Q @ L) @ L.T
        worst = max(worst, np.abs(2 * tree.prob[v] * Phi - F).max() / np.abs(F).max())
        assert stage[v] >= 1
    return worst


BARCELONA = dict(nx=63, nu=114, nd=88, ne=17)


def test_barcelona_network_collapses(driver):
    net = make_network(**BARCELONA, seed=1)
    tree = make_tree([4, 2, 2, 2] + [1] * 20, seed=2)
    dev = deviation(driver, tree, net.E, np.full(net.nu, 13.0))
    assert dev < 1e-12


def test_uneven_diagonal_weights_collapse(driver):
    net = make_network(16, 29, 22, 4, seed=11)
    tree = make_tree([2, 2, 1, 1, 1, 1], seed=2)
    w = np.random.default_rng(5).uniform(1.0, 100.0, net.nu)
    assert deviation(driver, tree, net.E, w) < 1e-11


def test_no_coupling(driver):
    net = make_network(8, 12, 6, 0, seed=3)
    tree = make_tree([3, 2, 1, 2, 1, 1, 1], seed=9)
    assert deviation(driver, tree, np.zeros((0, net.nu)), np.full(net.nu, 13.0)) < 1e-13


def test_single_scenario_tree(driver):
    net = make_network(8, 14, 6, 3, seed=4)
    tree = make_tree([1] * 6, seed=6)
    assert deviation(driver, tree, net.E, np.full(net.nu, 2.0)) < 1e-12


@pytest.mark.parametrize("scale", [1.0 + 1e-3, 0.9])
def test_scaled_schur_inverse_is_refused_and_matches_numpy(driver, scale):
    """A planted error in S^-1: the check exceeds the tolerance, and its
    value equals an independent numpy evaluation of the same recursion."""
    net = make_network(16, 29, 22, 4, seed=12)
    tree = make_tree([2, 2, 2, 1, 1], seed=3)
    w = np.random.default_rng(7).uniform(5.0, 20.0, net.nu)
    dev = deviation(driver, tree, net.E, w, scale=scale)
    assert dev > 100 * TOL
    ref = numpy_deviation(tree, net.E, w, w, scale)
    assert dev == pytest.approx(ref, rel=1e-8)


def test_schur_complement_of_another_weight_is_refused(driver):
    """S built with a different W_u than the one the kernels divide by."""
    net = make_network(16, 29, 22, 4, seed=13)
    tree = make_tree([2, 2, 1, 1], seed=4)
    w = np.full(net.nu, 13.0)
    wS = w.copy()
    wS[np.flatnonzero(np.abs(net.E).sum(0))[0]] *= 1.5
    dev = deviation(driver, tree, net.E, w, wS=wS)
    assert dev > 100 * TOL
    assert dev == pytest.approx(numpy_deviation(tree, net.E, w, wS, 1.0), rel=1e-8)
