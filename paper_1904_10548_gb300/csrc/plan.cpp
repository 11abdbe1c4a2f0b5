// Host-side validation of the scenario tree (paper §2.3) and the work
// schedule of the dual-gradient recursion (see rn::Plan).
#include <algorithm>
#include <cmath>
#include <cstdio>

#include "rn_internal.h"

namespace rn {

static thread_local std::string g_err;

void set_error(const char *fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
}
void clear_error() { g_err.clear(); }

Csr dense_to_csr(const double *M, int rows, int cols) {
  Csr c;
  c.ptr.assign(rows + 1, 0);
  for (int r = 0; r < rows; ++r) {
    for (int k = 0; k < cols; ++k) {
      double v = M[(size_t)r * cols + k];
      if (v != 0.0) {
        c.idx.push_back(k);
        c.val.push_back(v);
      }
    }
    c.ptr[r + 1] = (int)c.idx.size();
  }
  return c;
}

Csr dense_to_csc(const double *M, int rows, int cols) {
  Csr c;
  c.ptr.assign(cols + 1, 0);
  for (int k = 0; k < cols; ++k) {
    for (int r = 0; r < rows; ++r) {
      double v = M[(size_t)r * cols + k];
      if (v != 0.0) {
        c.idx.push_back(r);
        c.val.push_back(v);
      }
    }
    c.ptr[k + 1] = (int)c.idx.size();
  }
  return c;
}

int build_plan(const rn_tree *t, Plan &p, int max_groups) {
  if (!t || !t->stage_ptr || !t->anc || !t->prob) {
    set_error("tree: NULL pointer");
    return RN_ERR_INVAL;
  }
  const int N = t->N, n = t->n_nodes;
  if (N < 1 || n < 2) {
    set_error("tree: need N >= 1 and n_nodes >= 2 (got N=%d, n_nodes=%d)", N, n);
    return RN_ERR_INVAL;
  }
  const int *sp = t->stage_ptr;
  if (sp[0] != 0 || sp[1] != 1 || sp[N + 1] != n) {
    set_error("tree: stage_ptr must start 0, 1 and end at n_nodes");
    return RN_ERR_INVAL;
  }
  for (int s = 0; s <= N; ++s)
    if (sp[s + 1] <= sp[s]) {
      set_error("tree: stage %d is empty", s);
      return RN_ERR_INVAL;
    }
  if (t->anc[0] != -1) {
    set_error("tree: anc[0] must be -1");
    return RN_ERR_INVAL;
  }
  if (!(std::fabs(t->prob[0] - 1.0) <= 1e-9)) {
    set_error("tree: prob[0] must be 1");
    return RN_ERR_INVAL;
  }
  std::vector<int> first_child(n, -1), nchild(n, 0), stage(n, 0);
  for (int s = 1; s <= N; ++s) {
    int prev = -1;
    for (int v = sp[s]; v < sp[s + 1]; ++v) {
      int a = t->anc[v];
      stage[v] = s;
      if (a < sp[s - 1] || a >= sp[s]) {
        set_error("tree: anc[%d]=%d is not a node of stage %d", v, a, s - 1);
        return RN_ERR_INVAL;
      }
      if (a < prev) {
        set_error("tree: children must be contiguous and in parent order (node %d)", v);
        return RN_ERR_INVAL;
      }
      if (!(t->prob[v] > 0.0) || !std::isfinite(t->prob[v])) {
        set_error("tree: prob[%d] must be positive and finite", v);
        return RN_ERR_INVAL;
      }
      if (a != prev) first_child[a] = v;
      prev = a;
      nchild[a]++;
    }
  }
  for (int v = 0; v < sp[N]; ++v)
    if (nchild[v] == 0) {
      set_error("tree: node %d at stage %d < N has no child (all leaves must be at stage N)",
                v, stage[v]);
      return RN_ERR_INVAL;
    }
  for (int v = 0; v < sp[N]; ++v) {
    double sum = 0.0;
    for (int c = first_child[v]; c < first_child[v] + nchild[v]; ++c) sum += t->prob[c];
    if (std::fabs(sum - t->prob[v]) > 1e-9 * t->prob[v]) {
      set_error("tree: children of node %d have probability %.17g, parent %.17g", v, sum,
                t->prob[v]);
      return RN_ERR_INVAL;
    }
  }

  // leaves below every node
  std::vector<int> leaves(n, 0);
  for (int v = n - 1; v >= 0; --v) {
    if (nchild[v] == 0) leaves[v] = 1;
    if (v > 0) leaves[t->anc[v]] += leaves[v];
  }

  p = Plan();
  p.n = n;
  p.N = N;
  p.perm.assign(n, -1);
  p.iperm.assign(n, -1);
  p.perm[0] = 0;
  p.iperm[0] = 0;
  int next = 1;
  // groups: breadth-first over the top nodes below each stage-1 top node.
  // A large stage-1 subtree whose stage-1 node has two or more top children
  // and no chain child is split: its top children are bundled into parts
  // (as many as max_groups leaves room for), each part a group, and the
  // stage-1 node becomes a *root*, summed by the last of its parts to
  // finish; roots follow all groups in the internal order.
  p.g_node.push_back(1);
  p.g_lvl.push_back(0);
  std::vector<int> group_of(n, -1), root_orig;
  auto add_group = [&](const std::vector<int> &tops, int root, int hp0) {
    const int g = p.n_groups++;
    p.g_root.push_back(root);
    p.g_hp.push_back(hp0);
    std::vector<int> level = tops;
    while (!level.empty()) {
      p.lvl.push_back(next);
      std::vector<int> below;
      for (int v : level) {
        p.perm[next] = v;
        p.iperm[v] = next++;
        group_of[v] = g;
        for (int c = first_child[v]; c < first_child[v] + nchild[v]; ++c)
          if (leaves[c] >= 2) below.push_back(c);
      }
      level.swap(below);
    }
    p.lvl.push_back(next);
    p.g_lvl.push_back((int)p.lvl.size());
    p.g_node.push_back(next);
    p.max_group = std::max(p.max_group, p.g_node[g + 1] - p.g_node[g]);
  };
  std::vector<int> subtree_top(n, 0);  // top nodes in each subtree
  for (int v = n - 1; v >= 1; --v) {
    if (leaves[v] >= 2) subtree_top[v] += 1;
    if (t->anc[v] > 0) subtree_top[t->anc[v]] += subtree_top[v];
  }
  std::vector<int> stage1, splittable;
  for (int b1 = sp[1]; b1 < sp[2]; ++b1) {
    if (leaves[b1] < 2) continue;
    stage1.push_back(b1);
    int tops = 0, chains = 0;
    for (int c = first_child[b1]; c < first_child[b1] + nchild[b1]; ++c) (leaves[c] >= 2 ? tops : chains)++;
    if (tops >= 2 && chains == 0 && subtree_top[b1] > kSplitAbove) splittable.push_back(b1);
  }
  const long long extra = (long long)max_groups - (long long)stage1.size();
  const int parts_each = splittable.empty() || extra <= 0
                             ? 1
                             : (int)std::min<long long>(1 + extra / (long long)splittable.size(), 1 << 20);
  int hp_rows = 0;
  for (int b1 : stage1) {
    std::vector<int> tops;
    for (int c = first_child[b1]; c < first_child[b1] + nchild[b1]; ++c)
      if (leaves[c] >= 2) tops.push_back(c);
    const bool split = parts_each >= 2 &&
                       std::find(splittable.begin(), splittable.end(), b1) != splittable.end();
    if (!split) {
      add_group({b1}, -1, -1);
      continue;
    }
    const int r = (int)root_orig.size(), nt = (int)tops.size();
    const int ns = std::min(nt, parts_each);
    root_orig.push_back(b1);
    p.r_part.push_back(p.n_groups);  // [begin, end) of the root's parts
    p.r_hp.push_back(hp_rows);
    for (int q = 0, c0 = 0; q < ns; ++q) {  // contiguous bundles, sizes differ by one at most
      const int cnt = nt / ns + (q < nt % ns ? 1 : 0);
      add_group(std::vector<int>(tops.begin() + c0, tops.begin() + c0 + cnt), r, hp_rows + c0);
      c0 += cnt;
    }
    p.r_part.push_back(p.n_groups);
    hp_rows += nt;
  }
  p.n_roots = (int)root_orig.size();
  p.r_hp.push_back(hp_rows);
  // one more row per root after the children's sums: a copy of the root's
  // own backward input, taken by its first part before it arrives
  p.hp_rows = hp_rows + p.n_roots;
  for (int b1 : root_orig) {
    p.perm[next] = b1;
    p.iperm[b1] = next;
    p.r_node.push_back(next++);
  }
  for (int r = 0; r < p.n_roots; ++r)
    p.max_root_children = std::max(p.max_root_children, p.r_hp[r + 1] - p.r_hp[r]);
  if (p.r_part.empty()) p.r_part.assign(2, 0);
  p.n_top = next - 1;
  // chains, ordered by their leaf (all leaves are at stage N, so this
  // keeps the chains below any node contiguous)
  std::vector<int> head_chain(n, -1);
  for (int leaf = sp[N]; leaf < n; ++leaf) {
    int head = leaf;
    while (t->anc[head] != 0 && leaves[t->anc[head]] == 1) head = t->anc[head];
    head_chain[head] = (int)p.ch_start.size();
    p.ch_start.push_back(next);
    int len = 0;
    for (int w = head;; w = first_child[w]) {
      p.perm[next] = w;
      p.iperm[w] = next++;
      ++len;
      if (nchild[w] == 0) break;
    }
    p.ch_len.push_back(len);
    p.max_chain_len = std::max(p.max_chain_len, len);
  }
  p.n_chains = (int)p.ch_start.size();
  if (next != n) {
    set_error("tree: internal error in the chain decomposition");
    return RN_ERR_INVAL;
  }
  p.parent.assign(n, -1);
  p.prob.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    int b = p.perm[i];
    p.prob[i] = t->prob[b];
    if (b > 0) p.parent[i] = p.iperm[t->anc[b]];
  }
  // children of the top nodes: top children (internal) and chain children
  p.tc_ptr.assign(p.n_top + 2, 0);
  p.cc_ptr.assign(p.n_top + 2, 0);
  for (int i = 0; i <= p.n_top; ++i) {
    p.tc_ptr[i + 1] = p.tc_ptr[i];
    p.cc_ptr[i + 1] = p.cc_ptr[i];
    if (i == 0) continue;
    const int b = p.perm[i];
    for (int c = first_child[b]; c < first_child[b] + nchild[b]; ++c) {
      if (leaves[c] >= 2) {
        p.tc.push_back(p.iperm[c]);
        p.tc_ptr[i + 1]++;
      } else {
        p.cc.push_back(head_chain[c]);
        p.cc_ptr[i + 1]++;
      }
    }
  }
  p.g_ccn.assign(1, 0);
  for (int g = 0; g < p.n_groups; ++g) {
    for (int v = p.g_node[g]; v < p.g_node[g + 1]; ++v)
      if (p.cc_ptr[v + 1] > p.cc_ptr[v]) p.ccn.push_back(v);
    p.g_ccn.push_back((int)p.ccn.size());
  }
  // chains: group, parent, owned top nodes (the first chain below a top
  // node owns it; owned ancestors form a suffix of the path from stage 1)
  std::vector<int> owner(n, -1);
  p.ch_own_ptr.assign(1, 0);
  p.g_chain.assign(2 * (size_t)p.n_groups, -1);
  for (int k = 0; k < p.n_chains; ++k) {
    const int head = p.ch_start[k];
    const int par = p.parent[head];
    p.ch_parent.push_back(par);
    std::vector<int> path;
    for (int a = par; a > 0; a = p.parent[a]) path.push_back(a);
    std::reverse(path.begin(), path.end());
    const int g = par > 0 ? group_of[p.perm[par]] : -1;
    if (par > 0 && g < 0) {
      set_error("tree: internal error, chain below a root");
      return RN_ERR_INVAL;
    }
    p.ch_group.push_back(g);
    if (g >= 0) {
      if (p.g_chain[2 * g] < 0) p.g_chain[2 * g] = k;
      if (p.g_chain[2 * g + 1] >= 0 && p.g_chain[2 * g + 1] != k) {
        set_error("tree: internal error, chains of a group are not contiguous");
        return RN_ERR_INVAL;
      }
      p.g_chain[2 * g + 1] = k + 1;
    }
    bool owning = false;
    for (int a : path) {
      if (owner[a] < 0) {
        owner[a] = k;
        owning = true;
        p.ch_own.push_back(a);
      } else if (owning) {
        set_error("tree: internal error in the ownership of top nodes");
        return RN_ERR_INVAL;
      }
    }
    p.ch_own_ptr.push_back((int)p.ch_own.size());
  }
  for (int g = 0; g < p.n_groups; ++g)
    p.max_group_chains = std::max(p.max_group_chains, p.g_chain[2 * g + 1] - p.g_chain[2 * g]);
  p.g_desc_ptr.assign(1, 0);
  for (int g = 0; g < p.n_groups; ++g) {
    const int g0 = p.g_node[g], m = p.g_node[g + 1] - g0, c0 = p.g_chain[2 * g];
    const int l0 = p.g_lvl[g], nl = p.g_lvl[g + 1] - l0 - 1;
    std::vector<int> d{m, nl, p.g_chain[2 * g + 1] - c0, 0};
    for (int l = 0; l <= nl; ++l) d.push_back(p.lvl[l0 + l] - g0);
    for (int li = 0; li < m; ++li) {
      const int pa = p.parent[g0 + li];
      d.push_back(pa >= g0 && pa < g0 + m ? pa - g0 : -1);  // -1: the tree root or the group's root
    }
    int acc = 0;
    for (int li = 0; li <= m; ++li) {
      d.push_back(acc);
      if (li < m) acc += p.tc_ptr[g0 + li + 1] - p.tc_ptr[g0 + li];
    }
    for (int li = 0; li < m; ++li)
      for (int c = p.tc_ptr[g0 + li]; c < p.tc_ptr[g0 + li + 1]; ++c) d.push_back(p.tc[c] - g0);
    acc = 0;
    for (int li = 0; li <= m; ++li) {
      d.push_back(acc);
      if (li < m) acc += p.cc_ptr[g0 + li + 1] - p.cc_ptr[g0 + li];
    }
    for (int li = 0; li < m; ++li)
      for (int c = p.cc_ptr[g0 + li]; c < p.cc_ptr[g0 + li + 1]; ++c) d.push_back(p.cc[c] - c0);
    int ncn = 0;
    for (int li = 0; li < m; ++li) ncn += p.cc_ptr[g0 + li + 1] > p.cc_ptr[g0 + li];
    d[3] = ncn;
    for (int li = 0; li < m; ++li)
      if (p.cc_ptr[g0 + li + 1] > p.cc_ptr[g0 + li]) d.push_back(li);
    // children table (16-byte aligned): per node kChildSlots entries, chain
    // heads first (-2 - head position), then top children (local index),
    // -1 for none; a node with more children makes the whole group use
    // the lists above instead (flag in the word after the table offset)
    while (d.size() % 4) d.push_back(0);
    const int tab = (int)d.size() + 4;
    bool fits = true;
    for (int li = 0; li < m; ++li) {
      const int nc = (p.cc_ptr[g0 + li + 1] - p.cc_ptr[g0 + li]) + (p.tc_ptr[g0 + li + 1] - p.tc_ptr[g0 + li]);
      if (nc > kChildSlots) fits = false;
    }
    d.push_back(tab);
    d.push_back(fits ? 1 : 0);
    d.push_back(0);
    d.push_back(0);
    for (int li = 0; li < m; ++li) {
      int k = 0;
      for (int c = p.cc_ptr[g0 + li]; c < p.cc_ptr[g0 + li + 1] && k < kChildSlots; ++c, ++k)
        d.push_back(-2 - (p.cc[c] - c0));
      for (int c = p.tc_ptr[g0 + li]; c < p.tc_ptr[g0 + li + 1] && k < kChildSlots; ++c, ++k)
        d.push_back(p.tc[c] - g0);
      for (; k < kChildSlots; ++k) d.push_back(-1);
    }
    p.max_desc = std::max(p.max_desc, (int)d.size());
    p.g_desc.insert(p.g_desc.end(), d.begin(), d.end());
    p.g_desc_ptr.push_back((int)p.g_desc.size());
  }
  if (p.g_desc.empty()) p.g_desc.assign(4, 0);
  for (int i = 1; i <= p.n_top; ++i)
    if (owner[i] < 0) {
      set_error("tree: internal error, top node without a chain");
      return RN_ERR_INVAL;
    }
  return RN_OK;
}

}  // namespace rn

extern "C" const char *rapidnet_last_error(void) { return rn::g_err.c_str(); }
