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

int build_plan(const rn_tree *t, Plan &p) {
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
  for (int v = 1; v < n; ++v)
    if (leaves[v] >= 2) {
      p.perm[next] = v;
      p.iperm[v] = next++;
    }
  p.n_top = next - 1;
  // chains, ordered by their leaf (all leaves are at stage N, so this
  // keeps the chains below any node contiguous)
  for (int leaf = sp[N]; leaf < n; ++leaf) {
    int head = leaf;
    while (t->anc[head] != 0 && leaves[t->anc[head]] == 1) head = t->anc[head];
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
  // top nodes: children lists in breadth-first order, flags at stage 1
  p.top_nchild.assign(n, 0);
  p.top_child_ptr.assign(n + 1, 0);
  p.top_flag.assign(n, -1);
  for (int i = 1; i <= p.n_top; ++i) {
    int b = p.perm[i];
    p.top_nchild[i] = nchild[b];
    if (stage[b] == 1) p.top_flag[i] = p.n_flags++;
  }
  for (int i = 0; i < n; ++i) {
    p.top_child_ptr[i + 1] = p.top_child_ptr[i];
    if (i >= 1 && i <= p.n_top) {
      int b = p.perm[i];
      for (int c = first_child[b]; c < first_child[b] + nchild[b]; ++c)
        p.top_child.push_back(p.iperm[c]);
      p.top_child_ptr[i + 1] = (int)p.top_child.size();
    }
  }
  // chain paths (top ancestors from stage 1 down) and ownership: the
  // first chain below a top node computes that node's proximal step
  std::vector<int> owner(n, -1);
  p.ch_path_ptr.assign(1, 0);
  for (int k = 0; k < p.n_chains; ++k) {
    int head = p.ch_start[k];
    p.ch_parent.push_back(p.parent[head]);
    std::vector<int> path;
    for (int a = p.parent[head]; a > 0; a = p.parent[a]) path.push_back(a);
    std::reverse(path.begin(), path.end());
    int own_from = (int)path.size();
    for (int j = 0; j < (int)path.size(); ++j)
      if (owner[path[j]] < 0) {
        owner[path[j]] = k;
        own_from = std::min(own_from, j);
      }
    // owned ancestors form a suffix of the path
    for (int j = own_from; j < (int)path.size(); ++j)
      if (owner[path[j]] != k) {
        set_error("tree: internal error in the ownership of top nodes");
        return RN_ERR_INVAL;
      }
    p.ch_own_from.push_back(own_from);
    p.ch_flag.push_back(path.empty() ? -1 : p.top_flag[path[0]]);
    p.max_path_len = std::max(p.max_path_len, (int)path.size());
    for (int a : path) p.ch_path.push_back(a);
    p.ch_path_ptr.push_back((int)p.ch_path.size());
  }
  for (int i = 1; i <= p.n_top; ++i)
    if (owner[i] < 0) {
      set_error("tree: internal error, top node without a chain");
      return RN_ERR_INVAL;
    }
  return RN_OK;
}

}  // namespace rn

extern "C" const char *rapidnet_last_error(void) { return rn::g_err.c_str(); }
