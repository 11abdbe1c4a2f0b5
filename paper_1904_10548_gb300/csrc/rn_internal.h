// Internal declarations shared by the host and device translation units.
#pragma once

#include <cstdarg>
#include <string>
#include <vector>

#include "rapidnet.h"

namespace rn {

constexpr int kChildSlots = 8;  // children per node in a group's children table
constexpr int kSplitAbove = 24; // a stage-1 subtree with more top nodes is split

// thread-local error message behind rapidnet_last_error()
void set_error(const char *fmt, ...);
void clear_error();

// Compressed sparse rows of a dense row-major matrix (exact zeros dropped).
struct Csr {
  std::vector<int> ptr, idx;
  std::vector<double> val;
};
Csr dense_to_csr(const double *M, int rows, int cols);
Csr dense_to_csc(const double *M, int rows, int cols);  // "rows" of the result = columns of M

// Work schedule over the scenario tree.
//
// A node whose subtree holds exactly one leaf lies on a *chain*: the path
// from the highest such node (the chain head) down to its leaf.  Every
// other non-root node is a *top* node (two or more leaves below it).  The
// dual gradient is a subtree sum going up and a path sum going down
// (eq. dual-gradient evaluated by the recursion of §4.4).  A chain is
// scanned by one team of threads.  The top nodes below one stage-1 node
// form a *group* (the stage-1 subtrees are independent given x0): one
// thread block sums the group level by level from the chain-head sums,
// applies F, rolls the path sums back down and publishes them; the chain
// below each top node that comes first in chain order (its *owner*)
// performs that node's per-node step.
//
// Internal node order: 0 = root, then the top nodes group by group, each
// group in breadth-first order (so its levels are contiguous ranges),
// then the chains one after another, each from head to leaf.  Chains are
// ordered by their leaf; all leaves are at stage N, so the chains below
// any node form a contiguous range.
struct Plan {
  int n = 0, N = 0, n_top = 0, n_chains = 0, n_groups = 0, max_chain_len = 0;
  int max_group = 0, max_group_chains = 0, n_roots = 0, max_root_children = 0, hp_rows = 0;
  std::vector<int> perm;     // internal -> breadth-first index
  std::vector<int> iperm;    // breadth-first -> internal
  std::vector<int> parent;   // internal parent index (-1 for the root)
  std::vector<double> prob;  // internal order
  // groups: top nodes [g_node[g], g_node[g+1]), chains [g_chain[2g],
  // g_chain[2g+1]), level boundaries lvl[g_lvl[g]] .. lvl[g_lvl[g+1] - 1]
  std::vector<int> g_node, g_chain, g_lvl, lvl;
  // per group its root (-1 unless the group is a part of a split stage-1
  // subtree) and the first hp row of its top nodes' sums; roots: internal
  // node r_node[r], parts [r_part[2r], r_part[2r+1]), the sums of its
  // children in hp rows [r_hp[r], r_hp[r+1]); hp row r_hp[n_roots] + r
  // holds root r's own backward input (hp_rows counts both kinds)
  std::vector<int> g_root, g_hp, r_node, r_part, r_hp;
  // per group the top nodes with chain children: ccn[g_ccn[g] .. g_ccn[g+1])
  std::vector<int> g_ccn, ccn;
  // per group a compact descriptor in local indices (li = internal - g_node[g],
  // chain positions relative to g_chain[2g]), at g_desc[g_desc_ptr[g]],
  // padded to a multiple of 4 ints:
  //   m, nl, nch, ncn | lvl[nl + 1] | par[m] (-1: the root) |
  //   tcp[m + 1], tcl[..] (top children) | ccp[m + 1], ccl[..] (chain children) |
  //   cn[ncn] (the nodes with chain children) | pad to 4 | tab, fits, 0, 0 |
  //   children table at desc + tab: per node kChildSlots entries, chain heads
  //   first (-2 - head position), then top children (local index), -1 none;
  //   fits = 0 when some node has more children (the lists are used then)
  std::vector<int> g_desc_ptr, g_desc;
  int max_desc = 0;
  // top nodes (indexed by internal index 0..n_top): top children and
  // chain children (chain ids)
  std::vector<int> tc_ptr, tc, cc_ptr, cc;
  // chains: first node, length, group (-1 below the root), parent, owned
  // top nodes [ch_own_ptr[k], ch_own_ptr[k+1]) from stage 1 down
  std::vector<int> ch_start, ch_len, ch_group, ch_parent, ch_own_ptr, ch_own;
};

// Validates the tree (see rn_tree) and builds the schedule with at most
// max_groups groups where a split is possible (at least one group per
// stage-1 subtree).  Returns RN_OK or RN_ERR_INVAL with the error message
// set.
int build_plan(const rn_tree *tree, Plan &plan, int max_groups = 1 << 30);

// Dense FP64 helpers of the factor step (factor_check.cpp).  cholesky:
// A = R R' of an SPD m x m matrix in place (lower); false if a pivot is
// not positive relative to the diagonal scale.  chol_inverse: the inverse
// from that factor.
bool cholesky(std::vector<double> &A, int m);
std::vector<double> chol_inverse(const std::vector<double> &R, int m);

// Largest relative deviation max|2 p Phi - F| / max|F| of one step of the
// general per-node recursion (paper §4.4) from the shared operator
// F = W^-1 - W^-1 E' S^-1 E W^-1, at the first node of stages 1, N/2 and N,
// with the children's P_c formed from F.  E: ne x nu row-major; winv: the
// diagonal of W_u^-1; Sinv: (E W^-1 E')^-1, ne x ne.  Infinity if L' Q L is
// not positive definite or E' loses rank.
double collapse_deviation(const rn_tree *tree, int nu, int ne, const double *E,
                          const double *winv, const double *Sinv);
// The same for a dense W_u (nu x nu) and the dense F (nu x nu) the factor
// step computed from it.
double collapse_deviation_dense(const rn_tree *tree, int nu, int ne, const double *E,
                                const double *W, const double *F);
constexpr double kCollapseTol = 1e-8;

}  // namespace rn
