// Internal declarations shared by the host and device translation units.
#pragma once

#include <cstdarg>
#include <string>
#include <vector>

#include "rapidnet.h"

namespace rn {

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
// (eq. dual-gradient evaluated by the recursion of §4.4), so a chain is
// processed sequentially by one thread block, and top nodes are reduced
// by whichever block completes their last child.
//
// Internal node order: 0 = root, then the top nodes in breadth-first
// order (internal 1..n_top), then the chains one after another, each
// from head to leaf.  Chains are ordered by their leaf; all leaves are at
// stage N, so the chains below any node form a contiguous range.
struct Plan {
  int n = 0, N = 0, n_top = 0, n_chains = 0, max_chain_len = 0, max_path_len = 0;
  int n_flags = 0;
  std::vector<int> perm;     // internal -> breadth-first index
  std::vector<int> iperm;    // breadth-first -> internal
  std::vector<int> parent;   // internal parent index (-1 for the root)
  std::vector<double> prob;  // internal order
  // top nodes, indexed by internal index (entries for non-top nodes unused)
  std::vector<int> top_nchild, top_child_ptr, top_child, top_flag;
  // chains
  std::vector<int> ch_start, ch_len, ch_parent, ch_path_ptr, ch_path, ch_own_from, ch_flag;
};

// Validates the tree (see rn_tree) and builds the schedule.  Returns
// RN_OK or RN_ERR_INVAL with the error message set.
int build_plan(const rn_tree *tree, Plan &plan);

}  // namespace rn
