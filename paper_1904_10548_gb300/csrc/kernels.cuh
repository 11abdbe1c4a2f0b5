// Device-side data of a factor handle and the persistent solve kernel.
//
// Layout in HBM (internal node order, see rn::Plan), row-major per node,
// every row padded to a multiple of 4 elements so that rows start on
// 16-byte boundaries in FP32 and FP64 alike:
//   s   [n][SP]  SP = NXP + NUP : backward input (w1 + w2 | w3)
//   ya, yb [n][YP] YP = 2 NXP + NUP : dual iterates y^nu, y^{nu-1}
//                                      (y1 | y2 | y3), swapped every iteration
//   ub  [n][NUP] : input offset u0 = x*(0) inputs (or ubar + K q at preparation)
//   gb  [n][NXP] : Gd d
//   z   [n][NUP] : F ghat / (2p) of the current dual-gradient evaluation
//   up  [n][SP]  : subtree sums (lambda | ghat) handed from a node to its parent
//   uo, xo       : inputs and states of the last checked iteration
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace rn {

constexpr int kSeg = 16;                    // chain nodes held in shared memory at once
constexpr long long kWaitNs = 2000000000LL; // bound of every device-side wait (2 s)

template <typename T>
struct NetDev {
  int nx, nu, ne, nd, NXP, NUP, SP, YP, NEP;
  // B by columns (flow j -> tanks) and by rows (tank i -> flows)
  const int *Bc_ptr, *Bc_idx;
  const T *Bc_val;
  const int *Br_ptr, *Br_idx;
  const T *Br_val;
  // E by rows (mixing node r -> flows) and by columns (flow j -> mixing nodes)
  const int *Er_ptr, *Er_idx;
  const T *Er_val;
  const int *Ec_ptr, *Ec_idx;
  const T *Ec_val;
  const T *winv;  // diagonal of W_u^{-1}
  const T *Sinv;  // (E W_u^{-1} E')^{-1}, ne x ne
  const T *xmin, *xmax, *xs, *umin, *umax;
  T Wx, Ws;
};

struct PlanDev {
  int n, n_top, n_chains, n_flags;
  const int *parent, *top_nchild, *top_child_ptr, *top_child, *top_flag;
  const int *ch_start, *ch_len, *ch_parent, *ch_path_ptr, *ch_path, *ch_own_from, *ch_flag;
};

template <typename T>
struct StateDev {
  T *s, *ya, *yb, *ub, *gb, *z, *up, *uo, *xo;
  const T *inv2p;   // 1 / (2 p) per internal node
  const T *xroot;   // x0 (nx); unused when linear
  const double *beta;  // beta_0 .. beta_iters (APG)
  unsigned *count, *flags, *barrier;
  unsigned long long *res;  // per check: bits of the non-negative residual
  int *err;                 // 0 ok, 1 timeout
  int *info;                // [iters done, checks done, stop reason]
};

template <typename T>
struct KParams {
  NetDev<T> net;
  PlanDev plan;
  StateDev<T> st;
  int iters;        // APG iterations (1 for a plain solve step)
  int check_every;
  int linear;       // 1: constants of the dual gradient are zero
  unsigned step_base;
  double gamma, invgamma, tol;
};

// dynamic shared memory of the persistent kernel (layout in solve_kernels.cu)
template <typename T>
inline size_t smem_bytes(int SP, int NEP, int NUP) {
  size_t b = sizeof(T) * ((size_t)kSeg * SP + 2 * (size_t)kSeg * NEP + kSeg + NUP + 72);
  b = (b + 15) & ~(size_t)15;
  return b + 40 * sizeof(unsigned long long) + 4 * sizeof(int);
}

// host launchers of the persistent kernel (cooperative launch: every block
// must be resident because blocks wait on flags that other blocks set)
template <typename T, bool APG>
cudaError_t launch_solve(const KParams<T> &P, int grid, int block, size_t smem, cudaStream_t st);
template <typename T, bool APG>
cudaError_t solve_occupancy(int block, size_t smem, int *blocks_per_sm);

}  // namespace rn
