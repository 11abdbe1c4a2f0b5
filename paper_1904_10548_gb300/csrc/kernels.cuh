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
//   z   [n][NUP] : F ghat / (2p) of chain nodes (chains longer than a segment)
//   up  [n][SP]  : rows 0..K-1: chain-head subtree sums (lambda | ghat) of
//                  chain k; rows K + v: a group's rows that exceed its
//                  shared-memory capacity
//   ux  [n][SP]  : chain nodes: local path sums (X | U) of the chain;
//                  top nodes: the published (x | Z), Z = sum of z over the path
//   uo, xo       : inputs and states of the last checked iteration
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace rn {

constexpr int kSeg = 16;                    // ints of a team's node list (halved)
constexpr long long kWaitNs = 2000000000LL; // default bound of every device-side wait (2 s)
constexpr int kChildSlotsDev = 8;           // children per node in a group's children table
constexpr int kTcTiles = 4;                 // n-tiles of 8 columns of F a warp keeps (dense W_u)

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
  const T *Erw_val;  // E_rj W^-1_jj, aligned with Er_val
  const int *Ec_ptr, *Ec_idx;
  const T *Ec_val;
  const T *winv;  // diagonal of W_u^{-1}
  const T *Sinv;  // (E W_u^{-1} E')^{-1}, ne x ne
  // dense W_u (null for a diagonal one): F = W^-1 - W^-1 E' S^-1 E W^-1
  // (nu x nu, row-major), its TF32 fragments for the tensor cores (FP32
  // steps, dense_f.cuh) and W^-1 E' S^-1 (nu x ne) for the data terms
  const T *Fd;
  const float4 *Ft;
  const T *Gm;
  const T *xmin, *xmax, *xs, *umin, *umax;
  T Wx, Ws;
};

// the work schedule (rn::Plan) on the device
struct PlanDev {
  int n, n_top, n_chains, n_groups, n_roots;
  int hp_rows;  // rows of partial sums of the parts per step parity (hp holds 2 x hp_rows)
  const int *parent;
  // parts of split stage-1 subtrees: root of each group, its first hp row;
  // roots: node, parts [r_part[2r], r_part[2r+1]), hp rows [r_hp[r], r_hp[r+1])
  const int *g_root, *g_hp, *r_node, *r_part, *r_hp;
  const int *g_node, *g_chain, *g_lvl, *lvl, *g_ccn, *ccn;
  const int *g_desc_ptr, *g_desc;  // per-group descriptors (rn::Plan)
  const int *tc_ptr, *tc, *cc_ptr, *cc;
  const int *ch_start, *ch_len, *ch_group, *ch_parent, *ch_own_ptr, *ch_own;
};

template <typename T>
struct StateDev {
  T *s, *ya, *yb, *ub, *gb, *z, *up, *ux, *uo, *xo;
  T *hp;            // [2][hp_rows][SP]: sums (lambda | ghat) at the top nodes of the parts,
                    // one buffer per parity of the step
  float *uo32, *xo32;  // optional FP32 copies of uo / xo (plain step)
  const T *inv2p;   // 1 / (2 p) per internal node
  const T *xroot;   // x0 (nx); unused when linear
  const double *beta;  // beta_0 .. beta_iters (APG)
  const double *theta; // theta_0 .. theta_iters (APG, the averaged primal)
  double *uavg, *xavg; // averaged primal iterate (internal rows of NUP / NXP),
                       // updated in FP64 by the APG iterations; null = off
  unsigned *count, *flags, *barrier;  // per group: chain arrivals, completion flag; grid
  unsigned *arrive;  // per group that is a part of a split subtree: step + 1 once its sums are out
  unsigned long long *res;  // per check: bits of the non-negative residual
  int *err;                 // 0 ok, else the site of the wait that gave up (1-4)
  int *info;                // [iters done, checks done, stop reason, 0, t_begin, t_end]:
                            // %globaltimer at the start and end of an APG launch as
                            // 64-bit words at info + 4 (8-byte aligned)
  long long wait_ns;        // bound of every device-side wait
};

template <typename T>
struct KParams {
  NetDev<T> net;
  PlanDev plan;
  StateDev<T> st;
  int iters;        // APG iterations (1 for a plain solve step)
  int check_every;
  int linear;       // 1: constants of the dual gradient are zero
  int maxc;         // state components per lane in the dual update: 2, 4 or 8
  int buf_elems;    // work buffer of a team (elements of T)
  int gbuf_elems;   // work buffer of a group (elements of T, the block's two team regions)
  int segb;         // chain rows per backward segment
  int gcap;         // group rows held in shared memory
  int hchunk;       // chain-head rows staged at once by a group
  int fslots;       // staged nodes per warp in the forward sweep (1 to 3)
  int fbrows;       // group rows per batch of the F application
  int tpb;          // chain teams per block
  int team_bytes;   // bytes of one team region
  int net_bytes;    // bytes of the block's shared-memory copy of the network
  unsigned step_base;
  double gamma, invgamma, tol;
};

// Mixed precision (FP32 iteration around an FP64 reference): the dual is
// y = yb + d with the FP64 base yb refreshed every R iterations and the
// FP32 delta d; ybh = fl32(yb) serves the proximal decisions.  The
// primal of the FP32 solve step is x = xref + x_lin(dw), dw = w - yb,
// with xref = x*(yb) computed in FP64 at each refresh.
struct MixedDev {
  double *yb;         // n x YP  FP64 base of the dual
  float *ybh;         // n x YP  fl32(yb)
  float *da, *db;     // n x YP  FP32 deltas (swapped every iteration)
  const float *uref;  // n x NUP inputs of x*(yb)
  const float *xref;  // n x NXP states of x*(yb)
  float *sw;          // n x SP  (dw1 + dw2 | dw3) of the last checked iteration
  double *s64;        // n x SP  FP64 backward input of the refresh step
  int refresh_every;
};

struct MixedParams {
  KParams<float> f;   // FP32 iterations (linear dual gradient on dw)
  KParams<double> d;  // FP64 refresh / final evaluations
  MixedDev mx;
};

cudaError_t launch_mixed(const MixedParams &M, int maxc, int grid, int block, size_t smem,
                         cudaStream_t st);

// Batched mode: independent problems (each a factor handle in mixed
// precision) in one cooperative launch.  Work items are (problem, sub)
// with sub numbered as in the single-problem kernels (groups, then sets
// of tpb chains), sorted by problem; block b processes items
// [cta_begin[b], cta_begin[b+1]).
constexpr int kBatchMaxDistinct = 32;  // problems one block may touch

struct BatchDev {
  int n_problems;
  const MixedParams *probs;  // per problem (device copy; their err words are `err`)
  const int *item_prob, *item_sub, *cta_begin;
  unsigned *barrier;         // grid barrier of the batch
  int *err;                  // shared error word (a wait gave up)
  int *prob_info;            // per problem: iterations, checks, stop reason
  int iters, check_every, refresh_every;
  long long wait_ns;         // bound of every device-side wait
  int net_bytes;             // network region: FP32 copy, then the FP64 header
  int net_bytes_f;           // offset of the FP64 header in the network region
  int team_bytes;            // team region (max over problems)
  int tpb;                   // chain teams per block
  double tol;
};

cudaError_t launch_batch(const BatchDev &B, int maxc, int grid, int block, size_t smem,
                         cudaStream_t st);
cudaError_t batch_occupancy(int maxc, int block, size_t smem, int *blocks_per_sm);
cudaError_t batch_static_smem(int maxc, int *bytes);
cudaError_t mixed_occupancy(int maxc, bool dense, int block, size_t smem, int *blocks_per_sm);

// Shared memory of the persistent kernels.  A block is tpb teams of equal
// width; a team scans one chain, the whole block sums one group.  Dynamic
// shared memory: [block header | network copy | team 0 | team 1 | ...],
// the group work area spanning all team regions.  Buffers in elements
// of T (nw: warps of a team, nwb: of the block):
//   chain backward: segb rows of SP, E/S^-1 work space, 1/(2p), a vector
//   forward: the path vectors x_p | Z_p | B Z_p, then per warp `slots`
//     staged nodes
//   group: gcap rows, hchunk head rows, E/S^-1 work space for fbrows rows,
//     the descriptor
__host__ __device__ inline int round4(int e) { return (e + 3) & ~3; }

__host__ __device__ inline int fwd_elems_per_node(int NXP, int NUP, int YP, int SP, int mode) {
  return SP + (mode == 1 ? 2 * YP : (mode == 2 ? 3 * YP + NUP + NXP : 0));
}

__host__ __device__ inline int chain_vec_off(int segb, int SP, int NEP) {
  return round4(segb * SP) + round4(2 * segb * NEP + segb);
}

__host__ __device__ inline int chain_back_elems(int segb, int SP, int NEP, int NXP, int NUP) {
  return chain_vec_off(segb, SP, NEP) + round4(2 * NXP + NUP);
}

__host__ __device__ inline int fwd_elems(int nw, int slots, int NXP, int NUP, int YP, int SP,
                                         int mode) {
  return round4(2 * NXP + NUP) + nw * slots * fwd_elems_per_node(NXP, NUP, YP, SP, mode);
}

__host__ __device__ inline int group_elems(int gcap, int hchunk, int SP, int NEP, int fbrows,
                                           int desc_elems) {
  return (gcap + hchunk) * SP + round4(2 * fbrows * NEP + fbrows) + desc_elems;
}

constexpr int kHdrBytes = 512;  // block header: reduction words and flags

__host__ __device__ inline size_t round16(size_t b) { return (b + 15) & ~(size_t)15; }

// bytes of a team region holding buf_elems elements of T (plus the team's
// reduction words and node lists)
template <typename T>
inline size_t team_region_bytes(int buf_elems) {
  return round16(sizeof(T) * ((size_t)buf_elems + 72)) + round16((4 + 2 * kSeg) * sizeof(int));
}

// bytes of a block's shared-memory copy of the network data: the NetDev
// header, the sparse index arrays and the values in elements of elem bytes
__host__ __device__ inline size_t net_smem_bytes(int nx, int nu, int ne, int nnzB, int nnzE,
                                                 int elem) {
  const size_t ints = (size_t)(nu + 1) + nnzB + (nx + 1) + nnzB + (ne + 1) + nnzE + (nu + 1) + nnzE;
  const size_t vals = 2 * (size_t)nnzB + 3 * (size_t)nnzE + nu + (size_t)ne * ne + 3 * nx + 2 * nu;
  return round16(sizeof(NetDev<double>)) + round16(ints * 4) + round16(vals * elem);
}

// The kernel translation units (solve_kernels.cu, mixed_kernels.cu,
// batch_kernels.cu) are compiled once per component count C = RN_CVAL in
// {1, 2, 4, 8}, in parallel; each exports its instantiations through these
// functions and dispatch.cu picks one at run time.
#define RN_CAT2(a, b) a##b
#define RN_CAT(a, b) RN_CAT2(a, b)
// work-buffer sizes of one precision in one kernel's shared-memory layout
struct Sizes {
  int team_bytes = 0, net_bytes = 0;  // layout of the block
  int buf = 0, gbuf = 0, segb = 1, gcap = 0, hchunk = 1, fslots = 1, fbrows = 1, tpb = 2;
};
// padded row lengths of a factor's network (elements)
struct RowDims {
  int NXP, NUP, YP, SP, NEP;
};
// host layout rules (layout.cpp)
struct Plan;
int layout_sizes(const Plan &p, const RowDims &f, int eb, int team_bytes, int net_bytes, int tw,
                 int tpb, int mode, Sizes *z);
int team_layout(int block_threads, int nx, int nu, int *tw_out, int *tpb_out, int *maxc_out);
int team_bytes_for(int sms, int optin, int per_sm, int reserved, int n_items, int tpb, int block,
                   int net_bytes, int static_smem, int *team_bytes, int *blocks_per_sm);
int check_layout(const Plan &p, const Sizes &z, int n_items, int grid, const char *what);

#define RN_DECLARE_KERNELS(c)                          \
  const void *RN_CAT(solve_kernel_c, c##_d0)(bool apg); \
  const void *RN_CAT(solve_kernel_c, c##_d1)(bool apg); \
  const void *RN_CAT(mixed_kernel_c, c##_d0)();         \
  const void *RN_CAT(mixed_kernel_c, c##_d1)();         \
  const void *RN_CAT(batch_kernel_c, c)();
RN_DECLARE_KERNELS(1)
RN_DECLARE_KERNELS(2)
RN_DECLARE_KERNELS(4)
RN_DECLARE_KERNELS(8)

// Raise a kernel's dynamic shared-memory limit to the device's opt-in
// maximum, once per kernel: launches then use what they need.  Changing
// the attribute between launches of a kernel that is running on another
// stream would serialise the two.
cudaError_t allow_max_smem(const void *fn);

// host launchers of the persistent kernel (cooperative launch: every block
// must be resident because blocks wait on flags that other blocks set)
template <typename T, bool APG>
cudaError_t launch_solve(const KParams<T> &P, int grid, int block, size_t smem, cudaStream_t st);
template <typename T, bool APG>
cudaError_t solve_occupancy(int maxc, bool dense, int block, size_t smem, int *blocks_per_sm);

}  // namespace rn
