// Per-node factor form of the dual gradient (paper §4.4 and the stage-wise
// products of its GPU design, §5.2): one matrix pair (Phi_nu, K_nu) per
// node, streamed from device memory at every evaluation.  Declarations
// shared by the host factor step (pernode_factor.cpp), the kernels and the
// host driver (pernode.cu) and the C ABI (rapidnet.cu).
#pragma once

#include <cuda_runtime.h>

#include <memory>
#include <vector>

#include "rn_internal.h"

namespace rn {

// Receives the FP64 matrices of node v from the factor step's worker
// threads (each node once; Phi, K: nu x nu, Mc: nu x ne, row-major).
typedef void (*PnSink)(void *ctx, int v, const double *Phi, const double *K, const double *Mc);

// The general recursion on the host (FP64, `threads` worker threads per
// stage); Sd_out (nullable) receives -(E E')^-1 Ed (ne x nd).  RN_OK,
// RN_ERR_RANK (E loses rank), RN_ERR_INVAL (L' Q L not positive definite).
int pn_factor_host(const rn_network *net, const rn_tree *tree, const rn_cost *cost, int threads,
                   PnSink sink, void *ctx, std::vector<double> *Sd_out);

// Validation of network, tree and cost for the per-node form (any A;
// nx, nu <= kPnMaxDim).  RN_OK or an error with the message set.
int pn_validate(const rn_network *net, const rn_tree *tree, const rn_cost *cost);
constexpr int kPnMaxDim = 1024;

// Work items of the persistent kernel: node index with flags.
constexpr int kPnNodeMask = (1 << 26) - 1;
constexpr int kPnK = 1 << 26;      // the item streams K (forward), else Phi (backward)
constexpr int kPnFirst = 1 << 27;  // first node of a chain in this sweep (leaf / head)
constexpr int kPnLast = 1 << 28;   // last node of a chain in this sweep (head / leaf)
constexpr int kPnTop = 1 << 29;    // a node with two or more leaves below it
constexpr int kPnWarps = 4;        // warps of a team

template <typename T>
struct PnParams {
  int nx, nu, n, NXP, NUP, YP, ldm;
  long long mstride;
  const int *anc, *cbeg, *cend;
  const double *prob;
  // shared operators, compressed rows: A, A', B, B', W_u
  const int *Ap, *Ai, *Atp, *Ati, *Bp, *Bi, *Btp, *Bti, *Wp, *Wi;
  const T *Av, *Atv, *Bv, *Btv, *Wv;
  const T *xmin, *xmax, *xs, *umin, *umax;
  T Wx, Ws;
  const T *Phi, *K;            // per node, nu rows of ldm
  const T *c0, *mc, *gd;       // per-solve constants (NUP, NUP, NXP per node)
  const T *x0, *q;             // root state and input (zero when linear)
  T *ya, *yb;                  // dual iterates (YP per node), swapped every iteration
  T *m, *lam, *r, *uo, *xo;    // m (NUP), published sums (NXP, NUP), outputs (NUP, NXP)
  double *uavg, *xavg;         // averaged primal (nullable), NUP / NXP per node
  const double *beta, *theta;  // APG sequences
  unsigned long long *res;     // per check: max |y+ - w| as ordered bits
  unsigned *bar;               // grid barrier counter (residual checks)
  unsigned *nflag;             // per node: backward sums [0, n), forward values [n, 2n)
                               // published for iteration k (value k + 1)
  int *err, *info;             // error word; info: iters, checks, reason, -, stamps
  long long wait_ns;
  double gamma, invgamma, tol;
  int iters, check_every, apg;
  // iterations [it0, it0 + iters) of a solve of iters_total iterations
  // (the APG sequences, the ping-pong of y and the checks count from 0)
  int it0, iters_total;
  // delta form (RN_PREC_MIXED, FP32 handle): y holds the FP32 delta d from
  // the FP64 base yb; the evaluation is linear and x*(w) = x*(yb) + x_lin(dw)
  // with ybh = fl32(yb), uref/xref = x*(yb); swy receives dw at the checks
  int delta;
  const T *ybh, *uref, *xref;
  T *swy;
  // schedule: per team its items, cut into 2 T + 2 segments (chain
  // backward, top backward stage T .. 1, top forward stage 1 .. T, chain
  // forward) at seg[team * (n_seg + 1) + s]
  const int *items, *seg;
  int n_seg, t_top;
  int team_threads, teams;
  // matrix ring of every team: slots of slot_elems T; a matrix is nch
  // column blocks of qw 16-byte units (ldm columns in all)
  int qw, nch, slots, slot_elems, vec_elems;
  // prefetched rows of an item: yc | yp | b1 (max(NUP, NXP)) | b2 (NUP), vb in all
  int b1, vb;
};

// A handle of the per-node form (owned by an rn_factor).
struct PnFactor;
struct PnOptions {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool fp32 = false;         // matrices and iteration in FP32 (else FP64)
  bool mixed = false;        // RN_PREC_MIXED: FP32 delta iterations around an FP64
                             // base, with an FP64 twin handle for the base
  double gamma = 0.0;        // 0: power iteration
  int power_iters = 200, check_every = 10, theta_rule = 0, max_ctas = 0, refresh_every = 20;
  long long wait_ns = 0;
};
int pn_create(const rn_network *net, const rn_tree *tree, const rn_cost *cost,
              const PnOptions &o, PnFactor **out);
void pn_destroy(PnFactor *f);
// device pointers throughout, as rapidnet_solve_device / _dual_gradient_device
int pn_solve_device(PnFactor *f, const double *x0, const double *q, const double *demand,
                    const double *alpha, int max_iters, double tol, const double *y_warm,
                    rn_result *out);
int pn_dual_gradient_device(PnFactor *f, const double *x0, const double *q,
                            const double *demand, const double *alpha, const double *w,
                            double *u, double *x);
void pn_info(const PnFactor *f, rn_factor_info *info);
double pn_gamma(const PnFactor *f);

}  // namespace rn
