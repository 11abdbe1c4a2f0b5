// Persistent kernel of the dual APG iteration on a scenario tree
// (paper §4.3 eqs. apg:1 / apg:2, dual gradient by the tree recursion of
// §4.4) and the small kernels around it.
//
// The dual gradient x*(w) = grad f*(-H'w) (eq. dual-gradient) is computed
// in the form that the general Riccati recursion takes when A = I: with
// F = W^-1 - W^-1 E'(E W^-1 E')^-1 E W^-1 shared by all nodes,
//   lambda_nu = sum over subtree(nu) of (w1 + w2)
//   ghat_nu   = sum over subtree(nu) of (w3 + B' lambda)      (+ c0 at preparation)
//   z_nu      = F ghat_nu / (2 p_nu)
//   u_nu      = ub_nu - sum over path(root -> nu) of z
//   x_nu      = x_a(nu) + B u_nu + Gd d_nu
// where ub = x*(0)'s inputs carries all data terms (c0, the particular
// solution of E u + Ed d = 0 and the projection of q).  The backward sweep
// is a subtree sum and the forward sweep a path sum, so there is no
// dependent matrix product along the tree: each chain (single-leaf path)
// is scanned by a team of threads, the top nodes below each stage-1 node
// (a group) are summed, rolled back down and published by one block, and
// each chain turns the published path sums of its parent into its own by
// an elementwise correction of its precomputed local sums.
#include "solve_device.cuh"

namespace rn {

// ---------------------------------------------------------------------------
// the persistent kernel: `iters` APG iterations (APG = true) or one
// evaluation of the dual gradient (APG = false)
// ---------------------------------------------------------------------------
namespace RN_CAT(kv, RN_DENSE) {  // one kernel per (C, W_u diagonal or dense)

template <typename T, bool APG, int C>
__global__ void __launch_bounds__(512) k_solve(KParams<T> P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (APG && blockIdx.x == 0 && threadIdx.x == 0) stamp_time(P.st.info, 0);
  const BlockMem bm = block_mem(smem_raw, P.net_bytes, P.team_bytes);
  const NetDev<T> *net = stage_net(P.net, bm.net_raw);
  const Team tc = chain_team(P.tpb), tb = block_team();
  const Smem<T> smc = carve<T>(bm.team_raw(team_index(P.tpb)), P.buf_elems, net);
  const Smem<T> smg = carve<T>(bm.team_raw(0), P.gbuf_elems, net);
  const int G = P.plan.n_groups, n_items = G + (P.plan.n_chains + P.tpb - 1) / P.tpb;
  const bool keep = (int)gridDim.x >= n_items && (int)blockIdx.x >= G;
  int it = 0, ci = 0, reason = 0;  // reason: 0 max iters, 1 converged, 2 non-finite, 3 timeout
  for (; it < P.iters; ++it) {
    const unsigned step = P.step_base + (unsigned)it;
    FwdCtx<T> c;
    c.ycur = (it & 1) ? P.st.yb : P.st.ya;
    c.yprv = (it & 1) ? P.st.ya : P.st.yb;
    c.beta = APG ? (T)P.st.beta[it] : T(0);
    c.beta_n = APG ? (T)P.st.beta[it + 1] : T(0);
    const bool check = APG && (((it + 1) % P.check_every) == 0 || it + 1 == P.iters);
    c.write_out = !APG || check;
    c.avg = APG && P.st.uavg != nullptr;
    c.theta = APG ? P.st.theta[it] : 0.0;
    c.rbits = 0ull;
    eval_step<T, APG ? kFwdApg : kFwdPlain, C>(P, c, nullptr, smc, smg, tc, tb, step, keep);
    if (block_err(bm, P.st.err)) {
      reason = 3;
      ++it;
      break;
    }
    if (check) {
      if (!grid_check(bm, c.rbits, P.st.res, P.st.barrier, ci, P.st.err, P.st.wait_ns)) {
        reason = 3;
        ++ci;
        ++it;
        break;
      }
      const unsigned long long rb = ld_l2(P.st.res + ci);
      ++ci;
      const double rv = __longlong_as_double((long long)rb) * P.invgamma;
      if (!(rv <= 1.7976931348623157e308)) {  // NaN or infinite
        reason = 2;
        ++it;
        break;
      }
      if (P.tol > 0.0 && rv <= P.tol) {
        reason = 1;
        ++it;
        break;
      }
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    P.st.info[0] = it;
    P.st.info[1] = ci;
    P.st.info[2] = reason;
    if (APG) stamp_time(P.st.info, 1);
  }
}

}  // namespace

// this translation unit is compiled once per component count RN_CVAL and
// kind of W_u RN_DENSE
const void *RN_CAT(RN_CAT(solve_kernel_c, RN_CVAL), RN_CAT(_d, RN_DENSE))(bool apg) {
  return apg ? (const void *)RN_CAT(kv, RN_DENSE)::k_solve<double, true, RN_CVAL>
             : (const void *)RN_CAT(kv, RN_DENSE)::k_solve<double, false, RN_CVAL>;
}

}  // namespace rn
