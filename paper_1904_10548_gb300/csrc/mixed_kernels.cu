// Mixed-precision persistent kernel of the dual APG (paper §4.3 eqs.
// apg:1 / apg:2) on the scenario tree.
//
// The dual iterate is y = yb + d: an FP64 base yb and an FP32 delta d.  The
// dual gradient is affine in w, x*(w) = x*(yb) + x_lin(w - yb), so an
// iteration evaluates only the linear part on the FP32 delta dw = w - yb
// (the same backward/forward sweeps as the FP64 path, in FP32) and adds
// xref = x*(yb).  Every R iterations the base absorbs the delta (FP64) and
// xref is recomputed by an FP64 evaluation of the dual gradient; the last
// iteration's primal x*(w) is evaluated in FP64 as well, so the returned
// (u, x) satisfy the dynamics and couplings to FP64 rounding.  All three
// kinds of steps run in one cooperative launch and share its counters and
// flags, numbered by a common step counter.
#include "solve_device.cuh"

namespace rn {

namespace RN_CAT(kv, RN_DENSE) {  // one kernel per (C, W_u diagonal or dense)

template <int C>
__global__ void __launch_bounds__(512) k_mixed(MixedParams M) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (blockIdx.x == 0 && threadIdx.x == 0) stamp_time(M.f.st.info, 0);
  // network region: the FP32 copy (for the iterations), then the header of
  // the FP64 data (the rarely run FP64 steps read its arrays from global
  // memory) at offset M.d.net_bytes
  const BlockMem bm = block_mem(smem_raw, M.f.net_bytes, M.f.team_bytes);
  const NetDev<float> *netf = stage_net(M.f.net, bm.net_raw);
  const NetDev<double> *netd = stage_net(M.d.net, bm.net_raw + M.d.net_bytes, false);
  const int tpb = M.f.tpb;
  const Team tc = chain_team(tpb), tb = block_team();
  const int ti = team_index(tpb);
  const Smem<float> sfc = carve<float>(bm.team_raw(ti), M.f.buf_elems, netf);
  const Smem<float> sfg = carve<float>(bm.team_raw(0), M.f.gbuf_elems, netf);
  const Smem<double> sdc = carve<double>(bm.team_raw(ti), M.d.buf_elems, netd);
  const Smem<double> sdg = carve<double>(bm.team_raw(0), M.d.gbuf_elems, netd);
  const KParams<float> &P = M.f;
  const int G = P.plan.n_groups, K = P.plan.n_chains, n_items = G + (K + tpb - 1) / tpb;
  const bool keep = (int)gridDim.x >= n_items && (int)blockIdx.x >= G;
  auto owned = [&](auto fn) {
    for (int i = blockIdx.x; i < n_items; i += gridDim.x) {
      const int k = tpb * (i - G) + ti;
      if (i < G || k >= K) continue;
      int idx = 0;
      for_owned(P.plan, k, [&](int v) {
        if ((idx++ % tc.nwarps()) == tc.warp()) fn(v);
      });
    }
    tc.sync();
  };
  unsigned step = P.step_base;
  int it = 0, ci = 0, reason = 0;  // reason: 0 max iters, 1 converged, 2 non-finite, 3 timeout
  FwdCtx<double> c64{};
  eval_step<double, kFwdPlain, C>(M.d, c64, nullptr, sdc, sdg, tc, tb, step++, keep);
  bool ok = !block_err(bm, P.st.err);
  if (!ok) reason = 3;
  for (; it < P.iters && ok; ++it) {
    FwdCtx<float> c;
    float *dcur = (it & 1) ? M.mx.db : M.mx.da;
    float *dprv = (it & 1) ? M.mx.da : M.mx.db;
    c.ycur = dcur;
    c.yprv = dprv;
    c.beta = (float)P.st.beta[it];
    c.beta_n = (float)P.st.beta[it + 1];
    const bool check = ((it + 1) % P.check_every) == 0 || it + 1 == P.iters;
    c.write_out = check;
    c.avg = P.st.uavg != nullptr;
    c.theta = P.st.theta[it];
    c.rbits = 0ull;
    eval_step<float, kFwdMixed, C>(P, c, &M.mx, sfc, sfg, tc, tb, step++, keep);
    if (block_err(bm, P.st.err)) {
      ok = false;
      reason = 3;
      ++it;
      break;
    }
    if (check) {
      if (!grid_check(bm, widen_bits(c.rbits), P.st.res, P.st.barrier, ci, P.st.err,
                      P.st.wait_ns)) {
        ok = false;
        reason = 3;
        ++it;
        break;
      }
      // residual bits were taken from FP32 |y+ - w|; widen to FP64 units
      const unsigned long long rb = ld_l2(P.st.res + ci);
      ++ci;
      const double rv = (double)__longlong_as_double((long long)rb) * P.invgamma;
      if (!(rv <= 1.7976931348623157e308)) {
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
    if ((it + 1) % M.mx.refresh_every == 0 && it + 1 < P.iters) {
      const float bn = (float)P.st.beta[it + 1];
      owned([&](int v) { refresh_node(M, v, dprv, dcur, bn); });
      eval_step<double, kFwdPlain, C>(M.d, c64, nullptr, sdc, sdg, tc, tb, step++, keep);
      if (block_err(bm, P.st.err)) {
        ok = false;
        reason = 3;
        ++it;
        break;
      }
    }
  }
  if (ok) {
    owned([&](int v) { final_node(M, v); });
    eval_step<double, kFwdPlain, C>(M.d, c64, nullptr, sdc, sdg, tc, tb, step++, keep);
    if (block_err(bm, P.st.err)) reason = 3;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    P.st.info[0] = it;
    P.st.info[1] = ci;
    P.st.info[2] = reason;
    stamp_time(P.st.info, 1);
  }
}

}  // namespace

// this translation unit is compiled once per component count RN_CVAL and
// kind of W_u RN_DENSE
const void *RN_CAT(RN_CAT(mixed_kernel_c, RN_CVAL), RN_CAT(_d, RN_DENSE))() {
  return (const void *)RN_CAT(kv, RN_DENSE)::k_mixed<RN_CVAL>;
}

}  // namespace rn
