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

// one FP64 evaluation of the dual gradient from mx.s64 into d.st.uo / xo
// (and the FP32 copies uref / xref); false on timeout
template <int C>
__device__ bool fp64_step(const MixedParams &M, unsigned step, Smem<double> &sm) {
  const KParams<double> &P = M.d;
  for (int k = blockIdx.x; k < P.plan.n_chains; k += gridDim.x) {
    chain_backward<double, C>(P, k, sm);
    climb(P, k, step, sm);
  }
  FwdCtx<double> c{};
  for (int k = blockIdx.x; k < P.plan.n_chains; k += gridDim.x) {
    const int f = P.plan.ch_flag[k];
    if (f >= 0) {
      if (threadIdx.x == 0) sm.flag[1] = spin_geq(P.st.flags + f, step + 1u, P.st.err);
      __syncthreads();
      if (!sm.flag[1]) return false;
    }
    chain_forward<double, kFwdPlain, C>(P, k, c, sm, nullptr);
  }
  return true;
}

template <int C>
__global__ void __launch_bounds__(256) k_mixed(MixedParams M) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<double> smd = carve<double>(smem_raw, M.d.net, M.d.buf_elems);
  Smem<float> smf = carve<float>(smem_raw, M.f.net, M.f.buf_elems);
  // the FP32 iterations use a shared-memory copy of the network data; the
  // FP64 refresh steps read theirs from global memory (header only here)
  unsigned char *net_raw = smf.net_raw > smd.net_raw ? smf.net_raw : smd.net_raw;
  smf.net = stage_net(M.f.net, net_raw);
  smd.net = stage_net(M.d.net, net_raw + M.f.net_bytes, false);
  const KParams<float> &P = M.f;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  unsigned step = P.step_base;
  int it = 0, ci = 0, reason = 0;  // reason: 0 max iters, 1 converged, 2 non-finite, 3 timeout
  bool ok = fp64_step<C>(M, step++, smd);
  if (!ok) reason = 3;
  for (; it < P.iters && ok; ++it) {
    for (int k = blockIdx.x; k < P.plan.n_chains; k += gridDim.x) {
      chain_backward<float, C>(P, k, smf);
      climb(P, k, step, smf);
    }
    FwdCtx<float> c;
    float *dcur = (it & 1) ? M.mx.db : M.mx.da;
    float *dprv = (it & 1) ? M.mx.da : M.mx.db;
    c.ycur = dcur;
    c.yprv = dprv;
    c.beta = (float)P.st.beta[it];
    c.beta_n = (float)P.st.beta[it + 1];
    const bool check = ((it + 1) % P.check_every) == 0 || it + 1 == P.iters;
    c.write_out = check;
    c.rbits = 0ull;
    for (int k = blockIdx.x; k < P.plan.n_chains; k += gridDim.x) {
      const int f = P.plan.ch_flag[k];
      if (f >= 0) {
        if (tid == 0) smf.flag[1] = spin_geq(P.st.flags + f, step + 1u, P.st.err);
        __syncthreads();
        if (!smf.flag[1]) {
          ok = false;
          reason = 3;
          break;
        }
      }
      chain_forward<float, kFwdMixed, C>(P, k, c, smf, &M.mx);
    }
    ++step;
    if (!ok) break;
    bool stop = false;
    if (check) {
      const unsigned long long r = block_max_u64(c.rbits, smf.redu);
      if (tid == 0) {
        atomicMax(P.st.res + ci, r);
        __threadfence();
        atomicAdd(P.st.barrier, 1u);
        smf.flag[2] = spin_geq(P.st.barrier, (unsigned)(ci + 1) * gridDim.x, P.st.err);
      }
      __syncthreads();
      if (!smf.flag[2]) {
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
        stop = true;
      } else if (P.tol > 0.0 && rv <= P.tol) {
        reason = 1;
        stop = true;
      }
    }
    if (*(volatile int *)P.st.err != 0) {
      ok = false;
      reason = 3;
      ++it;
      break;
    }
    if (stop) {
      ++it;
      break;
    }
    if ((it + 1) % M.mx.refresh_every == 0 && it + 1 < P.iters) {
      const float bn = (float)P.st.beta[it + 1];
      for (int k = blockIdx.x; k < P.plan.n_chains; k += gridDim.x) {
        int idx = 0;
        for_owned(P.plan, k, [&](int v) {
          if ((idx++ % nw) == warp) refresh_node(M, v, dprv, dcur, bn);
        });
      }
      __syncthreads();
      if (!fp64_step<C>(M, step++, smd)) {
        ok = false;
        reason = 3;
        ++it;
        break;
      }
    }
  }
  if (ok) {
    for (int k = blockIdx.x; k < P.plan.n_chains; k += gridDim.x) {
      int idx = 0;
      for_owned(P.plan, k, [&](int v) {
        if ((idx++ % nw) == warp) final_node(M, v);
      });
    }
    __syncthreads();
    if (!fp64_step<C>(M, step++, smd)) reason = 3;
  }
  (void)lane;
  if (blockIdx.x == 0 && tid == 0) {
    P.st.info[0] = it;
    P.st.info[1] = ci;
    P.st.info[2] = reason;
  }
}

static const void *mixed_fn(int c) {
  switch (c) {
    case 1: return (const void *)k_mixed<1>;
    case 2: return (const void *)k_mixed<2>;
    case 4: return (const void *)k_mixed<4>;
    default: return (const void *)k_mixed<8>;
  }
}

cudaError_t launch_mixed(const MixedParams &M, int maxc, int grid, int block, size_t smem,
                         cudaStream_t st) {
  const void *fn = mixed_fn(maxc);
  cudaError_t e = allow_max_smem(fn);
  if (e != cudaSuccess) return e;
  MixedParams p = M;
  void *args[] = {&p};
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(block), args, smem, st);
}

cudaError_t mixed_occupancy(int maxc, int block, size_t smem, int *blocks_per_sm) {
  const void *fn = mixed_fn(maxc);
  cudaError_t e = allow_max_smem(fn);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, block, smem);
}

}  // namespace rn
