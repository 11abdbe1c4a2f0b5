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
// is scanned by one thread block, top nodes are summed by the block that
// completes their last child, and every block recomputes the path sums of
// its chain's top ancestors instead of waiting for them.
#include <mutex>
#include <set>

#include "solve_device.cuh"

namespace rn {

cudaError_t allow_max_smem(const void *fn) {
  static std::mutex mu;
  static std::set<std::pair<int, const void *>> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  if (done.count({dev, fn})) return cudaSuccess;
  int optin = 0;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa{};
  e = cudaFuncGetAttributes(&fa, fn);  // static shared memory counts against the limit
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           optin - (int)fa.sharedSizeBytes);
  if (e == cudaSuccess) done.insert({dev, fn});
  return e;
}

// ---------------------------------------------------------------------------
// the persistent kernel: `iters` APG iterations (APG = true) or one
// evaluation of the dual gradient (APG = false)
// ---------------------------------------------------------------------------
template <typename T, bool APG, int C>
__global__ void __launch_bounds__(256) k_solve(KParams<T> P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<T> sm = carve<T>(smem_raw, P.net, P.buf_elems);
  sm.net = stage_net(P.net, sm.net_raw);
  const int tid = threadIdx.x;
  int it = 0, ci = 0, reason = 0;  // reason: 0 max iters, 1 converged, 2 non-finite, 3 timeout
  bool ok = true;
  for (; it < P.iters && ok; ++it) {
    const unsigned step = P.step_base + (unsigned)it;
    for (int k = blockIdx.x; k < P.plan.n_chains; k += gridDim.x) {
      chain_backward<T, C>(P, k, sm);
      climb(P, k, step, sm);
    }
    FwdCtx<T> c;
    c.ycur = (it & 1) ? P.st.yb : P.st.ya;
    c.yprv = (it & 1) ? P.st.ya : P.st.yb;
    c.beta = APG ? (T)P.st.beta[it] : T(0);
    c.beta_n = APG ? (T)P.st.beta[it + 1] : T(0);
    const bool check = APG && (((it + 1) % P.check_every) == 0 || it + 1 == P.iters);
    c.write_out = !APG || check;
    c.rbits = 0ull;
    for (int k = blockIdx.x; k < P.plan.n_chains; k += gridDim.x) {
      const int f = P.plan.ch_flag[k];
      if (f >= 0) {
        if (tid == 0) sm.flag[1] = spin_geq(P.st.flags + f, step + 1u, P.st.err);
        __syncthreads();
        if (!sm.flag[1]) {
          ok = false;
          reason = 3;
          break;
        }
      }
      chain_forward<T, APG ? kFwdApg : kFwdPlain, C>(P, k, c, sm, nullptr);
    }
    if (!ok) break;
    if (check) {
      const unsigned long long r = block_max_u64(c.rbits, sm.redu);
      if (tid == 0) {
        atomicMax(P.st.res + ci, r);
        __threadfence();
        atomicAdd(P.st.barrier, 1u);
        sm.flag[2] = spin_geq(P.st.barrier, (unsigned)(ci + 1) * gridDim.x, P.st.err);
      }
      __syncthreads();
      if (!sm.flag[2]) {
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
    if (*(volatile int *)P.st.err != 0) {
      reason = 3;
      ++it;
      break;
    }
  }
  if (blockIdx.x == 0 && tid == 0) {
    P.st.info[0] = it;
    P.st.info[1] = ci;
    P.st.info[2] = reason;
  }
}

template <typename T, bool APG>
static const void *solve_fn(int c) {
  switch (c) {
    case 1: return (const void *)k_solve<T, APG, 1>;
    case 2: return (const void *)k_solve<T, APG, 2>;
    case 4: return (const void *)k_solve<T, APG, 4>;
    default: return (const void *)k_solve<T, APG, 8>;
  }
}

template <typename T, bool APG>
cudaError_t launch_solve(const KParams<T> &P, int grid, int block, size_t smem, cudaStream_t st) {
  const void *fn = solve_fn<T, APG>(P.maxc);
  cudaError_t e = allow_max_smem(fn);
  if (e != cudaSuccess) return e;
  KParams<T> p = P;
  void *args[] = {&p};
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(block), args, smem, st);
}

template <typename T, bool APG>
cudaError_t solve_occupancy(int maxc, int block, size_t smem, int *blocks_per_sm) {
  const void *fn = solve_fn<T, APG>(maxc);
  cudaError_t e = allow_max_smem(fn);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, block, smem);
}

template cudaError_t launch_solve<double, true>(const KParams<double> &, int, int, size_t, cudaStream_t);
template cudaError_t launch_solve<double, false>(const KParams<double> &, int, int, size_t, cudaStream_t);
template cudaError_t solve_occupancy<double, true>(int, int, size_t, int *);
template cudaError_t solve_occupancy<double, false>(int, int, size_t, int *);

}  // namespace rn
