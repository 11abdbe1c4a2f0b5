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
#include <cuda/atomic>

#include "kernels.cuh"

namespace rn {

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <typename T>
__device__ __forceinline__ T ld_l2(const T *p) {
  return __ldcg(p);
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  cuda::atomic_ref<const unsigned, cuda::thread_scope_device> a(*p);
  return a.load(cuda::memory_order_acquire);
}

__device__ __forceinline__ void st_release(unsigned *p, unsigned v) {
  cuda::atomic_ref<unsigned, cuda::thread_scope_device> a(*p);
  a.store(v, cuda::memory_order_release);
}

// bounded spin of one thread until *p >= target; false on timeout or error
__device__ bool spin_geq(const unsigned *p, unsigned target, int *err) {
  if (ld_acquire(p) >= target) return true;
  const unsigned long long t0 = global_ns();
  while (true) {
    if (ld_acquire(p) >= target) return true;
    if (*(volatile int *)err != 0) return false;
    if ((long long)(global_ns() - t0) > kWaitNs) {
      atomicExch(err, 1);
      return false;
    }
    __nanosleep(64);
  }
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// sums of a and b over the block, returned to every thread; red holds 66 T
template <typename T>
__device__ void block_sum2(T &a, T &b, T *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  a = warp_sum(a);
  b = warp_sum(b);
  if (lane == 0) {
    red[warp] = a;
    red[32 + warp] = b;
  }
  __syncthreads();
  if (warp == 0) {
    T x = lane < nw ? red[lane] : T(0);
    T y = lane < nw ? red[32 + lane] : T(0);
    x = warp_sum(x);
    y = warp_sum(y);
    if (lane == 0) {
      red[64] = x;
      red[65] = y;
    }
  }
  __syncthreads();
  a = red[64];
  b = red[65];
}

__device__ __forceinline__ unsigned long long block_max_u64(unsigned long long v,
                                                            unsigned long long *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < nw; ++i) v = red[i] > v ? red[i] : v;
    red[32] = v;
  }
  __syncthreads();
  v = red[32];
  __syncthreads();
  return v;
}

// bits of |d| as an unsigned integer: monotone in |d| (NaN compares above inf)
__device__ __forceinline__ unsigned long long abs_bits(double d) {
  return (unsigned long long)__double_as_longlong(d) & 0x7fffffffffffffffULL;
}
__device__ __forceinline__ unsigned long long abs_bits(float f) {
  return abs_bits((double)f);
}

// ---------------------------------------------------------------------------
// shared memory of the persistent kernel
// ---------------------------------------------------------------------------
template <typename T>
struct Smem {
  T *buf;   // kSeg * SP   chain rows (s, then lambda | ghat)
  T *eb;    // kSeg * NEP  E W^-1 ghat
  T *fb;    // kSeg * NEP  S^-1 E W^-1 ghat
  T *i2p;   // kSeg
  T *ubuf;  // NUP        inputs of the node in the forward sweep
  T *red;   // 72
  unsigned long long *redu;  // 40
  int *flag;                 // 4
};

template <typename T>
__device__ Smem<T> carve(unsigned char *raw, const NetDev<T> &nt) {
  Smem<T> s;
  T *p = reinterpret_cast<T *>(raw);
  s.buf = p;
  p += (size_t)kSeg * nt.SP;
  s.eb = p;
  p += (size_t)kSeg * nt.NEP;
  s.fb = p;
  p += (size_t)kSeg * nt.NEP;
  s.i2p = p;
  p += kSeg;
  s.ubuf = p;
  p += nt.NUP;
  s.red = p;
  p += 72;
  size_t off = (reinterpret_cast<unsigned char *>(p) - raw + 15) & ~(size_t)15;
  s.redu = reinterpret_cast<unsigned long long *>(raw + off);
  s.flag = reinterpret_cast<int *>(raw + off + 40 * sizeof(unsigned long long));
  return s;
}

// ---------------------------------------------------------------------------
// z = F ghat / (2p) for m rows of sm.buf (ghat at offset NXP of each row)
// F ghat = W^-1 (ghat - E' S^-1 E W^-1 ghat)
// ---------------------------------------------------------------------------
template <typename T>
__device__ void apply_F(const NetDev<T> &nt, int m, Smem<T> &sm, T *zrows) {
  const int tid = threadIdx.x, bd = blockDim.x, ne = nt.ne, nu = nt.nu;
  if (ne > 0) {
    for (int idx = tid; idx < m * ne; idx += bd) {
      const int q = idx / ne, r = idx - q * ne;
      const T *g = sm.buf + q * nt.SP + nt.NXP;
      T acc = T(0);
      for (int e = nt.Er_ptr[r]; e < nt.Er_ptr[r + 1]; ++e) {
        const int j = nt.Er_idx[e];
        acc += nt.Er_val[e] * (nt.winv[j] * g[j]);
      }
      sm.eb[q * nt.NEP + r] = acc;
    }
    __syncthreads();
    for (int idx = tid; idx < m * ne; idx += bd) {
      const int q = idx / ne, r = idx - q * ne;
      const T *Si = nt.Sinv + (size_t)r * ne;
      const T *e = sm.eb + q * nt.NEP;
      T acc = T(0);
      for (int c = 0; c < ne; ++c) acc += Si[c] * e[c];
      sm.fb[q * nt.NEP + r] = acc;
    }
    __syncthreads();
  }
  for (int idx = tid; idx < m * nu; idx += bd) {
    const int q = idx / nu, j = idx - q * nu;
    T acc = sm.buf[q * nt.SP + nt.NXP + j];
    for (int e = nt.Ec_ptr[j]; e < nt.Ec_ptr[j + 1]; ++e)
      acc -= nt.Ec_val[e] * sm.fb[q * nt.NEP + nt.Ec_idx[e]];
    zrows[(size_t)q * nt.NUP + j] = (nt.winv[j] * acc) * sm.i2p[q];
  }
}

// ---------------------------------------------------------------------------
// backward sweep over one chain: suffix sums from the leaf to the head
// ---------------------------------------------------------------------------
template <typename T>
__device__ void chain_backward(const KParams<T> &P, int k, Smem<T> &sm) {
  const NetDev<T> &nt = P.net;
  const int tid = threadIdx.x, bd = blockDim.x;
  const int start = P.plan.ch_start[k], L = P.plan.ch_len[k];
  T accL = T(0), accG = T(0);
  for (int hi = L; hi > 0; hi -= kSeg) {
    const int lo = hi > kSeg ? hi - kSeg : 0, m = hi - lo;
    const T *src = P.st.s + (size_t)(start + lo) * nt.SP;
    for (int e = tid; e < m * nt.SP; e += bd) sm.buf[e] = src[e];
    if (tid < m) sm.i2p[tid] = P.st.inv2p[start + lo + tid];
    __syncthreads();
    if (tid < nt.nx) {
      for (int q = m - 1; q >= 0; --q) {
        accL += sm.buf[q * nt.SP + tid];
        sm.buf[q * nt.SP + tid] = accL;
      }
    }
    __syncthreads();
    if (tid < nt.nu) {
      const int b0 = nt.Bc_ptr[tid], b1 = nt.Bc_ptr[tid + 1];
      for (int q = m - 1; q >= 0; --q) {
        const T *row = sm.buf + q * nt.SP;
        T t = row[nt.NXP + tid];
        for (int e = b0; e < b1; ++e) t += nt.Bc_val[e] * row[nt.Bc_idx[e]];
        accG += t;
        sm.buf[q * nt.SP + nt.NXP + tid] = accG;
      }
    }
    __syncthreads();
    apply_F(nt, m, sm, P.st.z + (size_t)(start + lo) * nt.NUP);
    if (lo == 0) {
      T *dst = P.st.up + (size_t)start * nt.SP;
      for (int e = tid; e < nt.SP; e += bd) dst[e] = sm.buf[e];
    }
    __syncthreads();
  }
}

// backward step at a top node: own terms plus the children's subtree sums
template <typename T>
__device__ void top_backward(const KParams<T> &P, int v, Smem<T> &sm) {
  const NetDev<T> &nt = P.net;
  const int tid = threadIdx.x, bd = blockDim.x;
  const int c0 = P.plan.top_child_ptr[v], c1 = P.plan.top_child_ptr[v + 1];
  const T *sv = P.st.s + (size_t)v * nt.SP;
  if (tid < nt.nx) {
    T acc = ld_l2(sv + tid);
    for (int c = c0; c < c1; ++c) acc += ld_l2(P.st.up + (size_t)P.plan.top_child[c] * nt.SP + tid);
    sm.buf[tid] = acc;
  }
  if (tid == 0) sm.i2p[0] = P.st.inv2p[v];
  __syncthreads();
  if (tid < nt.nu) {
    T acc = ld_l2(sv + nt.NXP + tid);
    for (int e = nt.Bc_ptr[tid]; e < nt.Bc_ptr[tid + 1]; ++e)
      acc += nt.Bc_val[e] * sm.buf[nt.Bc_idx[e]];
    for (int c = c0; c < c1; ++c)
      acc += ld_l2(P.st.up + (size_t)P.plan.top_child[c] * nt.SP + nt.NXP + tid);
    sm.buf[nt.NXP + tid] = acc;
  }
  __syncthreads();
  apply_F(nt, 1, sm, P.st.z + (size_t)v * nt.NUP);
  T *dst = P.st.up + (size_t)v * nt.SP;
  for (int e = tid; e < nt.SP; e += bd) {
    const bool pad = (e >= nt.nx && e < nt.NXP) || e >= nt.NXP + nt.nu;
    dst[e] = pad ? T(0) : sm.buf[e];
  }
  __syncthreads();
}

// After a chain's backward sweep: arrive at the parent; the last child to
// arrive completes the parent and climbs on.  Completing a stage-1 node
// releases its flag for the forward sweep.  Returns false on timeout.
template <typename T>
__device__ void climb(const KParams<T> &P, int k, unsigned step, Smem<T> &sm) {
  int v = P.plan.ch_parent[k];
  while (v > 0) {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned old = atomicAdd(P.st.count + v, 1u);
      sm.flag[0] = ((old + 1u) % (unsigned)P.plan.top_nchild[v]) == 0u;
    }
    __syncthreads();
    if (!sm.flag[0]) break;
    __threadfence();
    top_backward(P, v, sm);
    __threadfence();
    __syncthreads();
    const int f = P.plan.top_flag[v];
    if (f >= 0) {
      if (threadIdx.x == 0) st_release(P.st.flags + f, step + 1u);
      break;
    }
    v = P.plan.parent[v];
  }
}

// ---------------------------------------------------------------------------
// forward sweep
// ---------------------------------------------------------------------------
template <typename T>
struct FwdCtx {
  T Zp;   // running path sum of z (thread j < nu)
  T xa;   // state of the ancestor (thread i < nx)
  const T *ycur;
  T *yprv;
  T beta, beta_n;
  bool write_out;
  unsigned long long rbits;  // running max of |y+ - w| (bits)
};

// dual update at one node: y+ = prox_{gamma g*}(w + gamma H x) in the closed
// form e * min(gamma, W / |e|) with e = v - proj_C(v), v = Hx + w / gamma
// (distance-to-set prox of §4.3 through the Moreau decomposition of §4.2),
// and the next extrapolated w folded into the backward input s.
template <typename T>
__device__ void prox_update(const KParams<T> &P, int v, T uj, T xi, FwdCtx<T> &c, Smem<T> &sm) {
  const NetDev<T> &nt = P.net;
  const int tid = threadIdx.x;
  const T g = (T)P.gamma, ig = (T)P.invgamma;
  const T *yc = c.ycur + (size_t)v * nt.YP;
  T *yp = c.yprv + (size_t)v * nt.YP;
  T e1 = T(0), e2 = T(0), w1 = T(0), w2 = T(0), a1 = T(0), a2 = T(0);
  if (tid < nt.nx) {
    a1 = yc[tid];
    a2 = yc[nt.NXP + tid];
    const T b1 = yp[tid], b2 = yp[nt.NXP + tid];
    w1 = a1 + c.beta * (a1 - b1);
    w2 = a2 + c.beta * (a2 - b2);
    const T v1 = xi + w1 * ig;
    const T v2 = xi + w2 * ig;
    e1 = v1 - fmin(fmax(v1, nt.xmin[tid]), nt.xmax[tid]);
    e2 = fmin(v2 - nt.xs[tid], T(0));
  }
  T n1 = e1 * e1, n2 = e2 * e2;
  block_sum2(n1, n2, sm.red);
  if (tid < nt.nx) {
    const T s1 = n1 > T(0) ? fmin(g, nt.Wx / sqrt(n1)) : T(0);
    const T s2 = n2 > T(0) ? fmin(g, nt.Ws / sqrt(n2)) : T(0);
    const T y1 = e1 * s1, y2 = e2 * s2;
    unsigned long long r = abs_bits(y1 - w1), r2 = abs_bits(y2 - w2);
    r = r2 > r ? r2 : r;
    c.rbits = r > c.rbits ? r : c.rbits;
    yp[tid] = y1;
    yp[nt.NXP + tid] = y2;
    const T wn1 = y1 + c.beta_n * (y1 - a1);
    const T wn2 = y2 + c.beta_n * (y2 - a2);
    P.st.s[(size_t)v * nt.SP + tid] = wn1 + wn2;
    if (c.write_out) P.st.xo[(size_t)v * nt.NXP + tid] = xi;
  }
  if (tid < nt.nu) {
    const T a3 = yc[2 * nt.NXP + tid], b3 = yp[2 * nt.NXP + tid];
    const T w3 = a3 + c.beta * (a3 - b3);
    const T v3 = uj + w3 * ig;
    const T y3 = g * (v3 - fmin(fmax(v3, nt.umin[tid]), nt.umax[tid]));
    const unsigned long long r = abs_bits(y3 - w3);
    c.rbits = r > c.rbits ? r : c.rbits;
    yp[2 * nt.NXP + tid] = y3;
    P.st.s[(size_t)v * nt.SP + nt.NXP + tid] = y3 + c.beta_n * (y3 - a3);
    if (c.write_out) P.st.uo[(size_t)v * nt.NUP + tid] = uj;
  }
}

template <typename T, bool APG>
__device__ void forward_node(const KParams<T> &P, int v, bool owned, bool cross, FwdCtx<T> &c,
                             Smem<T> &sm) {
  const NetDev<T> &nt = P.net;
  const int tid = threadIdx.x;
  T uj = T(0), xi = T(0);
  if (tid < nt.nu) {
    const T *zp = P.st.z + (size_t)v * nt.NUP + tid;
    c.Zp += cross ? ld_l2(zp) : *zp;
    const T base = P.linear ? T(0) : P.st.ub[(size_t)v * nt.NUP + tid];
    uj = base - c.Zp;
    sm.ubuf[tid] = uj;
  }
  __syncthreads();
  if (tid < nt.nx) {
    T acc = c.xa;
    for (int e = nt.Br_ptr[tid]; e < nt.Br_ptr[tid + 1]; ++e)
      acc += nt.Br_val[e] * sm.ubuf[nt.Br_idx[e]];
    if (!P.linear) acc += P.st.gb[(size_t)v * nt.NXP + tid];
    c.xa = acc;
    xi = acc;
  }
  if (owned) {
    if (APG) {
      prox_update(P, v, uj, xi, c, sm);
    } else {
      if (tid < nt.nu) P.st.uo[(size_t)v * nt.NUP + tid] = uj;
      if (tid < nt.nx) P.st.xo[(size_t)v * nt.NXP + tid] = xi;
    }
  }
  __syncthreads();
}

template <typename T, bool APG>
__device__ void chain_forward(const KParams<T> &P, int k, FwdCtx<T> &c, Smem<T> &sm) {
  const int tid = threadIdx.x;
  c.Zp = T(0);
  c.xa = (tid < P.net.nx && !P.linear) ? P.st.xroot[tid] : T(0);
  const int p0 = P.plan.ch_path_ptr[k], p1 = P.plan.ch_path_ptr[k + 1];
  const int own_from = P.plan.ch_own_from[k];
  for (int q = p0; q < p1; ++q)
    forward_node<T, APG>(P, P.plan.ch_path[q], (q - p0) >= own_from, true, c, sm);
  const int start = P.plan.ch_start[k], L = P.plan.ch_len[k];
  for (int q = 0; q < L; ++q) forward_node<T, APG>(P, start + q, true, false, c, sm);
}

// ---------------------------------------------------------------------------
// the persistent kernel: `iters` APG iterations (APG = true) or one
// evaluation of the dual gradient (APG = false)
// ---------------------------------------------------------------------------
template <typename T, bool APG>
__global__ void __launch_bounds__(256) k_solve(KParams<T> P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<T> sm = carve<T>(smem_raw, P.net);
  const int tid = threadIdx.x;
  int it = 0, ci = 0, reason = 0;  // reason: 0 max iters, 1 converged, 2 non-finite, 3 timeout
  bool ok = true;
  for (; it < P.iters && ok; ++it) {
    const unsigned step = P.step_base + (unsigned)it;
    for (int k = blockIdx.x; k < P.plan.n_chains; k += gridDim.x) {
      chain_backward(P, k, sm);
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
      chain_forward<T, APG>(P, k, c, sm);
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
cudaError_t launch_solve(const KParams<T> &P, int grid, int block, size_t smem, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_solve<T, APG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  KParams<T> p = P;
  void *args[] = {&p};
  return cudaLaunchCooperativeKernel((const void *)k_solve<T, APG>, dim3(grid), dim3(block), args,
                                     smem, st);
}

template <typename T, bool APG>
cudaError_t solve_occupancy(int block, size_t smem, int *blocks_per_sm) {
  cudaError_t e = cudaFuncSetAttribute(k_solve<T, APG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_solve<T, APG>, block, smem);
}

template cudaError_t launch_solve<double, true>(const KParams<double> &, int, int, size_t, cudaStream_t);
template cudaError_t launch_solve<double, false>(const KParams<double> &, int, int, size_t, cudaStream_t);
template cudaError_t solve_occupancy<double, true>(int, size_t, int *);
template cudaError_t solve_occupancy<double, false>(int, size_t, int *);

}  // namespace rn
