// Device building blocks of the persistent solve kernels (solve_kernels.cu,
// mixed_kernels.cu): bounded waits, block/warp reductions, the backward
// sweep over chains and top nodes, and the forward sweep with the dual
// update.
#pragma once

#include <cuda/atomic>

#include <type_traits>

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
static __device__ bool spin_geq(const unsigned *p, unsigned target, int *err) {
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
  T *buf;   // backward: kSeg x SP rows (s, then lambda | ghat), then eb, fb, i2p;
            // forward: the staged rows of one segment (see chain_forward)
  T *eb;    // kSeg * NEP  E W^-1 ghat
  T *fb;    // kSeg * NEP  S^-1 E W^-1 ghat
  T *i2p;   // kSeg
  T *red;   // 72
  unsigned long long *redu;  // 40
  int *flag;                 // 4
  int *node;                 // 2 x kSeg: node ids and ownership of a forward segment
  const NetDev<T> *net;      // the network data in use (a shared-memory copy)
  unsigned char *net_raw;    // where the block's copy lives
};

template <typename T>
__device__ Smem<T> carve(unsigned char *raw, const NetDev<T> &nt, int buf_elems) {
  Smem<T> s;
  T *p = reinterpret_cast<T *>(raw);
  s.buf = p;
  s.eb = p + (size_t)kSeg * nt.SP;
  s.fb = s.eb + (size_t)kSeg * nt.NEP;
  s.i2p = s.fb + (size_t)kSeg * nt.NEP;
  p += buf_elems;
  s.red = p;
  p += 72;
  size_t off = (reinterpret_cast<unsigned char *>(p) - raw + 15) & ~(size_t)15;
  s.redu = reinterpret_cast<unsigned long long *>(raw + off);
  s.flag = reinterpret_cast<int *>(raw + off + 40 * sizeof(unsigned long long));
  s.node = s.flag + 4;
  off = round16(off + 40 * sizeof(unsigned long long) + (4 + 2 * kSeg) * sizeof(int));
  s.net_raw = raw + off;
  s.net = nullptr;
  return s;
}

// Copy the network data into shared memory at raw (net_smem_bytes of
// room) and return the copy; every block calls it once at start.  With
// arrays = false only the header is copied (the arrays stay in global
// memory; for rarely run steps).
template <typename T>
__device__ const NetDev<T> *stage_net(const NetDev<T> &g, unsigned char *raw, bool arrays = true) {
  if (!arrays) {
    NetDev<T> *h = reinterpret_cast<NetDev<T> *>(raw);
    if (threadIdx.x == 0) *h = g;
    __syncthreads();
    return h;
  }
  const int nu = g.nu, nx = g.nx, ne = g.ne;
  const int nnzB = g.Bc_ptr[nu], nnzE = ne > 0 ? g.Er_ptr[ne] : 0;
  NetDev<T> *s = reinterpret_cast<NetDev<T> *>(raw);
  int *ip = reinterpret_cast<int *>(raw + round16(sizeof(NetDev<double>)));
  int *Bc_ptr = ip, *Bc_idx = Bc_ptr + nu + 1, *Br_ptr = Bc_idx + nnzB, *Br_idx = Br_ptr + nx + 1;
  int *Er_ptr = Br_idx + nnzB, *Er_idx = Er_ptr + ne + 1, *Ec_ptr = Er_idx + nnzE;
  int *Ec_idx = Ec_ptr + nu + 1;
  const size_t nints = (size_t)(nu + 1) + nnzB + (nx + 1) + nnzB + (ne + 1) + nnzE + (nu + 1) + nnzE;
  T *vp = reinterpret_cast<T *>(reinterpret_cast<unsigned char *>(ip) + round16(nints * 4));
  T *Bc_val = vp, *Br_val = Bc_val + nnzB, *Er_val = Br_val + nnzB, *Ec_val = Er_val + nnzE;
  T *winv = Ec_val + nnzE, *Sinv = winv + nu, *xmin = Sinv + (size_t)ne * ne, *xmax = xmin + nx;
  T *xs = xmax + nx, *umin = xs + nx, *umax = umin + nu;
  const int tid = threadIdx.x, bd = blockDim.x;
  auto cpi = [&](int *dst, const int *src, int m) {
    for (int i = tid; i < m; i += bd) dst[i] = src[i];
  };
  auto cpv = [&](T *dst, const T *src, int m) {
    for (int i = tid; i < m; i += bd) dst[i] = src[i];
  };
  cpi(Bc_ptr, g.Bc_ptr, nu + 1);
  cpi(Bc_idx, g.Bc_idx, nnzB);
  cpi(Br_ptr, g.Br_ptr, nx + 1);
  cpi(Br_idx, g.Br_idx, nnzB);
  cpi(Er_ptr, g.Er_ptr, ne + 1);
  cpi(Er_idx, g.Er_idx, nnzE);
  cpi(Ec_ptr, g.Ec_ptr, nu + 1);
  cpi(Ec_idx, g.Ec_idx, nnzE);
  cpv(Bc_val, g.Bc_val, nnzB);
  cpv(Br_val, g.Br_val, nnzB);
  cpv(Er_val, g.Er_val, nnzE);
  cpv(Ec_val, g.Ec_val, nnzE);
  cpv(winv, g.winv, nu);
  cpv(Sinv, g.Sinv, ne * ne);
  cpv(xmin, g.xmin, nx);
  cpv(xmax, g.xmax, nx);
  cpv(xs, g.xs, nx);
  cpv(umin, g.umin, nu);
  cpv(umax, g.umax, nu);
  if (tid == 0) {
    *s = g;
    s->Bc_ptr = Bc_ptr;
    s->Bc_idx = Bc_idx;
    s->Bc_val = Bc_val;
    s->Br_ptr = Br_ptr;
    s->Br_idx = Br_idx;
    s->Br_val = Br_val;
    s->Er_ptr = Er_ptr;
    s->Er_idx = Er_idx;
    s->Er_val = Er_val;
    s->Ec_ptr = Ec_ptr;
    s->Ec_idx = Ec_idx;
    s->Ec_val = Ec_val;
    s->winv = winv;
    s->Sinv = Sinv;
    s->xmin = xmin;
    s->xmax = xmax;
    s->xs = xs;
    s->umin = umin;
    s->umax = umax;
  }
  __syncthreads();
  return s;
}

// copy rows `nodes[0..m)` of a row-major array (pitch elements, a multiple
// of 4) into consecutive shared-memory rows, 16 bytes per load, all
// threads of the block in flight at once; L2-only loads for data other
// blocks write in the same launch
template <typename T>
__device__ __forceinline__ void stage_rows(T *dst, const T *src, int pitch, const int *nodes, int m,
                                           bool l2) {
  using V = typename std::conditional<sizeof(T) == 8, double2, float4>::type;
  constexpr int per = 16 / sizeof(T);
  const int nv = pitch / per;
  V *d = reinterpret_cast<V *>(dst);
  for (int e = threadIdx.x; e < m * nv; e += blockDim.x) {
    const int q = e / nv, c = e - q * nv;
    const V *s = reinterpret_cast<const V *>(src + (size_t)nodes[q] * pitch) + c;
    d[e] = l2 ? __ldcg(s) : *s;
  }
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
template <typename T, int C>
__device__ void chain_backward(const KParams<T> &P, int k, Smem<T> &sm) {
  const NetDev<T> &nt = *sm.net;
  const int tid = threadIdx.x, bd = blockDim.x;
  const int start = P.plan.ch_start[k], L = P.plan.ch_len[k];
  T accL[C], accG[C];
#pragma unroll
  for (int c = 0; c < C; ++c) accL[c] = accG[c] = T(0);
  for (int hi = L; hi > 0; hi -= kSeg) {
    const int lo = hi > kSeg ? hi - kSeg : 0, m = hi - lo;
    {
      using V = typename std::conditional<sizeof(T) == 8, double2, float4>::type;
      constexpr int per = 16 / sizeof(T);
      const V *src = reinterpret_cast<const V *>(P.st.s + (size_t)(start + lo) * nt.SP);
      V *dst = reinterpret_cast<V *>(sm.buf);
      for (int e = tid; e < m * nt.SP / per; e += bd) dst[e] = src[e];
    }
    if (tid < m) sm.i2p[tid] = P.st.inv2p[start + lo + tid];
    __syncthreads();
    // lambda: suffix sums of w1 + w2 (thread owns components tid + c bd)
    for (int q = m - 1; q >= 0; --q) {
      T *row = sm.buf + q * nt.SP;
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const int i = tid + c * bd;
        if (i < nt.nx) {
          accL[c] += row[i];
          row[i] = accL[c];
        }
      }
    }
    __syncthreads();
    // ghat: suffix sums of w3 + B' lambda
    for (int q = m - 1; q >= 0; --q) {
      T *row = sm.buf + q * nt.SP;
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const int j = tid + c * bd;
        if (j < nt.nu) {
          T t = row[nt.NXP + j];
          for (int e = nt.Bc_ptr[j]; e < nt.Bc_ptr[j + 1]; ++e) t += nt.Bc_val[e] * row[nt.Bc_idx[e]];
          accG[c] += t;
          row[nt.NXP + j] = accG[c];
        }
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
  const NetDev<T> &nt = *sm.net;
  const int tid = threadIdx.x, bd = blockDim.x;
  const int c0 = P.plan.top_child_ptr[v], c1 = P.plan.top_child_ptr[v + 1];
  const T *sv = P.st.s + (size_t)v * nt.SP;
  for (int i = tid; i < nt.nx; i += bd) {
    T acc = ld_l2(sv + i);
    for (int c = c0; c < c1; ++c) acc += ld_l2(P.st.up + (size_t)P.plan.top_child[c] * nt.SP + i);
    sm.buf[i] = acc;
  }
  if (tid == 0) sm.i2p[0] = P.st.inv2p[v];
  __syncthreads();
  for (int j = tid; j < nt.nu; j += bd) {
    T acc = ld_l2(sv + nt.NXP + j);
    for (int e = nt.Bc_ptr[j]; e < nt.Bc_ptr[j + 1]; ++e) acc += nt.Bc_val[e] * sm.buf[nt.Bc_idx[e]];
    for (int c = c0; c < c1; ++c)
      acc += ld_l2(P.st.up + (size_t)P.plan.top_child[c] * nt.SP + nt.NXP + j);
    sm.buf[nt.NXP + j] = acc;
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
  const T *ycur;
  T *yprv;
  T beta, beta_n;
  bool write_out;
  unsigned long long rbits;  // running max of |y+ - w| (bits)
};

// Dual update at one node by one warp: y+ = prox_{gamma g*}(w + gamma H x)
// in the closed form e * min(gamma, W / |e|), e = v - proj_C(v),
// v = Hx + w / gamma (distance-to-set prox of §4.3 through the Moreau
// decomposition of §4.2), the next extrapolated w folded into the backward
// input s.  Lanes own components i = lane + 32 c (c < MAXC) of the state
// blocks and j = lane + 32 c of the input block.  yc / yp: staged rows of
// y^nu and y^{nu-1}; y^{nu+1} is written over y^{nu-1} in global memory.
template <typename T, int MAXC>
__device__ void prox_node_warp(const KParams<T> &P, const NetDev<T> &nt, int v, const T *Uq,
                               const T *Xq, const T *yc, const T *yp, FwdCtx<T> &c) {
  const int lane = threadIdx.x & 31;
  const T g = (T)P.gamma, ig = (T)P.invgamma;
  T *ypg = c.yprv + (size_t)v * nt.YP;
  T e1[MAXC], e2[MAXC], w1[MAXC], w2[MAXC], a1[MAXC], a2[MAXC];
  T n1 = T(0), n2 = T(0);
#pragma unroll
  for (int cc = 0; cc < MAXC; ++cc) {
    const int i = lane + 32 * cc;
    e1[cc] = e2[cc] = w1[cc] = w2[cc] = a1[cc] = a2[cc] = T(0);
    if (i < nt.nx) {
      a1[cc] = yc[i];
      a2[cc] = yc[nt.NXP + i];
      w1[cc] = a1[cc] + c.beta * (a1[cc] - yp[i]);
      w2[cc] = a2[cc] + c.beta * (a2[cc] - yp[nt.NXP + i]);
      const T xi = Xq[i];
      const T v1 = xi + w1[cc] * ig;
      const T v2 = xi + w2[cc] * ig;
      e1[cc] = v1 - fmin(fmax(v1, nt.xmin[i]), nt.xmax[i]);
      e2[cc] = fmin(v2 - nt.xs[i], T(0));
      n1 += e1[cc] * e1[cc];
      n2 += e2[cc] * e2[cc];
    }
  }
  n1 = warp_sum(n1);
  n2 = warp_sum(n2);
  const T s1 = n1 > T(0) ? fmin(g, nt.Wx / sqrt(n1)) : T(0);
  const T s2 = n2 > T(0) ? fmin(g, nt.Ws / sqrt(n2)) : T(0);
  T *srow = P.st.s + (size_t)v * nt.SP;
#pragma unroll
  for (int cc = 0; cc < MAXC; ++cc) {
    const int i = lane + 32 * cc;
    if (i < nt.nx) {
      const T y1 = e1[cc] * s1, y2 = e2[cc] * s2;
      unsigned long long r = abs_bits(y1 - w1[cc]), r2 = abs_bits(y2 - w2[cc]);
      r = r2 > r ? r2 : r;
      c.rbits = r > c.rbits ? r : c.rbits;
      ypg[i] = y1;
      ypg[nt.NXP + i] = y2;
      srow[i] = (y1 + c.beta_n * (y1 - a1[cc])) + (y2 + c.beta_n * (y2 - a2[cc]));
      if (c.write_out) P.st.xo[(size_t)v * nt.NXP + i] = Xq[i];
    }
  }
  for (int j = lane; j < nt.nu; j += 32) {
    const T a3 = yc[2 * nt.NXP + j];
    const T w3 = a3 + c.beta * (a3 - yp[2 * nt.NXP + j]);
    const T uj = Uq[j];
    const T v3 = uj + w3 * ig;
    const T y3 = g * (v3 - fmin(fmax(v3, nt.umin[j]), nt.umax[j]));
    const unsigned long long r = abs_bits(y3 - w3);
    c.rbits = r > c.rbits ? r : c.rbits;
    ypg[2 * nt.NXP + j] = y3;
    srow[nt.NXP + j] = y3 + c.beta_n * (y3 - a3);
    if (c.write_out) P.st.uo[(size_t)v * nt.NUP + j] = uj;
  }
}

// Dual update of one node in delta form, one warp.  With c_lo/c_hi the
// box edges scaled by gamma and shifted by the state (input),
//   gamma e = w - clamp(w, c_lo, c_hi)           (distance-to-set prox, §4.3)
//   y+      = gamma e * min(1, W / |gamma e|)     (Moreau, §4.2; W = inf on y3)
// is evaluated on d = y+ - yb: the clamp decision compares ybh + dw with
// the edges, the value is dw - edge (or -ybh when the component leaves its
// edge), so the small increments of a small step gamma survive in FP32.
template <int MAXC>
__device__ void prox_node_warp_mixed(const KParams<float> &P, const NetDev<float> &nt,
                                     const MixedDev &mx, int v, const float *Uq, const float *Xq,
                                     const float *dc, const float *dp, const float *bh,
                                     const float *ur, const float *xr, FwdCtx<float> &c) {
  const int lane = threadIdx.x & 31;
  const float g = (float)P.gamma;
  float *dpg = c.yprv + (size_t)v * nt.YP;
  float g1[MAXC], g2[MAXC], w1[MAXC], w2[MAXC], a1[MAXC], a2[MAXC], h1[MAXC], h2[MAXC];
  float n1 = 0.f, n2 = 0.f;
#pragma unroll
  for (int cc = 0; cc < MAXC; ++cc) {
    const int i = lane + 32 * cc;
    g1[cc] = g2[cc] = w1[cc] = w2[cc] = a1[cc] = a2[cc] = h1[cc] = h2[cc] = 0.f;
    if (i < nt.nx) {
      a1[cc] = dc[i];
      a2[cc] = dc[nt.NXP + i];
      w1[cc] = a1[cc] + c.beta * (a1[cc] - dp[i]);
      w2[cc] = a2[cc] + c.beta * (a2[cc] - dp[nt.NXP + i]);
      h1[cc] = bh[i];
      h2[cc] = bh[nt.NXP + i];
      const float x = xr[i] + Xq[i];
      const float lo = g * (nt.xmin[i] - x), hi = g * (nt.xmax[i] - x);
      const float wa = h1[cc] + w1[cc];
      g1[cc] = wa > hi ? w1[cc] - hi : (wa < lo ? w1[cc] - lo : -h1[cc]);
      const float sa = g * (nt.xs[i] - x);
      g2[cc] = (h2[cc] + w2[cc]) < sa ? w2[cc] - sa : -h2[cc];
      const float t1 = h1[cc] + g1[cc], t2 = h2[cc] + g2[cc];
      n1 += t1 * t1;
      n2 += t2 * t2;
    }
  }
  n1 = warp_sum(n1);
  n2 = warp_sum(n2);
  const float q1 = n1 > 0.f ? nt.Wx * rsqrtf(n1) : 1.f;
  const float q2 = n2 > 0.f ? nt.Ws * rsqrtf(n2) : 1.f;
  float *srow = P.st.s + (size_t)v * nt.SP;
  float *swrow = mx.sw + (size_t)v * nt.SP;
#pragma unroll
  for (int cc = 0; cc < MAXC; ++cc) {
    const int i = lane + 32 * cc;
    if (i < nt.nx) {
      // scale toward the ball |y| <= W only when the ball is active (one
      // fixed rounding sequence, the same in every instantiation)
      const float d1 = q1 < 1.f ? __fmaf_rn(h1[cc], q1 - 1.f, __fmul_rn(g1[cc], q1)) : g1[cc];
      const float d2 = q2 < 1.f ? __fmaf_rn(h2[cc], q2 - 1.f, __fmul_rn(g2[cc], q2)) : g2[cc];
      unsigned long long r = abs_bits(d1 - w1[cc]), r2 = abs_bits(d2 - w2[cc]);
      r = r2 > r ? r2 : r;
      c.rbits = r > c.rbits ? r : c.rbits;
      dpg[i] = d1;
      dpg[nt.NXP + i] = d2;
      srow[i] = (d1 + c.beta_n * (d1 - a1[cc])) + (d2 + c.beta_n * (d2 - a2[cc]));
      if (c.write_out) swrow[i] = w1[cc] + w2[cc];
    }
  }
  for (int j = lane; j < nt.nu; j += 32) {
    const float a3 = dc[2 * nt.NXP + j];
    const float w3 = a3 + c.beta * (a3 - dp[2 * nt.NXP + j]);
    const float h3 = bh[2 * nt.NXP + j];
    const float u = ur[j] + Uq[j];
    const float lo = g * (nt.umin[j] - u), hi = g * (nt.umax[j] - u);
    const float wa = h3 + w3;
    const float d3 = wa > hi ? w3 - hi : (wa < lo ? w3 - lo : -h3);
    const unsigned long long r = abs_bits(d3 - w3);
    c.rbits = r > c.rbits ? r : c.rbits;
    dpg[2 * nt.NXP + j] = d3;
    srow[nt.NXP + j] = d3 + c.beta_n * (d3 - a3);
    if (c.write_out) swrow[nt.NXP + j] = w3;
  }
}

// Forward sweep along the path of chain k: its top ancestors (stage 1
// down; recomputed here, their per-node step done only by the owner) and
// then the chain itself, in segments of SEGF nodes.  Each segment first
// stages the rows it reads (z, the data terms, the dual rows of the owned
// nodes) into shared memory in one round of 16-byte loads, then
//   A (thread j): Zp += z_nu, u_nu = ub_nu - Zp          (path sum of z)
//   B (thread i): x_nu = x_a + Gd d_nu + B u_nu           (path sum of B u + Gd d)
//   C (warp per owned node): MODE 0 writes the outputs of a plain step,
//     MODE 1 the dual update, MODE 2 the dual update in delta form.
// Shared layout of a segment (elements): Zs, Us [SEGF][NUP]; Xs [SEGF][NXP];
// Bs [SEGF][NUP], Gs [SEGF][NXP] (ub, gb; in MODE 2 uref, xref of owned
// nodes); Yc, Yp [, Yh] [SEGF][YP] of owned nodes (MODE 1, 2).
constexpr int kFwdPlain = 0, kFwdApg = 1, kFwdMixed = 2;

template <typename T>
struct SegF {
  static constexpr int value = sizeof(T) == 8 ? 4 : 8;
};

__host__ __device__ inline int fwd_elems_per_node(int NXP, int NUP, int YP, int mode) {
  return 3 * NUP + 2 * NXP + (mode == 1 ? 2 * YP : (mode == 2 ? 3 * YP : 0));
}

template <typename T, int MODE, int C>
__device__ void chain_forward(const KParams<T> &P, int k, FwdCtx<T> &c, Smem<T> &sm,
                              const MixedDev *mx) {
  constexpr int SEGF = SegF<T>::value;
  const NetDev<T> &nt = *sm.net;
  const int tid = threadIdx.x, warp = tid >> 5, nw = blockDim.x >> 5;
  const int p0 = P.plan.ch_path_ptr[k], m = P.plan.ch_path_ptr[k + 1] - p0;
  const int own_from = P.plan.ch_own_from[k];
  const int start = P.plan.ch_start[k], K = m + P.plan.ch_len[k];
  const int *path = P.plan.ch_path + p0;
  T *Zs = sm.buf;
  T *Us = Zs + SEGF * nt.NUP;
  T *Xs = Us + SEGF * nt.NUP;
  T *Bs = Xs + SEGF * nt.NXP;
  T *Gs = Bs + SEGF * nt.NUP;
  T *Yc = Gs + SEGF * nt.NXP;
  T *Yp = Yc + SEGF * nt.YP;
  T *Yh = Yp + SEGF * nt.YP;
  int *nodes = sm.node, *owned = sm.node + kSeg;
  const bool data = (MODE == kFwdMixed) || !P.linear;
  T Zp[C], xa[C];
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const int i = tid + c * blockDim.x;
    Zp[c] = T(0);
    xa[c] = (i < nt.nx && !P.linear) ? P.st.xroot[i] : T(0);
  }
  for (int q0 = 0; q0 < K; q0 += SEGF) {
    const int ms = K - q0 < SEGF ? K - q0 : SEGF;
    if (tid == 0) {
      int mo = 0;
      for (int q = 0; q < ms; ++q) {
        const int gq = q0 + q;
        nodes[q] = gq < m ? path[gq] : start + (gq - m);
        if (gq >= m || gq >= own_from) owned[mo++] = q;
      }
      sm.flag[3] = mo;
      for (int q = 0; q < mo; ++q) nodes[SEGF + q] = nodes[owned[q]];
    }
    __syncthreads();
    const int mo = sm.flag[3];
    stage_rows(Zs, P.st.z, nt.NUP, nodes, ms, true);
    if constexpr (MODE == kFwdMixed) {
      stage_rows(Bs, mx->uref, nt.NUP, nodes + SEGF, mo, false);
      stage_rows(Gs, mx->xref, nt.NXP, nodes + SEGF, mo, false);
      stage_rows(Yc, c.ycur, nt.YP, nodes + SEGF, mo, false);
      stage_rows(Yp, c.yprv, nt.YP, nodes + SEGF, mo, false);
      stage_rows(Yh, (const T *)mx->ybh, nt.YP, nodes + SEGF, mo, false);
    } else {
      if (data) {
        stage_rows(Bs, P.st.ub, nt.NUP, nodes, ms, false);
        stage_rows(Gs, P.st.gb, nt.NXP, nodes, ms, false);
      }
      if constexpr (MODE == kFwdApg) {
        stage_rows(Yc, c.ycur, nt.YP, nodes + SEGF, mo, false);
        stage_rows(Yp, c.yprv, nt.YP, nodes + SEGF, mo, false);
      }
    }
    __syncthreads();
    for (int q = 0; q < ms; ++q) {
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const int j = tid + c * blockDim.x;
        if (j < nt.nu) {
          Zp[c] += Zs[q * nt.NUP + j];
          const T base = (data && MODE != kFwdMixed) ? Bs[q * nt.NUP + j] : T(0);
          Us[q * nt.NUP + j] = base - Zp[c];
        }
      }
    }
    __syncthreads();
    for (int q = 0; q < ms; ++q) {
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const int i = tid + c * blockDim.x;
        if (i < nt.nx) {
          T acc = (data && MODE != kFwdMixed) ? Gs[q * nt.NXP + i] : T(0);
          for (int e = nt.Br_ptr[i]; e < nt.Br_ptr[i + 1]; ++e)
            acc += nt.Br_val[e] * Us[q * nt.NUP + nt.Br_idx[e]];
          xa[c] += acc;
          Xs[q * nt.NXP + i] = xa[c];
        }
      }
    }
    __syncthreads();
    for (int o = warp; o < mo; o += nw) {
      const int q = owned[o];
      const int v = nodes[q];
      if constexpr (MODE == kFwdApg) {
        prox_node_warp<T, C>(P, nt, v, Us + q * nt.NUP, Xs + q * nt.NXP, Yc + o * nt.YP,
                                Yp + o * nt.YP, c);
      } else if constexpr (MODE == kFwdMixed) {
        prox_node_warp_mixed<C>(P, nt, *mx, v, Us + q * nt.NUP, Xs + q * nt.NXP, Yc + o * nt.YP,
                                   Yp + o * nt.YP, Yh + o * nt.YP, Bs + o * nt.NUP,
                                   Gs + o * nt.NXP, c);
      } else {
        const int lane = tid & 31;
        for (int j = lane; j < nt.nu; j += 32) {
          const T val = Us[q * nt.NUP + j];
          P.st.uo[(size_t)v * nt.NUP + j] = val;
          if (P.st.uo32) P.st.uo32[(size_t)v * nt.NUP + j] = (float)val;
        }
        for (int i = lane; i < nt.nx; i += 32) {
          const T val = Xs[q * nt.NXP + i];
          P.st.xo[(size_t)v * nt.NXP + i] = val;
          if (P.st.xo32) P.st.xo32[(size_t)v * nt.NXP + i] = (float)val;
        }
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// per-node steps of the mixed-precision scheme
// ---------------------------------------------------------------------------
// apply fn to every node whose per-node work chain k owns
template <typename F>
__device__ void for_owned(const PlanDev &pl, int k, F fn) {
  const int p0 = pl.ch_path_ptr[k], m = pl.ch_path_ptr[k + 1] - p0;
  for (int q = pl.ch_own_from[k]; q < m; ++q) fn(pl.ch_path[p0 + q]);
  const int start = pl.ch_start[k], L = pl.ch_len[k];
  for (int q = 0; q < L; ++q) fn(start + q);
}

// Refresh of node v by one warp: yb += d_new, d_old -= d_new, d_new = 0,
// ybh = fl32(yb); the FP64 step input s64 = (yb1 + yb2 | yb3) and the next
// FP32 step input dw = -beta_next d_old.
static __device__ void refresh_node(const MixedParams &M, int v, float *dnew, float *dold,
                             float beta_next) {
  const NetDev<float> &nt = M.f.net;
  const int lane = threadIdx.x & 31;
  const size_t ro = (size_t)v * nt.YP;
  for (int e = lane; e < nt.YP; e += 32) {
    const double yb = M.mx.yb[ro + e] + (double)dnew[ro + e];
    M.mx.yb[ro + e] = yb;
    M.mx.ybh[ro + e] = (float)yb;
    dold[ro + e] -= dnew[ro + e];
    dnew[ro + e] = 0.f;
  }
  __syncwarp();
  double *s64 = M.mx.s64 + (size_t)v * nt.SP;
  float *s32 = M.f.st.s + (size_t)v * nt.SP;
  for (int i = lane; i < nt.nx; i += 32) {
    s64[i] = M.mx.yb[ro + i] + M.mx.yb[ro + nt.NXP + i];
    s32[i] = -beta_next * (dold[ro + i] + dold[ro + nt.NXP + i]);
  }
  for (int j = lane; j < nt.nu; j += 32) {
    s64[nt.NXP + j] = M.mx.yb[ro + 2 * nt.NXP + j];
    s32[nt.NXP + j] = -beta_next * dold[ro + 2 * nt.NXP + j];
  }
}

// input of the final FP64 evaluation at w = yb + dw of the last iteration
static __device__ void final_node(const MixedParams &M, int v) {
  const NetDev<float> &nt = M.f.net;
  const int lane = threadIdx.x & 31;
  const size_t ro = (size_t)v * nt.YP;
  double *s64 = M.mx.s64 + (size_t)v * nt.SP;
  const float *sw = M.mx.sw + (size_t)v * nt.SP;
  for (int i = lane; i < nt.nx; i += 32)
    s64[i] = (M.mx.yb[ro + i] + M.mx.yb[ro + nt.NXP + i]) + (double)sw[i];
  for (int j = lane; j < nt.nu; j += 32)
    s64[nt.NXP + j] = M.mx.yb[ro + 2 * nt.NXP + j] + (double)sw[nt.NXP + j];
}

}  // namespace rn
