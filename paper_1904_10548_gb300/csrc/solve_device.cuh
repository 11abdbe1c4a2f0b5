// Device building blocks of the persistent solve kernels (solve_kernels.cu,
// mixed_kernels.cu, batch_kernels.cu): bounded waits, reductions, teams
// and shared-memory staging, the backward and forward sweeps over chains
// and groups of top nodes, and the dual update.
#pragma once

#include <cuda/atomic>

#include <type_traits>

#include "kernels.cuh"

// Each kernel unit is compiled once for a diagonal W_u (RN_DENSE = 0: F in
// its sparse Schur form) and once for a dense W_u (RN_DENSE = 1: F as a
// dense product), so that neither kernel carries the other's code.
#ifndef RN_DENSE
#define RN_DENSE 0
#endif

namespace rn {

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// %globaltimer into the k-th 64-bit stamp word at info + 4 (0: launch began,
// 1: block 0 finished)
__device__ __forceinline__ void stamp_time(int *info, int k) {
  reinterpret_cast<unsigned long long *>(info + 4)[k] = global_ns();
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

// bounded spin of one thread until *p >= target; false on timeout or error.
// The first wait to give up (after limit_ns) records `site` in *err (1 chain
// arrivals at a group, 2 a group's flag, 3 a root's flag, 4 the grid barrier).
static __device__ bool spin_geq(const unsigned *p, unsigned target, int *err, long long limit_ns,
                                int site) {
  if (ld_acquire(p) >= target) return true;
  const unsigned long long t0 = global_ns();
  while (true) {
    if (ld_acquire(p) >= target) return true;
    if (*(volatile int *)err != 0) return false;
    if ((long long)(global_ns() - t0) > limit_ns) {
      atomicCAS(err, 0, site);
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
// bits of |f| for an FP32 value (monotone in |f| as well); the FP32 path
// keeps its running maximum in these and widens it once per check
__device__ __forceinline__ unsigned long long abs_bits(float f) {
  return (unsigned long long)(__float_as_uint(f) & 0x7fffffffu);
}
__device__ __forceinline__ unsigned long long widen_bits(unsigned long long fbits) {
  return abs_bits((double)__uint_as_float((unsigned)fbits));
}

// ---------------------------------------------------------------------------
// teams, block layout and shared-memory carving
// ---------------------------------------------------------------------------
// A team is a warp-aligned set of threads with its own barrier: the block
// is tpb teams (one chain each; named barriers 1 .. tpb) or, for a group,
// one team of the whole block (barrier 0).
struct Team {
  int tid, nt, bar;
  __device__ __forceinline__ void sync() const {
    if (bar == 0)
      __syncthreads();
    else
      asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(nt) : "memory");
  }
  __device__ __forceinline__ int lane() const { return tid & 31; }
  __device__ __forceinline__ int warp() const { return tid >> 5; }
  __device__ __forceinline__ int nwarps() const { return nt >> 5; }
};

// a block of tpb chain teams: team t is threads [t tw, (t + 1) tw)
__device__ __forceinline__ Team chain_team(int tpb) {
  const int tw = blockDim.x / tpb;
  return Team{(int)threadIdx.x % tw, tw, 1 + (int)threadIdx.x / tw};
}
__device__ __forceinline__ Team block_team() { return Team{(int)threadIdx.x, (int)blockDim.x, 0}; }
__device__ __forceinline__ int team_index(int tpb) {
  return (int)threadIdx.x / (int)(blockDim.x / tpb);
}

// [header | network copy | team 0 | team 1 | ...]
struct BlockMem {
  unsigned long long *redu;  // 40 words for block reductions
  int *bflag;                // 8 block-wide flags
  unsigned char *net_raw;
  unsigned char *team0;
  int team_bytes;
  __device__ __forceinline__ unsigned char *team_raw(int t) const { return team0 + (size_t)t * team_bytes; }
};

__device__ __forceinline__ BlockMem block_mem(unsigned char *raw, int net_bytes, int team_bytes) {
  BlockMem b;
  b.redu = reinterpret_cast<unsigned long long *>(raw);
  b.bflag = reinterpret_cast<int *>(raw + 40 * sizeof(unsigned long long));
  b.net_raw = raw + kHdrBytes;
  b.team0 = raw + kHdrBytes + net_bytes;
  b.team_bytes = team_bytes;
  return b;
}

template <typename T>
struct Smem {
  T *buf;                    // work buffer (layouts in kernels.cuh)
  T *red;                    // 72
  int *flag;                 // 4
  int *node;                 // 2 x kSeg: node ids of a staged forward segment
  const NetDev<T> *net;      // the network data in use
};

template <typename T>
__device__ __forceinline__ Smem<T> carve(unsigned char *raw, int buf_elems, const NetDev<T> *net) {
  Smem<T> s;
  s.buf = reinterpret_cast<T *>(raw);
  s.red = s.buf + buf_elems;
  const size_t off = round16(sizeof(T) * ((size_t)buf_elems + 72));
  s.flag = reinterpret_cast<int *>(raw + off);
  s.node = s.flag + 4;
  s.net = net;
  return s;
}

// ---------------------------------------------------------------------------
// asynchronous staging global -> shared, 16 bytes per copy, all copies of
// a team in flight at once, read through L2 (the shared-memory carve-out
// leaves a small L1, which streamed rows would only evict).  cg marks the
// copies of data other blocks wrote during this launch, which must not
// come from L1.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp16(void *dst, const void *src, bool cg) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  (void)cg;  // always through L2: staged rows must not evict the small L1
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// n contiguous elements (n * sizeof(T) a multiple of 16)
template <typename T>
__device__ __forceinline__ void stage_span(T *dst, const T *src, int n, const Team &tm, bool cg) {
  constexpr int per = 16 / sizeof(T);
  for (int e = tm.tid; e < n / per; e += tm.nt) cp16(dst + e * per, src + e * per, cg);
}

// the first len elements of rows nodes[0..m) of src (pitch spitch) into
// rows of dst (pitch dpitch); len, pitches multiples of 16 bytes
template <typename T>
__device__ __forceinline__ void stage_rows(T *dst, int dpitch, const T *src, int spitch, int len,
                                           const int *nodes, int m, const Team &tm, bool cg) {
  constexpr int per = 16 / sizeof(T);
  const int nv = len / per;
  for (int e = tm.tid; e < m * nv; e += tm.nt) {
    const int q = e / nv, c = e - q * nv;
    cp16(dst + (size_t)q * dpitch + c * per, src + (size_t)nodes[q] * spitch + c * per, cg);
  }
}

// ---------------------------------------------------------------------------
// loops over (row, component) pairs: thread t takes component c0 + k cw of
// rows r0, r0 + rs, ... (cw the smallest power of two >= the component
// count, at most the team width), so consecutive lanes take consecutive
// components and a thread's rows are independent of each other
// ---------------------------------------------------------------------------
struct Map2 {
  int c0, cw, r0, rs;
};

__device__ __forceinline__ Map2 map2(const Team &tm, int nc) {
  int cw = nc <= 1 ? 1 : 1 << (32 - __clz(nc - 1));
  if (cw > tm.nt) cw = tm.nt;
  return Map2{tm.tid % cw, cw, tm.tid / cw, tm.nt / cw};
}

// ---------------------------------------------------------------------------
// One row of a compressed sparse matrix held in registers for a loop over
// many nodes (the structure is shared by all nodes): the first CAP entries
// in registers, any further ones read from the arrays.  dot() adds the
// entries in storage order, like a plain loop over the row.
// ---------------------------------------------------------------------------
template <typename T, int CAP>
struct Slice {
  int n, p;
  int idx[CAP];
  T val[CAP];
  __device__ __forceinline__ void load(const int *ptr, const int *ix, const T *vl, int r) {
    p = ptr[r];
    n = ptr[r + 1] - p;
#pragma unroll
    for (int k = 0; k < CAP; ++k) {
      idx[k] = k < n ? ix[p + k] : 0;
      val[k] = k < n ? vl[p + k] : T(0);
    }
  }
  // acc + sum_k val_k f(idx_k)
  template <typename F>
  __device__ __forceinline__ T dot(T acc, F f, const int *ix, const T *vl) const {
#pragma unroll
    for (int k = 0; k < CAP; ++k)
      if (k < n) acc += val[k] * f(idx[k]);
    for (int e = CAP; e < n; ++e) acc += vl[p + e] * f(ix[p + e]);
    return acc;
  }
};

}  // namespace rn
#include "dense_f.cuh"
namespace rn {

// ---------------------------------------------------------------------------
// z = F ghat / (2p) in place for m rows (ghat at offset NXP of row(q)),
// F ghat = W^-1 (ghat - E' S^-1 E W^-1 ghat) for a diagonal W_u; eb, fb:
// m x NEP work space.  A dense W_u takes the dense product (dense_f.cuh).
// ---------------------------------------------------------------------------
template <typename T, typename RowF>
__device__ void apply_F(const NetDev<T> &nt, int m, RowF row, const T *i2p, T *eb, T *fb,
                        const Team &tm) {
#if RN_DENSE
  if constexpr (sizeof(T) == 8)
    apply_F_dense(nt, m, row, i2p, tm);
  else
    apply_F_tc(nt, m, row, i2p, tm);
  (void)eb;
  (void)fb;
#else
  const int ne = nt.ne, nu = nt.nu, NXP = nt.NXP, NEP = nt.NEP;
  const int *Er_ptr = nt.Er_ptr, *Er_idx = nt.Er_idx, *Ec_ptr = nt.Ec_ptr, *Ec_idx = nt.Ec_idx;
  const T *Erw_val = nt.Erw_val, *Ec_val = nt.Ec_val, *winv = nt.winv, *Sinv = nt.Sinv;
  if (ne > 0) {
    const Map2 a = map2(tm, ne);
    for (int r = a.c0; r < ne; r += a.cw) {
      Slice<T, 6> er;
      er.load(Er_ptr, Er_idx, Erw_val, r);
#pragma unroll 2
      for (int q = a.r0; q < m; q += a.rs) {
        const T *g = row(q) + NXP;
        const T acc = er.dot(T(0), [&](int j) { return g[j]; }, Er_idx, Erw_val);
        eb[q * NEP + r] = acc;
      }
    }
    tm.sync();
    for (int r = a.c0; r < ne; r += a.cw) {
      const T *Si = Sinv + (size_t)r * ne;
#pragma unroll 2
      for (int q = a.r0; q < m; q += a.rs) {
        const T *e = eb + q * NEP;
        T acc = T(0);
        for (int c = 0; c < ne; ++c) acc += Si[c] * e[c];
        fb[q * NEP + r] = acc;
      }
    }
    tm.sync();
  }
  const Map2 b = map2(tm, nu);
  for (int j = b.c0; j < nu; j += b.cw) {
    Slice<T, 2> ec;
    ec.load(Ec_ptr, Ec_idx, Ec_val, j);
    const T wj = winv[j];
#pragma unroll 4
    for (int q = b.r0; q < m; q += b.rs) {
      T *g = row(q) + NXP;
      const T *f = fb + q * NEP;
      T acc = g[j];
#pragma unroll
      for (int k = 0; k < 2; ++k)
        if (k < ec.n) acc -= ec.val[k] * f[ec.idx[k]];
      for (int e = 2; e < ec.n; ++e) acc -= Ec_val[ec.p + e] * f[Ec_idx[ec.p + e]];
      g[j] = (wj * acc) * i2p[q];
    }
  }
#endif
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
  T *Erw_val = Ec_val + nnzE;
  T *winv = Erw_val + nnzE, *Sinv = winv + nu, *xmin = Sinv + (size_t)ne * ne, *xmax = xmin + nx;
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
  cpv(Erw_val, g.Erw_val, nnzE);
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
    s->Erw_val = Erw_val;
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

// state of the forward sweep of one iteration
template <typename T>
struct FwdCtx {
  const T *ycur;
  T *yprv;
  T beta, beta_n;
  bool write_out;
  bool avg;                  // update the averaged primal with weight theta
  double theta;
  unsigned long long rbits;  // running max of |y+ - w| (abs_bits of T)
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
      if (c.avg) {
        double *xa = P.st.xavg + (size_t)v * nt.NXP + i;
        *xa = (1.0 - c.theta) * *xa + c.theta * (double)Xq[i];
      }
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
    if (c.avg) {
      double *ua = P.st.uavg + (size_t)v * nt.NUP + j;
      *ua = (1.0 - c.theta) * *ua + c.theta * (double)uj;
    }
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
      if (c.avg) {
        double *xa = P.st.xavg + (size_t)v * nt.NXP + i;
        *xa = (1.0 - c.theta) * *xa + c.theta * (double)x;
      }
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
    if (c.avg) {
      double *ua = P.st.uavg + (size_t)v * nt.NUP + j;
      *ua = (1.0 - c.theta) * *ua + c.theta * (double)u;
    }
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

// ---------------------------------------------------------------------------
// chain backward, critical part: the subtree sums at the chain head,
//   lambda_h = sum_q (w1 + w2)_q,  ghat_h = sum_q w3_q + B' sum_q lambda_q,
// published in up[k] (then one arrival at the group's counter).  The rows
// of the segment nearest the head stay in shared memory with lambda_q in
// place of (w1 + w2)_q for chain_rest.  Thread t owns components t + c nt.
// ---------------------------------------------------------------------------
template <typename T, int C>
__device__ void chain_head(const KParams<T> &P, int k, const Smem<T> &sm, const Team &tm) {
  const NetDev<T> &nt = *sm.net;
  const int SP = nt.SP, NXP = nt.NXP, nx = nt.nx, nu = nt.nu;
  const int start = P.plan.ch_start[k], L = P.plan.ch_len[k], segb = P.segb;
  const int g = P.plan.ch_group[k];
  T *rows = sm.buf;
  T lam[C], Lam[C], g3[C];
#pragma unroll
  for (int c = 0; c < C; ++c) lam[c] = Lam[c] = g3[c] = T(0);
  for (int hi = L; hi > 0; hi -= segb) {
    const int lo = hi > segb ? hi - segb : 0, m = hi - lo;
    if (hi < L) tm.sync();
    stage_span(rows, P.st.s + (size_t)(start + lo) * SP, m * SP, tm, false);
    cp_wait();
    tm.sync();
    for (int q = m - 1; q >= 0; --q) {
      T *row = rows + q * SP;
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const int i = tm.tid + c * tm.nt;
        if (i < nx) {
          lam[c] += row[i];
          row[i] = lam[c];
          Lam[c] += lam[c];
        }
        if (i < nu) g3[c] += row[NXP + i];
      }
    }
  }
  if (g < 0) return;  // below the root: nobody reads the head sums
  T *vec = rows + chain_vec_off(segb, SP, nt.NEP);
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const int i = tm.tid + c * tm.nt;
    if (i < nx) vec[i] = Lam[c];
  }
  tm.sync();
  const int *Bc_ptr = nt.Bc_ptr, *Bc_idx = nt.Bc_idx;
  const T *Bc_val = nt.Bc_val;
  T *out = P.st.up + (size_t)k * SP;
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const int i = tm.tid + c * tm.nt;
    if (i < nx) out[i] = lam[c];
    if (i < nu) {
      Slice<T, 2> bc;
      bc.load(Bc_ptr, Bc_idx, Bc_val, i);
      out[NXP + i] = bc.dot(g3[c], [&](int t) { return vec[t]; }, Bc_idx, Bc_val);
    }
  }
  tm.sync();
  if (tm.tid == 0) {
    __threadfence();
    atomicAdd(P.st.count + g, 1u);
  }
}

// ---------------------------------------------------------------------------
// chain backward and forward, local part (no dependence on the top nodes):
// per node ghat_q = sum_{r >= q} (w3_r + B' lambda_r), z_q = F ghat_q/(2p),
// then from the head down U_q = ub_q - sum_{r <= q} z_r and
// X_q = sum_{r <= q} (B U_r + Gd d_r), written to ux (X | U).  With the
// path sum Z_p and state x_p at the chain's parent the forward sweep is
// then u_q = U_q - Z_p, x_q = x_p + X_q - (q + 1) B Z_p.  Per-node
// products run one warp per node, the sums along the chain one thread per
// component.  keep: the rows chain_head left in shared memory are this
// chain's (one segment).
// ---------------------------------------------------------------------------
template <typename T, int C>
__device__ void chain_rest(const KParams<T> &P, int k, const Smem<T> &sm, const Team &tm, bool keep) {
  const NetDev<T> &nt = *sm.net;
  const int SP = nt.SP, NXP = nt.NXP, NUP = nt.NUP, nx = nt.nx, nu = nt.nu, NEP = nt.NEP;
  const int *Bc_ptr = nt.Bc_ptr, *Bc_idx = nt.Bc_idx, *Br_ptr = nt.Br_ptr, *Br_idx = nt.Br_idx;
  const T *Bc_val = nt.Bc_val, *Br_val = nt.Br_val;
  const int start = P.plan.ch_start[k], L = P.plan.ch_len[k], segb = P.segb;
  const bool multi = L > segb, data = !P.linear;
  const Map2 mu = map2(tm, nu), mx = map2(tm, nx);
  T *rows = sm.buf;
  T *eb = rows + round4(segb * SP), *fb = eb + segb * NEP, *i2p = fb + segb * NEP;
  T accL[C], accG[C];
#pragma unroll
  for (int c = 0; c < C; ++c) accL[c] = accG[c] = T(0);
  // leaf -> head: ghat and z per node
  for (int hi = L; hi > 0; hi -= segb) {
    const int lo = hi > segb ? hi - segb : 0, m = hi - lo;
    tm.sync();
    if (multi || !keep) {
      stage_span(rows, P.st.s + (size_t)(start + lo) * SP, m * SP, tm, false);
      cp_wait();
      tm.sync();
      for (int q = m - 1; q >= 0; --q) {
        T *row = rows + q * SP;
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const int i = tm.tid + c * tm.nt;
          if (i < nx) {
            accL[c] += row[i];
            row[i] = accL[c];
          }
        }
      }
    }
    for (int q = tm.tid; q < m; q += tm.nt) i2p[q] = P.st.inv2p[start + lo + q];
    tm.sync();
    for (int j = mu.c0; j < nu; j += mu.cw) {  // w3 + B' lambda per node
      Slice<T, 2> bc;
      bc.load(Bc_ptr, Bc_idx, Bc_val, j);
#pragma unroll 4
      for (int q = mu.r0; q < m; q += mu.rs) {
        T *row = rows + q * SP;
        row[NXP + j] = bc.dot(row[NXP + j], [&](int t) { return row[t]; }, Bc_idx, Bc_val);
      }
    }
    tm.sync();
    for (int q = m - 1; q >= 0; --q) {  // suffix sums along the chain
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const int j = tm.tid + c * tm.nt;
        if (j < nu) {
          accG[c] += rows[q * SP + NXP + j];
          rows[q * SP + NXP + j] = accG[c];
        }
      }
    }
    tm.sync();
    apply_F(nt, m, [=](int q) { return rows + q * SP; }, i2p, eb, fb, tm);
    tm.sync();
    if (lo > 0) {
      T *z = P.st.z + (size_t)(start + lo) * NUP;
      for (int e = tm.tid; e < m * nu; e += tm.nt) {
        const int q = e / nu, j = e - q * nu;
        z[(size_t)q * NUP + j] = rows[q * SP + NXP + j];
      }
    }
  }
  // head -> leaf: local path sums (the head segment is still in place)
  T accZ[C], accX[C];
#pragma unroll
  for (int c = 0; c < C; ++c) accZ[c] = accX[c] = T(0);
  for (int lo = 0; lo < L; lo += segb) {
    const int m = L - lo < segb ? L - lo : segb;
    if (lo > 0) {
      tm.sync();
      const T *z = P.st.z + (size_t)(start + lo) * NUP;
      constexpr int per = 16 / sizeof(T);
      const int nv = NUP / per;
      for (int e = tm.tid; e < m * nv; e += tm.nt) {
        const int q = e / nv, c = e - q * nv;
        cp16(rows + q * SP + NXP + c * per, z + (size_t)q * NUP + c * per, false);
      }
      cp_wait();
      tm.sync();
    }
    for (int q = 0; q < m; ++q) {  // U = ub - path sums of z
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const int j = tm.tid + c * tm.nt;
        if (j < nu) {
          accZ[c] += rows[q * SP + NXP + j];
          const T base = data ? P.st.ub[(size_t)(start + lo + q) * NUP + j] : T(0);
          rows[q * SP + NXP + j] = base - accZ[c];
        }
      }
    }
    tm.sync();
    for (int i = mx.c0; i < nx; i += mx.cw) {  // B U + Gd d per node
      Slice<T, 6> br;
      br.load(Br_ptr, Br_idx, Br_val, i);
#pragma unroll 4
      for (int q = mx.r0; q < m; q += mx.rs) {
        T *row = rows + q * SP;
        const T base = data ? P.st.gb[(size_t)(start + lo + q) * NXP + i] : T(0);
        row[i] = br.dot(base, [&](int t) { return row[NXP + t]; }, Br_idx, Br_val);
      }
    }
    tm.sync();
    for (int q = 0; q < m; ++q) {  // prefix sums along the chain
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const int i = tm.tid + c * tm.nt;
        if (i < nx) {
          accX[c] += rows[q * SP + i];
          rows[q * SP + i] = accX[c];
        }
      }
    }
    tm.sync();
    {
      using V = typename std::conditional<sizeof(T) == 8, double2, float4>::type;
      constexpr int per = 16 / sizeof(T);
      const V *src = reinterpret_cast<const V *>(rows);
      V *dst = reinterpret_cast<V *>(P.st.ux + (size_t)(start + lo) * SP);
      for (int e = tm.tid; e < m * SP / per; e += tm.nt) dst[e] = src[e];
    }
  }
}

// ---------------------------------------------------------------------------
// The root of a split stage-1 subtree (one node), whole block, computed by
// every part of it once all parts have published their top nodes' sums
// (the parts' hp rows of this step's buffer): own terms plus the
// children's sums, F, then (x | Z) with the tree root as parent, left in W's
// first row for the part's forward levels; the first part also publishes it
// in ux for the chain that owns the root node.  W: rows of work space
// (children + 1), eb/fb/i2p as for F.
// ---------------------------------------------------------------------------
template <typename T>
__device__ void root_compute(const KParams<T> &P, int root, const Smem<T> &sm, const Team &tm,
                             unsigned step, T *W, T *eb, T *fb, T *i2p, bool publish) {
  const NetDev<T> &nt = *sm.net;
  const PlanDev &pl = P.plan;
  const int SP = nt.SP, NXP = nt.NXP, NUP = nt.NUP, nx = nt.nx, nu = nt.nu;
  const int v = pl.r_node[root], q0 = pl.r_hp[root], np = pl.r_hp[root + 1] - q0;
  const bool data = !P.linear;
  T *Rr = W, *Hp = W + SP;
  // the root's own row from the copy its first part took before arriving:
  // the chain that owns the root may already have written the next
  // iteration's row into s by the time a late part gets here
  const T *hpb = P.st.hp + (size_t)(step & 1u) * pl.hp_rows * SP;
  stage_span(Rr, hpb + (size_t)(pl.r_hp[pl.n_roots] + root) * SP, SP, tm, true);
  stage_span(Hp, hpb + (size_t)q0 * SP, np * SP, tm, true);
  if (tm.tid == 0) i2p[0] = P.st.inv2p[v];
  cp_wait();
  tm.sync();
  for (int i = tm.tid; i < nx; i += tm.nt) {
    T acc = Rr[i];
    for (int q = 0; q < np; ++q) acc += Hp[(size_t)q * SP + i];
    Rr[i] = acc;
  }
  tm.sync();
  for (int j = tm.tid; j < nu; j += tm.nt) {
    Slice<T, 2> bc;
    bc.load(nt.Bc_ptr, nt.Bc_idx, nt.Bc_val, j);
    T acc = bc.dot(Rr[NXP + j], [&](int t) { return Rr[t]; }, nt.Bc_idx, nt.Bc_val);
    for (int q = 0; q < np; ++q) acc += Hp[(size_t)q * SP + NXP + j];
    Rr[NXP + j] = acc;
  }
  tm.sync();
  apply_F(nt, 1, [=](int) { return Rr; }, i2p, eb, fb, tm);
  tm.sync();
  // Z = z (the parent is the tree root), x = x0 + Gd d + B u, in place of
  // the state sums (which no thread reads any more)
  for (int i = tm.tid; i < nx; i += tm.nt) {
    Slice<T, 6> br;
    br.load(nt.Br_ptr, nt.Br_idx, nt.Br_val, i);
    T acc = data ? P.st.xroot[i] + P.st.gb[(size_t)v * NXP + i] : T(0);
    const T *ubv = P.st.ub + (size_t)v * NUP;
    Rr[i] = br.dot(acc, [&](int t) { return (data ? ubv[t] : T(0)) - Rr[NXP + t]; }, nt.Br_idx,
                   nt.Br_val);
  }
  tm.sync();
  if (publish) {
    T *out = P.st.ux + (size_t)v * SP;
    for (int e = tm.tid; e < NXP + NUP; e += tm.nt) out[e] = Rr[e];
  }
}

// ---------------------------------------------------------------------------
// One group of top nodes, whole block: wait for the group's chains, sum
// the subtree level by level from the deepest, apply F to every node, roll
// the path sums Z and states x back down and publish (x | Z) in ux, then
// release the group's flag.  The group's descriptor (levels, parents,
// children in local indices) is staged with its rows; rows of a group
// larger than the shared-memory capacity live in up[K + v].
//
// A group that is a part of a split stage-1 subtree sums the part,
// publishes the sums at its top nodes in hp and its arrival, applies F to
// its rows, waits until every part of the root has arrived, completes the
// root node itself (root_compute; every part does, so no part waits for
// another's result) and rolls down from it.  phase -1 does all of this in
// one call (a block with one work item); a block with several items (the
// batched kernel) calls phase 0 (up to the arrival, z rows left in ux) for
// all its groups before phase 1 (the wait, the root and the roll-down), so
// that no part waits for a part that its own block has still to start.
// False on timeout.
// ---------------------------------------------------------------------------
template <typename T>
__device__ bool group_step(const KParams<T> &P, int g, const Smem<T> &sm, const Team &tm,
                           unsigned step, int phase = -1) {
  const NetDev<T> &nt = *sm.net;
  const PlanDev &pl = P.plan;
  const int SP = nt.SP, NXP = nt.NXP, NUP = nt.NUP, nx = nt.nx, nu = nt.nu, NEP = nt.NEP;
  const int *Bc_ptr = nt.Bc_ptr, *Bc_idx = nt.Bc_idx, *Br_ptr = nt.Br_ptr, *Br_idx = nt.Br_idx;
  const T *Bc_val = nt.Bc_val, *Br_val = nt.Br_val;
  const int g0 = pl.g_node[g], c0 = pl.g_chain[2 * g], c1 = pl.g_chain[2 * g + 1];
  const int m = pl.g_node[g + 1] - g0;
  const int d0 = pl.g_desc_ptr[g], dn = pl.g_desc_ptr[g + 1] - d0;
  const bool data = !P.linear;
  const int gcap = P.gcap, hchunk = P.hchunk, fbr = P.fbrows;
  const Map2 mx = map2(tm, nx), mu = map2(tm, nu);
  T *R = sm.buf;
  T *H = R + (size_t)gcap * SP;
  T *eb = H + (size_t)hchunk * SP, *fb = eb + fbr * NEP, *i2p = fb + fbr * NEP;
  int *desc = reinterpret_cast<int *>(eb + round4(2 * fbr * NEP + fbr));
  // all rows in shared memory, or (a group larger than gcap) all in up[K + v]
  T *const rb = m <= gcap ? R : P.st.up + (size_t)(pl.n_chains + g0) * SP;
  const int root = pl.g_root[g];
  T *base = nullptr;  // (x | Z) at the parent of the group's top node, if not the tree root
  int nl = 0;
  const int *lvl = nullptr, *par = nullptr;
  const int p0 = root >= 0 ? pl.r_part[2 * root] : 0, p1 = root >= 0 ? pl.r_part[2 * root + 1] : 0;
  // every part waits until all parts of its root have arrived (bounded)
  auto wait_parts = [&]() {
    if (tm.tid == 0) {
      bool ok = true;
      for (int q = p0; q < p1 && ok; ++q)
        ok = spin_geq(P.st.arrive + q, step + 1u, P.st.err, P.st.wait_ns, 3);
      sm.flag[0] = ok;
    }
    tm.sync();
    return sm.flag[0] != 0;
  };
  if (phase == 1) {
    // second half of a part (a block that holds several items): the
    // descriptor and the z rows the first half left in ux, then the root
    if (root < 0) return true;
    if (!wait_parts()) return false;
    for (int e = tm.tid; e < dn / 4; e += tm.nt) cp16(desc + 4 * e, pl.g_desc + d0 + 4 * e, false);
    constexpr int per = 16 / sizeof(T);
    const int nv = NUP / per;
    if (m <= gcap) {
      for (int e = tm.tid; e < m * nv; e += tm.nt) {
        const int li = e / nv, c = e - li * nv;
        cp16(rb + (size_t)li * SP + NXP + c * per,
             P.st.ux + (size_t)(g0 + li) * SP + NXP + c * per, true);
      }
    } else {
      // rows in global memory: the asynchronous copy writes shared memory only
      for (int e = tm.tid; e < m * NUP; e += tm.nt) {
        const int li = e / NUP, j = e - li * NUP;
        rb[(size_t)li * SP + NXP + j] = __ldcg(P.st.ux + (size_t)(g0 + li) * SP + NXP + j);
      }
    }
    cp_wait();
    tm.sync();
    nl = desc[1];
    lvl = desc + 4;
    par = lvl + nl + 1;
    root_compute(P, root, sm, tm, step, H, eb, fb, i2p, g == p0);
    base = H;
  } else {
  // all chains of the group have arrived; the counter restarts for the
  // next evaluation (no chain arrives again before the flag below)
  if (tm.tid == 0) {
    sm.flag[0] = spin_geq(P.st.count + g, (unsigned)(c1 - c0), P.st.err, P.st.wait_ns, 1);
    if (sm.flag[0]) atomicExch(P.st.count + g, 0u);
  }
  tm.sync();
  if (!sm.flag[0]) return false;
  // own terms (w1 + w2 | w3) of the group's nodes, the descriptor, heads
  if (m <= gcap) {
    stage_span(R, P.st.s + (size_t)g0 * SP, m * SP, tm, true);
  } else {
    for (int e = tm.tid; e < m * SP; e += tm.nt) rb[e] = __ldcg(P.st.s + (size_t)g0 * SP + e);
  }
  for (int e = tm.tid; e < dn / 4; e += tm.nt) cp16(desc + 4 * e, pl.g_desc + d0 + 4 * e, false);
  const int nch = c1 - c0;
  // chain heads: all at once (added in the first backward pass below), or
  // in chunks added to their parents first
  const bool heads_all = nch <= hchunk;
  for (int h0 = 0; h0 < nch; h0 += hchunk) {
    const int h1 = nch - h0 < hchunk ? nch : h0 + hchunk;
    if (h0 > 0) tm.sync();
    stage_span(H, P.st.up + (size_t)(c0 + h0) * SP, (h1 - h0) * SP, tm, true);
    if (heads_all) break;
    cp_wait();
    tm.sync();
    const int nl = desc[1], ncn = desc[3];
    const int *tcp = desc + 4 + (nl + 1) + m;
    const int *ccp = tcp + (m + 1) + tcp[m], *ccl = ccp + m + 1, *cn = ccl + ccp[m];
    // heads into their parents (fixed order of the chain children)
    for (int o = mx.r0; o < ncn; o += mx.rs) {
      const int li = cn[o], cs = ccp[li], ce = ccp[li + 1];
      T *r = rb + (size_t)li * SP;
      for (int i = mx.c0; i < nx; i += mx.cw) {
        T acc = T(0);
        bool any = false;
        for (int c = cs; c < ce; ++c) {
          const int kk = ccl[c];
          if (kk >= h0 && kk < h1) {
            acc += H[(size_t)(kk - h0) * SP + i];
            any = true;
          }
        }
        if (any) r[i] += acc;
      }
    }
    for (int o = mu.r0; o < ncn; o += mu.rs) {
      const int li = cn[o], cs = ccp[li], ce = ccp[li + 1];
      T *r = rb + (size_t)li * SP + NXP;
      for (int j = mu.c0; j < nu; j += mu.cw) {
        T acc = T(0);
        bool any = false;
        for (int c = cs; c < ce; ++c) {
          const int kk = ccl[c];
          if (kk >= h0 && kk < h1) {
            acc += H[(size_t)(kk - h0) * SP + NXP + j];
            any = true;
          }
        }
        if (any) r[j] += acc;
      }
    }
  }
  cp_wait();
  tm.sync();
  nl = desc[1];
  lvl = desc + 4;
  par = lvl + nl + 1;
  const int *tcp = par + m, *tcl = tcp + m + 1;
  const int *ccp = tcl + tcp[m], *ccl = ccp + m + 1;
  // children table (one row of kChildSlotsDev references per node)
  const int *cn_end = ccl + ccp[m] + desc[3];
  const int thdr = round4((int)(cn_end - desc));
  const int *ctab = desc + desc[thdr];
  const bool table = desc[thdr + 1] != 0 && heads_all;
  // backward over the levels, deepest first
  for (int l = nl - 1; l >= 0; --l) {
    const int a = lvl[l], b = lvl[l + 1];
    if (table) {
      // four nodes per thread at a time: all child references, then all
      // child values, then the sums (no store before the last load)
      constexpr int NB = 4;
      for (int i = mx.c0; i < nx; i += mx.cw) {
        for (int l0 = a + mx.r0; l0 < b; l0 += NB * mx.rs) {
          T acc[NB];
#pragma unroll
          for (int k = 0; k < NB; ++k) {
            const int li = l0 + k * mx.rs;
            acc[k] = T(0);
            if (li < b) {
              const int4 c0v = reinterpret_cast<const int4 *>(ctab + li * kChildSlotsDev)[0];
              const int4 c1v = reinterpret_cast<const int4 *>(ctab + li * kChildSlotsDev)[1];
              const int cr[8] = {c0v.x, c0v.y, c0v.z, c0v.w, c1v.x, c1v.y, c1v.z, c1v.w};
              T v = rb[(size_t)li * SP + i];
#pragma unroll
              for (int e = 0; e < 8; ++e) {
                const int x = cr[e];
                if (x != -1) v += x >= 0 ? rb[(size_t)x * SP + i] : H[(size_t)(-2 - x) * SP + i];
              }
              acc[k] = v;
            }
          }
#pragma unroll
          for (int k = 0; k < NB; ++k) {
            const int li = l0 + k * mx.rs;
            if (li < b) rb[(size_t)li * SP + i] = acc[k];
          }
        }
      }
      tm.sync();
      for (int j = mu.c0; j < nu; j += mu.cw) {
        Slice<T, 2> bc;
        bc.load(Bc_ptr, Bc_idx, Bc_val, j);
        for (int l0 = a + mu.r0; l0 < b; l0 += NB * mu.rs) {
          T acc[NB];
#pragma unroll
          for (int k = 0; k < NB; ++k) {
            const int li = l0 + k * mu.rs;
            acc[k] = T(0);
            if (li < b) {
              const int4 c0v = reinterpret_cast<const int4 *>(ctab + li * kChildSlotsDev)[0];
              const int4 c1v = reinterpret_cast<const int4 *>(ctab + li * kChildSlotsDev)[1];
              const int cr[8] = {c0v.x, c0v.y, c0v.z, c0v.w, c1v.x, c1v.y, c1v.z, c1v.w};
              const T *r = rb + (size_t)li * SP;
              T v = r[NXP + j];
              // heads (negative references) before B' lambda, top children after
#pragma unroll
              for (int e = 0; e < 8; ++e)
                if (cr[e] < -1) v += H[(size_t)(-2 - cr[e]) * SP + NXP + j];
              v = bc.dot(v, [&](int t) { return r[t]; }, Bc_idx, Bc_val);
#pragma unroll
              for (int e = 0; e < 8; ++e)
                if (cr[e] >= 0) v += rb[(size_t)cr[e] * SP + NXP + j];
              acc[k] = v;
            }
          }
#pragma unroll
          for (int k = 0; k < NB; ++k) {
            const int li = l0 + k * mu.rs;
            if (li < b) rb[(size_t)li * SP + NXP + j] = acc[k];
          }
        }
      }
      tm.sync();
      continue;
    }
#pragma unroll 2
    for (int li = a + mx.r0; li < b; li += mx.rs) {
      T *r = rb + (size_t)li * SP;
      const int ts = tcp[li], te = tcp[li + 1];
      const int cs = heads_all ? ccp[li] : 0, ce = heads_all ? ccp[li + 1] : 0;
      for (int i = mx.c0; i < nx; i += mx.cw) {
        T acc = r[i];
        for (int c = cs; c < ce; ++c) acc += H[(size_t)ccl[c] * SP + i];
        for (int c = ts; c < te; ++c) acc += rb[(size_t)tcl[c] * SP + i];
        r[i] = acc;
      }
    }
    tm.sync();
    for (int j = mu.c0; j < nu; j += mu.cw) {
      Slice<T, 2> bc;
      bc.load(Bc_ptr, Bc_idx, Bc_val, j);
#pragma unroll 2
      for (int li = a + mu.r0; li < b; li += mu.rs) {
        T *r = rb + (size_t)li * SP;
        const int ts = tcp[li], te = tcp[li + 1];
        const int cs = heads_all ? ccp[li] : 0, ce = heads_all ? ccp[li + 1] : 0;
        T acc = r[NXP + j];
        for (int c = cs; c < ce; ++c) acc += H[(size_t)ccl[c] * SP + NXP + j];
        acc = bc.dot(acc, [&](int t) { return r[t]; }, Bc_idx, Bc_val);
        for (int c = ts; c < te; ++c) acc += rb[(size_t)tcl[c] * SP + NXP + j];
        r[NXP + j] = acc;
      }
    }
    tm.sync();
  }
  if (root >= 0) {
    // a part: its top nodes' sums to the root (buffer of this step's
    // parity: a part that runs one step ahead writes the other one), then
    // its arrival
    const int m0 = lvl[1] - lvl[0];
    T *hpb = P.st.hp + (size_t)(step & 1u) * pl.hp_rows * SP;
    T *hpg = hpb + (size_t)pl.g_hp[g] * SP;
    for (int e = tm.tid; e < m0 * SP; e += tm.nt) hpg[e] = rb[e];
    if (g == p0) {
      // the first part copies the root's own row while no chain can write it
      const T *src = P.st.s + (size_t)pl.r_node[root] * SP;
      T *dst = hpb + (size_t)(pl.r_hp[pl.n_roots] + root) * SP;
      for (int e = tm.tid; e < SP; e += tm.nt) dst[e] = __ldcg(src + e);
    }
    tm.sync();
    if (tm.tid == 0) {
      __threadfence();
      st_release(P.st.arrive + g, step + 1u);
    }
  }
  // z = F ghat / (2p) at every node of the group
  for (int q0 = 0; q0 < m; q0 += fbr) {
    const int mm = m - q0 < fbr ? m - q0 : fbr;
    if (q0 > 0) tm.sync();
    for (int q = tm.tid; q < mm; q += tm.nt) i2p[q] = P.st.inv2p[g0 + q0 + q];
    tm.sync();
    apply_F(nt, mm, [=](int q) { return rb + (size_t)(q0 + q) * SP; }, i2p, eb, fb, tm);
  }
  tm.sync();
  if (root >= 0) {
    if (phase == 0) {
      // first half of a part: leave the z rows in ux for the second half
      constexpr int per = 16 / sizeof(T);
      const int nv = NUP / per;
      using V = typename std::conditional<sizeof(T) == 8, double2, float4>::type;
      for (int e = tm.tid; e < m * nv; e += tm.nt) {
        const int li = e / nv, c = e - li * nv;
        reinterpret_cast<V *>(P.st.ux + (size_t)(g0 + li) * SP + NXP)[c] =
            reinterpret_cast<const V *>(rb + (size_t)li * SP + NXP)[c];
      }
      return true;
    }
    // every part completes the root itself once all parts have arrived
    if (!wait_parts()) return false;
    root_compute(P, root, sm, tm, step, H, eb, fb, i2p, g == p0);
    base = H;
  }
  }
  // forward over the levels: Z_v = Z_a(v) + z_v, x_v = x_a(v) + B u_v + Gd d_v
  // (four nodes per thread at a time: loads, then sums, then stores)
  constexpr int NF = 4;
  for (int l = 0; l < nl; ++l) {
    const int a = lvl[l], b = lvl[l + 1];
    for (int j = mu.c0; j < nu; j += mu.cw) {
      for (int l0 = a + mu.r0; l0 < b; l0 += NF * mu.rs) {
        T zv[NF];
#pragma unroll
        for (int k = 0; k < NF; ++k) {
          const int li = l0 + k * mu.rs;
          zv[k] = T(0);
          if (li < b) {
            const int pa = par[li];
            const T own = rb[(size_t)li * SP + NXP + j];
            zv[k] = pa >= 0 ? own + rb[(size_t)pa * SP + NXP + j]
                            : (base ? own + base[NXP + j] : own);
          }
        }
#pragma unroll
        for (int k = 0; k < NF; ++k) {
          const int li = l0 + k * mu.rs;
          if (li < b) rb[(size_t)li * SP + NXP + j] = zv[k];
        }
      }
    }
    tm.sync();
    for (int i = mx.c0; i < nx; i += mx.cw) {
      Slice<T, 6> br;
      br.load(Br_ptr, Br_idx, Br_val, i);
      for (int l0 = a + mx.r0; l0 < b; l0 += NF * mx.rs) {
        T xv[NF];
#pragma unroll
        for (int k = 0; k < NF; ++k) {
          const int li = l0 + k * mx.rs;
          xv[k] = T(0);
          if (li < b) {
            const int pa = par[li], v = g0 + li;
            const T *r = rb + (size_t)li * SP;
            T acc = pa >= 0 ? rb[(size_t)pa * SP + i]
                            : (base ? base[i] : (data ? P.st.xroot[i] : T(0)));
            if (data) acc += P.st.gb[(size_t)v * NXP + i];
            const T *ubv = P.st.ub + (size_t)v * NUP;
            xv[k] = br.dot(acc, [&](int t) { return (data ? ubv[t] : T(0)) - r[NXP + t]; }, Br_idx,
                           Br_val);
          }
        }
#pragma unroll
        for (int k = 0; k < NF; ++k) {
          const int li = l0 + k * mx.rs;
          if (li < b) rb[(size_t)li * SP + i] = xv[k];
        }
      }
    }
    tm.sync();
  }
  // publish (x | Z)
  {
    using V = typename std::conditional<sizeof(T) == 8, double2, float4>::type;
    constexpr int per = 16 / sizeof(T);
    const int nv = SP / per;
    V *dst = reinterpret_cast<V *>(P.st.ux + (size_t)g0 * SP);
    for (int e = tm.tid; e < m * nv; e += tm.nt) {
      const int li = e / nv, c = e - li * nv;
      dst[e] = reinterpret_cast<const V *>(rb + (size_t)li * SP)[c];
    }
  }
  tm.sync();
  if (tm.tid == 0) {
    __threadfence();
    st_release(P.st.flags + g, step + 1u);
  }
  return true;
}

// ---------------------------------------------------------------------------
// forward sweep of chain k after its group: the top nodes it owns, then its
// own nodes.  Warp w takes nodes w, w + nw, ...; it stages a node's rows
// into one of its P.fslots slots (the copies of the next nodes in flight
// while it works on the current one), forms (x | u) in place from the published
// (x | Z) of a top node (u = ub - Z) or from the chain's local sums, then
//   MODE 0 writes the outputs of a plain step,
//   MODE 1 the dual update, MODE 2 the dual update in delta form.
// Slot layout (elements): row [SP]; Yc, Yp [YP] (MODE 1); Yc, Yp, Yh [YP],
// Ur [NUP], Xr [NXP] (MODE 2).  False on timeout.
// ---------------------------------------------------------------------------
constexpr int kFwdPlain = 0, kFwdApg = 1, kFwdMixed = 2;

__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait_group() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <typename T, int MODE, int C>
__device__ bool chain_forward(const KParams<T> &P, int k, FwdCtx<T> &c, const Smem<T> &sm,
                              const Team &tm, const MixedDev *mx, unsigned step) {
  const NetDev<T> &nt = *sm.net;
  const PlanDev &pl = P.plan;
  const int SP = nt.SP, NXP = nt.NXP, NUP = nt.NUP, YP = nt.YP, nx = nt.nx, nu = nt.nu;
  const int start = pl.ch_start[k], L = pl.ch_len[k], g = pl.ch_group[k], par = pl.ch_parent[k];
  const int own0 = pl.ch_own_ptr[k], nown = pl.ch_own_ptr[k + 1] - own0;
  const bool data = !P.linear;
  const int lane = tm.lane(), warp = tm.warp(), nw = tm.nwarps(), S = P.fslots;
  T *xp = sm.buf, *Zp = xp + NXP, *BZ = Zp + NUP;
  const int fpn = fwd_elems_per_node(NXP, NUP, YP, SP, MODE);
  T *slots = sm.buf + round4(2 * NXP + NUP) + (size_t)warp * S * fpn;
  // nodes in the order the warps take them: the chain's own nodes (head to
  // leaf) first, then the top nodes the chain owns
  const int K = nown + L;
  constexpr int per = 16 / sizeof(T);
  auto node_of = [&](int q) { return q < L ? start + q : pl.ch_own[own0 + (q - L)]; };
  auto copy_row = [&](T *dst, const T *src, int len, bool cg) {
    for (int e = lane; e < len / per; e += 32) cp16(dst + e * per, src + e * per, cg);
  };
  auto issue = [&](int q, T *dst) {
    const int v = node_of(q);
    copy_row(dst, P.st.ux + (size_t)v * SP, SP, q >= L);
    if constexpr (MODE == kFwdApg) {
      copy_row(dst + SP, c.ycur + (size_t)v * YP, YP, false);
      copy_row(dst + SP + YP, c.yprv + (size_t)v * YP, YP, false);
    } else if constexpr (MODE == kFwdMixed) {
      copy_row(dst + SP, c.ycur + (size_t)v * YP, YP, false);
      copy_row(dst + SP + YP, c.yprv + (size_t)v * YP, YP, false);
      copy_row(dst + SP + 2 * YP, mx->ybh + (size_t)v * YP, YP, false);
      copy_row(dst + SP + 3 * YP, mx->uref + (size_t)v * NUP, NUP, false);
      copy_row(dst + SP + 3 * YP + NUP, mx->xref + (size_t)v * NXP, NXP, false);
    }
    cp_commit();
  };
  // ring of S slots per warp: node t of the warp (q = warp + t nw) lives
  // in slot t % S; up to S - 1 nodes ahead are in flight.  The first nodes
  // of the chain itself (their rows come from this team and from the
  // previous iteration) are requested before the wait for the group; a
  // top node's row is published by its group and requested after it.
  int issued = 0;
  tm.sync();  // the team's chain rows (chain_rest) are written
  for (; issued < S && warp + issued * nw < L; ++issued)
    issue(warp + issued * nw, slots + (size_t)issued * fpn);
  if (g >= 0) {
    if (tm.tid == 0) sm.flag[1] = spin_geq(P.st.flags + g, step + 1u, P.st.err, P.st.wait_ns, 2);
    tm.sync();
    if (!sm.flag[1]) {
      cp_wait_group<0>();
      return false;
    }
    const T *src = P.st.ux + (size_t)par * SP;
    for (int e = tm.tid; e < NXP + NUP; e += tm.nt) xp[e] = __ldcg(src + e);
  } else {
    for (int e = tm.tid; e < NXP + NUP; e += tm.nt)
      xp[e] = (e < nx && data) ? P.st.xroot[e] : T(0);
  }
  tm.sync();
  {
    const int *Br_ptr = nt.Br_ptr, *Br_idx = nt.Br_idx;
    const T *Br_val = nt.Br_val;
    for (int i = tm.tid; i < nx; i += tm.nt) {
      Slice<T, 6> br;
      br.load(Br_ptr, Br_idx, Br_val, i);
      BZ[i] = br.dot(T(0), [&](int t) { return Zp[t]; }, Br_idx, Br_val);
    }
  }
  tm.sync();
  for (; issued < S && warp + issued * nw < K; ++issued)
    issue(warp + issued * nw, slots + (size_t)issued * fpn);
  int t = 0;
  for (int q = warp; q < K; q += nw, ++t) {
    T *r = slots + (size_t)(t % S) * fpn;
    const int ahead = issued - t - 1;  // groups allowed to stay pending
    if (ahead >= 2)
      cp_wait_group<2>();
    else if (ahead == 1)
      cp_wait_group<1>();
    else
      cp_wait_group<0>();
    __syncwarp();
    const int v = node_of(q);
    if (q >= L) {
      for (int j = lane; j < nu; j += 32) {
        const T base = data ? P.st.ub[(size_t)v * NUP + j] : T(0);
        r[NXP + j] = base - r[NXP + j];
      }
    } else {
      const T depth = (T)(q + 1);
      for (int i = lane; i < nx; i += 32) r[i] = (xp[i] + r[i]) - depth * BZ[i];
      for (int j = lane; j < nu; j += 32) r[NXP + j] -= Zp[j];
    }
    __syncwarp();
    if constexpr (MODE == kFwdApg) {
      prox_node_warp<T, C>(P, nt, v, r + NXP, r, r + SP, r + SP + YP, c);
    } else if constexpr (MODE == kFwdMixed) {
      prox_node_warp_mixed<C>(P, nt, *mx, v, r + NXP, r, r + SP, r + SP + YP, r + SP + 2 * YP,
                              r + SP + 3 * YP, r + SP + 3 * YP + NUP, c);
    } else {
      for (int j = lane; j < nu; j += 32) {
        const T val = r[NXP + j];
        P.st.uo[(size_t)v * NUP + j] = val;
        if (P.st.uo32) P.st.uo32[(size_t)v * NUP + j] = (float)val;
      }
      for (int i = lane; i < nx; i += 32) {
        const T val = r[i];
        P.st.xo[(size_t)v * NXP + i] = val;
        if (P.st.xo32) P.st.xo32[(size_t)v * NXP + i] = (float)val;
      }
    }
    __syncwarp();
    const int qn = warp + issued * nw;
    if (qn < K) {
      issue(qn, r);
      ++issued;
    }
  }
  tm.sync();
  return true;
}

// ---------------------------------------------------------------------------
// per-node steps of the mixed-precision scheme
// ---------------------------------------------------------------------------
// apply fn to every node whose per-node work chain k owns
template <typename F>
__device__ void for_owned(const PlanDev &pl, int k, F fn) {
  for (int q = pl.ch_own_ptr[k]; q < pl.ch_own_ptr[k + 1]; ++q) fn(pl.ch_own[q]);
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


// ---------------------------------------------------------------------------
// one evaluation of the dual gradient (with the per-node step of MODE) by a
// block whose items are i = blockIdx.x, blockIdx.x + gridDim.x, ...: items
// below n_groups are groups (whole block), the rest sets of tpb chains
// (one per team).  Phases: chain heads, groups, the chains' local parts,
// the forward sweeps.
// keep: the block holds one chain set and no group.
// False (for the calling team) on timeout.
// ---------------------------------------------------------------------------
template <typename T, int MODE, int C>
__device__ bool eval_step(const KParams<T> &P, FwdCtx<T> &c, const MixedDev *mx,
                          const Smem<T> &smc, const Smem<T> &smg, const Team &tc,
                          const Team &tb, unsigned step, bool keep) {
  const int G = P.plan.n_groups, K = P.plan.n_chains, tpb = P.tpb;
  const int n_items = G + (K + tpb - 1) / tpb, team = team_index(tpb);
  bool ok = true;
  for (int i = blockIdx.x; i < n_items; i += gridDim.x) {
    const int k = tpb * (i - G) + team;
    if (i >= G && k < K) chain_head<T, C>(P, k, smc, tc);
  }
  for (int i = blockIdx.x; i < G; i += gridDim.x) {
    __syncthreads();
    if (!group_step<T>(P, i, smg, tb, step)) ok = false;
  }
  for (int i = blockIdx.x; i < n_items; i += gridDim.x) {
    const int k = tpb * (i - G) + team;
    if (i >= G && k < K) chain_rest<T, C>(P, k, smc, tc, keep);
  }
  for (int i = blockIdx.x; i < n_items && ok; i += gridDim.x) {
    const int k = tpb * (i - G) + team;
    if (i >= G && k < K) ok = chain_forward<T, MODE, C>(P, k, c, smc, tc, mx, step);
  }
  return ok;
}

// the block agrees on whether a wait has given up anywhere (every thread
// of the block calls it)
__device__ __forceinline__ bool block_err(const BlockMem &bm, int *err) {
  __syncthreads();
  if (threadIdx.x == 0) bm.bflag[0] = *(volatile int *)err;
  __syncthreads();
  const bool e = bm.bflag[0] != 0;
  __syncthreads();
  return e;
}

// residual check: the grid-wide maximum of r (bits of a non-negative
// value) lands in res[ci]; false on timeout (every thread calls it)
__device__ __forceinline__ bool grid_check(const BlockMem &bm, unsigned long long r,
                                           unsigned long long *res, unsigned *barrier, int ci,
                                           int *err, long long wait_ns) {
  r = block_max_u64(r, bm.redu);
  if (threadIdx.x == 0) {
    atomicMax(res + ci, r);
    __threadfence();
    atomicAdd(barrier, 1u);
    bm.bflag[1] = spin_geq(barrier, (unsigned)(ci + 1) * gridDim.x, err, wait_ns, 4);
  }
  __syncthreads();
  const bool ok = bm.bflag[1] != 0;
  __syncthreads();
  return ok;
}

}  // namespace rn
