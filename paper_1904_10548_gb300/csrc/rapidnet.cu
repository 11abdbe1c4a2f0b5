// C ABI of the solver: factor step, solve, dual gradient (include/rapidnet.h).
//
// Host orchestration around the persistent kernel of solve_kernels.cu:
//   factor:  validation, tree schedule, Schur complement S = E W^-1 E' and
//            S^-1 in FP64 (Cholesky), uploads, step size by power iteration
//   solve:   per-solve constants -> x*(0) (one dual-gradient evaluation
//            with the data terms) -> APG iterations -> outputs, cost,
//            input-box violation, optional duality gap.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <vector>

#include "kernels.cuh"
#include "pernode.h"
#include "rn_internal.h"

using namespace rn;
static_assert(kChildSlots == kChildSlotsDev, "children table width differs between host and device");

// ---------------------------------------------------------------------------
// helper kernels (FP64)
// ---------------------------------------------------------------------------
namespace {

constexpr int kRedBlocks = 304;  // partial sums of the node reductions

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// kq = q - W^-1 E' S^-1 E q: the input q projected on ker E in the W metric
// (dense W_u: kq = q - Gm E q with Gm = W^-1 E' S^-1)
__global__ void k_kq(NetDev<double> nt, const double *q, double *kq) {
  extern __shared__ double sh[];
  double *e = sh, *f = sh + nt.NEP;
  const int tid = threadIdx.x;
  for (int r = tid; r < nt.ne; r += blockDim.x) {
    double acc = 0.0;
    for (int k = nt.Er_ptr[r]; k < nt.Er_ptr[r + 1]; ++k) acc += nt.Er_val[k] * q[nt.Er_idx[k]];
    e[r] = acc;
  }
  __syncthreads();
  if (nt.Gm) {
    for (int j = tid; j < nt.nu; j += blockDim.x) {
      double acc = 0.0;
      for (int r = 0; r < nt.ne; ++r) acc += nt.Gm[(size_t)j * nt.ne + r] * e[r];
      kq[j] = q[j] - acc;
    }
    return;
  }
  for (int r = tid; r < nt.ne; r += blockDim.x) {
    double acc = 0.0;
    for (int c = 0; c < nt.ne; ++c) acc += nt.Sinv[(size_t)r * nt.ne + c] * e[c];
    f[r] = acc;
  }
  __syncthreads();
  for (int j = tid; j < nt.nu; j += blockDim.x) {
    double acc = 0.0;
    for (int k = nt.Ec_ptr[j]; k < nt.Ec_ptr[j + 1]; ++k) acc += nt.Ec_val[k] * f[nt.Ec_idx[k]];
    kq[j] = q[j] - nt.winv[j] * acc;
  }
}

struct PrepArgs {
  const int *perm;
  const double *prob;
  const double *demand, *alpha, *alpha0, *kq;
  const int *Gd_ptr, *Gd_idx;
  const double *Gd_val;
  const int *Ed_ptr, *Ed_idx;
  const double *Ed_val;
  double W_alpha;
  int nd;
};

// per node: s = (0 | c0), ub = ubar + kq, gb = Gd d, with
// c0 = p W_alpha (alpha0 + alpha_nu) and ubar = -W^-1 E' S^-1 Ed d
__global__ void k_prep(NetDev<double> nt, PrepArgs a, int n, double *s, double *ub, double *gb) {
  extern __shared__ double sh[];
  double *e = sh, *f = sh + nt.NEP;
  const int tid = threadIdx.x;
  for (int v = blockIdx.x + 1; v < n; v += gridDim.x) {
    const int b = a.perm[v];
    const double *d = a.demand + (size_t)b * a.nd;
    const double *al = a.alpha + (size_t)b * nt.nu;
    const double p = a.prob[v];
    for (int r = tid; r < nt.ne; r += blockDim.x) {
      double acc = 0.0;
      for (int k = a.Ed_ptr[r]; k < a.Ed_ptr[r + 1]; ++k) acc += a.Ed_val[k] * d[a.Ed_idx[k]];
      e[r] = acc;
    }
    __syncthreads();
    for (int r = tid; r < nt.ne && !nt.Gm; r += blockDim.x) {
      double acc = 0.0;
      for (int c = 0; c < nt.ne; ++c) acc += nt.Sinv[(size_t)r * nt.ne + c] * e[c];
      f[r] = acc;
    }
    __syncthreads();
    for (int j = tid; j < nt.NUP; j += blockDim.x) {
      double c0 = 0.0, u = 0.0;
      if (j < nt.nu) {
        c0 = p * a.W_alpha * (a.alpha0[j] + al[j]);
        double acc = 0.0;
        if (nt.Gm) {  // dense W_u: W^-1 E' S^-1 (Ed d)
          for (int r = 0; r < nt.ne; ++r) acc += nt.Gm[(size_t)j * nt.ne + r] * e[r];
          u = a.kq[j] - acc;
        } else {
          for (int k = nt.Ec_ptr[j]; k < nt.Ec_ptr[j + 1]; ++k)
            acc += nt.Ec_val[k] * f[nt.Ec_idx[k]];
          u = a.kq[j] - nt.winv[j] * acc;
        }
      }
      s[(size_t)v * nt.SP + nt.NXP + j] = c0;
      ub[(size_t)v * nt.NUP + j] = u;
    }
    for (int i = tid; i < nt.NXP; i += blockDim.x) {
      double g = 0.0;
      if (i < nt.nx)
        for (int k = a.Gd_ptr[i]; k < a.Gd_ptr[i + 1]; ++k) g += a.Gd_val[k] * d[a.Gd_idx[k]];
      gb[(size_t)v * nt.NXP + i] = g;
      s[(size_t)v * nt.SP + i] = 0.0;
    }
    __syncthreads();
  }
}

// y^0 = y^{-1} = y_warm (or 0) in the internal layout, s = (y1 + y2 | y3)
__global__ void k_init_apg(NetDev<double> nt, const int *perm, int n, const double *y_warm,
                           double *ya, double *yb, double *s) {
  const int ny = 2 * nt.nx + nt.nu;
  for (int v = blockIdx.x + 1; v < n; v += gridDim.x) {
    const double *src = y_warm ? y_warm + (size_t)perm[v] * ny : nullptr;
    for (int e = threadIdx.x; e < nt.YP; e += blockDim.x) {
      double val = 0.0;
      if (src) {
        if (e < nt.nx) val = src[e];
        else if (e >= nt.NXP && e < nt.NXP + nt.nx) val = src[nt.nx + e - nt.NXP];
        else if (e >= 2 * nt.NXP && e < 2 * nt.NXP + nt.nu) val = src[2 * nt.nx + e - 2 * nt.NXP];
      }
      ya[(size_t)v * nt.YP + e] = val;
      yb[(size_t)v * nt.YP + e] = val;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nt.SP; e += blockDim.x) {
      const double *y = ya + (size_t)v * nt.YP;
      double val = 0.0;
      if (e < nt.nx) val = y[e] + y[nt.NXP + e];
      else if (e >= nt.NXP && e < nt.NXP + nt.nu) val = y[2 * nt.NXP + (e - nt.NXP)];
      s[(size_t)v * nt.SP + e] = val;
    }
  }
}

// s = (y1 + y2 | y3) from a dual vector given in breadth-first rows
__global__ void k_s_from_w(NetDev<double> nt, const int *perm, int n, const double *w, double *s) {
  const int ny = 2 * nt.nx + nt.nu;
  for (int v = blockIdx.x + 1; v < n; v += gridDim.x) {
    const double *src = w + (size_t)perm[v] * ny;
    for (int e = threadIdx.x; e < nt.SP; e += blockDim.x) {
      double val = 0.0;
      if (e < nt.nx) val = src[e] + src[nt.nx + e];
      else if (e >= nt.NXP && e < nt.NXP + nt.nu) val = src[2 * nt.nx + (e - nt.NXP)];
      s[(size_t)v * nt.SP + e] = val;
    }
  }
}

// internal rows -> breadth-first rows of u, x (and y if given); root rows q, x0, 0
__global__ void k_gather(NetDev<double> nt, const int *perm, int n, const double *uo,
                         const double *xo, const double *yin, const double *q, const double *x0,
                         double *u, double *x, double *y) {
  const int ny = 2 * nt.nx + nt.nu;
  for (int v = blockIdx.x; v < n; v += gridDim.x) {
    const int b = perm[v];
    for (int j = threadIdx.x; j < nt.nu; j += blockDim.x)
      u[(size_t)b * nt.nu + j] = v == 0 ? q[j] : uo[(size_t)v * nt.NUP + j];
    for (int i = threadIdx.x; i < nt.nx; i += blockDim.x)
      x[(size_t)b * nt.nx + i] = v == 0 ? x0[i] : xo[(size_t)v * nt.NXP + i];
    if (y) {
      for (int e = threadIdx.x; e < ny; e += blockDim.x) {
        double val = 0.0;
        if (v != 0) {
          const double *r = yin + (size_t)v * nt.YP;
          if (e < nt.nx) val = r[e];
          else if (e < 2 * nt.nx) val = r[nt.NXP + e - nt.nx];
          else val = r[2 * nt.NXP + e - 2 * nt.nx];
        }
        y[(size_t)b * ny + e] = val;
      }
    }
  }
}

struct ReduceArgs {
  const int *parent, *perm;
  const double *prob, *alpha, *alpha0, *wdiag, *q;
  const double *wdense;    // dense W_u (nu x nu) or null (diagonal: wdiag)
  const double *uo, *xo;   // internal rows
  const double *y;         // internal rows (gap) or null
  double W_alpha;
  int mode;                // 0: cost + ubox, 1: gap terms
};

// Per-node terms reduced over the tree, one warp per node.
// mode 0: [smooth cost, soft cost, u-box violation (max)]
// mode 1: [gap terms, domain violation count]
__global__ void k_node_reduce(NetDev<double> nt, ReduceArgs a, int n, double *partial) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __shared__ double sh[3][32];
  double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0;
  for (int v = 1 + blockIdx.x * nw + warp; v < n; v += gridDim.x * nw) {
    const double *u = a.uo + (size_t)v * nt.NUP;
    const double *x = a.xo + (size_t)v * nt.NXP;
    double d1 = 0.0, d2 = 0.0, t = 0.0, m = 0.0;
    if (a.mode == 0) {
      const int pa = a.parent[v];
      const double *ua = pa == 0 ? a.q : a.uo + (size_t)pa * nt.NUP;
      const double *al = a.alpha + (size_t)a.perm[v] * nt.nu;
      const double p = a.prob[v];
      for (int j = lane; j < nt.nu; j += 32) {
        const double du = u[j] - ua[j];
        double wdu = a.wdiag[j] * du;
        if (a.wdense) {
          wdu = 0.0;
          for (int k = 0; k < nt.nu; ++k) wdu += a.wdense[(size_t)j * nt.nu + k] * (u[k] - ua[k]);
        }
        t += p * (a.W_alpha * (a.alpha0[j] + al[j]) * u[j] + wdu * du);
        m = fmax(m, fmax(nt.umin[j] - u[j], u[j] - nt.umax[j]));
      }
      for (int i = lane; i < nt.nx; i += 32) {
        const double e1 = x[i] - fmin(fmax(x[i], nt.xmin[i]), nt.xmax[i]);
        const double e2 = fmin(x[i] - nt.xs[i], 0.0);
        d1 += e1 * e1;
        d2 += e2 * e2;
      }
      t = warp_sum(t);
      d1 = warp_sum(d1);
      d2 = warp_sum(d2);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
      if (lane == 0) {
        acc0 += t;
        acc1 += nt.Wx * sqrt(d1) + nt.Ws * sqrt(d2);
        acc2 = fmax(acc2, m);
      }
    } else {
      // soft(x) - <y1 + y2, x> - <y3, u> + sigma_X(y1) + <y2, xs> + sigma_U(y3)
      const double *y = a.y + (size_t)v * nt.YP;
      double n1 = 0.0, n2 = 0.0, pos = 0.0;
      for (int i = lane; i < nt.nx; i += 32) {
        const double e1 = x[i] - fmin(fmax(x[i], nt.xmin[i]), nt.xmax[i]);
        const double e2 = fmin(x[i] - nt.xs[i], 0.0);
        d1 += e1 * e1;
        d2 += e2 * e2;
        const double y1 = y[i], y2 = y[nt.NXP + i];
        n1 += y1 * y1;
        n2 += y2 * y2;
        pos = fmax(pos, y2);
        t += -(y1 + y2) * x[i] + fmax(y1 * nt.xmax[i], y1 * nt.xmin[i]) + y2 * nt.xs[i];
      }
      for (int j = lane; j < nt.nu; j += 32) {
        const double y3 = y[2 * nt.NXP + j];
        t += -y3 * u[j] + fmax(y3 * nt.umax[j], y3 * nt.umin[j]);
      }
      t = warp_sum(t);
      d1 = warp_sum(d1);
      d2 = warp_sum(d2);
      n1 = warp_sum(n1);
      n2 = warp_sum(n2);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) pos = fmax(pos, __shfl_xor_sync(0xffffffffu, pos, o));
      if (lane == 0) {
        acc0 += t + nt.Wx * sqrt(d1) + nt.Ws * sqrt(d2);
        const bool bad = sqrt(n1) > nt.Wx * (1.0 + 1e-9) + 1e-300 ||
                         sqrt(n2) > nt.Ws * (1.0 + 1e-9) + 1e-300 ||
                         pos > 1e-9 * fmax(nt.Ws, 1e-300);
        acc1 += bad ? 1.0 : 0.0;
      }
    }
  }
  if (lane == 0) {
    sh[0][warp] = acc0;
    sh[1][warp] = acc1;
    sh[2][warp] = acc2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int w = 0; w < nw; ++w) {
      s0 += sh[0][w];
      s1 += sh[1][w];
      s2 = fmax(s2, sh[2][w]);
    }
    partial[3 * blockIdx.x + 0] = s0;
    partial[3 * blockIdx.x + 1] = s1;
    partial[3 * blockIdx.x + 2] = s2;
  }
}

// sum (max for the third entry) of the per-block partials, one warp, fixed order
__global__ void k_final_reduce(const double *partial, int nb, double *out) {
  const int lane = threadIdx.x;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (int b = lane; b < nb; b += 32) {
    s0 += partial[3 * b];
    s1 += partial[3 * b + 1];
    s2 = fmax(s2, partial[3 * b + 2]);
  }
  s0 = warp_sum(s0);
  s1 = warp_sum(s1);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s2 = fmax(s2, __shfl_xor_sync(0xffffffffu, s2, o));
  if (lane == 0) {
    out[0] = s0;
    out[1] = s1;
    out[2] = s2;
  }
}

// Power iteration on M v = -H x_lin(v).  The iterate v is never stored:
// only s = (v1 + v2 | v3) enters the dual gradient.
//   start: v = 1 + SplitMix64 over (breadth-first node, component), not
//          normalised (the estimate after one step does not depend on it)
//   step:  v <- M v / |M v| with M v = -(x, x, u), |M v|^2 = sum 2|x|^2 + |u|^2
__device__ __forceinline__ double splitmix_unit(unsigned long long i) {
  unsigned long long z = (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  return (double)(z >> 11) * 0x1.0p-53;
}

__global__ void k_power_start(NetDev<double> nt, const int *perm, int n, double *s) {
  const int ny = 2 * nt.nx + nt.nu;
  for (int v = blockIdx.x + 1; v < n; v += gridDim.x) {
    const unsigned long long base = (unsigned long long)(perm[v] - 1) * ny;
    for (int e = threadIdx.x; e < nt.SP; e += blockDim.x) {
      double val = 0.0;
      if (e < nt.nx)
        val = (1.0 + splitmix_unit(base + e)) + (1.0 + splitmix_unit(base + nt.nx + e));
      else if (e >= nt.NXP && e < nt.NXP + nt.nu)
        val = 1.0 + splitmix_unit(base + 2 * nt.nx + (e - nt.NXP));
      s[(size_t)v * nt.SP + e] = val;
    }
  }
}

// per-block partial sums of sum_nu 2 |x_nu|^2 + |u_nu|^2
__global__ void k_norm2(NetDev<double> nt, int n, const double *uo, const double *xo,
                        double *partial) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int v = blockIdx.x + 1; v < n; v += gridDim.x) {
    for (int j = threadIdx.x; j < nt.nu; j += blockDim.x) {
      const double a = uo[(size_t)v * nt.NUP + j];
      acc += a * a;
    }
    for (int i = threadIdx.x; i < nt.nx; i += blockDim.x) {
      const double a = xo[(size_t)v * nt.NXP + i];
      acc += 2.0 * a * a;
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    partial[3 * blockIdx.x] = t;
    partial[3 * blockIdx.x + 1] = 0.0;
    partial[3 * blockIdx.x + 2] = 0.0;
  }
}

// s = (-2x | -u) / sqrt(norm2)
__global__ void k_power_scale(NetDev<double> nt, int n, const double *uo, const double *xo,
                              const double *norm2, double *s) {
  const double inv = 1.0 / sqrt(norm2[0]);
  for (int v = blockIdx.x + 1; v < n; v += gridDim.x) {
    for (int e = threadIdx.x; e < nt.SP; e += blockDim.x) {
      double val = 0.0;
      if (e < nt.nx) val = -2.0 * xo[(size_t)v * nt.NXP + e] * inv;
      else if (e >= nt.NXP && e < nt.NXP + nt.nu) val = -uo[(size_t)v * nt.NUP + (e - nt.NXP)] * inv;
      s[(size_t)v * nt.SP + e] = val;
    }
  }
}

// mixed precision: base yb = y_warm (or 0), ybh = fl32(yb), deltas 0,
// FP64 step input s64 = (yb1 + yb2 | yb3), FP32 step input 0
__global__ void k_mixed_init(NetDev<double> nt, const int *perm, int n, const double *y_warm,
                             double *yb, float *ybh, float *da, float *db, double *s64,
                             float *s32) {
  const int ny = 2 * nt.nx + nt.nu;
  for (int v = blockIdx.x + 1; v < n; v += gridDim.x) {
    const double *src = y_warm ? y_warm + (size_t)perm[v] * ny : nullptr;
    for (int e = threadIdx.x; e < nt.YP; e += blockDim.x) {
      double val = 0.0;
      if (src) {
        if (e < nt.nx) val = src[e];
        else if (e >= nt.NXP && e < nt.NXP + nt.nx) val = src[nt.nx + e - nt.NXP];
        else if (e >= 2 * nt.NXP && e < 2 * nt.NXP + nt.nu) val = src[2 * nt.nx + e - 2 * nt.NXP];
      }
      const size_t o = (size_t)v * nt.YP + e;
      yb[o] = val;
      ybh[o] = (float)val;
      da[o] = 0.f;
      db[o] = 0.f;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nt.SP; e += blockDim.x) {
      const double *y = yb + (size_t)v * nt.YP;
      double val = 0.0;
      if (e < nt.nx) val = y[e] + y[nt.NXP + e];
      else if (e >= nt.NXP && e < nt.NXP + nt.nu) val = y[2 * nt.NXP + (e - nt.NXP)];
      s64[(size_t)v * nt.SP + e] = val;
      s32[(size_t)v * nt.SP + e] = 0.f;
    }
  }
}

// final dual y = yb + d into breadth-first rows (FP64)
__global__ void k_gather_mixed_y(NetDev<double> nt, const int *perm, int n, const double *yb,
                                 const float *d, double *y) {
  const int ny = 2 * nt.nx + nt.nu;
  for (int v = blockIdx.x; v < n; v += gridDim.x) {
    const int b = perm[v];
    for (int e = threadIdx.x; e < ny; e += blockDim.x) {
      double val = 0.0;
      if (v != 0) {
        const int c = e < nt.nx ? e : (e < 2 * nt.nx ? nt.NXP + e - nt.nx : 2 * nt.NXP + e - 2 * nt.nx);
        val = yb[(size_t)v * nt.YP + c] + (double)d[(size_t)v * nt.YP + c];
      }
      y[(size_t)b * ny + e] = val;
    }
  }
}

// the same for a batched solve: the last iteration's parity from the
// problem's info on the device (iterations in info[0])
__global__ void k_gather_mixed_y_batch(NetDev<double> nt, const int *perm, int n, const double *yb,
                                       const float *da, const float *db, const int *info,
                                       double *y) {
  const float *d = ((info[0] - 1) & 1) ? da : db;
  const int ny = 2 * nt.nx + nt.nu;
  for (int v = blockIdx.x; v < n; v += gridDim.x) {
    const int b = perm[v];
    for (int e = threadIdx.x; e < ny; e += blockDim.x) {
      double val = 0.0;
      if (v != 0) {
        const int c = e < nt.nx ? e : (e < 2 * nt.nx ? nt.NXP + e - nt.nx : 2 * nt.NXP + e - 2 * nt.nx);
        val = yb[(size_t)v * nt.YP + c] + (double)d[(size_t)v * nt.YP + c];
      }
      y[(size_t)b * ny + e] = val;
    }
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// factor handle
// ---------------------------------------------------------------------------
struct rn_factor {
  unsigned long long serial = 0;  // unique per handle of the process (batch caches)
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  rn_opts opts{};
  Plan plan;
  int nx = 0, nu = 0, nd = 0, ne = 0, NXP = 0, NUP = 0, SP = 0, YP = 0, NEP = 0;
  double W_alpha = 0.0, Ws = 0.0, Wx = 0.0;
  double gamma = 0.0, L = 0.0;
  double collapse_dev = 0.0;  // factor check of the shared operator
  // launch layout of the FP64 kernel (APG and plain evaluations)
  int grid = 0, block = 0, maxc = 2, tw = 64, tpb = 2;
  size_t smem = 0;
  Sizes sz_d{};   // its buffers
  // launch layout of the mixed-precision kernel (FP32 iterations, FP64 steps)
  Sizes sz_f{}, sz_dm{};
  int net_bytes_d = 0, net_bytes_f = 0;
  std::vector<void *> allocs;
  long long bytes = 0;
  NetDev<double> net{};
  PlanDev pd{};
  StateDev<double> st{};
  // mixed precision: FP32 network data and state, delta form of the dual
  NetDev<float> netf{};
  StateDev<float> stf{};
  MixedDev mx{};
  int grid_mixed = 0;
  size_t smem_mixed = 0;
  int net_region_m = 0;  // network region of the mixed kernel
  // device copies of host data
  int *perm = nullptr;
  double *prob = nullptr, *inv2p = nullptr, *alpha0 = nullptr, *wdiag = nullptr;
  double *wdense = nullptr;  // a dense W_u (null for a diagonal one)
  bool dense_w = false;
  int *Gd_ptr = nullptr, *Gd_idx = nullptr, *Ed_ptr = nullptr, *Ed_idx = nullptr;
  double *Gd_val = nullptr, *Ed_val = nullptr;
  // per-solve data owned by the handle
  double *x0 = nullptr, *q = nullptr, *kq = nullptr, *demand = nullptr, *alpha = nullptr;
  double *partial = nullptr, *scal = nullptr;
  double *beta = nullptr;
  int beta_cap = 0;
  unsigned long long *res = nullptr;
  int res_cap = 0;
  unsigned *sync = nullptr;  // counts | flags | barrier
  size_t sync_words = 0;
  int *err = nullptr, *info = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  bool have_data = false;
  // host staging for rapidnet_solve (host pointers)
  double *io_y = nullptr, *io_u = nullptr, *io_x = nullptr, *io_hist = nullptr;
  // averaged primal iterate (internal rows) and its host staging
  double *uavg = nullptr, *xavg = nullptr, *io_uavg = nullptr, *io_xavg = nullptr;
  int io_hist_cap = 0;
  // the per-node form (null for the shared-operator form)
  rn::PnFactor *pn = nullptr;

  ~rn_factor() {
    if (pn) rn::pn_destroy(pn);
    if (device >= 0) cudaSetDevice(device);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    for (void *p : allocs) cudaFree(p);
    if (own_stream && stream) cudaStreamDestroy(stream);
  }
};

namespace {

#define RN_CUDA(call)                                                              \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      set_error("CUDA error %s at %s:%d: %s", #call, __FILE__, __LINE__,           \
                cudaGetErrorString(e_));                                           \
      return e_ == cudaErrorMemoryAllocation ? RN_ERR_NOMEM : RN_ERR_CUDA;         \
    }                                                                              \
  } while (0)

template <typename T>
int dalloc(rn_factor *f, T **p, size_t count) {
  if (count == 0) count = 1;
  void *ptr = nullptr;
  cudaError_t e = cudaMalloc(&ptr, count * sizeof(T));
  if (e != cudaSuccess) {
    set_error("cudaMalloc of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? RN_ERR_NOMEM : RN_ERR_CUDA;
  }
  f->allocs.push_back(ptr);
  f->bytes += (long long)(count * sizeof(T));
  *p = static_cast<T *>(ptr);
  return RN_OK;
}

template <typename T>
int upload(rn_factor *f, T **p, const std::vector<T> &h) {
  int rc = dalloc(f, p, h.size());
  if (rc) return rc;
  if (!h.empty()) RN_CUDA(cudaMemcpy(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  return RN_OK;
}

void release(rn_factor *f, void *p) {
  if (!p) return;
  auto it = std::find(f->allocs.begin(), f->allocs.end(), p);
  if (it != f->allocs.end()) f->allocs.erase(it);
  cudaFree(p);
}

inline int ceil4(int v) { return (v + 3) & ~3; }

bool finite_all(const double *p, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

template <typename T>
void set_sizes(KParams<T> &P, const Sizes &z) {
  P.buf_elems = z.buf;
  P.gbuf_elems = z.gbuf;
  P.segb = z.segb;
  P.gcap = z.gcap;
  P.hchunk = z.hchunk;
  P.fslots = z.fslots;
  P.fbrows = z.fbrows;
  P.tpb = z.tpb;
  P.team_bytes = z.team_bytes;
  P.net_bytes = z.net_bytes;
}

// parameters of the FP64 kernel; mixed: of the FP64 steps of the mixed kernel
KParams<double> base_params(rn_factor *f, bool mixed = false) {
  KParams<double> P{};
  P.net = f->net;
  P.plan = f->pd;
  P.st = f->st;
  P.iters = 1;
  P.check_every = 1;
  P.linear = 0;
  P.step_base = 0;
  P.gamma = f->gamma;
  P.invgamma = f->gamma > 0 ? 1.0 / f->gamma : 0.0;
  P.tol = 0.0;
  P.maxc = f->maxc;
  set_sizes(P, mixed ? f->sz_dm : f->sz_d);
  return P;
}

KParams<float> base_params_f(rn_factor *f) {
  KParams<float> P{};
  P.net = f->netf;
  P.plan = f->pd;
  P.st = f->stf;
  P.st.res = f->st.res;
  P.st.beta = f->st.beta;
  P.st.theta = f->st.theta;
  P.iters = 1;
  P.check_every = 1;
  P.linear = 1;
  P.step_base = 0;
  P.gamma = f->gamma;
  P.invgamma = f->gamma > 0 ? 1.0 / f->gamma : 0.0;
  P.tol = 0.0;
  P.maxc = f->maxc;
  set_sizes(P, f->sz_f);
  return P;
}

// the mixed kernel's parameters for max_iters iterations
MixedParams mixed_params(rn_factor *f, int max_iters, double tol) {
  MixedParams M;
  M.f = base_params_f(f);
  M.f.iters = max_iters;
  M.f.check_every = f->opts.check_every;
  M.f.tol = tol > 0.0 ? tol : 0.0;
  M.d = base_params(f, true);
  M.d.st.uo32 = const_cast<float *>(f->mx.uref);
  M.d.st.xo32 = const_cast<float *>(f->mx.xref);
  M.mx = f->mx;
  return M;
}

// counters, flags and the grid barrier start at zero for every launch
int reset_sync(rn_factor *f) {
  RN_CUDA(cudaMemsetAsync(f->sync, 0, f->sync_words * sizeof(unsigned), f->stream));
  return RN_OK;
}

// the error word is cleared once per call of the ABI, so that a wait that
// gave up in any launch of the call is reported (and later launches of the
// call leave their waits at once)
int clear_err(rn_factor *f) {
  RN_CUDA(cudaMemsetAsync(f->err, 0, sizeof(int), f->stream));
  return RN_OK;
}

// the error word of a kernel that recorded a timed-out wait (site 1-4)
int timeout_error(const char *who, int e, long long wait_ns) {
  static const char *site[] = {"?", "chain arrivals at a group", "a group's flag",
                               "a root's flag", "the grid barrier"};
  set_error("%sa device-side wait (%s, site %d) gave up after %.6g s", who,
            site[e >= 1 && e <= 4 ? e : 0], e, wait_ns * 1e-9);
  return RN_ERR_TIMEOUT;
}

int check_err(rn_factor *f) {
  int e = 0;
  RN_CUDA(cudaMemcpyAsync(&e, f->err, sizeof(int), cudaMemcpyDeviceToHost, f->stream));
  RN_CUDA(cudaStreamSynchronize(f->stream));
  if (e) return timeout_error("", e, f->st.wait_ns);
  return RN_OK;
}

// one evaluation of the dual gradient from f->st.s into uo / xo
int solve_step(rn_factor *f, int linear) {
  int rc = reset_sync(f);
  if (rc) return rc;
  KParams<double> P = base_params(f);
  P.linear = linear;
  RN_CUDA((launch_solve<double, false>(P, f->grid, f->block, f->smem, f->stream)));
  return RN_OK;
}

int node_blocks(int n) { return std::max(1, std::min(n - 1, 4096)); }

int power_iteration(rn_factor *f, int iters, double *L_out) {
  const int n = f->plan.n;
  if (int rc = clear_err(f)) return rc;
  k_power_start<<<node_blocks(n), 128, 0, f->stream>>>(f->net, f->perm, n, f->st.s);
  RN_CUDA(cudaGetLastError());
  for (int k = 0; k < iters; ++k) {
    int rc = solve_step(f, 1);
    if (rc) return rc;
    k_norm2<<<kRedBlocks, 256, 0, f->stream>>>(f->net, n, f->st.uo, f->st.xo, f->partial);
    k_final_reduce<<<1, 32, 0, f->stream>>>(f->partial, kRedBlocks, f->scal);
    k_power_scale<<<node_blocks(n), 128, 0, f->stream>>>(f->net, n, f->st.uo, f->st.xo, f->scal,
                                                         f->st.s);
    RN_CUDA(cudaGetLastError());
  }
  double nrm2 = 0.0;
  RN_CUDA(cudaMemcpyAsync(&nrm2, f->scal, sizeof(double), cudaMemcpyDeviceToHost, f->stream));
  int rc = check_err(f);
  if (rc) return rc;
  *L_out = std::sqrt(nrm2);
  return RN_OK;
}

// Bytes of one team region for a kernel whose blocks hold a network
// region of net_bytes, tpb team regions and static_smem bytes of static
// shared memory: enough blocks per SM that every work item gets a
// resident block (up to 4), split evenly.
int team_budget(int device, int n_items, int tpb, int block, int net_bytes, int static_smem,
                int *team_bytes) {
  int sms = 0, optin = 0, per_sm = 0, reserved = 0;
  RN_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  RN_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
  RN_CUDA(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device));
  RN_CUDA(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, device));
  return team_bytes_for(sms, optin, per_sm, reserved, n_items, tpb, block, net_bytes, static_smem,
                        team_bytes, nullptr);
}

int fit_sizes(const rn_factor *f, int eb, int team_bytes, int net_bytes, int tw, int tpb, int mode,
              Sizes *z) {
  return layout_sizes(f->plan, RowDims{f->NXP, f->NUP, f->YP, f->SP, f->NEP}, eb, team_bytes,
                      net_bytes, tw, tpb, mode, z);
}

// a W_u with a nonzero entry off the diagonal
bool is_dense(const double *W, int nu) {
  for (int i = 0; i < nu; ++i)
    for (int j = 0; j < nu; ++j)
      if (i != j && W[(size_t)i * nu + j] != 0.0) return true;
  return false;
}

// TF32 head of an FP32 value on the host, as the device's cvt.rna.tf32.f32:
// round to nearest, ties away from zero, keep 10 mantissa bits
float tf32_round(float a) {
  unsigned u;
  std::memcpy(&u, &a, 4);
  if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x1000u) & ~0x1fffu;
  float r;
  std::memcpy(&r, &u, 4);
  return r;
}

// B fragments of F for mma.m16n8k8 (row.col), per (k-step ks, n-tile nt,
// lane): b0 = B[8 ks + t][8 nt + g], b1 = B[8 ks + t + 4][8 nt + g] with
// g = lane / 4, t = lane % 4 and B[k][j] = F[j][k] (zero outside nu x nu),
// each as TF32 head and tail: {b0 head, b1 head, b0 tail, b1 tail}
std::vector<float> dense_f_fragments(const std::vector<double> &F, int nu) {
  const int NT = (nu + 7) / 8;
  std::vector<float> out((size_t)NT * NT * 32 * 4);
  auto Bkj = [&](int k, int j) { return (k < nu && j < nu) ? F[(size_t)j * nu + k] : 0.0; };
  for (int ks = 0; ks < NT; ++ks)
    for (int nt = 0; nt < NT; ++nt)
      for (int lane = 0; lane < 32; ++lane) {
        const int g = lane / 4, t = lane % 4;
        const double b[2] = {Bkj(8 * ks + t, 8 * nt + g), Bkj(8 * ks + t + 4, 8 * nt + g)};
        float *o = &out[(((size_t)ks * NT + nt) * 32 + lane) * 4];
        for (int e = 0; e < 2; ++e) {
          const float head = tf32_round((float)b[e]);
          o[e] = head;
          o[2 + e] = tf32_round((float)(b[e] - (double)head));
        }
      }
  return out;
}

bool is_identity(const double *A, int nx) {
  for (int i = 0; i < nx; ++i)
    for (int j = 0; j < nx; ++j)
      if (A[(size_t)i * nx + j] != (i == j ? 1.0 : 0.0)) return false;
  return true;
}

int validate_network(const rn_network *net, const rn_cost *cost, bool shared = true) {
  if (!net || !cost) {
    set_error("network or cost is NULL");
    return RN_ERR_INVAL;
  }
  const int nx = net->nx, nu = net->nu, nd = net->nd, ne = net->ne;
  if (nx < 1 || nu < 1 || nd < 1 || ne < 0) {
    set_error("network: need nx, nu, nd >= 1 and ne >= 0");
    return RN_ERR_INVAL;
  }
  if (!net->A || !net->B || !net->Gd || !net->xmin || !net->xmax || !net->xs || !net->umin ||
      !net->umax || (ne > 0 && (!net->E || !net->Ed))) {
    set_error("network: NULL matrix or bound");
    return RN_ERR_INVAL;
  }
  if (!cost->alpha0 || !cost->Wu) {
    set_error("cost: NULL alpha0 or Wu");
    return RN_ERR_INVAL;
  }
  if (!finite_all(net->A, (size_t)nx * nx) || !finite_all(net->B, (size_t)nx * nu) ||
      !finite_all(net->Gd, (size_t)nx * nd) || (ne > 0 && !finite_all(net->E, (size_t)ne * nu)) ||
      (ne > 0 && !finite_all(net->Ed, (size_t)ne * nd)) || !finite_all(cost->alpha0, nu) ||
      !finite_all(cost->Wu, (size_t)nu * nu) || !finite_all(net->xs, nx)) {
    set_error("network/cost: non-finite entry");
    return RN_ERR_INVAL;
  }
  for (int i = 0; i < nx; ++i)
    if (!(net->xmin[i] <= net->xmax[i])) {
      set_error("network: xmin[%d] > xmax[%d]", i, i);
      return RN_ERR_INVAL;
    }
  for (int j = 0; j < nu; ++j)
    if (!(net->umin[j] <= net->umax[j])) {
      set_error("network: umin[%d] > umax[%d]", j, j);
      return RN_ERR_INVAL;
    }
  if (!(cost->W_alpha >= 0.0) || !(cost->Ws >= 0.0) || !(cost->Wx >= 0.0) ||
      !std::isfinite(cost->W_alpha) || !std::isfinite(cost->Ws) || !std::isfinite(cost->Wx)) {
    set_error("cost: weights must be finite and non-negative");
    return RN_ERR_INVAL;
  }
  for (int i = 0; i < nu; ++i)
    for (int j = 0; j < nu; ++j)
      if (cost->Wu[(size_t)i * nu + j] != cost->Wu[(size_t)j * nu + i]) {
        set_error("cost: Wu is not symmetric");
        return RN_ERR_INVAL;
      }
  for (int i = 0; i < nu; ++i)
    if (!(cost->Wu[(size_t)i * nu + i] > 0.0)) {
      set_error("cost: Wu is not positive definite (diagonal entry %d)", i);
      return RN_ERR_INVAL;
    }
  if (is_dense(cost->Wu, nu)) {
    std::vector<double> R(cost->Wu, cost->Wu + (size_t)nu * nu);
    if (!cholesky(R, nu)) {
      set_error("cost: Wu is not positive definite (Cholesky breaks down)");
      return RN_ERR_INVAL;
    }
  }
  if (!shared) return RN_OK;
  if (!is_identity(net->A, nx)) {
    set_error("network: the shared-operator form handles A = I only (tank mass balance)");
    return RN_ERR_UNSUPPORTED;
  }
  if (std::max(nx, nu) > 256) {
    set_error("network: the library handles nx, nu <= 256");
    return RN_ERR_UNSUPPORTED;
  }
  return RN_OK;
}

int factor_impl(const rn_network *net, const rn_tree *tree, const rn_cost *cost,
                const rn_opts *opts, rn_factor *f) {
  int rc = validate_network(net, cost);
  if (rc) return rc;
  rc = build_plan(tree, f->plan);  // validation; rebuilt below for the device
  if (rc) return rc;
  f->opts = opts ? *opts : rn_opts{};
  if (f->opts.precision != RN_PREC_FP64 && f->opts.precision != RN_PREC_MIXED) {
    set_error("precision must be RN_PREC_FP64 or RN_PREC_MIXED");
    return RN_ERR_INVAL;
  }
  if (f->opts.power_iters <= 0) f->opts.power_iters = 200;
  if (f->opts.check_every <= 0) f->opts.check_every = 10;
  if (f->opts.refresh_every <= 0) f->opts.refresh_every = 40;
  if (f->opts.theta_rule != RN_THETA_EQUALITY && f->opts.theta_rule != RN_THETA_SIMPLE) {
    set_error("theta_rule must be RN_THETA_EQUALITY or RN_THETA_SIMPLE");
    return RN_ERR_INVAL;
  }
  if (f->opts.wait_us < 0) {
    set_error("wait_us must be >= 0");
    return RN_ERR_INVAL;
  }
  const long long wait_ns = f->opts.wait_us > 0 ? 1000LL * f->opts.wait_us : kWaitNs;
  f->device = f->opts.device;
  RN_CUDA(cudaSetDevice(f->device));
  if (f->opts.stream) {
    f->stream = static_cast<cudaStream_t>(f->opts.stream);
  } else {
    RN_CUDA(cudaStreamCreateWithFlags(&f->stream, cudaStreamNonBlocking));
    f->own_stream = true;
  }
  const int nx = net->nx, nu = net->nu, nd = net->nd, ne = net->ne;
  {
    // groups beyond one per stage-1 subtree only where one block per SM
    // leaves SMs free next to the chain blocks
    int sms = 0, tw = 0, tpb = 0;
    RN_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, f->device));
    team_layout(f->opts.block_threads, nx, nu, &tw, &tpb, nullptr);
    const int chain_blocks = (f->plan.n_chains + tpb - 1) / tpb;
    if ((rc = build_plan(tree, f->plan, std::max(1, sms - chain_blocks)))) return rc;
  }
  f->nx = nx;
  f->nu = nu;
  f->nd = nd;
  f->ne = ne;
  f->NXP = ceil4(nx);
  f->NUP = ceil4(nu);
  f->SP = f->NXP + f->NUP;
  f->YP = 2 * f->NXP + f->NUP;
  f->NEP = std::max(1, ne);
  f->W_alpha = cost->W_alpha;
  f->Ws = cost->Ws;
  f->Wx = cost->Wx;

  // Schur complement of the coupling: S = E W^-1 E', its Cholesky factor
  // (full row rank of E) and inverse, in FP64
  std::vector<double> winv(nu), wdiag(nu);
  for (int j = 0; j < nu; ++j) {
    wdiag[j] = cost->Wu[(size_t)j * nu + j];
    winv[j] = 1.0 / wdiag[j];
  }
  std::vector<double> Sinv(std::max(1, ne * ne), 0.0);
  // dense W_u: W^-1 by Cholesky, S = E W^-1 E', F = W^-1 - W^-1 E' S^-1 E W^-1
  // and Gm = W^-1 E' S^-1 as dense matrices (FP64)
  f->dense_w = is_dense(cost->Wu, nu);
  std::vector<double> Fdense, Gm;
  if (f->dense_w) {
    std::vector<double> R(cost->Wu, cost->Wu + (size_t)nu * nu);
    if (!cholesky(R, nu)) {
      set_error("cost: Wu is not positive definite (Cholesky breaks down)");
      return RN_ERR_INVAL;
    }
    const std::vector<double> Wi = chol_inverse(R, nu);
    for (int j = 0; j < nu; ++j) winv[j] = Wi[(size_t)j * nu + j];
    std::vector<double> EWi((size_t)std::max(1, ne) * nu, 0.0);  // E W^-1
    for (int r = 0; r < ne; ++r)
      for (int k = 0; k < nu; ++k) {
        const double e = net->E[(size_t)r * nu + k];
        if (e == 0.0) continue;
        for (int j = 0; j < nu; ++j) EWi[(size_t)r * nu + j] += e * Wi[(size_t)k * nu + j];
      }
    Gm.assign((size_t)nu * std::max(1, ne), 0.0);
    if (ne > 0) {
      std::vector<double> S((size_t)ne * ne, 0.0);
      for (int r = 0; r < ne; ++r)
        for (int c = 0; c < ne; ++c) {
          double acc = 0.0;
          for (int j = 0; j < nu; ++j) acc += EWi[(size_t)r * nu + j] * net->E[(size_t)c * nu + j];
          S[(size_t)r * ne + c] = acc;
        }
      std::vector<double> RS = S;
      if (!cholesky(RS, ne)) {
        set_error("E does not have full row rank (E W^-1 E' is singular)");
        return RN_ERR_RANK;
      }
      Sinv = chol_inverse(RS, ne);
      for (int j = 0; j < nu; ++j)
        for (int r = 0; r < ne; ++r) {
          double acc = 0.0;
          for (int c = 0; c < ne; ++c) acc += EWi[(size_t)c * nu + j] * Sinv[(size_t)c * ne + r];
          Gm[(size_t)j * ne + r] = acc;
        }
    }
    Fdense = Wi;
    for (int i = 0; i < nu; ++i)
      for (int r = 0; r < ne; ++r) {
        const double a = Gm[(size_t)i * ne + r];
        if (a == 0.0) continue;
        for (int j = 0; j < nu; ++j) Fdense[(size_t)i * nu + j] -= a * EWi[(size_t)r * nu + j];
      }
  }
  if (ne > 0 && !f->dense_w) {
    std::vector<double> S((size_t)ne * ne, 0.0);
    for (int r = 0; r < ne; ++r)
      for (int c = 0; c < ne; ++c) {
        double acc = 0.0;
        for (int j = 0; j < nu; ++j)
          acc += net->E[(size_t)r * nu + j] * winv[j] * net->E[(size_t)c * nu + j];
        S[(size_t)r * ne + c] = acc;
      }
    std::vector<double> R = S;
    if (!cholesky(R, ne)) {
      set_error("E does not have full row rank (E W^-1 E' is singular)");
      return RN_ERR_RANK;
    }
    Sinv = chol_inverse(R, ne);
  }
  // the shared operator must stand for every node's factor of the general
  // recursion (it does in exact arithmetic; this bounds the rounding)
  f->collapse_dev = f->dense_w ? collapse_deviation_dense(tree, nu, ne, net->E, cost->Wu,
                                                         Fdense.data())
                              : collapse_deviation(tree, nu, ne, net->E, winv.data(), Sinv.data());
  if (!(f->collapse_dev <= kCollapseTol)) {
    set_error("factor check: 2 p Phi differs from the shared operator F by %.3g (relative) at a "
              "sampled node; E W_u^-1 E' is too ill-conditioned", f->collapse_dev);
    return RN_ERR_RANK;
  }

  const Plan &p = f->plan;
  const int n = p.n;
  // sparse operators
  Csr Bc = dense_to_csc(net->B, nx, nu), Br = dense_to_csr(net->B, nx, nu);
  Csr Er, Ec, Gdr = dense_to_csr(net->Gd, nx, nd), Edr;
  if (ne > 0) {
    Er = dense_to_csr(net->E, ne, nu);
    Ec = dense_to_csc(net->E, ne, nu);
    Edr = dense_to_csr(net->Ed, ne, nd);
  } else {
    Er.ptr.assign(1, 0);
    Ec.ptr.assign(nu + 1, 0);
    Edr.ptr.assign(1, 0);
  }
  NetDev<double> &nt = f->net;
  nt.nx = nx;
  nt.nu = nu;
  nt.ne = ne;
  nt.nd = nd;
  nt.NXP = f->NXP;
  nt.NUP = f->NUP;
  nt.SP = f->SP;
  nt.YP = f->YP;
  nt.NEP = f->NEP;
  nt.Wx = cost->Wx;
  nt.Ws = cost->Ws;
  int *ip;
  double *dp;
#define UP_I(field, vec) \
  if ((rc = upload(f, &ip, vec))) return rc; \
  field = ip;
#define UP_D(field, vec) \
  if ((rc = upload(f, &dp, vec))) return rc; \
  field = dp;
  UP_I(nt.Bc_ptr, Bc.ptr) UP_I(nt.Bc_idx, Bc.idx) UP_D(nt.Bc_val, Bc.val)
  UP_I(nt.Br_ptr, Br.ptr) UP_I(nt.Br_idx, Br.idx) UP_D(nt.Br_val, Br.val)
  std::vector<double> Erw(Er.val.size());
  for (size_t e = 0; e < Er.val.size(); ++e) Erw[e] = Er.val[e] * winv[Er.idx[e]];
  UP_I(nt.Er_ptr, Er.ptr) UP_I(nt.Er_idx, Er.idx) UP_D(nt.Er_val, Er.val) UP_D(nt.Erw_val, Erw)
  UP_I(nt.Ec_ptr, Ec.ptr) UP_I(nt.Ec_idx, Ec.idx) UP_D(nt.Ec_val, Ec.val)
  UP_D(nt.winv, winv) UP_D(nt.Sinv, Sinv)
  UP_D(nt.xmin, std::vector<double>(net->xmin, net->xmin + nx))
  UP_D(nt.xmax, std::vector<double>(net->xmax, net->xmax + nx))
  UP_D(nt.xs, std::vector<double>(net->xs, net->xs + nx))
  UP_D(nt.umin, std::vector<double>(net->umin, net->umin + nu))
  UP_D(nt.umax, std::vector<double>(net->umax, net->umax + nu))
  UP_D(f->alpha0, std::vector<double>(cost->alpha0, cost->alpha0 + nu))
  UP_D(f->wdiag, wdiag)
  if (f->dense_w) {
    UP_D(nt.Fd, Fdense) UP_D(nt.Gm, Gm)
    UP_D(f->wdense, std::vector<double>(cost->Wu, cost->Wu + (size_t)nu * nu))
  }
  UP_I(f->Gd_ptr, Gdr.ptr) UP_I(f->Gd_idx, Gdr.idx) UP_D(f->Gd_val, Gdr.val)
  UP_I(f->Ed_ptr, Edr.ptr) UP_I(f->Ed_idx, Edr.idx) UP_D(f->Ed_val, Edr.val)

  PlanDev &pd = f->pd;
  pd.n = n;
  pd.n_top = p.n_top;
  pd.n_chains = p.n_chains;
  pd.n_groups = p.n_groups;
  pd.n_roots = p.n_roots;
  pd.hp_rows = std::max(1, p.hp_rows);
  UP_I(pd.g_root, p.g_root.empty() ? std::vector<int>(1, -1) : p.g_root)
  UP_I(pd.r_node, p.r_node.empty() ? std::vector<int>(1, 0) : p.r_node)
  UP_I(pd.r_part, p.r_part)
  UP_I(pd.g_hp, p.g_hp.empty() ? std::vector<int>(1, -1) : p.g_hp)
  UP_I(pd.r_hp, p.r_hp.empty() ? std::vector<int>(1, 0) : p.r_hp)
  UP_I(pd.parent, p.parent) UP_I(pd.g_node, p.g_node) UP_I(pd.g_chain, p.g_chain)
  UP_I(pd.g_lvl, p.g_lvl) UP_I(pd.lvl, p.lvl) UP_I(pd.g_ccn, p.g_ccn) UP_I(pd.ccn, p.ccn)
  UP_I(pd.g_desc_ptr, p.g_desc_ptr) UP_I(pd.g_desc, p.g_desc)
  UP_I(pd.tc_ptr, p.tc_ptr) UP_I(pd.tc, p.tc) UP_I(pd.cc_ptr, p.cc_ptr) UP_I(pd.cc, p.cc)
  UP_I(pd.ch_start, p.ch_start) UP_I(pd.ch_len, p.ch_len) UP_I(pd.ch_group, p.ch_group)
  UP_I(pd.ch_parent, p.ch_parent) UP_I(pd.ch_own_ptr, p.ch_own_ptr) UP_I(pd.ch_own, p.ch_own)
  UP_I(f->perm, p.perm) UP_D(f->prob, p.prob)
  std::vector<double> inv2p(n, 0.0);
  for (int i = 1; i < n; ++i) inv2p[i] = 1.0 / (2.0 * p.prob[i]);
  UP_D(f->inv2p, inv2p)
#undef UP_I
#undef UP_D

  // state
  StateDev<double> &st = f->st;
  double *s, *ya, *yb, *ub, *gb, *z, *up, *ux, *uo, *xo, *hp;
  if ((rc = dalloc(f, &s, (size_t)n * f->SP)) || (rc = dalloc(f, &ya, (size_t)n * f->YP)) ||
      (rc = dalloc(f, &yb, (size_t)n * f->YP)) || (rc = dalloc(f, &ub, (size_t)n * f->NUP)) ||
      (rc = dalloc(f, &gb, (size_t)n * f->NXP)) || (rc = dalloc(f, &z, (size_t)n * f->NUP)) ||
      (rc = dalloc(f, &up, (size_t)n * f->SP)) || (rc = dalloc(f, &ux, (size_t)n * f->SP)) ||
      (rc = dalloc(f, &uo, (size_t)n * f->NUP)) || (rc = dalloc(f, &xo, (size_t)n * f->NXP)) ||
      (rc = dalloc(f, &hp, 2 * (size_t)std::max(1, p.hp_rows) * f->SP)))
    return rc;
  RN_CUDA(cudaMemset(hp, 0, 2 * (size_t)std::max(1, p.hp_rows) * f->SP * sizeof(double)));
  RN_CUDA(cudaMemset(s, 0, (size_t)n * f->SP * sizeof(double)));
  RN_CUDA(cudaMemset(ya, 0, (size_t)n * f->YP * sizeof(double)));
  RN_CUDA(cudaMemset(yb, 0, (size_t)n * f->YP * sizeof(double)));
  RN_CUDA(cudaMemset(ub, 0, (size_t)n * f->NUP * sizeof(double)));
  RN_CUDA(cudaMemset(gb, 0, (size_t)n * f->NXP * sizeof(double)));
  RN_CUDA(cudaMemset(z, 0, (size_t)n * f->NUP * sizeof(double)));
  RN_CUDA(cudaMemset(up, 0, (size_t)n * f->SP * sizeof(double)));
  RN_CUDA(cudaMemset(ux, 0, (size_t)n * f->SP * sizeof(double)));
  RN_CUDA(cudaMemset(uo, 0, (size_t)n * f->NUP * sizeof(double)));
  RN_CUDA(cudaMemset(xo, 0, (size_t)n * f->NXP * sizeof(double)));
  st.s = s;
  st.ya = ya;
  st.yb = yb;
  st.ub = ub;
  st.gb = gb;
  st.z = z;
  st.up = up;
  st.ux = ux;
  st.hp = hp;
  st.uo = uo;
  st.xo = xo;
  st.inv2p = f->inv2p;
  if ((rc = dalloc(f, &f->x0, nx)) || (rc = dalloc(f, &f->q, nu)) || (rc = dalloc(f, &f->kq, nu)) ||
      (rc = dalloc(f, &f->demand, (size_t)n * nd)) || (rc = dalloc(f, &f->alpha, (size_t)n * nu)) ||
      (rc = dalloc(f, &f->partial, 3 * kRedBlocks)) || (rc = dalloc(f, &f->scal, 4)) ||
      (rc = dalloc(f, &f->err, 1)) || (rc = dalloc(f, &f->info, 8)))
    return rc;
  RN_CUDA(cudaMemset(f->x0, 0, nx * sizeof(double)));
  st.xroot = f->x0;
  const size_t ng = (size_t)std::max(1, p.n_groups + p.n_roots);
  f->sync_words = 3 * ng + 1;
  if ((rc = dalloc(f, &f->sync, f->sync_words))) return rc;
  st.count = f->sync;
  st.flags = f->sync + ng;
  st.arrive = f->sync + 2 * ng;
  st.barrier = f->sync + 3 * ng;
  st.err = f->err;
  st.info = f->info;
  st.res = nullptr;
  st.beta = nullptr;
  st.wait_ns = wait_ns;

  if (f->opts.precision == RN_PREC_MIXED) {
    // FP32 copies of the network data (index arrays shared) and FP32 state
    auto tof = [](const double *p, size_t m) { return std::vector<float>(p, p + m); };
    auto tofv = [](const std::vector<double> &v) { return std::vector<float>(v.begin(), v.end()); };
    NetDev<float> &nf = f->netf;
    nf.nx = nx;
    nf.nu = nu;
    nf.ne = ne;
    nf.nd = nd;
    nf.NXP = f->NXP;
    nf.NUP = f->NUP;
    nf.SP = f->SP;
    nf.YP = f->YP;
    nf.NEP = f->NEP;
    nf.Wx = (float)cost->Wx;
    nf.Ws = (float)cost->Ws;
    nf.Bc_ptr = nt.Bc_ptr;
    nf.Bc_idx = nt.Bc_idx;
    nf.Br_ptr = nt.Br_ptr;
    nf.Br_idx = nt.Br_idx;
    nf.Er_ptr = nt.Er_ptr;
    nf.Er_idx = nt.Er_idx;
    nf.Ec_ptr = nt.Ec_ptr;
    nf.Ec_idx = nt.Ec_idx;
    float *fp;
#define UP_F(field, vec) \
  if ((rc = upload(f, &fp, vec))) return rc; \
  field = fp;
    UP_F(nf.Bc_val, tofv(Bc.val)) UP_F(nf.Br_val, tofv(Br.val)) UP_F(nf.Er_val, tofv(Er.val))
    UP_F(nf.Erw_val, tofv(Erw))
    UP_F(nf.Ec_val, tofv(Ec.val)) UP_F(nf.winv, tofv(winv)) UP_F(nf.Sinv, tofv(Sinv))
    UP_F(nf.xmin, tof(net->xmin, nx)) UP_F(nf.xmax, tof(net->xmax, nx)) UP_F(nf.xs, tof(net->xs, nx))
    UP_F(nf.umin, tof(net->umin, nu)) UP_F(nf.umax, tof(net->umax, nu))
    UP_F(f->stf.inv2p, tofv(inv2p))
    if (f->dense_w) {
      UP_F(nf.Fd, tofv(Fdense))
      const std::vector<float> frag = dense_f_fragments(Fdense, nu);
      UP_F(fp, frag)
      nf.Ft = reinterpret_cast<const float4 *>(fp);
    }
#undef UP_F
    float *s32, *z32, *up32, *ux32, *hp32, *da, *db, *ybh, *uref, *xref, *sw;
    if ((rc = dalloc(f, &s32, (size_t)n * f->SP)) || (rc = dalloc(f, &z32, (size_t)n * f->NUP)) ||
        (rc = dalloc(f, &up32, (size_t)n * f->SP)) || (rc = dalloc(f, &ux32, (size_t)n * f->SP)) ||
        (rc = dalloc(f, &hp32, 2 * (size_t)std::max(1, p.hp_rows) * f->SP)) ||
        (rc = dalloc(f, &da, (size_t)n * f->YP)) ||
        (rc = dalloc(f, &db, (size_t)n * f->YP)) || (rc = dalloc(f, &ybh, (size_t)n * f->YP)) ||
        (rc = dalloc(f, &uref, (size_t)n * f->NUP)) || (rc = dalloc(f, &xref, (size_t)n * f->NXP)) ||
        (rc = dalloc(f, &sw, (size_t)n * f->SP)))
      return rc;
    for (auto pr : {std::make_pair((void *)s32, (size_t)n * f->SP), {(void *)z32, (size_t)n * f->NUP},
                    {(void *)up32, (size_t)n * f->SP}, {(void *)ux32, (size_t)n * f->SP},
                    {(void *)hp32, 2 * (size_t)std::max(1, p.hp_rows) * f->SP},
                    {(void *)da, (size_t)n * f->YP},
                    {(void *)db, (size_t)n * f->YP}, {(void *)ybh, (size_t)n * f->YP},
                    {(void *)uref, (size_t)n * f->NUP}, {(void *)xref, (size_t)n * f->NXP},
                    {(void *)sw, (size_t)n * f->SP}})
      RN_CUDA(cudaMemset(pr.first, 0, pr.second * sizeof(float)));
    StateDev<float> &sf = f->stf;
    sf.s = s32;
    sf.z = z32;
    sf.up = up32;
    sf.ux = ux32;
    sf.hp = hp32;
    sf.count = st.count;
    sf.flags = st.flags;
    sf.arrive = st.arrive;
    sf.barrier = st.barrier;
    sf.err = st.err;
    sf.info = st.info;
    sf.wait_ns = wait_ns;
    f->mx.yb = st.ya;  // the FP64 iterate buffer holds the base
    f->mx.ybh = ybh;
    f->mx.da = da;
    f->mx.db = db;
    f->mx.uref = uref;
    f->mx.xref = xref;
    f->mx.sw = sw;
    f->mx.s64 = st.s;
    f->mx.refresh_every = f->opts.refresh_every;
  }

  // launch configuration: a block is two chain teams of tw threads (one
  // thread per input component, at least 64); as many resident blocks as
  // there are work items (groups and chain pairs), up to what the device
  // holds
  if ((rc = team_layout(f->opts.block_threads, nx, nu, &f->tw, &f->tpb, &f->maxc))) return rc;
  f->block = f->tpb * f->tw;
  if (f->dense_w) {
    // the dense F product: at most two components per thread (FP64) and
    // kTcTiles column tiles per warp (tensor cores)
    const int ntiles = (nu + 7) / 8, nw = f->tw / 32;
    if (2 * f->tw < nu || (ntiles + nw - 1) / nw > kTcTiles) {
      set_error("a dense Wu needs chain teams of at least %d threads (block_threads)",
                std::max((nu + 1) / 2, 32 * ((ntiles + kTcTiles - 1) / kTcTiles)));
      return RN_ERR_UNSUPPORTED;
    }
  }
  {
    const int nnzB = (int)Bc.idx.size(), nnzE = (int)Er.idx.size();
    f->net_bytes_d = (int)net_smem_bytes(nx, nu, ne, nnzB, nnzE, 8);
    f->net_bytes_f = (int)net_smem_bytes(nx, nu, ne, nnzB, nnzE, 4);
  }
  const int n_items = p.n_groups + (p.n_chains + f->tpb - 1) / f->tpb;
  int sms = 0;
  RN_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, f->device));
  {
    int team_bytes = 0;
    if ((rc = team_budget(f->device, n_items, f->tpb, f->block, f->net_bytes_d, 0, &team_bytes)))
      return rc;
    if ((rc = fit_sizes(f, 8, team_bytes, f->net_bytes_d, f->tw, f->tpb, 1, &f->sz_d))) return rc;
    f->smem = kHdrBytes + f->net_bytes_d + (size_t)f->tpb * team_bytes;
    int bps1 = 0, bps2 = 0;
    RN_CUDA((solve_occupancy<double, true>(f->maxc, f->dense_w, f->block, f->smem, &bps1)));
    RN_CUDA((solve_occupancy<double, false>(f->maxc, f->dense_w, f->block, f->smem, &bps2)));
    const int resident = std::min(bps1, bps2) * sms;
    if (resident < 1) {
      set_error("the solve kernel does not fit on the device (block %d, smem %zu)", f->block,
                f->smem);
      return RN_ERR_UNSUPPORTED;
    }
    f->grid = std::min(n_items, resident);
    if (f->opts.max_ctas > 0) f->grid = std::min(f->grid, f->opts.max_ctas);
    if ((rc = check_layout(p, f->sz_d, n_items, f->grid, "the FP64 kernel"))) return rc;
  }
  if (f->opts.precision == RN_PREC_MIXED) {
    // network region: the FP32 copy, then the header of the FP64 data
    f->net_region_m = f->net_bytes_f + (int)round16(sizeof(NetDev<double>));
    int team_bytes = 0;
    if ((rc = team_budget(f->device, n_items, f->tpb, f->block, f->net_region_m, 0, &team_bytes)))
      return rc;
    if ((rc = fit_sizes(f, 4, team_bytes, f->net_region_m, f->tw, f->tpb, 2, &f->sz_f)) ||
        (rc = fit_sizes(f, 8, team_bytes, f->net_bytes_f, f->tw, f->tpb, 0, &f->sz_dm)))
      return rc;
    f->smem_mixed = kHdrBytes + f->net_region_m + (size_t)f->tpb * team_bytes;
    int bpm = 0;
    RN_CUDA(mixed_occupancy(f->maxc, f->dense_w, f->block, f->smem_mixed, &bpm));
    if (bpm < 1) {
      set_error("the mixed kernel does not fit on the device");
      return RN_ERR_UNSUPPORTED;
    }
    f->grid_mixed = std::min(n_items, bpm * sms);
    if (f->opts.max_ctas > 0) f->grid_mixed = std::min(f->grid_mixed, f->opts.max_ctas);
    if ((rc = check_layout(p, f->sz_f, n_items, f->grid_mixed, "the mixed kernel")) ||
        (rc = check_layout(p, f->sz_dm, n_items, f->grid_mixed, "the mixed kernel (FP64 steps)")))
      return rc;
  }

  if (f->opts.gamma > 0.0) {
    f->gamma = f->opts.gamma;
    f->L = 0.0;
  } else {
    double L = 0.0;
    rc = power_iteration(f, f->opts.power_iters, &L);
    if (rc) return rc;
    if (!(L > 0.0) || !std::isfinite(L)) {
      set_error("power iteration gave a non-positive Lipschitz estimate %g", L);
      return RN_ERR_INVAL;
    }
    f->L = L;
    f->gamma = 1.0 / (1.01 * L);
  }
  RN_CUDA(cudaEventCreate(&f->ev0));
  RN_CUDA(cudaEventCreate(&f->ev1));
  RN_CUDA(cudaStreamSynchronize(f->stream));
  return RN_OK;
}

// The per-node form (paper §4.4, general recursion): the checks every form
// shares, the staging buffers of the host entry point, then the handle of
// pernode.cu, which holds everything else.
int pernode_impl(const rn_network *net, const rn_tree *tree, const rn_cost *cost,
                 const rn_opts *opts, rn_factor *f) {
  int rc = validate_network(net, cost, false);
  if (rc) return rc;
  if ((rc = pn_validate(net, tree, cost))) return rc;
  if ((rc = build_plan(tree, f->plan))) return rc;  // sizes of the host staging
  f->opts = opts ? *opts : rn_opts{};
  if (f->opts.precision != RN_PREC_FP64 && f->opts.precision != RN_PREC_FP32 &&
      f->opts.precision != RN_PREC_MIXED) {
    set_error("precision must be RN_PREC_FP64, RN_PREC_MIXED or RN_PREC_FP32");
    return RN_ERR_INVAL;
  }
  if (f->opts.power_iters <= 0) f->opts.power_iters = 200;
  if (f->opts.check_every <= 0) f->opts.check_every = 10;
  if (f->opts.refresh_every <= 0) f->opts.refresh_every = 40;
  if (f->opts.theta_rule != RN_THETA_EQUALITY && f->opts.theta_rule != RN_THETA_SIMPLE) {
    set_error("theta_rule must be RN_THETA_EQUALITY or RN_THETA_SIMPLE");
    return RN_ERR_INVAL;
  }
  if (f->opts.wait_us < 0) {
    set_error("wait_us must be >= 0");
    return RN_ERR_INVAL;
  }
  f->device = f->opts.device;
  RN_CUDA(cudaSetDevice(f->device));
  if (f->opts.stream) {
    f->stream = static_cast<cudaStream_t>(f->opts.stream);
  } else {
    RN_CUDA(cudaStreamCreateWithFlags(&f->stream, cudaStreamNonBlocking));
    f->own_stream = true;
  }
  f->nx = net->nx;
  f->nu = net->nu;
  f->nd = net->nd;
  f->ne = net->ne;
  f->NXP = ceil4(f->nx);
  f->NUP = ceil4(f->nu);
  f->SP = f->NXP + f->NUP;
  f->YP = 2 * f->NXP + f->NUP;
  f->W_alpha = cost->W_alpha;
  f->Ws = cost->Ws;
  f->Wx = cost->Wx;
  const int n = f->plan.n;
  if ((rc = dalloc(f, &f->x0, f->nx)) || (rc = dalloc(f, &f->q, f->nu)) ||
      (rc = dalloc(f, &f->demand, (size_t)n * f->nd)) ||
      (rc = dalloc(f, &f->alpha, (size_t)n * f->nu)))
    return rc;
  PnOptions o;
  o.device = f->device;
  o.stream = f->stream;
  o.fp32 = f->opts.precision == RN_PREC_FP32;
  o.mixed = f->opts.precision == RN_PREC_MIXED;
  o.refresh_every = f->opts.refresh_every;
  o.gamma = f->opts.gamma > 0.0 ? f->opts.gamma : 0.0;
  o.power_iters = f->opts.power_iters;
  o.check_every = f->opts.check_every;
  o.theta_rule = f->opts.theta_rule;
  o.max_ctas = f->opts.max_ctas;
  o.wait_ns = f->opts.wait_us > 0 ? 1000LL * f->opts.wait_us : kWaitNs;
  if ((rc = pn_create(net, tree, cost, o, &f->pn))) return rc;
  f->gamma = pn_gamma(f->pn);
  return RN_OK;
}

int ensure_beta(rn_factor *f, int iters) {
  if (iters + 1 <= f->beta_cap) return RN_OK;
  int cap = std::max(iters + 1, 2 * f->beta_cap);
  // beta_nu = theta_nu (1 / theta_{nu-1} - 1) from theta_0 = theta_{-1} = 1
  // with theta_{nu+1} = (sqrt(theta^4 + 4 theta^2) - theta^2) / 2 or
  // theta_nu = 2 / (nu + 2) (paper §4.3)
  // beta at [0, cap), theta_0 .. theta_{cap-1} at [cap, 2 cap)
  std::vector<double> b(2 * (size_t)cap);
  double th = 1.0, prev = 1.0;
  for (int k = 0; k < cap; ++k) {
    b[k] = th * (1.0 / prev - 1.0);
    b[cap + k] = th;
    const double t2 = th * th;
    const double nt = f->opts.theta_rule == RN_THETA_SIMPLE
                          ? 2.0 / (k + 3)
                          : 0.5 * (std::sqrt(t2 * t2 + 4.0 * t2) - t2);
    prev = th;
    th = nt;
  }
  release(f, f->beta);
  f->beta = nullptr;
  int rc = upload(f, &f->beta, b);
  if (rc) return rc;
  f->beta_cap = cap;
  f->st.beta = f->beta;
  f->st.theta = f->beta + cap;
  return RN_OK;
}

int ensure_res(rn_factor *f, int checks) {
  if (checks <= f->res_cap) return RN_OK;
  int cap = std::max(checks, 2 * f->res_cap);
  release(f, f->res);
  f->res = nullptr;
  int rc = dalloc(f, &f->res, cap);
  if (rc) return rc;
  f->res_cap = cap;
  f->st.res = f->res;
  return RN_OK;
}

// per-solve constants and the offset x*(0): s = (0 | c0), ub = ubar + Kq,
// gb = Gd d, then one dual-gradient evaluation; its inputs become ub
int prepare(rn_factor *f, const double *x0, const double *q, const double *demand,
            const double *alpha) {
  const int n = f->plan.n;
  // the host entry point stages its inputs directly in the handle's buffers
  if (x0 != f->x0)
    RN_CUDA(cudaMemcpyAsync(f->x0, x0, f->nx * sizeof(double), cudaMemcpyDeviceToDevice, f->stream));
  if (q != f->q)
    RN_CUDA(cudaMemcpyAsync(f->q, q, f->nu * sizeof(double), cudaMemcpyDeviceToDevice, f->stream));
  if (demand != f->demand)
    RN_CUDA(cudaMemcpyAsync(f->demand, demand, (size_t)n * f->nd * sizeof(double),
                            cudaMemcpyDeviceToDevice, f->stream));
  if (alpha != f->alpha)
    RN_CUDA(cudaMemcpyAsync(f->alpha, alpha, (size_t)n * f->nu * sizeof(double),
                            cudaMemcpyDeviceToDevice, f->stream));
  const size_t sh = 2 * f->NEP * sizeof(double);
  k_kq<<<1, 128, sh, f->stream>>>(f->net, f->q, f->kq);
  PrepArgs a{f->perm, f->prob, f->demand, f->alpha, f->alpha0, f->kq, f->Gd_ptr, f->Gd_idx,
             f->Gd_val, f->Ed_ptr, f->Ed_idx, f->Ed_val, f->W_alpha, f->nd};
  k_prep<<<node_blocks(n), 128, sh, f->stream>>>(f->net, a, n, f->st.s, f->st.ub, f->st.gb);
  RN_CUDA(cudaGetLastError());
  int rc = solve_step(f, 0);
  if (rc) return rc;
  RN_CUDA(cudaMemcpyAsync(f->st.ub, f->st.uo, (size_t)n * f->NUP * sizeof(double),
                          cudaMemcpyDeviceToDevice, f->stream));
  f->have_data = true;
  return RN_OK;
}

int reduce_nodes(rn_factor *f, int mode, const double *y, double out[3]) {
  ReduceArgs a{f->pd.parent, f->perm, f->prob, f->alpha, f->alpha0, f->wdiag, f->q,
               f->wdense, f->st.uo, f->st.xo, y, f->W_alpha, mode};
  k_node_reduce<<<kRedBlocks, 256, 0, f->stream>>>(f->net, a, f->plan.n, f->partial);
  k_final_reduce<<<1, 32, 0, f->stream>>>(f->partial, kRedBlocks, f->scal);
  RN_CUDA(cudaGetLastError());
  RN_CUDA(cudaMemcpyAsync(out, f->scal, 3 * sizeof(double), cudaMemcpyDeviceToHost, f->stream));
  RN_CUDA(cudaStreamSynchronize(f->stream));
  return RN_OK;
}

int solve_device_impl(rn_factor *f, const double *x0, const double *q, const double *demand,
                      const double *alpha, int max_iters, double tol, const double *y_warm,
                      rn_result *out) {
  if (!f || !x0 || !q || !demand || !alpha || !out || !out->u || !out->x || !out->y) {
    set_error("solve: NULL argument");
    return RN_ERR_INVAL;
  }
  if (max_iters < 1) {
    set_error("solve: max_iters must be >= 1");
    return RN_ERR_INVAL;
  }
  if (!(tol >= 0.0) && !(tol < 0.0)) {
    set_error("solve: tol is NaN");
    return RN_ERR_INVAL;
  }
  if ((out->u_avg == nullptr) != (out->x_avg == nullptr)) {
    set_error("solve: give both u_avg and x_avg, or neither");
    return RN_ERR_INVAL;
  }
  const bool avg = out->u_avg != nullptr;
  if (f->pn) return pn_solve_device(f->pn, x0, q, demand, alpha, max_iters, tol, y_warm, out);
  RN_CUDA(cudaSetDevice(f->device));
  const int n = f->plan.n;
  const int checks = (max_iters + f->opts.check_every - 1) / f->opts.check_every + 1;
  int rc;
  if ((rc = ensure_beta(f, max_iters)) || (rc = ensure_res(f, checks))) return rc;
  if ((rc = clear_err(f)) || (rc = prepare(f, x0, q, demand, alpha))) return rc;
  const bool mixed = f->opts.precision == RN_PREC_MIXED;
  if (mixed)
    k_mixed_init<<<node_blocks(n), 128, 0, f->stream>>>(f->net, f->perm, n, y_warm, f->mx.yb,
                                                        f->mx.ybh, f->mx.da, f->mx.db, f->st.s,
                                                        f->stf.s);
  else
    k_init_apg<<<node_blocks(n), 128, 0, f->stream>>>(f->net, f->perm, n, y_warm, f->st.ya,
                                                      f->st.yb, f->st.s);
  RN_CUDA(cudaGetLastError());
  if ((rc = reset_sync(f))) return rc;
  RN_CUDA(cudaMemsetAsync(f->res, 0, checks * sizeof(unsigned long long), f->stream));
  if (avg) {
    // the averaged primal starts at zero (theta_0 = 1 replaces it by x*(w^0))
    if (!f->uavg && ((rc = dalloc(f, &f->uavg, (size_t)n * f->NUP)) ||
                     (rc = dalloc(f, &f->xavg, (size_t)n * f->NXP))))
      return rc;
    RN_CUDA(cudaMemsetAsync(f->uavg, 0, (size_t)n * f->NUP * sizeof(double), f->stream));
    RN_CUDA(cudaMemsetAsync(f->xavg, 0, (size_t)n * f->NXP * sizeof(double), f->stream));
  }
  RN_CUDA(cudaEventRecord(f->ev0, f->stream));
  if (mixed) {
    MixedParams M = mixed_params(f, max_iters, tol);
    M.f.st.uavg = avg ? f->uavg : nullptr;
    M.f.st.xavg = avg ? f->xavg : nullptr;
    RN_CUDA(launch_mixed(M, f->maxc, f->grid_mixed, f->block, f->smem_mixed, f->stream));
  } else {
    KParams<double> P = base_params(f);
    P.iters = max_iters;
    P.check_every = f->opts.check_every;
    P.tol = tol > 0.0 ? tol : 0.0;
    P.st.uavg = avg ? f->uavg : nullptr;
    P.st.xavg = avg ? f->xavg : nullptr;
    RN_CUDA((launch_solve<double, true>(P, f->grid, f->block, f->smem, f->stream)));
  }
  RN_CUDA(cudaEventRecord(f->ev1, f->stream));
  int info[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  RN_CUDA(cudaMemcpyAsync(info, f->info, 8 * sizeof(int), cudaMemcpyDeviceToHost, f->stream));
  if ((rc = check_err(f))) return rc;
  const int iters = info[0], nchk = info[1], reason = info[2];
  {
    unsigned long long stamps[2];
    std::memcpy(stamps, info + 4, sizeof stamps);
    out->t_begin_ns = (long long)stamps[0];
    out->t_end_ns = (long long)stamps[1];
  }
  float apg_ms = 0.f;
  RN_CUDA(cudaEventElapsedTime(&apg_ms, f->ev0, f->ev1));
  out->apg_ms = apg_ms;
  // y^{iters} was written into the buffer that held y^{iters-2}
  if (mixed) {
    const float *dfin = ((iters - 1) & 1) ? f->mx.da : f->mx.db;
    k_gather<<<node_blocks(n) + 1, 128, 0, f->stream>>>(f->net, f->perm, n, f->st.uo, f->st.xo,
                                                        nullptr, f->q, f->x0, out->u, out->x,
                                                        nullptr);
    k_gather_mixed_y<<<node_blocks(n) + 1, 128, 0, f->stream>>>(f->net, f->perm, n, f->mx.yb,
                                                                dfin, out->y);
  } else {
    const double *yfin = ((iters - 1) & 1) ? f->st.ya : f->st.yb;
    k_gather<<<node_blocks(n) + 1, 128, 0, f->stream>>>(f->net, f->perm, n, f->st.uo, f->st.xo,
                                                        yfin, f->q, f->x0, out->u, out->x, out->y);
  }
  if (avg)
    k_gather<<<node_blocks(n) + 1, 128, 0, f->stream>>>(f->net, f->perm, n, f->uavg, f->xavg,
                                                        nullptr, f->q, f->x0, out->u_avg,
                                                        out->x_avg, nullptr);
  RN_CUDA(cudaGetLastError());
  std::vector<unsigned long long> hist(std::max(1, nchk));
  if (nchk > 0)
    RN_CUDA(cudaMemcpyAsync(hist.data(), f->res, nchk * sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, f->stream));
  double red[3];
  if ((rc = reduce_nodes(f, 0, nullptr, red))) return rc;
  out->cost = red[0] + red[1];
  out->ubox_viol = red[2];
  out->iters = iters;
  out->n_checks = nchk;
  out->gamma = f->gamma;
  std::vector<double> rh(std::max(1, nchk));
  for (int i = 0; i < nchk; ++i) {
    double d;
    std::memcpy(&d, &hist[i], sizeof d);
    rh[i] = d * (1.0 / f->gamma);  // as the kernel's termination test
  }
  out->primal_res = nchk > 0 ? rh[nchk - 1] : NAN;
  if (out->res_hist && out->res_hist_len > 0 && nchk > 0) {
    const int m = std::min(out->res_hist_len, nchk);
    RN_CUDA(cudaMemcpyAsync(out->res_hist, rh.data(), m * sizeof(double), cudaMemcpyHostToDevice,
                            f->stream));
  }
  out->gap = NAN;
  if (out->compute_gap) {
    // x*(y) with s = (y1 + y2 | y3) of the final dual iterate
    k_init_apg<<<node_blocks(n), 128, 0, f->stream>>>(f->net, f->perm, n, out->y, f->st.ya,
                                                      f->st.yb, f->st.s);
    RN_CUDA(cudaGetLastError());
    if ((rc = solve_step(f, 0))) return rc;
    double g[3];
    if ((rc = reduce_nodes(f, 1, f->st.ya, g))) return rc;
    if ((rc = check_err(f))) return rc;
    out->gap = g[1] > 0.0 ? INFINITY : g[0];
  }
  RN_CUDA(cudaStreamSynchronize(f->stream));
  if (reason == 2) {
    set_error("the residual became non-finite after %d iterations", iters);
    return RN_ERR_DIVERGED;
  }
  if (reason == 3) return timeout_error("", 0, f->st.wait_ns);
  if (tol > 0.0 && reason != 1) return RN_NOT_CONVERGED;
  return RN_OK;
}

// Scratch of the allocation-free dual gradient: doubles for s, up, ux (SP
// per node), z, uo (NUP), xo (NXP) and the partial sums hp (SP per row, two
// buffers), then 32-bit words for the counters, flags and arrivals of the
// groups, the grid barrier, the error word and the info words.
void noalloc_need(const rn_factor *f, size_t *need_d, size_t *need_w) {
  const size_t rows = (size_t)f->plan.n;
  const size_t ng = (size_t)std::max(1, f->plan.n_groups + f->plan.n_roots);
  const size_t hrows = (size_t)std::max(1, f->plan.hp_rows);
  *need_d = rows * (3 * (size_t)f->SP + 2 * (size_t)f->NUP + (size_t)f->NXP) +
            2 * hrows * f->SP;
  *need_w = 3 * ng + 1 + 1 + 4;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" int rapidnet_factor(const rn_network *net, const rn_tree *tree, const rn_cost *cost,
                               const rn_opts *opts, rn_factor **out) {
  clear_error();
  if (!out) {
    set_error("factor: out is NULL");
    return RN_ERR_INVAL;
  }
  *out = nullptr;
  std::unique_ptr<rn_factor> f(new (std::nothrow) rn_factor());
  if (!f) {
    set_error("factor: host allocation failed");
    return RN_ERR_NOMEM;
  }
  static std::atomic<unsigned long long> next_serial{1};
  f->serial = next_serial.fetch_add(1);
  f->device = opts ? opts->device : 0;
  const int form = opts ? opts->factor_form : RN_FACTOR_AUTO;
  const int prec = opts ? opts->precision : RN_PREC_FP64;
  if (form != RN_FACTOR_AUTO && form != RN_FACTOR_SHARED && form != RN_FACTOR_PER_NODE) {
    set_error("factor_form must be RN_FACTOR_AUTO, RN_FACTOR_SHARED or RN_FACTOR_PER_NODE");
    return RN_ERR_INVAL;
  }
  bool per_node = form == RN_FACTOR_PER_NODE;
  if (form == RN_FACTOR_AUTO && net && net->A && net->nx > 0)
    per_node = prec == RN_PREC_FP32 || !is_identity(net->A, net->nx);
  int rc = per_node ? pernode_impl(net, tree, cost, opts, f.get())
                    : factor_impl(net, tree, cost, opts, f.get());
  if (rc == RN_ERR_UNSUPPORTED && form == RN_FACTOR_AUTO && !per_node &&
      prec == RN_PREC_FP64) {
    // outside what the shared-operator form lays out: the per-node form
    const std::string why = rapidnet_last_error();
    f.reset(new (std::nothrow) rn_factor());
    if (!f) {
      set_error("factor: host allocation failed");
      return RN_ERR_NOMEM;
    }
    f->serial = next_serial.fetch_add(1);
    f->device = opts ? opts->device : 0;
    clear_error();
    rc = pernode_impl(net, tree, cost, opts, f.get());
    if (rc == RN_ERR_UNSUPPORTED) set_error("%s; per-node form: %s", why.c_str(),
                                            rapidnet_last_error());
  }
  if (rc) return rc;
  *out = f.release();
  return RN_OK;
}

extern "C" void rapidnet_factor_free(rn_factor *f) { delete f; }

extern "C" int rapidnet_factor_info(const rn_factor *f, rn_factor_info *info) {
  clear_error();
  if (!f || !info) {
    set_error("factor_info: NULL argument");
    return RN_ERR_INVAL;
  }
  info->nx = f->nx;
  info->nu = f->nu;
  info->nd = f->nd;
  info->ne = f->ne;
  info->N = f->plan.N;
  info->n_nodes = f->plan.n;
  info->n_chains = f->plan.n_chains;
  info->n_top = f->plan.n_top;
  info->grid_ctas = f->grid;
  info->block_threads = f->block;
  info->L = f->L;
  info->gamma = f->gamma;
  info->precision = f->opts.precision;
  info->device_bytes = f->bytes;
  info->collapse_dev = f->collapse_dev;
  size_t need_d = 0, need_w = 0;
  noalloc_need(f, &need_d, &need_w);
  info->noalloc_bytes = (long long)(8 * (need_d + (need_w + 1) / 2));
  info->factor_form = RN_FACTOR_SHARED;
  if (f->pn) {
    pn_info(f->pn, info);
    info->device_bytes += f->bytes;
    info->collapse_dev = 0.0;
    info->noalloc_bytes = 0;
    info->factor_form = RN_FACTOR_PER_NODE;
  }
  return RN_OK;
}

extern "C" int rapidnet_solve_device(rn_factor *f, const double *x0, const double *q,
                                     const double *demand, const double *alpha, int max_iters,
                                     double tol, const double *y_warm, rn_result *out) {
  clear_error();
  return solve_device_impl(f, x0, q, demand, alpha, max_iters, tol, y_warm, out);
}

extern "C" int rapidnet_solve(rn_factor *f, const double *x0, const double *q,
                              const double *demand, const double *alpha, int max_iters, double tol,
                              const double *y_warm, rn_result *out) {
  clear_error();
  if (!f || !x0 || !q || !demand || !alpha || !out || !out->u || !out->x || !out->y) {
    set_error("solve: NULL argument");
    return RN_ERR_INVAL;
  }
  RN_CUDA(cudaSetDevice(f->device));
  const int n = f->plan.n, ny = 2 * f->nx + f->nu;
  int rc;
  // device staging of the caller's host arrays (kept by the handle)
  if (!f->io_y) {
    if ((rc = dalloc(f, &f->io_y, (size_t)n * ny)) || (rc = dalloc(f, &f->io_u, (size_t)n * f->nu)) ||
        (rc = dalloc(f, &f->io_x, (size_t)n * f->nx)))
      return rc;
  }
  // inputs: x0, q, demand, alpha land in the handle's own buffers
  RN_CUDA(cudaMemcpyAsync(f->x0, x0, f->nx * sizeof(double), cudaMemcpyHostToDevice, f->stream));
  RN_CUDA(cudaMemcpyAsync(f->q, q, f->nu * sizeof(double), cudaMemcpyHostToDevice, f->stream));
  RN_CUDA(cudaMemcpyAsync(f->demand, demand, (size_t)n * f->nd * sizeof(double),
                          cudaMemcpyHostToDevice, f->stream));
  RN_CUDA(cudaMemcpyAsync(f->alpha, alpha, (size_t)n * f->nu * sizeof(double),
                          cudaMemcpyHostToDevice, f->stream));
  if (y_warm)
    RN_CUDA(cudaMemcpyAsync(f->io_y, y_warm, (size_t)n * ny * sizeof(double),
                            cudaMemcpyHostToDevice, f->stream));
  rn_result dres = *out;
  dres.u = f->io_u;
  dres.x = f->io_x;
  dres.y = f->io_y;
  if ((out->u_avg == nullptr) != (out->x_avg == nullptr)) {
    set_error("solve: give both u_avg and x_avg, or neither");
    return RN_ERR_INVAL;
  }
  if (out->u_avg) {
    if (!f->io_uavg && ((rc = dalloc(f, &f->io_uavg, (size_t)n * f->nu)) ||
                        (rc = dalloc(f, &f->io_xavg, (size_t)n * f->nx))))
      return rc;
    dres.u_avg = f->io_uavg;
    dres.x_avg = f->io_xavg;
  }
  std::vector<double> hist;
  if (out->res_hist && out->res_hist_len > 0) {
    if (out->res_hist_len > f->io_hist_cap) {
      release(f, f->io_hist);
      f->io_hist = nullptr;
      if ((rc = dalloc(f, &f->io_hist, out->res_hist_len))) return rc;
      f->io_hist_cap = out->res_hist_len;
    }
    dres.res_hist = f->io_hist;
  } else {
    dres.res_hist = nullptr;
  }
  rc = solve_device_impl(f, f->x0, f->q, f->demand, f->alpha, max_iters, tol,
                         y_warm ? f->io_y : nullptr, &dres);
  if (rc < 0) return rc;
  RN_CUDA(cudaMemcpyAsync(out->u, f->io_u, (size_t)n * f->nu * sizeof(double),
                          cudaMemcpyDeviceToHost, f->stream));
  RN_CUDA(cudaMemcpyAsync(out->x, f->io_x, (size_t)n * f->nx * sizeof(double),
                          cudaMemcpyDeviceToHost, f->stream));
  RN_CUDA(cudaMemcpyAsync(out->y, f->io_y, (size_t)n * ny * sizeof(double),
                          cudaMemcpyDeviceToHost, f->stream));
  if (out->u_avg) {
    RN_CUDA(cudaMemcpyAsync(out->u_avg, f->io_uavg, (size_t)n * f->nu * sizeof(double),
                            cudaMemcpyDeviceToHost, f->stream));
    RN_CUDA(cudaMemcpyAsync(out->x_avg, f->io_xavg, (size_t)n * f->nx * sizeof(double),
                            cudaMemcpyDeviceToHost, f->stream));
  }
  if (dres.res_hist)
    RN_CUDA(cudaMemcpyAsync(out->res_hist, f->io_hist,
                            std::min(out->res_hist_len, std::max(dres.n_checks, 0)) * sizeof(double),
                            cudaMemcpyDeviceToHost, f->stream));
  RN_CUDA(cudaStreamSynchronize(f->stream));
  double *hu = out->u, *hx = out->x, *hy = out->y, *hh = out->res_hist;
  double *hua = out->u_avg, *hxa = out->x_avg;
  *out = dres;
  out->u = hu;
  out->x = hx;
  out->y = hy;
  out->res_hist = hh;
  out->u_avg = hua;
  out->x_avg = hxa;
  return rc;
}

extern "C" int rapidnet_dual_gradient_device(rn_factor *f, const double *x0, const double *q,
                                             const double *demand, const double *alpha,
                                             const double *w, double *u, double *x) {
  clear_error();
  if (!f || !w || !u || !x) {
    set_error("dual_gradient: NULL argument");
    return RN_ERR_INVAL;
  }
  if (f->pn) return pn_dual_gradient_device(f->pn, x0, q, demand, alpha, w, u, x);
  RN_CUDA(cudaSetDevice(f->device));
  int rc;
  if (x0 || q || demand || alpha) {
    if (!(x0 && q && demand && alpha)) {
      set_error("dual_gradient: give all of x0, q, demand, alpha or none");
      return RN_ERR_INVAL;
    }
    if ((rc = clear_err(f)) || (rc = prepare(f, x0, q, demand, alpha))) return rc;
  } else if (!f->have_data) {
    set_error("dual_gradient: no data yet (give x0, q, demand, alpha)");
    return RN_ERR_INVAL;
  }
  if (!(x0 || q || demand || alpha) && (rc = clear_err(f))) return rc;
  const int n = f->plan.n;
  k_s_from_w<<<node_blocks(n), 128, 0, f->stream>>>(f->net, f->perm, n, w, f->st.s);
  RN_CUDA(cudaGetLastError());
  if ((rc = solve_step(f, 0))) return rc;
  k_gather<<<node_blocks(n) + 1, 128, 0, f->stream>>>(f->net, f->perm, n, f->st.uo, f->st.xo,
                                                      nullptr, f->q, f->x0, u, x, nullptr);
  RN_CUDA(cudaGetLastError());
  return check_err(f);
}

// ---------------------------------------------------------------------------
// Dual gradient without any allocation
//
// For callers that must not allocate device memory once they are running:
// a real-time control loop that forbids allocation after start-up for
// predictable timing, a host application that owns the device memory pool
// and hands none of it to libraries, or an embedding that counts every byte.
// Such a caller creates the factor handle (and runs one solve or
// rapidnet_dual_gradient_device with data) during set-up; afterwards
// rapidnet_dual_gradient_noalloc evaluates x*(w) with the per-call scratch
// (backward inputs, subtree sums, path terms, outputs in internal order,
// counters and flags) taken from the fixed array below instead of the
// handle's buffers.  It calls no cudaMalloc, cudaFree or allocating
// library routine.
// ---------------------------------------------------------------------------
namespace {

// 8 MiB of doubles, held by every device that loads the library until exit
constexpr size_t kNoAllocDoubles = (size_t)1 << 20;
static_assert(kNoAllocDoubles * sizeof(double) == (size_t)RN_NOALLOC_SCRATCH_BYTES,
              "scratch size differs from the header");
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double *g_noalloc_addr[kMaxDevices] = {};

// device address of the scratch array on the current device (looked up once
// per device; the host-side name is only a stand-in for the symbol)
int noalloc_scratch(int device, double **out) {
  if (device < 0 || device >= kMaxDevices) {
    set_error("noalloc: device ordinal %d out of range", device);
    return RN_ERR_INVAL;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[device]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_error("noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return RN_ERR_CUDA;
    }
    g_noalloc_addr[device] = static_cast<double *>(p);
  }
  *out = g_noalloc_addr[device];
  return RN_OK;
}

}  // namespace

extern "C" int rapidnet_dual_gradient_noalloc(rn_factor *f, const double *w, double *u,
                                              double *x) {
  clear_error();
  if (!f || !w || !u || !x) {
    set_error("dual_gradient_noalloc: NULL argument");
    return RN_ERR_INVAL;
  }
  if (f->pn) {
    set_error("dual_gradient_noalloc: a handle of the per-node form has no allocation-free "
              "entry point");
    return RN_ERR_UNSUPPORTED;
  }
  if (!f->have_data) {
    set_error("dual_gradient_noalloc: no data yet (run a solve or "
              "rapidnet_dual_gradient_device with data during set-up)");
    return RN_ERR_INVAL;
  }
  const int n = f->plan.n;
  const size_t rows = (size_t)n;
  const size_t ng = (size_t)std::max(1, f->plan.n_groups + f->plan.n_roots);
  const size_t hrows = (size_t)std::max(1, f->plan.hp_rows);
  size_t need_d = 0, need_w = 0;
  noalloc_need(f, &need_d, &need_w);
  const size_t need = need_d + (need_w + 1) / 2;
  if (need > kNoAllocDoubles) {
    set_error("dual_gradient_noalloc: this tree needs %zu bytes of scratch, more than the "
              "static %zu bytes (n_nodes = %d)", need * sizeof(double),
              kNoAllocDoubles * sizeof(double), n);
    return RN_ERR_INVAL;
  }
  RN_CUDA(cudaSetDevice(f->device));
  double *base = nullptr;
  int rc = noalloc_scratch(f->device, &base);
  if (rc) return rc;
  StateDev<double> st = f->st;
  double *p = base;
  st.s = p;
  p += rows * f->SP;
  st.up = p;
  p += rows * f->SP;
  st.ux = p;
  p += rows * f->SP;
  st.z = p;
  p += rows * f->NUP;
  st.uo = p;
  p += rows * f->NUP;
  st.xo = p;
  p += rows * f->NXP;
  st.hp = p;
  p += 2 * hrows * f->SP;
  unsigned *words = reinterpret_cast<unsigned *>(p);
  st.count = words;
  st.flags = words + ng;
  st.arrive = words + 2 * ng;
  st.barrier = words + 3 * ng;
  st.err = reinterpret_cast<int *>(words + 3 * ng + 1);
  st.info = st.err + 1;
  st.res = nullptr;
  st.beta = nullptr;
  // the array keeps the previous call's contents: counters, flags and the
  // error word must start at zero; padding columns of s, up and ux as well
  RN_CUDA(cudaMemsetAsync(words, 0, need_w * sizeof(unsigned), f->stream));
  RN_CUDA(cudaMemsetAsync(st.s, 0, rows * 3 * f->SP * sizeof(double), f->stream));
  k_s_from_w<<<node_blocks(n), 128, 0, f->stream>>>(f->net, f->perm, n, w, st.s);
  RN_CUDA(cudaGetLastError());
  KParams<double> P = base_params(f);
  P.st = st;
  RN_CUDA((launch_solve<double, false>(P, f->grid, f->block, f->smem, f->stream)));
  k_gather<<<node_blocks(n) + 1, 128, 0, f->stream>>>(f->net, f->perm, n, st.uo, st.xo, nullptr,
                                                      f->q, f->x0, u, x, nullptr);
  RN_CUDA(cudaGetLastError());
  int e = 0;
  RN_CUDA(cudaMemcpyAsync(&e, st.err, sizeof(int), cudaMemcpyDeviceToHost, f->stream));
  RN_CUDA(cudaStreamSynchronize(f->stream));
  if (e) return timeout_error("dual_gradient_noalloc: ", e, st.wait_ns);
  return RN_OK;
}

// ---------------------------------------------------------------------------
// batched solve (many handles, one cooperative launch)
//
// A call runs, on the stream of the first handle: every problem's
// preparation (data terms, x*(0), initial dual), the persistent batched
// kernel, every problem's outputs and reductions, and one gathering kernel
// that packs each problem's scalars into a record read back with a single
// copy.  The whole sequence is captured once into a CUDA graph per set of
// handles, requests, iteration cap and tolerance, and replayed by later
// calls with the same arguments.  The launch layout (team width, teams per
// block) of a set of handles is chosen once by timing the candidates on a
// short run of the same batch (rn_opts.batch_tune of the first handle).
// ---------------------------------------------------------------------------
namespace {

// one problem's scalars after a batched solve
struct BatchRec {
  double res_last;      // residual bits of the last check (as a double's bits)
  double cost[3];       // smooth cost, soft cost, input-box violation
  int iters, nchk, reason, err;
};

struct BatchSrc {
  const int *info;                 // iterations, checks, stop reason
  const unsigned long long *res;   // residual history
  const double *scal;              // reductions of k_final_reduce
  const int *err;                  // the handle's error word (preparation)
};

__global__ void k_batch_collect(int n, const BatchSrc *src, BatchRec *out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const BatchSrc s = src[i];
    BatchRec r;
    r.iters = s.info[0];
    r.nchk = s.info[1];
    r.reason = s.info[2];
    r.err = *s.err;
    const unsigned long long b = r.nchk > 0 ? s.res[r.nchk - 1] : 0ull;
    r.res_last = __longlong_as_double((long long)b);
    r.cost[0] = s.scal[0];
    r.cost[1] = s.scal[1];
    r.cost[2] = s.scal[2];
    out[i] = r;
  }
}

// launch layout of the batched kernel for a set of handles
struct BatchLayout {
  int tw = 64, tpb = 4, block = 256, maxc = 1, grid = 0, net_f = 0, net_region = 0;
  int team_bytes = 0;
  long long items = 0;
  size_t smem = 0;
  std::vector<Sizes> szf, szd;
};

// the layout for teams of tw threads, tpb to a block (tw at least each
// problem's own team width); RN_OK or the reason the layout does not fit
int batch_layout(rn_factor *const *fs, int n, int tw, int tpb, BatchLayout *L) {
  const int dev = fs[0]->device;
  int rc;
  L->tw = tw;
  L->tpb = tpb;
  L->block = tpb * tw;
  L->net_f = 0;
  L->items = 0;
  L->maxc = 1;
  for (int i = 0; i < n; ++i) {
    L->net_f = std::max(L->net_f, fs[i]->net_bytes_f);
    L->items += fs[i]->plan.n_groups + (fs[i]->plan.n_chains + tpb - 1) / tpb;
    const int m = std::max(fs[i]->nx, fs[i]->nu);
    int c = std::max((m + tw - 1) / tw, (fs[i]->nx + 31) / 32);
    if (c > 8) {
      set_error("solve_batch: teams of %d threads are too narrow for nx = %d, nu = %d", tw,
                fs[i]->nx, fs[i]->nu);
      return RN_ERR_UNSUPPORTED;
    }
    c = c <= 1 ? 1 : (c <= 2 ? 2 : (c <= 4 ? 4 : 8));
    L->maxc = std::max(L->maxc, c);
  }
  L->net_region = L->net_f + (int)round16(sizeof(NetDev<double>));
  int static_smem = 0;
  RN_CUDA(batch_static_smem(L->maxc, &static_smem));
  if ((rc = team_budget(dev, (int)std::min<long long>(L->items, 1 << 30), tpb, L->block,
                        L->net_region, static_smem, &L->team_bytes)))
    return rc;
  L->szf.assign(n, Sizes{});
  L->szd.assign(n, Sizes{});
  for (int i = 0; i < n; ++i)
    if ((rc = fit_sizes(fs[i], 4, L->team_bytes, L->net_region, tw, tpb, 2, &L->szf[i])) ||
        (rc = fit_sizes(fs[i], 8, L->team_bytes, L->net_f, tw, tpb, 0, &L->szd[i])) ||
        (rc = check_layout(fs[i]->plan, L->szf[i], 0, 0, "solve_batch")) ||
        (rc = check_layout(fs[i]->plan, L->szd[i], 0, 0, "solve_batch")))
      return rc;
  L->smem = kHdrBytes + L->net_region + (size_t)tpb * L->team_bytes;
  int bps = 0, sms = 0;
  RN_CUDA(batch_occupancy(L->maxc, L->block, L->smem, &bps));
  RN_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (bps < 1) {
    set_error("solve_batch: the batched kernel does not fit on the device");
    return RN_ERR_UNSUPPORTED;
  }
  L->grid = (int)std::min<long long>(L->items, (long long)bps * sms);
  if (fs[0]->opts.max_ctas > 0) L->grid = std::min(L->grid, fs[0]->opts.max_ctas);
  return RN_OK;
}

// the node reductions of one handle (cost, input-box violation) into its
// scal, without reading them back
int reduce_nodes_async(rn_factor *f) {
  ReduceArgs a{f->pd.parent, f->perm, f->prob, f->alpha, f->alpha0, f->wdiag, f->q,
               f->wdense, f->st.uo, f->st.xo, nullptr, f->W_alpha, 0};
  k_node_reduce<<<kRedBlocks, 256, 0, f->stream>>>(f->net, a, f->plan.n, f->partial);
  k_final_reduce<<<1, 32, 0, f->stream>>>(f->partial, kRedBlocks, f->scal);
  RN_CUDA(cudaGetLastError());
  return RN_OK;
}

// a batch prepared for launch: its device workspace (parameters, work
// items, barrier, error and info words, result records), the pinned host
// copy of the records and, once captured, the graph
struct BatchRun {
  std::vector<unsigned long long> key;
  BatchLayout L;
  unsigned char *dev = nullptr;
  BatchRec *host = nullptr;
  size_t o_probs = 0, o_ip = 0, o_ic = 0, o_cb = 0, o_bar = 0, o_err = 0, o_info = 0, o_src = 0,
         o_rec = 0;
  cudaGraphExec_t exec = nullptr;
  bool graph = false;  // the sequence replays as a graph
  ~BatchRun() {
    if (exec) cudaGraphExecDestroy(exec);
    if (dev) cudaFree(dev);
    if (host) cudaFreeHost(host);
  }
};

// workspace, parameters and work items of a batch (host to device, before
// any capture)
int batch_setup(rn_factor *const *fs, const rn_solve_req *req, int n, int max_iters, double tol,
                BatchRun &R) {
  const BatchLayout &L = R.L;
  const int grid = L.grid;
  const long long items = L.items;
  std::vector<int> ip, ic, cb(grid + 1);
  ip.reserve(items);
  ic.reserve(items);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < fs[i]->plan.n_groups + (fs[i]->plan.n_chains + L.tpb - 1) / L.tpb; ++k) {
      ip.push_back(i);
      ic.push_back(k);
    }
  for (int b = 0; b <= grid; ++b) cb[b] = (int)((long long)b * items / grid);
  for (int b = 0; b < grid; ++b) {
    int distinct = 0;
    for (int it = cb[b]; it < cb[b + 1]; ++it)
      if (it == cb[b] || ip[it] != ip[it - 1]) ++distinct;
    if (distinct > kBatchMaxDistinct) {
      set_error("solve_batch: a block would touch %d problems (more than %d); "
                "too many small problems for this batch size", distinct, kBatchMaxDistinct);
      return RN_ERR_UNSUPPORTED;
    }
  }
  R.o_probs = 0;
  R.o_ip = round16(R.o_probs + n * sizeof(MixedParams));
  R.o_ic = round16(R.o_ip + items * sizeof(int));
  R.o_cb = round16(R.o_ic + items * sizeof(int));
  R.o_bar = round16(R.o_cb + (grid + 1) * sizeof(int));
  R.o_err = round16(R.o_bar + sizeof(unsigned));
  R.o_info = round16(R.o_err + sizeof(int));
  R.o_src = round16(R.o_info + 3 * n * sizeof(int));
  R.o_rec = round16(R.o_src + n * sizeof(BatchSrc));
  const size_t total = round16(R.o_rec + n * sizeof(BatchRec));
  void *p = nullptr;
  cudaError_t e = cudaMalloc(&p, total);
  if (e != cudaSuccess) {
    set_error("solve_batch: cudaMalloc of %zu bytes failed: %s", total, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? RN_ERR_NOMEM : RN_ERR_CUDA;
  }
  R.dev = static_cast<unsigned char *>(p);
  e = cudaMallocHost(&p, n * sizeof(BatchRec));
  if (e != cudaSuccess) {
    set_error("solve_batch: cudaMallocHost failed: %s", cudaGetErrorString(e));
    return RN_ERR_NOMEM;
  }
  R.host = static_cast<BatchRec *>(p);
  int *berr = reinterpret_cast<int *>(R.dev + R.o_err);
  std::vector<MixedParams> probs(n);
  std::vector<BatchSrc> src(n);
  const int *binfo = reinterpret_cast<const int *>(R.dev + R.o_info);
  for (int i = 0; i < n; ++i) {
    MixedParams &M = probs[i];
    M = mixed_params(fs[i], max_iters, tol);
    set_sizes(M.f, L.szf[i]);
    set_sizes(M.d, L.szd[i]);
    M.f.st.err = berr;
    M.d.st.err = berr;
    src[i] = BatchSrc{binfo + 3 * i, fs[i]->res, fs[i]->scal, fs[i]->err};
  }
  RN_CUDA(cudaMemcpy(R.dev + R.o_probs, probs.data(), n * sizeof(MixedParams),
                     cudaMemcpyHostToDevice));
  RN_CUDA(cudaMemcpy(R.dev + R.o_ip, ip.data(), items * sizeof(int), cudaMemcpyHostToDevice));
  RN_CUDA(cudaMemcpy(R.dev + R.o_ic, ic.data(), items * sizeof(int), cudaMemcpyHostToDevice));
  RN_CUDA(cudaMemcpy(R.dev + R.o_cb, cb.data(), (grid + 1) * sizeof(int), cudaMemcpyHostToDevice));
  RN_CUDA(cudaMemcpy(R.dev + R.o_src, src.data(), n * sizeof(BatchSrc), cudaMemcpyHostToDevice));
  (void)req;
  return RN_OK;
}

// the device work of a batch on stream bs (every handle's stream set to bs
// by the caller): preparations, the batched kernel between the timing
// events of the first handle, outputs, reductions, records and their copy
// to the pinned host buffer
int batch_enqueue(rn_factor *const *fs, const rn_solve_req *req, int n, int max_iters,
                  double tol, BatchRun &R, cudaStream_t bs) {
  const BatchLayout &L = R.L;
  int rc;
  for (int i = 0; i < n; ++i) {
    rn_factor *f = fs[i];
    const int ck = (max_iters + f->opts.check_every - 1) / f->opts.check_every + 1;
    if ((rc = clear_err(f)) || (rc = prepare(f, req[i].x0, req[i].q, req[i].demand, req[i].alpha)))
      return rc;
    const int nn = f->plan.n;
    k_mixed_init<<<node_blocks(nn), 128, 0, bs>>>(f->net, f->perm, nn, req[i].y_warm, f->mx.yb,
                                                  f->mx.ybh, f->mx.da, f->mx.db, f->st.s,
                                                  f->stf.s);
    RN_CUDA(cudaGetLastError());
    if ((rc = reset_sync(f))) return rc;
    RN_CUDA(cudaMemsetAsync(f->res, 0, ck * sizeof(unsigned long long), bs));
  }
  unsigned char *W = R.dev;
  int *berr = reinterpret_cast<int *>(W + R.o_err);
  RN_CUDA(cudaMemsetAsync(W + R.o_bar, 0, sizeof(unsigned), bs));
  RN_CUDA(cudaMemsetAsync(berr, 0, sizeof(int), bs));
  RN_CUDA(cudaMemsetAsync(W + R.o_info, 0, 3 * n * sizeof(int), bs));
  BatchDev B{};
  B.n_problems = n;
  B.probs = reinterpret_cast<const MixedParams *>(W + R.o_probs);
  B.item_prob = reinterpret_cast<const int *>(W + R.o_ip);
  B.item_sub = reinterpret_cast<const int *>(W + R.o_ic);
  B.cta_begin = reinterpret_cast<const int *>(W + R.o_cb);
  B.barrier = reinterpret_cast<unsigned *>(W + R.o_bar);
  B.err = berr;
  B.prob_info = reinterpret_cast<int *>(W + R.o_info);
  B.iters = max_iters;
  B.check_every = fs[0]->opts.check_every;
  B.refresh_every = fs[0]->opts.refresh_every;
  B.wait_ns = fs[0]->st.wait_ns;
  B.net_bytes = L.net_region;
  B.net_bytes_f = L.net_f;
  B.team_bytes = L.team_bytes;
  B.tpb = L.tpb;
  B.tol = tol > 0.0 ? tol : 0.0;
  RN_CUDA(launch_batch(B, L.maxc, L.grid, L.block, L.smem, bs));
  for (int i = 0; i < n; ++i) {
    rn_factor *f = fs[i];
    rn_result *out = req[i].out;
    const int nn = f->plan.n;
    // the final dual sits in the delta buffer of the last iteration's
    // parity, read from the problem's info on the device
    k_gather<<<node_blocks(nn) + 1, 128, 0, bs>>>(f->net, f->perm, nn, f->st.uo, f->st.xo,
                                                  nullptr, f->q, f->x0, out->u, out->x, nullptr);
    k_gather_mixed_y_batch<<<node_blocks(nn) + 1, 128, 0, bs>>>(
        f->net, f->perm, nn, f->mx.yb, f->mx.da, f->mx.db, B.prob_info + 3 * i, out->y);
    RN_CUDA(cudaGetLastError());
    if ((rc = reduce_nodes_async(f))) return rc;
  }
  k_batch_collect<<<(n + 127) / 128, 128, 0, bs>>>(
      n, reinterpret_cast<const BatchSrc *>(W + R.o_src), reinterpret_cast<BatchRec *>(W + R.o_rec));
  RN_CUDA(cudaGetLastError());
  RN_CUDA(cudaMemcpyAsync(R.host, W + R.o_rec, n * sizeof(BatchRec), cudaMemcpyDeviceToHost, bs));
  return RN_OK;
}

// every handle's stream set to bs for the duration of a batch, restored after
struct StreamSwap {
  std::vector<cudaStream_t> saved;
  rn_factor *const *fs;
  int n;
  StreamSwap(rn_factor *const *fs_, int n_, cudaStream_t bs) : fs(fs_), n(n_) {
    for (int i = 0; i < n; ++i) {
      saved.push_back(fs[i]->stream);
      fs[i]->stream = bs;
    }
  }
  ~StreamSwap() {
    for (int i = 0; i < n; ++i) fs[i]->stream = saved[i];
  }
};

// enqueue the batch: by graph (captured on first use, replayed after) or,
// where the capture fails, directly
int batch_launch(rn_factor *const *fs, const rn_solve_req *req, int n, int max_iters, double tol,
                 BatchRun &R, cudaStream_t bs, bool try_graph) {
  StreamSwap swap(fs, n, bs);
  // the first handle's events bracket the whole sequence on the device
  if (!R.exec && try_graph) {
    cudaGraph_t g = nullptr;
    RN_CUDA(cudaStreamBeginCapture(bs, cudaStreamCaptureModeThreadLocal));
    const int rc = batch_enqueue(fs, req, n, max_iters, tol, R, bs);
    const cudaError_t e = cudaStreamEndCapture(bs, &g);
    if (rc == RN_OK && e == cudaSuccess && g && cudaGraphInstantiate(&R.exec, g, 0) == cudaSuccess) {
      R.graph = true;
    } else {
      R.exec = nullptr;
      cudaGetLastError();  // the failed capture leaves no sticky error; clear the last one
    }
    if (g) cudaGraphDestroy(g);
    clear_error();
  }
  RN_CUDA(cudaEventRecord(fs[0]->ev0, bs));
  if (R.exec) {
    RN_CUDA(cudaGraphLaunch(R.exec, bs));
  } else {
    R.graph = false;
    if (const int rc = batch_enqueue(fs, req, n, max_iters, tol, R, bs)) return rc;
  }
  RN_CUDA(cudaEventRecord(fs[0]->ev1, bs));
  return RN_OK;
}

std::mutex g_batch_mu;
std::unique_ptr<BatchRun> g_batch_run[kMaxDevices];        // the last batch per device
std::map<std::vector<unsigned long long>, std::pair<int, int>> g_batch_tuned[kMaxDevices];

int batch_impl(rn_factor *const *fs, const rn_solve_req *req, int n, int max_iters, double tol) {
  if (!fs || !req || n < 1) {
    set_error("solve_batch: need n >= 1 handles and requests");
    return RN_ERR_INVAL;
  }
  if (max_iters < 1) {
    set_error("solve_batch: max_iters must be >= 1");
    return RN_ERR_INVAL;
  }
  const int dev = fs[0] ? fs[0]->device : -1;
  for (int i = 0; i < n; ++i) {
    rn_factor *f = fs[i];
    const rn_solve_req &r = req[i];
    if (!f || !r.x0 || !r.q || !r.demand || !r.alpha || !r.out || !r.out->u || !r.out->x ||
        !r.out->y) {
      set_error("solve_batch: NULL handle or argument in request %d", i);
      return RN_ERR_INVAL;
    }
    if (f->pn) {
      set_error("solve_batch: handle %d is of the per-node form (solve it alone)", i);
      return RN_ERR_UNSUPPORTED;
    }
    if (f->opts.precision != RN_PREC_MIXED) {
      set_error("solve_batch: handle %d is not RN_PREC_MIXED", i);
      return RN_ERR_INVAL;
    }
    if (f->dense_w) {
      set_error("solve_batch: handle %d has a dense Wu (the batched kernel applies F in its "
                "sparse form only; solve it alone)", i);
      return RN_ERR_UNSUPPORTED;
    }
    if (r.out->u_avg || r.out->x_avg) {
      set_error("solve_batch: the averaged primal iterate is not available in a batch "
                "(request %d)", i);
      return RN_ERR_UNSUPPORTED;
    }
    if (f->device != dev) {
      set_error("solve_batch: handles on different devices");
      return RN_ERR_INVAL;
    }
    if (f->opts.check_every != fs[0]->opts.check_every ||
        f->opts.refresh_every != fs[0]->opts.refresh_every) {
      set_error("solve_batch: all handles need the same check_every and refresh_every");
      return RN_ERR_INVAL;
    }
    for (int j = 0; j < i; ++j)
      if (fs[j] == f) {
        set_error("solve_batch: handle %d appears twice", i);
        return RN_ERR_INVAL;
      }
  }
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("solve_batch: device ordinal out of range");
    return RN_ERR_INVAL;
  }
  RN_CUDA(cudaSetDevice(dev));
  cudaStream_t bs = fs[0]->stream;
  int rc;
  // earlier work of every handle on its own stream ends first; buffers
  // that depend on the iteration cap are sized now (no allocation below)
  for (int i = 0; i < n; ++i) {
    rn_factor *f = fs[i];
    if (f->stream != bs) RN_CUDA(cudaStreamSynchronize(f->stream));
    const int ck = (max_iters + f->opts.check_every - 1) / f->opts.check_every + 1;
    if ((rc = ensure_beta(f, max_iters)) || (rc = ensure_res(f, ck))) return rc;
  }
  std::lock_guard<std::mutex> lock(g_batch_mu);
  // the layout: rule-based, or the fastest of the candidates timed on the
  // first batch of this set of handles
  std::vector<unsigned long long> set_key;
  int tw0 = 64;
  for (int i = 0; i < n; ++i) {
    set_key.push_back(fs[i]->serial);
    tw0 = std::max(tw0, fs[i]->tw);
  }
  const int tpb0 = tw0 <= 128 ? 4 : 2;
  std::pair<int, int> choice{tw0, tpb0};
  auto &tuned = g_batch_tuned[dev];
  if (fs[0]->opts.batch_tune == 0) {
    auto it = tuned.find(set_key);
    if (it != tuned.end()) {
      choice = it->second;
    } else {
      std::vector<std::pair<int, int>> cand{{tw0, tpb0}};
      if (tpb0 == 4) cand.push_back({tw0, 2});
      if (2 * tw0 <= 256) cand.push_back({2 * tw0, 2});
      const int titers = std::min(max_iters, 30);
      float best = 0.f;
      for (const auto &c : cand) {
        BatchRun T;
        if (batch_layout(fs, n, c.first, c.second, &T.L) != RN_OK) continue;
        if ((rc = batch_setup(fs, req, n, titers, 0.0, T))) return rc;
        if ((rc = batch_launch(fs, req, n, titers, 0.0, T, bs, false))) return rc;
        RN_CUDA(cudaStreamSynchronize(bs));
        float ms = 0.f;
        RN_CUDA(cudaEventElapsedTime(&ms, fs[0]->ev0, fs[0]->ev1));
        if (best == 0.f || ms < best) {
          best = ms;
          choice = c;
        }
      }
      clear_error();
      tuned[set_key] = choice;
    }
  }
  // the prepared batch (and its graph) of the same arguments, or a new one
  std::vector<unsigned long long> key = set_key;
  unsigned long long tb;
  std::memcpy(&tb, &tol, sizeof tb);
  key.insert(key.end(), {(unsigned long long)n, (unsigned long long)max_iters, tb,
                         (unsigned long long)choice.first, (unsigned long long)choice.second});
  for (int i = 0; i < n; ++i) {
    const rn_solve_req &r = req[i];
    for (const void *p : {(const void *)r.x0, (const void *)r.q, (const void *)r.demand,
                          (const void *)r.alpha, (const void *)r.y_warm, (const void *)r.out->u,
                          (const void *)r.out->x, (const void *)r.out->y,
                          (const void *)fs[i]->beta, (const void *)fs[i]->res})
      key.push_back((unsigned long long)(uintptr_t)p);
  }
  std::unique_ptr<BatchRun> &run = g_batch_run[dev];
  if (!run || run->key != key) {
    run.reset(new BatchRun());
    run->key = key;
    if ((rc = batch_layout(fs, n, choice.first, choice.second, &run->L)) ||
        (rc = batch_setup(fs, req, n, max_iters, tol, *run))) {
      run.reset();
      return rc;
    }
  }
  if ((rc = batch_launch(fs, req, n, max_iters, tol, *run, bs, fs[0]->opts.batch_tune != 2))) {
    run.reset();
    return rc;
  }
  RN_CUDA(cudaStreamSynchronize(bs));
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, fs[0]->ev0, fs[0]->ev1) != cudaSuccess) {
    ms = NAN;
    cudaGetLastError();
  }
  const int berr_host = [&] {
    int e = 0;
    for (int i = 0; i < n; ++i) e = e ? e : run->host[i].err;
    return e;
  }();
  int any_err = 0;
  RN_CUDA(cudaMemcpy(&any_err, run->dev + run->o_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (berr_host) return timeout_error("solve_batch (preparation): ", berr_host, fs[0]->st.wait_ns);
  if (any_err) return timeout_error("solve_batch: ", any_err, fs[0]->st.wait_ns);
  int status = RN_OK;
  for (int i = 0; i < n; ++i) {
    rn_factor *f = fs[i];
    rn_result *out = req[i].out;
    const BatchRec &r = run->host[i];
    out->iters = r.iters;
    out->n_checks = r.nchk;
    out->primal_res = r.nchk > 0 ? r.res_last * (1.0 / f->gamma) : NAN;
    out->cost = r.cost[0] + r.cost[1];
    out->ubox_viol = r.cost[2];
    out->gap = NAN;
    out->gamma = f->gamma;
    out->apg_ms = ms;
    out->t_begin_ns = out->t_end_ns = 0;
    if (r.reason == 2) status = RN_ERR_DIVERGED;
    else if (tol > 0.0 && r.reason != 1 && status == RN_OK) status = RN_NOT_CONVERGED;
  }
  if (status == RN_ERR_DIVERGED) set_error("solve_batch: a residual became non-finite");
  return status;
}

}  // namespace

extern "C" int rapidnet_solve_batch(rn_factor *const *f, const rn_solve_req *req, int n,
                                    int max_iters, double tol) {
  clear_error();
  return batch_impl(f, req, n, max_iters, tol);
}
