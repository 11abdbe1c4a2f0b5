// Per-node factor form of the dual gradient: kernels and host driver.
//
// Paper §4.4 evaluates x*(w) by a Riccati-type recursion with one set of
// matrices per node, and §5.2 runs its products stage by stage as batched
// matrix-vector products.  This form keeps one (Phi_nu, K_nu) pair per node
// (from the factor step in pernode_factor.cpp) and streams both from
// device memory at every evaluation:
//   backward (stage N .. 1):
//     lambda_nu = w1 + w2 + A' sum_c lambda_c
//     g_nu      = c0_nu + w3 + B' lambda_nu + sum_c r_c
//     m_nu      = mc_nu - Phi_nu g_nu
//     r_nu      = -2 p_nu W_u m_nu
//   forward (stage 1 .. N):
//     u_nu = m_nu + K_nu u_a(nu),  x_nu = A x_a(nu) + B u_nu + Gd d_nu
// followed at every node by the dual update of eqs. apg:1 / apg:2.  Unlike
// the shared-operator kernels it needs neither A = I nor the collapse of
// the per-node factors, and it is bound by the stream of 2 nu^2 matrix
// entries per node and iteration.
//
// One persistent cooperative launch runs all iterations.  A block is a set
// of teams (four warps each); every team owns whole chains (the path below
// a node with a single leaf under it) and some top nodes (two or more
// leaves below), and walks a fixed list of work items per iteration: its
// chains leaf to head, the top nodes stage by stage up, then down, then its
// chains head to leaf.  Grid barriers separate the stages of the top nodes
// only; a chain needs no synchronisation beyond its team.  The matrices of
// the team's items arrive in order through a ring of shared-memory slots
// filled by bulk copies (cp.async.bulk, completion on an mbarrier per
// slot), issued as far ahead as the ring allows, independent of the data:
// the copy engine streams the next rows while the warps work on the
// current ones.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <thread>
#include <vector>

#include "pernode.h"

namespace rn {
namespace {

__device__ __forceinline__ unsigned long long pn_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void team_sync(int team, int nt) {
  asm volatile("bar.sync %0, %1;" ::"r"(team + 1), "r"(nt) : "memory");
}

template <typename T>
__device__ __forceinline__ T wsum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ unsigned long long res_bits(double d) {
  return (unsigned long long)__double_as_longlong(fabs(d));
}

// mbarrier and bulk copy (PTX ISA: mbarrier.*, cp.async.bulk)
__device__ __forceinline__ void mb_init(unsigned long long *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mb_expect_tx(unsigned long long *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mb_try_wait(unsigned long long *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes,
                                         unsigned long long *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// 16-byte copies global -> shared (L2 only) in commit groups
__device__ __forceinline__ void cp16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Ring of matrix chunks of one team.  A node's matrix is stored as nch
// column blocks of qw 16-byte units (the last one narrower), each block nu
// rows in row-major order; chunk i is block c = i mod nch of the matrix of
// the team's item (i / nch) mod n_items, in slot i mod slots; its mbarrier
// completes phase (i / slots) mod 2.
template <typename T>
struct Ring {
  const PnParams<T> *P;
  T *slot0;
  unsigned long long *bar;
  const int *items;  // the team's items of one iteration
  int n_items;
  long long issued, cons, limit;
  // incremental positions (no 64-bit division on the way): slot and phase
  // parity of the next chunk to consume and to issue, the issued chunk's
  // block within its matrix; thread 0 also keeps the item of the chunks
  // being issued, the next one (loaded ahead) and its index
  int cslot, islot, ic;
  unsigned cpar;
  int icur, inext, iidx;
  __device__ void issue_one(int tid) {
    if (tid == 0) {
      constexpr int VW = 16 / sizeof(T);
      if (ic == 0 && issued > 0) {  // the next item; the one after it is loaded ahead
        iidx = iidx + 1 == n_items ? 0 : iidx + 1;
        icur = inext;
        inext = items[iidx + 1 == n_items ? 0 : iidx + 1];
      }
      const int v = icur & kPnNodeMask;
      const int w = min(P->qw, P->ldm / VW - ic * P->qw);  // 16-byte units of this block
      const unsigned bytes = (unsigned)(P->nu * w * 16);
      const T *src = ((icur & kPnK) ? P->K : P->Phi) + (size_t)v * P->mstride +
                     (size_t)P->nu * ic * P->qw * VW;
      // the slot's previous chunk was read by the team before the barrier
      // that precedes this call: the reads are complete, and the copy that
      // overwrites them is ordered after them (as a consumer release before
      // a producer's refill)
      mb_expect_tx(bar + islot, bytes);
      bulk_g2s(slot0 + (size_t)islot * P->slot_elems, src, bytes, bar + islot);
    }
    ++issued;
    if (++ic == P->nch) ic = 0;
    if (++islot == P->slots) islot = 0;
  }
  // wait for the next chunk to consume (every thread of the team); false on
  // timeout (after an error elsewhere it returns false at once: the launch
  // is being abandoned, and the drain at the end waits for what is in flight)
  __device__ bool wait(bool drain = false) const {
    unsigned long long *b = bar + cslot;
    if (mb_try_wait(b, cpar)) return true;
    if (!drain && *(volatile int *)P->err != 0) return false;
    // a copy of device memory completes by itself: the drain waits for it
    // whatever the handle's wait bound (up to 2 s)
    const long long lim = drain ? 2000000000LL : P->wait_ns;
    const unsigned long long t0 = pn_ns();
    while (!mb_try_wait(b, cpar))
      if ((long long)(pn_ns() - t0) > lim) return false;
    return true;
  }
  __device__ const T *slot() const { return slot0 + (size_t)cslot * P->slot_elems; }
  __device__ void consumed() {
    ++cons;
    if (++cslot == P->slots) {
      cslot = 0;
      cpar ^= 1u;
    }
  }
};

// out[i] = base[i] + sgn * (M_i . vec) for the nu rows of the team's current
// item, block of columns by block out of the ring; vec (smem) is zero
// beyond nu.  Thread t owns rows t, t + nt, ... and keeps their sums in
// registers over the blocks: no reduction between threads.  A block's row
// pitch is an odd number of 16-byte units (but for the last block), so the
// 8 threads of a shared-memory phase read 8 distinct bank groups; vec is
// read by all threads at once (broadcast).
template <typename T, int MR>  // MR: rows per thread (nu <= 128 MR)
__device__ void ring_matvec(Ring<T> &R, const T *vec, const T *base, T sgn, T *out, T *gout,
                            bool base_pending, int team, int tid, int nt) {
  const PnParams<T> &P = *R.P;
  constexpr int VW = 16 / sizeof(T);
  using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  const V *vq = reinterpret_cast<const V *>(vec);
  T acc[MR], acc2[MR];
#pragma unroll
  for (int r = 0; r < MR; ++r) acc[r] = acc2[r] = T(0);
  const int nqt = P.ldm / VW;
  for (int c = 0; c < P.nch; ++c) {
    if (!R.wait()) {
      if (tid == 0) atomicCAS(P.err, 0, 5);
      R.limit = R.issued;  // no further copies into a ring that is being abandoned
    }
    const V *S = reinterpret_cast<const V *>(R.slot());
    const int q0 = c * P.qw, w = min(P.qw, nqt - q0);
#pragma unroll
    for (int r = 0; r < MR; ++r) {
      const int i = tid + r * nt;
      if (i < P.nu) {
        const V *row = S + (size_t)i * w;
        T a0 = acc[r], a1 = acc2[r];
        for (int k = 0; k < w; ++k) {
          const V a = row[k], b = vq[q0 + k];
          if constexpr (sizeof(T) == 4) {
            a0 = fmaf(a.x, b.x, a0);
            a1 = fmaf(a.y, b.y, a1);
            a0 = fmaf(a.z, b.z, a0);
            a1 = fmaf(a.w, b.w, a1);
          } else {
            a0 = fma(a.x, b.x, a0);
            a1 = fma(a.y, b.y, a1);
          }
        }
        acc[r] = a0;
        acc2[r] = a1;
      }
    }
    team_sync(team, nt);  // the slot is free again
    R.consumed();
    if (R.issued < R.limit) R.issue_one(tid);
  }
  // a base row still in flight (the second newest copy group) lands first
  if (base_pending) {
    cp_wait<1>();
    team_sync(team, nt);
  }
#pragma unroll
  for (int r = 0; r < MR; ++r) {
    const int i = tid + r * nt;
    if (i < P.nu) {
      const T val = (base ? base[i] : T(0)) + sgn * (acc[r] + acc2[r]);
      out[i] = val;
      if (gout) gout[i] = val;
    }
  }
  team_sync(team, nt);
}

// sum over a compressed row
template <typename T>
__device__ __forceinline__ T csr_dot(const int *p, const int *ix, const T *val, int row,
                                     const T *x) {
  T s = T(0);
  for (int e = p[row]; e < p[row + 1]; ++e) s = fma(val[e], x[ix[e]], s);
  return s;
}

template <typename T>
__device__ __forceinline__ T clampv(T v, T lo, T hi) {
  return v < lo ? lo : (v > hi ? hi : v);
}

// grid barrier of the persistent launch (all blocks resident); false on
// timeout or an error raised elsewhere
__device__ bool grid_barrier(unsigned *bar, unsigned target, int *err, long long wait_ns) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    __threadfence();
    atomicAdd(bar, 1u);
    const unsigned long long t0 = pn_ns();
    while (true) {
      unsigned v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
      if (v >= target) break;
      if (*(volatile int *)err != 0) {
        ok = 0;
        break;
      }
      if ((long long)(pn_ns() - t0) > wait_ns) {
        atomicCAS(err, 0, 4);
        ok = 0;
        break;
      }
    }
    if (ok && *(volatile int *)err != 0) ok = 0;
  }
  __syncthreads();
  return ok != 0;
}

// the flag of another team's node reached `target` (bounded spin by one
// thread; the caller's team barrier then orders the team's reads after it)
__device__ bool wait_flag(const unsigned *f, unsigned target, int *err, long long wait_ns) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(f) : "memory");
  if (v >= target) return true;
  const unsigned long long t0 = pn_ns();
  while (true) {
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(f) : "memory");
    if (v >= target) return true;
    if (*(volatile int *)err != 0) return false;
    if ((long long)(pn_ns() - t0) > wait_ns) {
      atomicCAS(err, 0, 6);
      return false;
    }
  }
}

// publish a node's results of iteration `stamp - 1` (after the team barrier
// that follows their stores)
__device__ __forceinline__ void set_flag(unsigned *f, unsigned stamp) {
  __threadfence();
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(f), "r"(stamp) : "memory");
}

}  // namespace

// ---------------------------------------------------------------------------
// the persistent kernel: P.iters APG iterations (P.apg = 1) or one
// evaluation of x*(w) with w = ya (P.apg = 0)
// ---------------------------------------------------------------------------
template <typename T>
struct TeamVec {
  T *sl, *sr, *lamb, *rr, *g, *mv;  // backward: child sums, own sums, g, m
  T *xa, *ua, *x, *u;               // forward: parent values, own values
  T *red;                           // 2 * 32 reduction slots
  T *pf, *mb;                       // prefetched rows: 3 buffers of P.vb, 2 m rows of vup
  int vup;
};

// The rows an item reads besides its matrix, copied ahead into shared
// memory (one copy group per thread): y^nu and y^{nu-1} of the node, then
// c0 and mc (backward) or Gd d (forward).  Buffer layout: yc (YP) | yp (YP)
// | b1 (max(NUP, NXP)) | b2 (NUP).
template <typename T>
__device__ void prefetch_item(const PnParams<T> &P, int item, const T *ycur, const T *yprv,
                              T *dst, int tid, int nt) {
  constexpr int per = 16 / sizeof(T);
  const int v = item & kPnNodeMask;
  const bool fw = (item & kPnK) != 0;
  const int YP = P.YP;
  if (P.delta && fw) {  // the base rows of the delta form: ybh (YP) | xref (NXP) | uref (NUP)
    const T *yc = ycur + (size_t)v * YP, *yp = yprv + (size_t)v * YP;
    const T *bh = P.ybh + (size_t)v * YP, *xr = P.xref + (size_t)v * P.NXP,
            *ur = P.uref + (size_t)v * P.NUP;
    const int uY = YP / per, uX = P.NXP / per, uU = P.NUP / per;
    for (int e = tid; e < 3 * uY + uX + uU; e += nt) {
      if (e < uY)
        cp16(dst + e * per, yc + e * per);
      else if (e < 2 * uY)
        cp16(dst + YP + (e - uY) * per, yp + (e - uY) * per);
      else if (e < 3 * uY)
        cp16(dst + 2 * YP + (e - 2 * uY) * per, bh + (e - 2 * uY) * per);
      else if (e < 3 * uY + uX)
        cp16(dst + 3 * YP + (e - 3 * uY) * per, xr + (e - 3 * uY) * per);
      else
        cp16(dst + 3 * YP + P.NXP + (e - 3 * uY - uX) * per, ur + (e - 3 * uY - uX) * per);
    }
    cp_commit();
    return;
  }
  const T *b1 = fw ? (P.gd ? P.gd + (size_t)v * P.NXP : nullptr)
                   : (P.c0 ? P.c0 + (size_t)v * P.NUP : nullptr);
  const T *b2 = (!fw && P.mc) ? P.mc + (size_t)v * P.NUP : nullptr;
  const int uY = YP / per, u1 = b1 ? (fw ? P.NXP : P.NUP) / per : 0, u2 = b2 ? P.NUP / per : 0;
  const T *yc = ycur + (size_t)v * YP, *yp = yprv + (size_t)v * YP;
  for (int e = tid; e < 2 * uY + u1 + u2; e += nt) {
    if (e < uY)
      cp16(dst + e * per, yc + e * per);
    else if (e < 2 * uY)
      cp16(dst + YP + (e - uY) * per, yp + (e - uY) * per);
    else if (e < 2 * uY + u1)
      cp16(dst + 2 * YP + (e - 2 * uY) * per, b1 + (e - 2 * uY) * per);
    else
      cp16(dst + 2 * YP + P.b1 + (e - 2 * uY - u1) * per, b2 + (e - 2 * uY - u1) * per);
  }
  cp_commit();
}

template <typename T, int MR>
__device__ void backward_item(const PnParams<T> &P, Ring<T> &R, TeamVec<T> &V, int item,
                              const T *pf, T beta, unsigned stamp, int team, int tid, int nt) {
  const int v = item & kPnNodeMask;
  const int nx = P.nx, nu = P.nu, NXP = P.NXP, NUP = P.NUP;
  if (item & kPnTop) {
    const int c0 = P.cbeg[v], c1 = P.cend[v];
    // the children's sums of this iteration (other teams)
    if (tid == 0)
      for (int c = c0; c < c1; ++c) wait_flag(P.nflag + c, stamp, P.err, P.wait_ns);
    team_sync(team, nt);
    for (int i = tid; i < nx; i += nt) {
      T s = T(0);
      for (int c = c0; c < c1; ++c) s += __ldcg(P.lam + (size_t)c * NXP + i);
      V.sl[i] = s;
    }
    for (int j = tid; j < nu; j += nt) {
      T s = T(0);
      for (int c = c0; c < c1; ++c) s += __ldcg(P.r + (size_t)c * NUP + j);
      V.sr[j] = s;
    }
  } else if (item & kPnFirst) {  // a leaf
    for (int i = tid; i < nx; i += nt) V.sl[i] = T(0);
    for (int j = tid; j < nu; j += nt) V.sr[j] = T(0);
  }
  team_sync(team, nt);
  const bool publish = (item & (kPnTop | kPnLast)) != 0;
  const T *yc = pf, *yp = pf + P.YP;  // prefetched rows (see prefetch_item)
  const T *c0 = P.c0 ? pf + 2 * P.YP : nullptr, *mc = P.mc ? pf + 2 * P.YP + P.b1 : nullptr;
  for (int i = tid; i < nx; i += nt) {
    const T a1 = yc[i], a2 = yc[NXP + i];
    const T w1 = a1 + beta * (a1 - yp[i]), w2 = a2 + beta * (a2 - yp[NXP + i]);
    const T l = (w1 + w2) + csr_dot(P.Atp, P.Ati, P.Atv, i, V.sl);
    V.lamb[i] = l;
    if (publish) P.lam[(size_t)v * NXP + i] = l;
  }
  team_sync(team, nt);
  for (int j = tid; j < nu; j += nt) {
    const T a3 = yc[2 * NXP + j];
    const T w3 = a3 + beta * (a3 - yp[2 * NXP + j]);
    const T c = c0 ? c0[j] : T(0);
    V.g[j] = (c + w3) + csr_dot(P.Btp, P.Bti, P.Btv, j, V.lamb) + V.sr[j];
  }
  team_sync(team, nt);
  // m = mc - Phi g (the matrix streams through the ring)
  ring_matvec<T, MR>(R, V.g, mc, T(-1), V.mv, P.m + (size_t)v * NUP, false, team, tid, nt);
  const T w2p = T(-2.0 * P.prob[v]);
  for (int j = tid; j < nu; j += nt) {
    const T rv = w2p * csr_dot(P.Wp, P.Wi, P.Wv, j, V.mv);
    V.rr[j] = rv;
    if (publish) P.r[(size_t)v * NUP + j] = rv;
  }
  if (publish) {  // a chain head's or top node's sums, for its parent
    team_sync(team, nt);
    if (tid == 0) set_flag(P.nflag + v, stamp);
  }
  // this node's sums are its parent's child sums when the chain goes on
  T *t = V.sl;
  V.sl = V.lamb;
  V.lamb = t;
  t = V.sr;
  V.sr = V.rr;
  V.rr = t;
}

// The dual update in delta form (RN_PREC_MIXED): with h = fl32(yb), the
// delta dw of w and x = xref + x_lin(dw), the clamp of w = h + dw onto
// gamma (box - x) decides, and the new delta d+ = y+ - h is formed from
// small terms (dw - edge, or -h) so that the increments of a small step
// survive in FP32:
//   g = t - h with t = w - clamp(w, gamma (lo - x), gamma (hi - x)),
//   d+ = g, or h (q - 1) + g q when the ball |t| <= W is active
//   (q = W / |t|), and d+ = dw - edge, or -h, on the input block.
template <typename T>
__device__ void delta_prox(const PnParams<T> &P, TeamVec<T> &V, int v, const T *pf, T *yprv,
                           T beta, bool write_out, unsigned long long &rbits, int team, int tid,
                           int nt) {
  const int nx = P.nx, nu = P.nu, NXP = P.NXP, YP = P.YP;
  const T g = (T)P.gamma;
  const T *dc = pf, *dp = pf + YP, *bh = pf + 2 * YP, *xr = pf + 3 * YP, *ur = xr + NXP;
  T *dn = yprv + (size_t)v * YP;
  T *sw = (write_out && P.swy) ? P.swy + (size_t)v * YP : nullptr;
  T n1 = T(0), n2 = T(0);
  for (int i = tid; i < nx; i += nt) {
    const T w1 = dc[i] + beta * (dc[i] - dp[i]), w2 = dc[NXP + i] + beta * (dc[NXP + i] - dp[NXP + i]);
    const T h1 = bh[i], h2 = bh[NXP + i];
    const T x = xr[i] + V.x[i];
    const T lo = g * (P.xmin[i] - x), hi = g * (P.xmax[i] - x), wa = h1 + w1;
    const T g1 = wa > hi ? w1 - hi : (wa < lo ? w1 - lo : -h1);
    const T sa = g * (P.xs[i] - x);
    const T g2 = (h2 + w2) < sa ? w2 - sa : -h2;
    const T t1 = h1 + g1, t2 = h2 + g2;
    n1 += t1 * t1;
    n2 += t2 * t2;
  }
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  n1 = wsum(n1);
  n2 = wsum(n2);
  if (lane == 0) {
    V.red[warp] = n1;
    V.red[32 + warp] = n2;
  }
  team_sync(team, nt);
  n1 = T(0);
  n2 = T(0);
  for (int w = 0; w < nw; ++w) {
    n1 += V.red[w];
    n2 += V.red[32 + w];
  }
  const T q1 = n1 > T(0) ? P.Wx / sqrt(n1) : T(1);
  const T q2 = n2 > T(0) ? P.Ws / sqrt(n2) : T(1);
  for (int i = tid; i < nx; i += nt) {
    const T w1 = dc[i] + beta * (dc[i] - dp[i]), w2 = dc[NXP + i] + beta * (dc[NXP + i] - dp[NXP + i]);
    const T h1 = bh[i], h2 = bh[NXP + i];
    const T x = xr[i] + V.x[i];
    const T lo = g * (P.xmin[i] - x), hi = g * (P.xmax[i] - x), wa = h1 + w1;
    const T g1 = wa > hi ? w1 - hi : (wa < lo ? w1 - lo : -h1);
    const T sa = g * (P.xs[i] - x);
    const T g2 = (h2 + w2) < sa ? w2 - sa : -h2;
    const T d1 = q1 < T(1) ? fma(h1, q1 - T(1), g1 * q1) : g1;
    const T d2 = q2 < T(1) ? fma(h2, q2 - T(1), g2 * q2) : g2;
    rbits = max(rbits, max(res_bits((double)(d1 - w1)), res_bits((double)(d2 - w2))));
    dn[i] = d1;
    dn[NXP + i] = d2;
    if (sw) {
      sw[i] = w1;
      sw[NXP + i] = w2;
    }
  }
  for (int j = tid; j < nu; j += nt) {
    const T a3 = dc[2 * NXP + j];
    const T w3 = a3 + beta * (a3 - dp[2 * NXP + j]);
    const T h3 = bh[2 * NXP + j];
    const T u = ur[j] + V.u[j];
    const T lo = g * (P.umin[j] - u), hi = g * (P.umax[j] - u), wa = h3 + w3;
    const T d3 = wa > hi ? w3 - hi : (wa < lo ? w3 - lo : -h3);
    rbits = max(rbits, res_bits((double)(d3 - w3)));
    dn[2 * NXP + j] = d3;
    if (sw) sw[2 * NXP + j] = w3;
  }
}

template <typename T, int MR>
__device__ void forward_item(const PnParams<T> &P, Ring<T> &R, TeamVec<T> &V, int item,
                             const T *pf, const T *mrow, T *yprv, T beta, bool write_out,
                             double theta, unsigned long long &rbits, unsigned stamp, int team,
                             int tid, int nt) {
  const int v = item & kPnNodeMask;
  const int nx = P.nx, nu = P.nu, NXP = P.NXP, NUP = P.NUP;
  if (item & (kPnTop | kPnFirst)) {
    const int a = P.anc[v];
    if (a == 0) {
      for (int i = tid; i < nx; i += nt) V.xa[i] = P.x0 ? P.x0[i] : T(0);
      for (int j = tid; j < nu; j += nt) V.ua[j] = P.q ? P.q[j] : T(0);
    } else {
      // the parent's values of this iteration (another team)
      if (tid == 0) wait_flag(P.nflag + P.n + a, stamp, P.err, P.wait_ns);
      team_sync(team, nt);
      for (int i = tid; i < nx; i += nt) V.xa[i] = __ldcg(P.xo + (size_t)a * NXP + i);
      for (int j = tid; j < nu; j += nt) V.ua[j] = __ldcg(P.uo + (size_t)a * NUP + j);
    }
  }
  team_sync(team, nt);
  // u = m + K u_a
  const bool top = (item & kPnTop) != 0;
  const bool store = top || write_out || !P.apg;
  ring_matvec<T, MR>(R, V.ua, mrow, T(1), V.u, store ? P.uo + (size_t)v * NUP : (T *)nullptr, true,
              team, tid, nt);
  const T *gdr = P.gd ? pf + 2 * P.YP : nullptr;
  for (int i = tid; i < nx; i += nt) {
    const T gd = gdr ? gdr[i] : T(0);
    const T xv = (gd + csr_dot(P.Ap, P.Ai, P.Av, i, V.xa)) + csr_dot(P.Bp, P.Bi, P.Bv, i, V.u);
    V.x[i] = xv;
    if (store) P.xo[(size_t)v * NXP + i] = xv;
  }
  if (P.uavg) {  // (the delta form adds x*(yb))
    const T *xr = P.delta ? pf + 3 * P.YP : nullptr, *ur = P.delta ? xr + NXP : nullptr;
    for (int i = tid; i < nx; i += nt) {
      double *xa = P.xavg + (size_t)v * NXP + i;
      *xa = (1.0 - theta) * *xa + theta * (double)(V.x[i] + (xr ? xr[i] : T(0)));
    }
    for (int j = tid; j < nu; j += nt) {
      double *ua = P.uavg + (size_t)v * NUP + j;
      *ua = (1.0 - theta) * *ua + theta * (double)(V.u[j] + (ur ? ur[j] : T(0)));
    }
  }
  if (P.apg && P.delta) {
    delta_prox(P, V, v, pf, yprv, beta, write_out, rbits, team, tid, nt);
  } else if (P.apg) {
    // y+ = prox_{gamma g*}(w + gamma H x): distance-to-set prox of the soft
    // state terms (§4.3) through the Moreau decomposition (§4.2), box
    // projection on the input block
    const T g = (T)P.gamma, ig = (T)P.invgamma;
    const T *yc = pf, *yo = pf + P.YP;  // y^nu, y^{nu-1} (prefetched)
    T *yn = yprv + (size_t)v * P.YP;   // y^{nu+1} replaces y^{nu-1}
    T n1 = T(0), n2 = T(0);
    for (int i = tid; i < nx; i += nt) {
      const T a1 = yc[i], a2 = yc[NXP + i];
      const T w1 = a1 + beta * (a1 - yo[i]), w2 = a2 + beta * (a2 - yo[NXP + i]);
      const T v1 = V.x[i] + w1 * ig, v2 = V.x[i] + w2 * ig;
      const T e1 = v1 - clampv(v1, P.xmin[i], P.xmax[i]);
      const T e2 = fmin(v2 - P.xs[i], T(0));
      n1 += e1 * e1;
      n2 += e2 * e2;
    }
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    n1 = wsum(n1);
    n2 = wsum(n2);
    if (lane == 0) {
      V.red[warp] = n1;
      V.red[32 + warp] = n2;
    }
    team_sync(team, nt);
    n1 = T(0);
    n2 = T(0);
    for (int w = 0; w < nw; ++w) {
      n1 += V.red[w];
      n2 += V.red[32 + w];
    }
    const T s1 = n1 > T(0) ? fmin(g, P.Wx / sqrt(n1)) : T(0);
    const T s2 = n2 > T(0) ? fmin(g, P.Ws / sqrt(n2)) : T(0);
    for (int i = tid; i < nx; i += nt) {
      const T a1 = yc[i], a2 = yc[NXP + i];
      const T w1 = a1 + beta * (a1 - yo[i]), w2 = a2 + beta * (a2 - yo[NXP + i]);
      const T v1 = V.x[i] + w1 * ig, v2 = V.x[i] + w2 * ig;
      const T y1 = (v1 - clampv(v1, P.xmin[i], P.xmax[i])) * s1;
      const T y2 = fmin(v2 - P.xs[i], T(0)) * s2;
      const unsigned long long b1 = res_bits((double)(y1 - w1)), b2 = res_bits((double)(y2 - w2));
      rbits = max(rbits, max(b1, b2));
      yn[i] = y1;
      yn[NXP + i] = y2;
    }
    for (int j = tid; j < nu; j += nt) {
      const T a3 = yc[2 * NXP + j];
      const T w3 = a3 + beta * (a3 - yo[2 * NXP + j]);
      const T v3 = V.u[j] + w3 * ig;
      const T y3 = g * (v3 - clampv(v3, P.umin[j], P.umax[j]));
      rbits = max(rbits, res_bits((double)(y3 - w3)));
      yn[2 * NXP + j] = y3;
    }
  }
  if (top) {  // a top node's values, for its children
    team_sync(team, nt);
    if (tid == 0) set_flag(P.nflag + P.n + v, stamp);
  }
  T *t = V.xa;
  V.xa = V.x;
  V.x = t;
  t = V.ua;
  V.ua = V.u;
  V.u = t;
}

template <typename T, int MR>
__global__ void __launch_bounds__(512, 1) k_pn_solve(PnParams<T> P) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int nt = P.team_threads, team = threadIdx.x / nt, tid = threadIdx.x % nt;
  const int gteam = blockIdx.x * P.teams + team;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const unsigned long long t = pn_ns();
    memcpy(P.info + 4, &t, sizeof t);
  }
  const size_t mb_bytes = ((size_t)P.teams * 8 * 8 + 127) & ~(size_t)127;  // up to 8 slots
  const size_t ring_bytes = ((size_t)P.slots * P.slot_elems * sizeof(T) + 127) & ~(size_t)127;
  const size_t vec_bytes = ((size_t)P.vec_elems * sizeof(T) + 127) & ~(size_t)127;
  unsigned char *base = smem + mb_bytes + (size_t)team * (ring_bytes + vec_bytes);
  unsigned long long *bars = reinterpret_cast<unsigned long long *>(smem) + team * P.slots;
  T *vec = reinterpret_cast<T *>(base + ring_bytes);
  for (int e = tid; e < P.vec_elems; e += nt) vec[e] = T(0);
  if (tid == 0) {
    for (int s = 0; s < P.slots; ++s) mb_init(bars + s, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  TeamVec<T> V;
  {
    T *p = vec;
    V.sl = p; p += P.NXP;
    V.lamb = p; p += P.NXP;
    // vectors of nu read against a matrix row span the row pitch ldm
    const int vup = (max(P.NUP, P.ldm) + 3) & ~3;
    V.sr = p; p += vup;
    V.rr = p; p += vup;
    V.g = p; p += vup;
    V.mv = p; p += vup;
    V.red = p; p += 64;
    V.pf = p; p += 3 * P.vb;
    V.mb = p;
    V.vup = vup;
    V.xa = V.sl;  // the forward reuses the backward's region
    V.x = V.lamb;
    V.ua = V.sr;
    V.u = V.rr;
  }
  const int *seg = P.seg + (size_t)gteam * (P.n_seg + 1);
  Ring<T> R;
  R.P = &P;
  R.slot0 = reinterpret_cast<T *>(base);
  R.bar = bars;
  R.items = P.items + seg[0];
  R.n_items = seg[P.n_seg] - seg[0];
  R.issued = R.cons = 0;
  R.cslot = R.islot = R.ic = 0;
  R.cpar = 0u;
  R.limit = R.n_items > 0 ? (long long)R.n_items * P.nch * (P.apg ? P.iters : 1) : 0;
  if (tid == 0 && R.n_items > 0) {
    R.iidx = 0;
    R.icur = R.items[0];
    R.inext = R.items[R.n_items > 1 ? 1 : 0];
  }
  for (int s = 0; s < P.slots && R.issued < R.limit; ++s) R.issue_one(tid);
  unsigned nbar = 0;
  int it = 0, ci = 0, reason = 0;  // reason: 0 max iters, 1 converged, 2 non-finite, 3 wait
  bool pend = false;
  const int TT = P.t_top;
  const int n_it = P.apg ? P.iters : 1;
  for (; it < n_it; ++it) {
    const int git = P.it0 + it;  // iteration of the solve
    const T *ycur = (git & 1) ? P.yb : P.ya;
    T *yprv = P.apg ? ((git & 1) ? P.ya : P.yb) : P.ya;
    const T beta = P.apg ? (T)P.beta[git] : T(0);
    const double theta = P.apg ? P.theta[git] : 1.0;
    const bool check =
        P.apg && (((git + 1) % P.check_every) == 0 || git + 1 == P.iters_total);
    const bool wout = !P.apg || check;
    const unsigned stamp = (unsigned)it + 1u;  // flags of this iteration's results
    unsigned long long rbits = 0ull;
    // one item: the rows of the next item are requested before this one's
    // wait (three row buffers, two m buffers, in item order; nothing is
    // requested across the end of an iteration, whose last item may write
    // rows the next one reads)
    const int k0 = seg[0], kend = seg[P.n_seg];
    // items k and k + 1 in registers, k + 2 on its way (called for k = k0, k0 + 1, ...)
    int ia = k0 < kend ? P.items[k0] : 0, ib = k0 + 1 < kend ? P.items[k0 + 1] : 0;
    auto run_item = [&](int k) {
      const int item = ia, next = ib, kk = k - k0;
      ia = ib;
      ib = k + 2 < kend ? P.items[k + 2] : 0;
      const bool fw = (item & kPnK) != 0;
      T *pfk = V.pf + (kk % 3) * P.vb;
      if (kk == 0) {
        team_sync(team, nt);  // the rows the previous iteration wrote
        prefetch_item(P, item, ycur, yprv, pfk, tid, nt);
      }
      T *mrow = V.mb + (kk & 1) * V.vup;
      if (fw) {  // m of this node, written by its backward step
        constexpr int per = 16 / sizeof(T);
        const T *src = P.m + (size_t)(item & kPnNodeMask) * P.NUP;
        for (int e = tid; e < P.NUP / per; e += nt) cp16(mrow + e * per, src + e * per);
        cp_commit();
      }
      if (k + 1 < kend)
        prefetch_item(P, next, ycur, yprv, V.pf + ((kk + 1) % 3) * P.vb, tid, nt);
      else
        cp_commit();
      if (fw) {
        cp_wait<2>();
        forward_item<T, MR>(P, R, V, item, pfk, mrow, yprv, beta, wout, theta, rbits, stamp, team,
                            tid, nt);
      } else {
        cp_wait<1>();
        backward_item<T, MR>(P, R, V, item, pfk, beta, stamp, team, tid, nt);
      }
    };
    // chains, leaf to head
    for (int k = seg[0]; k < seg[1]; ++k) run_item(k);
    if (pend) {  // the check of the previous iteration, once every block has added to it
      if (!grid_barrier(P.bar, ++nbar * gridDim.x, P.err, P.wait_ns)) {
        reason = 3;
        break;
      }
      pend = false;
      const double rv =
          __longlong_as_double((long long)__ldcg(P.res + ci - 1)) * P.invgamma;
      if (!(rv <= 1.7976931348623157e308)) {
        reason = 2;
        break;
      }
      if (P.tol > 0.0 && rv <= P.tol) {
        reason = 1;
        break;
      }
    }
    // top nodes, stage T .. 1, then 1 .. T: every item waits for the flags
    // of the nodes it reads (children going up, the parent going down),
    // which earlier stages of other teams set; a node and its forward step
    // have the same team
    // (a wait that gave up has set the error word: the launch ends at the
    // next residual check, where every block sees it)
    for (int k = seg[1]; k < seg[2 * TT + 1]; ++k) run_item(k);
    // chains, head to leaf
    for (int k = seg[2 * TT + 1]; k < seg[2 * TT + 2]; ++k) run_item(k);
    if (check) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long b = __shfl_xor_sync(0xffffffffu, rbits, o);
        rbits = b > rbits ? b : rbits;
      }
      if ((tid & 31) == 0 && rbits) atomicMax(P.res + ci, rbits);
      ++ci;
      pend = true;
    }
  }
  if (reason == 0 && pend) {
    if (grid_barrier(P.bar, ++nbar * gridDim.x, P.err, P.wait_ns)) {
      const double rv =
          __longlong_as_double((long long)__ldcg(P.res + ci - 1)) * P.invgamma;
      if (!(rv <= 1.7976931348623157e308))
        reason = 2;
      else if (P.tol > 0.0 && rv <= P.tol)
        reason = 1;
    } else {
      reason = 3;
    }
  }
  // no copy may still be writing into this block's memory when it ends
  cp_wait<0>();
  while (R.cons < R.issued) {
    R.wait(true);
    R.consumed();
  }
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    P.info[0] = P.apg ? it : 1;
    P.info[1] = ci;
    P.info[2] = reason;
    const unsigned long long t = pn_ns();
    memcpy(P.info + 6, &t, sizeof t);
  }
}

namespace {

// ---------------------------------------------------------------------------
// kernels around the persistent launch (one block or warp per node)
// ---------------------------------------------------------------------------
struct PnPrepArgs {
  const double *prob, *demand, *alpha, *alpha0;  // demand n x nd, alpha n x nu
  const int *Gp, *Gi;                            // Gd rows
  const double *Gv;
  const double *Mc, *Sd;                         // n x nu x ne, ne x nd
  double W_alpha;
  int nx, nu, nd, ne, n, NXP, NUP;
};

// c0 = p W_alpha (alpha0 + alpha), gd = Gd d, mc = Mc (Sd d) per node
// (FP64, stored in T); the root row is zero
template <typename T>
__global__ void k_pn_prep(PnPrepArgs a, T *c0, T *mc, T *gd) {
  extern __shared__ double sv[];  // ne
  for (int v = blockIdx.x; v < a.n; v += gridDim.x) {
    const double *d = a.demand + (size_t)v * a.nd;
    __syncthreads();
    for (int e = threadIdx.x; e < a.ne; e += blockDim.x) {
      double s = 0.0;
      for (int k = 0; k < a.nd; ++k) s += a.Sd[(size_t)e * a.nd + k] * d[k];
      sv[e] = s;
    }
    __syncthreads();
    const bool root = v == 0;
    for (int j = threadIdx.x; j < a.NUP; j += blockDim.x) {
      double cv = 0.0, mv = 0.0;
      if (!root && j < a.nu) {
        cv = a.prob[v] * a.W_alpha * (a.alpha0[j] + a.alpha[(size_t)v * a.nu + j]);
        const double *row = a.Mc + ((size_t)v * a.nu + j) * a.ne;
        for (int e = 0; e < a.ne; ++e) mv += row[e] * sv[e];
      }
      c0[(size_t)v * a.NUP + j] = (T)cv;
      mc[(size_t)v * a.NUP + j] = (T)mv;
    }
    for (int i = threadIdx.x; i < a.NXP; i += blockDim.x) {
      double gv = 0.0;
      if (!root && i < a.nx)
        for (int e = a.Gp[i]; e < a.Gp[i + 1]; ++e) gv += a.Gv[e] * d[a.Gi[e]];
      gd[(size_t)v * a.NXP + i] = (T)gv;
    }
  }
}

// y^0 = y^{-1} = src (n x (2nx + nu) doubles, row 0 ignored) or 0, in the
// padded layout; also the T copies of x0 and q
template <typename T>
__global__ void k_pn_init(int n, int nx, int nu, int NXP, int YP, const double *src, T *ya,
                          T *yb, const double *x0, const double *q, T *x0t, T *qt) {
  const int ny = 2 * nx + nu;
  for (int v = blockIdx.x; v < n; v += gridDim.x)
    for (int e = threadIdx.x; e < YP; e += blockDim.x) {
      int k = -1;
      if (e < nx) k = e;
      else if (e >= NXP && e < NXP + nx) k = nx + (e - NXP);
      else if (e >= 2 * NXP && e < 2 * NXP + nu) k = 2 * nx + (e - 2 * NXP);
      const T val = (v > 0 && k >= 0 && src) ? (T)src[(size_t)v * ny + k] : T(0);
      ya[(size_t)v * YP + e] = val;
      yb[(size_t)v * YP + e] = val;
    }
  if (blockIdx.x == 0 && x0t) {
    for (int i = threadIdx.x; i < nx; i += blockDim.x) x0t[i] = (T)x0[i];
    for (int j = threadIdx.x; j < nu; j += blockDim.x) qt[j] = (T)q[j];
  }
}

// outputs in the caller's layout (doubles): u, x (root rows q, x0), y
// (root row 0); any of them may be null
template <typename T>
__global__ void k_pn_gather(int n, int nx, int nu, int NXP, int NUP, int YP, const T *uo,
                            const T *xo, const T *y, const double *q, const double *x0,
                            double *u, double *x, double *yout) {
  const int ny = 2 * nx + nu;
  for (int v = blockIdx.x; v < n; v += gridDim.x) {
    if (u)
      for (int j = threadIdx.x; j < nu; j += blockDim.x)
        u[(size_t)v * nu + j] = v == 0 ? q[j] : (double)uo[(size_t)v * NUP + j];
    if (x)
      for (int i = threadIdx.x; i < nx; i += blockDim.x)
        x[(size_t)v * nx + i] = v == 0 ? x0[i] : (double)xo[(size_t)v * NXP + i];
    if (yout)
      for (int k = threadIdx.x; k < ny; k += blockDim.x) {
        const int e = k < nx ? k : (k < 2 * nx ? NXP + (k - nx) : 2 * NXP + (k - 2 * nx));
        yout[(size_t)v * ny + k] = v == 0 ? 0.0 : (double)y[(size_t)v * YP + e];
      }
  }
}

template <typename T>
__global__ void k_pn_gather_avg(int n, int nx, int nu, int NXP, int NUP, const double *ua,
                                const double *xa, const double *q, const double *x0, double *u,
                                double *x) {
  for (int v = blockIdx.x; v < n; v += gridDim.x) {
    for (int j = threadIdx.x; j < nu; j += blockDim.x)
      u[(size_t)v * nu + j] = v == 0 ? q[j] : ua[(size_t)v * NUP + j];
    for (int i = threadIdx.x; i < nx; i += blockDim.x)
      x[(size_t)v * nx + i] = v == 0 ? x0[i] : xa[(size_t)v * NXP + i];
  }
}

__device__ __forceinline__ double pn_splitmix_unit(unsigned long long i) {
  // SplitMix64 (Steele, Lea, Flood 2014) from seed 0, top 53 bits
  unsigned long long z = (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

// power iteration start: 1 + SplitMix64 over the non-root dual entries in
// node order
template <typename T>
__global__ void k_pn_power_start(int n, int nx, int nu, int NXP, int YP, T *ya) {
  const int ny = 2 * nx + nu;
  for (int v = blockIdx.x + 1; v < n; v += gridDim.x)
    for (int k = threadIdx.x; k < ny; k += blockDim.x) {
      const int e = k < nx ? k : (k < 2 * nx ? NXP + (k - nx) : 2 * NXP + (k - 2 * nx));
      ya[(size_t)v * YP + e] = (T)(1.0 + pn_splitmix_unit((unsigned long long)(v - 1) * ny + k));
    }
}

// per-block partial sums of |H x|^2 = sum 2 |x_nu|^2 + |u_nu|^2
template <typename T>
__global__ void k_pn_norm2(int n, int nx, int nu, int NXP, int NUP, const T *uo, const T *xo,
                           double *partial) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int v = blockIdx.x + 1; v < n; v += gridDim.x) {
    for (int j = threadIdx.x; j < nu; j += blockDim.x) {
      const double a = uo[(size_t)v * NUP + j];
      acc += a * a;
    }
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      const double a = xo[(size_t)v * NXP + i];
      acc += 2.0 * a * a;
    }
  }
  acc = wsum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    partial[blockIdx.x] = t;
  }
}

// v = -H x / |H x| as the next input (the partial sums of every block
// are added up again by each block)
template <typename T>
__global__ void k_pn_power_scale(int n, int nx, int nu, int NXP, int NUP, int YP, const T *uo,
                                 const T *xo, const double *partial, int nparts, T *ya,
                                 double *norm2) {
  __shared__ double inv;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int b = 0; b < nparts; ++b) t += partial[b];
    inv = 1.0 / sqrt(t);
    if (blockIdx.x == 0) *norm2 = t;
  }
  __syncthreads();
  for (int v = blockIdx.x + 1; v < n; v += gridDim.x) {
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
      const T a = (T)(-(double)xo[(size_t)v * NXP + i] * inv);
      ya[(size_t)v * YP + i] = a;
      ya[(size_t)v * YP + NXP + i] = a;
    }
    for (int j = threadIdx.x; j < nu; j += blockDim.x)
      ya[(size_t)v * YP + 2 * NXP + j] = (T)(-(double)uo[(size_t)v * NUP + j] * inv);
  }
}

struct PnCostArgs {
  const int *anc;
  const double *prob, *alpha, *alpha0, *xmin, *xmax, *xs, *umin, *umax;
  const int *Wp, *Wi;
  const double *Wv;
  const double *u, *x;  // caller layout, root rows q, x0
  double W_alpha, Wx, Ws;
  int n, nx, nu;
};

// per-block partials: smooth cost, soft cost, max input-box violation (one
// warp per node, FP64)
__global__ void k_pn_cost(PnCostArgs a, double *partial) {
  __shared__ double sh[3][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double sm = 0.0, so = 0.0, vb = 0.0;
  for (int v = 1 + blockIdx.x * nw + warp; v < a.n; v += gridDim.x * nw) {
    const double *u = a.u + (size_t)v * a.nu, *ua = a.u + (size_t)a.anc[v] * a.nu;
    const double *x = a.x + (size_t)v * a.nx;
    const double p = a.prob[v];
    double lin = 0.0, quad = 0.0, dx = 0.0, ds = 0.0;
    for (int j = lane; j < a.nu; j += 32) {
      lin += p * a.W_alpha * (a.alpha0[j] + a.alpha[(size_t)v * a.nu + j]) * u[j];
      double wd = 0.0;
      for (int e = a.Wp[j]; e < a.Wp[j + 1]; ++e) wd += a.Wv[e] * (u[a.Wi[e]] - ua[a.Wi[e]]);
      quad += (u[j] - ua[j]) * wd;
      vb = fmax(vb, fmax(a.umin[j] - u[j], u[j] - a.umax[j]));
    }
    for (int i = lane; i < a.nx; i += 32) {
      const double e1 = x[i] - fmin(fmax(x[i], a.xmin[i]), a.xmax[i]);
      const double e2 = fmin(x[i] - a.xs[i], 0.0);
      dx += e1 * e1;
      ds += e2 * e2;
    }
    lin = wsum(lin);
    quad = wsum(quad);
    dx = wsum(dx);
    ds = wsum(ds);
    if (lane == 0) {
      sm += lin + p * quad;
      so += a.Wx * sqrt(dx) + a.Ws * sqrt(ds);
    }
  }
  vb = fmax(vb, 0.0);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) vb = fmax(vb, __shfl_xor_sync(0xffffffffu, vb, o));
  if (lane == 0) {
    sh[0][warp] = sm;
    sh[1][warp] = so;
    sh[2][warp] = vb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int w = 0; w < nw; ++w) {
      s0 += sh[0][w];
      s1 += sh[1][w];
      s2 = fmax(s2, sh[2][w]);
    }
    partial[3 * blockIdx.x] = s0;
    partial[3 * blockIdx.x + 1] = s1;
    partial[3 * blockIdx.x + 2] = s2;
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------
struct PnFactor {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool fp32 = false;
  int nx = 0, nu = 0, nd = 0, ne = 0, n = 0, N = 0, NXP = 0, NUP = 0, YP = 0, ldm = 0;
  long long mstride = 0;
  double W_alpha = 0.0, Wx = 0.0, Ws = 0.0;
  int theta_rule = 0, check_every = 10;
  double gamma = 0.0, L = 0.0;
  long long wait_ns = 0;
  std::vector<void *> allocs;
  long long bytes = 0;
  // tree and operators
  int *anc = nullptr, *cbeg = nullptr, *cend = nullptr;
  double *prob = nullptr;
  int *Ap = nullptr, *Ai = nullptr, *Atp = nullptr, *Ati = nullptr, *Bp = nullptr, *Bi = nullptr;
  int *Btp = nullptr, *Bti = nullptr, *Wp = nullptr, *Wi = nullptr, *Gp = nullptr, *Gi = nullptr;
  void *Av = nullptr, *Atv = nullptr, *Bv = nullptr, *Btv = nullptr, *Wv = nullptr;
  double *Wv64 = nullptr, *Gv = nullptr;
  void *xmin = nullptr, *xmax = nullptr, *xs = nullptr, *umin = nullptr, *umax = nullptr;
  double *bnd64 = nullptr;  // xmin, xmax, xs (nx each), umin, umax (nu each)
  double *alpha0 = nullptr;
  void *Phi = nullptr, *K = nullptr;
  double *Mc = nullptr, *Sd = nullptr;
  // per solve
  void *c0 = nullptr, *mc = nullptr, *gd = nullptr, *x0t = nullptr, *qt = nullptr;
  double *x0 = nullptr, *q = nullptr, *alpha = nullptr;  // copies of the last data
  void *ya = nullptr, *yb = nullptr, *m = nullptr, *lam = nullptr, *r = nullptr;
  void *uo = nullptr, *xo = nullptr;
  double *uavg = nullptr, *xavg = nullptr;
  double *beta = nullptr;
  int beta_cap = 0;
  unsigned long long *res = nullptr;
  int res_cap = 0;
  unsigned *bar = nullptr, *nflag = nullptr;
  int *err = nullptr, *info = nullptr;
  double *partial = nullptr, *norm2 = nullptr;
  bool have_data = false;
  // schedule and launch layout
  int *items = nullptr, *seg = nullptr;
  int n_seg = 0, t_top = 0, n_chains = 0, n_top = 0;
  int grid = 0, block = 0, team_threads = 128, teams = 4;
  int qw = 0, nch = 0, slots = 0, slot_elems = 0, vec_elems = 0, b1 = 0, vb = 0;
  size_t smem = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // RN_PREC_MIXED: this FP32 handle iterates on the delta d = y - yb; the
  // FP64 twin evaluates x*(yb) at every refresh and the final x*(w)
  bool mixed = false;
  int refresh_every = 20;
  PnFactor *twin = nullptr;
  double *ybase = nullptr;                              // yb, n x YP
  float *ybh = nullptr, *uref = nullptr, *xref = nullptr, *swy = nullptr;

  ~PnFactor() {
    delete twin;
    cudaSetDevice(device);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    for (void *p : allocs) cudaFree(p);
  }
};

namespace {

constexpr int kPnParts = 304;  // blocks of the reductions

#define PN_CUDA(call)                                                       \
  do {                                                                      \
    cudaError_t e_ = (call);                                                \
    if (e_ != cudaSuccess) {                                                \
      set_error("per-node path: %s failed: %s", #call, cudaGetErrorString(e_)); \
      return e_ == cudaErrorMemoryAllocation ? RN_ERR_NOMEM : RN_ERR_CUDA;  \
    }                                                                       \
  } while (0)

template <typename U>
int pn_alloc(PnFactor *f, U **p, size_t count) {
  void *q = nullptr;
  PN_CUDA(cudaMalloc(&q, std::max<size_t>(1, count) * sizeof(U)));
  f->allocs.push_back(q);
  f->bytes += (long long)(std::max<size_t>(1, count) * sizeof(U));
  *p = static_cast<U *>(q);
  return RN_OK;
}

template <typename U>
int pn_upload(PnFactor *f, U **p, const std::vector<U> &h) {
  int rc = pn_alloc(f, p, h.size());
  if (rc) return rc;
  if (!h.empty())
    PN_CUDA(cudaMemcpyAsync(*p, h.data(), h.size() * sizeof(U), cudaMemcpyHostToDevice, f->stream));
  return RN_OK;
}

// a vector of T (float or double) from doubles, uploaded
template <typename T>
int pn_upload_t(PnFactor *f, void **p, const double *src, size_t count) {
  std::vector<T> h(src, src + count);
  T *d = nullptr;
  int rc = pn_upload(f, &d, h);
  *p = d;
  return rc;
}

int pn_upload_csr(PnFactor *f, const Csr &c, int **p, int **i, void **v, bool fp32,
                  double **v64 = nullptr) {
  int rc;
  if ((rc = pn_upload(f, p, c.ptr)) || (rc = pn_upload(f, i, c.idx))) return rc;
  rc = fp32 ? pn_upload_t<float>(f, v, c.val.data(), c.val.size())
            : pn_upload_t<double>(f, v, c.val.data(), c.val.size());
  if (rc) return rc;
  if (v64) rc = pn_upload(f, v64, c.val);
  return rc;
}

template <typename T>
PnParams<T> pn_params(const PnFactor *f) {
  PnParams<T> P{};
  P.nx = f->nx;
  P.nu = f->nu;
  P.n = f->n;
  P.NXP = f->NXP;
  P.NUP = f->NUP;
  P.YP = f->YP;
  P.ldm = f->ldm;
  P.mstride = f->mstride;
  P.anc = f->anc;
  P.cbeg = f->cbeg;
  P.cend = f->cend;
  P.prob = f->prob;
  P.Ap = f->Ap;
  P.Ai = f->Ai;
  P.Atp = f->Atp;
  P.Ati = f->Ati;
  P.Bp = f->Bp;
  P.Bi = f->Bi;
  P.Btp = f->Btp;
  P.Bti = f->Bti;
  P.Wp = f->Wp;
  P.Wi = f->Wi;
  P.Av = static_cast<const T *>(f->Av);
  P.Atv = static_cast<const T *>(f->Atv);
  P.Bv = static_cast<const T *>(f->Bv);
  P.Btv = static_cast<const T *>(f->Btv);
  P.Wv = static_cast<const T *>(f->Wv);
  P.xmin = static_cast<const T *>(f->xmin);
  P.xmax = static_cast<const T *>(f->xmax);
  P.xs = static_cast<const T *>(f->xs);
  P.umin = static_cast<const T *>(f->umin);
  P.umax = static_cast<const T *>(f->umax);
  P.Wx = (T)f->Wx;
  P.Ws = (T)f->Ws;
  P.Phi = static_cast<const T *>(f->Phi);
  P.K = static_cast<const T *>(f->K);
  P.ya = static_cast<T *>(f->ya);
  P.yb = static_cast<T *>(f->yb);
  P.m = static_cast<T *>(f->m);
  P.lam = static_cast<T *>(f->lam);
  P.r = static_cast<T *>(f->r);
  P.uo = static_cast<T *>(f->uo);
  P.xo = static_cast<T *>(f->xo);
  P.bar = f->bar;
  P.nflag = f->nflag;
  P.err = f->err;
  P.info = f->info;
  P.wait_ns = f->wait_ns;
  P.gamma = f->gamma;
  P.invgamma = f->gamma > 0.0 ? 1.0 / f->gamma : 0.0;
  P.items = f->items;
  P.seg = f->seg;
  P.n_seg = f->n_seg;
  P.t_top = f->t_top;
  P.team_threads = f->team_threads;
  P.teams = f->teams;
  P.qw = f->qw;
  P.nch = f->nch;
  P.slots = f->slots;
  P.slot_elems = f->slot_elems;
  P.vec_elems = f->vec_elems;
  P.b1 = f->b1;
  P.vb = f->vb;
  return P;
}

// the instantiation for the handle's precision and rows per thread
const void *pn_kernel(bool fp32, int mr) {
  if (fp32)
    return mr <= 1 ? (const void *)k_pn_solve<float, 1>
         : mr <= 2 ? (const void *)k_pn_solve<float, 2>
         : mr <= 4 ? (const void *)k_pn_solve<float, 4>
                   : (const void *)k_pn_solve<float, 8>;
  return mr <= 1 ? (const void *)k_pn_solve<double, 1>
       : mr <= 2 ? (const void *)k_pn_solve<double, 2>
       : mr <= 4 ? (const void *)k_pn_solve<double, 4>
                 : (const void *)k_pn_solve<double, 8>;
}

template <typename T>
int pn_launch(PnFactor *f, PnParams<T> &P) {
  PN_CUDA(cudaMemsetAsync(f->bar, 0, sizeof(unsigned), f->stream));
  PN_CUDA(cudaMemsetAsync(f->nflag, 0, 2 * (size_t)f->n * sizeof(unsigned), f->stream));
  void *args[] = {&P};
  PN_CUDA(cudaLaunchCooperativeKernel(pn_kernel(f->fp32, (f->nu + 127) / 128), f->grid, f->block,
                                      args, f->smem, f->stream));
  return RN_OK;
}

int pn_check_err(PnFactor *f) {
  int e = 0;
  PN_CUDA(cudaMemcpyAsync(&e, f->err, sizeof(int), cudaMemcpyDeviceToHost, f->stream));
  PN_CUDA(cudaStreamSynchronize(f->stream));
  if (e) {
    PN_CUDA(cudaMemsetAsync(f->err, 0, sizeof(int), f->stream));
    set_error("per-node path: a device-side wait gave up after %.3g s (%s)", f->wait_ns * 1e-9,
              e == 4 ? "grid barrier" : "matrix copy");
    return RN_ERR_TIMEOUT;
  }
  return RN_OK;
}

// one evaluation of x*(w), w in ya; `linear` drops every data term
template <typename T>
int pn_eval(PnFactor *f, bool linear) {
  PnParams<T> P = pn_params<T>(f);
  P.apg = 0;
  P.iters = 1;
  P.it0 = 0;
  P.iters_total = 1;
  P.check_every = 1;
  if (!linear) {
    P.c0 = static_cast<const T *>(f->c0);
    P.mc = static_cast<const T *>(f->mc);
    P.gd = static_cast<const T *>(f->gd);
    P.x0 = static_cast<const T *>(f->x0t);
    P.q = static_cast<const T *>(f->qt);
  }
  return pn_launch<T>(f, P);
}

template <typename T>
int pn_power(PnFactor *f, int iters, double *L) {
  const int nb = std::max(1, std::min(f->n - 1, 4096));
  k_pn_power_start<T><<<nb, 128, 0, f->stream>>>(f->n, f->nx, f->nu, f->NXP, f->YP,
                                                static_cast<T *>(f->ya));
  PN_CUDA(cudaGetLastError());
  for (int k = 0; k < iters; ++k) {
    int rc = pn_eval<T>(f, true);
    if (rc) return rc;
    k_pn_norm2<T><<<kPnParts, 256, 0, f->stream>>>(f->n, f->nx, f->nu, f->NXP, f->NUP,
                                                   static_cast<const T *>(f->uo),
                                                   static_cast<const T *>(f->xo), f->partial);
    k_pn_power_scale<T><<<nb, 128, 0, f->stream>>>(
        f->n, f->nx, f->nu, f->NXP, f->NUP, f->YP, static_cast<const T *>(f->uo),
        static_cast<const T *>(f->xo), f->partial, kPnParts, static_cast<T *>(f->ya), f->norm2);
    PN_CUDA(cudaGetLastError());
  }
  double n2 = 0.0;
  PN_CUDA(cudaMemcpyAsync(&n2, f->norm2, sizeof(double), cudaMemcpyDeviceToHost, f->stream));
  int rc = pn_check_err(f);
  if (rc) return rc;
  *L = std::sqrt(n2);
  return RN_OK;
}

}  // namespace

int pn_validate(const rn_network *net, const rn_tree *tree, const rn_cost *cost) {
  if (!net || !tree || !cost) {
    set_error("network, tree or cost is NULL");
    return RN_ERR_INVAL;
  }
  if (std::max(net->nx, net->nu) > kPnMaxDim) {
    set_error("per-node path: nx, nu <= %d", kPnMaxDim);
    return RN_ERR_UNSUPPORTED;
  }
  Plan p;
  return build_plan(tree, p);  // the tree's structure (see rn_tree)
}

namespace {

// Work lists of the teams (see PnParams): chains by longest-first onto the
// least loaded team (teams taken in an order that visits every block before
// a second team of any block), top nodes of a stage one per team in the
// same order.
int pn_schedule(PnFactor *f, const rn_tree *tree, int n_teams) {
  const int n = tree->n_nodes, N = tree->N;
  std::vector<int> stage(n), cbeg(n, 0), cend(n, 0), nleaf(n, 0);
  for (int t = 0; t <= N; ++t)
    for (int v = tree->stage_ptr[t]; v < tree->stage_ptr[t + 1]; ++v) stage[v] = t;
  for (int v = 1; v < n; ++v) {
    const int a = tree->anc[v];
    if (cend[a] == 0) cbeg[a] = v;
    cend[a] = v + 1;
  }
  for (int v = n - 1; v >= 1; --v) {
    if (cend[v] == 0) nleaf[v] = 1;
    nleaf[tree->anc[v]] += nleaf[v];
  }
  std::vector<char> top(n, 0);
  int t_top = 0;
  for (int v = 1; v < n; ++v)
    if (nleaf[v] >= 2) {
      top[v] = 1;
      t_top = std::max(t_top, stage[v]);
    }
  // chains: head (parent is the root or a top node) down to the leaf
  std::vector<std::vector<int>> chains;
  for (int v = 1; v < n; ++v)
    if (!top[v] && (tree->anc[v] == 0 || top[tree->anc[v]])) {
      std::vector<int> c{v};
      int u = v;
      while (cend[u] > 0) {
        u = cbeg[u];
        c.push_back(u);
      }
      chains.push_back(std::move(c));
    }
  const int grid = std::max(1, n_teams / f->teams);
  std::vector<int> ord(n_teams);
  for (int k = 0; k < n_teams; ++k) ord[k] = (k % grid) * f->teams + (k / grid);
  std::vector<int> corder(chains.size());
  std::iota(corder.begin(), corder.end(), 0);
  std::stable_sort(corder.begin(), corder.end(),
                   [&](int a, int b) { return chains[a].size() > chains[b].size(); });
  std::vector<long long> load(n_teams, 0);
  std::vector<std::vector<int>> team_chains(n_teams);
  {
    // least loaded team, ties to the earliest in the spread order
    std::vector<std::pair<long long, int>> heap;
    for (int k = 0; k < n_teams; ++k) heap.push_back({0, k});
    auto cmp = [](const std::pair<long long, int> &a, const std::pair<long long, int> &b) {
      return a.first != b.first ? a.first > b.first : a.second > b.second;
    };
    std::make_heap(heap.begin(), heap.end(), cmp);
    for (int c : corder) {
      std::pop_heap(heap.begin(), heap.end(), cmp);
      auto h = heap.back();
      heap.pop_back();
      team_chains[ord[h.second]].push_back(c);
      h.first += (long long)chains[c].size();
      heap.push_back(h);
      std::push_heap(heap.begin(), heap.end(), cmp);
    }
  }
  std::vector<std::vector<std::vector<int>>> team_top(n_teams,
                                                      std::vector<std::vector<int>>(t_top + 1));
  for (int t = 1; t <= t_top; ++t) {
    int j = 0;
    for (int v = tree->stage_ptr[t]; v < tree->stage_ptr[t + 1]; ++v)
      if (top[v]) team_top[ord[j++ % n_teams]][t].push_back(v);
  }
  const int n_seg = 2 * t_top + 2;
  std::vector<int> items, seg;
  for (int tm = 0; tm < n_teams; ++tm) {
    seg.push_back((int)items.size());
    for (int c : team_chains[tm]) {  // chain backward: leaf to head
      const auto &ch = chains[c];
      for (int q = (int)ch.size() - 1; q >= 0; --q) {
        int it = ch[q];
        if (q == (int)ch.size() - 1) it |= kPnFirst;
        if (q == 0) it |= kPnLast;
        items.push_back(it);
      }
    }
    for (int t = t_top; t >= 1; --t) {
      seg.push_back((int)items.size());
      for (int v : team_top[tm][t]) items.push_back(v | kPnTop);
    }
    for (int t = 1; t <= t_top; ++t) {
      seg.push_back((int)items.size());
      for (int v : team_top[tm][t]) items.push_back(v | kPnTop | kPnK);
    }
    seg.push_back((int)items.size());
    for (int c : team_chains[tm]) {  // chain forward: head to leaf
      const auto &ch = chains[c];
      for (int q = 0; q < (int)ch.size(); ++q) {
        int it = ch[q] | kPnK;
        if (q == 0) it |= kPnFirst;
        if (q == (int)ch.size() - 1) it |= kPnLast;
        items.push_back(it);
      }
    }
  }
  seg.push_back((int)items.size());
  // seg holds n_teams * (n_seg + 1) entries: each team's n_seg + 1 offsets
  // (its last offset is the next team's first)
  std::vector<int> segs;
  for (int tm = 0; tm < n_teams; ++tm)
    for (int s = 0; s <= n_seg; ++s) segs.push_back(seg[(size_t)tm * n_seg + s]);
  int rc;
  if ((rc = pn_upload(f, &f->items, items)) || (rc = pn_upload(f, &f->seg, segs))) return rc;
  if ((rc = pn_upload(f, &f->cbeg, cbeg)) || (rc = pn_upload(f, &f->cend, cend))) return rc;
  f->n_seg = n_seg;
  f->t_top = t_top;
  f->n_chains = (int)chains.size();
  int ntop = 0;
  for (int v = 1; v < n; ++v) ntop += top[v];
  f->n_top = ntop;
  return RN_OK;
}

// widest work of one phase: chains, or the top nodes of one stage
int pn_width(const rn_tree *tree) {
  const int n = tree->n_nodes;
  std::vector<int> nleaf(n, 0), nch(n, 0);
  for (int v = 1; v < n; ++v) ++nch[tree->anc[v]];
  for (int v = n - 1; v >= 1; --v) {
    if (nch[v] == 0) nleaf[v] = 1;
    nleaf[tree->anc[v]] += nleaf[v];
  }
  int w = 1;
  for (int t = 1; t <= tree->N; ++t) {
    int k = 0;
    for (int v = tree->stage_ptr[t]; v < tree->stage_ptr[t + 1]; ++v) k += nleaf[v] >= 2;
    w = std::max(w, k);
  }
  return std::max(w, nleaf[0]);
}

// the matrices in the layout of the ring: column blocks of qw 16-byte units
// (the last block narrower), each block nu rows, row-major; padding zero
template <typename T>
struct PnMatSink {
  T *Phi, *K;
  double *Mc;
  int nu, ne, ldm, qw;
  static void put(void *ctx, int v, const double *P, const double *Kv, const double *M) {
    PnMatSink *s = static_cast<PnMatSink *>(ctx);
    constexpr int VW = 16 / sizeof(T);
    const size_t ms = (size_t)s->nu * s->ldm;
    const int cw = s->qw * VW;  // columns of a full block
    for (int j = 0; j < s->nu; ++j) {
      const int b = j / cw, wb = std::min(cw, s->ldm - b * cw), jj = j - b * cw;
      const size_t col = (size_t)s->nu * b * cw + jj;
      for (int i = 0; i < s->nu; ++i) {
        const size_t o = (size_t)v * ms + col + (size_t)i * wb;
        s->Phi[o] = (T)P[(size_t)i * s->nu + j];
        s->K[o] = (T)Kv[(size_t)i * s->nu + j];
      }
    }
    if (s->ne > 0)
      std::copy(M, M + (size_t)s->nu * s->ne, s->Mc + (size_t)v * s->nu * s->ne);
  }
};

template <typename T>
int pn_matrices(PnFactor *f, const rn_network *net, const rn_tree *tree, const rn_cost *cost) {
  const size_t ms = (size_t)f->nu * f->ldm;
  std::vector<T> hP((size_t)f->n * ms, T(0)), hK((size_t)f->n * ms, T(0));
  std::vector<double> hM((size_t)f->n * f->nu * std::max(1, f->ne), 0.0), Sd;
  PnMatSink<T> sink{hP.data(), hK.data(), hM.data(), f->nu, f->ne, f->ldm, f->qw};
  const int threads = (int)std::max(1u, std::thread::hardware_concurrency());
  int rc = pn_factor_host(net, tree, cost, threads, &PnMatSink<T>::put, &sink, &Sd);
  if (rc) return rc;
  T *dP = nullptr, *dK = nullptr;
  if ((rc = pn_upload(f, &dP, hP)) || (rc = pn_upload(f, &dK, hK)) ||
      (rc = pn_upload(f, &f->Mc, hM)) || (rc = pn_upload(f, &f->Sd, Sd)))
    return rc;
  f->Phi = dP;
  f->K = dK;
  // the host copies go when this returns: the uploads must be done
  PN_CUDA(cudaStreamSynchronize(f->stream));
  return RN_OK;
}

// launch layout: teams of team_threads threads, a ring of matrix chunks per
// team in the shared memory left after its vectors
int pn_layout(PnFactor *f, int max_ctas, int width) {
  const int sz = f->fp32 ? 4 : 8;
  int sms = 0, optin = 0;
  PN_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, f->device));
  PN_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, f->device));
  const size_t avail = (size_t)optin - 1024;  // static shared memory of the kernel
  const int vup = (std::max(f->NUP, f->ldm) + 3) & ~3;
  f->b1 = std::max(f->NUP, f->NXP);
  // the delta form's forward rows: ybh | xref | uref after y and y_prev
  if (f->mixed) f->b1 = std::max(f->b1, f->YP + f->NXP + f->NUP);
  f->vb = 2 * f->YP + f->b1 + f->NUP;
  f->vec_elems = 2 * f->NXP + 4 * vup + 64 + 3 * f->vb + 2 * vup;
  const size_t vec_bytes = ((size_t)f->vec_elems * sz + 127) & ~(size_t)127;
  const size_t colb = (size_t)f->nu * 16;  // bytes of one 16-byte column unit of a matrix
  const int nq = f->ldm / (16 / sz);
  for (int teams = 4; teams >= 1; teams /= 2) {
    const size_t mb = ((size_t)teams * 8 * 8 + 127) & ~(size_t)127;
    if (avail < mb + teams * vec_bytes) continue;
    const size_t per = ((avail - mb) / teams - vec_bytes) & ~(size_t)127;
    const int max_units = (int)(per / colb);  // column units the ring holds
    if (max_units < 2) continue;
    // blocks of an odd number of units, as wide as two slots allow (fewer,
    // larger copies: measured 275 us per iteration at barcelona512 against
    // 310 with three slots and 319 with four)
    int qw = std::max(1, std::min(nq, max_units / 2));
    if (qw % 2 == 0) qw = std::max(1, qw - 1);
    f->qw = qw;
    f->nch = (nq + qw - 1) / qw;
    f->slots = std::min(8, max_units / qw);
    f->slot_elems = (int)((size_t)f->nu * qw * (16 / sz));
    f->teams = teams;
    f->block = teams * f->team_threads;
    f->smem = mb + teams * ((((size_t)f->slots * f->slot_elems * sz + 127) & ~(size_t)127) +
                            vec_bytes);
    const void *k = pn_kernel(f->fp32, (f->nu + 127) / 128);
    PN_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)f->smem));
    int occ = 0;
    PN_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, f->block, f->smem));
    if (occ < 1) continue;
    int grid = std::min(sms * occ, (width + teams - 1) / teams);
    if (max_ctas > 0) grid = std::min(grid, max_ctas);
    f->grid = std::max(1, grid);
    return RN_OK;
  }
  set_error("per-node path: nu = %d does not fit the shared memory of a block", f->nu);
  return RN_ERR_UNSUPPORTED;
}

}  // namespace

void pn_destroy(PnFactor *f) { delete f; }

int pn_create(const rn_network *net, const rn_tree *tree, const rn_cost *cost,
              const PnOptions &o, PnFactor **out) {
  *out = nullptr;
  int rc = pn_validate(net, tree, cost);
  if (rc) return rc;
  std::unique_ptr<PnFactor> f(new (std::nothrow) PnFactor());
  if (!f) {
    set_error("per-node path: host allocation failed");
    return RN_ERR_NOMEM;
  }
  PnFactor *F = f.get();
  F->device = o.device;
  F->stream = o.stream;
  F->fp32 = o.fp32 || o.mixed;
  F->mixed = o.mixed;
  F->refresh_every = std::max(1, o.refresh_every);
  PnOptions o2 = o;  // the FP64 twin of a mixed handle: its step size serves both
  if (o.mixed) {
    o2.mixed = false;
    o2.fp32 = false;
    PnFactor *tw = nullptr;
    if ((rc = pn_create(net, tree, cost, o2, &tw))) return rc;
    F->twin = tw;
  }
  F->nx = net->nx;
  F->nu = net->nu;
  F->nd = net->nd;
  F->ne = net->ne;
  F->n = tree->n_nodes;
  F->N = tree->N;
  F->NXP = (F->nx + 3) & ~3;
  F->NUP = (F->nu + 3) & ~3;
  F->YP = 2 * F->NXP + F->NUP;
  // columns padded to 16 bytes
  {
    const int vw = F->fp32 ? 4 : 2;
    F->ldm = (F->nu + vw - 1) / vw * vw;
  }
  F->mstride = (long long)F->nu * F->ldm;
  F->W_alpha = cost->W_alpha;
  F->Wx = cost->Wx;
  F->Ws = cost->Ws;
  F->theta_rule = o.theta_rule;
  F->check_every = o.check_every;
  F->wait_ns = o.wait_ns;
  PN_CUDA(cudaSetDevice(F->device));
  PN_CUDA(cudaEventCreate(&F->ev0));
  PN_CUDA(cudaEventCreate(&F->ev1));
  if ((rc = pn_layout(F, o.max_ctas, pn_width(tree)))) return rc;
  if ((rc = pn_schedule(F, tree, F->grid * F->teams))) return rc;
  const int nx = F->nx, nu = F->nu, n = F->n;
  // tree, operators, bounds
  {
    std::vector<int> anc(tree->anc, tree->anc + n);
    anc[0] = 0;
    std::vector<double> prob(tree->prob, tree->prob + n);
    if ((rc = pn_upload(F, &F->anc, anc)) || (rc = pn_upload(F, &F->prob, prob))) return rc;
  }
  const Csr Ar = dense_to_csr(net->A, nx, nx), At = dense_to_csc(net->A, nx, nx);
  const Csr Br = dense_to_csr(net->B, nx, nu), Bt = dense_to_csc(net->B, nx, nu);
  const Csr Wr = dense_to_csr(cost->Wu, nu, nu), Gr = dense_to_csr(net->Gd, nx, F->nd);
  if ((rc = pn_upload_csr(F, Ar, &F->Ap, &F->Ai, &F->Av, F->fp32)) ||
      (rc = pn_upload_csr(F, At, &F->Atp, &F->Ati, &F->Atv, F->fp32)) ||
      (rc = pn_upload_csr(F, Br, &F->Bp, &F->Bi, &F->Bv, F->fp32)) ||
      (rc = pn_upload_csr(F, Bt, &F->Btp, &F->Bti, &F->Btv, F->fp32)) ||
      (rc = pn_upload_csr(F, Wr, &F->Wp, &F->Wi, &F->Wv, F->fp32, &F->Wv64)) ||
      (rc = pn_upload(F, &F->Gp, Gr.ptr)) || (rc = pn_upload(F, &F->Gi, Gr.idx)) ||
      (rc = pn_upload(F, &F->Gv, Gr.val)))
    return rc;
  {
    std::vector<double> b;
    b.insert(b.end(), net->xmin, net->xmin + nx);
    b.insert(b.end(), net->xmax, net->xmax + nx);
    b.insert(b.end(), net->xs, net->xs + nx);
    b.insert(b.end(), net->umin, net->umin + nu);
    b.insert(b.end(), net->umax, net->umax + nu);
    if ((rc = pn_upload(F, &F->bnd64, b))) return rc;
    auto up = [&](void **p, const double *s, int k) {
      return F->fp32 ? pn_upload_t<float>(F, p, s, k) : pn_upload_t<double>(F, p, s, k);
    };
    if ((rc = up(&F->xmin, net->xmin, nx)) || (rc = up(&F->xmax, net->xmax, nx)) ||
        (rc = up(&F->xs, net->xs, nx)) || (rc = up(&F->umin, net->umin, nu)) ||
        (rc = up(&F->umax, net->umax, nu)))
      return rc;
    std::vector<double> a0(cost->alpha0, cost->alpha0 + nu);
    if ((rc = pn_upload(F, &F->alpha0, a0))) return rc;
  }
  // the per-node matrices (general recursion, FP64 on the host)
  rc = F->fp32 ? pn_matrices<float>(F, net, tree, cost) : pn_matrices<double>(F, net, tree, cost);
  if (rc) return rc;
  // state and per-solve buffers
  const int sz = F->fp32 ? 4 : 8;
  auto talloc = [&](void **p, size_t count) -> int {
    if (F->fp32) {
      float *q = nullptr;
      int r2 = pn_alloc(F, &q, count);
      *p = q;
      return r2;
    }
    double *q = nullptr;
    int r2 = pn_alloc(F, &q, count);
    *p = q;
    return r2;
  };
  (void)sz;
  if ((rc = talloc(&F->c0, (size_t)n * F->NUP)) || (rc = talloc(&F->mc, (size_t)n * F->NUP)) ||
      (rc = talloc(&F->gd, (size_t)n * F->NXP)) || (rc = talloc(&F->x0t, F->NXP)) ||
      (rc = talloc(&F->qt, F->NUP)) || (rc = talloc(&F->ya, (size_t)n * F->YP)) ||
      (rc = talloc(&F->yb, (size_t)n * F->YP)) || (rc = talloc(&F->m, (size_t)n * F->NUP)) ||
      (rc = talloc(&F->lam, (size_t)n * F->NXP)) || (rc = talloc(&F->r, (size_t)n * F->NUP)) ||
      (rc = talloc(&F->uo, (size_t)n * F->NUP)) || (rc = talloc(&F->xo, (size_t)n * F->NXP)) ||
      (rc = pn_alloc(F, &F->x0, nx)) || (rc = pn_alloc(F, &F->q, nu)) ||
      (rc = pn_alloc(F, &F->alpha, (size_t)n * nu)) || (rc = pn_alloc(F, &F->bar, 1)) || (rc = pn_alloc(F, &F->nflag, 2 * (size_t)n)) ||
      (rc = pn_alloc(F, &F->err, 1)) || (rc = pn_alloc(F, &F->info, 8)) ||
      (rc = pn_alloc(F, &F->partial, 3 * kPnParts)) || (rc = pn_alloc(F, &F->norm2, 1)))
    return rc;
  if (F->mixed &&
      ((rc = pn_alloc(F, &F->ybase, (size_t)n * F->YP)) || (rc = pn_alloc(F, &F->ybh, (size_t)n * F->YP)) ||
       (rc = pn_alloc(F, &F->uref, (size_t)n * F->NUP)) ||
       (rc = pn_alloc(F, &F->xref, (size_t)n * F->NXP)) ||
       (rc = pn_alloc(F, &F->swy, (size_t)n * F->YP))))
    return rc;
  PN_CUDA(cudaMemsetAsync(F->err, 0, sizeof(int), F->stream));
  PN_CUDA(cudaMemsetAsync(F->uo, 0, (size_t)n * F->NUP * (F->fp32 ? 4 : 8), F->stream));
  PN_CUDA(cudaMemsetAsync(F->xo, 0, (size_t)n * F->NXP * (F->fp32 ? 4 : 8), F->stream));
  // step size: gamma = 1 / (1.01 L), L by power iteration on the dual Hessian
  if (F->twin) {
    F->gamma = F->twin->gamma;
    F->L = F->twin->L;
  } else if (o.gamma > 0.0) {
    F->gamma = o.gamma;
  } else {
    rc = F->fp32 ? pn_power<float>(F, o.power_iters, &F->L)
                 : pn_power<double>(F, o.power_iters, &F->L);
    if (rc) return rc;
    if (!(F->L > 0.0) || !std::isfinite(F->L)) {
      set_error("per-node path: power iteration gave L = %g", F->L);
      return RN_ERR_INVAL;
    }
    F->gamma = 1.0 / (1.01 * F->L);
  }
  PN_CUDA(cudaStreamSynchronize(F->stream));
  *out = f.release();
  return RN_OK;
}

namespace {

int pn_beta(PnFactor *f, int iters) {
  if (iters + 1 <= f->beta_cap) return RN_OK;
  const int cap = std::max(iters + 1, 2 * f->beta_cap);
  // beta_nu = theta_nu (1 / theta_{nu-1} - 1) from theta_0 = theta_{-1} = 1
  // (paper §4.3: the equality rule, or theta_nu = 2 / (nu + 2))
  std::vector<double> b(2 * (size_t)cap);
  double th = 1.0, prev = 1.0;
  for (int k = 0; k < cap; ++k) {
    b[k] = th * (1.0 / prev - 1.0);
    b[cap + k] = th;
    const double t2 = th * th;
    const double nt = f->theta_rule == RN_THETA_SIMPLE ? 2.0 / (k + 3)
                                                       : 0.5 * (std::sqrt(t2 * t2 + 4.0 * t2) - t2);
    prev = th;
    th = nt;
  }
  double *d = nullptr;
  int rc = pn_upload(f, &d, b);
  if (rc) return rc;
  f->beta = d;
  f->beta_cap = cap;
  return RN_OK;
}

int pn_res(PnFactor *f, int checks) {
  if (checks <= f->res_cap) return RN_OK;
  const int cap = std::max(checks, 2 * f->res_cap);
  int rc = pn_alloc(f, &f->res, cap);
  if (rc) return rc;
  f->res_cap = cap;
  return RN_OK;
}

// per-solve constants from device inputs
template <typename T>
int pn_prepare_t(PnFactor *f, const double *x0, const double *q, const double *demand,
                 const double *alpha) {
  PN_CUDA(cudaMemcpyAsync(f->x0, x0, f->nx * sizeof(double), cudaMemcpyDeviceToDevice, f->stream));
  PN_CUDA(cudaMemcpyAsync(f->q, q, f->nu * sizeof(double), cudaMemcpyDeviceToDevice, f->stream));
  PN_CUDA(cudaMemcpyAsync(f->alpha, alpha, (size_t)f->n * f->nu * sizeof(double),
                          cudaMemcpyDeviceToDevice, f->stream));
  PnPrepArgs a{f->prob, demand, f->alpha, f->alpha0, f->Gp, f->Gi, f->Gv, f->Mc, f->Sd,
               f->W_alpha, f->nx, f->nu, f->nd, f->ne, f->n, f->NXP, f->NUP};
  const int nb = std::max(1, std::min(f->n, 4096));
  k_pn_prep<T><<<nb, 128, std::max(1, f->ne) * sizeof(double), f->stream>>>(
      a, static_cast<T *>(f->c0), static_cast<T *>(f->mc), static_cast<T *>(f->gd));
  PN_CUDA(cudaGetLastError());
  f->have_data = true;
  return RN_OK;
}

int pn_prepare(PnFactor *f, const double *x0, const double *q, const double *demand,
               const double *alpha) {
  return f->fp32 ? pn_prepare_t<float>(f, x0, q, demand, alpha)
                 : pn_prepare_t<double>(f, x0, q, demand, alpha);
}

template <typename T>
int pn_init(PnFactor *f, const double *src) {
  const int nb = std::max(1, std::min(f->n, 4096));
  k_pn_init<T><<<nb, 128, 0, f->stream>>>(f->n, f->nx, f->nu, f->NXP, f->YP, src,
                                          static_cast<T *>(f->ya), static_cast<T *>(f->yb),
                                          f->x0, f->q, static_cast<T *>(f->x0t),
                                          static_cast<T *>(f->qt));
  PN_CUDA(cudaGetLastError());
  return RN_OK;
}

template <typename T>
int pn_gather(PnFactor *f, const T *yfin, double *u, double *x, double *y) {
  const int nb = std::max(1, std::min(f->n, 4096));
  k_pn_gather<T><<<nb, 128, 0, f->stream>>>(f->n, f->nx, f->nu, f->NXP, f->NUP, f->YP,
                                            static_cast<const T *>(f->uo),
                                            static_cast<const T *>(f->xo), yfin, f->q, f->x0, u,
                                            x, y);
  PN_CUDA(cudaGetLastError());
  return RN_OK;
}

int pn_cost(PnFactor *f, const double *u, const double *x, double out[3]) {
  PnCostArgs a{f->anc, f->prob, f->alpha, f->alpha0, f->bnd64, f->bnd64 + f->nx,
               f->bnd64 + 2 * f->nx, f->bnd64 + 3 * f->nx, f->bnd64 + 3 * f->nx + f->nu,
               f->Wp, f->Wi, f->Wv64, u, x, f->W_alpha, f->Wx, f->Ws, f->n, f->nx, f->nu};
  k_pn_cost<<<kPnParts, 256, 0, f->stream>>>(a, f->partial);
  PN_CUDA(cudaGetLastError());
  std::vector<double> h(3 * kPnParts);
  PN_CUDA(cudaMemcpyAsync(h.data(), f->partial, h.size() * sizeof(double), cudaMemcpyDeviceToHost,
                          f->stream));
  PN_CUDA(cudaStreamSynchronize(f->stream));
  out[0] = out[1] = out[2] = 0.0;
  for (int b = 0; b < kPnParts; ++b) {
    out[0] += h[3 * b];
    out[1] += h[3 * b + 1];
    out[2] = std::max(out[2], h[3 * b + 2]);
  }
  return RN_OK;
}

template <typename T>
int pn_solve_t(PnFactor *f, const double *x0, const double *q, const double *demand,
               const double *alpha, int max_iters, double tol, const double *y_warm,
               rn_result *out) {
  const bool avg = out->u_avg != nullptr;
  const int checks = (max_iters + f->check_every - 1) / f->check_every + 1;
  int rc;
  if ((rc = pn_beta(f, max_iters)) || (rc = pn_res(f, checks))) return rc;
  if ((rc = pn_prepare_t<T>(f, x0, q, demand, alpha)) || (rc = pn_init<T>(f, y_warm))) return rc;
  PN_CUDA(cudaMemsetAsync(f->res, 0, checks * sizeof(unsigned long long), f->stream));
  PN_CUDA(cudaMemsetAsync(f->err, 0, sizeof(int), f->stream));
  if (avg) {
    if (!f->uavg && ((rc = pn_alloc(f, &f->uavg, (size_t)f->n * f->NUP)) ||
                     (rc = pn_alloc(f, &f->xavg, (size_t)f->n * f->NXP))))
      return rc;
    PN_CUDA(cudaMemsetAsync(f->uavg, 0, (size_t)f->n * f->NUP * sizeof(double), f->stream));
    PN_CUDA(cudaMemsetAsync(f->xavg, 0, (size_t)f->n * f->NXP * sizeof(double), f->stream));
  }
  PnParams<T> P = pn_params<T>(f);
  P.apg = 1;
  P.iters = max_iters;
  P.it0 = 0;
  P.iters_total = max_iters;
  P.check_every = f->check_every;
  P.tol = tol > 0.0 ? tol : 0.0;
  P.c0 = static_cast<const T *>(f->c0);
  P.mc = static_cast<const T *>(f->mc);
  P.gd = static_cast<const T *>(f->gd);
  P.x0 = static_cast<const T *>(f->x0t);
  P.q = static_cast<const T *>(f->qt);
  P.uavg = avg ? f->uavg : nullptr;
  P.xavg = avg ? f->xavg : nullptr;
  P.beta = f->beta;
  P.theta = f->beta + f->beta_cap;
  P.res = f->res;
  PN_CUDA(cudaEventRecord(f->ev0, f->stream));
  if ((rc = pn_launch<T>(f, P))) return rc;
  PN_CUDA(cudaEventRecord(f->ev1, f->stream));
  int info[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  PN_CUDA(cudaMemcpyAsync(info, f->info, sizeof info, cudaMemcpyDeviceToHost, f->stream));
  if ((rc = pn_check_err(f))) return rc;
  const int iters = info[0], nchk = info[1], reason = info[2];
  {
    unsigned long long st[2];
    std::memcpy(st, info + 4, sizeof st);
    out->t_begin_ns = (long long)st[0];
    out->t_end_ns = (long long)st[1];
  }
  float ms = 0.f;
  PN_CUDA(cudaEventElapsedTime(&ms, f->ev0, f->ev1));
  out->apg_ms = ms;
  // y^{iters} was written into the buffer that held y^{iters-2}
  const T *yfin = static_cast<const T *>(((iters - 1) & 1) ? f->ya : f->yb);
  if ((rc = pn_gather<T>(f, yfin, out->u, out->x, out->y))) return rc;
  if (avg) {
    const int nb = std::max(1, std::min(f->n, 4096));
    k_pn_gather_avg<T><<<nb, 128, 0, f->stream>>>(f->n, f->nx, f->nu, f->NXP, f->NUP, f->uavg,
                                                  f->xavg, f->q, f->x0, out->u_avg, out->x_avg);
    PN_CUDA(cudaGetLastError());
  }
  std::vector<unsigned long long> hist(std::max(1, nchk));
  if (nchk > 0)
    PN_CUDA(cudaMemcpyAsync(hist.data(), f->res, nchk * sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, f->stream));
  double red[3];
  if ((rc = pn_cost(f, out->u, out->x, red))) return rc;
  out->cost = red[0] + red[1];
  out->ubox_viol = red[2];
  out->iters = iters;
  out->n_checks = nchk;
  out->gamma = f->gamma;
  std::vector<double> rh(std::max(1, nchk));
  for (int i = 0; i < nchk; ++i) {
    double d;
    std::memcpy(&d, &hist[i], sizeof d);
    rh[i] = d / f->gamma;
  }
  out->primal_res = nchk > 0 ? rh[nchk - 1] : NAN;
  if (out->res_hist && out->res_hist_len > 0 && nchk > 0)
    PN_CUDA(cudaMemcpyAsync(out->res_hist, rh.data(),
                            std::min(out->res_hist_len, nchk) * sizeof(double),
                            cudaMemcpyHostToDevice, f->stream));
  out->gap = NAN;
  PN_CUDA(cudaStreamSynchronize(f->stream));
  if (reason == 2) {
    set_error("the residual became non-finite after %d iterations", iters);
    return RN_ERR_DIVERGED;
  }
  if (reason == 3) {
    set_error("per-node path: a device-side wait gave up after %.3g s", f->wait_ns * 1e-9);
    return RN_ERR_TIMEOUT;
  }
  if (tol > 0.0 && reason != 1) return RN_NOT_CONVERGED;
  return RN_OK;
}

}  // namespace

namespace {

// ---------------------------------------------------------------------------
// RN_PREC_MIXED on the per-node form: FP32 iterations on the delta d = y - yb
// (linear evaluations of the FP32 matrices, x*(w) = x*(yb) + x_lin(dw), the
// dual update in delta form), the FP64 twin evaluating x*(yb) at the start
// and after every refresh (yb += d every refresh_every iterations), and the
// final x*(w) in FP64 (the same scheme as the shared-operator mixed kernel)
// ---------------------------------------------------------------------------
// yb = y_warm (padded, FP64) or 0, ybh = fl32(yb), d = 0 in both buffers
__global__ void k_pnm_init(int n, int nx, int nu, int NXP, int YP, const double *src,
                           double *yb, float *ybh, float *da, float *db) {
  const int ny = 2 * nx + nu;
  for (int v = blockIdx.x; v < n; v += gridDim.x)
    for (int e = threadIdx.x; e < YP; e += blockDim.x) {
      int k = -1;
      if (e < nx) k = e;
      else if (e >= NXP && e < NXP + nx) k = nx + (e - NXP);
      else if (e >= 2 * NXP && e < 2 * NXP + nu) k = 2 * nx + (e - 2 * NXP);
      const double val = (v > 0 && k >= 0 && src) ? src[(size_t)v * ny + k] : 0.0;
      const size_t o = (size_t)v * YP + e;
      yb[o] = val;
      ybh[o] = (float)val;
      da[o] = 0.f;
      db[o] = 0.f;
    }
}

// refresh: yb += dnew (FP64), ybh = fl32(yb), dold -= dnew, dnew = 0; the
// next iteration's w then starts from the same value relative to the new base
__global__ void k_pnm_refresh(size_t count, double *yb, float *ybh, float *dnew, float *dold) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count;
       e += (size_t)gridDim.x * blockDim.x) {
    const double y = yb[e] + (double)dnew[e];
    yb[e] = y;
    ybh[e] = (float)y;
    dold[e] -= dnew[e];
    dnew[e] = 0.f;
  }
}

__global__ void k_pnm_to32(size_t cu, size_t cx, const double *uo, const double *xo, float *uref,
                           float *xref) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < cu + cx;
       e += (size_t)gridDim.x * blockDim.x) {
    if (e < cu) uref[e] = (float)uo[e];
    else xref[e - cu] = (float)xo[e - cu];
  }
}

// out = yb + delta (FP64), padded layout
__global__ void k_pnm_add(size_t count, const double *yb, const float *dlt, double *out) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count;
       e += (size_t)gridDim.x * blockDim.x)
    out[e] = yb[e] + (double)dlt[e];
}

int pnm_grid(size_t count) { return (int)std::max<size_t>(1, std::min<size_t>((count + 255) / 256, 4096)); }

// x*(w) in FP64 on the twin for w = yb (+ delta, if given): its uo/xo
int pnm_eval64(PnFactor *f, const float *dlt) {
  PnFactor *T64 = f->twin;
  const size_t cnt = (size_t)f->n * f->YP;
  if (dlt) {
    k_pnm_add<<<pnm_grid(cnt), 256, 0, f->stream>>>(cnt, f->ybase, dlt,
                                                   static_cast<double *>(T64->ya));
  } else {
    PN_CUDA(cudaMemcpyAsync(T64->ya, f->ybase, cnt * sizeof(double), cudaMemcpyDeviceToDevice,
                            f->stream));
  }
  PN_CUDA(cudaGetLastError());
  return pn_eval<double>(T64, false);
}

int pnm_refs(PnFactor *f) {
  PnFactor *T64 = f->twin;
  const size_t cu = (size_t)f->n * f->NUP, cx = (size_t)f->n * f->NXP;
  k_pnm_to32<<<pnm_grid(cu + cx), 256, 0, f->stream>>>(cu, cx, static_cast<double *>(T64->uo),
                                                       static_cast<double *>(T64->xo), f->uref,
                                                       f->xref);
  PN_CUDA(cudaGetLastError());
  return RN_OK;
}

int pn_solve_mixed(PnFactor *f, const double *x0, const double *q, const double *demand,
                   const double *alpha, int max_iters, double tol, const double *y_warm,
                   rn_result *out) {
  PnFactor *T64 = f->twin;
  const bool avg = out->u_avg != nullptr;
  const int n = f->n;
  const int checks = (max_iters + f->check_every - 1) / f->check_every + 1;
  int rc;
  if ((rc = pn_beta(f, max_iters)) || (rc = pn_res(f, checks))) return rc;
  // the twin's data terms, and its FP64 copies of x0 and q
  if ((rc = pn_prepare_t<double>(T64, x0, q, demand, alpha)) || (rc = pn_init<double>(T64, nullptr)))
    return rc;
  PN_CUDA(cudaMemsetAsync(f->res, 0, checks * sizeof(unsigned long long), f->stream));
  PN_CUDA(cudaMemsetAsync(f->err, 0, sizeof(int), f->stream));
  PN_CUDA(cudaMemsetAsync(T64->err, 0, sizeof(int), f->stream));
  if (avg) {
    if (!f->uavg && ((rc = pn_alloc(f, &f->uavg, (size_t)n * f->NUP)) ||
                     (rc = pn_alloc(f, &f->xavg, (size_t)n * f->NXP))))
      return rc;
    PN_CUDA(cudaMemsetAsync(f->uavg, 0, (size_t)n * f->NUP * sizeof(double), f->stream));
    PN_CUDA(cudaMemsetAsync(f->xavg, 0, (size_t)n * f->NXP * sizeof(double), f->stream));
  }
  const int nb = std::max(1, std::min(n, 4096));
  PN_CUDA(cudaEventRecord(f->ev0, f->stream));
  k_pnm_init<<<nb, 128, 0, f->stream>>>(n, f->nx, f->nu, f->NXP, f->YP, y_warm, f->ybase, f->ybh,
                                        static_cast<float *>(f->ya), static_cast<float *>(f->yb));
  PN_CUDA(cudaGetLastError());
  if ((rc = pnm_eval64(f, nullptr)) || (rc = pnm_refs(f))) return rc;
  int done = 0, nchk = 0, reason = 0;
  unsigned long long t_begin = 0, t_end = 0;
  while (done < max_iters) {
    const int len = std::min(f->refresh_every, max_iters - done);
    PnParams<float> P = pn_params<float>(f);
    P.apg = 1;
    P.delta = 1;
    P.it0 = done;
    P.iters = len;
    P.iters_total = max_iters;
    P.check_every = f->check_every;
    P.tol = tol > 0.0 ? tol : 0.0;
    P.ybh = f->ybh;
    P.uref = f->uref;
    P.xref = f->xref;
    P.swy = f->swy;
    P.uavg = avg ? f->uavg : nullptr;
    P.xavg = avg ? f->xavg : nullptr;
    P.beta = f->beta;
    P.theta = f->beta + f->beta_cap;
    P.res = f->res + nchk;
    if ((rc = pn_launch<float>(f, P))) return rc;
    int info[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    PN_CUDA(cudaMemcpyAsync(info, f->info, sizeof info, cudaMemcpyDeviceToHost, f->stream));
    if ((rc = pn_check_err(f))) return rc;
    {
      unsigned long long st[2];
      std::memcpy(st, info + 4, sizeof st);
      if (done == 0) t_begin = st[0];
      t_end = st[1];
    }
    done += info[0];
    nchk += info[1];
    reason = info[2];
    if (reason != 0) break;
    if (done < max_iters) {
      // y^done sits in the buffer that iteration done - 1 wrote
      float *dnew = static_cast<float *>(((done - 1) & 1) ? f->ya : f->yb);
      float *dold = static_cast<float *>(((done - 1) & 1) ? f->yb : f->ya);
      const size_t cnt = (size_t)n * f->YP;
      k_pnm_refresh<<<pnm_grid(cnt), 256, 0, f->stream>>>(cnt, f->ybase, f->ybh, dnew, dold);
      PN_CUDA(cudaGetLastError());
      if ((rc = pnm_eval64(f, nullptr)) || (rc = pnm_refs(f))) return rc;
    }
  }
  // the primal of the last iteration, x*(yb + dw), in FP64
  if ((rc = pnm_eval64(f, f->swy))) return rc;
  PN_CUDA(cudaEventRecord(f->ev1, f->stream));
  if ((rc = pn_check_err(T64))) return rc;
  float ms = 0.f;
  PN_CUDA(cudaEventElapsedTime(&ms, f->ev0, f->ev1));
  out->apg_ms = ms;
  out->t_begin_ns = (long long)t_begin;
  out->t_end_ns = (long long)t_end;
  // outputs: (u, x) of the FP64 evaluation, y = yb + d^done
  if ((rc = pn_gather<double>(T64, nullptr, out->u, out->x, nullptr))) return rc;
  {
    const float *dfin = static_cast<const float *>(((done - 1) & 1) ? f->ya : f->yb);
    const size_t cnt = (size_t)n * f->YP;
    double *yfull = static_cast<double *>(T64->yb);  // scratch of the twin
    k_pnm_add<<<pnm_grid(cnt), 256, 0, f->stream>>>(cnt, f->ybase, dfin, yfull);
    PN_CUDA(cudaGetLastError());
    k_pn_gather<double><<<nb, 128, 0, f->stream>>>(n, f->nx, f->nu, f->NXP, f->NUP, f->YP, nullptr,
                                                   nullptr, yfull, T64->q, T64->x0, nullptr,
                                                   nullptr, out->y);
    PN_CUDA(cudaGetLastError());
  }
  if (avg) {
    k_pn_gather_avg<float><<<nb, 128, 0, f->stream>>>(n, f->nx, f->nu, f->NXP, f->NUP, f->uavg,
                                                      f->xavg, T64->q, T64->x0, out->u_avg,
                                                      out->x_avg);
    PN_CUDA(cudaGetLastError());
  }
  std::vector<unsigned long long> hist(std::max(1, nchk));
  if (nchk > 0)
    PN_CUDA(cudaMemcpyAsync(hist.data(), f->res, nchk * sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, f->stream));
  double red[3];
  if ((rc = pn_cost(T64, out->u, out->x, red))) return rc;
  out->cost = red[0] + red[1];
  out->ubox_viol = red[2];
  out->iters = done;
  out->n_checks = nchk;
  out->gamma = f->gamma;
  std::vector<double> rh(std::max(1, nchk));
  for (int i = 0; i < nchk; ++i) {
    double d;
    std::memcpy(&d, &hist[i], sizeof d);
    rh[i] = d / f->gamma;
  }
  out->primal_res = nchk > 0 ? rh[nchk - 1] : NAN;
  if (out->res_hist && out->res_hist_len > 0 && nchk > 0)
    PN_CUDA(cudaMemcpyAsync(out->res_hist, rh.data(),
                            std::min(out->res_hist_len, nchk) * sizeof(double),
                            cudaMemcpyHostToDevice, f->stream));
  out->gap = NAN;
  PN_CUDA(cudaStreamSynchronize(f->stream));
  if (reason == 2) {
    set_error("the residual became non-finite after %d iterations", done);
    return RN_ERR_DIVERGED;
  }
  if (reason == 3) {
    set_error("per-node path: a device-side wait gave up after %.3g s", f->wait_ns * 1e-9);
    return RN_ERR_TIMEOUT;
  }
  if (tol > 0.0 && reason != 1) return RN_NOT_CONVERGED;
  return RN_OK;
}

}  // namespace

int pn_solve_device(PnFactor *f, const double *x0, const double *q, const double *demand,
                    const double *alpha, int max_iters, double tol, const double *y_warm,
                    rn_result *out) {
  if (out->compute_gap) {
    set_error("solve: the per-node factor form does not evaluate the duality gap");
    return RN_ERR_UNSUPPORTED;
  }
  PN_CUDA(cudaSetDevice(f->device));
  if (f->mixed) return pn_solve_mixed(f, x0, q, demand, alpha, max_iters, tol, y_warm, out);
  return f->fp32 ? pn_solve_t<float>(f, x0, q, demand, alpha, max_iters, tol, y_warm, out)
                 : pn_solve_t<double>(f, x0, q, demand, alpha, max_iters, tol, y_warm, out);
}

namespace {
template <typename T>
int pn_dual_gradient_t(PnFactor *f, const double *w, double *u, double *x) {
  int rc;
  if ((rc = pn_init<T>(f, w))) return rc;
  PN_CUDA(cudaMemsetAsync(f->err, 0, sizeof(int), f->stream));
  if ((rc = pn_eval<T>(f, false))) return rc;
  if ((rc = pn_gather<T>(f, nullptr, u, x, nullptr))) return rc;
  return pn_check_err(f);
}
}  // namespace

int pn_dual_gradient_device(PnFactor *f, const double *x0, const double *q,
                            const double *demand, const double *alpha, const double *w,
                            double *u, double *x) {
  if (f->mixed) return pn_dual_gradient_device(f->twin, x0, q, demand, alpha, w, u, x);
  PN_CUDA(cudaSetDevice(f->device));
  int rc;
  if (x0 || q || demand || alpha) {
    if (!(x0 && q && demand && alpha)) {
      set_error("dual_gradient: give all of x0, q, demand, alpha or none");
      return RN_ERR_INVAL;
    }
    if ((rc = pn_prepare(f, x0, q, demand, alpha))) return rc;
  } else if (!f->have_data) {
    set_error("dual_gradient: no data yet (give x0, q, demand, alpha)");
    return RN_ERR_INVAL;
  }
  return f->fp32 ? pn_dual_gradient_t<float>(f, w, u, x)
                 : pn_dual_gradient_t<double>(f, w, u, x);
}

void pn_info(const PnFactor *f, rn_factor_info *info) {
  info->grid_ctas = f->grid;
  info->block_threads = f->block;
  info->L = f->L;
  info->gamma = f->gamma;
  info->device_bytes = f->bytes + (f->twin ? f->twin->bytes : 0);
  info->n_chains = f->n_chains;
  info->n_top = f->n_top;
}

double pn_gamma(const PnFactor *f) { return f->gamma; }

}  // namespace rn
