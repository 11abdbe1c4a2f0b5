// Batched mode: many independent scenario-tree problems, each with its own
// network, tree and step size, solved by the mixed-precision dual APG
// (mixed_kernels.cu) in one cooperative launch.
//
// Work items are (problem, group) and (problem, pair of chains), numbered
// within a problem as in the single-problem kernels (groups first), sorted
// by problem and dealt to blocks in contiguous ranges, so a block touches
// few problems; when it moves to another problem it loads that problem's
// parameters and network copy into shared memory.  Every problem keeps its
// own counters, flags and residual slots; the blocks share one grid
// barrier at the residual checks, after which each block decides, for the
// problems it touches, whether they stop (all blocks read the same
// residuals, so they agree).  A stopped problem's items are skipped; its
// final FP64 evaluation runs with everybody's at the end.
#include "solve_device.cuh"

namespace rn {

struct BatchCtx {
  int n;                          // distinct problems of this block
  int prob[kBatchMaxDistinct];
  int active[kBatchMaxDistinct];
  unsigned long long rbits[kBatchMaxDistinct];
  int loaded;                     // problem whose parameters sit in mp
};

// parameters of problem p into shared memory (with its network copy);
// every thread of the block calls it at the same points
static __device__ void load_problem(const BatchDev &B, int p, BatchCtx &bc, MixedParams &mp,
                             const BlockMem &bm) {
  if (bc.loaded == p) return;
  __syncthreads();
  if (threadIdx.x == 0) mp = B.probs[p];
  __syncthreads();
  stage_net(mp.f.net, bm.net_raw);
  stage_net(mp.d.net, bm.net_raw + B.net_bytes_f, false);
  if (threadIdx.x == 0) bc.loaded = p;
  __syncthreads();
}

static __device__ int slot_of(const BatchCtx &bc, int p) {
  for (int s = 0; s < bc.n; ++s)
    if (bc.prob[s] == p) return s;
  return -1;
}

// one evaluation of the dual gradient for the participating problems
// (all, or the active ones); the phases of eval_step over the block's items
template <typename T, int MODE, int C, typename CtxF>
__device__ bool batch_eval(const BatchDev &B, BatchCtx &bc, MixedParams &mp, const BlockMem &bm,
                           unsigned step, bool all, CtxF make_ctx) {
  const int i0 = B.cta_begin[blockIdx.x], i1 = B.cta_begin[blockIdx.x + 1];
  const Team tc = chain_team(B.tpb), tb = block_team();
  const int ti = team_index(B.tpb);
  auto params = [&]() -> const KParams<T> & {
    if constexpr (sizeof(T) == 4) return mp.f; else return mp.d;
  };
  auto smem_c = [&]() {
    const KParams<T> &P = params();
    return carve<T>(bm.team_raw(ti), P.buf_elems,
                    reinterpret_cast<const NetDev<T> *>(sizeof(T) == 4 ? bm.net_raw
                                                                       : bm.net_raw + B.net_bytes_f));
  };
  auto smem_g = [&]() {
    const KParams<T> &P = params();
    return carve<T>(bm.team_raw(0), P.gbuf_elems,
                    reinterpret_cast<const NetDev<T> *>(sizeof(T) == 4 ? bm.net_raw
                                                                       : bm.net_raw + B.net_bytes_f));
  };
  auto use = [&](int i) {
    const int p = B.item_prob[i];
    return all || bc.active[slot_of(bc, p)];
  };
  for (int i = i0; i < i1; ++i) {
    if (!use(i)) continue;
    load_problem(B, B.item_prob[i], bc, mp, bm);
    const KParams<T> &P = params();
    const int G = P.plan.n_groups, sub = B.item_sub[i], k = B.tpb * (sub - G) + ti;
    if (sub >= G && k < P.plan.n_chains) chain_head<T, C>(P, k, smem_c(), tc);
  }
  bool ok = true;
  for (int i = i0; i < i1; ++i) {
    if (!use(i)) continue;
    load_problem(B, B.item_prob[i], bc, mp, bm);
    const KParams<T> &P = params();
    const int sub = B.item_sub[i];
    if (sub < P.plan.n_groups) {
      __syncthreads();
      if (!group_step<T>(P, sub, smem_g(), tb, step, 0)) ok = false;
    }
  }
  for (int i = i0; i < i1; ++i) {
    if (!use(i)) continue;
    load_problem(B, B.item_prob[i], bc, mp, bm);
    const KParams<T> &P = params();
    const int G = P.plan.n_groups, sub = B.item_sub[i], k = B.tpb * (sub - G) + ti;
    if (sub >= G && k < P.plan.n_chains) chain_rest<T, C>(P, k, smem_c(), tc, false);
  }
  // parts of split subtrees complete their root once every part of it has
  // arrived: a block may hold several parts, so no part waits before the
  // block has done the first half of all of its groups
  for (int i = i0; i < i1; ++i) {
    if (!use(i)) continue;
    load_problem(B, B.item_prob[i], bc, mp, bm);
    const KParams<T> &P = params();
    const int sub = B.item_sub[i];
    if (sub < P.plan.n_groups && P.plan.g_root[sub] >= 0) {
      __syncthreads();
      if (!group_step<T>(P, sub, smem_g(), tb, step, 1)) ok = false;
    }
  }
  for (int i = i0; i < i1; ++i) {
    if (!use(i)) continue;
    load_problem(B, B.item_prob[i], bc, mp, bm);
    const KParams<T> &P = params();
    const int G = P.plan.n_groups, sub = B.item_sub[i], k = B.tpb * (sub - G) + ti;
    if (sub >= G && k < P.plan.n_chains && ok) {
      FwdCtx<T> *c = make_ctx(slot_of(bc, B.item_prob[i]));
      ok = chain_forward<T, MODE, C>(P, k, *c, smem_c(), tc, &mp.mx, step);
    }
  }
  return ok;
}

template <int C>
__global__ void __launch_bounds__(512) k_batch(BatchDev B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ MixedParams mp;
  __shared__ BatchCtx bc;
  const BlockMem bm = block_mem(smem_raw, B.net_bytes, B.team_bytes);
  const Team tc = chain_team(B.tpb);
  const int ti = team_index(B.tpb);
  const int i0 = B.cta_begin[blockIdx.x], i1 = B.cta_begin[blockIdx.x + 1];
  if (threadIdx.x == 0) {
    bc.n = 0;
    bc.loaded = -1;
    for (int i = i0; i < i1; ++i) {
      const int p = B.item_prob[i];
      if (bc.n == 0 || bc.prob[bc.n - 1] != p) {
        bc.prob[bc.n] = p;
        bc.active[bc.n] = 1;
        bc.rbits[bc.n] = 0ull;
        ++bc.n;
      }
    }
  }
  __syncthreads();
  unsigned step = 0;
  int it = 0, ci = 0;
  FwdCtx<double> c64{};
  auto ctx64 = [&](int) { return &c64; };
  batch_eval<double, kFwdPlain, C>(B, bc, mp, bm, step++, true, ctx64);
  bool ok = !block_err(bm, B.err);
  // per-problem FP32 contexts differ only in their residual accumulator
  FwdCtx<float> cf;
  unsigned long long rb_local[kBatchMaxDistinct];
  for (; it < B.iters && ok; ++it) {
    const bool check = ((it + 1) % B.check_every) == 0 || it + 1 == B.iters;
    for (int s = 0; s < kBatchMaxDistinct; ++s) rb_local[s] = 0ull;
    int cur = -1;
    auto ctx32 = [&](int sl) {
      if (sl != cur) {
        if (cur >= 0) rb_local[cur] = cf.rbits;
        cur = sl;
        cf.ycur = (it & 1) ? mp.mx.db : mp.mx.da;
        cf.yprv = (it & 1) ? mp.mx.da : mp.mx.db;
        cf.beta = (float)mp.f.st.beta[it];
        cf.beta_n = (float)mp.f.st.beta[it + 1];
        cf.write_out = check;
        cf.avg = false;
        cf.theta = 0.0;
        cf.rbits = rb_local[sl];
      }
      return &cf;
    };
    batch_eval<float, kFwdMixed, C>(B, bc, mp, bm, step++, false, ctx32);
    if (cur >= 0) rb_local[cur] = cf.rbits;
    if (block_err(bm, B.err)) {
      ok = false;
      break;
    }
    if (check) {
      // per problem: block maximum, then one grid barrier for all
      for (int s = 0; s < bc.n; ++s) {
        const unsigned long long r = block_max_u64(widen_bits(rb_local[s]), bm.redu);
        if (threadIdx.x == 0 && bc.active[s]) atomicMax(B.probs[bc.prob[s]].f.st.res + ci, r);
      }
      if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(B.barrier, 1u);
        bm.bflag[1] = spin_geq(B.barrier, (unsigned)(ci + 1) * gridDim.x, B.err, B.wait_ns, 4);
      }
      __syncthreads();
      if (!bm.bflag[1]) {
        ok = false;
        break;
      }
      // the same residuals are visible to every block: consistent stops
      if (threadIdx.x == 0) {
        for (int s = 0; s < bc.n; ++s) {
          if (!bc.active[s]) continue;
          const MixedParams &q = B.probs[bc.prob[s]];
          const unsigned long long rbv = __ldcg(q.f.st.res + ci);
          const double rv = __longlong_as_double((long long)rbv) * q.f.invgamma;
          int reason = -1;
          if (!(rv <= 1.7976931348623157e308)) reason = 2;
          else if (B.tol > 0.0 && rv <= B.tol) reason = 1;
          if (reason >= 0) {
            bc.active[s] = 0;
            int *info = B.prob_info + 3 * bc.prob[s];
            info[0] = it + 1;
            info[1] = ci + 1;
            info[2] = reason;
          }
        }
      }
      ++ci;
      __syncthreads();
    }
    if ((it + 1) % B.refresh_every == 0 && it + 1 < B.iters) {
      for (int i = i0; i < i1; ++i) {
        const int p = B.item_prob[i];
        if (!bc.active[slot_of(bc, p)]) continue;
        load_problem(B, p, bc, mp, bm);
        const int G = mp.f.plan.n_groups, sub = B.item_sub[i], k = B.tpb * (sub - G) + ti;
        if (sub >= G && k < mp.f.plan.n_chains) {
          float *dcur = (it & 1) ? mp.mx.db : mp.mx.da;
          float *dprv = (it & 1) ? mp.mx.da : mp.mx.db;
          const float bn = (float)mp.f.st.beta[it + 1];
          int idx = 0;
          for_owned(mp.f.plan, k, [&](int v) {
            if ((idx++ % tc.nwarps()) == tc.warp()) refresh_node(mp, v, dprv, dcur, bn);
          });
        }
        tc.sync();
      }
      batch_eval<double, kFwdPlain, C>(B, bc, mp, bm, step++, false, ctx64);
      if (block_err(bm, B.err)) {
        ok = false;
        break;
      }
    }
  }
  if (ok) {
    for (int i = i0; i < i1; ++i) {
      load_problem(B, B.item_prob[i], bc, mp, bm);
      const int G = mp.f.plan.n_groups, sub = B.item_sub[i], k = B.tpb * (sub - G) + ti;
      if (sub >= G && k < mp.f.plan.n_chains) {
        int idx = 0;
        for_owned(mp.f.plan, k, [&](int v) {
          if ((idx++ % tc.nwarps()) == tc.warp()) final_node(mp, v);
        });
      }
      tc.sync();
    }
    batch_eval<double, kFwdPlain, C>(B, bc, mp, bm, step++, true, ctx64);
    ok = !block_err(bm, B.err);
  }
  // problems that ran to the end
  if (threadIdx.x == 0) {
    for (int s = 0; s < bc.n; ++s) {
      if (!bc.active[s]) continue;
      int *info = B.prob_info + 3 * bc.prob[s];
      info[0] = it;
      info[1] = ci;
      info[2] = ok ? 0 : 3;
    }
  }
}

// this translation unit is compiled once per component count RN_CVAL
const void *RN_CAT(batch_kernel_c, RN_CVAL)() { return (const void *)k_batch<RN_CVAL>; }

}  // namespace rn
