// Batched mode: many independent scenario-tree problems, each with its own
// network, tree and step size, solved by the mixed-precision dual APG
// (mixed_kernels.cu) in one cooperative launch.
//
// Work items (problem, chain) are sorted by problem and dealt to blocks in
// contiguous ranges, so a block touches few problems; when it moves to
// another problem it loads that problem's parameters and network copy into
// shared memory.  Every problem keeps its own counters, flags and residual
// slots; the blocks share one grid barrier at the residual checks, after
// which each block decides, for the problems it touches, whether they stop
// (all blocks read the same residuals, so they agree).  A stopped problem's
// items are skipped; its final FP64 evaluation runs with everybody's at the
// end.
#include "solve_device.cuh"

namespace rn {

struct BatchCtx {
  int n;                          // distinct problems of this block
  int prob[kBatchMaxDistinct];
  int active[kBatchMaxDistinct];
  unsigned long long rbits[kBatchMaxDistinct];
  int loaded;                     // problem whose parameters sit in mp
};

// parameters of problem p into shared memory (with its network copy)
__device__ void load_problem(const BatchDev &B, int p, BatchCtx &bc, MixedParams &mp,
                             unsigned char *raw, Smem<float> &smf, Smem<double> &smd) {
  if (bc.loaded == p) return;
  __syncthreads();
  if (threadIdx.x == 0) mp = B.probs[p];
  __syncthreads();
  smf = carve<float>(raw, mp.f.net, B.buf_f);
  smd = carve<double>(raw, mp.d.net, B.buf_d);
  unsigned char *net_raw = smf.net_raw > smd.net_raw ? smf.net_raw : smd.net_raw;
  smf.net = stage_net(mp.f.net, net_raw);
  smd.net = stage_net(mp.d.net, net_raw + B.net_bytes_f, false);
  if (threadIdx.x == 0) bc.loaded = p;
  __syncthreads();
}

__device__ int slot_of(const BatchCtx &bc, int p) {
  for (int s = 0; s < bc.n; ++s)
    if (bc.prob[s] == p) return s;
  return -1;
}

// one FP64 evaluation of the dual gradient for the participating problems
template <int C>
__device__ bool batch_fp64_step(const BatchDev &B, BatchCtx &bc, MixedParams &mp,
                                unsigned char *raw, Smem<float> &smf, Smem<double> &smd,
                                unsigned step, bool all) {
  const int i0 = B.cta_begin[blockIdx.x], i1 = B.cta_begin[blockIdx.x + 1];
  for (int i = i0; i < i1; ++i) {
    const int p = B.item_prob[i];
    if (!all && !bc.active[slot_of(bc, p)]) continue;
    load_problem(B, p, bc, mp, raw, smf, smd);
    chain_backward<double, C>(mp.d, B.item_chain[i], smd);
    climb(mp.d, B.item_chain[i], step, smd);
  }
  FwdCtx<double> c{};
  for (int i = i0; i < i1; ++i) {
    const int p = B.item_prob[i];
    if (!all && !bc.active[slot_of(bc, p)]) continue;
    load_problem(B, p, bc, mp, raw, smf, smd);
    const int k = B.item_chain[i];
    const int f = mp.d.plan.ch_flag[k];
    if (f >= 0) {
      if (threadIdx.x == 0) smd.flag[1] = spin_geq(mp.d.st.flags + f, step + 1u, mp.d.st.err);
      __syncthreads();
      if (!smd.flag[1]) return false;
    }
    chain_forward<double, kFwdPlain, C>(mp.d, k, c, smd, nullptr);
  }
  return true;
}

template <int C>
__global__ void __launch_bounds__(256) k_batch(BatchDev B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ MixedParams mp;
  __shared__ BatchCtx bc;
  Smem<float> smf{};
  Smem<double> smd{};
  const int tid = threadIdx.x, warp = tid >> 5, nw = blockDim.x >> 5;
  const int i0 = B.cta_begin[blockIdx.x], i1 = B.cta_begin[blockIdx.x + 1];
  if (tid == 0) {
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
  bool ok = batch_fp64_step<C>(B, bc, mp, smem_raw, smf, smd, step++, true);
  for (; it < B.iters && ok; ++it) {
    // FP32 backward sweep and top-node reductions
    for (int i = i0; i < i1; ++i) {
      const int p = B.item_prob[i];
      if (!bc.active[slot_of(bc, p)]) continue;
      load_problem(B, p, bc, mp, smem_raw, smf, smd);
      chain_backward<float, C>(mp.f, B.item_chain[i], smf);
      climb(mp.f, B.item_chain[i], step, smf);
    }
    const bool check = ((it + 1) % B.check_every) == 0 || it + 1 == B.iters;
    // FP32 forward sweep with the dual update
    for (int i = i0; i < i1 && ok; ++i) {
      const int p = B.item_prob[i];
      const int sl = slot_of(bc, p);
      if (!bc.active[sl]) continue;
      load_problem(B, p, bc, mp, smem_raw, smf, smd);
      const int k = B.item_chain[i];
      FwdCtx<float> c;
      c.ycur = (it & 1) ? mp.mx.db : mp.mx.da;
      c.yprv = (it & 1) ? mp.mx.da : mp.mx.db;
      c.beta = (float)mp.f.st.beta[it];
      c.beta_n = (float)mp.f.st.beta[it + 1];
      c.write_out = check;
      c.rbits = 0ull;
      const int f = mp.f.plan.ch_flag[k];
      if (f >= 0) {
        if (tid == 0) smf.flag[1] = spin_geq(mp.f.st.flags + f, step + 1u, mp.f.st.err);
        __syncthreads();
        if (!smf.flag[1]) {
          ok = false;
          break;
        }
      }
      chain_forward<float, kFwdMixed, C>(mp.f, k, c, smf, &mp.mx);
      const unsigned long long r = block_max_u64(c.rbits, smf.redu);
      if (tid == 0 && r > bc.rbits[sl]) bc.rbits[sl] = r;
    }
    ++step;
    if (!ok) break;
    if (check) {
      __syncthreads();
      if (tid == 0) {
        for (int s = 0; s < bc.n; ++s) {
          if (!bc.active[s]) continue;
          atomicMax(B.probs[bc.prob[s]].f.st.res + ci, bc.rbits[s]);
          bc.rbits[s] = 0ull;
        }
        __threadfence();
        atomicAdd(B.barrier, 1u);
        smf.flag[2] = spin_geq(B.barrier, (unsigned)(ci + 1) * gridDim.x, mp.f.st.err);
      }
      __syncthreads();
      if (!smf.flag[2]) {
        ok = false;
        break;
      }
      // the same residuals are visible to every block: consistent stops
      if (tid == 0) {
        for (int s = 0; s < bc.n; ++s) {
          if (!bc.active[s]) continue;
          const MixedParams &q = B.probs[bc.prob[s]];
          const unsigned long long rb = __ldcg(q.f.st.res + ci);
          const double rv = __longlong_as_double((long long)rb) * q.f.invgamma;
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
        load_problem(B, p, bc, mp, smem_raw, smf, smd);
        float *dcur = (it & 1) ? mp.mx.db : mp.mx.da;
        float *dprv = (it & 1) ? mp.mx.da : mp.mx.db;
        const float bn = (float)mp.f.st.beta[it + 1];
        int idx = 0;
        for_owned(mp.f.plan, B.item_chain[i], [&](int v) {
          if ((idx++ % nw) == warp) refresh_node(mp, v, dprv, dcur, bn);
        });
        __syncthreads();
      }
      if (!batch_fp64_step<C>(B, bc, mp, smem_raw, smf, smd, step++, false)) {
        ok = false;
        break;
      }
    }
  }
  if (ok) {
    for (int i = i0; i < i1; ++i) {
      load_problem(B, B.item_prob[i], bc, mp, smem_raw, smf, smd);
      int idx = 0;
      for_owned(mp.f.plan, B.item_chain[i], [&](int v) {
        if ((idx++ % nw) == warp) final_node(mp, v);
      });
      __syncthreads();
    }
    ok = batch_fp64_step<C>(B, bc, mp, smem_raw, smf, smd, step++, true);
  }
  // problems that ran to the end
  if (tid == 0) {
    for (int s = 0; s < bc.n; ++s) {
      if (!bc.active[s]) continue;
      int *info = B.prob_info + 3 * bc.prob[s];
      info[0] = it;
      info[1] = ci;
      info[2] = ok ? 0 : 3;
    }
  }
}

static const void *batch_fn(int c) {
  switch (c) {
    case 1: return (const void *)k_batch<1>;
    case 2: return (const void *)k_batch<2>;
    case 4: return (const void *)k_batch<4>;
    default: return (const void *)k_batch<8>;
  }
}

cudaError_t launch_batch(const BatchDev &B, int maxc, int grid, int block, size_t smem,
                         cudaStream_t st) {
  const void *fn = batch_fn(maxc);
  cudaError_t e = allow_max_smem(fn);
  if (e != cudaSuccess) return e;
  BatchDev b = B;
  void *args[] = {&b};
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(block), args, smem, st);
}

cudaError_t batch_occupancy(int maxc, int block, size_t smem, int *blocks_per_sm) {
  const void *fn = batch_fn(maxc);
  cudaError_t e = allow_max_smem(fn);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, block, smem);
}

}  // namespace rn
