// Scenario tree from sampled paths (include/rapidnet.h,
// rapidnet_scenario_tree): paper §2.3 and §6.2, where Monte-Carlo scenarios
// of the forecast errors are reduced into a tree by the method of Heitsch
// and Römisch.
//
// The tree is built forward, stage by stage.  Every node of stage t holds
// a bundle of the paths (the root all of them); its b_t children are
// representatives chosen from the bundle by fast forward selection on the
// distance between the paths' remaining parts (stages t+1 .. N):
//   d(i, j) = || x_i[t:] - x_j[t:] ||  (Euclidean over stages and dimensions)
//   z(u)    = sum_j p_j min(m_j, d(j, u)),  m_j = min over chosen c of d(j, c)
// one representative at a time, the one with the smallest z (lowest index
// on ties, a tie being a value within 1e-12 relative of the smallest);
// every path of the bundle then goes to its nearest representative (first
// chosen on ties).  Per bundle on the GPU:
//   k_tail_dist   the bundle's distance matrix (FP64, tiles of 32 x 32 pairs,
//                 the tails staged through shared memory);
//   k_ffs_z       z for every candidate: one warp per candidate reads one
//                 row of the matrix (it is symmetric) with the weights and
//                 the current minima: the matrix streams from HBM once per
//                 choice, the bound of this step;
//   k_ffs_pick    the smallest z (one block), marks the choice;
//   k_ffs_update  m_j = min(m_j, d(j, chosen));
//   k_assign      each path's nearest representative.
// The host keeps the bundles (index lists) and writes the tree in
// breadth-first order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "rn_internal.h"

namespace {

constexpr int kTile = 32;

// D[a][b] = || X[idx[a], t0:] - X[idx[b], t0:] || for a bundle of M paths;
// X is S x R row-major (R = N dim), the tail is columns [c0, R)
__global__ void k_tail_dist(const double *X, int R, const int *idx, int M, int c0, double *D) {
  __shared__ double A[kTile][kTile + 1], Bt[kTile][kTile + 1];
  const int a0 = blockIdx.y * kTile, b0 = blockIdx.x * kTile;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8 threads
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int c = c0; c < R; c += kTile) {
    for (int r = ty; r < kTile; r += 8) {
      const int a = a0 + r, b = b0 + r, col = c + tx;
      A[r][tx] = (a < M && col < R) ? X[(size_t)idx[a] * R + col] : 0.0;
      Bt[r][tx] = (b < M && col < R) ? X[(size_t)idx[b] * R + col] : 0.0;
    }
    __syncthreads();
    const int kmax = min(kTile, R - c);
    for (int k = 0; k < kmax; ++k) {
      const double bv = Bt[tx][k];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const double diff = A[ty + 8 * q][k] - bv;
        acc[q] = fma(diff, diff, acc[q]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int a = a0 + ty + 8 * q, b = b0 + tx;
    if (a < M && b < M) D[(size_t)a * M + b] = sqrt(acc[q]);
  }
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// z[u] = sum_j p_j min(m_j, D[u][j]) for every candidate u not yet chosen
// (a chosen one gets +inf); one warp per candidate
__global__ void k_ffs_z(const double *D, int M, const double *p, const double *m,
                        const int *chosen, double *z) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < M; u += warps) {
    const double *row = D + (size_t)u * M;
    double acc = 0.0;
    for (int j = lane; j < M; j += 32) acc += p[j] * fmin(m[j], __ldcs(row + j));
    acc = warp_sum_d(acc);
    if (lane == 0) z[u] = chosen[u] ? INFINITY : acc;
  }
}

// values within kTie (relative) of the smallest count as ties: they are real
// (in one dimension the median of an even number of paths is an interval),
// and sums added in different orders must still take the same decision
constexpr double kTie = 1e-12;

// the lowest candidate whose z is within kTie of the smallest becomes
// choice k (one block: the smallest value, then the first index within it)
__global__ void k_ffs_pick(const double *z, int M, int k, int *chosen, int *sel) {
  __shared__ double red[32];
  __shared__ int ired[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double lo = INFINITY;
  for (int u = threadIdx.x; u < M; u += blockDim.x) lo = fmin(lo, z[u]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
  if (lane == 0) red[w] = lo;
  __syncthreads();
  lo = red[0];
  for (int q = 1; q < nw; ++q) lo = fmin(lo, red[q]);
  const double thr = lo + kTie * fabs(lo);
  int first = M;
  for (int u = threadIdx.x; u < M; u += blockDim.x)
    if (z[u] <= thr) {
      first = u;
      break;
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) first = min(first, __shfl_xor_sync(0xffffffffu, first, o));
  if (lane == 0) ired[w] = first;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < nw; ++q) first = min(first, ired[q]);
    first = min(first, ired[0]);
    if (first >= M) first = 0;  // every candidate chosen (not reached: k < M)
    sel[k] = first;
    chosen[first] = 1;
  }
}

// m_j = min(m_j, D[sel[k]][j])
__global__ void k_ffs_update(const double *D, int M, const int *sel, int k, double *m) {
  const double *row = D + (size_t)sel[k] * M;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < M; j += gridDim.x * blockDim.x)
    m[j] = fmin(m[j], row[j]);
}

// owner[j] = the first chosen representative within kTie of the nearest
__global__ void k_assign(const double *D, int M, const int *sel, int K, int *owner) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < M; j += gridDim.x * blockDim.x) {
    double best = INFINITY;
    for (int c = 0; c < K; ++c) best = fmin(best, D[(size_t)j * M + sel[c]]);
    const double thr = best + kTie * best;
    int o = 0;
    for (int c = 0; c < K; ++c)
      if (D[(size_t)j * M + sel[c]] <= thr) {
        o = c;
        break;
      }
    owner[j] = o;
  }
}

#define ST_CUDA(call)                                                              \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      rn::set_error("scenario_tree: %s failed: %s", #call, cudaGetErrorString(e_));  \
      rc = e_ == cudaErrorMemoryAllocation ? RN_ERR_NOMEM : RN_ERR_CUDA;           \
      goto done;                                                                   \
    }                                                                              \
  } while (0)

}  // namespace

extern "C" int rapidnet_scenario_tree(const double *paths, const double *prob, int S, int N,
                                      int dim, const int *branching, int device,
                                      rn_tree_out *out) {
  rn::clear_error();
  if (!paths || !branching || !out || !out->stage_ptr || !out->anc || !out->prob ||
      !out->value || !out->leaf_of || !out->rep || S < 1 || N < 1 || dim < 1) {
    rn::set_error("scenario_tree: NULL argument or a size below 1");
    return RN_ERR_INVAL;
  }
  for (int t = 0; t < N; ++t)
    if (branching[t] < 1) {
      rn::set_error("scenario_tree: branching[%d] = %d (need >= 1)", t, branching[t]);
      return RN_ERR_INVAL;
    }
  const int R = N * dim;
  std::vector<double> p(S, 1.0 / S);
  if (prob) {
    double sum = 0.0;
    for (int s = 0; s < S; ++s) {
      if (!(prob[s] >= 0.0) || !std::isfinite(prob[s])) {
        rn::set_error("scenario_tree: prob[%d] is negative or not finite", s);
        return RN_ERR_INVAL;
      }
      sum += prob[s];
    }
    if (!(std::fabs(sum - 1.0) <= 1e-9)) {
      rn::set_error("scenario_tree: the probabilities add up to %.17g, not 1", sum);
      return RN_ERR_INVAL;
    }
    p.assign(prob, prob + S);
  }
  for (size_t e = 0; e < (size_t)S * R; ++e)
    if (!std::isfinite(paths[e])) {
      rn::set_error("scenario_tree: a path value is not finite");
      return RN_ERR_INVAL;
    }
  int maxb = 1;
  for (int t = 0; t < N; ++t) maxb = std::max(maxb, branching[t]);
  int rc = RN_OK;
  double *dX = nullptr, *dD = nullptr, *dp = nullptr, *dm = nullptr, *dz = nullptr;
  int *didx = nullptr, *dch = nullptr, *dsel = nullptr, *down = nullptr;
  cudaStream_t st = nullptr;
  // breadth-first output; bundles of the current stage's nodes
  std::vector<std::vector<int>> bundles(1), next;
  std::vector<int> anc{-1}, rep{-1}, sel(maxb), owner(S);
  std::vector<double> pr{1.0}, val((size_t)dim, 0.0), pb, minit(S, INFINITY);
  std::vector<int> stage_ptr{0, 1};
  bundles[0].resize(S);
  for (int s = 0; s < S; ++s) bundles[0][s] = s;
  ST_CUDA(cudaSetDevice(device));
  ST_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  ST_CUDA(cudaMalloc(&dX, (size_t)S * R * sizeof(double)));
  ST_CUDA(cudaMalloc(&dD, (size_t)S * S * sizeof(double)));
  ST_CUDA(cudaMalloc(&dp, (size_t)S * sizeof(double)));
  ST_CUDA(cudaMalloc(&dm, (size_t)S * sizeof(double)));
  ST_CUDA(cudaMalloc(&dz, (size_t)S * sizeof(double)));
  ST_CUDA(cudaMalloc(&didx, (size_t)S * sizeof(int)));
  ST_CUDA(cudaMalloc(&dch, (size_t)S * sizeof(int)));
  ST_CUDA(cudaMalloc(&dsel, (size_t)maxb * sizeof(int)));
  ST_CUDA(cudaMalloc(&down, (size_t)S * sizeof(int)));
  ST_CUDA(cudaMemcpyAsync(dX, paths, (size_t)S * R * sizeof(double), cudaMemcpyHostToDevice, st));
  for (int t = 0; t < N; ++t) {
    next.clear();
    for (size_t off = 0; off < bundles.size(); ++off) {
      const std::vector<int> &idx = bundles[off];
      const int parent = stage_ptr[t] + (int)off, M = (int)idx.size();
      const int K = std::min(branching[t], M);
      pb.resize(M);
      for (int a = 0; a < M; ++a) pb[a] = p[idx[a]];
      ST_CUDA(cudaMemcpyAsync(didx, idx.data(), M * sizeof(int), cudaMemcpyHostToDevice, st));
      ST_CUDA(cudaMemcpyAsync(dp, pb.data(), M * sizeof(double), cudaMemcpyHostToDevice, st));
      ST_CUDA(cudaMemcpyAsync(dm, minit.data(), M * sizeof(double), cudaMemcpyHostToDevice, st));
      ST_CUDA(cudaMemsetAsync(dch, 0, M * sizeof(int), st));
      const int tiles = (M + kTile - 1) / kTile;
      k_tail_dist<<<dim3(tiles, tiles), dim3(32, 8), 0, st>>>(dX, R, didx, M, t * dim, dD);
      const int zblocks = std::min(4096, (M + 7) / 8);
      for (int k = 0; k < K; ++k) {
        k_ffs_z<<<zblocks, 256, 0, st>>>(dD, M, dp, dm, dch, dz);
        k_ffs_pick<<<1, 1024, 0, st>>>(dz, M, k, dch, dsel);
        k_ffs_update<<<std::min(1024, (M + 255) / 256), 256, 0, st>>>(dD, M, dsel, k, dm);
      }
      k_assign<<<std::min(1024, (M + 255) / 256), 256, 0, st>>>(dD, M, dsel, K, down);
      ST_CUDA(cudaGetLastError());
      ST_CUDA(cudaMemcpyAsync(sel.data(), dsel, K * sizeof(int), cudaMemcpyDeviceToHost, st));
      ST_CUDA(cudaMemcpyAsync(owner.data(), down, M * sizeof(int), cudaMemcpyDeviceToHost, st));
      ST_CUDA(cudaStreamSynchronize(st));
      for (int c = 0; c < K; ++c) {
        std::vector<int> members;
        double mass = 0.0;
        for (int a = 0; a < M; ++a)
          if (owner[a] == c) {
            members.push_back(idx[a]);
            mass += p[idx[a]];
          }
        const int r = idx[sel[c]];
        anc.push_back(parent);
        pr.push_back(mass);
        rep.push_back(r);
        for (int d = 0; d < dim; ++d) val.push_back(paths[(size_t)r * R + t * dim + d]);
        next.push_back(std::move(members));
      }
    }
    bundles.swap(next);
    stage_ptr.push_back((int)anc.size());
  }
  if ((int)anc.size() > out->max_nodes) {
    rn::set_error("scenario_tree: the tree has %d nodes, more than max_nodes = %d",
                  (int)anc.size(), out->max_nodes);
    rc = RN_ERR_INVAL;
    goto done;
  }
  out->n_nodes = (int)anc.size();
  std::copy(stage_ptr.begin(), stage_ptr.end(), out->stage_ptr);
  std::copy(anc.begin(), anc.end(), out->anc);
  std::copy(pr.begin(), pr.end(), out->prob);
  std::copy(rep.begin(), rep.end(), out->rep);
  std::copy(val.begin(), val.end(), out->value);
  for (size_t off = 0; off < bundles.size(); ++off)
    for (int s : bundles[off]) out->leaf_of[s] = stage_ptr[N] + (int)off;
done:
  if (st) cudaStreamSynchronize(st);
  for (void *q : {(void *)dX, (void *)dD, (void *)dp, (void *)dm, (void *)dz, (void *)didx,
                  (void *)dch, (void *)dsel, (void *)down})
    if (q) cudaFree(q);
  if (st) cudaStreamDestroy(st);
  return rc;
}
