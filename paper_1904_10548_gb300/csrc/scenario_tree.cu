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
// chosen on ties).
//
// The bundles of a stage partition the paths, so a stage is processed with
// one set of launches over all its bundles: the paths in bundle order
// (pos[], offsets boff[]), every bundle's distance matrix at doff[] in one
// array (sum of M_b^2 <= S^2 doubles).
//   k_tail_dist  the distance matrices (FP64, tiles of 32 x 32 pairs from a
//                tile table of the upper triangle, each tile written with
//                its mirror; the tails staged through shared memory);
//   k_ffs_z      z for every candidate of every bundle still choosing: a
//                block reads the rows of four candidates of its bundle's
//                matrix (it is symmetric) with the weights and the current
//                minima: the matrices stream from HBM once per choice, the
//                bound of this step;
//   k_ffs_pick   one block per bundle: the smallest z, then the first
//                candidate within the tie tolerance;
//   k_ffs_update m_j = min(m_j, d(j, chosen));
//   k_assign     each path's nearest representative.
// The host keeps the bundles (index lists) and writes the tree in
// breadth-first order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "rn_internal.h"

namespace {

constexpr int kTile = 32;
// values within kTie (relative) of the smallest count as ties: they are real
// (in one dimension the median of an even number of paths is an interval),
// and sums added in different orders must still take the same decision
constexpr double kTie = 1e-12;

// one stage's bundles on the device
struct StageDev {
  const int *pos;        // S: path of each position, bundle by bundle
  const int *boff;       // B + 1: first position of each bundle
  const long long *doff; // B: first entry of each bundle's distance matrix
  const int *bundle_of;  // S: bundle of each position
  const int *K;          // B: representatives the bundle chooses
  int B;
};

// D_b[a][c] = || X[pos[a], c0:] - X[pos[c], c0:] || for the pairs of one
// 32 x 32 tile and its mirror (tile table: bundle, tile row, tile column,
// row <= column); X is S x R.  The differences are squared exactly alike
// either way round, so D_b is symmetric bit for bit.
__global__ void k_tail_dist(const double *X, int R, StageDev sd, const int4 *tiles, int c0,
                            double *D) {
  __shared__ double A[kTile][kTile + 1], Bt[kTile][kTile + 1];
  const int4 tl = tiles[blockIdx.x];
  const int b = tl.x, first = sd.boff[b], M = sd.boff[b + 1] - first;
  const int a0 = tl.y * kTile, b0 = tl.z * kTile;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8 threads
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int c = c0; c < R; c += kTile) {
    for (int r = ty; r < kTile; r += 8) {
      const int a = a0 + r, e = b0 + r, col = c + tx;
      A[r][tx] = (a < M && col < R) ? X[(size_t)sd.pos[first + a] * R + col] : 0.0;
      Bt[r][tx] = (e < M && col < R) ? X[(size_t)sd.pos[first + e] * R + col] : 0.0;
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
  // the tile, then (off the diagonal) its mirror: the table holds the tiles
  // with tile row <= tile column only, D being symmetric
  double *Db = D + sd.doff[b];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int r = ty + 8 * q, a = a0 + r, e = b0 + tx;
    const double d = sqrt(acc[q]);
    if (a < M && e < M) Db[(size_t)a * M + e] = d;
    A[r][tx] = d;
  }
  if (tl.y == tl.z) return;
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int r = ty + 8 * q, e = b0 + r, a = a0 + tx;
    if (e < M && a < M) Db[(size_t)e * M + a] = A[tx][r];
  }
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

constexpr int kZRows = 4, kZThreads = 256;  // candidates and threads per block of k_ffs_z

// choice k: z[u] = sum_j p_j min(m_j, D_b[u][j]) for every position u of a
// bundle with k < K_b (a chosen one gets +inf).  One block takes kZRows
// consecutive positions and splits the columns over its threads: when the
// positions share a bundle their rows stream together, with p and m read
// once for all of them.
__global__ void __launch_bounds__(kZThreads)
    k_ffs_z(const double *D, StageDev sd, int S, int k, const double *p, const double *m,
            const int *chosen, double *z) {
  __shared__ double red[kZThreads / 32][kZRows];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int groups = (S + kZRows - 1) / kZRows;
  for (int g = blockIdx.x; g < groups; g += gridDim.x) {
    const int u0 = g * kZRows, nr = min(kZRows, S - u0);
    const int b0 = sd.bundle_of[u0];
    const bool one = sd.bundle_of[u0 + nr - 1] == b0;  // bundles are contiguous
    if (one && k >= sd.K[b0]) continue;                 // the same for the whole block
    double acc[kZRows];
#pragma unroll
    for (int r = 0; r < kZRows; ++r) acc[r] = 0.0;
    if (one) {
      const int first = sd.boff[b0], M = sd.boff[b0 + 1] - first;
      const double *row = D + sd.doff[b0] + (size_t)(u0 - first) * M;
      const double *pb = p + first, *mb = m + first;
      for (int j = threadIdx.x; j < M; j += kZThreads) {
        const double pj = pb[j], mj = mb[j];
#pragma unroll
        for (int r = 0; r < kZRows; ++r)
          if (r < nr) acc[r] += pj * fmin(mj, __ldcs(row + (size_t)r * M + j));
      }
    } else {
#pragma unroll
      for (int r = 0; r < kZRows; ++r) {
        const int u = u0 + r;
        if (r >= nr) continue;
        const int b = sd.bundle_of[u];
        if (k >= sd.K[b]) continue;
        const int first = sd.boff[b], M = sd.boff[b + 1] - first;
        const double *row = D + sd.doff[b] + (size_t)(u - first) * M;
        for (int j = threadIdx.x; j < M; j += kZThreads)
          acc[r] += p[first + j] * fmin(m[first + j], __ldcs(row + j));
      }
    }
#pragma unroll
    for (int r = 0; r < kZRows; ++r) {
      const double v = warp_sum_d(acc[r]);
      if (lane == 0) red[w][r] = v;
    }
    __syncthreads();
    if (threadIdx.x < nr) {
      const int u = u0 + threadIdx.x;
      if (k < sd.K[sd.bundle_of[u]]) {
        double v = 0.0;
        for (int q = 0; q < kZThreads / 32; ++q) v += red[q][threadIdx.x];
        z[u] = chosen[u] ? INFINITY : v;
      }
    }
    __syncthreads();
  }
}

// one block per bundle with k < K_b: the first candidate within kTie of the
// smallest z becomes choice k (sel[b * kmax + k], a position in the bundle)
__global__ void k_ffs_pick(const double *z, StageDev sd, int k, int kmax, int *chosen, int *sel) {
  __shared__ double red[32];
  __shared__ int ired[32];
  const int b = blockIdx.x;
  if (k >= sd.K[b]) return;
  const int first = sd.boff[b], M = sd.boff[b + 1] - first;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double lo = INFINITY;
  for (int a = threadIdx.x; a < M; a += blockDim.x) lo = fmin(lo, z[first + a]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
  if (lane == 0) red[w] = lo;
  __syncthreads();
  lo = red[0];
  for (int q = 1; q < nw; ++q) lo = fmin(lo, red[q]);
  const double thr = lo + kTie * fabs(lo);
  int fa = M;
  for (int a = threadIdx.x; a < M; a += blockDim.x)
    if (z[first + a] <= thr) {
      fa = a;
      break;
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) fa = min(fa, __shfl_xor_sync(0xffffffffu, fa, o));
  if (lane == 0) ired[w] = fa;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 0; q < nw; ++q) fa = min(fa, ired[q]);
    if (fa >= M) fa = 0;  // every candidate chosen (not reached: k < K_b <= M)
    sel[b * kmax + k] = fa;
    chosen[first + fa] = 1;
  }
}

// choice k: m_j = min(m_j, D_b[sel_b][j]) for the positions of bundles with k < K_b
__global__ void k_ffs_update(const double *D, StageDev sd, int S, int k, int kmax,
                             const int *sel, double *m) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < S; j += gridDim.x * blockDim.x) {
    const int b = sd.bundle_of[j];
    if (k >= sd.K[b]) continue;
    const int first = sd.boff[b], M = sd.boff[b + 1] - first;
    m[j] = fmin(m[j], D[sd.doff[b] + (size_t)sel[b * kmax + k] * M + (j - first)]);
  }
}

// owner[j] = the first chosen representative within kTie of the nearest
__global__ void k_assign(const double *D, StageDev sd, int S, int kmax, const int *sel,
                         int *owner) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < S; j += gridDim.x * blockDim.x) {
    const int b = sd.bundle_of[j], K = sd.K[b];
    const int first = sd.boff[b], M = sd.boff[b + 1] - first, a = j - first;
    const double *Db = D + sd.doff[b] + (size_t)a * M;
    double best = INFINITY;
    for (int c = 0; c < K; ++c) best = fmin(best, Db[sel[b * kmax + c]]);
    const double thr = best + kTie * best;
    int o = 0;
    for (int c = 0; c < K; ++c)
      if (Db[sel[b * kmax + c]] <= thr) {
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
  int rc = RN_OK;
  double *dX = nullptr, *dD = nullptr, *dp = nullptr, *dm = nullptr, *dz = nullptr;
  int *dpos = nullptr, *dboff = nullptr, *dbof = nullptr, *dK = nullptr, *dch = nullptr;
  int *dsel = nullptr, *down = nullptr;
  long long *ddoff = nullptr;
  int4 *dtiles = nullptr;
  size_t tiles_cap = 0;
  cudaStream_t st = nullptr;
  // breadth-first output; the bundles of the current stage's nodes
  std::vector<std::vector<int>> bundles(1), next;
  std::vector<int> anc{-1}, rep{-1}, stage_ptr{0, 1};
  std::vector<double> pr{1.0}, val((size_t)dim, 0.0);
  std::vector<int> pos(S), boff, bof(S), Kb, sel, owner(S);
  std::vector<long long> doff;
  std::vector<int4> tiles;
  std::vector<double> pb(S), minit(S, INFINITY);
  bundles[0].resize(S);
  for (int s = 0; s < S; ++s) bundles[0][s] = s;
  int maxb = 1;
  for (int t = 0; t < N; ++t) maxb = std::max(maxb, branching[t]);
  ST_CUDA(cudaSetDevice(device));
  ST_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  ST_CUDA(cudaMalloc(&dX, (size_t)S * R * sizeof(double)));
  ST_CUDA(cudaMalloc(&dD, (size_t)S * S * sizeof(double)));
  ST_CUDA(cudaMalloc(&dp, (size_t)S * sizeof(double)));
  ST_CUDA(cudaMalloc(&dm, (size_t)S * sizeof(double)));
  ST_CUDA(cudaMalloc(&dz, (size_t)S * sizeof(double)));
  ST_CUDA(cudaMalloc(&dpos, (size_t)S * sizeof(int)));
  ST_CUDA(cudaMalloc(&dboff, (size_t)(S + 1) * sizeof(int)));
  ST_CUDA(cudaMalloc(&dbof, (size_t)S * sizeof(int)));
  ST_CUDA(cudaMalloc(&dK, (size_t)S * sizeof(int)));
  ST_CUDA(cudaMalloc(&ddoff, (size_t)S * sizeof(long long)));
  ST_CUDA(cudaMalloc(&dch, (size_t)S * sizeof(int)));
  ST_CUDA(cudaMalloc(&dsel, (size_t)S * maxb * sizeof(int)));
  ST_CUDA(cudaMalloc(&down, (size_t)S * sizeof(int)));
  ST_CUDA(cudaMemcpyAsync(dX, paths, (size_t)S * R * sizeof(double), cudaMemcpyHostToDevice, st));
  for (int t = 0; t < N; ++t) {
    // the stage's bundles in order: positions, offsets, matrices, tiles
    const int B = (int)bundles.size(), kmax = branching[t];
    boff.assign(B + 1, 0);
    doff.assign(B, 0);
    Kb.assign(B, 0);
    tiles.clear();
    long long dsum = 0;
    for (int b = 0; b < B; ++b) {
      const int M = (int)bundles[b].size(), f = boff[b];
      boff[b + 1] = f + M;
      doff[b] = dsum;
      dsum += (long long)M * M;
      Kb[b] = std::min(kmax, M);
      for (int a = 0; a < M; ++a) {
        pos[f + a] = bundles[b][a];
        bof[f + a] = b;
        pb[f + a] = p[bundles[b][a]];
      }
      const int nt = (M + kTile - 1) / kTile;
      for (int i = 0; i < nt; ++i)
        for (int j = i; j < nt; ++j) tiles.push_back(make_int4(b, i, j, 0));
    }
    if (tiles.size() > tiles_cap) {
      if (dtiles) cudaFree(dtiles);
      dtiles = nullptr;
      tiles_cap = tiles.size();
      ST_CUDA(cudaMalloc(&dtiles, tiles_cap * sizeof(int4)));
    }
    ST_CUDA(cudaMemcpyAsync(dpos, pos.data(), S * sizeof(int), cudaMemcpyHostToDevice, st));
    ST_CUDA(cudaMemcpyAsync(dboff, boff.data(), (B + 1) * sizeof(int), cudaMemcpyHostToDevice, st));
    ST_CUDA(cudaMemcpyAsync(dbof, bof.data(), S * sizeof(int), cudaMemcpyHostToDevice, st));
    ST_CUDA(cudaMemcpyAsync(dK, Kb.data(), B * sizeof(int), cudaMemcpyHostToDevice, st));
    ST_CUDA(cudaMemcpyAsync(ddoff, doff.data(), B * sizeof(long long), cudaMemcpyHostToDevice, st));
    ST_CUDA(cudaMemcpyAsync(dp, pb.data(), S * sizeof(double), cudaMemcpyHostToDevice, st));
    ST_CUDA(cudaMemcpyAsync(dm, minit.data(), S * sizeof(double), cudaMemcpyHostToDevice, st));
    ST_CUDA(cudaMemcpyAsync(dtiles, tiles.data(), tiles.size() * sizeof(int4),
                            cudaMemcpyHostToDevice, st));
    ST_CUDA(cudaMemsetAsync(dch, 0, S * sizeof(int), st));
    const StageDev sd{dpos, dboff, ddoff, dbof, dK, B};
    k_tail_dist<<<(unsigned)tiles.size(), dim3(32, 8), 0, st>>>(dX, R, sd, dtiles, t * dim, dD);
    const int zblocks = std::min(1 << 16, (S + kZRows - 1) / kZRows), eblocks = std::min(2048, (S + 255) / 256);
    for (int k = 0; k < kmax; ++k) {
      k_ffs_z<<<zblocks, kZThreads, 0, st>>>(dD, sd, S, k, dp, dm, dch, dz);
      k_ffs_pick<<<B, 1024, 0, st>>>(dz, sd, k, kmax, dch, dsel);
      k_ffs_update<<<eblocks, 256, 0, st>>>(dD, sd, S, k, kmax, dsel, dm);
    }
    k_assign<<<eblocks, 256, 0, st>>>(dD, sd, S, kmax, dsel, down);
    ST_CUDA(cudaGetLastError());
    sel.resize((size_t)B * kmax);
    ST_CUDA(cudaMemcpyAsync(sel.data(), dsel, (size_t)B * kmax * sizeof(int),
                            cudaMemcpyDeviceToHost, st));
    ST_CUDA(cudaMemcpyAsync(owner.data(), down, S * sizeof(int), cudaMemcpyDeviceToHost, st));
    ST_CUDA(cudaStreamSynchronize(st));
    // the children, bundle by bundle in the order of their choices
    next.clear();
    for (int b = 0; b < B; ++b) {
      const int f = boff[b], M = boff[b + 1] - f, parent = stage_ptr[t] + b;
      for (int c = 0; c < Kb[b]; ++c) {
        std::vector<int> members;
        double mass = 0.0;
        for (int a = 0; a < M; ++a)
          if (owner[f + a] == c) {
            members.push_back(pos[f + a]);
            mass += p[pos[f + a]];
          }
        const int r = pos[f + sel[(size_t)b * kmax + c]];
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
  for (void *q : {(void *)dX, (void *)dD, (void *)dp, (void *)dm, (void *)dz, (void *)dpos,
                  (void *)dboff, (void *)dbof, (void *)dK, (void *)ddoff, (void *)dch,
                  (void *)dsel, (void *)down, (void *)dtiles})
    if (q) cudaFree(q);
  if (st) cudaStreamDestroy(st);
  return rc;
}
