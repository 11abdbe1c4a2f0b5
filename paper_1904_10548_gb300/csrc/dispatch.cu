// Run-time choice of the kernel instantiation (components per thread C)
// and the launch helpers of the persistent kernels.
#include <mutex>
#include <set>

#include "kernels.cuh"

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

// dense: the instantiation for a dense W_u (F as a dense product)
static const void *solve_kernel(int c, bool apg, bool dense) {
  switch (c) {
    case 1: return dense ? solve_kernel_c1_d1(apg) : solve_kernel_c1_d0(apg);
    case 2: return dense ? solve_kernel_c2_d1(apg) : solve_kernel_c2_d0(apg);
    case 4: return dense ? solve_kernel_c4_d1(apg) : solve_kernel_c4_d0(apg);
    default: return dense ? solve_kernel_c8_d1(apg) : solve_kernel_c8_d0(apg);
  }
}
static const void *mixed_kernel(int c, bool dense) {
  switch (c) {
    case 1: return dense ? mixed_kernel_c1_d1() : mixed_kernel_c1_d0();
    case 2: return dense ? mixed_kernel_c2_d1() : mixed_kernel_c2_d0();
    case 4: return dense ? mixed_kernel_c4_d1() : mixed_kernel_c4_d0();
    default: return dense ? mixed_kernel_c8_d1() : mixed_kernel_c8_d0();
  }
}
static const void *batch_kernel(int c) {
  switch (c) {
    case 1: return batch_kernel_c1();
    case 2: return batch_kernel_c2();
    case 4: return batch_kernel_c4();
    default: return batch_kernel_c8();
  }
}

static cudaError_t launch_coop(const void *fn, void *arg, int grid, int block, size_t smem,
                               cudaStream_t st) {
  cudaError_t e = allow_max_smem(fn);
  if (e != cudaSuccess) return e;
  void *args[] = {arg};
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(block), args, smem, st);
}

static cudaError_t occupancy(const void *fn, int block, size_t smem, int *blocks_per_sm) {
  cudaError_t e = allow_max_smem(fn);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, block, smem);
}

template <typename T, bool APG>
cudaError_t launch_solve(const KParams<T> &P, int grid, int block, size_t smem, cudaStream_t st) {
  KParams<T> p = P;
  return launch_coop(solve_kernel(P.maxc, APG, P.net.Fd != nullptr), &p, grid, block, smem, st);
}

template <typename T, bool APG>
cudaError_t solve_occupancy(int maxc, bool dense, int block, size_t smem, int *blocks_per_sm) {
  return occupancy(solve_kernel(maxc, APG, dense), block, smem, blocks_per_sm);
}

template cudaError_t launch_solve<double, true>(const KParams<double> &, int, int, size_t, cudaStream_t);
template cudaError_t launch_solve<double, false>(const KParams<double> &, int, int, size_t, cudaStream_t);
template cudaError_t solve_occupancy<double, true>(int, bool, int, size_t, int *);
template cudaError_t solve_occupancy<double, false>(int, bool, int, size_t, int *);

cudaError_t launch_mixed(const MixedParams &M, int maxc, int grid, int block, size_t smem,
                         cudaStream_t st) {
  MixedParams p = M;
  return launch_coop(mixed_kernel(maxc, M.f.net.Fd != nullptr), &p, grid, block, smem, st);
}

cudaError_t mixed_occupancy(int maxc, bool dense, int block, size_t smem, int *blocks_per_sm) {
  return occupancy(mixed_kernel(maxc, dense), block, smem, blocks_per_sm);
}

cudaError_t launch_batch(const BatchDev &B, int maxc, int grid, int block, size_t smem,
                         cudaStream_t st) {
  BatchDev b = B;
  return launch_coop(batch_kernel(maxc), &b, grid, block, smem, st);
}

cudaError_t batch_occupancy(int maxc, int block, size_t smem, int *blocks_per_sm) {
  return occupancy(batch_kernel(maxc), block, smem, blocks_per_sm);
}

cudaError_t batch_static_smem(int maxc, int *bytes) {
  cudaFuncAttributes fa{};
  cudaError_t e = cudaFuncGetAttributes(&fa, batch_kernel(maxc));
  if (e == cudaSuccess) *bytes = (int)fa.sharedSizeBytes;
  return e;
}

}  // namespace rn
