// Launch of the persistent solver kernel without the IC(0) preconditioner, and the launch-time
// queries over every solver kernel (the lockstep kernels and the IC(0) instantiations live in
// their own translation units, compiled in parallel).
#include "solver.cuh"

namespace mpcg {

cudaError_t launch_cg(const Launch& L, int grid, size_t smem, cudaStream_t s) {
  if (L.ic) return launch_cg_ic(L, grid, smem, s);
  void* args[] = {(void*)&L};
  return cudaLaunchCooperativeKernel((const void*)cg_persistent<false>, dim3(grid), dim3(kThreads), args, smem, s);
}

// Resident CTAs per SM of the solver kernels (the smallest over all of them, so that one grid
// size serves every launch).
cudaError_t cg_occupancy(int* blocks_per_sm, size_t smem) {
  int best = 0, a = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&best, cg_persistent<false>, kThreads, smem);
  if (e != cudaSuccess) return e;
  cudaError_t (*others[3])(int*, size_t) = {cg_occupancy_ic, lockstep_occupancy, lockstep_occupancy_ic};
  for (auto f : others) {
    e = f(&a, smem);
    if (e != cudaSuccess) return e;
    best = a < best ? a : best;
  }
  *blocks_per_sm = best;
  return cudaSuccess;
}

cudaError_t cg_set_smem_limit(size_t bytes) {
  cudaError_t e = cudaFuncSetAttribute(cg_persistent<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  cudaError_t (*others[3])(size_t) = {cg_set_smem_limit_ic, lockstep_set_smem_limit, lockstep_set_smem_limit_ic};
  for (auto f : others) {
    e = f(bytes);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

size_t cg_static_smem() { return sizeof(Smem); }

}  // namespace mpcg
