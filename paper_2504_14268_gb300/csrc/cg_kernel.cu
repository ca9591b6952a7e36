// Launches of the solver kernels without the IC(0) preconditioner, and the launch-time
// queries over both instantiations (the IC(0) ones live in cg_kernel_ic.cu).
#include "solver.cuh"

namespace mpcg {

cudaError_t launch_cg(const Launch& L, int grid, size_t smem, cudaStream_t s) {
  if (L.ic) return launch_cg_ic(L, grid, smem, s);
  void* args[] = {(void*)&L};
  return cudaLaunchCooperativeKernel((const void*)cg_persistent<false>, dim3(grid), dim3(kThreads), args, smem, s);
}

cudaError_t launch_cg_lockstep(const Launch& L, int grid, size_t smem, cudaStream_t s) {
  if (L.ic) return launch_cg_lockstep_ic(L, grid, smem, s);
  void* args[] = {(void*)&L};
  return cudaLaunchCooperativeKernel((const void*)cg_lockstep<false>, dim3(grid), dim3(kThreads), args, smem, s);
}

// Resident CTAs per SM of the solver kernels (the smallest over all of them, so that one grid
// size serves every launch).
cudaError_t cg_occupancy(int* blocks_per_sm, size_t smem) {
  int best = 0;
  cudaError_t e = cg_occupancy_ic(&best, smem);
  if (e != cudaSuccess) return e;
  const void* ks[2] = {(const void*)cg_persistent<false>, (const void*)cg_lockstep<false>};
  for (const void* k : ks) {
    int a = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k, kThreads, smem);
    if (e != cudaSuccess) return e;
    best = a < best ? a : best;
  }
  *blocks_per_sm = best;
  return cudaSuccess;
}

cudaError_t cg_set_smem_limit(size_t bytes) {
  const void* ks[2] = {(const void*)cg_persistent<false>, (const void*)cg_lockstep<false>};
  for (const void* k : ks) {
    const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
  }
  return cg_set_smem_limit_ic(bytes);
}

size_t cg_static_smem() { return sizeof(Smem); }

}  // namespace mpcg
