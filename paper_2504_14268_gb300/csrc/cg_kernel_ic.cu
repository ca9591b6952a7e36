// Launches of the solver kernels with the IC(0) preconditioner (their own translation unit,
// compiled in parallel with cg_kernel.cu).
#include "solver.cuh"

namespace mpcg {

cudaError_t launch_cg_ic(const Launch& L, int grid, size_t smem, cudaStream_t s) {
  void* args[] = {(void*)&L};
  return cudaLaunchCooperativeKernel((const void*)cg_persistent<true>, dim3(grid), dim3(kThreads), args, smem, s);
}

cudaError_t launch_cg_lockstep_ic(const Launch& L, int grid, size_t smem, cudaStream_t s) {
  void* args[] = {(void*)&L};
  return cudaLaunchCooperativeKernel((const void*)cg_lockstep<true>, dim3(grid), dim3(kThreads), args, smem, s);
}

cudaError_t cg_occupancy_ic(int* blocks_per_sm, size_t smem) {
  int a = 0, b = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, cg_persistent<true>, kThreads, smem);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, cg_lockstep<true>, kThreads, smem);
  if (e != cudaSuccess) return e;
  *blocks_per_sm = a < b ? a : b;
  return cudaSuccess;
}

cudaError_t cg_set_smem_limit_ic(size_t bytes) {
  cudaError_t e = cudaFuncSetAttribute(cg_persistent<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(cg_lockstep<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace mpcg
