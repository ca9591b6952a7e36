// Launch of the persistent solver kernel with the IC(0) preconditioner (its own translation
// unit, compiled in parallel with the others).
#include "solver.cuh"

namespace mpcg {

cudaError_t launch_cg_ic(const Launch& L, int grid, size_t smem, cudaStream_t s) {
  void* args[] = {(void*)&L};
  return cudaLaunchCooperativeKernel((const void*)cg_persistent<true>, dim3(grid), dim3(kThreads), args, smem, s);
}

cudaError_t cg_occupancy_ic(int* blocks_per_sm, size_t smem) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, cg_persistent<true>, kThreads, smem);
}

cudaError_t cg_set_smem_limit_ic(size_t bytes) {
  return cudaFuncSetAttribute(cg_persistent<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace mpcg
