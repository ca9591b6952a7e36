// Launch of the lockstep batch kernel with the IC(0) preconditioner.
#include "solver.cuh"

namespace mpcg {

cudaError_t launch_cg_lockstep_ic(const Launch& L, int grid, size_t smem, cudaStream_t s) {
  void* args[] = {(void*)&L};
  return cudaLaunchCooperativeKernel((const void*)cg_lockstep<true>, dim3(grid), dim3(kThreads), args, smem, s);
}

cudaError_t lockstep_occupancy_ic(int* blocks_per_sm, size_t smem) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, cg_lockstep<true>, kThreads, smem);
}

cudaError_t lockstep_set_smem_limit_ic(size_t bytes) {
  return cudaFuncSetAttribute(cg_lockstep<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace mpcg
