// Launch of the lockstep batch kernel without the IC(0) preconditioner.
#include "solver.cuh"

namespace mpcg {

cudaError_t launch_cg_lockstep(const Launch& L, int grid, size_t smem, cudaStream_t s) {
  if (L.ic) return launch_cg_lockstep_ic(L, grid, smem, s);
  void* args[] = {(void*)&L};
  return cudaLaunchCooperativeKernel((const void*)cg_lockstep<false>, dim3(grid), dim3(kThreads), args, smem, s);
}

cudaError_t lockstep_occupancy(int* blocks_per_sm, size_t smem) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, cg_lockstep<false>, kThreads, smem);
}

cudaError_t lockstep_set_smem_limit(size_t bytes) {
  return cudaFuncSetAttribute(cg_lockstep<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace mpcg
