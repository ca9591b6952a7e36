// Stepped single solve: the phases of the mixed-precision CG iteration (Section 3 Eq. (1)-(4)
// with the operation precisions of Section 4.2; Algorithm 2's greedy policy between
// iterations) as one kernel launch each, repeated by a conditional while-loop CUDA graph until
// the system's phase machine is done. Used for single systems large enough that a phase
// takes far longer than a launch: every phase kernel then has its own register allocation and
// occupancy (the product kernel carries none of the other phases' live state), and the grid-
// wide barriers of the persistent kernel become kernel boundaries.
//
// Body of the loop, in order: the product kernel (phase A: q = fl_p1(A fl_p1(p)), nu partials),
// the residual kernel (phase B: r -= alpha q, ||r||^2, sigma partials), the direction kernel
// (phase C: x += alpha p, p = z + beta p, p's copy in the next product format), a kernel for the
// other phases (initialisation, p's first low copy, x-only update, residual recomputation,
// restarts, closing residual), and a one-thread control kernel. A kernel whose phase is not the
// system's current phase returns at once, so one pass through the body runs a whole ordinary
// iteration (A, B, C). In each phase kernel the CTA that finishes last (a counter, no waiting)
// sums the CTA partials in CTA order (deterministic for a given grid), runs the phase's scalar
// step (the same device code as the batched lockstep kernel: alpha, the stopping tests,
// beta, the policy, the history record) and sets the next phase. The control kernel ends the
// loop when the system is done, when the device status word is set, or after a bounded number
// of passes (then it sets the status word: no unbounded loop).
#include <cstring>

#include "solver.cuh"

namespace mpcg {
namespace {

// Arrival at the end of a phase kernel: true in the CTA that arrives last (its view of the
// other CTAs' partials is then complete). The counter (bars[0]) is reset by that CTA.
__device__ __forceinline__ bool arrive_last(const Launch& L, Smem& sm) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned old = atomicAdd(L.bars, 1u);
    sm.last = (old == gridDim.x - 1u) ? 1 : 0;
    if (sm.last) __threadfence();
  }
  __syncthreads();
  return sm.last != 0;
}

// Rows of CTA c of G: by nonzeros (product), by rows (vector phases) or by nonzeros + 3 rows
// (the mixed phases of the other kernel).
template <int PH>
__device__ __forceinline__ int stepped_row(const DevSys& S, int c, int G) {
  if (c <= 0) return 0;
  if (c >= G) return S.A.n;
  if constexpr (PH == PH_A || PH == PH_W) {
    return part_row(S.A.rp, S.A.n, S.A.nnz, c, G);
  } else if constexpr (PH == PH_B || PH == PH_C || PH == PH_U) {
    return (int)(((long long)S.A.n * c) / G);
  } else {
    return lk_row_at(S, ((S.A.nnz + 3LL * S.A.n) * c) / G);
  }
}

// PH = PH_A, PH_B, PH_C (or PH_W, PH_U of the single-reduction iteration): that phase alone;
// PH = -1: any other phase.
// At least four CTAs per SM (at most 64 registers): the phase kernels stream HBM, and the
// loads in flight per SM come from resident threads.
template <int PH>
__global__ void __launch_bounds__(kThreads, 4) cg_phase(const Launch L) {
  __shared__ Smem sm;
  extern __shared__ __align__(128) unsigned char dyn[];
  if (threadIdx.x == 0) {
    sm.lk_phase = ((const volatile SysState*)L.st)->phase;
    sm.ok = *(volatile unsigned*)L.err == 0u ? 1 : 0;
  }
  __syncthreads();
  const int ph = sm.lk_phase;
  const bool mine = PH >= 0 ? ph == PH
                            : (ph != PH_A && ph != PH_B && ph != PH_C && ph != PH_W && ph != PH_U && ph != PH_DONE);
  if (!mine || !sm.ok) return;
  const bool ring = L.stream_stage > 0 && (PH == PH_A || PH == PH_W || PH < 0);
  StreamCtx scx{dyn, sm.mbar, &sm.mbar_phase, L.err, L.stream_stage};
  if (ring) {
    if (threadIdx.x == 0) {
      mbar_init(sm.mbar + 0, 1);
      mbar_init(sm.mbar + 1, 1);
      mbar_fence_init();
      sm.mbar_phase = 0;
    }
    __syncthreads();
  }
  const DevSys& S = L.sys[0];
  if (threadIdx.x == 0) {
    sm.r0 = stepped_row<PH>(S, blockIdx.x, gridDim.x);
    sm.r1 = stepped_row<PH>(S, blockIdx.x + 1, gridDim.x);
  }
  __syncthreads();
  lk_slice_rows<false, PH>(L, 0, Rows{sm.r0, sm.r1}, blockIdx.x, sm, ring ? &scx : nullptr);
  if (!arrive_last(L, sm)) return;
  lk_step_slots<PH>(L, 0, 0, gridDim.x, sm);
  if (threadIdx.x == 0) atomicExch(L.bars, 0u);
}

// End of a pass through the loop body: continue while the system is not done. bars[16]
// counts the passes; beyond `limit` the phase machine is taken to be stuck (status word).
__global__ void cg_loop_ctrl(const Launch L, cudaGraphConditionalHandle h, unsigned limit) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  volatile unsigned* cnt = L.bars + 16;
  const unsigned c = *cnt + 1u;
  *cnt = c;
  const int ph = ((const volatile SysState*)L.st)->phase;
  const bool err = *(volatile unsigned*)L.err != 0u;
  if (!err && ph != PH_DONE && c >= limit) atomicCAS(L.err, 0u, (unsigned)DERR_BAD_STATE);
  if (ph == PH_DONE || err || c >= limit) cudaGraphSetConditional(h, 0u);
}

const void* phase_kernel(int which) {
  switch (which) {
    case 0: return (const void*)cg_phase<PH_A>;
    case 1: return (const void*)cg_phase<PH_B>;
    case 2: return (const void*)cg_phase<PH_C>;
    case 4: return (const void*)cg_phase<PH_W>;
    case 5: return (const void*)cg_phase<PH_U>;
    default: return (const void*)cg_phase<-1>;
  }
}

}  // namespace

cudaError_t stepped_occupancy(int which, int* blocks_per_sm, size_t smem) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, phase_kernel(which), kThreads, smem);
}

cudaError_t stepped_set_smem_limit(size_t bytes) {
  for (int w = 0; w < 6; ++w) {
    const cudaError_t e = cudaFuncSetAttribute(phase_kernel(w), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// One pass through the body's phase kernels launched on `s` (the host-driven form of the loop:
// the caller checks the system's phase between passes).
cudaError_t stepped_pass(const Launch& L, const int grids[kPhaseKernels], size_t smem, cudaStream_t s) {
  const int std_body[4] = {0, 1, 2, 3}, sr_body[3] = {4, 5, 3};
  const int* body_k = L.opt.variant ? sr_body : std_body;
  const int nbody = L.opt.variant ? 3 : 4;
  Launch Lc = L;
  void* args[] = {(void*)&Lc};
  for (int i = 0; i < nbody; ++i) {
    const int w = body_k[i];
    const cudaError_t e = cudaLaunchKernel(phase_kernel(w), dim3(grids[w]), dim3(kThreads), args,
                                           (w == 0 || w == 3 || w == 4) ? smem : 0, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// The graph of one stepped solve: a while-loop node whose body chains the phase kernels
// (kernels 0, 1, 2, 3 for the CG of Section 3, or 4, 5, 3 for the single-reduction iteration;
// grids[w] CTAs for kernel w, dynamic shared memory smem for the product kernels and the
// other-phases kernel when the launch uses the stream schedule) and the control kernel.
cudaError_t stepped_graph(const Launch& L, const int grids[6], size_t smem, unsigned limit, cudaGraph_t* out) {
  *out = nullptr;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return e;
  cudaGraphConditionalHandle h;
  e = cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault);
  // (the parameter struct holds a union whose default constructor is deleted: zeroed storage)
  alignas(cudaGraphNodeParams) unsigned char cpbuf[sizeof(cudaGraphNodeParams)];
  memset(cpbuf, 0, sizeof(cpbuf));
  cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cpbuf);
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cnode;
  if (e == cudaSuccess) e = cudaGraphAddNode(&cnode, g, nullptr, nullptr, 0, &cp);
  cudaGraph_t body = e == cudaSuccess ? cp.conditional.phGraph_out[0] : nullptr;
  Launch Lc = L;
  void* args[] = {(void*)&Lc};
  cudaGraphNode_t prev = nullptr;
  const int std_body[4] = {0, 1, 2, 3}, sr_body[3] = {4, 5, 3};
  const int* body_k = L.opt.variant ? sr_body : std_body;
  const int nbody = L.opt.variant ? 3 : 4;
  for (int i = 0; i < nbody && e == cudaSuccess; ++i) {
    const int w = body_k[i];
    cudaKernelNodeParams kp;
    memset(&kp, 0, sizeof(kp));
    kp.func = (void*)phase_kernel(w);
    kp.gridDim = dim3(grids[w]);
    kp.blockDim = dim3(kThreads);
    kp.sharedMemBytes = (w == 0 || w == 3 || w == 4) ? (unsigned)smem : 0u;
    kp.kernelParams = args;
    cudaGraphNode_t nd;
    e = cudaGraphAddKernelNode(&nd, body, prev ? &prev : nullptr, prev ? 1 : 0, &kp);
    prev = nd;
  }
  if (e == cudaSuccess) {
    void* cargs[] = {(void*)&Lc, (void*)&h, (void*)&limit};
    cudaKernelNodeParams kp;
    memset(&kp, 0, sizeof(kp));
    kp.func = (void*)cg_loop_ctrl;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(32);
    kp.kernelParams = cargs;
    cudaGraphNode_t nd;
    e = cudaGraphAddKernelNode(&nd, body, &prev, 1, &kp);
  }
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return e;
  }
  *out = g;
  return cudaSuccess;
}

}  // namespace mpcg
