// Internal layouts shared by the host runtime (api.cu) and the kernels (cg_kernel.cu,
// setup_kernels.cu). Not part of the C ABI.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "mpcg.h"
#include "formats.cuh"

namespace mpcg {

constexpr int kThreads = 256;       // threads per CTA of every kernel
constexpr int kMaxRBins = 32;       // residual bins supported by the device policy
constexpr int kMaxBBins = 64;       // iteration bins
constexpr int kNSlot = 8;           // partial sums per CTA and phase
constexpr int kNFeat = 16;          // MLP input features
constexpr int kMaxHidden = 128;     // MLP hidden width bound
constexpr int kBarStride = 32;      // uint32 words between team barriers (128 bytes)
constexpr int kStageBytes = 24 * 1024;  // one stage of the stream schedule's shared-memory ring

enum Sched : int { SCHED_VECTOR = 0, SCHED_STREAM = 1, SCHED_VLOAD = 2, SCHED_MERGE = 3, SCHED_XSTAGE = 4 };

// Device view of a matrix: CSR structure plus the value copy of every format.
struct DevMatrix {
  int n;
  int pad0;
  long long nnz;
  const int* rp;
  const int* ci;
  const double* v64;
  const float* v32;
  const float* vtf;
  const __half* v16;
  const __nv_bfloat16* vbf;
  const __half* v16r;
  const __nv_bfloat16* vbfr;
  const q52_t* v8;          // q52 values (Table 1's quarter precision)
  const short* rexp;        // e_i of the row scales s_i = 2^e_i of the row-scaled formats
  int sched[8];             // SpMV schedule per format
  int lanes[8];             // lanes per row per format
  int tile_rows[8];         // stream schedule: rows per shared-memory tile (kThreads / lanes)
  int tile_bytes[8];        // stream schedule: bytes of a stage's value region (columns follow)
  int cols_sorted;          // every row's column indices strictly increase
  const double* dinv;       // Jacobi: 1 / a_ii in fp64 when the launch preconditions, else nullptr
  const float* icf;         // IC(0) factor in fp32 when the launch preconditions with it, else
                            // nullptr: l_ij at (i, j) for j <= i, l_ji at (i, j) for j > i
  const int* icd;           // IC(0): position of the diagonal entry of each row
  const int* icpf;          // IC(0): the rows sorted by level of L y = r (level 0 first), then
  const int* icpb;          // ... of L^T w = y; a row's level is 1 + the largest level of the rows
  int icwf, icwb;           // its sum reads (0 if none); icw*: the widest level's row count
  const int* icof;          // IC(0): start of each level in icpf (nlevf + 1 entries), then
  const int* icob;          // ... in icpb (nlevb + 1 entries)
  int nlevf, nlevb;
};

// One transition of an exploration episode (Algorithm 1), recorded for the end-of-round merge.
struct Transition {
  int s, s_next;
  int act[4];
  double reward;
  int terminal, pad;
};

// One system of a launch: matrix, right-hand side, solution, work vectors, limits.
struct DevSys {
  DevMatrix A;
  const double* b;
  double* x;
  double* r;
  double* p;
  void* plow;               // p in the product's input format (fp32 / tf32 / fp16 / bf16)
  void* q;                  // q = A p in the product's format
  double tol;
  int max_iter;
  int lane;                 // index of the system in its batch
  mpcg_iter_record* hist;   // device array or nullptr
  int hist_cap;
  int pad1;
  double* Qpriv;            // training: lane-private copy of the tables
  Transition* trans;        // training: transitions of this lane's episode
  int trans_cap;
  int pad2;
  float feat_static[5];     // MLP static features of the matrix
  int feat_cap;             // capacity of feat_log in feature vectors
  float* feat_log;          // when set: the 16 features of every visited state, [k][16]
  unsigned long long* icw;  // IC(0): the substitutions' work vector [n], per row the fp32 value
                            // (y_i, then w_i = (M^-1 r)_i) in the low word and its mark above
  double* sv;               // single-reduction iteration: s = A p by recurrence (nullptr otherwise);
                            // plow then holds u = fl_p2(M^-1 r) in the product's format, fp64 included
};

// Per-system state that persists across phases; written only by the CTA that arrives
// last at a team barrier, read by every CTA of the team after the barrier.
struct SysState {
  double alpha, beta, nu, sigma, rho, bnorm, rho_true;
  double rho_hist[9];
  double alpha_prev, beta_prev, gap_log;
  double rew;
  int k, mode, outcome, iters;
  int fmt[4];
  int act[4];
  int prev_act[4];
  int have_prev, n_true, ntrans, true_known;
  int explored, s_cur;      // exploration flag and state index of the current iteration
  int zfmt;                 // p2 of the iteration whose direction update is pending
  int phase;                // lockstep batches: the phase the system runs next (0 = initialisation)
  unsigned icep;            // phases completed since initialisation: the IC(0) marks' epoch
  int fp64_lock, n_restart;   // after a breakdown restart every operation runs in fp64
  unsigned long long t_last;  // globaltimer at the previous team barrier
  unsigned ns_a, ns_b;        // phase times of the current iteration
  int near_edge, pad_ne;      // greedy tabular decisions taken near a residual-bin edge
  double sr_gamma, sr_alpha;  // single-reduction iteration: gamma and alpha of the last iteration
  int restart_sr;             // single-reduction iteration: 1 = the next iteration restarts (beta = 0)
  int wfmt;                   // single-reduction iteration: product format of the finished iteration
  long long counts[4][8];
};

struct PolicyView {
  int kind;                 // 0 fixed, 1 schedule, 2 qtable, 3 mlp
  int fixed[4];
  int sched_len;
  const int* sched;         // [len][4] format codes
  const double* Q;          // [4][S][nprec]
  const int* visits;        // [4][S] or nullptr
  const float* mlp;         // flat parameters
  int H;
  int pad;
};

struct OptView {
  int b_bins, r_bins, t_width, min_k;
  int nprec;
  int precs[8];
  double cost[8];
  double thr[kMaxRBins];    // residual-bin thresholds theta_m = 10^(-m delta), m = 1..r-1
  double log_cap;           // -log10(eps_min)
  double eps_min;
  double w1, w2, w3, lr, gamma;
  unsigned long long seed;
  int fallback_fmt;         // unvisited-row action (format code), -1 = argmax
  int fallback_idx;         // its index in precs (-1 if absent)
  int true_every, true_at_conv, warm_start, t_bin;
  int on_breakdown, precond;
  int op_mask[4];           // allowed action indices per operation (all bits set = no restriction)
  double edge_tol;          // relative distance to a residual-bin threshold counted as near an edge
  int variant;              // 0: the CG of Section 3; 1: the single-reduction iteration
  int joint;                // 1: one Q-table over the joint actions ([S][nprec^4], visits [S])
};

// Arguments of one launch of the persistent kernel.
struct Launch {
  const DevSys* sys;
  SysState* st;
  int nsys;
  int nteams;
  const int* cta_team;      // [grid] team of each CTA
  const int* cta_rank;      // [grid] rank of each CTA inside its team
  const int* team_size;     // [nteams]
  const int* team_first;    // [nteams] first CTA of the team
  const int* team_sys_off;  // [nteams + 1] offsets into team_sys
  const int* team_sys;      // systems of each team, solved in this order
  unsigned* bars;           // [nteams * kBarStride]: count at +0, generation at +16
  double* partials;         // [grid * kNSlot]
  mpcg_result* res;         // [nsys]
  unsigned* err;            // device status word (0 = fine)
  PolicyView pol;
  OptView opt;
  int train;                // 1: epsilon-greedy episode with online private updates
  int stream_stage;         // bytes of one stage of the stream ring (0: no stream schedule)
  unsigned long long episode;
  double eps;
  long long timeout_cycles;
  // Lockstep batches (lockstep != 0): at every super-step each CTA works on a slice of every
  // active system, the slices re-cut whenever systems finish.
  int lockstep;
  int ic;                   // IC(0) preconditioning: the solver kernels' IC instantiations run
  const long long* lk_w;    // [nsys] row work of each system: nnz + 3 n (at least 1)
  long long* lk_pref;       // [nsys + 1] prefix of the work of the active systems
  int* lk_cfirst;           // [nsys] first CTA holding rows of the system (-1: finished)
  int* lk_clast;            // [nsys] last such CTA
  int* lk_base;             // [nsys] partial slot of the system's first slice
  int* lk_done;             // number of finished systems
  int4* lk_seg;             // [grid][nsys + 1] slices of each CTA: (system, r0, r1, partial slot)
  int* lk_nseg;             // [grid] number of slices of each CTA
};

// max over the entries a of a Q-table row that bit a of `mask` allows (the bootstrap term
// of the Section 4.1 update over an operation's customised precision set).
__device__ __forceinline__ double row_max_allowed(const double* row, int n, unsigned mask) {
  double m = -__longlong_as_double(0x7ff0000000000000ll);
  for (int a = 0; a < n; ++a)
    if (((mask >> a) & 1u) && row[a] > m) m = row[a];
  return m;
}

// Joint actions (one Q-table over the four operations' formats, the |P|^4 alternative of
// Section 4.1): a = ((a_1 P + a_2) P + a_3) P + a_4 is allowed when each a_j is in operation
// j's set (bit a_j of m[j]).
template <class MT>
__device__ __forceinline__ bool joint_allowed(int a, int P, const MT* m) {
  for (int j = 3; j >= 0; --j) {
    if (!(((unsigned)m[j] >> (a % P)) & 1u)) return false;
    a /= P;
  }
  return true;
}

// max over the allowed joint actions of a joint row (the bootstrap term of the update).
template <class MT>
__device__ __forceinline__ double joint_row_max(const double* row, int P, const MT* m) {
  double mx = -__longlong_as_double(0x7ff0000000000000ll);
  const int n = P * P * P * P;
  for (int a = 0; a < n; ++a)
    if (joint_allowed(a, P, m) && row[a] > mx) mx = row[a];
  return mx;
}

// Device status word values.
enum DevErr : unsigned { DERR_NONE = 0, DERR_TIMEOUT = 1, DERR_BAD_STATE = 2 };

// Host entry points of the kernels (cg_kernel.cu, setup_kernels.cu).
cudaError_t launch_cg(const Launch& L, int grid, size_t smem, cudaStream_t s);
cudaError_t launch_cg_lockstep(const Launch& L, int grid, size_t smem, cudaStream_t s);
// Stepped single solve (stepped.cu): kernels 0..3 are the product, residual, direction and
// other-phases kernels, 4 and 5 the single-reduction iteration's product and update kernels;
// the graph repeats them (grids[w] CTAs each, smem bytes of dynamic shared memory for the
// product kernels and kernel 3) until the system is done or `limit` passes ran.
constexpr int kPhaseKernels = 6;
constexpr int kPhaseDone = 10;  // the phase machine's final phase (PH_DONE in solver.cuh)
cudaError_t stepped_occupancy(int which, int* blocks_per_sm, size_t smem);
cudaError_t stepped_set_smem_limit(size_t bytes);
cudaError_t stepped_graph(const Launch& L, const int grids[kPhaseKernels], size_t smem, unsigned limit,
                          cudaGraph_t* out);
cudaError_t stepped_pass(const Launch& L, const int grids[kPhaseKernels], size_t smem, cudaStream_t s);
// the IC(0) instantiations (cg_kernel_ic.cu)
cudaError_t launch_cg_ic(const Launch& L, int grid, size_t smem, cudaStream_t s);
cudaError_t launch_cg_lockstep_ic(const Launch& L, int grid, size_t smem, cudaStream_t s);
cudaError_t cg_occupancy_ic(int* blocks_per_sm, size_t smem);
cudaError_t cg_set_smem_limit_ic(size_t bytes);
// the lockstep kernels (cg_lockstep.cu, cg_lockstep_ic.cu)
cudaError_t lockstep_occupancy(int* blocks_per_sm, size_t smem);
cudaError_t lockstep_occupancy_ic(int* blocks_per_sm, size_t smem);
cudaError_t lockstep_set_smem_limit(size_t bytes);
cudaError_t lockstep_set_smem_limit_ic(size_t bytes);
cudaError_t cg_occupancy(int* blocks_per_sm, size_t smem);
size_t cg_static_smem();
cudaError_t launch_validate(int n, long long nnz, const int* rp, const int* ci, const double* v,
                            unsigned* flags, int* bad_row, cudaStream_t s);
cudaError_t launch_convert(const DevMatrix& A, float* v32, float* vtf, __half* v16, __nv_bfloat16* vbf,
                           __half* v16r, __nv_bfloat16* vbfr, q52_t* v8, short* rexp, cudaStream_t s);
long long mlp_nparams_dev(int H, int nprec);
size_t mlp_grad_smem(int H, int nprec);
cudaError_t mlp_set_smem_limit(size_t bytes);
// Allowed precision entries per operation (bit p = entry p of precs), for the MLP targets.
struct OpMask {
  unsigned m[4];
};
cudaError_t launch_mlp_grad(const float* w, const float* wt, int H, int nprec, const float* feats,
                            const float* feats_next, const int* acts, const float* rew, const int* done, const float* y,
                            const long long* idx, int B, int chunk, float gamma, OpMask mask, float* part,
                            double* lpart, cudaStream_t s);
cudaError_t launch_mlp_targets(const float* wt, int H, int nprec, const float* feats_next, const float* rew,
                               const int* done, int B, float gamma, OpMask mask, float* y, cudaStream_t s);
cudaError_t launch_mlp_reduce_adam(const float* part, int nparts, long long np, float* grad, float* w, float* m,
                                   float* v, int t, float lr, const double* lpart, double* loss, cudaStream_t s);
cudaError_t launch_mlp_sample(long long* idx, int B, long long count, unsigned long long seed, unsigned long long t,
                              cudaStream_t s);
// IC(0) factorization in fp32 (sync-free: one thread per row, rows in increasing order per
// thread, each row waiting on the completion marks of the rows it depends on; all CTAs
// resident, cooperative launch). err bits: 1 breakdown, 2 unusable pattern, 4 time limit.
cudaError_t launch_ic0_factor(int n, const int* rp, const int* ci, const double* v, float* F, int* icd,
                              unsigned* done, unsigned* err, long long timeout_cycles, int nsm, cudaStream_t s);
cudaError_t launch_jacobi_diag(int n, const int* rp, const int* ci, const double* v, double* dinv, unsigned* bad,
                               cudaStream_t s);
cudaError_t launch_row_features(int n, const int* rp, const int* ci, const double* v, unsigned long long* out,
                                cudaStream_t s);
cudaError_t launch_to_format(const double* x, void* xlow, int n, int f, cudaStream_t s);
cudaError_t launch_from_q(const void* q, const short* rexp, double* y, int n, int f, cudaStream_t s);
cudaError_t launch_spmv_only(const DevSys& S, int fmt, int grid, int stream_stage, unsigned* err, cudaStream_t s);
cudaError_t spmv_occupancy(int* blocks_per_sm, size_t smem);
cudaError_t set_smem_limits(size_t bytes);
cudaError_t launch_qcopy(const double* Q, double* Qpriv, int nlanes, long long qsize, cudaStream_t s);
cudaError_t launch_qmerge(double* Q, int* visits, const Transition* trans, const SysState* st, int nlanes, int cap,
                          int S, int nprec, double lr, double gamma, OpMask mask, int joint, cudaStream_t s);
// Entries of a tabular policy's Q array and of its visit counts.
inline long long qtable_size(int S, int nprec, int joint) {
  return joint ? (long long)S * nprec * nprec * nprec * nprec : 4LL * S * nprec;
}
inline long long visits_size(int S, int joint) { return joint ? (long long)S : 4LL * S; }

}  // namespace mpcg
