/*
 * mpcg.h -- C ABI of the GB300 (sm_103a) mixed-precision conjugate gradient library.
 *
 * The library solves sparse symmetric positive definite systems A x = b (A in CSR) with
 * the conjugate gradient method of arXiv 2504.14268, Section 3, Eq. (1)-(4), in which the
 * four operations of Section 4.2 run at a precision chosen at every iteration by a
 * policy:
 *     op 1  q_k      = fl_p1(A p_k)          (sparse matrix-vector product)
 *     op 2  z_{k+1}  = fl_p2(M^-1 r_{k+1})   (preconditioner solve; M = I here, so a rounding of r)
 *     op 3  nu_k     = fl_p3(p_k^T q_k)      (inner product for alpha)
 *     op 4  sigma_k+1= fl_p4(r^T z)          (inner product for beta)
 * while the residual update r_{k+1} = r_k - alpha_k q_k and the scalars alpha_k = sigma_k /
 * nu_k, beta_k = sigma_{k+1} / sigma_k stay in fp64 (Section 4.2). Policies are the
 * Q-learning tables of Section 4.1 (greedy inference as in Algorithm 2, epsilon-greedy
 * training as in Algorithm 1), fixed assignments, replayed schedules, or a small MLP
 * Q-function.
 *
 * Conventions (every entry point):
 *   - Every call returns an mpcg_status. A solver outcome (converged, iteration cap,
 *     breakdown) is not an error; it is reported in mpcg_result.outcome.
 *   - Arguments are validated on the host before any kernel launch; device-side problems
 *     (a barrier wait that exceeded its time limit) are reported through a device status
 *     word and returned as MPCG_ERR_TIMEOUT. No kernel traps.
 *   - Memory the caller passes in (CSR arrays, b, x, history) stays owned by the caller;
 *     the library neither frees nor keeps pointers to it past the call. Objects the
 *     library creates (context, matrix, policy) are freed by the matching *_destroy.
 *   - Pointers to vectors and CSR arrays may be host memory (pageable or pinned) or device
 *     memory of the context's device; the library tells them apart with
 *     cudaPointerGetAttributes and stages host data through its own device buffers.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream). Work is enqueued on
 *     it; calls that return host-side results synchronise that stream before returning.
 *   - A context is used by one host thread at a time.
 *   - On error, mpcg_last_error(ctx) returns a message describing the failure.
 */
#ifndef MPCG_H
#define MPCG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mpcg_ctx_s* mpcg_ctx_t;       /* library-owned, opaque */
typedef struct mpcg_matrix_s* mpcg_matrix_t; /* library-owned device copies of A in every format */
typedef struct mpcg_policy_s* mpcg_policy_t; /* FIXED | SCHEDULE | QTABLE | MLP */

/* Number formats. 0..4 are the precision set of Section 5, in the order used for argmax
 * ties (first index wins). fp16/bf16/fp32/fp64 follow Table 1; tf32 (not in Table 1) is
 * read as 11 significand digits with the fp32 exponent range. BF16R / FP16R store the
 * matrix values of row i as fl(a_ij / s_i) with s_i = 2^floor(log2 max_j |a_ij|) (an
 * extension: power-of-two row scaling); for ops 2-4 they round like BF16 / FP16. Q52 is
 * Table 1's quarter precision (u = 2^-3: 3 significand digits, e_min = -14, e_max = 15,
 * x_max = 57344), stored in one byte (the fp8 E5M2 layout); it is not in Section 5's set
 * and is offered as an extra action. */
typedef enum {
  MPCG_FP16 = 0,
  MPCG_BF16 = 1,
  MPCG_TF32 = 2,
  MPCG_FP32 = 3,
  MPCG_FP64 = 4,
  MPCG_BF16R = 5,
  MPCG_FP16R = 6,
  MPCG_Q52 = 7
} mpcg_prec;
#define MPCG_NUM_FORMATS 8
#define MPCG_NUM_OPS 4
#define MPCG_MAX_PREC 8

typedef enum {
  MPCG_OK = 0,
  MPCG_ERR_INVALID_ARG = 1, /* bad pointer, size, CSR structure or option     */
  MPCG_ERR_CUDA = 2,        /* a CUDA runtime call failed                      */
  MPCG_ERR_OOM = 3,         /* device allocation failed                        */
  MPCG_ERR_BAD_POLICY = 4,  /* policy incompatible with the context's options  */
  MPCG_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up              */
  MPCG_ERR_INTERNAL = 6
} mpcg_status;

typedef enum { MPCG_CONVERGED = 0, MPCG_MAX_ITER = 1, MPCG_BREAKDOWN = 2 } mpcg_outcome;

/* CSR matrix: n rows, nnz stored entries, row_ptr[n+1] (row_ptr[0] = 0, non-decreasing,
 * row_ptr[n] = nnz), col[nnz] in [0, n), val[nnz] fp64. Every row must hold its diagonal
 * entry with a positive value (a necessary condition for SPD). Symmetry is not checked.
 * nnz < 2^31. Host or device pointers (all three in the same space). */
typedef struct {
  int32_t n;
  int64_t nnz;
  const int32_t* row_ptr;
  const int32_t* col;
  const double* val;
} mpcg_csr;

/* Method options. mpcg_options_default() fills the values of Sections 4.1 and 5. */
typedef struct {
  int32_t b_bins;          /* b iteration bins (10)                                     */
  int32_t r_bins;          /* r residual bins (10)                                      */
  int32_t t_bin;           /* T_max used by the iteration bins (1000)                   */
  int32_t min_k;           /* a solve may stop at iteration k only if k >= min_k (10)   */
  double eps_min;          /* residual floor of the bins and reward (1e-16)             */
  int32_t nprec;           /* size of the precision set P (5), <= MPCG_MAX_PREC         */
  int32_t precs[MPCG_MAX_PREC]; /* P as mpcg_prec codes, in argmax tie order            */
  double cost[MPCG_MAX_PREC];   /* c(p) for each entry of precs (cost setting C1)       */
  double w1, w2, w3;       /* reward weights (1.0, 0.1, 10.0)                           */
  double lr, gamma;        /* Q-learning rate alpha and discount gamma (0.1, 0.9)       */
  double eps0, eps_floor;  /* exploration: eps_e = max(eps_floor, eps0 (1 - e/E)) (1, 0.1) */
  uint64_t seed;           /* key of the Philox4x64-10 exploration draws                */
  int32_t unvisited_fallback; /* greedy action for a (state, op) never updated in
                                 training: an mpcg_prec code (default MPCG_FP64), or -1
                                 for the plain first-index argmax                      */
  int32_t true_res_every;  /* >0: replace r by b - A x (fp64) every this many iterations */
  int32_t true_res_at_conv;/* 1: confirm a claimed convergence with b - A x (fp64)      */
  int32_t warm_start;      /* 1: x holds x_0 on entry; 0: x_0 = 0 (Algorithms 1 and 2)  */
  int32_t op_mask[4];      /* per operation, bitmask of the entries of precs the policy may
                              choose (bit a = precs[a]); 0 allows all. Section 5 notes the
                              precision set can be customised; a mask customises it per
                              operation: greedy choice, exploration, the unvisited
                              fallback and the bootstrap max of the Section 4.1 update
                              (max over the operation's allowed entries) respect it     */
  int32_t on_breakdown;    /* 0: a breakdown ends the solve (paper); 1: inference solves
                              recompute r = b - A x in fp64, restart with p = r and finish
                              with every operation in fp64 (at most once per solve)     */
  int32_t mlp_hidden;      /* hidden width of the MLP policy (64)                       */
  int32_t batch_mode;      /* launches with several systems: 0 = automatic (lockstep),
                            * 1 = teams (each system solved by its own group of CTAs from
                            * start to end), 2 = lockstep (every CTA works on a slice of
                            * every unfinished system at every phase; slices re-cut as
                            * systems finish)                                            */
  int32_t precond;         /* 0: M = I (op 2 is z = fl_p2(r)); 1: Jacobi, M = diag(A): op 2
                            * is z = fl_p2(r_i d_i) with d_i = 1 / a_ii in fp64, and the
                            * first and restart directions are p = M^-1 r. Solves of a
                            * matrix with a row lacking a positive diagonal entry fail
                            * with MPCG_ERR_INVALID_ARG. 2: incomplete Cholesky IC(0) in
                            * fp32 (Section 5's fixed-precision fp32 preconditioner, in its
                            * symmetric zero-fill form; see mpcg_matrix_ic0): op 2 is
                            * z = fl_p2(L^-T L^-1 fl32(r)) with both substitutions in fp32,
                            * and the first and restart directions are p = L^-T L^-1 r.
                            * The factor is computed on the first such solve of a matrix
                            * and kept with it.                                          */
  double edge_tol;         /* greedy decisions of a tabular policy taken at a residual rho_k
                            * with |rho_k / theta_m - 1| <= edge_tol for a residual-bin
                            * threshold theta_m (Section 4.1's bin edges) are counted in
                            * mpcg_result.near_edge_count: there a rounding-level change of
                            * rho can move the state to the next bin (5e-3)              */
  int32_t stepped;         /* single solves (mpcg_solve): 0 = automatic (stepped for systems
                            * of at least 2^24 nonzeros without IC(0)), 1 = one persistent
                            * cooperative launch, 2 = stepped: one kernel per phase of the
                            * iteration, repeated on the device by a conditional while-loop
                            * CUDA graph, 3 = the same kernels with each pass launched by the
                            * host, which reads the phase back after every pass (for tools
                            * that cannot follow kernels inside graphs with conditional
                            * nodes; slower) (precond = 2 always runs the persistent launch,
                            * whose substitutions need every CTA resident)              */
  int32_t variant;         /* 0: the CG of Section 3 (three reductions per iteration); 1: the
                            * single-reduction iteration of Chronopoulos and Gear (an
                            * extension, equal to CG in exact arithmetic): u = fl_p2(M^-1 r),
                            * w = fl_p1(A fl_p1(u)), gamma = fl_p4(r^T u) (op 4),
                            * delta = fl_p3(w^T u) (op 3), beta = gamma / gamma_prev,
                            * alpha = gamma / (delta - beta gamma / alpha_prev), p = u + beta p,
                            * s = w + beta s, x += alpha p, r -= alpha s, and ||r_{k+1}||^2
                            * expanded from inner products of the same pass, so that one
                            * reduction serves an iteration. Runs in the lockstep and
                            * stepped kernels (every launch with variant 1 uses them), with
                            * M = I or Jacobi (precond 2 is refused); mpcg_solve_noalloc
                            * refuses it                                                  */
  int32_t joint;           /* tabular policies: 0 = one table per operation (Section 4.1), 1 =
                            * one table over the joint actions (the |P|^m alternative that
                            * Section 4.1 weighs): Q[S][nprec^4], entry ((a1 P + a2) P + a3) P
                            * + a4, update counts visits[S]; the allowed joint actions are the
                            * product of the op_mask sets, greedy is the first largest allowed
                            * entry, exploration draws op 1's u and each operation's pick    */
  int32_t reserved_joint;
} mpcg_options;

/* Result of one solve. */
typedef struct {
  int32_t outcome;         /* mpcg_outcome                                              */
  int32_t iters;           /* completed iterations (Algorithm 2 logs k+1 at the stop)   */
  double rel_res_rec;      /* ||r|| / ||b|| of the recursive residual at the end        */
  double rel_res_true;     /* ||b - A x|| / ||b|| computed in fp64 at the end           */
  int32_t n_true_checks;   /* residual recomputations during the solve                  */
  int32_t n_restarts;      /* fp64 restarts after a breakdown (option on_breakdown)      */
  int64_t action_hist[MPCG_NUM_OPS][MPCG_MAX_PREC]; /* iterations per (op, format)       */
  int32_t near_edge_count; /* greedy tabular decisions taken within edge_tol of a residual-bin
                              edge (options.edge_tol); 0 for other policies             */
  int32_t kernel_launches; /* the library's solver-kernel launches of the call: 1 for one
                              persistent or lockstep launch (shared by a batch), passes x
                              kernels for the stepped solve (the phase kernels and the loop
                              control kernel of every pass of the graph)               */
} mpcg_result;

/* One record per iteration k (80 bytes). rho is rho_{k+1} after the iteration (the true
 * relative residual when r was replaced). flags: bit0 converged here, bit1 breakdown here,
 * bit2 r replaced by b - A x, bit3 an operation explored (training), bit4 restarted in fp64
 * after the breakdown. ns_a / ns_b / ns_c:
 * device time (globaltimer, ns) from the previous team barrier to the barriers that close
 * phase A (product and nu), phase B (residual update, norms) and phase C (x and p update)
 * of the iteration, including the barrier itself. */
typedef struct {
  int32_t k, state;
  int8_t fmt[4];
  int8_t act[4];
  double rho, nu, alpha, sigma, beta, reward;
  int32_t flags;
  uint32_t ns_a, ns_b, ns_c;
} mpcg_iter_record;

/* Matrix statistics filled by mpcg_matrix_info. */
typedef struct {
  int32_t n;
  int64_t nnz;
  double mean_row_nnz, max_row_nnz, cv_row_nnz;
  int32_t spmv_sched[MPCG_NUM_FORMATS]; /* SpMV schedule chosen per value format          */
  int32_t spmv_lanes[MPCG_NUM_FORMATS]; /* lanes per row of that schedule                 */
  int64_t device_bytes;                 /* library-owned device memory of the matrix      */
  double static_features[5];            /* MLP policy's static matrix features            */
} mpcg_matrix_stats;

/* ---- context ---------------------------------------------------------------------- */

/* Fills *opt with the paper's defaults (Sections 4.1 and 5, cost setting C1, P = {fp16,
 * bf16, tf32, fp32, fp64}). */
void mpcg_options_default(mpcg_options* opt);

/* Creates a context on CUDA device `device` with a copy of *opt (NULL = defaults).
 * Errors: INVALID_ARG (bad options), CUDA, OOM. */
mpcg_status mpcg_create(mpcg_ctx_t* out, int device, const mpcg_options* opt);
mpcg_status mpcg_destroy(mpcg_ctx_t ctx);
/* Message of the last failed call on ctx ("" if none). Valid until the next call. */
const char* mpcg_last_error(mpcg_ctx_t ctx);
/* Returns the number of SMs and the co-resident CTAs per SM of the solver kernel. */
mpcg_status mpcg_device_info(mpcg_ctx_t ctx, int32_t* num_sms, int32_t* ctas_per_sm);

/* ---- matrices --------------------------------------------------------------------- */

/* Copies A into library-owned device memory, validates it on the device (row_ptr
 * monotone, col in range, finite values, positive diagonal present in every row), builds
 * the value copies in every format (a single rounding from fp64 each; Table 1 formats and
 * the row-scaled extensions) and picks an SpMV schedule per format. Enqueued on `stream`
 * and synchronised. Errors: INVALID_ARG (structure; message names the first bad row),
 * CUDA, OOM. */
mpcg_status mpcg_matrix_create(mpcg_ctx_t ctx, const mpcg_csr* A, mpcg_matrix_t* out, void* stream);
mpcg_status mpcg_matrix_destroy(mpcg_matrix_t A);
mpcg_status mpcg_matrix_info(mpcg_matrix_t A, mpcg_matrix_stats* info);
/* Times every SpMV schedule on A for each value format (a few launches each) and keeps
 * the fastest (the autotuner). `reps` timed launches per candidate. Matrices with fewer
 * than 2^22 nonzeros, whose products are too short to time apart, keep the row-length rule
 * that mpcg_matrix_create applies (vector loads for a mean row length up to ~32 nonzeros,
 * K lanes with about 24 nonzeros per lane beyond). Results are cached in the context by
 * matrix bucket (half-octave of the mean row length, quarter of its coefficient of
 * variation, octave of the longest row and of n, column order): a matrix of a bucket tuned
 * before takes that bucket's schedules without timing when they all apply to it; with
 * reps < 0 the matrix is timed (|reps| launches per candidate) and replaces the entry. */
mpcg_status mpcg_matrix_autotune(mpcg_ctx_t ctx, mpcg_matrix_t A, int32_t reps, void* stream);
/* IC(0) factor of A in fp32, computed on the device once per matrix and kept with it
 * (Section 5 preconditions with an fp32 incomplete factorization; for SPD A this is its
 * symmetric zero-fill form M = L L^T, L on the pattern of A's lower triangle). Each entry:
 * l_ij = (fl32(a_ij) - sum_{k<j} l_ik l_jk) / l_jj for j < i and l_ii = sqrt(fl32(a_ii) -
 * sum_{k<i} l_ik^2), every operation in fp32, sums in increasing k over the columns stored
 * in both rows. If `factor` (device, nnz floats, caller-owned; may be NULL) is given, it
 * receives one value per stored entry of A in A's CSR order: l_ij at (i, j) for j <= i and
 * l_ji at (i, j) for j > i. Needs strictly increasing column indices in every row, a
 * diagonal entry in every row and a symmetric pattern (INVALID_ARG otherwise); a
 * non-positive pivot (IC(0) exists for M-matrices, not for every SPD matrix) is INVALID_ARG
 * "breaks down". Synchronises `stream`. */
mpcg_status mpcg_matrix_ic0(mpcg_ctx_t ctx, mpcg_matrix_t A, float* factor, void* stream);
/* Dependency levels of the two triangular substitutions of a CSR pattern (host pointers,
 * no device work; the scheduling analysis of the IC(0) substitutions): level_lower[i] =
 * 0 for a row without stored columns j < i, else 1 + the largest level_lower[j] over them
 * (rows of one level of L y = r are independent once the earlier levels are done);
 * level_upper[i] the same over the columns j > i (for L^T w = y, rows taken from the last).
 * depth[0], depth[1] receive the number of levels of each. The caller owns all arrays
 * (level arrays of n int32). INVALID_ARG for n < 0, NULL arrays, a decreasing row_ptr or a
 * column outside [0, n). */
mpcg_status mpcg_csr_levels(int32_t n, const int32_t* row_ptr, const int32_t* col, int32_t* level_lower,
                            int32_t* level_upper, int32_t* depth);
/* Forces the SpMV schedule of value format `fmt` (sched: 0 = sub-warp vector CSR with
 * `lanes` lanes per row (1, 2, 4, 8, 16 or 32); 1 = staged stream CSR, shared-memory tiles
 * filled by bulk copies, `lanes` = 1, 2 or 4 lanes per row; 2 = one thread per row reading
 * columns and values with 16-byte loads, `lanes` = 1; 3 = merge-path CSR (Merrill and
 * Garland, SC 2016): every thread of a CTA an equal share of the merged list of the CTA's row
 * ends and products, rows split over threads merged exactly before the one rounding, `lanes`
 * = 1; 4 = staged x: one thread per row as schedule 2, gathering from a copy in shared memory
 * of the window of x that the CTA's rows read, when it fits (otherwise from x), `lanes` = 1,
 * for matrices whose column indices increase in every row). In schedules 0, 2 and 4 a row
 * longer than 1024 nonzeros (a power-law hub) is summed by a whole CTA after the CTA's other
 * rows.
 * INVALID_ARG for other combinations and for a stream tile that does not fit its
 * shared-memory stage. */
mpcg_status mpcg_matrix_set_schedule(mpcg_matrix_t A, int32_t fmt, int32_t sched, int32_t lanes);

/* y = fl_fmt(A fl_fmt(x)) with the matrix's schedule for `fmt` (op 1 of Section 4.2 on its
 * own; x and y fp64 device vectors of length n). `reps` > 1 repeats the product (for timing);
 * if ms_per_rep is non-NULL it receives the mean device time of one product. */
mpcg_status mpcg_spmv(mpcg_ctx_t ctx, mpcg_matrix_t A, int32_t fmt, const double* x, double* y,
                      int32_t reps, double* ms_per_rep, void* stream);

/* ---- policies --------------------------------------------------------------------- */

/* Same four formats at every iteration (op order p1..p4). Any mpcg_prec codes. */
mpcg_status mpcg_policy_fixed(mpcg_ctx_t ctx, const int32_t fmt[4], mpcg_policy_t* out);
/* Iteration k uses row min(k, len-1) of the host array fmts[len][4] (replay). */
mpcg_status mpcg_policy_schedule(mpcg_ctx_t ctx, const int32_t* fmts, int32_t len, mpcg_policy_t* out);
/* Tabular policy (Section 4.1): Q[4][b*r][nprec] fp64 and visits[4][b*r] (host arrays,
 * visits may be NULL = all visited), shaped by the context's options; with options.joint,
 * Q[b*r][nprec^4] and visits[b*r]. */
mpcg_status mpcg_policy_qtable(mpcg_ctx_t ctx, const double* Q, const int32_t* visits, mpcg_policy_t* out);
/* MLP Q-function 16 -> H -> H -> 4*nprec (ReLU), fp32 parameters in the layout W1[H][16],
 * b1[H], W2[H][H], b2[H], W3[4*nprec][H], b3[4*nprec] (host array of mpcg_mlp_nparams
 * floats), H = options.mlp_hidden. Greedy: per operation, the first-index argmax over its
 * nprec outputs. Features of iteration k (an extension; the paper's state is the pair of
 * bins): f0 = log10(n)/8, f1 = mean nnz per row / 64, f2 = log10(max a_ii / min a_ii)/16,
 * f3 = log10(max_i sum_j |a_ij| / a_ii)/16, f4 = fraction of |a_ij| outside the fp16 normal
 * range, f5 = k / t_bin, f6 = -log10(max(rho_k, eps_min))/16, f7 = log10(rho_k / rho_{k-1}),
 * f8 = log10(rho_k / rho_{k-8}) / 8, f9 = log10|alpha_{k-1}| / 8, f10 = log10|beta_{k-1}| / 8,
 * f11 = log10(true / recursive residual) at the last recomputation, f12..f15 = previous
 * action indices / (nprec - 1); unavailable history terms are 0. */
mpcg_status mpcg_policy_mlp(mpcg_ctx_t ctx, const float* params, mpcg_policy_t* out);
int64_t mpcg_mlp_nparams(int32_t hidden, int32_t nprec);
/* Copies a QTABLE policy's tables back to host arrays (either may be NULL). */
mpcg_status mpcg_policy_get_qtable(mpcg_policy_t P, double* Q, int32_t* visits);
/* Copies an MLP policy's parameters back to a host array. */
mpcg_status mpcg_policy_get_mlp(mpcg_policy_t P, float* params);
/* Serialises a policy to a host buffer. With blob == NULL, *bytes receives the size. The
 * blob holds a header (magic "MPCGPOL1", kind, b, r, t_bin, eps_min, nprec, precs, costs)
 * followed by the tables or parameters. */
mpcg_status mpcg_policy_save(mpcg_policy_t P, void* blob, size_t* bytes);
/* Creates a policy from a blob written by mpcg_policy_save (host buffer). Errors:
 * INVALID_ARG (bad magic or size), BAD_POLICY (shape differs from the context's options). */
mpcg_status mpcg_policy_load(mpcg_ctx_t ctx, const void* blob, size_t bytes, mpcg_policy_t* out);
mpcg_status mpcg_policy_destroy(mpcg_policy_t P);

/* ---- solves ----------------------------------------------------------------------- */

/* Solves A x = b with the policy (Algorithm 2 for QTABLE/MLP policies) until
 * ||r_{k+1}|| / ||b|| < tol with k >= min_k, max_iter iterations, or breakdown
 * (non-positive or non-finite p^T A p, non-finite residual). One cooperative launch of the
 * persistent kernel runs every iteration on the device. b and x: n doubles, host or device.
 * history (optional): device or host array of history_cap records. Synchronises `stream`.
 * Errors: INVALID_ARG, BAD_POLICY, CUDA, OOM, TIMEOUT. */
mpcg_status mpcg_solve(mpcg_ctx_t ctx, mpcg_matrix_t A, const double* b, double* x, double tol,
                       int32_t max_iter, mpcg_policy_t policy, mpcg_result* res,
                       mpcg_iter_record* history, int32_t history_cap, void* stream);

/* Solves nsys independent systems in one persistent launch: the systems are assigned
 * longest-first to teams of CTAs sized by their nonzeros. b[i], x[i]: device pointers.
 * tol and max_iter: per system (host arrays). res: host array of nsys results.
 * Synchronises `stream`. */
mpcg_status mpcg_solve_batched(mpcg_ctx_t ctx, int32_t nsys, const mpcg_matrix_t* A,
                               const double* const* b, double* const* x, const double* tol,
                               const int32_t* max_iter, mpcg_policy_t policy, mpcg_result* res,
                               void* stream);

/* Batched solve captured once into a CUDA graph (device pointers only): create, replay,
 * read results (host array), destroy. Replays reuse the same inputs and outputs. */
typedef struct mpcg_graph_s* mpcg_graph_t;
mpcg_status mpcg_graph_create(mpcg_ctx_t ctx, int32_t nsys, const mpcg_matrix_t* A,
                              const double* const* b, double* const* x, const double* tol,
                              const int32_t* max_iter, mpcg_policy_t policy, void* stream,
                              mpcg_graph_t* out);
mpcg_status mpcg_graph_launch(mpcg_graph_t g, void* stream);
mpcg_status mpcg_graph_results(mpcg_graph_t g, mpcg_result* res, void* stream);
mpcg_status mpcg_graph_destroy(mpcg_graph_t g);

/* Same solve as mpcg_solve (no history) for callers that cannot allocate device memory
 * while they solve, e.g. code running under a fixed device-memory budget or inside a pool
 * that must not grow. The paper has no counterpart; this is a property of the library.
 * This call allocates nothing: its scratch (work vectors, team barriers, partial sums,
 * state) lives in a static device array of 1 MiB + 28 bytes per row for at most
 * 1,048,576 rows (about 29 MiB), which every GPU that loads the library holds until the
 * process exits. Systems with more rows are rejected with MPCG_ERR_INVALID_ARG. b and x must
 * be device pointers; the matrix and the policy are created beforehand with the calls
 * above. Each call looks up the array's device address with the context's device current;
 * the first lookup on a device loads the library's device code, so make the first call on
 * a device before any stream capture. The call synchronises `stream` before it returns.
 * All calls share the one array and it keeps the last call's contents (the barriers and
 * status word are cleared by each call): calls whose work overlaps on the GPU (other
 * streams, other host threads) race and must not be issued. The system always runs as one
 * team of CTAs (options.batch_mode is ignored). Contexts with precond = 2 (IC(0), whose
 * factor and marks need memory) are rejected with MPCG_ERR_INVALID_ARG. */
mpcg_status mpcg_solve_noalloc(mpcg_ctx_t ctx, mpcg_matrix_t A, const double* b, double* x, double tol,
                               int32_t max_iter, mpcg_policy_t policy, mpcg_result* res, void* stream);

/* ---- training --------------------------------------------------------------------- */

/* Tabular Q-learning (Algorithm 1) on nsys training systems, batched: in every round
 * e = 1..episodes each system runs one epsilon-greedy episode of at most t_max iterations
 * from x_0 = 0 on a private copy of the tables, updating the copy online; at the end of the
 * round the shared tables are rebuilt by replaying every recorded transition (system 0..
 * nsys-1, then iteration order) onto the round-start tables. With nsys = 1 this is
 * Algorithm 1. `inout` is a QTABLE policy updated in place. iters_out (optional, host,
 * [episodes][nsys]) receives each episode's iteration count. b[i]: device pointers. */
mpcg_status mpcg_train_qtable(mpcg_ctx_t ctx, int32_t nsys, const mpcg_matrix_t* A,
                              const double* const* b, double tol, int32_t t_max, int32_t episodes,
                              mpcg_policy_t inout, int32_t* iters_out, void* stream);

/* ---- learned policy (MLP Q-function; an extension, not in the paper) ----------------- */

/* One transition of the MLP's training data (152 bytes). */
typedef struct {
  float f[16];      /* features of state s_k (see mpcg_policy_mlp for their definition)   */
  float f_next[16]; /* features of state s_{k+1} (unused when done = 1)                   */
  int32_t act[4];   /* action of each operation as an index into options.precs            */
  float reward;     /* reward of Section 4.1                                              */
  int32_t done;     /* 1 when the episode ended with this transition                      */
} mpcg_transition;

/* Runs one epsilon-greedy episode (at most max_iter iterations, x_0 = 0) per system with
 * the behaviour policy (QTABLE: its tables are copied and updated privately as in
 * Algorithm 1, the policy itself is unchanged; MLP: greedy on its Q-values) and exploration
 * rate eps, episode counter `episode` for the draws. The transitions of all systems are
 * written to the host array out (system order, then iteration order), at most cap of them;
 * *count receives the number written. b[i]: device pointers. */
mpcg_status mpcg_collect(mpcg_ctx_t ctx, int32_t nsys, const mpcg_matrix_t* A, const double* const* b, double tol,
                         int32_t max_iter, mpcg_policy_t behavior, double eps, uint64_t episode,
                         mpcg_transition* out, int64_t cap, int64_t* count, void* stream);

/* Loss (1/(4B)) sum_b sum_j 1/2 (Q(f_b)[j, a_bj] - y_bj)^2 of the MLP with parameters
 * `params` (host, mpcg_mlp_nparams floats) on B samples (host arrays feats[B][16],
 * acts[B][4], y[B][4]) and its gradient (host array, same layout as params). */
mpcg_status mpcg_mlp_loss_grad(mpcg_ctx_t ctx, const float* params, int64_t B, const float* feats,
                               const int32_t* acts, const float* y, float* grad, double* loss, void* stream);

/* Fitted-Q training of an MLP policy in place: `steps` Adam steps (lr, betas 0.9 / 0.999,
 * eps 1e-8) on minibatches of `batch` transitions drawn from data[count] (host array) with
 * Philox4x64-10 (key seed), targets r + gamma (1 - done) max_p Q_target(f_next)[j, p] (p over
 * the entries the options' op_mask[j] allows, as mpcg_mlp_targets) from a target network
 * copied from the trained one every target_sync steps. loss_out (optional, host [steps])
 * receives each step's loss. */
mpcg_status mpcg_mlp_train(mpcg_ctx_t ctx, mpcg_policy_t mlp, const mpcg_transition* data, int64_t count,
                           int32_t steps, int32_t batch, float lr, int32_t target_sync, uint64_t seed,
                           float* loss_out, void* stream);

/* One Adam step (Kingma & Ba, ICLR 2015; the optimiser of mpcg_mlp_train) on host arrays of
 * mpcg_mlp_nparams(options.mlp_hidden, options.nprec) floats: m = 0.9 m + 0.1 g,
 * v = 0.999 v + 0.001 g^2, params -= lr (m / (1 - 0.9^t)) / (sqrt(v / (1 - 0.999^t)) + 1e-8),
 * in fp32 on the device with the kernel mpcg_mlp_train uses. params, m, v are updated in
 * place; grad is read. t >= 1 is the step number. Errors: INVALID_ARG (NULL, t < 1), CUDA,
 * OOM. */
mpcg_status mpcg_mlp_adam(mpcg_ctx_t ctx, float* params, float* m, float* v, const float* grad, int32_t t, float lr,
                          void* stream);

/* The fitted-Q regression targets of the MLP Q-function (the one-step backup of the
 * Section 4.1 update with the table replaced by the network): y[b][j] = rew[b] +
 * gamma (1 - done[b]) max over the entries p of precs allowed by the options' op_mask[j] of
 * Q_target(feats_next[b])[j, p], Q_target the network with parameters target_params (host,
 * mpcg_mlp_nparams floats). Host arrays feats_next[B][16], rew[B], done[B], y[B][4]. Errors:
 * INVALID_ARG (NULL, B < 1), CUDA, OOM. */
mpcg_status mpcg_mlp_targets(mpcg_ctx_t ctx, const float* target_params, int64_t B, const float* feats_next,
                             const float* rew, const int32_t* done, float* y, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MPCG_H */
