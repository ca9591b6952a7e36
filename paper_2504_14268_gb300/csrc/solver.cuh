// Persistent mixed-precision CG kernel (Section 3 Eq. (1)-(4) with the operation
// precisions of Section 4.2, Algorithm 2 for inference and Algorithm 1's episode for
// training).
//
// One cooperative launch runs every iteration of every system on the device. The CTAs of
// the grid are grouped into teams; a team solves its systems one after another. A single
// large solve uses one team made of the whole grid; a batch of small systems uses many
// teams, down to one CTA per system. Inside a team the rows of a system are split between
// the CTAs by nonzeros. Each iteration has three phases separated by team barriers:
//   A  q = fl_p1(A fl_p1(p)) and the CTA partial of nu = p^T q (op 3, precision p3)
//   B  r -= alpha q (fp64), partials of ||r||^2 (fp64) and sigma = r^T z (op 4, z = fl_p2(r))
//   C  x += alpha p, p = z + beta p (fp64) and p's copy in the next product's format
// At a team barrier the CTA that arrives last reduces the partials of all CTAs of the team
// in a fixed order (deterministic), evaluates the scalars alpha, beta, rho in fp64, the
// stopping tests, the policy (state bins of Section 4.1, argmax / epsilon-greedy over the
// Q-tables, or the MLP Q-function) and, in training, the reward and Q update; then it
// releases the others. Every wait is bounded; a wait that runs out sets the device status
// word and the kernel returns.
// Solver kernels shared by two translation units: cg_kernel.cu instantiates them without
// the IC(0) preconditioner, cg_kernel_ic.cu with it (two nvcc processes in parallel, and
// the unpreconditioned kernels keep their own register allocation).
#pragma once
#include "internal.h"
#include "spmv.cuh"
#include "ic0.cuh"

namespace mpcg {

namespace {

enum Mode : int { M_CONT = 0, M_DONE = 1, M_X_THEN_DONE = 2, M_TCHK = 3, M_RESTART = 4, M_RESTART64 = 5,
                  M_X_THEN_RESTART64 = 6 };

struct TeamCtx {
  int team, rank, size, first;
  unsigned* bar;
};

// Values every thread needs after a barrier.
struct Bcast {
  double alpha, beta;
  int k, mode;
  int fmt[4];
  int zfmt;
  int wfmt;       // single-reduction iteration: product format of the finished iteration
  unsigned icep;  // epoch of the IC(0) application in this phase
};

struct Smem {
  double red[2 * (kThreads / 32)];
  double tmp;  // a scalar handed from thread 0 to the CTA
  Bcast bc;
  int last;
  int ok;
  unsigned gen;
  int need_action;
  int flag;
  int r0, r1;
  int lk_phase, lk_known, lk_done;
  int a_fmt[4], a_act[4], a_expl, a_state;
  unsigned long long mbar[2];
  unsigned mbar_phase;
  float feat[kNFeat];
  float h1[kMaxHidden];
  float h2[kMaxHidden];
  float out[4 * 8];
};

// ----------------------------------------------------------------------------------------
// Reductions
// ----------------------------------------------------------------------------------------

// Sum over the CTA in a fixed order: xor butterfly inside each warp, then the warp sums in
// warp order. Every thread returns the same value.
template <typename T>
__device__ __forceinline__ T cta_sum(T v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)v;
  __syncthreads();
  T s = 0;
#pragma unroll
  for (int w = 0; w < kThreads / 32; ++w) s += (T)red[w];
  return s;
}

// Reduction of a dot accumulator over the CTA in a fixed order: the fp64 part by
// cta_sum, the compensated fp32 pair by an xor butterfly of TwoSum steps, then the warp
// pairs in warp order; returns d + s + c in fp64.
__device__ __forceinline__ double cta_dot(DotAcc a, double* red) {
  const double d = cta_sum(a.d, red);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float s2 = __shfl_xor_sync(kFull, a.s, o), c2 = __shfl_xor_sync(kFull, a.c, o);
    float t;
    two_sum(a.s, s2, a.s, t);
    a.c = __fadd_rn(__fadd_rn(a.c, c2), t);
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5] = (double)a.s;
    red[(threadIdx.x >> 5) + kThreads / 32] = (double)a.c;
  }
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int w = 0; w < kThreads / 32; ++w) s += red[w] + red[w + kThreads / 32];
  return d + s;
}

__device__ __forceinline__ void write_partial(const Launch& L, int slot, double v) {
  if (threadIdx.x == 0) L.partials[(long long)blockIdx.x * kNSlot + slot] = v;
}

// Sum of one partial slot over the CTAs of the team, in rank order per thread and a fixed
// tree across threads (deterministic for a given team size). Run by the last CTA.
__device__ __forceinline__ double team_sum(const Launch& L, const TeamCtx& T, int slot, double* red) {
  double v = 0.0;
  for (int c = threadIdx.x; c < T.size; c += kThreads)
    v += __ldcg(&L.partials[(long long)(T.first + c) * kNSlot + slot]);
  return cta_sum(v, red);
}

// ----------------------------------------------------------------------------------------
// Team barrier
// ----------------------------------------------------------------------------------------

__device__ __forceinline__ bool err_set(const Launch& L) { return *(volatile unsigned*)L.err != 0u; }

// Arrival: returns true in the CTA that arrives last; that CTA does the team work and then
// calls team_release. Other CTAs call team_wait.
__device__ __forceinline__ bool team_arrive(const TeamCtx& T, Smem& sm) {
  __syncthreads();
  if (T.size == 1) return true;
  if (threadIdx.x == 0) {
    const unsigned g = *(volatile unsigned*)(T.bar + 16);  // generation before our arrival
    __threadfence();                                      // release this CTA's writes
    const unsigned old = atomicAdd(T.bar, 1u);
    sm.last = (old == (unsigned)T.size - 1u) ? 1 : 0;
    sm.gen = g;
    if (sm.last) __threadfence();                         // acquire the others' writes
  }
  __syncthreads();
  return sm.last != 0;
}

__device__ __forceinline__ void team_release(const TeamCtx& T) {
  __syncthreads();
  if (T.size > 1 && threadIdx.x == 0) {
    atomicExch(T.bar, 0u);
    __threadfence();
    atomicAdd(T.bar + 16, 1u);
  }
  __syncthreads();
}

// Bounded wait for the generation to move on. Returns false (and sets the status word)
// when the wait exceeds the time limit or another CTA reported an error.
__device__ __forceinline__ bool team_wait(const Launch& L, const TeamCtx& T, Smem& sm) {
  if (threadIdx.x == 0) {
    int ok = 1;
    const long long t0 = clock64();
    unsigned spins = 0;
    while (*(volatile unsigned*)(T.bar + 16) == sm.gen) {
      if ((++spins & 255u) == 0u) {
        if (err_set(L)) { ok = 0; break; }
        if (clock64() - t0 > L.timeout_cycles) {
          atomicCAS(L.err, 0u, (unsigned)DERR_TIMEOUT);
          ok = 0;
          break;
        }
      }
      __nanosleep(64);
    }
    __threadfence();
    sm.ok = ok;
  }
  __syncthreads();
  return sm.ok != 0;
}

// Loads the broadcast values of a system's state into shared memory (after a barrier).
__device__ __forceinline__ void load_bcast(const SysState* st, Smem& sm) {
  if (threadIdx.x == 0) {
    const volatile SysState* v = st;
    sm.bc.alpha = v->alpha;
    sm.bc.beta = v->beta;
    sm.bc.k = v->k;
    sm.bc.mode = v->mode;
    sm.bc.zfmt = v->zfmt;
    sm.bc.wfmt = v->wfmt;
    sm.bc.icep = v->icep;
#pragma unroll
    for (int j = 0; j < 4; ++j) sm.bc.fmt[j] = v->fmt[j];
  }
  __syncthreads();
}

// ----------------------------------------------------------------------------------------
// Policy (Section 4.1): state, action, reward, Q update
// ----------------------------------------------------------------------------------------

__device__ __forceinline__ int state_of(const OptView& o, int k, double rho) {
  int i = k / o.t_width;
  if (i > o.b_bins - 1) i = o.b_bins - 1;
  int j = 0;
  for (int m = 1; m < o.r_bins; ++m) j += (rho <= o.thr[m]) ? 1 : 0;
  return i * o.r_bins + j;
}

// Reward of Section 4.1, evaluated with separately rounded operations in the order
// w1 min(-log10 rho, cap) - w2 c(p_1) - ... - w2 c(p_4) [+ w3].
__device__ double reward_of(const OptView& o, double rho, const int* act, double tau, bool breakdown) {
  double acc;
  if (breakdown) {
    acc = -o.log_cap;
  } else {
    const double l = rho > 0.0 ? -log10(rho) : __longlong_as_double(0x7ff0000000000000ll);
    acc = l < o.log_cap ? l : o.log_cap;
  }
  double r = __dmul_rn(o.w1, acc);
  for (int j = 0; j < 4; ++j)
    if (act[j] >= 0 && act[j] < o.nprec) r = __dsub_rn(r, __dmul_rn(o.w2, o.cost[act[j]]));
  if (!breakdown && rho < tau) r = __dadd_rn(r, o.w3);
  return r;
}


// First-index argmax over the allowed entries (bit a of mask).
__device__ __forceinline__ int row_argmax(const double* row, int n, unsigned mask) {
  int b = -1;
  for (int a = 0; a < n; ++a)
    if ((mask >> a) & 1u)
      if (b < 0 || row[a] > row[b]) b = a;
  return b;
}

// The k-th allowed index (k < popcount(mask)).
__device__ __forceinline__ int kth_allowed(unsigned mask, int k) {
  for (int a = 0; a < 32; ++a)
    if ((mask >> a) & 1u) {
      if (k == 0) return a;
      --k;
    }
  return 0;
}

// The exploration draws of operation j at iteration k (Philox4x64-10 keyed by the seed, counter
// (episode, lane, k, j)): u uniform in [0, 1) from 53 bits of the first word, pick the low 32
// bits of the second.
__device__ __forceinline__ void policy_draw(const Launch& L, const DevSys& S, int k, int j, double& u, unsigned& pick) {
  U64x4 c;
  c.v[0] = L.episode;
  c.v[1] = (unsigned long long)S.lane;
  c.v[2] = (unsigned long long)k;
  c.v[3] = (unsigned long long)j;
  const U64x4 w = philox4x64_10(c, L.opt.seed, 0x6d706367ull);
  u = (double)(w.v[0] >> 11) * 0x1.0p-53;
  pick = (unsigned)(w.v[1] & 0xffffffffull);
}

// Q_j(s, a_j) += lr (R + gamma max_{p in P_j} Q_j(s', p) - Q_j(s, a_j)), terminal without the max
// term; P_j = the entries operation j may choose (op_mask).
__device__ void q_update(double* Q, const OptView& o, const Transition& t) {
  const int S = o.b_bins * o.r_bins;
  if (o.joint) {  // one entry of the joint table, bootstrap max over the allowed joint actions
    const int np4 = o.nprec * o.nprec * o.nprec * o.nprec;
    const int a = ((t.act[0] * o.nprec + t.act[1]) * o.nprec + t.act[2]) * o.nprec + t.act[3];
    double* row = Q + (long long)t.s * np4;
    double target = t.reward;
    if (!t.terminal)
      target = __dadd_rn(target, __dmul_rn(o.gamma, joint_row_max(Q + (long long)t.s_next * np4, o.nprec, o.op_mask)));
    const double cur = row[a];
    row[a] = __dadd_rn(cur, __dmul_rn(o.lr, __dsub_rn(target, cur)));
    return;
  }
  for (int j = 0; j < 4; ++j) {
    double* row = Q + ((long long)j * S + t.s) * o.nprec;
    double target = t.reward;
    if (!t.terminal)
      target = __dadd_rn(target, __dmul_rn(o.gamma, row_max_allowed(Q + ((long long)j * S + t.s_next) * o.nprec,
                                                                     o.nprec, (unsigned)o.op_mask[j])));
    const double cur = row[t.act[j]];
    row[t.act[j]] = __dadd_rn(cur, __dmul_rn(o.lr, __dsub_rn(target, cur)));
  }
}

// MLP forward pass by the whole CTA, fp32, weights read through the read-only path.
__device__ void mlp_forward(const float* __restrict__ w, int H, int nout, Smem& sm) {
  const float* W1 = w;
  const float* b1 = W1 + H * kNFeat;
  const float* W2 = b1 + H;
  const float* b2 = W2 + H * H;
  const float* W3 = b2 + H;
  const float* b3 = W3 + nout * H;
  for (int i = threadIdx.x; i < H; i += kThreads) {
    float s = __ldg(b1 + i);
    for (int j = 0; j < kNFeat; ++j) s = fmaf(__ldg(W1 + i * kNFeat + j), sm.feat[j], s);
    sm.h1[i] = s > 0.f ? s : 0.f;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < H; i += kThreads) {
    float s = __ldg(b2 + i);
    for (int j = 0; j < H; ++j) s = fmaf(__ldg(W2 + i * H + j), sm.h1[j], s);
    sm.h2[i] = s > 0.f ? s : 0.f;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nout; i += kThreads) {
    float s = __ldg(b3 + i);
    for (int j = 0; j < H; ++j) s = fmaf(__ldg(W3 + i * H + j), sm.h2[j], s);
    sm.out[i] = s;
  }
  __syncthreads();
}

__device__ __forceinline__ float safe_log10f(double v) { return v > 0.0 ? (float)log10(v) : 0.f; }

// Features of the MLP policy at iteration k (static part from the matrix, dynamic part from
// the solver state): k / t_bin, -log10 max(rho, eps_min) / 16, one- and eight-step log10
// residual ratios, log10 |alpha|, log10 |beta| (/ 8), log10 of the last true/recursive
// residual gap, previous action indices / (nprec - 1).
__device__ void mlp_features(const Launch& L, const DevSys& S, const SysState* st, int k, Smem& sm) {
  const OptView& o = L.opt;
  for (int j = 0; j < 5; ++j) sm.feat[j] = S.feat_static[j];
  const double rho = st->rho_hist[0];
  const double rr = rho > o.eps_min ? rho : o.eps_min;
  sm.feat[5] = (float)((double)k / (double)o.t_bin);
  sm.feat[6] = (float)(-log10(rr) / 16.0);
  sm.feat[7] = (st->rho_hist[1] > 0.0 && rho > 0.0) ? (float)log10(rho / st->rho_hist[1]) : 0.f;
  sm.feat[8] = (st->rho_hist[8] > 0.0 && rho > 0.0) ? (float)(log10(rho / st->rho_hist[8]) / 8.0) : 0.f;
  sm.feat[9] = st->have_prev ? safe_log10f(fabs(st->alpha_prev)) / 8.f : 0.f;
  sm.feat[10] = st->have_prev ? safe_log10f(fabs(st->beta_prev)) / 8.f : 0.f;
  sm.feat[11] = (float)st->gap_log;
  for (int j = 0; j < 4; ++j)
    sm.feat[12 + j] = (st->have_prev && o.nprec > 1) ? (float)st->prev_act[j] / (float)(o.nprec - 1) : 0.f;
}

// Chooses the action of iteration k in state of residual rho. Called by every thread of the
// CTA that holds the team work; the result is left in sm.a_*.
__device__ void choose_action(const Launch& L, const DevSys& S, SysState* st, int k, double rho, Smem& sm) {
  const OptView& o = L.opt;
  const PolicyView& P = L.pol;
  const int s = state_of(o, k, rho);
  if (P.kind == 3 || S.feat_log) {
    if (threadIdx.x == 0) {
      mlp_features(L, S, st, k, sm);
      if (S.feat_log && k < S.feat_cap)
        for (int j = 0; j < kNFeat; ++j) S.feat_log[(long long)k * kNFeat + j] = sm.feat[j];
    }
    __syncthreads();
    if (P.kind == 3 && !st->fp64_lock) mlp_forward(P.mlp, P.H, 4 * o.nprec, sm);
  }
  if (threadIdx.x == 0) {
    int expl = 0;
    int jact[4] = {0, 0, 0, 0};
    if (P.kind == 2 && o.joint && !st->fp64_lock) {
      // the joint table: exploration decided by operation 1's draw, each operation's pick from
      // its own draw; greedy: first largest allowed joint entry; unvisited state: the fallback
      // format for all four operations when each allows it
      bool done = false;
      if (L.train) {
        double u[4];
        unsigned pick[4];
        for (int j = 0; j < 4; ++j) policy_draw(L, S, k, j, u[j], pick[j]);
        if (u[0] < L.eps) {
          for (int j = 0; j < 4; ++j)
            jact[j] = kth_allowed((unsigned)o.op_mask[j], (int)(pick[j] % (unsigned)__popc((unsigned)o.op_mask[j])));
          expl = 1;
          done = true;
        }
      } else {
        int near = 0;
        for (int m = 1; m < o.r_bins; ++m) near |= fabs(rho / o.thr[m] - 1.0) <= o.edge_tol ? 1 : 0;
        st->near_edge += near;
        if (P.visits && o.fallback_fmt >= 0 && o.fallback_idx >= 0 && P.visits[s] == 0) {
          bool all = true;
          for (int j = 0; j < 4; ++j) all = all && (((unsigned)o.op_mask[j] >> o.fallback_idx) & 1u);
          if (all) {
            for (int j = 0; j < 4; ++j) jact[j] = o.fallback_idx;
            done = true;
          }
        }
      }
      if (!done) {
        const int np4 = o.nprec * o.nprec * o.nprec * o.nprec;
        const double* row = (L.train ? S.Qpriv : P.Q) + (long long)s * np4;
        int best = -1;
        for (int a = 0; a < np4; ++a)
          if (joint_allowed(a, o.nprec, o.op_mask) && (best < 0 || row[a] > row[best])) best = a;
        for (int j = 3; j >= 0; --j) {
          jact[j] = best % o.nprec;
          best /= o.nprec;
        }
      }
    }
    for (int j = 0; j < 4; ++j) {
      int fmt, act = -1;
      if (st->fp64_lock) {
        fmt = F64;
      } else if (P.kind == 2 && o.joint) {
        act = jact[j];
        fmt = o.precs[act];
      } else if (P.kind == 0) {
        fmt = P.fixed[j];
      } else if (P.kind == 1) {
        const int row = k < P.sched_len ? k : P.sched_len - 1;
        fmt = P.sched[row * 4 + j];
      } else {
        const unsigned mask = (unsigned)o.op_mask[j];
        if (P.kind == 2) {
          const double* Qsrc = L.train ? S.Qpriv : P.Q;
          const double* row = Qsrc + ((long long)j * (o.b_bins * o.r_bins) + s) * o.nprec;
          act = row_argmax(row, o.nprec, mask);
          if (!L.train && j == 0) {  // one count per decision: rho within edge_tol of a bin edge
            int near = 0;
            for (int m = 1; m < o.r_bins; ++m) near |= fabs(rho / o.thr[m] - 1.0) <= o.edge_tol ? 1 : 0;
            st->near_edge += near;
          }
          if (!L.train && P.visits && o.fallback_fmt >= 0 && o.fallback_idx >= 0 && ((mask >> o.fallback_idx) & 1u) &&
              P.visits[j * (o.b_bins * o.r_bins) + s] == 0)
            act = o.fallback_idx;
        } else {
          int b = -1;
          for (int a = 0; a < o.nprec; ++a)
            if ((mask >> a) & 1u)
              if (b < 0 || sm.out[j * o.nprec + a] > sm.out[j * o.nprec + b]) b = a;
          act = b;
        }
        if (L.train) {
          double u;
          unsigned pick;
          policy_draw(L, S, k, j, u, pick);
          if (u < L.eps) {
            act = kth_allowed(mask, (int)(pick % (unsigned)__popc(mask)));
            expl = 1;
          }
        }
        fmt = o.precs[act];
      }
      if (act < 0)
        for (int a = 0; a < o.nprec; ++a)
          if (o.precs[a] == fmt) { act = a; break; }
      sm.a_fmt[j] = fmt;
      sm.a_act[j] = act;
    }
    sm.a_expl = expl;
    sm.a_state = s;
  }
  __syncthreads();
}

// ----------------------------------------------------------------------------------------
// Row phases
// ----------------------------------------------------------------------------------------

// M^-1 r_i in fp64: with IC(0) the element of the last application (ic_rows), with Jacobi
// r_i times the fp64 reciprocal of the diagonal (dinv set), r_i itself otherwise (M = I).
__device__ __forceinline__ double minv_r(const DevSys& S, int i, double ri) {
  if (S.icw) return (double)__uint_as_float((unsigned)__ldcg(S.icw + i));
  return S.A.dinv ? ri * __ldg(S.A.dinv + i) : ri;
}

// IC(0) application over the rows R in the phase with epoch ep (all CTAs that hold rows of
// the system run it in the same phase); consume(i, r_i, w_i) per row, w = M^-1 r.
template <class F>
__device__ __forceinline__ void ic_rows(const Launch& L, const DevSys& S, Rows R, unsigned ep, F&& consume) {
  ic_apply(S, R, ep, L.err, (unsigned)DERR_TIMEOUT, L.timeout_cycles, consume);
}


// sigma term of row i: fl_p4(r_i) fl_p4(z_i) with z_i = fl_p2(w_i), w_i = M^-1 r_i: a DFMA
// when p4 = fp64, otherwise the compensated fp32 pair. Roundings that are identities
// (p4's value set contains p2's) are skipped.
__device__ __forceinline__ void sigma_term(double ri, double wi, int p2, int p4, DotAcc& sg) {
  if (p4 == F64) {
    const double z = (p2 == F64) ? wi : f2d(round_d2f(wi, p2));
    sg.d = fma(ri, z, sg.d);
  } else {
    const float a = round_d2f(ri, p4);
    float b;
    // z_i = r_i (M = I): compared on the bit patterns, an integer test (an fp64 comparison
    // would take the narrow fp64 pipe once per row)
    if (__double_as_longlong(wi) == __double_as_longlong(ri) && (p2 == F64 || base_fmt(p2) == base_fmt(p4))) b = a;
    else if (p2 == F64) b = round_d2f(wi, p4);
    else {
      const float zf = round_d2f(wi, p2);
      b = contains_fmt(p4, p2) ? zf : round_f2f(zf, p4);
    }
    dot_low(sg, a, b, p4);
  }
}

// z = fl_p2(w) as fp64, w = M^-1 r.
__device__ __forceinline__ double z_of(double wi, int p2) { return p2 == F64 ? wi : f2d(round_d2f(wi, p2)); }

// The IC(0) applications of the solver phases, out of line so that the preconditioner's
// code does not enter the register allocation of the unpreconditioned phases. With copy_p
// the direction becomes p = w and sg.d collects r^T w in fp64; with p2 >= 0 sg collects
// the sigma terms of z = fl_p2(w).
__device__ __noinline__ void ic_phase(const Launch& L, const DevSys& S, Rows R, unsigned ep, int p2, int p4,
                                      bool copy_p, DotAcc& sg) {
  DotAcc acc = sg;
  ic_rows(L, S, R, ep, [&](int i, double ri, double wi) {
    if (copy_p) {
      S.p[i] = wi;
      acc.d = fma(ri, wi, acc.d);
    }
    if (p2 >= 0) sigma_term(ri, wi, p2, p4, acc);
  });
  sg = acc;
}

// Element i of q (stored in p1's format) as fp64, times 2^e_i for the row-scaled formats.
__device__ __forceinline__ double load_q(const DevSys& S, int i, int p1) {
  double v;
  switch (store_of(p1)) {
    case ST_Q52: v = f2d(to_acc(((const q52_t*)S.q)[i])); break;
    case ST_HALF: v = f2d(__half2float(((const __half*)S.q)[i])); break;
    case ST_BF16: v = f2d(__bfloat162float(((const __nv_bfloat16*)S.q)[i])); break;
    case ST_FLOAT: v = f2d(((const float*)S.q)[i]); break;
    default: return ((const double*)S.q)[i];
  }
  return row_scaled(p1) ? scale2(v, __ldg(S.A.rexp + i)) : v;
}

// Stores fl_f(v) (f other than fp64) in the low-precision copy of p.
__device__ __forceinline__ void store_low(void* plow, int i, double v, int f) {
  const float r = round_d2f(v, f);
  switch (store_of(f)) {
    case ST_Q52: ((q52_t*)plow)[i] = q52_from_exact(r); break;
    case ST_HALF: ((__half*)plow)[i] = __float2half_rn(r); break;
    case ST_BF16: ((__nv_bfloat16*)plow)[i] = __float2bfloat16_rn(r); break;
    default: ((float*)plow)[i] = r; break;
  }
}

// r = b - A x in fp64 (residual recomputation), with ||r||^2 and, when p2 >= 0, sigma partials.
// With copy_p the new residual is also written to p (warm-start initialisation).
template <int K, bool IC>
__device__ void true_res_vec(const DevSys& S, Rows R, int p2, int p4, bool copy_p, double& rr, DotAcc& sg) {
  constexpr int NG = kThreads / K;
  const int lane = threadIdx.x & (K - 1);
  const int grp = threadIdx.x / K;
  const unsigned mask = (K == 32) ? kFull : (((1u << K) - 1u) << ((threadIdx.x & 31) & ~(K - 1)));
  const int* __restrict__ rp = S.A.rp;
  const int* __restrict__ ci = S.A.ci;
  const double* __restrict__ v = S.A.v64;
  for (int row = R.r0 + grp; row < R.r1; row += NG) {
    const int e0 = __ldg(rp + row), e1 = __ldg(rp + row + 1);
    double acc = 0.0;
    for (int e = e0 + lane; e < e1; e += K) acc = fma(__ldg(v + e), S.x[__ldg(ci + e)], acc);
#pragma unroll
    for (int o = K / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(mask, acc, o);
    if (lane == 0) {
      const double ri = __ldg(S.b + row) - acc;
      S.r[row] = ri;
      rr = fma(ri, ri, rr);
      if (!(IC && S.icw)) {  // with IC(0), M^-1 r needs every row of r first (true_res_rows)
        const double wi = minv_r(S, row, ri);
        if (copy_p) {  // restart direction p = M^-1 r, sigma = r^T M^-1 r in fp64
          S.p[row] = wi;
          sg.d = fma(ri, wi, sg.d);
        }
        if (p2 >= 0) sigma_term(ri, wi, p2, p4, sg);
      }
    }
  }
}

// ep: the phase's IC(0) epoch (used when the launch preconditions with IC(0) and the
// caller wants M^-1 r: copy_p or p2 >= 0).
template <bool IC>
__device__ void true_res_rows(const Launch& L, const DevSys& S, Rows R, int p2, int p4, bool copy_p, double& rr,
                              DotAcc& sg, unsigned ep) {
  switch (S.A.lanes[F64]) {
    case 1: true_res_vec<1, IC>(S, R, p2, p4, copy_p, rr, sg); break;
    case 2: true_res_vec<2, IC>(S, R, p2, p4, copy_p, rr, sg); break;
    case 4: true_res_vec<4, IC>(S, R, p2, p4, copy_p, rr, sg); break;
    case 8: true_res_vec<8, IC>(S, R, p2, p4, copy_p, rr, sg); break;
    case 16: true_res_vec<16, IC>(S, R, p2, p4, copy_p, rr, sg); break;
    default: true_res_vec<32, IC>(S, R, p2, p4, copy_p, rr, sg); break;
  }
  if (IC && S.icw && (copy_p || p2 >= 0)) ic_phase(L, S, R, ep, p2, p4, copy_p, sg);
}

// ----------------------------------------------------------------------------------------
// Team steps (run by every thread of the CTA that arrived last)
// ----------------------------------------------------------------------------------------

__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Nanoseconds since the previous team barrier of this system (and restarts the clock).
__device__ __forceinline__ unsigned stamp(SysState* st) {
  const unsigned long long t = gtime();
  const unsigned long long d = t - st->t_last;
  st->t_last = t;
  return d > 0xffffffffull ? 0xffffffffu : (unsigned)d;
}

__device__ void write_record(const DevSys& S, SysState* st, int flags, double rho, double sigma, double beta,
                             double reward) {
  const int k = st->k;
  if (S.hist && k < S.hist_cap) {
    mpcg_iter_record rec;
    rec.k = k;
    rec.state = st->s_cur;
    for (int j = 0; j < 4; ++j) {
      rec.fmt[j] = (int8_t)st->fmt[j];
      rec.act[j] = (int8_t)st->act[j];
    }
    rec.rho = rho;
    rec.nu = st->nu;
    rec.alpha = st->alpha;
    rec.sigma = sigma;
    rec.beta = beta;
    rec.reward = reward;
    rec.flags = flags | (st->explored ? 8 : 0);
    rec.ns_a = st->ns_a;
    rec.ns_b = st->ns_b;
    rec.ns_c = 0;
    S.hist[k] = rec;
  }
}

__device__ void push_transition(const Launch& L, const DevSys& S, SysState* st, int s_next, double R,
                                int terminal) {
  if (!L.train) return;
  Transition t;
  t.s = st->s_cur;
  t.s_next = s_next;
  for (int j = 0; j < 4; ++j) t.act[j] = st->act[j];
  t.reward = R;
  t.terminal = terminal;
  t.pad = 0;
  if (L.pol.kind == 2 && S.Qpriv) q_update(S.Qpriv, L.opt, t);
  if (S.trans && st->ntrans < S.trans_cap) S.trans[st->ntrans] = t;
  st->ntrans += 1;
}

// Applies a chosen action (sm.a_*) as the action of iteration st->k.
__device__ void adopt_action(SysState* st, const Smem& sm) {
  for (int j = 0; j < 4; ++j) {
    st->fmt[j] = sm.a_fmt[j];
    st->act[j] = sm.a_act[j];
    st->counts[j][sm.a_fmt[j] & 7] += 1;
  }
  st->explored = sm.a_expl;
  st->s_cur = sm.a_state;
}

// A breakdown of an inference solve restarts in fp64 when the option asks for it (once).
__device__ __forceinline__ bool restart_ok(const Launch& L, const SysState* st) {
  return !L.train && L.opt.on_breakdown && !st->fp64_lock;
}

// After the initial phase: ||b||, rho_0, sigma_0 = r_0^T r_0, action of iteration 0.
__device__ void step_init(const Launch& L, const DevSys& S, SysState* st, double bb, double rr, double sig,
                          Smem& sm) {
  if (threadIdx.x == 0) {
    const double bnorm = sqrt(bb);
    st->bnorm = bnorm;
    st->rho = bnorm > 0.0 ? sqrt(rr) / bnorm : 0.0;
    st->sigma = sig;
    st->k = 0;
    st->icep = 0u;  // the phase after initialisation applies IC(0) with epoch 1
    st->alpha = 0.0;
    st->beta = 0.0;
    st->nu = 0.0;
    st->rho_true = 0.0;
    for (int h = 0; h < 9; ++h) st->rho_hist[h] = 0.0;
    st->rho_hist[0] = st->rho;
    st->alpha_prev = st->beta_prev = st->gap_log = 0.0;
    st->have_prev = 0;
    st->n_true = 0;
    st->ntrans = 0;
    st->true_known = 0;
    st->explored = 0;
    st->s_cur = 0;
    st->zfmt = F64;
    st->fp64_lock = 0;
    st->n_restart = 0;
    st->ns_a = st->ns_b = 0;
    st->near_edge = 0;
    st->restart_sr = 1;  // the single-reduction recurrence starts with beta = 0
    st->sr_gamma = st->sr_alpha = 0.0;
    st->t_last = gtime();
    for (int j = 0; j < 4; ++j) {
      st->prev_act[j] = 0;
      for (int f = 0; f < 8; ++f) st->counts[j][f] = 0;
    }
    sm.need_action = 0;
    if (S.A.n == 0 || bnorm == 0.0) {
      st->outcome = MPCG_CONVERGED;
      st->iters = 0;
      st->rho = 0.0;
      st->rho_true = 0.0;
      st->true_known = 1;
      st->mode = M_DONE;
    } else if (S.max_iter <= 0) {
      st->outcome = MPCG_MAX_ITER;
      st->iters = 0;
      st->mode = M_DONE;
    } else {
      st->mode = M_CONT;
      sm.need_action = 1;
    }
  }
  __syncthreads();
  if (sm.need_action) {
    choose_action(L, S, st, 0, st->rho, sm);
    if (threadIdx.x == 0) adopt_action(st, sm);
  }
}

// After phase A: nu = fl_p3(sum), alpha = sigma / nu, curvature breakdown test.
__device__ void step_A(const Launch& L, const DevSys& S, SysState* st, double nu_sum) {
  if (threadIdx.x != 0) return;
  st->ns_a = stamp(st);
  st->ns_b = 0;
  const int p3 = st->fmt[2];
  const double nu = (p3 == F64) ? nu_sum : round_fmt(nu_sum, p3);
  const double alpha = st->sigma / nu;
  st->nu = nu;
  st->alpha = alpha;
  if (!(nu > 0.0) || !isfinite(nu) || !isfinite(alpha)) {
    const int k = st->k;
    if (st->rho < S.tol && isfinite(nu)) {
      // The residual is already below tol (exact solution reached before k >= min_k).
      st->outcome = MPCG_CONVERGED;
      const double R = !L.train ? 0.0 : reward_of(L.opt, st->rho, st->act, S.tol, false);
      write_record(S, st, 1, st->rho, 0.0, 0.0, L.train ? R : 0.0);
      push_transition(L, S, st, st->s_cur, R, 1);
    } else if (restart_ok(L, st)) {
      write_record(S, st, 2 | 16, st->rho, 0.0, 0.0, 0.0);
      st->mode = M_RESTART64;
      return;
    } else {
      st->outcome = MPCG_BREAKDOWN;
      const double R = !L.train ? 0.0 : reward_of(L.opt, st->rho, st->act, S.tol, true);
      write_record(S, st, 2, st->rho, 0.0, 0.0, L.train ? R : 0.0);
      push_transition(L, S, st, st->s_cur, R, 1);
    }
    st->iters = k;
    st->mode = M_DONE;
  } else {
    st->mode = M_CONT;
  }
}

// Continues after the residual of iteration k is known (recursive, or replaced when
// `replaced`): sigma_{k+1}, beta_k (0 after a replacement), reward, next state and action.
__device__ void continue_step(const Launch& L, const DevSys& S, SysState* st, double rho_new, double sig_sum,
                              int replaced, Smem& sm) {
  if (threadIdx.x == 0) {
    sm.need_action = 0;
    const int p4 = st->fmt[3];
    const double sigma_new = (p4 == F64) ? sig_sum : round_fmt(sig_sum, p4);
    const double beta = replaced ? 0.0 : sigma_new / st->sigma;
    const int k = st->k;
    const int flags = replaced ? 4 : 0;
    if ((!isfinite(sigma_new) || !isfinite(beta)) && restart_ok(L, st)) {
      write_record(S, st, flags | 2 | 16, rho_new, sigma_new, beta, 0.0);
      st->mode = replaced ? M_RESTART64 : M_X_THEN_RESTART64;
    } else if (!isfinite(sigma_new) || !isfinite(beta)) {
      st->outcome = MPCG_BREAKDOWN;
      st->iters = k + 1;
      const double R = !L.train ? 0.0 : reward_of(L.opt, rho_new, st->act, S.tol, true);
      write_record(S, st, flags | 2, rho_new, sigma_new, beta, L.train ? R : 0.0);
      push_transition(L, S, st, st->s_cur, R, 1);
      st->rho = rho_new;
      st->mode = replaced ? M_DONE : M_X_THEN_DONE;
    } else {
      const int s_next = state_of(L.opt, k + 1, rho_new);
      const double R = !L.train ? 0.0 : reward_of(L.opt, rho_new, st->act, S.tol, false);
      write_record(S, st, flags, rho_new, sigma_new, beta, L.train ? R : 0.0);
      push_transition(L, S, st, s_next, R, 0);
      for (int h = 8; h > 0; --h) st->rho_hist[h] = st->rho_hist[h - 1];
      st->rho_hist[0] = rho_new;
      st->alpha_prev = st->alpha;
      st->beta_prev = beta;
      st->have_prev = 1;
      for (int j = 0; j < 4; ++j) st->prev_act[j] = st->act[j] >= 0 ? st->act[j] : 0;
      st->sigma = sigma_new;
      st->beta = beta;
      st->rho = rho_new;
      st->zfmt = st->fmt[1];
      st->k = k + 1;
      st->mode = replaced ? M_RESTART : M_CONT;
      if (k + 1 >= S.max_iter) {
        st->outcome = MPCG_MAX_ITER;
        st->iters = S.max_iter;
        if (S.feat_log && k + 1 < S.feat_cap) {  // the bootstrap state of the last transition
          mlp_features(L, S, st, k + 1, sm);
          for (int j = 0; j < kNFeat; ++j) S.feat_log[(long long)(k + 1) * kNFeat + j] = sm.feat[j];
        }
      } else {
        sm.need_action = 1;
      }
    }
  }
  __syncthreads();
  if (sm.need_action) {
    choose_action(L, S, st, st->k, st->rho, sm);
    if (threadIdx.x == 0) adopt_action(st, sm);
  }
}

// Single-reduction iteration: continues after the residual norm of iteration k's end is known
// (from the recurrence, or recomputed when `replaced`): record, reward, transition, next state
// and action. gamma and alpha of iteration k become the recurrence's previous values; a
// replaced residual restarts the recurrence (beta = 0 next).
__device__ void continue_sr(const Launch& L, const DevSys& S, SysState* st, double rho_new, int replaced, Smem& sm) {
  if (threadIdx.x == 0) {
    sm.need_action = 0;
    const int k = st->k;
    const int s_next = state_of(L.opt, k + 1, rho_new);
    const double R = !L.train ? 0.0 : reward_of(L.opt, rho_new, st->act, S.tol, false);
    write_record(S, st, replaced ? 4 : 0, rho_new, st->sigma, st->beta, L.train ? R : 0.0);
    push_transition(L, S, st, s_next, R, 0);
    for (int h = 8; h > 0; --h) st->rho_hist[h] = st->rho_hist[h - 1];
    st->rho_hist[0] = rho_new;
    st->alpha_prev = st->alpha;
    st->beta_prev = st->beta;
    st->have_prev = 1;
    for (int j = 0; j < 4; ++j) st->prev_act[j] = st->act[j] >= 0 ? st->act[j] : 0;
    st->sr_gamma = st->sigma;
    st->sr_alpha = st->alpha;
    st->restart_sr = replaced;
    st->rho = rho_new;
    st->k = k + 1;
    st->mode = replaced ? M_RESTART : M_CONT;
    if (k + 1 >= S.max_iter) {
      st->outcome = MPCG_MAX_ITER;
      st->iters = S.max_iter;
      if (S.feat_log && k + 1 < S.feat_cap) {
        mlp_features(L, S, st, k + 1, sm);
        for (int j = 0; j < kNFeat; ++j) S.feat_log[(long long)(k + 1) * kNFeat + j] = sm.feat[j];
      }
    } else {
      sm.need_action = 1;
    }
  }
  __syncthreads();
  if (sm.need_action) {
    choose_action(L, S, st, st->k, st->rho, sm);
    if (threadIdx.x == 0) adopt_action(st, sm);
  }
}

// After the single-reduction product phase W: gamma = fl_p4(sum), delta = fl_p3(sum), then in
// fp64 beta = gamma / gamma_prev, nu = delta - beta gamma / alpha_prev (beta = 0, nu = delta
// at a restart), alpha = gamma / nu; breakdown tests as after phase A; the next residual norm
// rr - 2 alpha (r.w + beta r.s) + alpha^2 (w.w + 2 beta w.s + beta^2 s.s) (clamped at 0) and the
// stopping tests as after phase B. dots = r.r, r.w, r.s, w.w, w.s, s.s (fp64 sums).
__device__ void step_W(const Launch& L, const DevSys& S, SysState* st, double gsum, double dsum, const double* dots,
                       Smem& sm) {
  if (threadIdx.x == 0) {
    st->ns_a = stamp(st);
    st->ns_b = 0;
    sm.flag = 0;
    const OptView& o = L.opt;
    const int k = st->k;
    const int p3 = st->fmt[2], p4 = st->fmt[3];
    const double gamma = (p4 == F64) ? gsum : round_fmt(gsum, p4);
    const double delta = (p3 == F64) ? dsum : round_fmt(dsum, p3);
    const bool rs = st->restart_sr != 0;
    const double beta = rs ? 0.0 : gamma / st->sr_gamma;
    const double nu = rs ? delta : delta - beta * gamma / st->sr_alpha;
    const double alpha = gamma / nu;
    st->nu = nu;
    st->alpha = alpha;
    st->beta = beta;
    st->sigma = gamma;
    st->wfmt = st->fmt[0];
    st->zfmt = st->fmt[1];
    if (!(nu > 0.0) || !isfinite(nu) || !isfinite(alpha) || !isfinite(beta)) {
      if (st->rho < S.tol && isfinite(nu)) {
        st->outcome = MPCG_CONVERGED;
        const double R = !L.train ? 0.0 : reward_of(o, st->rho, st->act, S.tol, false);
        write_record(S, st, 1, st->rho, gamma, beta, L.train ? R : 0.0);
        push_transition(L, S, st, st->s_cur, R, 1);
        st->iters = k;
        st->mode = M_DONE;
      } else if (restart_ok(L, st)) {
        write_record(S, st, 2 | 16, st->rho, gamma, beta, 0.0);
        st->mode = M_RESTART64;
      } else {
        st->outcome = MPCG_BREAKDOWN;
        const double R = !L.train ? 0.0 : reward_of(o, st->rho, st->act, S.tol, true);
        write_record(S, st, 2, st->rho, gamma, beta, L.train ? R : 0.0);
        push_transition(L, S, st, st->s_cur, R, 1);
        st->iters = k;
        st->mode = M_DONE;
      }
    } else {
      double rr = dots[0] - 2.0 * alpha * (dots[1] + beta * dots[2]) +
                  alpha * alpha * (dots[3] + 2.0 * beta * dots[4] + beta * beta * dots[5]);
      if (rr < 0.0) rr = 0.0;
      const double rho_rec = sqrt(rr) / st->bnorm;
      const bool check = (o.true_every > 0 && (k + 1) % o.true_every == 0) ||
                         (o.true_at_conv && rho_rec < S.tol && k >= o.min_k);
      if (check && isfinite(rho_rec)) {
        st->rho_true = rho_rec;
        st->mode = M_TCHK;
      } else if (!isfinite(rho_rec) && restart_ok(L, st)) {
        write_record(S, st, 2 | 16, rho_rec, gamma, beta, 0.0);
        st->mode = M_X_THEN_RESTART64;
      } else if (!isfinite(rho_rec)) {
        st->outcome = MPCG_BREAKDOWN;
        st->iters = k + 1;
        const double R = !L.train ? 0.0 : reward_of(o, rho_rec, st->act, S.tol, true);
        write_record(S, st, 2, rho_rec, gamma, beta, L.train ? R : 0.0);
        push_transition(L, S, st, st->s_cur, R, 1);
        st->rho = rho_rec;
        st->mode = M_X_THEN_DONE;
      } else if (rho_rec < S.tol && k >= o.min_k) {
        st->outcome = MPCG_CONVERGED;
        st->iters = k + 1;
        const double R = !L.train ? 0.0 : reward_of(o, rho_rec, st->act, S.tol, false);
        write_record(S, st, 1, rho_rec, gamma, beta, L.train ? R : 0.0);
        push_transition(L, S, st, st->s_cur, R, 1);
        st->rho = rho_rec;
        st->mode = M_X_THEN_DONE;
      } else {
        sm.flag = 1;
        sm.tmp = rho_rec;
      }
    }
  }
  __syncthreads();
  if (sm.flag) continue_sr(L, S, st, sm.tmp, 0, sm);
}

// After phase B: rho_{k+1} of the recursive residual, stopping tests.
__device__ void step_B(const Launch& L, const DevSys& S, SysState* st, double rr, double sig_sum, Smem& sm) {
  if (threadIdx.x == 0) {
    st->ns_b = stamp(st);
    sm.need_action = 0;
    const double rho_rec = sqrt(rr) / st->bnorm;
    const OptView& o = L.opt;
    const int k = st->k;
    const bool check = (o.true_every > 0 && (k + 1) % o.true_every == 0) ||
                       (o.true_at_conv && rho_rec < S.tol && k >= o.min_k);
    sm.flag = 0;
    if (check && isfinite(rho_rec)) {
      st->rho_true = rho_rec;  // recursive value, kept for the gap feature
      st->mode = M_TCHK;
    } else if (!isfinite(rho_rec) && restart_ok(L, st)) {
      write_record(S, st, 2 | 16, rho_rec, 0.0, 0.0, 0.0);
      st->mode = M_X_THEN_RESTART64;
    } else if (!isfinite(rho_rec)) {
      st->outcome = MPCG_BREAKDOWN;
      st->iters = k + 1;
      const double R = !L.train ? 0.0 : reward_of(o, rho_rec, st->act, S.tol, true);
      write_record(S, st, 2, rho_rec, 0.0, 0.0, L.train ? R : 0.0);
      push_transition(L, S, st, st->s_cur, R, 1);
      st->rho = rho_rec;
      st->mode = M_X_THEN_DONE;
    } else if (rho_rec < S.tol && k >= o.min_k) {
      st->outcome = MPCG_CONVERGED;
      st->iters = k + 1;
      const double R = !L.train ? 0.0 : reward_of(o, rho_rec, st->act, S.tol, false);
      write_record(S, st, 1, rho_rec, 0.0, 0.0, L.train ? R : 0.0);
      push_transition(L, S, st, st->s_cur, R, 1);
      st->rho = rho_rec;
      st->mode = M_X_THEN_DONE;
    } else {
      sm.flag = 1;
    }
  }
  __syncthreads();
  if (sm.flag) continue_step(L, S, st, sqrt(rr) / st->bnorm, sig_sum, 0, sm);
}

// After a residual recomputation inside the iteration (phase T).
__device__ void step_T(const Launch& L, const DevSys& S, SysState* st, double rr, double sig_sum, Smem& sm) {
  if (threadIdx.x == 0) {
    const double rho_t = sqrt(rr) / st->bnorm;
    const double rho_rec = st->rho_true;
    st->n_true += 1;
    st->gap_log = (rho_t > 0.0 && rho_rec > 0.0) ? log10(rho_t / rho_rec) : 0.0;
    const int k = st->k;
    sm.flag = 0;
    if (!isfinite(rho_t) && restart_ok(L, st)) {
      write_record(S, st, 4 | 2 | 16, rho_t, 0.0, 0.0, 0.0);
      st->mode = M_RESTART64;
    } else if (!isfinite(rho_t)) {
      st->outcome = MPCG_BREAKDOWN;
      st->iters = k + 1;
      const double R = !L.train ? 0.0 : reward_of(L.opt, rho_t, st->act, S.tol, true);
      write_record(S, st, 4 | 2, rho_t, 0.0, 0.0, L.train ? R : 0.0);
      push_transition(L, S, st, st->s_cur, R, 1);
      st->rho = rho_t;
      st->rho_true = rho_t;
      st->true_known = 1;
      st->mode = M_DONE;
    } else if (rho_t < S.tol && k >= L.opt.min_k) {
      st->outcome = MPCG_CONVERGED;
      st->iters = k + 1;
      const double R = !L.train ? 0.0 : reward_of(L.opt, rho_t, st->act, S.tol, false);
      write_record(S, st, 4 | 1, rho_t, 0.0, 0.0, L.train ? R : 0.0);
      push_transition(L, S, st, st->s_cur, R, 1);
      st->rho = rho_t;
      st->rho_true = rho_t;
      st->true_known = 1;
      st->mode = M_DONE;
    } else {
      sm.flag = 1;
    }
  }
  __syncthreads();
  if (sm.flag) {
    if (L.opt.variant) continue_sr(L, S, st, sqrt(rr) / st->bnorm, 1, sm);
    else continue_step(L, S, st, sqrt(rr) / st->bnorm, sig_sum, 1, sm);
  }
}

// After the fp64 restart's residual recomputation (r = b - A x, p = r): iteration k counts
// as done; sigma = ||r||^2, every later operation in fp64; stop test as after any iteration.
__device__ void step_restart(const Launch& L, const DevSys& S, SysState* st, double rr, double sig, Smem& sm) {
  if (threadIdx.x == 0) {
    sm.need_action = 0;
    const double rho = sqrt(rr) / st->bnorm;
    const int k = st->k;
    st->fp64_lock = 1;
    st->n_restart += 1;
    st->n_true += 1;
    st->restart_sr = 1;  // the single-reduction recurrence restarts with beta = 0
    st->sigma = sig;
    st->beta = 0.0;
    st->rho = rho;
    for (int h = 8; h > 0; --h) st->rho_hist[h] = st->rho_hist[h - 1];
    st->rho_hist[0] = rho;
    st->zfmt = F64;
    st->k = k + 1;
    if (!isfinite(rho)) {
      st->outcome = MPCG_BREAKDOWN;
      st->iters = k + 1;
      st->rho_true = rho;
      st->true_known = 1;
      st->mode = M_DONE;
    } else if (rho < S.tol && k >= L.opt.min_k) {
      st->outcome = MPCG_CONVERGED;
      st->iters = k + 1;
      st->rho_true = rho;
      st->true_known = 1;
      st->mode = M_DONE;
    } else if (k + 1 >= S.max_iter) {
      st->outcome = MPCG_MAX_ITER;
      st->iters = S.max_iter;
      st->mode = M_DONE;
    } else {
      st->mode = M_CONT;
      sm.need_action = 1;
    }
  }
  __syncthreads();
  if (sm.need_action) {
    choose_action(L, S, st, st->k, st->rho, sm);
    if (threadIdx.x == 0) adopt_action(st, sm);
  }
}

__device__ void step_final(const Launch& L, const DevSys& S, SysState* st, int sid, double rr) {
  if (threadIdx.x != 0) return;
  if (!st->true_known) st->rho_true = st->bnorm > 0.0 ? sqrt(rr) / st->bnorm : 0.0;
  mpcg_result res;
  res.outcome = st->outcome;
  res.iters = st->iters;
  res.rel_res_rec = st->rho;
  res.rel_res_true = st->rho_true;
  res.n_true_checks = st->n_true;
  res.n_restarts = st->n_restart;
  for (int j = 0; j < 4; ++j)
    for (int f = 0; f < 8; ++f) res.action_hist[j][f] = st->counts[j][f];
  res.near_edge_count = st->near_edge;
  res.kernel_launches = 0;
  L.res[sid] = res;
}

// ----------------------------------------------------------------------------------------
// One system, solved by one team
// ----------------------------------------------------------------------------------------

// Barrier plus team work: `work` runs in all threads of the last CTA.
template <class F>
__device__ __forceinline__ bool team_step(const Launch& L, const TeamCtx& T, SysState* st, Smem& sm, F&& work) {
  const bool last = team_arrive(T, sm);
  bool ok = true;
  if (last) {
    work();
    if (threadIdx.x == 0) st->icep += 1u;
    team_release(T);
  } else {
    ok = team_wait(L, T, sm);
  }
  if (ok) load_bcast(st, sm);
  return ok;
}

// Stage-C stamp: phase C of the finished iteration closes at this barrier.
__device__ __forceinline__ void stamp_c(const DevSys& S, SysState* st) {
  if (threadIdx.x == 0) {
    const unsigned d = stamp(st);
    const int kd = st->k - 1;
    if (S.hist && kd >= 0 && kd < S.hist_cap) S.hist[kd].ns_c = d;
  }
}

constexpr int kUnroll = 4;  // rows per thread in flight in the vector phases

// Storage types of q (phase B) and of p's low copy (phase C), one instantiation each, so that
// the loads of a thread's kUnroll rows are issued together before any use.
template <typename T>
__device__ __forceinline__ double stored_as_double(T v) {
  if constexpr (sizeof(T) == 8) return v;
  else return f2d(to_acc(v));
}
template <typename T>
__device__ __forceinline__ T to_storage(float v);
template <>
__device__ __forceinline__ float to_storage<float>(float v) { return v; }
template <>
__device__ __forceinline__ __half to_storage<__half>(float v) { return __float2half_rn(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 to_storage<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <>
__device__ __forceinline__ q52_t to_storage<q52_t>(float v) { return q52_from_exact(v); }

// Phase B rows: r -= alpha q (fp64), ||r||^2 (fp64) and, unless sigma is ||r||^2 itself,
// the sigma terms. QT: storage of q; SCALED: q carries the row scale 2^e_i.
template <typename QT, bool SCALED>
__device__ __forceinline__ void phase_b_rows(const DevSys& S, Rows R, double alpha, int p2, int p4, bool sig_rr,
                                             double& rr, DotAcc& sg) {
  const QT* __restrict__ q = (const QT*)S.q;
  for (int i0 = R.r0 + threadIdx.x; i0 < R.r1; i0 += kUnroll * kThreads) {
    QT qv[kUnroll];
    double ro[kUnroll];
    short ev[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int i = i0 + u * kThreads;
      if (i < R.r1) {
        qv[u] = q[i];
        ro[u] = S.r[i];
        if constexpr (SCALED) ev[u] = __ldg(S.A.rexp + i);
      }
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int i = i0 + u * kThreads;
      if (i < R.r1) {
        double qd = stored_as_double(qv[u]);
        if constexpr (SCALED) qd = scale2(qd, ev[u]);
        const double ri = fma(-alpha, qd, ro[u]);
        S.r[i] = ri;
        rr = fma(ri, ri, rr);
        if (!sig_rr) sigma_term(ri, minv_r(S, i, ri), p2, p4, sg);
      }
    }
  }
}

// Phase C rows: x += alpha p; p = z + beta p (fp64) with z = fl_p2(r); p's copy in the next
// product's format p1n, stored as PT (PT = double: no copy, the next product is fp64).
template <typename PT>
__device__ __forceinline__ void phase_c_rows(const DevSys& S, Rows R, double alpha, double beta, int p2, int p1n) {
  const bool zlow = p2 != F64;
  for (int i0 = R.r0 + threadIdx.x; i0 < R.r1; i0 += kUnroll * kThreads) {
    double pv[kUnroll], xv[kUnroll], rv[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int i = i0 + u * kThreads;
      if (i < R.r1) {
        pv[u] = S.p[i];
        xv[u] = S.x[i];
        rv[u] = S.r[i];
      }
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int i = i0 + u * kThreads;
      if (i < R.r1) {
        S.x[i] = fma(alpha, pv[u], xv[u]);
        const double w = minv_r(S, i, rv[u]);
        const double z = zlow ? f2d(round_d2f(w, p2)) : w;
        const double pn = fma(beta, pv[u], z);
        S.p[i] = pn;
        if constexpr (sizeof(PT) != 8) ((PT*)S.plow)[i] = to_storage<PT>(round_d2f(pn, p1n));
      }
    }
  }
}

// Pair-vectorised variants: a thread takes rows 2j and 2j+1 with one 16-byte load of each
// fp64 vector (and one load of two q / p-copy elements); the odd first and last rows of the
// range go through the element-wise code. Used when every vector is 16-byte aligned.
template <typename T> struct PairOf;
template <> struct PairOf<double> { using type = double2; };
template <> struct PairOf<float> { using type = float2; };
template <> struct PairOf<__half> { using type = __half2; };
template <> struct PairOf<__nv_bfloat16> { using type = __nv_bfloat162; };
template <> struct PairOf<q52_t> { using type = q52x2_t; };

constexpr int kPairs = 2;  // row pairs per thread in flight

template <typename QT, bool SCALED>
__device__ __forceinline__ void phase_b_row(const DevSys& S, int i, double alpha, int p2, int p4, bool sig_rr,
                                            double& rr, DotAcc& sg) {
  double qd = stored_as_double(((const QT*)S.q)[i]);
  if constexpr (SCALED) qd = scale2(qd, __ldg(S.A.rexp + i));
  const double ri = fma(-alpha, qd, S.r[i]);
  S.r[i] = ri;
  rr = fma(ri, ri, rr);
  if (!sig_rr) sigma_term(ri, minv_r(S, i, ri), p2, p4, sg);
}

template <typename QT, bool SCALED>
__device__ __forceinline__ void phase_b_pairs(const DevSys& S, Rows R, double alpha, int p2, int p4, bool sig_rr,
                                              double& rr, DotAcc& sg) {
  using Q2 = typename PairOf<QT>::type;
  int a = R.r0, e = R.r1;
  if (a < e && (a & 1)) {
    if (threadIdx.x == 0) phase_b_row<QT, SCALED>(S, a, alpha, p2, p4, sig_rr, rr, sg);
    ++a;
  }
  if (a < e && (e & 1)) {
    if (threadIdx.x == 1) phase_b_row<QT, SCALED>(S, e - 1, alpha, p2, p4, sig_rr, rr, sg);
    --e;
  }
  const Q2* __restrict__ q2 = (const Q2*)S.q;
  double2* r2 = (double2*)S.r;
  const short2* e2 = (const short2*)S.A.rexp;
  const int j1 = e >> 1;
  for (int j0 = (a >> 1) + threadIdx.x; j0 < j1; j0 += kPairs * kThreads) {
    Q2 qv[kPairs];
    double2 ro[kPairs];
    short2 ev[kPairs];
#pragma unroll
    for (int u = 0; u < kPairs; ++u) {
      const int j = j0 + u * kThreads;
      if (j < j1) {
        qv[u] = q2[j];
        ro[u] = r2[j];
        if constexpr (SCALED) ev[u] = __ldg(e2 + j);
      }
    }
#pragma unroll
    for (int u = 0; u < kPairs; ++u) {
      const int j = j0 + u * kThreads;
      if (j < j1) {
        double qa = stored_as_double(qv[u].x), qb = stored_as_double(qv[u].y);
        if constexpr (SCALED) {
          qa = scale2(qa, ev[u].x);
          qb = scale2(qb, ev[u].y);
        }
        double2 rn;
        rn.x = fma(-alpha, qa, ro[u].x);
        rn.y = fma(-alpha, qb, ro[u].y);
        r2[j] = rn;
        rr = fma(rn.x, rn.x, rr);
        rr = fma(rn.y, rn.y, rr);
        if (!sig_rr) {
          sigma_term(rn.x, minv_r(S, 2 * j, rn.x), p2, p4, sg);
          sigma_term(rn.y, minv_r(S, 2 * j + 1, rn.y), p2, p4, sg);
        }
      }
    }
  }
}

template <typename PT>
__device__ __forceinline__ void phase_c_row(const DevSys& S, int i, double alpha, double beta, int p2, int p1n) {
  const double pv = S.p[i];
  S.x[i] = fma(alpha, pv, S.x[i]);
  const double rv = S.r[i];
  const double w = minv_r(S, i, rv);
  const double z = p2 != F64 ? f2d(round_d2f(w, p2)) : w;
  const double pn = fma(beta, pv, z);
  S.p[i] = pn;
  if constexpr (sizeof(PT) != 8) ((PT*)S.plow)[i] = to_storage<PT>(round_d2f(pn, p1n));
}

template <typename PT>
__device__ __forceinline__ void phase_c_pairs(const DevSys& S, Rows R, double alpha, double beta, int p2, int p1n) {
  const bool zlow = p2 != F64;
  int a = R.r0, e = R.r1;
  if (a < e && (a & 1)) {
    if (threadIdx.x == 0) phase_c_row<PT>(S, a, alpha, beta, p2, p1n);
    ++a;
  }
  if (a < e && (e & 1)) {
    if (threadIdx.x == 1) phase_c_row<PT>(S, e - 1, alpha, beta, p2, p1n);
    --e;
  }
  double2* p2v = (double2*)S.p;
  double2* x2v = (double2*)S.x;
  const double2* r2v = (const double2*)S.r;
  const int j1 = e >> 1;
  for (int j0 = (a >> 1) + threadIdx.x; j0 < j1; j0 += kPairs * kThreads) {
    double2 pv[kPairs], xv[kPairs], rv[kPairs];
#pragma unroll
    for (int u = 0; u < kPairs; ++u) {
      const int j = j0 + u * kThreads;
      if (j < j1) {
        pv[u] = p2v[j];
        xv[u] = x2v[j];
        rv[u] = r2v[j];
      }
    }
#pragma unroll
    for (int u = 0; u < kPairs; ++u) {
      const int j = j0 + u * kThreads;
      if (j < j1) {
        double2 xn, pn;
        xn.x = fma(alpha, pv[u].x, xv[u].x);
        xn.y = fma(alpha, pv[u].y, xv[u].y);
        x2v[j] = xn;
        const double wa = minv_r(S, 2 * j, rv[u].x), wb = minv_r(S, 2 * j + 1, rv[u].y);
        const double za = zlow ? f2d(round_d2f(wa, p2)) : wa;
        const double zb = zlow ? f2d(round_d2f(wb, p2)) : wb;
        pn.x = fma(beta, pv[u].x, za);
        pn.y = fma(beta, pv[u].y, zb);
        p2v[j] = pn;
        if constexpr (sizeof(PT) != 8) {
          typename PairOf<PT>::type lw;
          lw.x = to_storage<PT>(round_d2f(pn.x, p1n));
          lw.y = to_storage<PT>(round_d2f(pn.y, p1n));
          ((typename PairOf<PT>::type*)S.plow)[j] = lw;
        }
      }
    }
  }
}

__device__ __forceinline__ bool aligned16(const void* a, const void* b, const void* c) {
  return ((reinterpret_cast<unsigned long long>(a) | reinterpret_cast<unsigned long long>(b) |
           reinterpret_cast<unsigned long long>(c)) & 15ull) == 0ull;
}

// Row phases B and C, out of line (one register allocation each, as for the product).
__device__ __noinline__ void phase_b(const DevSys& S, Rows R, double alpha, int p1, int p2, int p4, bool sig_rr,
                                     double& rr, DotAcc& sg) {
  if (aligned16(S.r, S.q, S.r)) {
    switch (p1) {
      case F64: phase_b_pairs<double, false>(S, R, alpha, p2, p4, sig_rr, rr, sg); return;
      case F32:
      case TF32: phase_b_pairs<float, false>(S, R, alpha, p2, p4, sig_rr, rr, sg); return;
      case F16: phase_b_pairs<__half, false>(S, R, alpha, p2, p4, sig_rr, rr, sg); return;
      case BF16: phase_b_pairs<__nv_bfloat16, false>(S, R, alpha, p2, p4, sig_rr, rr, sg); return;
      case F16R: phase_b_pairs<__half, true>(S, R, alpha, p2, p4, sig_rr, rr, sg); return;
      case Q52: phase_b_pairs<q52_t, false>(S, R, alpha, p2, p4, sig_rr, rr, sg); return;
      default: phase_b_pairs<__nv_bfloat16, true>(S, R, alpha, p2, p4, sig_rr, rr, sg); return;
    }
  }
  switch (p1) {
    case F64: phase_b_rows<double, false>(S, R, alpha, p2, p4, sig_rr, rr, sg); break;
    case F32:
    case TF32: phase_b_rows<float, false>(S, R, alpha, p2, p4, sig_rr, rr, sg); break;
    case F16: phase_b_rows<__half, false>(S, R, alpha, p2, p4, sig_rr, rr, sg); break;
    case BF16: phase_b_rows<__nv_bfloat16, false>(S, R, alpha, p2, p4, sig_rr, rr, sg); break;
    case F16R: phase_b_rows<__half, true>(S, R, alpha, p2, p4, sig_rr, rr, sg); break;
    case Q52: phase_b_rows<q52_t, false>(S, R, alpha, p2, p4, sig_rr, rr, sg); break;
    default: phase_b_rows<__nv_bfloat16, true>(S, R, alpha, p2, p4, sig_rr, rr, sg); break;
  }
}

__device__ __noinline__ void phase_c(const DevSys& S, Rows R, double alpha, double beta, int p2, int p1n) {
  if (aligned16(S.p, S.x, S.r)) {
    switch (store_of(p1n)) {
      case ST_DOUBLE: phase_c_pairs<double>(S, R, alpha, beta, p2, p1n); return;
      case ST_FLOAT: phase_c_pairs<float>(S, R, alpha, beta, p2, p1n); return;
      case ST_HALF: phase_c_pairs<__half>(S, R, alpha, beta, p2, p1n); return;
      case ST_Q52: phase_c_pairs<q52_t>(S, R, alpha, beta, p2, p1n); return;
      default: phase_c_pairs<__nv_bfloat16>(S, R, alpha, beta, p2, p1n); return;
    }
  }
  switch (store_of(p1n)) {
    case ST_DOUBLE: phase_c_rows<double>(S, R, alpha, beta, p2, p1n); break;
    case ST_FLOAT: phase_c_rows<float>(S, R, alpha, beta, p2, p1n); break;
    case ST_HALF: phase_c_rows<__half>(S, R, alpha, beta, p2, p1n); break;
    case ST_Q52: phase_c_rows<q52_t>(S, R, alpha, beta, p2, p1n); break;
    default: phase_c_rows<__nv_bfloat16>(S, R, alpha, beta, p2, p1n); break;
  }
}

// fp64 restart after a breakdown: r = b - A x and p = r in fp64, then step_restart.
template <bool IC>
__device__ bool restart64(const Launch& L, const TeamCtx& T, const DevSys& S, SysState* st, Rows R, Smem& sm) {
  double rr = 0.0;
  DotAcc sg{0.0, 0.f, 0.f};
  true_res_rows<IC>(L, S, R, -1, -1, true, rr, sg, sm.bc.icep);
  rr = cta_sum(rr, sm.red);
  const double sp = cta_dot(sg, sm.red);
  write_partial(L, 0, rr);
  write_partial(L, 1, sp);
  return team_step(L, T, st, sm, [&] {
    const double trr = team_sum(L, T, 0, sm.red);
    const double tsg = team_sum(L, T, 1, sm.red);
    step_restart(L, S, st, trr, tsg, sm);
  });
}

template <bool IC>
__device__ __forceinline__ bool solve_system(const Launch& L, const TeamCtx& T, int sid, Smem& sm, const StreamCtx* sc) {
  const DevSys& S = L.sys[sid];
  SysState* st = L.st + sid;
  const OptView& o = L.opt;
  if (threadIdx.x == 0) {
    sm.r0 = part_row(S.A.rp, S.A.n, S.A.nnz, T.rank, T.size);
    sm.r1 = part_row(S.A.rp, S.A.n, S.A.nnz, T.rank + 1, T.size);
  }
  __syncthreads();
  const Rows R{sm.r0, sm.r1, T.rank, T.size};

  // ---- initialisation: x_0, r_0 = b - A x_0, p_0 = z_0 = M^-1 r_0, ||b||^2, ||r_0||^2,
  //      sigma_0 = r_0^T z_0 ----
  {
    double bb = 0.0, rr = 0.0;
    DotAcc sg{0.0, 0.f, 0.f};
    const bool ic = IC && S.icw != nullptr;
    for (int i = R.r0 + threadIdx.x; i < R.r1; i += kThreads) {
      const double bi = __ldg(S.b + i);
      bb = fma(bi, bi, bb);
      if (!o.warm_start) {
        S.x[i] = 0.0;
        S.r[i] = bi;
        rr = fma(bi, bi, rr);
        if (!ic) {
          const double wi = minv_r(S, i, bi);
          S.p[i] = wi;
          sg.d = fma(bi, wi, sg.d);
        }
      }
    }
    // IC(0): epoch 0 (the marks are zeroed for every launch; later phases count from 1)
    if (o.warm_start) true_res_rows<IC>(L, S, R, -1, -1, true, rr, sg, 0u);
    else if (ic)
      ic_phase(L, S, R, 0u, -1, -1, true, sg);
    bb = cta_sum(bb, sm.red);
    rr = cta_sum(rr, sm.red);
    const double sp = cta_dot(sg, sm.red);
    write_partial(L, 0, bb);
    write_partial(L, 1, rr);
    write_partial(L, 2, sp);
    if (!team_step(L, T, st, sm, [&] {
          const double tb = team_sum(L, T, 0, sm.red);
          const double tr = team_sum(L, T, 1, sm.red);
          const double ts = team_sum(L, T, 2, sm.red);
          step_init(L, S, st, tb, tr, ts, sm);
        }))
      return false;
  }

  if (sm.bc.mode == M_CONT) {
    // p in the format of the first product
    {
      const int p1 = sm.bc.fmt[0];
      if (p1 != F64)
        for (int i = R.r0 + threadIdx.x; i < R.r1; i += kThreads) store_low(S.plow, i, S.p[i], p1);
      if (!team_step(L, T, st, sm, [] {})) return false;
    }
    while (true) {
      // ---- phase A: q = fl_p1(A p), nu partials ----
      {
        DotAcc nu{0.0, 0.f, 0.f};
        const int p1 = sm.bc.fmt[0], p3 = sm.bc.fmt[2];
        spmv_rows(S, R, p1, p3, nu, sc);
        write_partial(L, 0, cta_dot(nu, sm.red));
        if (!team_step(L, T, st, sm, [&] { step_A(L, S, st, team_sum(L, T, 0, sm.red)); })) return false;
        if (sm.bc.mode == M_RESTART64) {
          if (!restart64<IC>(L, T, S, st, R, sm)) return false;
          if (sm.bc.mode != M_CONT) break;
          continue;
        }
        if (sm.bc.mode != M_CONT) break;
      }
      // ---- phase B: r -= alpha q (fp64), ||r||^2 (fp64), sigma partials ----
      {
        const double alpha = sm.bc.alpha;
        const int p1 = sm.bc.fmt[0], p2 = sm.bc.fmt[1], p4 = sm.bc.fmt[3];
        // with z = r (no preconditioner) and an fp64 dot, sigma is ||r||^2 itself: one DFMA
        // per row saved
        const bool ic = IC && S.icw != nullptr;
        const bool sig_rr = (p2 == F64 && p4 == F64 && !S.A.dinv && !ic);
        double rr = 0.0;
        DotAcc sg{0.0, 0.f, 0.f};
        // with IC(0) the sigma terms follow the substitutions
        phase_b(S, R, alpha, p1, p2, p4, sig_rr || ic, rr, sg);
        if (ic) ic_phase(L, S, R, sm.bc.icep, p2, p4, false, sg);
        rr = cta_sum(rr, sm.red);
        const double sp = sig_rr ? rr : cta_dot(sg, sm.red);
        write_partial(L, 0, rr);
        write_partial(L, 1, sp);
        if (!team_step(L, T, st, sm, [&] {
              const double trr = team_sum(L, T, 0, sm.red);
              const double tsg = team_sum(L, T, 1, sm.red);
              step_B(L, S, st, trr, tsg, sm);
            }))
          return false;
      }
      const int mode = sm.bc.mode;
      if (mode == M_CONT) {
        // ---- phase C: x += alpha p; p = z + beta p (fp64); p in the next product's format ----
        const double alpha = sm.bc.alpha, beta = sm.bc.beta;
        const int p1n = sm.bc.fmt[0];  // next action's product format
        const int p2 = sm.bc.zfmt;     // z = fl_p2(r) of the finished iteration
        phase_c(S, R, alpha, beta, p2, p1n);
        if (!team_step(L, T, st, sm, [&] { stamp_c(S, st); })) return false;
        if (sm.bc.k >= S.max_iter) break;
        continue;
      }
      if (mode == M_DONE) break;
      // ---- phase X: x += alpha p ----
      {
        const double alpha = sm.bc.alpha;
        for (int i = R.r0 + threadIdx.x; i < R.r1; i += kThreads) S.x[i] = fma(alpha, S.p[i], S.x[i]);
        if (!team_step(L, T, st, sm, [] {})) return false;
      }
      if (mode == M_X_THEN_DONE) break;
      if (mode == M_X_THEN_RESTART64) {
        if (!restart64<IC>(L, T, S, st, R, sm)) return false;
        if (sm.bc.mode != M_CONT) break;
        continue;
      }
      // ---- phase T: r = b - A x (fp64), ||r||^2, sigma partials ----
      {
        const int p2 = sm.bc.fmt[1], p4 = sm.bc.fmt[3];
        double rr = 0.0;
        DotAcc sg{0.0, 0.f, 0.f};
        true_res_rows<IC>(L, S, R, p2, p4, false, rr, sg, sm.bc.icep);
        rr = cta_sum(rr, sm.red);
        const double sp = cta_dot(sg, sm.red);
        write_partial(L, 0, rr);
        write_partial(L, 1, sp);
        if (!team_step(L, T, st, sm, [&] {
              const double trr = team_sum(L, T, 0, sm.red);
              const double tsg = team_sum(L, T, 1, sm.red);
              step_T(L, S, st, trr, tsg, sm);
            }))
          return false;
      }
      if (sm.bc.mode == M_RESTART64) {
        if (!restart64<IC>(L, T, S, st, R, sm)) return false;
        if (sm.bc.mode != M_CONT) break;
        continue;
      }
      if (sm.bc.mode == M_RESTART) {
        // p = z (beta = 0) after the replacement; x is already up to date.
        const int p1n = sm.bc.fmt[0];
        const int p2 = sm.bc.zfmt;
        for (int i = R.r0 + threadIdx.x; i < R.r1; i += kThreads) {
          const double pn = z_of(minv_r(S, i, S.r[i]), p2);
          S.p[i] = pn;
          if (p1n != F64) store_low(S.plow, i, pn, p1n);
        }
        if (!team_step(L, T, st, sm, [] {})) return false;
        if (sm.bc.k >= S.max_iter) break;
        continue;
      }
      break;
    }
  }

  // ---- final: ||b - A x|| in fp64 unless already known ----
  {
    double rr = 0.0;
    DotAcc unused{0.0, 0.f, 0.f};
    int known = 0;
    if (threadIdx.x == 0) known = *(volatile int*)&st->true_known;
    known = __syncthreads_or(known);
    if (!known) true_res_rows<IC>(L, S, R, -1, -1, false, rr, unused, 0u);
    rr = cta_sum(rr, sm.red);
    write_partial(L, 0, rr);
    if (!team_step(L, T, st, sm, [&] { step_final(L, S, st, sid, team_sum(L, T, 0, sm.red)); })) return false;
  }
  return true;
}

// ----------------------------------------------------------------------------------------
// Single-reduction iteration: row work of its phases
// ----------------------------------------------------------------------------------------

// u_i in the product format p1 (fp64 included) in plow, the product's input.
__device__ __forceinline__ void store_u(const DevSys& S, int i, double u, int p1) {
  if (p1 == F64) ((double*)S.plow)[i] = u;
  else store_low(S.plow, i, u, p1);
}

// Phase UL: u = fl_p2(M^-1 r) in the product format, from the current r (after the
// initialisation, a residual replacement or the fp64 restart).
__device__ __noinline__ void sr_ul_rows(const DevSys& S, Rows R, int p1, int p2) {
  for (int i = R.r0 + threadIdx.x; i < R.r1; i += kThreads) store_u(S, i, z_of(minv_r(S, i, S.r[i]), p2), p1);
}

// Partial sums of phase W over the CTA's rows, after the product w = fl_p1(A u) is stored:
// gamma = sum fl_p4(r_i) fl_p4(u_i) and delta = sum fl_p3(w_i) fl_p3(u_i) (compensated fp32, or
// fp64 for fp64), and the fp64 sums r.r, r.w, r.s, w.w, w.s, s.s of the norm recurrence.
struct SrSums {
  DotAcc g, d;
  double rr, rw, rs, ww, ws, ss;
};
__device__ __noinline__ void sr_w_tail(const DevSys& S, Rows R, int p1, int p2, int p3, int p4, SrSums& a) {
  for (int i = R.r0 + threadIdx.x; i < R.r1; i += kThreads) {
    const double ri = S.r[i];
    const double wi = load_q(S, i, p1);
    const double si = S.sv[i];
    const double mi = minv_r(S, i, ri);
    const double ui = z_of(mi, p2);
    sigma_term(ri, mi, p2, p4, a.g);
    if (p3 == F64) a.d.d = fma(wi, ui, a.d.d);
    else dot_low(a.d, round_d2f(wi, p3), round_d2f(ui, p3), p3);
    a.rr = fma(ri, ri, a.rr);
    a.rw = fma(ri, wi, a.rw);
    a.rs = fma(ri, si, a.rs);
    a.ww = fma(wi, wi, a.ww);
    a.ws = fma(wi, si, a.ws);
    a.ss = fma(si, si, a.ss);
  }
}

// Phase U: p = u + beta p, s = w + beta s, x += alpha p, r -= alpha s (fp64) with u = fl_p2(M^-1 r)
// and w (stored in format p1w) of the finished iteration; with `next`, the next iteration's u
// in its product format (p1n, p2n) from the new r.
__device__ __noinline__ void sr_u_rows(const DevSys& S, Rows R, double alpha, double beta, int p2, int p1w, bool next,
                                       int p1n, int p2n) {
  for (int i = R.r0 + threadIdx.x; i < R.r1; i += kThreads) {
    const double ri = S.r[i];
    const double ui = z_of(minv_r(S, i, ri), p2);
    const double wi = load_q(S, i, p1w);
    const double pn = fma(beta, S.p[i], ui);
    const double sn = fma(beta, S.sv[i], wi);
    S.p[i] = pn;
    S.sv[i] = sn;
    S.x[i] = fma(alpha, pn, S.x[i]);
    const double rn = fma(-alpha, sn, ri);
    S.r[i] = rn;
    if (next) store_u(S, i, z_of(minv_r(S, i, rn), p2n), p1n);
  }
}

// ----------------------------------------------------------------------------------------
// Lockstep batches: all CTAs work on all active systems at every super-step
// ----------------------------------------------------------------------------------------
// Each system runs the same sequence of phases as solve_system, as a state machine: at a
// super-step every CTA does the row work of the current phase of each system it holds a
// slice of (partials per slice), a grid barrier follows, then the CTA that owns a system
// (system index modulo the grid) reduces the slices' partials in slice order, runs the
// phase's scalar step and sets the next phase, and a second grid barrier closes the
// super-step. The slices are cut from the active systems' row work (nnz + 3 n per system,
// rows located by bisection on rp[r] + 3 r) and re-cut whenever a system finishes, so the
// whole GPU keeps working on whatever systems are left.

// PH_W, PH_U, PH_UL: the single-reduction iteration's product-and-reduction phase, its update
// phase, and the write of u's product-format copy after an initialisation or a restart.
enum LkPhase : int { PH_INIT = 0, PH_PLOW, PH_A, PH_B, PH_C, PH_X, PH_T, PH_RZ, PH_R64, PH_FINAL, PH_DONE,
                     PH_W, PH_U, PH_UL };
static_assert(PH_DONE == kPhaseDone, "the host reads the final phase's code");

__device__ __forceinline__ bool grid_sync(const Launch& L, const TeamCtx& G, Smem& sm) {
  if (team_arrive(G, sm)) {
    team_release(G);
    return true;
  }
  return team_wait(L, G, sm);
}

// Exclusive prefix over the CTA's threads (thread order) of v; *total receives the sum.
__device__ __forceinline__ long long cta_excl_scan(long long v, long long* tmp, long long* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  long long x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  __syncthreads();
  if (lane == 31) tmp[w] = x;
  __syncthreads();
  long long before = 0, all = 0;
  for (int i = 0; i < kThreads / 32; ++i) {
    if (i < w) before += tmp[i];
    all += tmp[i];
  }
  *total = all;
  return before + x - v;
}

// Re-cuts the slices (run by CTA 0 with all threads): prefix of the active systems' work,
// the CTA range of each active system and the partial slot of its first slice.
__device__ void lk_partition(const Launch& L, Smem& sm) {
  long long* tmp = reinterpret_cast<long long*>(sm.red);
  const int ns = L.nsys;
  const long long G = gridDim.x;
  long long carry = 0;
  for (int c0 = 0; c0 < ns; c0 += kThreads) {
    const int s = c0 + threadIdx.x;
    long long w = 0;
    if (s < ns && ((const volatile SysState*)(L.st + s))->phase != PH_DONE) w = L.lk_w[s];
    long long tot;
    const long long ex = cta_excl_scan(w, tmp, &tot);
    if (s < ns) L.lk_pref[s] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) L.lk_pref[ns] = carry;
  __syncthreads();
  const long long W = carry;
  long long slots = 0;
  for (int c0 = 0; c0 < ns; c0 += kThreads) {
    const int s = c0 + threadIdx.x;
    long long cnt = 0;
    int cf = -1, cl = -1;
    if (s < ns && W > 0) {
      const long long a = L.lk_pref[s], b = L.lk_pref[s + 1];
      if (b > a) {
        cf = (int)((a * G) / W);
        cl = (int)(((b - 1) * G) / W);
        cnt = cl - cf + 1;
      }
    }
    long long tot;
    const long long ex = cta_excl_scan(cnt, tmp, &tot);
    if (s < ns) {
      L.lk_cfirst[s] = cf;
      L.lk_clast[s] = cl;
      L.lk_base[s] = (int)(slots + ex);
    }
    slots += tot;
  }
}

// First row r of system S with rp[r] + 3 r >= t (0 <= t <= nnz + 3 n).
__device__ __forceinline__ int lk_row_at(const DevSys& S, long long t) {
  int lo = 0, hi = S.A.n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if ((long long)__ldg(S.A.rp + mid) + 3LL * mid < t) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// The slices of this CTA under the current cut (thread 0 writes them, the CTA reads them
// after the barrier at the end of the function).
__device__ void lk_slices(const Launch& L, Smem& sm) {
  if (threadIdx.x == 0) {
    const int c = blockIdx.x, ns = L.nsys;
    const long long G = gridDim.x, W = L.lk_pref[ns];
    int4* out = L.lk_seg + (long long)c * (ns + 1);
    int cnt = 0;
    if (W > 0) {
      // positions x in [0, W) belong to CTA floor(x G / W): this CTA holds [a, b)
      const long long a = (W * c + G - 1) / G, b = (W * (c + 1) + G - 1) / G;
      // first system whose work ends after a
      int lo = 0, hi = ns;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (L.lk_pref[mid + 1] <= a) lo = mid + 1;
        else hi = mid;
      }
      for (int s = lo; s < ns && cnt <= ns; ++s) {
        const long long ps = L.lk_pref[s], pe = L.lk_pref[s + 1];
        if (ps >= b) break;
        if (pe <= ps || pe <= a) continue;
        const DevSys& S = L.sys[s];
        const long long t0 = (a > ps ? a : ps) - ps, t1 = (b < pe ? b : pe) - ps;
        const int r0 = lk_row_at(S, t0), r1 = lk_row_at(S, t1);
        out[cnt++] = make_int4(s, r0, r1, L.lk_base[s] + (c - L.lk_cfirst[s]));
      }
    }
    L.lk_nseg[c] = cnt;
  }
  __syncthreads();
}

__device__ __forceinline__ void lk_partial(const Launch& L, int slot, int k, double v) {
  if (threadIdx.x == 0) L.partials[(long long)slot * kNSlot + k] = v;
}

// Phase W row work: the product of u (no nu partial) and the iteration's partial sums (slots
// 0..7: gamma, delta, r.r, r.w, r.s, w.w, w.s, s.s).
__device__ __forceinline__ void sr_w_rows(const Launch& L, const DevSys& S, Rows R, int slot, Smem& sm,
                                          const StreamCtx* sc) {
  DotAcc none{0.0, 0.f, 0.f};
  spmv_rows(S, R, sm.bc.fmt[0], -1, none, sc);
  SrSums a{{0.0, 0.f, 0.f}, {0.0, 0.f, 0.f}, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  sr_w_tail(S, R, sm.bc.fmt[0], sm.bc.fmt[1], sm.bc.fmt[2], sm.bc.fmt[3], a);
  lk_partial(L, slot, 0, cta_dot(a.g, sm.red));
  lk_partial(L, slot, 1, cta_dot(a.d, sm.red));
  lk_partial(L, slot, 2, cta_sum(a.rr, sm.red));
  lk_partial(L, slot, 3, cta_sum(a.rw, sm.red));
  lk_partial(L, slot, 4, cta_sum(a.rs, sm.red));
  lk_partial(L, slot, 5, cta_sum(a.ww, sm.red));
  lk_partial(L, slot, 6, cta_sum(a.ws, sm.red));
  lk_partial(L, slot, 7, cta_sum(a.ss, sm.red));
}

// Phase U row work (updates; the next u's copy when the iteration continues normally).
__device__ __forceinline__ void sr_u_phase(const DevSys& S, Rows R, Smem& sm) {
  sr_u_rows(S, R, sm.bc.alpha, sm.bc.beta, sm.bc.zfmt, sm.bc.wfmt, sm.bc.mode == M_CONT, sm.bc.fmt[0], sm.bc.fmt[1]);
}

// Row work of one slice in the current phase of its system. ONLY >= 0 compiles the code of
// that phase alone (the per-phase kernels of the stepped solve; the caller has checked the
// phase), ONLY < 0 every phase behind a run-time switch.
template <bool IC, int ONLY = -1>
__device__ void lk_slice_rows(const Launch& L, int s, Rows R, int slot, Smem& sm, const StreamCtx* sc) {
  static_assert(!(IC && ONLY >= 0), "the single-phase forms carry no IC(0) substitutions");
  const DevSys& S = L.sys[s];
  SysState* st = L.st + s;
  if (threadIdx.x == 0) {
    const volatile SysState* v = st;
    sm.lk_phase = v->phase;
    sm.lk_known = v->true_known;
  }
  load_bcast(st, sm);  // ends with __syncthreads
  if constexpr (ONLY == PH_A) {
    DotAcc nu{0.0, 0.f, 0.f};
    spmv_rows(S, R, sm.bc.fmt[0], sm.bc.fmt[2], nu, sc);
    lk_partial(L, slot, 0, cta_dot(nu, sm.red));
    return;
  } else if constexpr (ONLY == PH_B) {
    const int p1 = sm.bc.fmt[0], p2 = sm.bc.fmt[1], p4 = sm.bc.fmt[3];
    const bool sig_rr = (p2 == F64 && p4 == F64 && !S.A.dinv);
    double rr = 0.0;
    DotAcc sg{0.0, 0.f, 0.f};
    phase_b(S, R, sm.bc.alpha, p1, p2, p4, sig_rr, rr, sg);
    rr = cta_sum(rr, sm.red);
    const double sp = sig_rr ? rr : cta_dot(sg, sm.red);
    lk_partial(L, slot, 0, rr);
    lk_partial(L, slot, 1, sp);
    return;
  } else if constexpr (ONLY == PH_C) {
    phase_c(S, R, sm.bc.alpha, sm.bc.beta, sm.bc.zfmt, sm.bc.fmt[0]);
    return;
  } else if constexpr (ONLY == PH_W) {
    sr_w_rows(L, S, R, slot, sm, sc);
    return;
  } else if constexpr (ONLY == PH_U) {
    sr_u_phase(S, R, sm);
    return;
  }
  const int phase = sm.lk_phase;
  switch (phase) {
    case PH_INIT: {
      double bb = 0.0, rr = 0.0;
      DotAcc sg{0.0, 0.f, 0.f};
      const bool warm = L.opt.warm_start != 0;
      const bool ic = IC && S.icw != nullptr;
      const bool sr = S.sv != nullptr;  // single-reduction iteration: p = s = 0, no sigma_0
      for (int i = R.r0 + threadIdx.x; i < R.r1; i += kThreads) {
        const double bi = __ldg(S.b + i);
        bb = fma(bi, bi, bb);
        if (sr) S.p[i] = S.sv[i] = 0.0;
        if (!warm) {
          S.x[i] = 0.0;
          S.r[i] = bi;
          rr = fma(bi, bi, rr);
          if (!ic && !sr) {
            const double wi = minv_r(S, i, bi);
            S.p[i] = wi;
            sg.d = fma(bi, wi, sg.d);
          }
        }
      }
      if (warm) true_res_rows<IC>(L, S, R, -1, -1, !sr, rr, sg, sm.bc.icep);
      else if (ic)
        ic_phase(L, S, R, sm.bc.icep, -1, -1, true, sg);
      bb = cta_sum(bb, sm.red);
      rr = cta_sum(rr, sm.red);
      const double sp = cta_dot(sg, sm.red);
      lk_partial(L, slot, 0, bb);
      lk_partial(L, slot, 1, rr);
      lk_partial(L, slot, 2, sp);
      break;
    }
    case PH_PLOW: {
      const int p1 = sm.bc.fmt[0];
      if (p1 != F64)
        for (int i = R.r0 + threadIdx.x; i < R.r1; i += kThreads) store_low(S.plow, i, S.p[i], p1);
      break;
    }
    case PH_A: {
      DotAcc nu{0.0, 0.f, 0.f};
      spmv_rows(S, R, sm.bc.fmt[0], sm.bc.fmt[2], nu, sc);
      lk_partial(L, slot, 0, cta_dot(nu, sm.red));
      break;
    }
    case PH_B: {
      const int p1 = sm.bc.fmt[0], p2 = sm.bc.fmt[1], p4 = sm.bc.fmt[3];
      const bool ic = IC && S.icw != nullptr;
      const bool sig_rr = (p2 == F64 && p4 == F64 && !S.A.dinv && !ic);
      double rr = 0.0;
      DotAcc sg{0.0, 0.f, 0.f};
      phase_b(S, R, sm.bc.alpha, p1, p2, p4, sig_rr || ic, rr, sg);
      if (ic) ic_phase(L, S, R, sm.bc.icep, p2, p4, false, sg);
      rr = cta_sum(rr, sm.red);
      const double sp = sig_rr ? rr : cta_dot(sg, sm.red);
      lk_partial(L, slot, 0, rr);
      lk_partial(L, slot, 1, sp);
      break;
    }
    case PH_C:
      phase_c(S, R, sm.bc.alpha, sm.bc.beta, sm.bc.zfmt, sm.bc.fmt[0]);
      break;
    case PH_X: {
      const double alpha = sm.bc.alpha;
      for (int i = R.r0 + threadIdx.x; i < R.r1; i += kThreads) S.x[i] = fma(alpha, S.p[i], S.x[i]);
      break;
    }
    case PH_T: {
      double rr = 0.0;
      DotAcc sg{0.0, 0.f, 0.f};
      true_res_rows<IC>(L, S, R, sm.bc.fmt[1], sm.bc.fmt[3], false, rr, sg, sm.bc.icep);
      rr = cta_sum(rr, sm.red);
      const double sp = cta_dot(sg, sm.red);
      lk_partial(L, slot, 0, rr);
      lk_partial(L, slot, 1, sp);
      break;
    }
    case PH_RZ: {
      const int p1n = sm.bc.fmt[0], p2 = sm.bc.zfmt;
      for (int i = R.r0 + threadIdx.x; i < R.r1; i += kThreads) {
        const double pn = z_of(minv_r(S, i, S.r[i]), p2);
        S.p[i] = pn;
        if (p1n != F64) store_low(S.plow, i, pn, p1n);
      }
      break;
    }
    case PH_R64: {
      double rr = 0.0;
      DotAcc sg{0.0, 0.f, 0.f};
      const bool sr = S.sv != nullptr;  // single-reduction iteration: the recurrence restarts from 0
      true_res_rows<IC>(L, S, R, -1, -1, !sr, rr, sg, sm.bc.icep);
      if (sr)
        for (int i = R.r0 + threadIdx.x; i < R.r1; i += kThreads) S.p[i] = S.sv[i] = 0.0;
      rr = cta_sum(rr, sm.red);
      const double sp = cta_dot(sg, sm.red);
      lk_partial(L, slot, 0, rr);
      lk_partial(L, slot, 1, sp);
      break;
    }
    case PH_FINAL: {
      double rr = 0.0;
      DotAcc unused{0.0, 0.f, 0.f};
      if (!sm.lk_known) true_res_rows<IC>(L, S, R, -1, -1, false, rr, unused, 0u);
      lk_partial(L, slot, 0, cta_sum(rr, sm.red));
      break;
    }
    case PH_UL:
      sr_ul_rows(S, R, sm.bc.fmt[0], sm.bc.fmt[1]);
      break;
    case PH_W:
      sr_w_rows(L, S, R, slot, sm, sc);
      break;
    case PH_U:
      sr_u_phase(S, R, sm);
      break;
    default:
      break;
  }
}

// Sum of partial k over the slices of a system (slice order per thread, fixed tree across
// threads: deterministic for a given cut).
__device__ __forceinline__ double lk_sum(const Launch& L, int base, int np, int k, Smem& sm) {
  double v = 0.0;
  for (int i = threadIdx.x; i < np; i += kThreads) v += __ldcg(&L.partials[(long long)(base + i) * kNSlot + k]);
  return cta_sum(v, sm.red);
}

// Scalar step of the phase system s has just run, by the CTA that owns s; sets the next
// phase (the transitions of solve_system). The phase's partials are the np slots from base.
// ONLY >= 0: the caller knows the phase and only that phase's step is compiled.
template <int ONLY = -1>
__device__ void lk_step_slots(const Launch& L, int s, int base, int np, Smem& sm) {
  const DevSys& S = L.sys[s];
  SysState* st = L.st + s;
  if (threadIdx.x == 0) sm.lk_phase = ((const volatile SysState*)st)->phase;
  __syncthreads();
  const int phase = ONLY >= 0 ? ONLY : sm.lk_phase;
  if (phase == PH_DONE) return;
  if constexpr (ONLY == PH_A) {
    step_A(L, S, st, lk_sum(L, base, np, 0, sm));
  } else if constexpr (ONLY == PH_B) {
    const double trr = lk_sum(L, base, np, 0, sm), tsg = lk_sum(L, base, np, 1, sm);
    step_B(L, S, st, trr, tsg, sm);
  } else if constexpr (ONLY == PH_C || ONLY == PH_U) {
    stamp_c(S, st);
  } else if constexpr (ONLY == PH_W) {
    double d[6];
    const double g = lk_sum(L, base, np, 0, sm), dl = lk_sum(L, base, np, 1, sm);
    for (int q = 0; q < 6; ++q) d[q] = lk_sum(L, base, np, 2 + q, sm);
    step_W(L, S, st, g, dl, d, sm);
  } else {
  switch (phase) {
    case PH_INIT: {
      const double tb = lk_sum(L, base, np, 0, sm), tr = lk_sum(L, base, np, 1, sm);
      const double ts = lk_sum(L, base, np, 2, sm);
      step_init(L, S, st, tb, tr, ts, sm);
      break;
    }
    case PH_A: step_A(L, S, st, lk_sum(L, base, np, 0, sm)); break;
    case PH_B: {
      const double trr = lk_sum(L, base, np, 0, sm), tsg = lk_sum(L, base, np, 1, sm);
      step_B(L, S, st, trr, tsg, sm);
      break;
    }
    case PH_C: stamp_c(S, st); break;
    case PH_T: {
      const double trr = lk_sum(L, base, np, 0, sm), tsg = lk_sum(L, base, np, 1, sm);
      step_T(L, S, st, trr, tsg, sm);
      break;
    }
    case PH_R64: {
      const double trr = lk_sum(L, base, np, 0, sm), tsg = lk_sum(L, base, np, 1, sm);
      step_restart(L, S, st, trr, tsg, sm);
      break;
    }
    case PH_FINAL: step_final(L, S, st, s, lk_sum(L, base, np, 0, sm)); break;
    case PH_W: {
      double d[6];
      const double g = lk_sum(L, base, np, 0, sm), dl = lk_sum(L, base, np, 1, sm);
      for (int q = 0; q < 6; ++q) d[q] = lk_sum(L, base, np, 2 + q, sm);
      step_W(L, S, st, g, dl, d, sm);
      break;
    }
    case PH_U: stamp_c(S, st); break;
    default: break;  // PH_PLOW, PH_X, PH_RZ, PH_UL: no scalar work
  }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const volatile SysState* v = st;
    const int mode = v->mode;
    int next = PH_FINAL;
    const bool sr = S.sv != nullptr;
    switch (phase) {
      case PH_INIT: next = mode == M_CONT ? (sr ? PH_UL : v->fmt[0] != F64 ? PH_PLOW : PH_A) : PH_FINAL; break;
      case PH_UL: next = PH_W; break;
      case PH_W: next = mode == M_RESTART64 ? PH_R64 : mode == M_DONE ? PH_FINAL : PH_U; break;
      case PH_U:
        next = mode == M_CONT ? (v->k >= S.max_iter ? PH_FINAL : PH_W)
               : mode == M_TCHK ? PH_T
               : mode == M_X_THEN_RESTART64 ? PH_R64
                                            : PH_FINAL;
        break;
      case PH_PLOW: next = PH_A; break;
      case PH_A: next = mode == M_RESTART64 ? PH_R64 : mode == M_CONT ? PH_B : PH_FINAL; break;
      case PH_B: next = mode == M_CONT ? PH_C : mode == M_DONE ? PH_FINAL : PH_X; break;
      case PH_C: next = v->k >= S.max_iter ? PH_FINAL : PH_A; break;
      case PH_X: next = mode == M_X_THEN_DONE ? PH_FINAL : mode == M_X_THEN_RESTART64 ? PH_R64 : PH_T; break;
      case PH_T:
        next = mode == M_RESTART64 ? PH_R64
               : mode == M_RESTART ? (sr ? (v->k >= S.max_iter ? PH_FINAL : PH_UL) : PH_RZ)
                                   : PH_FINAL;
        break;
      case PH_RZ: next = v->k >= S.max_iter ? PH_FINAL : PH_A; break;
      case PH_R64: next = mode == M_CONT ? (sr ? PH_UL : PH_A) : PH_FINAL; break;
      default: next = PH_DONE; break;  // PH_FINAL
    }
    st->phase = next;
    st->icep += 1u;  // a new epoch for the IC(0) marks of the next phase
    if (next == PH_DONE) atomicAdd(L.lk_done, 1);
  }
  __syncthreads();
}

__device__ __forceinline__ void lk_step(const Launch& L, int s, Smem& sm) {
  const int cf = L.lk_cfirst[s];
  const int np = cf < 0 ? 0 : L.lk_clast[s] - cf + 1;
  lk_step_slots<-1>(L, s, L.lk_base[s], np, sm);
}

template <bool IC>
__global__ void __launch_bounds__(kThreads, 4) cg_lockstep(const Launch L) {
  __shared__ Smem sm;
  extern __shared__ __align__(128) unsigned char dyn[];
  StreamCtx scx{dyn, sm.mbar, &sm.mbar_phase, L.err, L.stream_stage};
  if (L.stream_stage > 0) {
    if (threadIdx.x == 0) {
      mbar_init(sm.mbar + 0, 1);
      mbar_init(sm.mbar + 1, 1);
      mbar_fence_init();
      sm.mbar_phase = 0;
    }
    __syncthreads();
  }
  const StreamCtx* sc = L.stream_stage > 0 ? &scx : nullptr;
  TeamCtx G;
  G.team = 0;
  G.rank = blockIdx.x;
  G.size = gridDim.x;
  G.first = 0;
  G.bar = L.bars;
  int seen = -1;
  while (true) {
    if (threadIdx.x == 0) sm.lk_done = *(volatile int*)L.lk_done;
    __syncthreads();
    const int done = sm.lk_done;
    __syncthreads();
    if (done >= L.nsys) break;
    if (done != seen) {
      if (blockIdx.x == 0) lk_partition(L, sm);
      if (!grid_sync(L, G, sm)) return;
      lk_slices(L, sm);
      seen = done;
    }
    const int nseg = L.lk_nseg[blockIdx.x];
    for (int i = 0; i < nseg; ++i) {
      const int4 sg = L.lk_seg[(long long)blockIdx.x * (L.nsys + 1) + i];
      // the system's slices sit on its CTA range, one per CTA: this slice's index and count
      const int sg_g = sg.w - L.lk_base[sg.x];
      const int sg_n = L.lk_clast[sg.x] - L.lk_cfirst[sg.x] + 1;
      lk_slice_rows<IC>(L, sg.x, Rows{sg.y, sg.z, sg_g, sg_n}, sg.w, sm, sc);
    }
    if (!grid_sync(L, G, sm)) return;
    for (int s = blockIdx.x; s < L.nsys; s += gridDim.x) lk_step(L, s, sm);
    if (!grid_sync(L, G, sm)) return;
  }
}

// IC = true: the instantiation for launches that precondition with IC(0); the other one
// carries none of its code.
template <bool IC>
__global__ void __launch_bounds__(kThreads, 4) cg_persistent(const Launch L) {
  __shared__ Smem sm;
  extern __shared__ __align__(128) unsigned char dyn[];
  StreamCtx scx{dyn, sm.mbar, &sm.mbar_phase, L.err, L.stream_stage};
  if (L.stream_stage > 0) {
    if (threadIdx.x == 0) {
      mbar_init(sm.mbar + 0, 1);
      mbar_init(sm.mbar + 1, 1);
      mbar_fence_init();
      sm.mbar_phase = 0;
    }
    __syncthreads();
  }
  const StreamCtx* sc = L.stream_stage > 0 ? &scx : nullptr;
  TeamCtx T;
  T.team = L.cta_team[blockIdx.x];
  T.rank = L.cta_rank[blockIdx.x];
  T.size = L.team_size[T.team];
  T.first = L.team_first[T.team];
  T.bar = L.bars + (long long)T.team * kBarStride;
  for (int i = L.team_sys_off[T.team]; i < L.team_sys_off[T.team + 1]; ++i) {
    if (!solve_system<IC>(L, T, L.team_sys[i], sm, sc)) return;
  }
}

}  // namespace

}  // namespace mpcg
