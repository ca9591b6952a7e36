/*
 * mpcg CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline / reference
 * arm may load this file. The CUDA library never links, calls or includes it, and it
 * shares no code with that library.
 *
 * What it is: a plain, slow, single-threaded fp64 restatement of the method of
 * "Mixed-Precision Conjugate Gradient Solvers with RL-Driven Precision Tuning"
 * (arXiv 2504.14268):
 *   - the rounding model fl_p(x) = x(1+delta), |delta| <= u_p of Section 4, with
 *     the format parameters of Table 1 (t, e_min, e_max);
 *   - the CG recurrences Eq. (1)-(4) of Section 3 with the mixed-precision operation
 *     assignment of Section 4.2 (q = fl_p1(A p), z = fl_p2(M^-1 r), nu = fl_p3(p^T q),
 *     sigma = fl_p4(r^T z); residual update, alpha and beta in fp64);
 *   - the MDP of Section 4.1 (state discretisation, reward, Q-learning update,
 *     epsilon-greedy exploration) and Algorithms 1 (training) and 2 (inference), with
 *     per-operation tables or one table over the joint actions;
 *   - a small MLP Q-function (forward, backward, Adam) used by the learned policy;
 *   - the preconditioners of op 2: Jacobi and the fp32 incomplete Cholesky IC(0);
 *   - a single-reduction form of the iteration (Chronopoulos and Gear), beside the CG of
 *     Section 3.
 *
 * Every sum runs in fp64 in index order and the result is then rounded ("compute
 * high, round the output"), which is the emulation model the paper used (Section 5).
 *
 * Readings of passages that are silent or ambiguous are marked READING below.
 * Functions with no independent pin in the test suite say "parity unpinned".
 *
 * Build: gcc -O2 -std=c11 -fPIC -shared -ffp-contract=off (no FMA contraction, so
 * results are identical on x86-64 and aarch64 hosts).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Number formats (Table 1; tf32 and the row-scaled formats are READINGS).    */
/* ------------------------------------------------------------------------- */

enum {
  ORC_FP16 = 0, ORC_BF16 = 1, ORC_TF32 = 2, ORC_FP32 = 3, ORC_FP64 = 4,
  ORC_BF16R = 5, ORC_FP16R = 6, ORC_Q52 = 7, ORC_NFMT = 8
};

/* t = significand digits including the implicit bit, e_min, e_max (Table 1).
 * tf32 is not in Table 1: READING t = 11 with the fp32 exponent range.
 * q52 (Table 1's "quarter precision"): the t column is garbled; u = 1.25e-1 = 2^-3
 * gives t = 3. The row-scaled formats use their base format's parameters. */
static const int FMT_T[ORC_NFMT] = {11, 8, 11, 24, 53, 8, 11, 3};
static const int FMT_EMIN[ORC_NFMT] = {-14, -126, -126, -126, -1022, -126, -14, -14};
static const int FMT_EMAX[ORC_NFMT] = {15, 127, 127, 127, 1023, 127, 15, 15};

/* Round x to nearest (ties to even) in a binary format with t significand digits,
 * minimum normal exponent e_min (gradual underflow below it) and maximum exponent
 * e_max (Section 4: fl_p(x) = x(1+delta), |delta| <= u = 2^-t for normal results).
 * Step by step:
 *   e  = floor(log2 |x|), clamped below at e_min (subnormal range keeps the quantum of 2^e_min)
 *   q  = 2^(e - t + 1), the spacing of the format at that exponent
 *   y  = round_to_nearest_even(x / q) * q        (exact power-of-two scalings)
 *   |y| > x_max = 2^e_max (2 - 2^(1-t))  ->  +-inf (IEEE overflow under round to nearest). */
double orc_chop_tee(double x, int t, int emin, int emax) {
  if (x == 0.0 || !isfinite(x)) return x;
  int e2;
  frexp(x, &e2); /* x = f 2^e2 with 0.5 <= |f| < 1, so floor(log2|x|) = e2 - 1 */
  int e = e2 - 1;
  if (e < emin) e = emin;
  double scaled = ldexp(x, t - 1 - e);     /* exact */
  double y = ldexp(nearbyint(scaled), e - t + 1); /* nearbyint: round half to even */
  double xmax = ldexp(2.0 - ldexp(1.0, 1 - t), emax);
  if (fabs(y) > xmax) return copysign(INFINITY, x);
  return y;
}

/* fl_p(x): the rounding of a single value to format p; fp64 is the identity. The
 * row-scaled formats round like their base format (the scale enters only in A). */
double orc_chop(double x, int fmt) {
  if (fmt == ORC_FP64) return x;
  return orc_chop_tee(x, FMT_T[fmt], FMT_EMIN[fmt], FMT_EMAX[fmt]);
}

void orc_chop_vec(const double* x, double* y, int64_t n, int fmt) {
  for (int64_t i = 0; i < n; ++i) y[i] = orc_chop(x[i], fmt);
}

static int is_row_scaled(int fmt) { return fmt == ORC_BF16R || fmt == ORC_FP16R; }

/* READING (row-scaled value streams, an extension beside the paper's formats):
 * s_i = 2^floor(log2 max_j |a_ij|); the stored value is fl_f(a_ij / s_i); the
 * effective entry is s_i * stored. Division by a power of two is exact. */
double orc_row_scale(const int32_t* rp, const double* val, int i) {
  double m = 0.0;
  for (int32_t e = rp[i]; e < rp[i + 1]; ++e)
    if (fabs(val[e]) > m) m = fabs(val[e]);
  if (m == 0.0 || !isfinite(m)) return 1.0;
  int e2;
  frexp(m, &e2);
  return ldexp(1.0, e2 - 1);
}

/* ------------------------------------------------------------------------- */
/* Philox4x64-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11). */
/* Used for the epsilon-greedy draws of Algorithm 1.                          */
/* ------------------------------------------------------------------------- */

static void mulhilo64(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
  unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
  *hi = (uint64_t)(p >> 64);
  *lo = (uint64_t)p;
}

void orc_philox4x64(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4]) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
  uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint64_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t hi0, lo0, hi1, lo1;
    mulhilo64(M0, c0, &hi0, &lo0);
    mulhilo64(M1, c2, &hi1, &lo1);
    uint64_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += W0; k1 += W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------------- */
/* Options, policies and per-iteration records.                                */
/* ------------------------------------------------------------------------- */

typedef struct {
  int b_bins;        /* b: iteration bins (Section 4.1; 10 in Section 5)             */
  int r_bins;        /* r: residual bins (10 in Section 5)                            */
  int t_bin;         /* T_max used by the iteration bins (1000 in Section 5)          */
  int min_k;         /* stop only when k >= min_k (Section 5: "k >= 10")              */
  double eps_min;    /* residual floor (1e-16 in Section 5)                           */
  int nprec;         /* |P|                                                           */
  int precs[8];      /* P as format codes, in argmax tie order                        */
  double cost[8];    /* c(p) per entry of precs (Section 5, C1/C2)                    */
  double w1, w2, w3; /* reward weights (Section 4.1: 1.0, 0.1, 10.0)                  */
  double lr, gamma;  /* Q-learning alpha, gamma (0.1, 0.9)                            */
  double eps0, eps_floor; /* epsilon schedule: 1.0 decaying to 0.1                    */
  uint64_t seed;     /* Philox key                                                    */
  int unvisited_fallback; /* READING: action for never-updated (s, op) rows at inference;
                             -1 keeps the plain first-index argmax                    */
  int true_res_every;     /* >0: replace r by b - A x every this many iterations      */
  int true_res_at_conv;   /* 1: confirm a claimed convergence with b - A x            */
  int op_mask[4];         /* per operation, bitmask of allowed entries of precs (0 = all);
                             READING (extension): Section 5 allows customising P         */
  int on_breakdown;       /* 1: an inference solve that breaks down restarts once from
                             r = b - A x, p = r (fp64) and finishes in fp64            */
  int mlp_hidden;         /* MLP hidden width (64)                                     */
  int precond;            /* 0: M = I (the hot path); 1: Jacobi, M = diag(A): op 2 becomes
                             z = fl_p2(r_i d_i) with d_i = 1 / a_ii in fp64, and the
                             initial and restart directions and sigmas use z = d r;
                             2: IC(0) in fp32 (orc_ic0): z = fl_p2(L^-T L^-1 r) with
                             the solves in fp32, the initial and restart directions
                             z = L^-T L^-1 r unrounded beyond fp32                      */
  int variant;            /* 0: the CG of Section 3 (orc_run); 1: the single-reduction
                             iteration of orc_run_sr (M = I or Jacobi)                  */
  int joint;              /* 0: one Q-table per operation (Section 4.1); 1: one table over
                             the joint actions (orc_q_update_joint)                     */
} orc_opts;

enum { ORC_POL_FIXED = 0, ORC_POL_SCHEDULE = 1, ORC_POL_QTABLE = 2, ORC_POL_MLP = 3 };

typedef struct {
  int kind;
  int fixed[4];          /* FIXED: format codes of (p1, p2, p3, p4)                   */
  const int32_t* sched;  /* SCHEDULE: [len][4] format codes; rows past len repeat the last */
  int sched_len;
  double* Q;             /* QTABLE: [4][S][nprec]                                     */
  int32_t* visits;       /* QTABLE: [4][S] update counts                              */
  const double* mlp;     /* MLP: flat parameters (see mlp layout below)               */
  const double* feat_static; /* MLP: 5 static matrix features                        */
} orc_policy;

/* One record per iteration k (Algorithm 2 logs (k+1, p1..p4) at the stop; the oracle
 * logs every iteration so that trajectories can be compared). */
typedef struct {
  int32_t k, state, fmt[4], act[4]; /* act: index into precs, -1 if not in P        */
  double rho;      /* rho_{k+1} after the iteration (true residual if it was replaced) */
  double nu, alpha, sigma, beta, reward;
  int32_t flags;   /* bit0 converged, bit1 breakdown, bit2 r replaced, bit3 explored  */
  int32_t pad;
} orc_rec;

enum { ORC_CONVERGED = 0, ORC_MAX_ITER = 1, ORC_BREAKDOWN = 2 };

typedef struct {
  int32_t outcome, iters;
  int32_t nrec;     /* number of per-iteration records written                      */
  int32_t pad;
  double rho_rec;   /* last recursive relative residual                           */
  double rho_true;  /* ||b - A x|| / ||b|| at the end (always computed, fp64)      */
} orc_result;

/* ------------------------------------------------------------------------- */
/* Section 4.1: state discretisation.                                          */
/* ------------------------------------------------------------------------- */

/* i_k = min(floor(k / ceil(T_max / b)), b - 1)
 * j_k = min(floor(-log10 max(rho_k, eps_min) / delta), r - 1), delta = -log10(eps_min) / r
 * READING: rho_k > 1 makes j_k negative; it is clamped to 0.  s = i_k * r + j_k. */
int orc_state(const orc_opts* o, int k, double rho) {
  int width = (o->t_bin + o->b_bins - 1) / o->b_bins;
  int i = k / width;
  if (i > o->b_bins - 1) i = o->b_bins - 1;
  double delta = -log10(o->eps_min) / o->r_bins;
  double rr = rho > o->eps_min ? rho : o->eps_min;
  double jf = floor(-log10(rr) / delta);
  int j = (int)fmin(jf, (double)(o->r_bins - 1));
  if (j < 0) j = 0;
  return i * o->r_bins + j;
}

/* Section 4.1 reward: w1 min(-log10 rho', -log10 eps_min) - w2 sum_j c(p_j) + w3 1(rho' < tau).
 * READING: the sum runs over the four RL-controlled operations of Section 4.2.
 * READING: rho' = 0 takes the clamp value -log10(eps_min). */
double orc_reward(const orc_opts* o, double rho, const int act[4], double tau) {
  double acc = rho > 0 ? -log10(rho) : INFINITY;
  double cap = -log10(o->eps_min);
  double r = o->w1 * (acc < cap ? acc : cap);
  for (int j = 0; j < 4; ++j) r -= o->w2 * o->cost[act[j]];
  if (rho < tau) r += o->w3;
  return r;
}

/* READING: a breakdown ends the episode with the worst accuracy term. */
double orc_reward_breakdown(const orc_opts* o, const int act[4]) {
  double r = -o->w1 * (-log10(o->eps_min));
  for (int j = 0; j < 4; ++j) r -= o->w2 * o->cost[act[j]];
  return r;
}

/* Allowed actions of operation j: bit a of op_mask[j], all when the mask is 0. */
static int allowed(const orc_opts* o, int j, int a) {
  return o->op_mask[j] == 0 || ((o->op_mask[j] >> a) & 1);
}

/* First-index argmax over the allowed entries of a Q row. */
static int argmax_allowed(const orc_opts* o, int j, const double* row) {
  int best = -1;
  for (int a = 0; a < o->nprec; ++a)
    if (allowed(o, j, a) && (best < 0 || row[a] > row[best])) best = a;
  return best;
}

/* The random action of an exploring operation: the (pick mod #allowed)-th allowed entry. */
static int random_allowed(const orc_opts* o, int j, uint32_t pick) {
  int cnt = 0;
  for (int a = 0; a < o->nprec; ++a) cnt += allowed(o, j, a);
  int k = (int)(pick % (uint32_t)cnt);
  for (int a = 0; a < o->nprec; ++a)
    if (allowed(o, j, a) && k-- == 0) return a;
  return 0;
}

/* max_{p in P_j} Q_j(s', p): the bootstrap term of the Section 4.1 update, taken over the
 * entries operation j may choose. READING: Section 5 lets the precision set be customised;
 * with a per-operation set P_j (op_mask) the update's max runs over P_j, the same set the
 * greedy and exploring choices use (entries outside P_j are never updated and must not
 * enter the target). */
static double max_allowed(const orc_opts* o, int j, const double* row) {
  double m = -INFINITY;
  for (int a = 0; a < o->nprec; ++a)
    if (allowed(o, j, a) && row[a] > m) m = row[a];
  return m;
}

static int index_of(const orc_opts* o, int fmt) {
  for (int a = 0; a < o->nprec; ++a)
    if (o->precs[a] == fmt) return a;
  return -1;
}

/* Exploration schedule of Section 4.1 / Algorithm 1 with the floor of Section 5:
 * epsilon_e = max(eps_floor, eps0 (1 - e / E)), e = 1..E. */
double orc_epsilon(const orc_opts* o, int e, int E) {
  double v = o->eps0 * (1.0 - (double)e / (double)E);
  return v > o->eps_floor ? v : o->eps_floor;
}

/* Exploration draw for (episode e, lane, iteration k, operation j): Philox4x64-10 with
 * key (seed, 0x6d706367) and counter (e, lane, k, j). Word 0 gives u = (w0 >> 11) 2^-53,
 * the operation explores iff u < epsilon; word 1 mod |P| gives the random action. */
void orc_draw(uint64_t seed, uint64_t e, uint64_t lane, uint64_t k, uint64_t j,
              double* u, uint32_t* pick) {
  uint64_t ctr[4] = {e, lane, k, j}, key[2] = {seed, 0x6d706367ULL}, out[4];
  orc_philox4x64(ctr, key, out);
  *u = (double)(out[0] >> 11) * 0x1.0p-53;
  *pick = (uint32_t)(out[1] & 0xffffffffu);
}

/* ------------------------------------------------------------------------- */
/* MLP Q-function (an extension; the paper uses tables and names deep RL as    */
/* future work, Section 7). 16 -> H -> H -> 4*nprec, ReLU, fp64 here.          */
/* Layout of the flat parameter vector: W1[H][16], b1[H], W2[H][H], b2[H],     */
/* W3[4*nprec][H], b3[4*nprec] (row-major, out x in).                          */
/* ------------------------------------------------------------------------- */

#define ORC_NFEAT 16

int64_t orc_mlp_nparams(int H, int nout) {
  return (int64_t)H * ORC_NFEAT + H + (int64_t)H * H + H + (int64_t)nout * H + nout;
}

/* Forward pass for one feature vector. h1, h2 receive the post-ReLU activations. */
void orc_mlp_forward(const double* w, int H, int nout, const double* f, double* h1, double* h2,
                     double* out) {
  const double* W1 = w;
  const double* b1 = W1 + (int64_t)H * ORC_NFEAT;
  const double* W2 = b1 + H;
  const double* b2 = W2 + (int64_t)H * H;
  const double* W3 = b2 + H;
  const double* b3 = W3 + (int64_t)nout * H;
  for (int i = 0; i < H; ++i) {
    double s = b1[i];
    for (int j = 0; j < ORC_NFEAT; ++j) s += W1[(int64_t)i * ORC_NFEAT + j] * f[j];
    h1[i] = s > 0 ? s : 0;
  }
  for (int i = 0; i < H; ++i) {
    double s = b2[i];
    for (int j = 0; j < H; ++j) s += W2[(int64_t)i * H + j] * h1[j];
    h2[i] = s > 0 ? s : 0;
  }
  for (int i = 0; i < nout; ++i) {
    double s = b3[i];
    for (int j = 0; j < H; ++j) s += W3[(int64_t)i * H + j] * h2[j];
    out[i] = s;
  }
}

/* Fitted-Q regression loss over a batch and its gradient (READING, an extension):
 *   L = (1 / (B * 4)) sum_b sum_j 1/2 (Q(f_b)[j * nprec + a_bj] - y_bj)^2
 * Only the output of the taken action carries gradient. grad has the parameter layout.
 * Returns L. */
double orc_mlp_loss_grad(const double* w, int H, int nprec, int B, const double* feats,
                         const int32_t* acts, const double* y, double* grad) {
  int nout = 4 * nprec;
  int64_t np = orc_mlp_nparams(H, nout);
  memset(grad, 0, sizeof(double) * np);
  double* gW1 = grad;
  double* gb1 = gW1 + (int64_t)H * ORC_NFEAT;
  double* gW2 = gb1 + H;
  double* gb2 = gW2 + (int64_t)H * H;
  double* gW3 = gb2 + H;
  double* gb3 = gW3 + (int64_t)nout * H;
  const double* W2 = w + (int64_t)H * ORC_NFEAT + H;
  const double* W3 = W2 + (int64_t)H * H + H;
  double* h1 = malloc(sizeof(double) * H);
  double* h2 = malloc(sizeof(double) * H);
  double* out = malloc(sizeof(double) * nout);
  double* dout = malloc(sizeof(double) * nout);
  double* dh2 = malloc(sizeof(double) * H);
  double* dh1 = malloc(sizeof(double) * H);
  double loss = 0.0;
  double scale = 1.0 / ((double)B * 4.0);
  for (int b = 0; b < B; ++b) {
    const double* f = feats + (int64_t)b * ORC_NFEAT;
    orc_mlp_forward(w, H, nout, f, h1, h2, out);
    for (int i = 0; i < nout; ++i) dout[i] = 0.0;
    for (int j = 0; j < 4; ++j) {
      int o = j * nprec + acts[(int64_t)b * 4 + j];
      double d = out[o] - y[(int64_t)b * 4 + j];
      loss += 0.5 * d * d * scale;
      dout[o] += d * scale;
    }
    for (int i = 0; i < nout; ++i) {
      gb3[i] += dout[i];
      for (int j = 0; j < H; ++j) gW3[(int64_t)i * H + j] += dout[i] * h2[j];
    }
    for (int j = 0; j < H; ++j) {
      double s = 0.0;
      for (int i = 0; i < nout; ++i) s += W3[(int64_t)i * H + j] * dout[i];
      dh2[j] = h2[j] > 0 ? s : 0.0;
    }
    for (int i = 0; i < H; ++i) {
      gb2[i] += dh2[i];
      for (int j = 0; j < H; ++j) gW2[(int64_t)i * H + j] += dh2[i] * h1[j];
    }
    for (int j = 0; j < H; ++j) {
      double s = 0.0;
      for (int i = 0; i < H; ++i) s += W2[(int64_t)i * H + j] * dh2[i];
      dh1[j] = h1[j] > 0 ? s : 0.0;
    }
    for (int i = 0; i < H; ++i) {
      gb1[i] += dh1[i];
      for (int j = 0; j < ORC_NFEAT; ++j) gW1[(int64_t)i * ORC_NFEAT + j] += dh1[i] * f[j];
    }
  }
  free(h1); free(h2); free(out); free(dout); free(dh2); free(dh1);
  return loss;
}

/* Fitted-Q targets (the regression targets of the MLP Q-function): for each sample b and
 * operation j, y_bj = r_b + gamma (1 - done_b) max over the entries p allowed by op_mask[j]
 * (bit p; 0 = all) of Q_target(f_next_b)[j, p], with Q_target the network wt. This is the
 * one-step Bellman backup of the Q-learning update of Section 4.1 with the table replaced
 * by a function of the features. */
void orc_mlp_targets(const double* wt, int H, int nprec, int B, const double* feats_next, const double* rew,
                     const int32_t* done, double gamma, const int32_t* op_mask, double* y) {
  int nout = 4 * nprec;
  double* h1 = malloc(sizeof(double) * H);
  double* h2 = malloc(sizeof(double) * H);
  double* out = malloc(sizeof(double) * nout);
  for (int b = 0; b < B; ++b) {
    orc_mlp_forward(wt, H, nout, feats_next + (int64_t)b * ORC_NFEAT, h1, h2, out);
    for (int j = 0; j < 4; ++j) {
      unsigned mask = op_mask && op_mask[j] ? (unsigned)op_mask[j] : ~0u;
      double m = -INFINITY;
      for (int p = 0; p < nprec; ++p)
        if ((mask >> p) & 1u) m = out[j * nprec + p] > m ? out[j * nprec + p] : m;
      y[(int64_t)b * 4 + j] = rew[b] + (done[b] ? 0.0 : gamma * m);
    }
  }
  free(h1); free(h2); free(out);
}

/* Adam (Kingma & Ba, ICLR 2015), step t >= 1:
 *   m = b1 m + (1 - b1) g;  v = b2 v + (1 - b2) g^2
 *   w -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps) */
void orc_adam(double* w, double* m, double* v, const double* g, int64_t np, int t, double lr,
              double b1, double b2, double eps) {
  double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
  for (int64_t i = 0; i < np; ++i) {
    m[i] = b1 * m[i] + (1.0 - b1) * g[i];
    v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
    double mh = m[i] / c1, vh = v[i] / c2;
    w[i] -= lr * mh / (sqrt(vh) + eps);
  }
}

/* Static matrix features of the MLP policy (READING, an extension):
 *   f0 = log10(n) / 8, f1 = mean nnz per row / 64,
 *   f2 = log10(max a_ii / min a_ii) / 16,
 *   f3 = log10(max_i (sum_j |a_ij|) / a_ii) / 16   (Gershgorin radius over the diagonal),
 *   f4 = fraction of |a_ij| outside the fp16 normal range [2^-14, 65504]. */
void orc_static_features(int n, const int32_t* rp, const int32_t* ci, const double* val,
                         double* f) {
  double dmax = 0, dmin = INFINITY, gmax = 0;
  int64_t outside = 0;
  for (int i = 0; i < n; ++i) {
    double d = 0, rs = 0;
    for (int32_t e = rp[i]; e < rp[i + 1]; ++e) {
      double a = fabs(val[e]);
      rs += a;
      if (ci[e] == i) d = val[e];
      if (a != 0 && (a < 0x1.0p-14 || a > 65504.0)) ++outside;
    }
    if (d > dmax) dmax = d;
    if (d < dmin) dmin = d;
    double g = d > 0 ? rs / d : 0;
    if (g > gmax) gmax = g;
  }
  int64_t nnz = n > 0 ? rp[n] : 0;
  f[0] = n > 0 ? log10((double)n) / 8.0 : 0;
  f[1] = n > 0 ? ((double)nnz / n) / 64.0 : 0;
  f[2] = (dmin > 0 && dmax > 0) ? log10(dmax / dmin) / 16.0 : 0;
  f[3] = gmax > 0 ? log10(gmax) / 16.0 : 0;
  f[4] = nnz > 0 ? (double)outside / (double)nnz : 0;
}

/* Dynamic features at iteration k (READING, an extension):
 *   f5 = k / t_bin, f6 = -log10(max(rho_k, eps_min)) / 16,
 *   f7 = log10(rho_k / rho_{k-1}), f8 = log10(rho_k / rho_{k-8}) / 8  (0 when not available),
 *   f9 = log10|alpha_{k-1}| / 8, f10 = log10|beta_{k-1}| / 8 (0 when not available),
 *   f11 = log10(rho_true / rho_rec) at the last replacement (0 if none),
 *   f12..f15 = previous action indices / (nprec - 1) (0 at k = 0). */
typedef struct {
  double rho_hist[9];  /* rho_k, rho_{k-1}, ..., rho_{k-8} (0 = unknown) */
  double alpha_prev, beta_prev, gap_log;
  int prev_act[4];
  int have_prev;
} orc_feat_state;

static double safe_log10(double v) { return v > 0 ? log10(v) : 0.0; }

void orc_dynamic_features(const orc_opts* o, int k, const orc_feat_state* st, double* f) {
  double rho = st->rho_hist[0];
  double rr = rho > o->eps_min ? rho : o->eps_min;
  f[5] = (double)k / (double)o->t_bin;
  f[6] = -log10(rr) / 16.0;
  f[7] = (st->rho_hist[1] > 0 && rho > 0) ? log10(rho / st->rho_hist[1]) : 0.0;
  f[8] = (st->rho_hist[8] > 0 && rho > 0) ? log10(rho / st->rho_hist[8]) / 8.0 : 0.0;
  f[9] = st->have_prev ? safe_log10(fabs(st->alpha_prev)) / 8.0 : 0.0;
  f[10] = st->have_prev ? safe_log10(fabs(st->beta_prev)) / 8.0 : 0.0;
  f[11] = st->gap_log;
  for (int j = 0; j < 4; ++j)
    f[12 + j] = (st->have_prev && o->nprec > 1) ? (double)st->prev_act[j] / (double)(o->nprec - 1) : 0.0;
}

/* ------------------------------------------------------------------------- */
/* CG building blocks (Section 3, Section 4.2).                                */
/* ------------------------------------------------------------------------- */

/* q = fl_p1(A^(p1) fl_p1(p)), sums in fp64 in index order. For a row-scaled p1 the
 * entries are s_i fl_f(a_ij / s_i) and the output rounding is applied before the
 * scale: q_i = s_i fl_f(sum_j fl_f(a_ij / s_i) fl_f(p_j)). */
void orc_spmv(int n, const int32_t* rp, const int32_t* ci, const double* val, int fmt,
              const double* p, double* q) {
  for (int i = 0; i < n; ++i) {
    double s = is_row_scaled(fmt) ? orc_row_scale(rp, val, i) : 1.0;
    double acc = 0.0;
    for (int32_t e = rp[i]; e < rp[i + 1]; ++e)
      acc += orc_chop(val[e] / s, fmt) * orc_chop(p[ci[e]], fmt);
    q[i] = s * orc_chop(acc, fmt);
  }
}

/* fl_p(x^T y) = fl_p(sum_i fl_p(x_i) fl_p(y_i)), fp64 sum in index order. */
double orc_dot(int64_t n, const double* x, const double* y, int fmt) {
  double acc = 0.0;
  for (int64_t i = 0; i < n; ++i) acc += orc_chop(x[i], fmt) * orc_chop(y[i], fmt);
  return orc_chop(acc, fmt);
}

/* r_t = b - A x in fp64 (the residual recomputation kept in fp64, abstract). Returns ||r_t||^2. */
double orc_true_residual(int n, const int32_t* rp, const int32_t* ci, const double* val,
                         const double* b, const double* x, double* rt) {
  double nn = 0.0;
  for (int i = 0; i < n; ++i) {
    double acc = 0.0;
    for (int32_t e = rp[i]; e < rp[i + 1]; ++e) acc += val[e] * x[ci[e]];
    rt[i] = b[i] - acc;
    nn += rt[i] * rt[i];
  }
  return nn;
}

/* ------------------------------------------------------------------------- */
/* Incomplete Cholesky preconditioner in fp32 (Section 5's fixed-precision    */
/* preconditioner M ~ A, p_fixed = fp32).                                     */
/* ------------------------------------------------------------------------- */

/* READING: Section 5 factors with an fp32 incomplete LU (drop tolerance 1e-4, fill factor 10).
 * For SPD A this is taken as its symmetric, zero-fill form IC(0): M = L L^T with L lower
 * triangular on the pattern of A's lower triangle and (L L^T)_ij = a_ij wherever a_ij is
 * stored (Meijerink and van der Vorst 1977, the reference the paper cites for M). Every
 * operation runs in fp32 (the paper's p_fixed), rows in order, each sum over increasing
 * column index:
 *   l_ij = (fl32(a_ij) - sum_{k<j} l_ik l_jk) / l_jj   for stored j < i,
 *   l_ii = sqrt(fl32(a_ii) - sum_{k<i} l_ik^2),
 * the sums running over the columns k stored in both rows i and j.
 * Output layout: one fp32 per stored entry of A; position (i, j) holds l_ij for j <= i and
 * the transposed factor value l_ji for j > i (row i of L^T).
 * Returns 0; -2 for a non-positive or non-finite pivot (IC(0) breaks down; it exists for
 * M-matrices but not for every SPD matrix); -3 when a row lacks its diagonal, its columns are
 * not strictly increasing, or the pattern is not symmetric. */
int orc_ic0(int n, const int32_t* rp, const int32_t* ci, const double* val, float* L) {
  for (int i = 0; i < n; ++i) {
    for (int32_t e = rp[i] + 1; e < rp[i + 1]; ++e)
      if (ci[e] <= ci[e - 1]) return -3;
  }
  for (int i = 0; i < n; ++i) {
    int32_t di = -1;
    for (int32_t e = rp[i]; e < rp[i + 1]; ++e) {
      const int j = ci[e];
      if (j > i) break;
      if (j == i) {
        di = e;
        break;
      }
      /* l_ij: merge row i's entries left of column j with row j's entries left of column j */
      float s = (float)val[e];
      int32_t a = rp[i], c = rp[j];
      while (a < e && c < rp[j + 1] && ci[c] < j) {
        if (ci[a] < ci[c]) {
          ++a;
        } else if (ci[a] > ci[c]) {
          ++c;
        } else {
          s = s - L[a] * L[c];
          ++a;
          ++c;
        }
      }
      int32_t dj = -1;
      for (int32_t f = rp[j]; f < rp[j + 1]; ++f)
        if (ci[f] == j) dj = f;
      if (dj < 0) return -3;
      L[e] = s / L[dj];
    }
    if (di < 0) return -3;
    float s = (float)val[di];
    for (int32_t e = rp[i]; e < di; ++e) s = s - L[e] * L[e];
    if (!(s > 0.0f) || !isfinite(s)) return -2;
    L[di] = sqrtf(s);
  }
  /* upper part: position (i, j), j > i, takes l_ji from row j; every off-diagonal entry
   * needs its transposed partner */
  for (int i = 0; i < n; ++i) {
    for (int32_t e = rp[i]; e < rp[i + 1]; ++e) {
      const int j = ci[e];
      if (j == i) continue;
      int32_t t = -1;
      for (int32_t f = rp[j]; f < rp[j + 1]; ++f)
        if (ci[f] == i) t = f;
      if (t < 0) return -3;
      if (j > i) L[e] = L[t];
    }
  }
  return 0;
}

/* w = M^-1 r with M = L L^T from orc_ic0, in fp32: the input rounded to fp32, the forward
 * substitution L y = fl32(r) in increasing row order, then the backward substitution
 * L^T w = y in decreasing row order; each row's sum over its stored columns in increasing
 * order, then one division by l_ii. w is returned as fp64 (its values are fp32 numbers). */
void orc_ic0_apply(int n, const int32_t* rp, const int32_t* ci, const float* L, const double* r,
                   double* w) {
  float* y = malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
  float* z = malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
  for (int i = 0; i < n; ++i) {
    float s = (float)r[i];
    int32_t di = rp[i];
    for (int32_t e = rp[i]; e < rp[i + 1]; ++e) {
      if (ci[e] >= i) {
        di = e;
        break;
      }
      s = s - L[e] * y[ci[e]];
    }
    y[i] = s / L[di];
  }
  for (int i = n - 1; i >= 0; --i) {
    float s = y[i];
    int32_t di = rp[i];
    for (int32_t e = rp[i]; e < rp[i + 1]; ++e)
      if (ci[e] == i) di = e;
    for (int32_t e = di + 1; e < rp[i + 1]; ++e) s = s - L[e] * z[ci[e]];
    z[i] = s / L[di];
  }
  for (int i = 0; i < n; ++i) w[i] = (double)z[i];
  free(y);
  free(z);
}

/* ------------------------------------------------------------------------- */
/* One episode: Algorithm 2 (inference) or Algorithm 1's inner loop (training). */
/* ------------------------------------------------------------------------- */

enum { ORC_MODE_INFER = 0, ORC_MODE_TRAIN = 1 };

typedef struct {
  int32_t s, s_next, act[4];
  double reward;
  int32_t terminal, pad;
} orc_transition;

/* Select the action of operation-table j in state s.
 *   inference: greedy first-index argmax; a never-updated row falls back (READING)
 *   training : epsilon-greedy, draws from orc_draw(...) */
/* ---- One table over joint actions (Section 4.1's alternative to a table per operation) --
 * READING: Section 4.1 sets a table per operation against the |P|^m joint actions; the joint
 * form is Q(s, a) with a = (a_1, a_2, a_3, a_4), stored at index ((a_1 |P| + a_2) |P| + a_3) |P|
 * + a_4 of state s's row ([S][|P|^4]), update counts per state. The joint set is the product of
 * the operations' allowed sets (op_mask); greedy: the first joint index with the largest value
 * among the allowed ones (op 1 the most significant digit); a never-updated state takes the
 * fallback format for every operation when all four allow it; exploration: operation 1's draw
 * decides (u < epsilon), each operation's pick comes from its own draw (uniform over the
 * product set); update: Q(s, a) += lr (R + gamma max_{a' allowed} Q(s', a') - Q(s, a)). */
static int joint_size(const orc_opts* o) { return o->nprec * o->nprec * o->nprec * o->nprec; }

static void joint_decode(const orc_opts* o, int a, int act[4]) {
  for (int j = 3; j >= 0; --j) {
    act[j] = a % o->nprec;
    a /= o->nprec;
  }
}

static int joint_ok(const orc_opts* o, int a) {
  int act[4];
  joint_decode(o, a, act);
  for (int j = 0; j < 4; ++j)
    if (!allowed(o, j, act[j])) return 0;
  return 1;
}

static int joint_argmax(const orc_opts* o, const double* row) {
  int best = -1;
  for (int a = 0; a < joint_size(o); ++a)
    if (joint_ok(o, a) && (best < 0 || row[a] > row[best])) best = a;
  return best;
}

static double joint_max(const orc_opts* o, const double* row) {
  double m = -INFINITY;
  for (int a = 0; a < joint_size(o); ++a)
    if (joint_ok(o, a) && row[a] > m) m = row[a];
  return m;
}

static void select_joint(const orc_opts* o, const orc_policy* pol, int mode, int s, double eps, uint64_t ep,
                         uint64_t lane, int k, int act[4], int* explored) {
  const double* row = pol->Q + (int64_t)s * joint_size(o);
  if (mode == ORC_MODE_TRAIN) {
    double u[4];
    uint32_t pick[4];
    for (int j = 0; j < 4; ++j) orc_draw(o->seed, ep, lane, (uint64_t)k, (uint64_t)j, &u[j], &pick[j]);
    if (u[0] < eps) {
      *explored = 1;
      for (int j = 0; j < 4; ++j) act[j] = random_allowed(o, j, pick[j]);
      return;
    }
  } else if (o->unvisited_fallback >= 0 && pol->visits[s] == 0) {
    int a = index_of(o, o->unvisited_fallback);
    int all = a >= 0;
    for (int j = 0; j < 4; ++j) all = all && allowed(o, j, a);
    if (all) {
      for (int j = 0; j < 4; ++j) act[j] = a;
      return;
    }
  }
  joint_decode(o, joint_argmax(o, row), act);
}

static int select_qtable(const orc_opts* o, const orc_policy* pol, int mode, int j, int s,
                         double eps, uint64_t ep, uint64_t lane, int k, int* explored) {
  int S = o->b_bins * o->r_bins;
  const double* row = pol->Q + ((int64_t)j * S + s) * o->nprec;
  if (mode == ORC_MODE_TRAIN) {
    double u;
    uint32_t pick;
    orc_draw(o->seed, ep, lane, (uint64_t)k, (uint64_t)j, &u, &pick);
    if (u < eps) {
      *explored = 1;
      return random_allowed(o, j, pick);
    }
    return argmax_allowed(o, j, row);
  }
  if (o->unvisited_fallback >= 0 && pol->visits[(int64_t)j * S + s] == 0) {
    int a = index_of(o, o->unvisited_fallback);
    return (a >= 0 && allowed(o, j, a)) ? a : argmax_allowed(o, j, row);
  }
  return argmax_allowed(o, j, row);
}

/* Algorithm 2's decision at iteration k with residual rho_k: state s = (i_k, j_k) of
 * Section 4.1, then per operation the greedy entry of Q_j(s, .) (first-index argmax over the
 * allowed entries; a never-updated row takes the fallback). act[j] receives indices into
 * precs. Returns s. */
int orc_greedy_action(const orc_opts* o, const double* Q, const int32_t* visits, int k, double rho,
                      int32_t act[4]) {
  orc_policy pol;
  memset(&pol, 0, sizeof(pol));
  pol.kind = ORC_POL_QTABLE;
  pol.Q = (double*)Q;
  pol.visits = (int32_t*)visits;
  int s = orc_state(o, k, rho);
  int explored = 0;
  if (o->joint) {
    int a[4];
    select_joint(o, &pol, ORC_MODE_INFER, s, 0.0, 0, 0, k, a, &explored);
    for (int j = 0; j < 4; ++j) act[j] = a[j];
  } else {
    for (int j = 0; j < 4; ++j) act[j] = select_qtable(o, &pol, ORC_MODE_INFER, j, s, 0.0, 0, 0, k, &explored);
  }
  return s;
}

/* Q_j(s, a_j) += lr (R + gamma max_{p in P_j} Q_j(s', p) - Q_j(s, a_j))   (Section 4.1, Alg. 1 non-terminal)
 * Q_j(s, a_j) += lr (R - Q_j(s, a_j))                                    (Alg. 1 terminal)
 * P_j is operation j's allowed set (all of P unless op_mask[j] restricts it). */
void orc_q_update(const orc_opts* o, double* Q, int32_t* visits, const orc_transition* t) {
  int S = o->b_bins * o->r_bins;
  if (o->joint) {
    /* the joint table: one update of the joint action's entry */
    int a = 0;
    for (int j = 0; j < 4; ++j) a = a * o->nprec + t->act[j];
    double* row = Q + (int64_t)t->s * joint_size(o);
    double target = t->reward;
    if (!t->terminal) target += o->gamma * joint_max(o, Q + (int64_t)t->s_next * joint_size(o));
    row[a] += o->lr * (target - row[a]);
    if (visits) visits[t->s] += 1;
    return;
  }
  for (int j = 0; j < 4; ++j) {
    double* row = Q + ((int64_t)j * S + t->s) * o->nprec;
    double target = t->reward;
    if (!t->terminal) target += o->gamma * max_allowed(o, j, Q + ((int64_t)j * S + t->s_next) * o->nprec);
    row[t->act[j]] += o->lr * (target - row[t->act[j]]);
    if (visits) visits[(int64_t)j * S + t->s] += 1;
  }
}

/* Applies Algorithm 1's Q update for one transition (when the policy learns online)
 * and appends the transition to the caller's list (when one is given). */
static void learn_step(const orc_opts* o, orc_policy* pol, const orc_transition* t,
                       orc_transition* trans, int32_t* ntrans) {
  if (pol->kind == ORC_POL_QTABLE && pol->Q) orc_q_update(o, pol->Q, pol->visits, t);
  if (trans) trans[(*ntrans)++] = *t;
}

/* The action of iteration k in state s (Algorithm 1's epsilon-greedy choice in training,
 * Algorithm 2's greedy choice in inference, or the fixed / replayed formats): fmt[j] the
 * format of operation j, act[j] its index in P (-1 when the format is not in P). f holds the
 * MLP policy's features; h1, h2, qout are its work arrays. */
static void choose_formats(const orc_opts* o, const orc_policy* pol, int mode, int k, int s, double eps,
                           uint64_t ep, uint64_t lane, int locked, const double* f, int H, int nout,
                           double* h1, double* h2, double* qout, int fmt[4], int act[4], int* explored) {
  if (locked) {
    for (int j = 0; j < 4; ++j) fmt[j] = ORC_FP64;
  } else if (pol->kind == ORC_POL_FIXED) {
    for (int j = 0; j < 4; ++j) fmt[j] = pol->fixed[j];
  } else if (pol->kind == ORC_POL_SCHEDULE) {
    int row = k < pol->sched_len ? k : pol->sched_len - 1;
    for (int j = 0; j < 4; ++j) fmt[j] = pol->sched[(int64_t)row * 4 + j];
  } else if (pol->kind == ORC_POL_QTABLE && o->joint) {
    select_joint(o, pol, mode, s, eps, ep, lane, k, act, explored);
    for (int j = 0; j < 4; ++j) fmt[j] = o->precs[act[j]];
  } else if (pol->kind == ORC_POL_QTABLE) {
    for (int j = 0; j < 4; ++j) {
      int ex = 0;
      act[j] = select_qtable(o, pol, mode, j, s, eps, ep, lane, k, &ex);
      *explored |= ex;
      fmt[j] = o->precs[act[j]];
    }
  } else {
    /* Learned policy: greedy per operation on the MLP's Q-values (same tie rule). */
    orc_mlp_forward(pol->mlp, H, nout, f, h1, h2, qout);
    for (int j = 0; j < 4; ++j) {
      act[j] = argmax_allowed(o, j, qout + j * o->nprec);
      if (mode == ORC_MODE_TRAIN) {
        double u;
        uint32_t pick;
        orc_draw(o->seed, ep, lane, (uint64_t)k, (uint64_t)j, &u, &pick);
        if (u < eps) {
          act[j] = random_allowed(o, j, pick);
          *explored = 1;
        }
      }
      fmt[j] = o->precs[act[j]];
    }
  }
  if (locked || pol->kind == ORC_POL_FIXED || pol->kind == ORC_POL_SCHEDULE)
    for (int j = 0; j < 4; ++j) act[j] = index_of(o, fmt[j]);
}

/* ------------------------------------------------------------------------- */
/* Single-reduction variant of the iteration (a widening beyond the paper).    */
/* ------------------------------------------------------------------------- */

/* Chronopoulos and Gear's form of CG (J. Comput. Appl. Math. 25, 1989), identical to the CG
 * of Section 3 in exact arithmetic, in which every inner product of an iteration is formed
 * from vectors that exist at the same time, so that one global reduction serves a whole
 * iteration. The four operations of Section 4.2 keep their roles:
 *   u_k = fl_p2(M^-1 r_k)                                   (op 2, z of Section 3)
 *   w_k = fl_p1(A fl_p1(u_k))                               (op 1, the product)
 *   gamma_k = fl_p4(sum fl_p4(r_i) fl_p4(u_i))              (op 4, sigma)
 *   delta_k = fl_p3(sum fl_p3(w_i) fl_p3(u_i))              (op 3, the curvature product)
 *   beta_k = gamma_k / gamma_{k-1},  nu_k = delta_k - beta_k gamma_k / alpha_{k-1}
 *     (at k = 0 and after r was replaced: beta_k = 0, nu_k = delta_k)
 *   alpha_k = gamma_k / nu_k                                (fp64 scalars)
 *   p_k = u_k + beta_k p_{k-1},  s_k = w_k + beta_k s_{k-1} (s_k = A p_k in exact arithmetic)
 *   x_{k+1} = x_k + alpha_k p_k,  r_{k+1} = r_k - alpha_k s_k        (fp64)
 * READING (what the variant stops on): the residual norm of the next state comes from the
 * same reduction, expanding ||r_k - alpha_k s_k||^2 with s_k = w_k + beta_k s_{k-1}:
 *   rr_{k+1} = rr_k - 2 alpha_k (r_k.w_k + beta_k r_k.s_{k-1})
 *            + alpha_k^2 (w_k.w_k + 2 beta_k w_k.s_{k-1} + beta_k^2 s_{k-1}.s_{k-1}),
 * with every inner product in fp64 and rr_k = r_k.r_k formed directly, clamped at 0; rho_{k+1} =
 * sqrt(rr_{k+1}) / ||b|| drives the stopping test, the reward and the next state. The
 * breakdown rules, the residual replacement (which restarts the recurrence: beta = 0) and the
 * fp64 restart follow orc_run. Parity unpinned beyond the equality with orc_run's CG in fp64
 * and the step-by-step recomputation of its first iterations (tests). */
int orc_run_sr(const orc_opts* o, int n, const int32_t* rp, const int32_t* ci, const double* val,
               const double* b, double* x, double tau, int max_iter, orc_policy* pol, int mode,
               uint64_t ep, uint64_t lane, double eps, orc_transition* trans, int32_t* ntrans,
               orc_rec* hist, double* feat_out, orc_result* res) {
  size_t nb = sizeof(double) * (size_t)(n > 0 ? n : 1);
  double* r = malloc(nb);
  double* u = malloc(nb);
  double* w = malloc(nb);
  double* p = calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  double* sv = calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  double* rt = malloc(nb);
  double* dinv = malloc(nb);
  int nout = 4 * o->nprec;
  int H = o->mlp_hidden > 0 ? o->mlp_hidden : 1;
  double* h1 = malloc(sizeof(double) * H);
  double* h2 = malloc(sizeof(double) * H);
  double* qout = malloc(sizeof(double) * nout);
  orc_feat_state fs;
  memset(&fs, 0, sizeof(fs));
  if (ntrans) *ntrans = 0;
  for (int i = 0; i < n; ++i) dinv[i] = 1.0;
  if (o->precond == 1) {
    for (int i = 0; i < n; ++i) {
      double d = 0.0;
      for (int e = rp[i]; e < rp[i + 1]; ++e)
        if (ci[e] == i) d = val[e];
      if (!(d > 0.0)) {
        free(r); free(u); free(w); free(p); free(sv); free(rt); free(dinv); free(h1); free(h2); free(qout);
        return -1;
      }
      dinv[i] = 1.0 / d;
    }
  } else if (o->precond != 0) {
    free(r); free(u); free(w); free(p); free(sv); free(rt); free(dinv); free(h1); free(h2); free(qout);
    return -4;
  }
  double bb = 0.0;
  for (int i = 0; i < n; ++i) bb += b[i] * b[i];
  double bnorm = sqrt(bb);
  double rr = orc_true_residual(n, rp, ci, val, b, x, r);
  double rho = bnorm > 0 ? sqrt(rr) / bnorm : 0.0;
  int outcome = ORC_MAX_ITER, iters = max_iter, nrec = 0;
  if (n == 0 || bnorm == 0.0) {
    for (int i = 0; i < n; ++i) x[i] = 0.0;
    outcome = ORC_CONVERGED;
    iters = 0;
    rho = 0.0;
    max_iter = 0;
  }
  fs.rho_hist[0] = rho;
  int locked = 0, restart = 1;
  double gamma_prev = 0.0, alpha_prev = 0.0;
  double fstat[5] = {0, 0, 0, 0, 0};
  if (pol->feat_static) memcpy(fstat, pol->feat_static, sizeof(fstat));

  for (int k = 0; k < max_iter; ++k) {
    int s = orc_state(o, k, rho);
    int fmt[4], act[4], explored = 0;
    double f[ORC_NFEAT];
    for (int j = 0; j < 5; ++j) f[j] = fstat[j];
    orc_dynamic_features(o, k, &fs, f);
    if (feat_out) memcpy(feat_out + (int64_t)k * ORC_NFEAT, f, sizeof(f));
    choose_formats(o, pol, mode, k, s, eps, ep, lane, locked, f, H, nout, h1, h2, qout, fmt, act, &explored);
    int learn = mode == ORC_MODE_TRAIN && act[0] >= 0 && act[1] >= 0 && act[2] >= 0 && act[3] >= 0;
    orc_rec rec;
    memset(&rec, 0, sizeof(rec));
    rec.k = k;
    rec.state = s;
    for (int j = 0; j < 4; ++j) { rec.fmt[j] = fmt[j]; rec.act[j] = act[j]; }
    rec.flags = explored ? 8 : 0;
    rec.rho = rho;

    /* u_k = fl_p2(M^-1 r_k); w_k = fl_p1(A fl_p1(u_k)); gamma_k, delta_k */
    for (int i = 0; i < n; ++i) u[i] = orc_chop(o->precond == 1 ? r[i] * dinv[i] : r[i], fmt[1]);
    orc_spmv(n, rp, ci, val, fmt[0], u, w);
    double gamma = orc_dot(n, r, u, fmt[3]);
    double delta = orc_dot(n, w, u, fmt[2]);
    double beta = restart ? 0.0 : gamma / gamma_prev;
    double nu = restart ? delta : delta - beta * gamma / alpha_prev;
    double alpha = gamma / nu;
    rec.nu = nu;
    rec.alpha = alpha;
    rec.sigma = gamma;
    rec.beta = beta;
    int stop = 0;
    orc_transition t = {s, s, {act[0], act[1], act[2], act[3]}, 0.0, 1, 0};
    if (!(nu > 0.0) || !isfinite(nu) || !isfinite(alpha) || !isfinite(beta)) {
      if (rho < tau && isfinite(nu)) {
        outcome = ORC_CONVERGED;
        iters = k;
        rec.flags |= 1;
        t.reward = learn ? orc_reward(o, rho, act, tau) : 0.0;
      } else {
        outcome = ORC_BREAKDOWN;
        iters = k;
        rec.flags |= 2;
        t.reward = learn ? orc_reward_breakdown(o, act) : 0.0;
      }
      stop = 1;
    } else {
      /* the inner products of the norm recurrence (fp64, the vectors before the update) */
      double rr_k = 0.0, rw = 0.0, rs = 0.0, ww = 0.0, ws = 0.0, ss = 0.0;
      for (int i = 0; i < n; ++i) {
        rr_k += r[i] * r[i];
        rw += r[i] * w[i];
        rs += r[i] * sv[i];
        ww += w[i] * w[i];
        ws += w[i] * sv[i];
        ss += sv[i] * sv[i];
      }
      double rr_next = rr_k - 2.0 * alpha * (rw + beta * rs) + alpha * alpha * (ww + 2.0 * beta * ws + beta * beta * ss);
      if (rr_next < 0.0) rr_next = 0.0;
      double rho_rec = sqrt(rr_next) / bnorm;
      /* p_k, s_k, x_{k+1}, r_{k+1} (fp64) */
      for (int i = 0; i < n; ++i) {
        p[i] = u[i] + beta * p[i];
        sv[i] = w[i] + beta * sv[i];
        x[i] = x[i] + alpha * p[i];
        r[i] = r[i] - alpha * sv[i];
      }
      double rho_new = rho_rec;
      int check = (o->true_res_every > 0 && (k + 1) % o->true_res_every == 0) ||
                  (o->true_res_at_conv && rho_rec < tau && k >= o->min_k);
      int replaced = 0;
      if (check && isfinite(rho_rec)) {
        double nt = orc_true_residual(n, rp, ci, val, b, x, rt);
        for (int i = 0; i < n; ++i) r[i] = rt[i];
        double rho_t = sqrt(nt) / bnorm;
        fs.gap_log = (rho_t > 0 && rho_rec > 0) ? log10(rho_t / rho_rec) : 0.0;
        rho_new = rho_t;
        rec.flags |= 4;
        replaced = 1;
      }
      rec.rho = rho_new;
      if (!isfinite(rho_new)) {
        outcome = ORC_BREAKDOWN;
        iters = k + 1;
        rec.flags |= 2;
        t.reward = learn ? orc_reward_breakdown(o, act) : 0.0;
        stop = 1;
      } else if (rho_new < tau && k >= o->min_k) {
        outcome = ORC_CONVERGED;
        iters = k + 1;
        rec.flags |= 1;
        t.reward = learn ? orc_reward(o, rho_new, act, tau) : 0.0;
        rho = rho_new;
        stop = 1;
      } else {
        t.reward = learn ? orc_reward(o, rho_new, act, tau) : 0.0;
        t.s_next = orc_state(o, k + 1, rho_new);
        t.terminal = 0;
        gamma_prev = gamma;
        alpha_prev = alpha;
        restart = replaced;
        for (int h = 8; h > 0; --h) fs.rho_hist[h] = fs.rho_hist[h - 1];
        fs.rho_hist[0] = rho_new;
        fs.alpha_prev = alpha;
        fs.beta_prev = beta;
        fs.have_prev = 1;
        for (int j = 0; j < 4; ++j) fs.prev_act[j] = act[j] >= 0 ? act[j] : 0;
        rho = rho_new;
      }
    }
    if (stop && outcome == ORC_BREAKDOWN && mode == ORC_MODE_INFER && o->on_breakdown && !locked) {
      /* fp64 restart from the current x (as orc_run): r = b - A x, the recurrence restarts */
      double nt = orc_true_residual(n, rp, ci, val, b, x, r);
      for (int i = 0; i < n; ++i) p[i] = sv[i] = 0.0;
      rho = sqrt(nt) / bnorm;
      locked = 1;
      restart = 1;
      rec.flags |= 16;
      for (int h = 8; h > 0; --h) fs.rho_hist[h] = fs.rho_hist[h - 1];
      fs.rho_hist[0] = rho;
      stop = 0;
      outcome = ORC_MAX_ITER;
      iters = max_iter;
      if (!isfinite(rho)) {
        outcome = ORC_BREAKDOWN;
        iters = k + 1;
        stop = 1;
      } else if (rho < tau && k >= o->min_k) {
        outcome = ORC_CONVERGED;
        iters = k + 1;
        stop = 1;
      }
    }
    rec.reward = t.reward;
    if (learn) learn_step(o, pol, &t, trans, ntrans);
    if (hist) hist[k] = rec;
    nrec = k + 1;
    if (stop) break;
  }
  if (feat_out && outcome != ORC_CONVERGED && outcome != ORC_BREAKDOWN && max_iter > 0) {
    double f[ORC_NFEAT];
    for (int j = 0; j < 5; ++j) f[j] = fstat[j];
    orc_dynamic_features(o, max_iter, &fs, f);
    memcpy(feat_out + (int64_t)max_iter * ORC_NFEAT, f, sizeof(f));
  }
  if (res) {
    res->outcome = outcome;
    res->iters = iters;
    res->nrec = nrec;
    double nt = orc_true_residual(n, rp, ci, val, b, x, rt);
    res->rho_true = bnorm > 0 ? sqrt(nt) / bnorm : 0.0;
    double r2 = 0.0;
    for (int i = 0; i < n; ++i) r2 += r[i] * r[i];
    res->rho_rec = bnorm > 0 ? sqrt(r2) / bnorm : 0.0;
  }
  free(r); free(u); free(w); free(p); free(sv); free(rt); free(dinv); free(h1); free(h2); free(qout);
  return outcome;
}

/* Runs one CG solve with the given policy.
 *   mode INFER: Algorithm 2. mode TRAIN: Algorithm 1's episode body with epsilon-greedy
 *   selection; a QTABLE policy's tables are updated online after every iteration
 *   (Algorithm 1), and every transition is also appended to trans (if non-NULL).
 * x holds x_0 on entry (Algorithms 1 and 2 use x_0 = 0) and the final iterate on exit.
 * hist (optional) receives one record per iteration; feat_out (optional, [max_iter + 1][16])
 * receives the MLP feature vector of every visited state. */
int orc_run(const orc_opts* o, int n, const int32_t* rp, const int32_t* ci, const double* val,
            const double* b, double* x, double tau, int max_iter, orc_policy* pol, int mode,
            uint64_t ep, uint64_t lane, double eps, orc_transition* trans, int32_t* ntrans,
            orc_rec* hist, double* feat_out, orc_result* res) {
  if (o->variant == 1)
    return orc_run_sr(o, n, rp, ci, val, b, x, tau, max_iter, pol, mode, ep, lane, eps, trans, ntrans, hist,
                      feat_out, res);
  size_t nb = sizeof(double) * (size_t)(n > 0 ? n : 1);
  double* r = malloc(nb);
  double* p = malloc(nb);
  double* q = malloc(nb);
  double* z = malloc(nb);
  double* rt = malloc(nb);
  int nout = 4 * o->nprec;
  int H = o->mlp_hidden > 0 ? o->mlp_hidden : 1;
  double* h1 = malloc(sizeof(double) * H);
  double* h2 = malloc(sizeof(double) * H);
  double* qout = malloc(sizeof(double) * nout);
  orc_feat_state fs;
  memset(&fs, 0, sizeof(fs));
  if (ntrans) *ntrans = 0;

  /* M^-1 as the fp64 reciprocals of the diagonal (Jacobi) or the identity. A row without a
   * positive diagonal entry makes Jacobi undefined: the solve is refused (return -1). */
  double* dinv = malloc(nb);
  int64_t nnz = n > 0 ? rp[n] : 0;
  float* icl = malloc(sizeof(float) * (size_t)(nnz > 0 ? nnz : 1));
  for (int i = 0; i < n; ++i) dinv[i] = 1.0;
  if (o->precond == 1) {
    for (int i = 0; i < n; ++i) {
      double d = 0.0;
      for (int e = rp[i]; e < rp[i + 1]; ++e)
        if (ci[e] == i) d = val[e];
      if (!(d > 0.0)) {
        free(r); free(p); free(q); free(z); free(rt); free(h1); free(h2); free(qout); free(dinv); free(icl);
        return -1;
      }
      dinv[i] = 1.0 / d;
    }
  }
  /* IC(0) in fp32 (precond 2): factored once per solve; a breakdown refuses the solve. */
  if (o->precond == 2) {
    int rc = orc_ic0(n, rp, ci, val, icl);
    if (rc < 0) {
      free(r); free(p); free(q); free(z); free(rt); free(h1); free(h2); free(qout); free(dinv); free(icl);
      return rc;
    }
  }
  /* Initialisation (Algorithms 1 and 2): r_0 = b - A x_0, z_0 = M^-1 r_0, p_0 = z_0,
   * sigma_0 = r_0^T z_0, b_norm = ||b||_2; all in fp64. */
  double bb = 0.0;
  for (int i = 0; i < n; ++i) bb += b[i] * b[i];
  double bnorm = sqrt(bb);
  double rr0 = orc_true_residual(n, rp, ci, val, b, x, r);
  double sigma = 0.0;
  if (o->precond == 2) orc_ic0_apply(n, rp, ci, icl, r, z);
  for (int i = 0; i < n; ++i) {
    p[i] = o->precond == 2 ? z[i] : o->precond == 1 ? r[i] * dinv[i] : r[i];
    sigma += r[i] * p[i];
  }
  double rho = bnorm > 0 ? sqrt(rr0) / bnorm : 0.0;
  int outcome = ORC_MAX_ITER, iters = max_iter, nrec = 0;
  if (n == 0 || bnorm == 0.0) {
    /* b = 0: x = 0 solves the system exactly. */
    for (int i = 0; i < n; ++i) x[i] = 0.0;
    outcome = ORC_CONVERGED;
    iters = 0;
    rho = 0.0;
    max_iter = 0;
  }
  fs.rho_hist[0] = rho;
  int locked = 0, restarts = 0; /* fp64 restart after a breakdown (option on_breakdown) */
  double fstat[5] = {0, 0, 0, 0, 0};
  if (pol->feat_static) memcpy(fstat, pol->feat_static, sizeof(fstat));

  for (int k = 0; k < max_iter; ++k) {
    /* State s_k = discretize(k, ||r_k|| / b_norm)  (Section 4.1). */
    int s = orc_state(o, k, rho);
    int fmt[4], act[4], explored = 0;
    double f[ORC_NFEAT];
    for (int j = 0; j < 5; ++j) f[j] = fstat[j];
    orc_dynamic_features(o, k, &fs, f);
    if (feat_out) memcpy(feat_out + (int64_t)k * ORC_NFEAT, f, sizeof(f));
    choose_formats(o, pol, mode, k, s, eps, ep, lane, locked, f, H, nout, h1, h2, qout, fmt, act, &explored);
    int learn = mode == ORC_MODE_TRAIN && act[0] >= 0 && act[1] >= 0 && act[2] >= 0 && act[3] >= 0;

    orc_rec rec;
    memset(&rec, 0, sizeof(rec));
    rec.k = k;
    rec.state = s;
    for (int j = 0; j < 4; ++j) { rec.fmt[j] = fmt[j]; rec.act[j] = act[j]; }
    rec.flags = explored ? 8 : 0;
    rec.rho = rho;

    /* q_k = fl_p1(A p_k); nu_k = fl_p3(p_k^T q_k); alpha_k = sigma_k / nu_k (fp64). */
    orc_spmv(n, rp, ci, val, fmt[0], p, q);
    double nu = orc_dot(n, p, q, fmt[2]);
    double alpha = sigma / nu;
    rec.nu = nu;
    rec.alpha = alpha;
    int stop = 0;
    orc_transition t = {s, s, {act[0], act[1], act[2], act[3]}, 0.0, 1, 0};
    if (!(nu > 0.0) || !isfinite(nu) || !isfinite(alpha)) {
      if (rho < tau && isfinite(nu)) {
        /* READING: the residual is already below tau (it reached exactly zero before the
         * k >= min_k rule allowed a stop), so p = 0 and nu = 0: the solve is exact. */
        outcome = ORC_CONVERGED;
        iters = k;
        rec.flags |= 1;
        t.reward = learn ? orc_reward(o, rho, act, tau) : 0.0;
      } else {
        /* READING: breakdown (non-positive or non-finite curvature); x stays x_k. */
        outcome = ORC_BREAKDOWN;
        iters = k;
        rec.flags |= 2;
        t.reward = learn ? orc_reward_breakdown(o, act) : 0.0;
      }
      stop = 1;
    } else {
      /* x_{k+1} = x_k + alpha p_k; r_{k+1} = r_k - alpha q_k (fp64, Section 4.2). */
      double rr = 0.0;
      for (int i = 0; i < n; ++i) {
        x[i] = x[i] + alpha * p[i];
        r[i] = r[i] - alpha * q[i];
        rr += r[i] * r[i];
      }
      double rho_rec = sqrt(rr) / bnorm;
      double rho_new = rho_rec;
      /* Residual recomputation b - A x in fp64 (an extension): periodic replacement and
       * confirmation of a claimed convergence. */
      int check = (o->true_res_every > 0 && (k + 1) % o->true_res_every == 0) ||
                  (o->true_res_at_conv && rho_rec < tau && k >= o->min_k);
      if (check && isfinite(rho_rec)) {
        double nt = orc_true_residual(n, rp, ci, val, b, x, rt);
        for (int i = 0; i < n; ++i) r[i] = rt[i];
        double rho_t = sqrt(nt) / bnorm;
        fs.gap_log = (rho_t > 0 && rho_rec > 0) ? log10(rho_t / rho_rec) : 0.0;
        rho_new = rho_t;
        rec.flags |= 4;
      }
      rec.rho = rho_new;
      if (!isfinite(rho_new)) {
        outcome = ORC_BREAKDOWN;
        iters = k + 1;
        rec.flags |= 2;
        t.reward = learn ? orc_reward_breakdown(o, act) : 0.0;
        stop = 1;
      } else if (rho_new < tau && k >= o->min_k) {
        /* Stop test (Algorithms 1 and 2; Section 5 adds k >= 10). */
        outcome = ORC_CONVERGED;
        iters = k + 1;
        rec.flags |= 1;
        t.reward = learn ? orc_reward(o, rho_new, act, tau) : 0.0;
        rho = rho_new;
        stop = 1;
      } else {
        /* z_{k+1} = fl_p2(M^-1 r_{k+1}) (M = I; the fp64 product r_i d_i for Jacobi; the fp32
         * IC(0) solves), rounded once; sigma_{k+1} = fl_p4(r^T z); beta_k = sigma_{k+1} /
         * sigma_k (fp64). */
        if (o->precond == 2) orc_ic0_apply(n, rp, ci, icl, r, z);
        for (int i = 0; i < n; ++i)
          z[i] = orc_chop(o->precond == 2 ? z[i] : o->precond == 1 ? r[i] * dinv[i] : r[i], fmt[1]);
        double sigma_new = orc_dot(n, r, z, fmt[3]);
        /* READING: after r was replaced by b - A x the old direction no longer matches the
         * residual history, so the iteration restarts with beta = 0 (p_{k+1} = z_{k+1}). */
        double beta = (rec.flags & 4) ? 0.0 : sigma_new / sigma;
        rec.sigma = sigma_new;
        rec.beta = beta;
        if (!isfinite(sigma_new) || !isfinite(beta)) {
          outcome = ORC_BREAKDOWN;
          iters = k + 1;
          rec.flags |= 2;
          t.reward = learn ? orc_reward_breakdown(o, act) : 0.0;
          stop = 1;
        } else {
          /* p_{k+1} = z_{k+1} + beta_k p_k (fp64). */
          for (int i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
          t.reward = learn ? orc_reward(o, rho_new, act, tau) : 0.0;
          t.s_next = orc_state(o, k + 1, rho_new);
          t.terminal = 0;
          sigma = sigma_new;
          for (int h = 8; h > 0; --h) fs.rho_hist[h] = fs.rho_hist[h - 1];
          fs.rho_hist[0] = rho_new;
          fs.alpha_prev = alpha;
          fs.beta_prev = beta;
          fs.have_prev = 1;
          for (int j = 0; j < 4; ++j) fs.prev_act[j] = act[j] >= 0 ? act[j] : 0;
          rho = rho_new;
        }
      }
    }
    if (stop && outcome == ORC_BREAKDOWN && mode == ORC_MODE_INFER && o->on_breakdown && !locked) {
      /* READING (extension): restart from the current x (x_k after a curvature breakdown,
       * x_{k+1} after a later one) with r = b - A x, p = M^-1 r, sigma = r^T M^-1 r, every operation
       * in fp64 from here on; iteration k counts as done. */
      double nt = orc_true_residual(n, rp, ci, val, b, x, r);
      sigma = 0.0;
      if (o->precond == 2) orc_ic0_apply(n, rp, ci, icl, r, z);
      for (int i = 0; i < n; ++i) {
        p[i] = o->precond == 2 ? z[i] : o->precond == 1 ? r[i] * dinv[i] : r[i];
        sigma += r[i] * p[i];
      }
      rho = sqrt(nt) / bnorm;
      locked = 1;
      restarts += 1;
      rec.flags |= 16;
      for (int h = 8; h > 0; --h) fs.rho_hist[h] = fs.rho_hist[h - 1];
      fs.rho_hist[0] = rho;
      stop = 0;
      outcome = ORC_MAX_ITER;
      iters = max_iter;
      if (!isfinite(rho)) {
        outcome = ORC_BREAKDOWN;
        iters = k + 1;
        stop = 1;
      } else if (rho < tau && k >= o->min_k) {
        outcome = ORC_CONVERGED;
        iters = k + 1;
        stop = 1;
      }
    }
    rec.reward = t.reward;
    if (learn) learn_step(o, pol, &t, trans, ntrans);
    if (hist) hist[k] = rec;
    nrec = k + 1;
    if (stop) break;
  }
  if (feat_out && outcome != ORC_CONVERGED && outcome != ORC_BREAKDOWN && max_iter > 0) {
    double f[ORC_NFEAT];
    for (int j = 0; j < 5; ++j) f[j] = fstat[j];
    orc_dynamic_features(o, max_iter, &fs, f);
    memcpy(feat_out + (int64_t)max_iter * ORC_NFEAT, f, sizeof(f));
  }
  if (res) {
    res->outcome = outcome;
    res->iters = iters;
    res->nrec = nrec;
    double nt = orc_true_residual(n, rp, ci, val, b, x, rt);
    res->rho_true = bnorm > 0 ? sqrt(nt) / bnorm : 0.0;
    double rr = 0.0;
    for (int i = 0; i < n; ++i) rr += r[i] * r[i];
    res->rho_rec = bnorm > 0 ? sqrt(rr) / bnorm : 0.0;
  }
  free(r); free(p); free(q); free(z); free(rt);
  free(h1); free(h2); free(qout); free(dinv); free(icl);
  return outcome;
}

/* ------------------------------------------------------------------------- */
/* Training.                                                                   */
/* ------------------------------------------------------------------------- */

/* Algorithm 1 on one matrix: episodes e = 1..E with x_0 = 0, online Q updates.
 * ep_base offsets the episode counter of the exploration draws (training on several
 * matrices in sequence continues the count). Returns the number of episodes run. */
int orc_train_sequential(const orc_opts* o, int n, const int32_t* rp, const int32_t* ci,
                         const double* val, const double* b, double tau, int t_max, int E,
                         uint64_t ep_base, double* Q, int32_t* visits, int32_t* iters_out) {
  orc_policy pol;
  memset(&pol, 0, sizeof(pol));
  pol.kind = ORC_POL_QTABLE;
  pol.Q = Q;
  pol.visits = visits;
  double* x = malloc(sizeof(double) * (n > 0 ? n : 1));
  for (int e = 1; e <= E; ++e) {
    for (int i = 0; i < n; ++i) x[i] = 0.0;
    orc_result res;
    orc_run(o, n, rp, ci, val, b, x, tau, t_max, &pol, ORC_MODE_TRAIN, ep_base + (uint64_t)e, 0,
            orc_epsilon(o, e, E), NULL, NULL, NULL, NULL, &res);
    if (iters_out) iters_out[e - 1] = res.iters;
  }
  free(x);
  return E;
}

/* Batched training, one round e (READING, an extension for the batched GPU path):
 * every lane starts from a private copy of the shared tables, runs one episode of
 * Algorithm 1 on its own matrix with online updates to its private copy, and records
 * its transitions. At the end of the round the shared tables are rebuilt by replaying
 * all transitions (lane 0..B-1, then iteration order) with the update rule of
 * Section 4.1 onto the round-start shared tables. With B = 1 this is Algorithm 1. */
int orc_train_round(const orc_opts* o, int B, const int32_t* ns, const int32_t* const* rps,
                    const int32_t* const* cis, const double* const* vals,
                    const double* const* bs, double tau, int t_max, int e, int E, double* Q,
                    int32_t* visits, int32_t* iters_out) {
  int S = o->b_bins * o->r_bins;
  int64_t qsize = o->joint ? (int64_t)S * joint_size(o) : (int64_t)4 * S * o->nprec;
  double* Qp = malloc(sizeof(double) * qsize);
  orc_transition* all = malloc(sizeof(orc_transition) * (size_t)B * (size_t)(t_max > 0 ? t_max : 1));
  int32_t* counts = malloc(sizeof(int32_t) * (size_t)B);
  double eps = orc_epsilon(o, e, E);
  for (int l = 0; l < B; ++l) {
    memcpy(Qp, Q, sizeof(double) * qsize);
    orc_policy pol;
    memset(&pol, 0, sizeof(pol));
    pol.kind = ORC_POL_QTABLE;
    pol.Q = Qp;
    pol.visits = NULL;
    double* x = calloc((size_t)(ns[l] > 0 ? ns[l] : 1), sizeof(double));
    orc_result res;
    orc_run(o, ns[l], rps[l], cis[l], vals[l], bs[l], x, tau, t_max, &pol, ORC_MODE_TRAIN,
            (uint64_t)e, (uint64_t)l, eps, all + (size_t)l * (size_t)t_max, &counts[l], NULL, NULL,
            &res);
    if (iters_out) iters_out[l] = res.iters;
    free(x);
  }
  for (int l = 0; l < B; ++l)
    for (int32_t t = 0; t < counts[l]; ++t) orc_q_update(o, Q, visits, all + (size_t)l * (size_t)t_max + t);
  free(Qp);
  free(all);
  free(counts);
  return 0;
}
