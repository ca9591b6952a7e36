// Host runtime and C ABI of the mixed-precision CG library (see include/mpcg.h).
//
// Owns device memory (matrix copies, policies, launch plans), validates arguments,
// schedules systems onto teams of CTAs and launches the persistent kernel.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <numeric>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "internal.h"

using namespace mpcg;

namespace {

// Device buffer that grows on demand.
struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  cudaError_t ensure(size_t bytes) {
    if (bytes <= cap && p) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e == cudaSuccess) cap = bytes;
    return e;
  }
  template <typename T> T* as() const { return (T*)p; }
};

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

constexpr long long kTimeoutCycles = 4000000000ll;  // about two seconds at 2 GHz per wait
constexpr long long kTuneMinNnz = 4LL << 20;        // smallest matrix the autotuner times

}  // namespace

// ---------------------------------------------------------------------------------------
// Objects
// ---------------------------------------------------------------------------------------

struct Plan {
  int grid = 0, nsys = 0, nteams = 0;
  DevBuf sys, st, res, cta_team, cta_rank, team_size, team_first, team_sys_off, team_sys, bars, partials, err;
  DevBuf work, bstage, xstage, hstage;
  DevBuf qpriv, trans, feats;
  DevBuf lk_w, lk_pref, lk_cfirst, lk_clast, lk_base, lk_done, lk_seg, lk_nseg;
  DevBuf icwork;             // IC(0): every system's substitution words, zeroed per launch
  size_t icwork_bytes = 0;
  bool lockstep = false;
  bool stepped = false;      // one system, one kernel per phase in a while-loop graph
  bool stepped_host = false; // ... the passes launched by the host instead (option stepped = 3)
  unsigned host_passes = 0;  // passes the host launched (stepped_host)
  int sgrid[kPhaseKernels] = {0, 0, 0, 0, 0, 0};
  size_t ssmem = 0;
  cudaGraphExec_t sexec = nullptr;
  ~Plan() {
    if (sexec) cudaGraphExecDestroy(sexec);
  }
  std::vector<DevSys> hsys;
  std::vector<mpcg_result> hres;
  Launch L;
};

struct mpcg_ctx_s {
  int device = 0;
  mpcg_options opt;
  OptView ov;
  int nsm = 0;
  int occ = 0;      // CTAs per SM of the solver kernel without the stream ring
  int occ_s = 0;    // ... with the stream ring (2 * kStageBytes of dynamic shared memory)
  int socc = 0, socc_s = 0;  // same for the standalone product kernel
  int pocc[kPhaseKernels] = {}, pocc_s[kPhaseKernels] = {};  // the stepped solve's phase kernels
  std::string err;
  Plan plan;   // reused by mpcg_solve / mpcg_solve_batched / training
  // the autotuner's results by matrix bucket (mean row length, its spread, longest row, n,
  // column order): schedule and lanes of every format
  std::map<std::tuple<int, int, int, int, int>, std::pair<std::vector<int>, std::vector<int>>> tune_cache;
  DevBuf spmv_x, spmv_q, spmv_y, spmv_err;
};

struct mpcg_matrix_s {
  mpcg_ctx_t ctx = nullptr;
  DevMatrix dm;
  DevBuf rp, ci, v64, v32, vtf, v16, vbf, v16r, vbfr, v8, rexp, dinv;
  bool diag_ok = false;             // every row has a positive diagonal entry (Jacobi defined)
  DevBuf icf, icd;                  // IC(0) factor (fp32, one value per stored entry), diagonal positions
  DevBuf icpf, icpb;                // IC(0): rows in level order of the two substitutions
  DevBuf icof, icob;                // ... the start of each level in them
  int icwf = 0, icwb = 0;           // ... the widest level's row count
  int nlevf = 0, nlevb = 0;         // ... and the number of levels
  unsigned ic_fail = 0;             // 0: not factored or factored fine; else the factorization's error bits
  bool ic_ready = false;
  int device = 0;
  double mean = 0, maxr = 0, cv = 0;
  long long win[4] = {0, 0, 0, 0};  // largest nonzero count of 256, 128, 64, 32 consecutive rows
  bool force_stream_shape = false;  // autotuner: time every candidate in the stream launch shape
  float feat[5] = {0, 0, 0, 0, 0};
  long long bytes = 0;
};

struct mpcg_policy_s {
  mpcg_ctx_t ctx = nullptr;
  int kind = 0;
  int fixed[4] = {4, 4, 4, 4};
  int sched_len = 0;
  DevBuf sched, Q, visits, mlp;
  int S = 0, nprec = 0, H = 0;
  int joint = 0;  // tabular: one table over the joint actions
  int device = 0;
  mpcg_options shape;
};

struct mpcg_graph_s {
  mpcg_ctx_t ctx = nullptr;
  int device = 0;
  std::unique_ptr<Plan> plan;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

mpcg_status fail(mpcg_ctx_t ctx, mpcg_status s, const char* fmt, ...) {
  if (ctx) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    ctx->err = buf;
  }
  return s;
}

#define CK(ctx, call)                                                                                  \
  do {                                                                                                 \
    cudaError_t e_ = (call);                                                                           \
    if (e_ != cudaSuccess) {                                                                           \
      const mpcg_status s_ = (e_ == cudaErrorMemoryAllocation) ? MPCG_ERR_OOM : MPCG_ERR_CUDA;         \
      return fail(ctx, s_, "%s failed: %s", #call, cudaGetErrorString(e_));                           \
    }                                                                                                  \
  } while (0)

bool valid_fmt(int f) { return f >= 0 && f < NFMT; }

int lanes_index(int lanes) { return lanes == 1 ? 0 : lanes == 2 ? 1 : lanes == 4 ? 2 : lanes == 8 ? 3 : -1; }

// Value-region bytes of a stream-schedule stage for (format, lanes), or -1 when a tile of
// kThreads / lanes rows does not fit in one stage.
int stream_vreg(const mpcg_matrix_s* M, int fmt, int lanes) {
  const int li = lanes_index(lanes);
  if (li < 0) return -1;
  // a tile's byte range is rounded out to 16-byte boundaries at both ends (up to 30 extra bytes)
  const long long w = M->win[li];
  const long long vreg = (w * bytes_of(fmt) + 32 + 15) / 16 * 16;
  const long long creg = (w * 4 + 32 + 15) / 16 * 16;
  return vreg + creg <= kStageBytes ? (int)vreg : -1;
}

// The launch carries the shared-memory buffer (two stream stages) when some format's product
// uses it: the stream ring, or the staged x window.
bool uses_stream(const DevMatrix& d) {
  for (int f = 0; f < NFMT; ++f)
    if (d.sched[f] == SCHED_STREAM || d.sched[f] == SCHED_XSTAGE) return true;
  return false;
}

mpcg_status build_optview(mpcg_ctx_t ctx, const mpcg_options& o, OptView& v) {
  if (o.b_bins < 1 || o.b_bins > kMaxBBins) return fail(ctx, MPCG_ERR_INVALID_ARG, "b_bins must be in [1, %d]", kMaxBBins);
  if (o.r_bins < 1 || o.r_bins > kMaxRBins) return fail(ctx, MPCG_ERR_INVALID_ARG, "r_bins must be in [1, %d]", kMaxRBins);
  if (o.t_bin < 1) return fail(ctx, MPCG_ERR_INVALID_ARG, "t_bin must be >= 1");
  if (o.nprec < 1 || o.nprec > MPCG_MAX_PREC) return fail(ctx, MPCG_ERR_INVALID_ARG, "nprec must be in [1, 8]");
  if (!(o.eps_min > 0.0 && o.eps_min < 1.0)) return fail(ctx, MPCG_ERR_INVALID_ARG, "eps_min must be in (0, 1)");
  if (o.mlp_hidden < 1 || o.mlp_hidden > kMaxHidden) return fail(ctx, MPCG_ERR_INVALID_ARG, "mlp_hidden must be in [1, %d]", kMaxHidden);
  if (o.batch_mode < 0 || o.batch_mode > 2) return fail(ctx, MPCG_ERR_INVALID_ARG, "batch_mode must be 0, 1 or 2");
  if (o.precond < 0 || o.precond > 2) return fail(ctx, MPCG_ERR_INVALID_ARG, "precond must be 0, 1 or 2");
  if (!(o.edge_tol >= 0.0 && o.edge_tol < 1.0)) return fail(ctx, MPCG_ERR_INVALID_ARG, "edge_tol must be in [0, 1)");
  if (o.stepped < 0 || o.stepped > 3) return fail(ctx, MPCG_ERR_INVALID_ARG, "stepped must be 0, 1, 2 or 3");
  if (o.variant < 0 || o.variant > 1) return fail(ctx, MPCG_ERR_INVALID_ARG, "variant must be 0 or 1");
  if (o.joint < 0 || o.joint > 1) return fail(ctx, MPCG_ERR_INVALID_ARG, "joint must be 0 or 1");
  if (o.variant == 1 && o.precond == 2)
    return fail(ctx, MPCG_ERR_INVALID_ARG, "the single-reduction iteration runs with precond 0 or 1");
  for (int a = 0; a < o.nprec; ++a)
    if (!valid_fmt(o.precs[a])) return fail(ctx, MPCG_ERR_INVALID_ARG, "precs[%d] = %d is not a format code", a, o.precs[a]);
  if (o.unvisited_fallback != -1 && !valid_fmt(o.unvisited_fallback))
    return fail(ctx, MPCG_ERR_INVALID_ARG, "unvisited_fallback must be -1 or a format code");
  memset(&v, 0, sizeof(v));
  v.b_bins = o.b_bins;
  v.r_bins = o.r_bins;
  v.t_bin = o.t_bin;
  v.t_width = (o.t_bin + o.b_bins - 1) / o.b_bins;
  v.min_k = o.min_k;
  v.nprec = o.nprec;
  for (int a = 0; a < MPCG_MAX_PREC; ++a) {
    v.precs[a] = a < o.nprec ? o.precs[a] : 0;
    v.cost[a] = a < o.nprec ? o.cost[a] : 0.0;
  }
  // Residual bins (Section 4.1): j = min(floor(-log10 max(rho, eps_min) / delta), r - 1) with
  // delta = -log10(eps_min) / r, evaluated as the count of thresholds 10^(-m delta), m = 1..r-1,
  // that rho does not exceed.
  const double delta = -std::log10(o.eps_min) / o.r_bins;
  for (int m = 1; m < o.r_bins; ++m) v.thr[m] = std::pow(10.0, -m * delta);
  v.log_cap = -std::log10(o.eps_min);
  v.eps_min = o.eps_min;
  v.w1 = o.w1;
  v.w2 = o.w2;
  v.w3 = o.w3;
  v.lr = o.lr;
  v.gamma = o.gamma;
  v.seed = o.seed;
  v.fallback_fmt = o.unvisited_fallback;
  v.fallback_idx = -1;
  for (int a = 0; a < o.nprec; ++a)
    if (o.precs[a] == o.unvisited_fallback) { v.fallback_idx = a; break; }
  v.true_every = o.true_res_every;
  v.true_at_conv = o.true_res_at_conv;
  v.warm_start = o.warm_start;
  v.on_breakdown = o.on_breakdown;
  v.precond = o.precond;
  v.edge_tol = o.edge_tol;
  v.variant = o.variant;
  v.joint = o.joint ? 1 : 0;
  for (int j = 0; j < 4; ++j) {
    const unsigned all = (1u << o.nprec) - 1u;
    const unsigned m = o.op_mask[j] ? ((unsigned)o.op_mask[j] & all) : all;
    if (!m) return fail(ctx, MPCG_ERR_INVALID_ARG, "op_mask[%d] allows no entry of precs", j);
    v.op_mask[j] = (int)m;
  }
  return MPCG_OK;
}

// Team size for a system of `work` units (nonzeros plus vector work): about 24k units per
// CTA, at most the whole grid.
int team_size_for(long long work, int grid) {
  long long s = (work + 24575) / 24576;
  if (s < 1) s = 1;
  if (s > grid) s = grid;
  return (int)s;
}

struct SysIn {
  mpcg_matrix_t A;
  const double* b;   // device
  double* x;         // device
  double tol;
  int max_iter;
  mpcg_iter_record* hist;
  int hist_cap;
};

// Longest-processing-time assignment of systems to teams. Systems large enough for
// several CTAs get a team of their own sized by their work; the other CTAs form
// one-CTA teams. Remaining systems go, largest first, to the team whose load per CTA
// grows least.
void schedule(const std::vector<long long>& work, int grid, int force_team, std::vector<int>& team_size,
              std::vector<std::vector<int>>& team_sys) {
  const int nsys = (int)work.size();
  team_size.clear();
  team_sys.clear();
  if (nsys == 0) return;
  std::vector<int> order(nsys);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work[a] > work[b]; });
  if (force_team > 0) {
    // Fixed team size for every system (deterministic layouts for tests).
    const int ts = std::min(force_team, grid);
    const int nt = std::max(1, grid / ts);
    for (int t = 0; t < nt; ++t) {
      team_size.push_back(ts);
      team_sys.emplace_back();
    }
    std::vector<double> load(nt, 0.0);
    for (int i : order) {
      int best = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      team_sys[best].push_back(i);
      load[best] += (double)work[i];
    }
    return;
  }
  if (nsys == 1) {
    team_size.push_back(team_size_for(work[0], grid));
    team_sys.push_back({0});
    return;
  }
  const double total = (double)std::accumulate(work.begin(), work.end(), 0LL);
  const double per_cta = total / grid;
  int used = 0;
  std::vector<double> load;
  std::vector<char> placed(nsys, 0);
  for (int i : order) {
    int s = (int)std::floor((double)work[i] / per_cta);
    s = std::min(s, team_size_for(work[i], grid));
    if (s < 2) break;
    if (used + s > grid - 1) s = grid - 1 - used;
    if (s < 2) break;
    team_size.push_back(s);
    team_sys.push_back({i});
    load.push_back((double)work[i] / s);
    placed[i] = 1;
    used += s;
  }
  while (used < grid) {
    team_size.push_back(1);
    team_sys.emplace_back();
    load.push_back(0.0);
    ++used;
  }
  for (int i : order) {
    if (placed[i]) continue;
    int best = 0;
    double bestv = 1e300;
    for (size_t t = 0; t < team_size.size(); ++t) {
      const double v = load[t] + (double)work[i] / team_size[t];
      if (v < bestv) { bestv = v; best = (int)t; }
    }
    team_sys[best].push_back(i);
    load[best] = bestv;
  }
}

mpcg_status fill_policy(mpcg_ctx_t ctx, mpcg_policy_t P, PolicyView& pv) {
  memset(&pv, 0, sizeof(pv));
  if (!P) return fail(ctx, MPCG_ERR_INVALID_ARG, "policy is NULL");
  pv.kind = P->kind;
  for (int j = 0; j < 4; ++j) pv.fixed[j] = P->fixed[j];
  pv.sched = P->sched.as<int>();
  pv.sched_len = P->sched_len;
  pv.Q = P->Q.as<double>();
  pv.visits = P->visits.as<int>();
  pv.mlp = P->mlp.as<float>();
  pv.H = P->H;
  if (P->kind == 2 || P->kind == 3) {
    const mpcg_options& o = ctx->opt;
    if (P->nprec != o.nprec || (P->kind == 2 && (P->S != o.b_bins * o.r_bins || P->joint != (o.joint ? 1 : 0))) ||
        (P->kind == 3 && P->H != o.mlp_hidden))
      return fail(ctx, MPCG_ERR_BAD_POLICY, "policy shape (S=%d, nprec=%d, H=%d) differs from the context's options",
                  P->S, P->nprec, P->H);
  }
  return MPCG_OK;
}

mpcg_status ic0_error(mpcg_ctx_t ctx, unsigned bits) {
  if (bits & 4u) return fail(ctx, MPCG_ERR_TIMEOUT, "the incomplete Cholesky factorization exceeded its wait limit");
  if (bits & 2u)
    return fail(ctx, MPCG_ERR_INVALID_ARG,
                "incomplete Cholesky needs strictly increasing column indices, a diagonal entry in every row "
                "and a symmetric pattern");
  return fail(ctx, MPCG_ERR_INVALID_ARG, "incomplete Cholesky breaks down (a non-positive pivot)");
}

// IC(0) factor of A in fp32, computed once per matrix on the device (the factorization kernel
// and the transposed copy for the backward substitution); a failed factorization is
// remembered and reported again.
mpcg_status ensure_ic0(mpcg_ctx_t ctx, mpcg_matrix_s* M, cudaStream_t s) {
  if (M->ic_ready) return MPCG_OK;
  if (M->ic_fail) return ic0_error(ctx, M->ic_fail);
  const int n = M->dm.n;
  const long long nnz = M->dm.nnz;
  CK(ctx, M->icf.ensure(4 * (size_t)std::max(nnz, 1LL)));
  CK(ctx, M->icd.ensure(4 * (size_t)std::max(n, 1)));
  DevBuf done, err;
  CK(ctx, done.ensure(4 * (size_t)std::max(n, 1)));
  CK(ctx, err.ensure(sizeof(unsigned)));
  CK(ctx, cudaMemsetAsync(done.p, 0, 4 * (size_t)std::max(n, 1), s));
  CK(ctx, cudaMemsetAsync(err.p, 0, sizeof(unsigned), s));
  CK(ctx, launch_ic0_factor(n, M->dm.rp, M->dm.ci, M->dm.v64, M->icf.as<float>(), M->icd.as<int>(),
                            done.as<unsigned>(), err.as<unsigned>(), kTimeoutCycles, ctx->nsm, s));
  unsigned bits = 0;
  CK(ctx, cudaMemcpyAsync(&bits, err.p, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  CK(ctx, cudaStreamSynchronize(s));
  if (bits) {
    M->ic_fail = bits;
    return ic0_error(ctx, bits);
  }
  // level schedule of the substitutions (host pass over the pattern): rows sorted by level,
  // stable in the row index
  std::vector<int> hrp(n + 1), hci((size_t)std::max(nnz, 1LL)), hdp(std::max(n, 1));
  CK(ctx, cudaMemcpy(hrp.data(), M->dm.rp, 4 * (size_t)(n + 1), cudaMemcpyDeviceToHost));
  if (nnz) CK(ctx, cudaMemcpy(hci.data(), M->dm.ci, 4 * (size_t)nnz, cudaMemcpyDeviceToHost));
  if (n) CK(ctx, cudaMemcpy(hdp.data(), M->icd.p, 4 * (size_t)n, cudaMemcpyDeviceToHost));
  std::vector<int> lev(std::max(n, 1)), perm(std::max(n, 1));
  auto sort_by_level = [&](int depth, DevBuf& out, DevBuf& starts, int& width, int& nlev) -> mpcg_status {
    std::vector<int> cnt(depth + 1, 0);
    for (int i = 0; i < n; ++i) ++cnt[lev[i] + 1];
    width = 0;
    for (int l = 0; l < depth; ++l) width = std::max(width, cnt[l + 1]);
    for (int l = 0; l < depth; ++l) cnt[l + 1] += cnt[l];
    CK(ctx, starts.ensure(4 * (size_t)(depth + 1)));
    CK(ctx, cudaMemcpy(starts.p, cnt.data(), 4 * (size_t)(depth + 1), cudaMemcpyHostToDevice));
    nlev = depth;
    for (int i = 0; i < n; ++i) perm[cnt[lev[i]]++] = i;
    CK(ctx, out.ensure(4 * (size_t)std::max(n, 1)));
    if (n) CK(ctx, cudaMemcpy(out.p, perm.data(), 4 * (size_t)n, cudaMemcpyHostToDevice));
    return MPCG_OK;
  };
  int depth = 0;
  for (int i = 0; i < n; ++i) {  // L y = r: row i reads y_j, j < i, over its lower entries
    int l = 0;
    for (int e = hrp[i]; e < hdp[i]; ++e) l = std::max(l, lev[hci[e]] + 1);
    lev[i] = l;
    depth = std::max(depth, l + 1);
  }
  mpcg_status ls = sort_by_level(depth, M->icpf, M->icof, M->icwf, M->nlevf);
  if (ls != MPCG_OK) return ls;
  depth = 0;
  for (int i = n - 1; i >= 0; --i) {  // L^T w = y: row i reads w_j, j > i, over its upper entries
    int l = 0;
    for (int e = hdp[i] + 1; e < hrp[i + 1]; ++e) l = std::max(l, lev[hci[e]] + 1);
    lev[i] = l;
    depth = std::max(depth, l + 1);
  }
  ls = sort_by_level(depth, M->icpb, M->icob, M->icwb, M->nlevb);
  if (ls != MPCG_OK) return ls;
  M->ic_ready = true;
  M->bytes += 4 * nnz + 12LL * n;
  return MPCG_OK;
}

// Builds the device tables of a launch for `in` systems into `pl` and fills pl.L.
mpcg_status build_plan(mpcg_ctx_t ctx, Plan& pl, const std::vector<SysIn>& in, mpcg_policy_t policy, int train,
                       int trans_cap, int force_team, cudaStream_t s, int feat_cap = 0, bool stepped = false) {
  const int nsys = (int)in.size();
  if (stepped && (nsys != 1 || train || ctx->opt.precond == 2))
    return fail(ctx, MPCG_ERR_INTERNAL, "the stepped solve takes one inference system without IC(0)");
  if (ctx->opt.precond == 1)
    for (int i = 0; i < nsys; ++i)
      if (!in[i].A->diag_ok)
        return fail(ctx, MPCG_ERR_INVALID_ARG,
                    "system %d: Jacobi preconditioning needs a positive diagonal entry in every row", i);
  const bool ic = ctx->opt.precond == 2;
  if (ic)
    for (int i = 0; i < nsys; ++i) {
      mpcg_status st = ensure_ic0(ctx, in[i].A, s);
      if (st != MPCG_OK) return st;
    }
  bool stream_shape = false;
  for (int i = 0; i < nsys; ++i) stream_shape = stream_shape || uses_stream(in[i].A->dm);
  const int grid = ctx->nsm * (stream_shape ? ctx->occ_s : ctx->occ);
  std::vector<long long> work(nsys);
  for (int i = 0; i < nsys; ++i) work[i] = in[i].A->dm.nnz + 4LL * in[i].A->dm.n;
  std::vector<int> tsize;
  std::vector<std::vector<int>> tsys;
  schedule(work, grid, force_team, tsize, tsys);
  const int nteams = (int)tsize.size();
  std::vector<int> cta_team(grid, nteams), cta_rank(grid, 0), team_first(nteams + 1, 0), team_sys_off(nteams + 2, 0), team_sys_flat;
  int c = 0;
  for (int t = 0; t < nteams; ++t) {
    team_first[t] = c;
    for (int r = 0; r < tsize[t]; ++r, ++c) {
      cta_team[c] = t;
      cta_rank[c] = r;
    }
    team_sys_off[t] = (int)team_sys_flat.size();
    for (int i : tsys[t]) team_sys_flat.push_back(i);
  }
  team_sys_off[nteams] = (int)team_sys_flat.size();
  // CTAs beyond the scheduled teams form one extra empty team.
  std::vector<int> tsize_all(tsize);
  tsize_all.push_back(std::max(1, grid - c));
  team_first[nteams] = c;
  team_sys_off[nteams + 1] = team_sys_off[nteams];
  for (int cc = c; cc < grid; ++cc) {
    cta_team[cc] = nteams;
    cta_rank[cc] = cc - c;
  }
  const int nteams_all = nteams + 1;

  // Work vectors: r, p, q (8 bytes per row each) and p's low-precision copy (4 bytes).
  // IC(0) adds one 64-bit word per row (value and mark of the substitutions).
  size_t wbytes = 0, mbytes = 0;
  const bool sr = ctx->opt.variant == 1;  // single-reduction iteration: u in fp64 possible, and s
  for (int i = 0; i < nsys; ++i) wbytes += (sr ? 40 : 28) * (size_t)in[i].A->dm.n + 5 * 256;
  for (int i = 0; i < nsys; ++i) mbytes += ic ? 8 * (size_t)in[i].A->dm.n : 0;
  CK(ctx, pl.work.ensure(wbytes));
  pl.icwork_bytes = mbytes;
  if (mbytes) CK(ctx, pl.icwork.ensure(mbytes));
  unsigned long long* icw_next = pl.icwork.as<unsigned long long>();
  const int S = ctx->opt.b_bins * ctx->opt.r_bins;
  const long long qsize = qtable_size(S, ctx->opt.nprec, ctx->opt.joint ? 1 : 0);
  if (train) {
    CK(ctx, pl.qpriv.ensure(sizeof(double) * qsize * nsys));
    CK(ctx, pl.trans.ensure(sizeof(Transition) * (size_t)trans_cap * nsys));
  }
  if (feat_cap > 0) CK(ctx, pl.feats.ensure(sizeof(float) * kNFeat * (size_t)feat_cap * nsys));
  pl.hsys.resize(nsys);
  char* wp = pl.work.as<char>();
  auto take = [&](size_t bytes) {
    char* r = wp;
    wp += (bytes + 255) / 256 * 256;
    return (void*)r;
  };
  for (int i = 0; i < nsys; ++i) {
    DevSys& d = pl.hsys[i];
    memset(&d, 0, sizeof(d));
    d.A = in[i].A->dm;
    d.A.dinv = ctx->opt.precond == 1 ? in[i].A->dinv.as<double>() : nullptr;
    d.A.icf = ic ? in[i].A->icf.as<float>() : nullptr;
    d.A.icd = ic ? in[i].A->icd.as<int>() : nullptr;
    d.A.icpf = ic ? in[i].A->icpf.as<int>() : nullptr;
    d.A.icpb = ic ? in[i].A->icpb.as<int>() : nullptr;
    d.A.icwf = ic ? in[i].A->icwf : 0;
    d.A.icwb = ic ? in[i].A->icwb : 0;
    d.A.icof = ic ? in[i].A->icof.as<int>() : nullptr;
    d.A.icob = ic ? in[i].A->icob.as<int>() : nullptr;
    d.A.nlevf = ic ? in[i].A->nlevf : 0;
    d.A.nlevb = ic ? in[i].A->nlevb : 0;
    const int n = d.A.n;
    d.b = in[i].b;
    d.x = in[i].x;
    d.r = (double*)take(8 * (size_t)n);
    d.p = (double*)take(8 * (size_t)n);
    d.q = take(8 * (size_t)n);
    d.plow = take((sr ? 8 : 4) * (size_t)n);
    d.sv = sr ? (double*)take(8 * (size_t)n) : nullptr;
    if (ic) {
      d.icw = icw_next;
      icw_next += n;
    }
    d.tol = in[i].tol;
    d.max_iter = in[i].max_iter;
    d.lane = i;
    d.hist = in[i].hist;
    d.hist_cap = in[i].hist_cap;
    if (train) {
      d.Qpriv = pl.qpriv.as<double>() + qsize * i;
      d.trans = pl.trans.as<Transition>() + (size_t)trans_cap * i;
      d.trans_cap = trans_cap;
    }
    for (int j = 0; j < 5; ++j) d.feat_static[j] = in[i].A->feat[j];
    if (feat_cap > 0) {
      d.feat_log = pl.feats.as<float>() + (size_t)kNFeat * feat_cap * i;
      d.feat_cap = feat_cap;
    }
  }
  CK(ctx, pl.sys.ensure(sizeof(DevSys) * std::max(nsys, 1)));
  CK(ctx, pl.st.ensure(sizeof(SysState) * std::max(nsys, 1)));
  CK(ctx, pl.res.ensure(sizeof(mpcg_result) * std::max(nsys, 1)));
  CK(ctx, pl.cta_team.ensure(sizeof(int) * grid));
  CK(ctx, pl.cta_rank.ensure(sizeof(int) * grid));
  CK(ctx, pl.team_size.ensure(sizeof(int) * nteams_all));
  CK(ctx, pl.team_first.ensure(sizeof(int) * (nteams_all + 1)));
  CK(ctx, pl.team_sys_off.ensure(sizeof(int) * (nteams_all + 1)));
  CK(ctx, pl.team_sys.ensure(sizeof(int) * std::max<size_t>(1, team_sys_flat.size())));
  CK(ctx, pl.bars.ensure(sizeof(unsigned) * kBarStride * nteams_all));
  // Lockstep batches: every CTA works on a slice of every unfinished system.
  const int bm = ctx->opt.batch_mode;
  // the single-reduction iteration runs in the lockstep (or stepped) kernels only
  if (sr && force_team > 0) return fail(ctx, MPCG_ERR_INVALID_ARG, "the single-reduction iteration runs without teams");
  pl.lockstep = !stepped && force_team == 0 && ((bm == 0 && nsys >= 2) || bm == 2 || sr) && nsys >= 1;
  pl.stepped = stepped;
  pl.stepped_host = false;
  int pgrid = 0;
  if (stepped) {
    for (int w = 0; w < kPhaseKernels; ++w) {
      pl.sgrid[w] = ctx->nsm * (stream_shape ? ctx->pocc_s[w] : ctx->pocc[w]);
      pgrid = std::max(pgrid, pl.sgrid[w]);
    }
    pl.ssmem = stream_shape ? 2 * (size_t)kStageBytes : 0;
    CK(ctx, pl.lk_done.ensure(sizeof(int)));
  }
  CK(ctx, pl.partials.ensure(sizeof(double) * kNSlot * (size_t)(std::max(grid, pgrid) + (pl.lockstep ? nsys : 0))));
  if (pl.lockstep) {
    std::vector<long long> w(nsys);
    for (int i = 0; i < nsys; ++i) w[i] = std::max(1LL, in[i].A->dm.nnz + 3LL * in[i].A->dm.n);
    CK(ctx, pl.lk_w.ensure(sizeof(long long) * nsys));
    CK(ctx, pl.lk_pref.ensure(sizeof(long long) * (nsys + 1)));
    CK(ctx, pl.lk_cfirst.ensure(sizeof(int) * nsys));
    CK(ctx, pl.lk_clast.ensure(sizeof(int) * nsys));
    CK(ctx, pl.lk_base.ensure(sizeof(int) * nsys));
    CK(ctx, pl.lk_done.ensure(sizeof(int)));
    CK(ctx, pl.lk_seg.ensure(sizeof(int4) * (size_t)grid * (nsys + 1)));
    CK(ctx, pl.lk_nseg.ensure(sizeof(int) * grid));
    CK(ctx, cudaMemcpyAsync(pl.lk_w.p, w.data(), sizeof(long long) * nsys, cudaMemcpyHostToDevice, s));
    CK(ctx, cudaStreamSynchronize(s));
  }
  CK(ctx, pl.err.ensure(sizeof(unsigned)));
  if (nsys) CK(ctx, cudaMemcpyAsync(pl.sys.p, pl.hsys.data(), sizeof(DevSys) * nsys, cudaMemcpyHostToDevice, s));
  CK(ctx, cudaMemcpyAsync(pl.cta_team.p, cta_team.data(), sizeof(int) * grid, cudaMemcpyHostToDevice, s));
  CK(ctx, cudaMemcpyAsync(pl.cta_rank.p, cta_rank.data(), sizeof(int) * grid, cudaMemcpyHostToDevice, s));
  CK(ctx, cudaMemcpyAsync(pl.team_size.p, tsize_all.data(), sizeof(int) * nteams_all, cudaMemcpyHostToDevice, s));
  CK(ctx, cudaMemcpyAsync(pl.team_first.p, team_first.data(), sizeof(int) * (nteams_all + 1), cudaMemcpyHostToDevice, s));
  CK(ctx, cudaMemcpyAsync(pl.team_sys_off.p, team_sys_off.data(), sizeof(int) * (nteams_all + 1), cudaMemcpyHostToDevice, s));
  if (!team_sys_flat.empty())
    CK(ctx, cudaMemcpyAsync(pl.team_sys.p, team_sys_flat.data(), sizeof(int) * team_sys_flat.size(), cudaMemcpyHostToDevice, s));
  // The host vectors above are pageable; wait for the copies before they go out of scope.
  CK(ctx, cudaStreamSynchronize(s));
  pl.grid = grid;
  pl.nsys = nsys;
  pl.nteams = nteams_all;
  Launch& L = pl.L;
  memset(&L, 0, sizeof(L));
  L.sys = pl.sys.as<DevSys>();
  L.st = pl.st.as<SysState>();
  L.nsys = nsys;
  L.nteams = nteams_all;
  L.cta_team = pl.cta_team.as<int>();
  L.cta_rank = pl.cta_rank.as<int>();
  L.team_size = pl.team_size.as<int>();
  L.team_first = pl.team_first.as<int>();
  L.team_sys_off = pl.team_sys_off.as<int>();
  L.team_sys = pl.team_sys.as<int>();
  L.bars = pl.bars.as<unsigned>();
  L.partials = pl.partials.as<double>();
  L.res = pl.res.as<mpcg_result>();
  L.err = pl.err.as<unsigned>();
  mpcg_status st = fill_policy(ctx, policy, L.pol);
  if (st != MPCG_OK) return st;
  L.opt = ctx->ov;
  L.train = train;
  L.stream_stage = stream_shape ? kStageBytes : 0;
  L.timeout_cycles = kTimeoutCycles;
  if (const char* t = getenv("MPCG_TIMEOUT_CYCLES")) L.timeout_cycles = atoll(t);
  L.lockstep = pl.lockstep ? 1 : 0;
  L.ic = ctx->opt.precond == 2 ? 1 : 0;
  if (pl.stepped) L.lk_done = pl.lk_done.as<int>();
  if (pl.lockstep) {
    L.lk_w = pl.lk_w.as<long long>();
    L.lk_pref = pl.lk_pref.as<long long>();
    L.lk_cfirst = pl.lk_cfirst.as<int>();
    L.lk_clast = pl.lk_clast.as<int>();
    L.lk_base = pl.lk_base.as<int>();
    L.lk_done = pl.lk_done.as<int>();
    L.lk_seg = pl.lk_seg.as<int4>();
    L.lk_nseg = pl.lk_nseg.as<int>();
  }
  return MPCG_OK;
}

// Enqueues one launch of a built plan (barrier counters and status word cleared first).
mpcg_status enqueue_plan(mpcg_ctx_t ctx, Plan& pl, cudaStream_t s) {
  CK(ctx, cudaMemsetAsync(pl.bars.p, 0, sizeof(unsigned) * kBarStride * pl.nteams, s));
  CK(ctx, cudaMemsetAsync(pl.err.p, 0, sizeof(unsigned), s));
  if (pl.icwork_bytes) CK(ctx, cudaMemsetAsync(pl.icwork.p, 0, pl.icwork_bytes, s));
  const size_t smem = pl.L.stream_stage > 0 ? 2 * (size_t)pl.L.stream_stage : 0;
  if (pl.stepped) {
    // the phase machine starts in its initialisation phase; the while-loop graph of this
    // launch is built and instantiated here (a graph with a conditional node has at most one
    // instantiation at a time, so the previous one is destroyed first)
    CK(ctx, cudaMemsetAsync(pl.st.p, 0, sizeof(SysState), s));
    CK(ctx, cudaMemsetAsync(pl.lk_done.p, 0, sizeof(int), s));
    if (pl.sexec) {
      CK(ctx, cudaStreamSynchronize(s));
      cudaGraphExecDestroy(pl.sexec);
      pl.sexec = nullptr;
    }
    const unsigned limit = 8u * (unsigned)std::min(pl.hsys[0].max_iter + 4, 1 << 26) + 64u;
    if (pl.stepped_host) {
      // the same passes launched from the host, the phase read back after each pass (for tools
      // that do not follow kernels inside graphs with conditional nodes); bounded like the graph
      int phase = 0;
      unsigned herr = 0;
      pl.host_passes = 0;
      for (unsigned pass = 0; pass < limit; ++pass) {
        CK(ctx, stepped_pass(pl.L, pl.sgrid, pl.ssmem, s));
        pl.host_passes = pass + 1;
        CK(ctx, cudaMemcpyAsync(&phase, &pl.L.st->phase, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(ctx, cudaMemcpyAsync(&herr, pl.L.err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        CK(ctx, cudaStreamSynchronize(s));
        if (phase == kPhaseDone || herr) return MPCG_OK;
      }
      return fail(ctx, MPCG_ERR_INTERNAL, "the stepped solve did not finish within its pass limit");
    }
    cudaGraph_t g = nullptr;
    CK(ctx, stepped_graph(pl.L, pl.sgrid, pl.ssmem, limit, &g));
    const cudaError_t e = cudaGraphInstantiate(&pl.sexec, g, 0);
    cudaGraphDestroy(g);
    CK(ctx, e);
    CK(ctx, cudaGraphLaunch(pl.sexec, s));
    return MPCG_OK;
  }
  if (pl.lockstep) {
    // every system starts in its initialisation phase; no system has finished
    CK(ctx, cudaMemsetAsync(pl.st.p, 0, sizeof(SysState) * pl.nsys, s));
    CK(ctx, cudaMemsetAsync(pl.lk_done.p, 0, sizeof(int), s));
    cudaGetLastError();
    CK(ctx, launch_cg_lockstep(pl.L, pl.grid, smem, s));
    return MPCG_OK;
  }
  cudaGetLastError();
  CK(ctx, launch_cg(pl.L, pl.grid, smem, s));
  return MPCG_OK;
}

mpcg_status finish_plan(mpcg_ctx_t ctx, Plan& pl, mpcg_result* res, cudaStream_t s) {
  unsigned herr = 0;
  pl.hres.resize(std::max(pl.nsys, 1));
  if (pl.nsys) CK(ctx, cudaMemcpyAsync(pl.hres.data(), pl.res.p, sizeof(mpcg_result) * pl.nsys, cudaMemcpyDeviceToHost, s));
  CK(ctx, cudaMemcpyAsync(&herr, pl.err.p, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  unsigned passes = 0;  // the stepped graph's pass counter (bars[16], kept by its control kernel)
  if (pl.stepped && !pl.stepped_host)
    CK(ctx, cudaMemcpyAsync(&passes, pl.bars.as<unsigned>() + 16, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  CK(ctx, cudaStreamSynchronize(s));
  if (herr == DERR_TIMEOUT) return fail(ctx, MPCG_ERR_TIMEOUT, "a device-side barrier wait exceeded its limit");
  if (herr) return fail(ctx, MPCG_ERR_INTERNAL, "device status word %u", herr);
  int launches = 1;
  if (pl.stepped) {
    const int nbody = pl.L.opt.variant ? 3 : 4;  // phase kernels per pass (stepped.cu)
    launches = pl.stepped_host ? (int)pl.host_passes * nbody : (int)passes * (nbody + 1);
  }
  for (int i = 0; i < pl.nsys; ++i) pl.hres[i].kernel_launches = launches;
  if (res && pl.nsys) memcpy(res, pl.hres.data(), sizeof(mpcg_result) * pl.nsys);
  return MPCG_OK;
}

// Row-length rule for the product schedule (from timings on GB300 across the workloads'
// row lengths): one thread per row with 16-byte loads for a mean row length of up to about
// 32 nonzeros; longer rows get K lanes, K the power of two near mean / 24 (banded rows of 65
// nonzeros: 4 lanes, of 129: 8). Rows over 1024 nonzeros (power-law hubs) are summed by the
// whole CTA in both schedules.
void default_schedule(mpcg_matrix_s* M) {
  int sched = SCHED_VECTOR, lanes = 1;
  if (M->mean <= 32.0) {
    sched = SCHED_VLOAD;
  } else {
    while (lanes < 32 && lanes * 24 < M->mean) lanes *= 2;
  }
  for (int f = 0; f < 8; ++f) {
    M->dm.sched[f] = sched;
    M->dm.lanes[f] = lanes;
  }
}

}  // namespace

// ---------------------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------------------

extern "C" {

void mpcg_options_default(mpcg_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->b_bins = 10;
  o->r_bins = 10;
  o->t_bin = 1000;
  o->min_k = 10;
  o->eps_min = 1e-16;
  o->nprec = 5;
  const int precs[5] = {MPCG_FP16, MPCG_BF16, MPCG_TF32, MPCG_FP32, MPCG_FP64};
  const double cost[5] = {0.8, 0.6, 0.8, 1.0, 2.0};  // cost setting C1 (Section 5)
  for (int a = 0; a < 5; ++a) {
    o->precs[a] = precs[a];
    o->cost[a] = cost[a];
  }
  o->w1 = 1.0;
  o->w2 = 0.1;
  o->w3 = 10.0;
  o->lr = 0.1;
  o->gamma = 0.9;
  o->eps0 = 1.0;
  o->eps_floor = 0.1;
  o->seed = 0;
  o->unvisited_fallback = MPCG_FP64;
  o->true_res_every = 0;
  o->true_res_at_conv = 0;
  o->warm_start = 0;
  o->on_breakdown = 0;
  o->mlp_hidden = 64;
  o->batch_mode = 0;
  o->precond = 0;
  o->edge_tol = 5e-3;
  o->stepped = 0;
  o->variant = 0;
  o->joint = 0;
  o->reserved_joint = 0;
}

mpcg_status mpcg_create(mpcg_ctx_t* out, int device, const mpcg_options* opt) {
  if (!out) return MPCG_ERR_INVALID_ARG;
  *out = nullptr;
  std::unique_ptr<mpcg_ctx_s> c(new mpcg_ctx_s());
  if (opt) c->opt = *opt;
  else mpcg_options_default(&c->opt);
  mpcg_status s = build_optview(c.get(), c->opt, c->ov);
  if (s != MPCG_OK) return s;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return MPCG_ERR_INVALID_ARG;
  }
  c->device = device;
  if (cudaSetDevice(device) != cudaSuccess) return MPCG_ERR_CUDA;
  int coop = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device);
  cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, device);
  if (!coop) return MPCG_ERR_CUDA;
  if (set_smem_limits(2 * (size_t)kStageBytes) != cudaSuccess) return MPCG_ERR_CUDA;
  if (cg_occupancy(&c->occ, 0) != cudaSuccess || c->occ < 1) return MPCG_ERR_CUDA;
  if (cg_occupancy(&c->occ_s, 2 * (size_t)kStageBytes) != cudaSuccess || c->occ_s < 1) return MPCG_ERR_CUDA;
  if (spmv_occupancy(&c->socc, 0) != cudaSuccess || spmv_occupancy(&c->socc_s, 2 * (size_t)kStageBytes) != cudaSuccess)
    return MPCG_ERR_CUDA;
  if (mlp_set_smem_limit(mlp_grad_smem(kMaxHidden, MPCG_MAX_PREC)) != cudaSuccess) return MPCG_ERR_CUDA;
  if (stepped_set_smem_limit(2 * (size_t)kStageBytes) != cudaSuccess) return MPCG_ERR_CUDA;
  for (int w = 0; w < kPhaseKernels; ++w) {
    if (stepped_occupancy(w, &c->pocc[w], 0) != cudaSuccess || c->pocc[w] < 1) return MPCG_ERR_CUDA;
    if (stepped_occupancy(w, &c->pocc_s[w], 2 * (size_t)kStageBytes) != cudaSuccess || c->pocc_s[w] < 1)
      return MPCG_ERR_CUDA;
  }
  c->socc = std::min(c->socc, c->occ);
  c->socc_s = std::min(c->socc_s, c->occ_s);
  *out = c.release();
  return MPCG_OK;
}

mpcg_status mpcg_destroy(mpcg_ctx_t ctx) {
  if (!ctx) return MPCG_ERR_INVALID_ARG;
  cudaSetDevice(ctx->device);
  delete ctx;
  return MPCG_OK;
}

const char* mpcg_last_error(mpcg_ctx_t ctx) { return ctx ? ctx->err.c_str() : "no context"; }

mpcg_status mpcg_device_info(mpcg_ctx_t ctx, int32_t* num_sms, int32_t* ctas_per_sm) {
  if (!ctx) return MPCG_ERR_INVALID_ARG;
  if (num_sms) *num_sms = ctx->nsm;
  if (ctas_per_sm) *ctas_per_sm = ctx->occ;
  return MPCG_OK;
}

// ---- matrices ---------------------------------------------------------------------------

mpcg_status mpcg_matrix_create(mpcg_ctx_t ctx, const mpcg_csr* A, mpcg_matrix_t* out, void* stream) {
  if (!ctx || !A || !out) return fail(ctx, MPCG_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  ctx->err.clear();
  const int n = A->n;
  const long long nnz = A->nnz;
  if (n < 0 || nnz < 0 || nnz >= (1LL << 31)) return fail(ctx, MPCG_ERR_INVALID_ARG, "n = %d, nnz = %lld out of range", n, nnz);
  if (!A->row_ptr || (nnz > 0 && (!A->col || !A->val)))
    return fail(ctx, MPCG_ERR_INVALID_ARG, "CSR array pointer is NULL");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  std::unique_ptr<mpcg_matrix_s> M(new mpcg_matrix_s());
  M->ctx = ctx;
  M->device = ctx->device;
  const bool dev = is_device_ptr(A->row_ptr);
  const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const size_t pn = (size_t)nnz + 16;  // padding so that 16-byte rounded ranges stay in bounds
  CK(ctx, M->rp.ensure(sizeof(int) * ((size_t)n + 1)));
  CK(ctx, M->ci.ensure(sizeof(int) * pn));
  CK(ctx, M->v64.ensure(sizeof(double) * pn));
  CK(ctx, M->v32.ensure(sizeof(float) * pn));
  CK(ctx, M->vtf.ensure(sizeof(float) * pn));
  CK(ctx, M->v16.ensure(sizeof(__half) * pn));
  CK(ctx, M->vbf.ensure(sizeof(__nv_bfloat16) * pn));
  CK(ctx, M->v16r.ensure(sizeof(__half) * pn));
  CK(ctx, M->vbfr.ensure(sizeof(__nv_bfloat16) * pn));
  CK(ctx, M->v8.ensure(sizeof(q52_t) * pn));
  CK(ctx, M->rexp.ensure(sizeof(short) * ((size_t)n + 8)));
  M->bytes = (long long)(M->rp.cap + M->ci.cap + M->v64.cap + M->v32.cap + M->vtf.cap + M->v16.cap + M->vbf.cap +
                         M->v16r.cap + M->vbfr.cap + M->v8.cap + M->rexp.cap);
  CK(ctx, cudaMemcpyAsync(M->rp.p, A->row_ptr, sizeof(int) * ((size_t)n + 1), kind, s));
  CK(ctx, cudaMemsetAsync(M->ci.p, 0, sizeof(int) * pn, s));
  CK(ctx, cudaMemsetAsync(M->v64.p, 0, sizeof(double) * pn, s));
  if (nnz > 0) {
    CK(ctx, cudaMemcpyAsync(M->ci.p, A->col, sizeof(int) * (size_t)nnz, kind, s));
    CK(ctx, cudaMemcpyAsync(M->v64.p, A->val, sizeof(double) * (size_t)nnz, kind, s));
  }
  // Validation on the device.
  DevBuf flags;
  CK(ctx, flags.ensure(2 * sizeof(int)));
  const int init[2] = {0, 0x7fffffff};
  CK(ctx, cudaMemcpyAsync(flags.p, init, sizeof(init), cudaMemcpyHostToDevice, s));
  CK(ctx, launch_validate(n, nnz, M->rp.as<int>(), M->ci.as<int>(), M->v64.as<double>(), flags.as<unsigned>(),
                          flags.as<int>() + 1, s));
  int hf[2] = {0, 0};
  CK(ctx, cudaMemcpyAsync(hf, flags.p, sizeof(hf), cudaMemcpyDeviceToHost, s));
  CK(ctx, cudaStreamSynchronize(s));
  if (hf[0] & 31) {
    const unsigned f = (unsigned)hf[0];
    return fail(ctx, MPCG_ERR_INVALID_ARG, "invalid CSR at row %d:%s%s%s%s%s", hf[1], (f & 1) ? " row_ptr bounds" : "",
                (f & 2) ? " row_ptr decreasing" : "", (f & 4) ? " column out of range" : "",
                (f & 8) ? " non-finite value" : "", (f & 16) ? " missing or non-positive diagonal" : "");
  }
  DevMatrix& d = M->dm;
  memset(&d, 0, sizeof(d));
  d.n = n;
  d.nnz = nnz;
  d.rp = M->rp.as<int>();
  d.ci = M->ci.as<int>();
  d.v64 = M->v64.as<double>();
  d.v32 = M->v32.as<float>();
  d.vtf = M->vtf.as<float>();
  d.v16 = M->v16.as<__half>();
  d.vbf = M->vbf.as<__nv_bfloat16>();
  d.v16r = M->v16r.as<__half>();
  d.vbfr = M->vbfr.as<__nv_bfloat16>();
  d.v8 = M->v8.as<q52_t>();
  d.rexp = M->rexp.as<short>();
  d.cols_sorted = (hf[0] & 32) ? 0 : 1;
  CK(ctx, launch_convert(d, M->v32.as<float>(), M->vtf.as<float>(), M->v16.as<__half>(), M->vbf.as<__nv_bfloat16>(),
                         M->v16r.as<__half>(), M->vbfr.as<__nv_bfloat16>(), M->v8.as<q52_t>(), M->rexp.as<short>(), s));
  // Jacobi: fp64 reciprocals of the diagonal, and whether every row has a positive one.
  {
    DevBuf bad;
    CK(ctx, M->dinv.ensure(8 * (size_t)std::max(n, 1)));
    CK(ctx, bad.ensure(sizeof(unsigned)));
    CK(ctx, cudaMemsetAsync(bad.p, 0, sizeof(unsigned), s));
    CK(ctx, launch_jacobi_diag(n, d.rp, d.ci, d.v64, M->dinv.as<double>(), bad.as<unsigned>(), s));
    unsigned hb = 0;
    CK(ctx, cudaMemcpyAsync(&hb, bad.p, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    CK(ctx, cudaStreamSynchronize(s));
    M->diag_ok = hb == 0;
    M->bytes += 8LL * n;
  }
  // Row statistics (host) and static features of the MLP policy.
  std::vector<int> hrp((size_t)n + 1);
  CK(ctx, cudaMemcpyAsync(hrp.data(), M->rp.p, sizeof(int) * ((size_t)n + 1), cudaMemcpyDeviceToHost, s));
  CK(ctx, cudaStreamSynchronize(s));
  double sum = 0, sq = 0, mx = 0;
  for (int i = 0; i < n; ++i) {
    const double l = hrp[i + 1] - hrp[i];
    sum += l;
    sq += l * l;
    mx = std::max(mx, l);
  }
  M->mean = n ? sum / n : 0.0;
  M->maxr = mx;
  for (int li = 0; li < 4; ++li) {
    const int tr = kThreads >> li;
    long long w = 0;
    for (int i = 0; i < n; ++i) w = std::max(w, (long long)hrp[std::min(i + tr, n)] - hrp[i]);
    M->win[li] = w;
  }
  M->cv = (n && M->mean > 0) ? std::sqrt(std::max(0.0, sq / n - M->mean * M->mean)) / M->mean : 0.0;
  // Static features of the MLP policy: log10(n) / 8, mean nnz per row / 64,
  // log10(max a_ii / min a_ii) / 16, log10(max_i sum_j |a_ij| / a_ii) / 16, and the fraction
  // of entries outside the fp16 normal range.
  {
    DevBuf fb;
    CK(ctx, fb.ensure(4 * sizeof(unsigned long long)));
    const unsigned long long init4[4] = {0ull, 0x7ff0000000000000ull, 0ull, 0ull};
    CK(ctx, cudaMemcpyAsync(fb.p, init4, sizeof(init4), cudaMemcpyHostToDevice, s));
    CK(ctx, launch_row_features(n, d.rp, d.ci, d.v64, fb.as<unsigned long long>(), s));
    unsigned long long hfb[4];
    CK(ctx, cudaMemcpyAsync(hfb, fb.p, sizeof(hfb), cudaMemcpyDeviceToHost, s));
    CK(ctx, cudaStreamSynchronize(s));
    double dmax, dmin, gmax;
    memcpy(&dmax, &hfb[0], 8);
    memcpy(&dmin, &hfb[1], 8);
    memcpy(&gmax, &hfb[2], 8);
    M->feat[0] = n > 0 ? (float)(std::log10((double)n) / 8.0) : 0.f;
    M->feat[1] = n > 0 ? (float)(((double)nnz / n) / 64.0) : 0.f;
    M->feat[2] = (dmin > 0 && dmax > 0 && std::isfinite(dmin)) ? (float)(std::log10(dmax / dmin) / 16.0) : 0.f;
    M->feat[3] = gmax > 0 ? (float)(std::log10(gmax) / 16.0) : 0.f;
    M->feat[4] = nnz > 0 ? (float)((double)hfb[3] / (double)nnz) : 0.f;
  }
  default_schedule(M.get());
  *out = M.release();
  return MPCG_OK;
}

mpcg_status mpcg_matrix_destroy(mpcg_matrix_t A) {
  if (!A) return MPCG_ERR_INVALID_ARG;
  cudaSetDevice(A->device);
  delete A;
  return MPCG_OK;
}

mpcg_status mpcg_matrix_info(mpcg_matrix_t A, mpcg_matrix_stats* info) {
  if (!A || !info) return MPCG_ERR_INVALID_ARG;
  memset(info, 0, sizeof(*info));
  info->n = A->dm.n;
  info->nnz = A->dm.nnz;
  info->mean_row_nnz = A->mean;
  info->max_row_nnz = A->maxr;
  info->cv_row_nnz = A->cv;
  for (int f = 0; f < MPCG_NUM_FORMATS; ++f) {
    info->spmv_sched[f] = A->dm.sched[f];
    info->spmv_lanes[f] = A->dm.lanes[f];
  }
  info->device_bytes = A->bytes;
  for (int j = 0; j < 5; ++j) info->static_features[j] = A->feat[j];
  return MPCG_OK;
}

mpcg_status mpcg_csr_levels(int32_t n, const int32_t* row_ptr, const int32_t* col, int32_t* level_lower,
                            int32_t* level_upper, int32_t* depth) {
  if (n < 0 || !depth || (n > 0 && (!row_ptr || !col || !level_lower || !level_upper))) return MPCG_ERR_INVALID_ARG;
  depth[0] = depth[1] = 0;
  if (n == 0) return MPCG_OK;
  if (row_ptr[0] != 0) return MPCG_ERR_INVALID_ARG;
  for (int32_t i = 0; i < n; ++i) {
    if (row_ptr[i + 1] < row_ptr[i]) return MPCG_ERR_INVALID_ARG;
    for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
      if (col[e] < 0 || col[e] >= n) return MPCG_ERR_INVALID_ARG;
  }
  int32_t dl = 0, du = 0;
  for (int32_t i = 0; i < n; ++i) {
    int32_t l = 0;
    for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
      if (col[e] < i) l = std::max(l, level_lower[col[e]] + 1);
    level_lower[i] = l;
    dl = std::max(dl, l + 1);
  }
  for (int32_t i = n - 1; i >= 0; --i) {
    int32_t l = 0;
    for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
      if (col[e] > i) l = std::max(l, level_upper[col[e]] + 1);
    level_upper[i] = l;
    du = std::max(du, l + 1);
  }
  depth[0] = dl;
  depth[1] = du;
  return MPCG_OK;
}

mpcg_status mpcg_matrix_ic0(mpcg_ctx_t ctx, mpcg_matrix_t A, float* factor, void* stream) {
  if (!ctx || !A) return fail(ctx, MPCG_ERR_INVALID_ARG, "NULL argument");
  if (A->ctx != ctx) return fail(ctx, MPCG_ERR_INVALID_ARG, "matrix belongs to another context");
  if (factor && !is_device_ptr(factor)) return fail(ctx, MPCG_ERR_INVALID_ARG, "factor must be a device pointer");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  mpcg_status st = ensure_ic0(ctx, A, s);
  if (st != MPCG_OK) return st;
  if (factor && A->dm.nnz > 0)
    CK(ctx, cudaMemcpyAsync(factor, A->icf.p, 4 * (size_t)A->dm.nnz, cudaMemcpyDeviceToDevice, s));
  CK(ctx, cudaStreamSynchronize(s));
  return MPCG_OK;
}

mpcg_status mpcg_matrix_set_schedule(mpcg_matrix_t A, int32_t fmt, int32_t sched, int32_t lanes) {
  if (!A) return MPCG_ERR_INVALID_ARG;
  if (!valid_fmt(fmt) || lanes < 1 || lanes > 32 || (lanes & (lanes - 1)))
    return fail(A->ctx, MPCG_ERR_INVALID_ARG, "unsupported schedule (fmt %d, sched %d, lanes %d)", fmt, sched, lanes);
  if (sched == SCHED_STREAM) {
    if (lanes > 4) return fail(A->ctx, MPCG_ERR_INVALID_ARG, "the stream schedule takes 1, 2 or 4 lanes per row");
    const int vreg = stream_vreg(A, fmt, lanes);
    if (vreg < 0)
      return fail(A->ctx, MPCG_ERR_INVALID_ARG, "stream schedule with %d lanes does not fit a %d-byte stage", lanes,
                  kStageBytes);
    A->dm.tile_rows[fmt] = kThreads / lanes;
    A->dm.tile_bytes[fmt] = vreg;
  } else if (sched == SCHED_VLOAD) {
    if (lanes != 1) return fail(A->ctx, MPCG_ERR_INVALID_ARG, "the vector-load schedule takes one lane per row");
  } else if (sched == SCHED_MERGE) {
    if (lanes != 1) return fail(A->ctx, MPCG_ERR_INVALID_ARG, "the merge-path schedule takes lanes = 1");
  } else if (sched == SCHED_XSTAGE) {
    if (lanes != 1) return fail(A->ctx, MPCG_ERR_INVALID_ARG, "the staged-x schedule takes lanes = 1");
    if (!A->dm.cols_sorted)
      return fail(A->ctx, MPCG_ERR_INVALID_ARG, "the staged-x schedule needs increasing column indices in every row");
  } else if (sched != SCHED_VECTOR) {
    return fail(A->ctx, MPCG_ERR_INVALID_ARG, "unknown schedule %d", sched);
  }
  A->dm.sched[fmt] = sched;
  A->dm.lanes[fmt] = lanes;
  return MPCG_OK;
}

mpcg_status mpcg_spmv(mpcg_ctx_t ctx, mpcg_matrix_t A, int32_t fmt, const double* x, double* y, int32_t reps,
                      double* ms_per_rep, void* stream) {
  if (!ctx || !A || !x || !y) return fail(ctx, MPCG_ERR_INVALID_ARG, "NULL argument");
  if (!valid_fmt(fmt)) return fail(ctx, MPCG_ERR_INVALID_ARG, "bad format %d", fmt);
  if (!is_device_ptr(x) || !is_device_ptr(y)) return fail(ctx, MPCG_ERR_INVALID_ARG, "x and y must be device pointers");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const int n = A->dm.n;
  CK(ctx, ctx->spmv_x.ensure(4 * (size_t)n + 16));
  CK(ctx, ctx->spmv_q.ensure(8 * (size_t)n + 16));
  DevSys S;
  memset(&S, 0, sizeof(S));
  S.A = A->dm;
  S.p = const_cast<double*>(x);
  S.plow = ctx->spmv_x.p;
  S.q = ctx->spmv_q.p;
  if (fmt != F64) CK(ctx, launch_to_format(x, S.plow, n, fmt, s));
  // The launch shape the solver uses for this matrix: with the stream ring when any format
  // of the matrix uses the stream schedule.
  const bool stream_shape = A->force_stream_shape || uses_stream(A->dm);
  const int grid = ctx->nsm * (stream_shape ? ctx->occ_s : ctx->occ);
  const int stage = stream_shape ? kStageBytes : 0;
  CK(ctx, ctx->spmv_err.ensure(sizeof(unsigned)));
  CK(ctx, cudaMemsetAsync(ctx->spmv_err.p, 0, sizeof(unsigned), s));
  if (reps < 1) reps = 1;
  cudaEvent_t e0, e1;
  CK(ctx, cudaEventCreate(&e0));
  CK(ctx, cudaEventCreate(&e1));
  CK(ctx, launch_spmv_only(S, fmt, grid, stage, ctx->spmv_err.as<unsigned>(), s));  // warm-up
  CK(ctx, cudaEventRecord(e0, s));
  for (int r = 0; r < reps; ++r) CK(ctx, launch_spmv_only(S, fmt, grid, stage, ctx->spmv_err.as<unsigned>(), s));
  CK(ctx, cudaEventRecord(e1, s));
  CK(ctx, launch_from_q(S.q, A->dm.rexp, y, n, fmt, s));
  CK(ctx, cudaStreamSynchronize(s));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  unsigned herr = 0;
  CK(ctx, cudaMemcpy(&herr, ctx->spmv_err.p, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (herr) return fail(ctx, MPCG_ERR_TIMEOUT, "a bulk-copy wait of the product exceeded its limit");
  if (ms_per_rep) *ms_per_rep = ms / reps;
  return MPCG_OK;
}

namespace {
mpcg_status autotune_timed(mpcg_ctx_t ctx, mpcg_matrix_t A, int32_t reps, void* stream);

// Bucket of a matrix for the autotuner's cache: half-octaves of the mean row length, quarters
// of its coefficient of variation, octaves of the longest row and of n, and the column order.
std::tuple<int, int, int, int, int> tune_key(const mpcg_matrix_s* A) {
  const int lm = (int)std::floor(2.0 * std::log2(std::max(A->mean, 1.0)));
  const int lc = std::min(16, (int)std::floor(4.0 * A->cv));
  const int lx = (int)std::floor(std::log2(std::max(A->maxr, 1.0)));
  const int ln = (int)std::floor(std::log2((double)std::max(A->dm.n, 1)));
  return std::make_tuple(lm, lc, lx, ln, A->dm.cols_sorted);
}
}  // namespace

mpcg_status mpcg_matrix_autotune(mpcg_ctx_t ctx, mpcg_matrix_t A, int32_t reps, void* stream) {
  if (!ctx || !A) return fail(ctx, MPCG_ERR_INVALID_ARG, "NULL argument");
  cudaSetDevice(ctx->device);
  const int n = A->dm.n;
  if (n == 0) return MPCG_OK;
  // A product of a small matrix takes a few microseconds on the whole GPU, within the noise
  // of the launch itself: such matrices keep the row-length rule.
  if (A->dm.nnz < kTuneMinNnz) {
    default_schedule(A);
    return MPCG_OK;
  }
  // a matrix of a bucket tuned before in this context takes that bucket's schedules (when they
  // all apply to it); reps < 0 times it anyway and replaces the bucket's entry
  const auto key = tune_key(A);
  if (reps > 0) {
    auto it = ctx->tune_cache.find(key);
    if (it != ctx->tune_cache.end()) {
      bool ok = true;
      for (int f = 0; f < NFMT && ok; ++f)
        ok = mpcg_matrix_set_schedule(A, f, it->second.first[f], it->second.second[f]) == MPCG_OK;
      if (ok) return MPCG_OK;
    }
  }
  const mpcg_status st = autotune_timed(ctx, A, std::max(1, std::abs(reps)), stream);
  if (st != MPCG_OK) return st;
  std::vector<int> sc(NFMT), la(NFMT);
  for (int f = 0; f < NFMT; ++f) {
    sc[f] = A->dm.sched[f];
    la[f] = A->dm.lanes[f];
  }
  ctx->tune_cache[key] = std::make_pair(sc, la);
  return MPCG_OK;
}

namespace {
// Times every (schedule, lanes) per format and keeps the fastest configuration.
mpcg_status autotune_timed(mpcg_ctx_t ctx, mpcg_matrix_t A, int32_t reps, void* stream) {
  const int n = A->dm.n;
  DevBuf x, y;
  CK(ctx, x.ensure(8 * (size_t)n));
  CK(ctx, y.ensure(8 * (size_t)n));
  std::vector<double> ones((size_t)n, 1.0);
  CK(ctx, cudaMemcpy(x.p, ones.data(), 8 * (size_t)n, cudaMemcpyHostToDevice));
  reps = std::max(1, reps);
  auto time_it = [&](int f, int sched, int lanes, double& ms) -> mpcg_status {
    mpcg_status st = mpcg_matrix_set_schedule(A, f, sched, lanes);
    if (st != MPCG_OK) return st;
    return mpcg_spmv(ctx, A, f, x.as<double>(), y.as<double>(), reps, &ms, stream);
  };
  // Configuration P: every format on the sub-warp vector schedule, no stream ring.
  int bestP[NFMT];
  double sumP = 0;
  int schedP[NFMT];
  for (int f = 0; f < NFMT; ++f) A->dm.sched[f] = SCHED_VECTOR;
  for (int f = 0; f < NFMT; ++f) {
    double best = 1e30;
    bestP[f] = A->dm.lanes[f];
    schedP[f] = SCHED_VECTOR;
    for (int lanes = 1; lanes <= 32; lanes *= 2) {
      double ms = 0;
      mpcg_status st = time_it(f, SCHED_VECTOR, lanes, ms);
      if (st != MPCG_OK) return st;
      if (ms < best) { best = ms; bestP[f] = lanes; }
    }
    for (int sched : {SCHED_VLOAD, SCHED_MERGE}) {
      double ms = 0;
      mpcg_status st = time_it(f, sched, 1, ms);
      if (st != MPCG_OK) return st;
      if (ms < best) { best = ms; bestP[f] = 1; schedP[f] = sched; }
    }
    A->dm.sched[f] = schedP[f];
    A->dm.lanes[f] = bestP[f];
    sumP += best;
  }
  // Configuration S: launch shape with the stream ring; each format takes the faster of the
  // stream schedule and the vector schedule measured in that shape.
  bool any = A->dm.cols_sorted != 0;  // the staged-x schedule runs in this shape too
  for (int f = 0; f < NFMT && !any; ++f)
    for (int lanes = 1; lanes <= 4; lanes *= 2) any = any || stream_vreg(A, f, lanes) >= 0;
  if (any) {
    int schedS[NFMT], lanesS[NFMT];
    double sumS = 0;
    A->force_stream_shape = true;
    for (int f = 0; f < NFMT; ++f) {
      double best = 1e30;
      schedS[f] = schedP[f];
      lanesS[f] = bestP[f];
      for (int lanes = 1; lanes <= 32; lanes *= 2) {
        for (int sched = 0; sched < 5; ++sched) {
          if (sched == SCHED_STREAM && (lanes > 4 || stream_vreg(A, f, lanes) < 0)) continue;
          if ((sched == SCHED_VLOAD || sched == SCHED_MERGE || sched == SCHED_XSTAGE) && lanes != 1) continue;
          if (sched == SCHED_XSTAGE && !A->dm.cols_sorted) continue;
          double ms = 0;
          mpcg_status st = time_it(f, sched, lanes, ms);
          if (st != MPCG_OK) {
            A->force_stream_shape = false;
            return st;
          }
          if (ms < best) { best = ms; schedS[f] = sched; lanesS[f] = lanes; }
        }
      }
      mpcg_matrix_set_schedule(A, f, schedS[f], lanesS[f]);
      sumS += best;
    }
    A->force_stream_shape = false;
    bool s_uses = false;
    for (int f = 0; f < NFMT; ++f) s_uses = s_uses || schedS[f] == SCHED_STREAM || schedS[f] == SCHED_XSTAGE;
    if (s_uses && sumS < sumP) {
      for (int f = 0; f < NFMT; ++f) mpcg_matrix_set_schedule(A, f, schedS[f], lanesS[f]);
      return MPCG_OK;
    }
  }
  for (int f = 0; f < NFMT; ++f) mpcg_matrix_set_schedule(A, f, schedP[f], bestP[f]);
  return MPCG_OK;
}
}  // namespace

// ---- policies -----------------------------------------------------------------------------

static mpcg_policy_s* new_policy(mpcg_ctx_t ctx, int kind) {
  mpcg_policy_s* P = new mpcg_policy_s();
  P->ctx = ctx;
  P->device = ctx->device;
  P->kind = kind;
  P->shape = ctx->opt;
  P->nprec = ctx->opt.nprec;
  P->S = ctx->opt.b_bins * ctx->opt.r_bins;
  P->H = ctx->opt.mlp_hidden;
  P->joint = ctx->opt.joint ? 1 : 0;
  return P;
}

mpcg_status mpcg_policy_fixed(mpcg_ctx_t ctx, const int32_t fmt[4], mpcg_policy_t* out) {
  if (!ctx || !fmt || !out) return fail(ctx, MPCG_ERR_INVALID_ARG, "NULL argument");
  for (int j = 0; j < 4; ++j)
    if (!valid_fmt(fmt[j])) return fail(ctx, MPCG_ERR_INVALID_ARG, "fmt[%d] = %d is not a format code", j, fmt[j]);
  mpcg_policy_s* P = new_policy(ctx, 0);
  for (int j = 0; j < 4; ++j) P->fixed[j] = fmt[j];
  *out = P;
  return MPCG_OK;
}

mpcg_status mpcg_policy_schedule(mpcg_ctx_t ctx, const int32_t* fmts, int32_t len, mpcg_policy_t* out) {
  if (!ctx || !fmts || !out || len < 1) return fail(ctx, MPCG_ERR_INVALID_ARG, "bad schedule arguments");
  for (long long i = 0; i < 4LL * len; ++i)
    if (!valid_fmt(fmts[i])) return fail(ctx, MPCG_ERR_INVALID_ARG, "schedule entry %lld = %d is not a format code", i, fmts[i]);
  cudaSetDevice(ctx->device);
  std::unique_ptr<mpcg_policy_s> P(new_policy(ctx, 1));
  CK(ctx, P->sched.ensure(sizeof(int) * 4 * (size_t)len));
  CK(ctx, cudaMemcpy(P->sched.p, fmts, sizeof(int) * 4 * (size_t)len, cudaMemcpyHostToDevice));
  P->sched_len = len;
  *out = P.release();
  return MPCG_OK;
}

mpcg_status mpcg_policy_qtable(mpcg_ctx_t ctx, const double* Q, const int32_t* visits, mpcg_policy_t* out) {
  if (!ctx || !Q || !out) return fail(ctx, MPCG_ERR_INVALID_ARG, "NULL argument");
  cudaSetDevice(ctx->device);
  std::unique_ptr<mpcg_policy_s> P(new_policy(ctx, 2));
  const size_t qn = (size_t)qtable_size(P->S, P->nprec, P->joint);
  CK(ctx, P->Q.ensure(sizeof(double) * qn));
  CK(ctx, P->visits.ensure(sizeof(int) * (size_t)visits_size(P->S, P->joint)));
  CK(ctx, cudaMemcpy(P->Q.p, Q, sizeof(double) * qn, cudaMemcpyHostToDevice));
  std::vector<int> v((size_t)visits_size(P->S, P->joint), 1);
  if (visits) memcpy(v.data(), visits, sizeof(int) * v.size());
  CK(ctx, cudaMemcpy(P->visits.p, v.data(), sizeof(int) * v.size(), cudaMemcpyHostToDevice));
  *out = P.release();
  return MPCG_OK;
}

int64_t mpcg_mlp_nparams(int32_t H, int32_t nprec) {
  const int64_t nout = 4LL * nprec;
  return (int64_t)H * kNFeat + H + (int64_t)H * H + H + nout * H + nout;
}

mpcg_status mpcg_policy_mlp(mpcg_ctx_t ctx, const float* params, mpcg_policy_t* out) {
  if (!ctx || !params || !out) return fail(ctx, MPCG_ERR_INVALID_ARG, "NULL argument");
  cudaSetDevice(ctx->device);
  std::unique_ptr<mpcg_policy_s> P(new_policy(ctx, 3));
  const size_t np = (size_t)mpcg_mlp_nparams(P->H, P->nprec);
  CK(ctx, P->mlp.ensure(sizeof(float) * np));
  CK(ctx, cudaMemcpy(P->mlp.p, params, sizeof(float) * np, cudaMemcpyHostToDevice));
  *out = P.release();
  return MPCG_OK;
}

mpcg_status mpcg_policy_get_qtable(mpcg_policy_t P, double* Q, int32_t* visits) {
  if (!P || P->kind != 2) return MPCG_ERR_INVALID_ARG;
  cudaSetDevice(P->ctx->device);
  const size_t qn = (size_t)qtable_size(P->S, P->nprec, P->joint);
  if (Q) CK(P->ctx, cudaMemcpy(Q, P->Q.p, sizeof(double) * qn, cudaMemcpyDeviceToHost));
  if (visits)
    CK(P->ctx, cudaMemcpy(visits, P->visits.p, sizeof(int) * (size_t)visits_size(P->S, P->joint),
                          cudaMemcpyDeviceToHost));
  return MPCG_OK;
}

mpcg_status mpcg_policy_get_mlp(mpcg_policy_t P, float* params) {
  if (!P || P->kind != 3 || !params) return MPCG_ERR_INVALID_ARG;
  cudaSetDevice(P->ctx->device);
  CK(P->ctx, cudaMemcpy(params, P->mlp.p, sizeof(float) * (size_t)mpcg_mlp_nparams(P->H, P->nprec), cudaMemcpyDeviceToHost));
  return MPCG_OK;
}

namespace {
struct BlobHeader {
  char magic[8];
  int32_t kind, b_bins, r_bins, t_bin;
  double eps_min;
  int32_t nprec, H;
  int32_t precs[8];
  double cost[8];
  int32_t sched_len, fixed[4];
  int32_t joint, pad;
  int64_t payload;
};
}  // namespace

mpcg_status mpcg_policy_save(mpcg_policy_t P, void* blob, size_t* bytes) {
  if (!P || !bytes) return MPCG_ERR_INVALID_ARG;
  mpcg_ctx_t ctx = P->ctx;
  size_t payload = 0;
  if (P->kind == 1) payload = sizeof(int) * 4 * (size_t)P->sched_len;
  if (P->kind == 2)
    payload = sizeof(double) * (size_t)qtable_size(P->S, P->nprec, P->joint) +
              sizeof(int) * (size_t)visits_size(P->S, P->joint);
  if (P->kind == 3) payload = sizeof(float) * (size_t)mpcg_mlp_nparams(P->H, P->nprec);
  const size_t total = sizeof(BlobHeader) + payload;
  if (!blob) {
    *bytes = total;
    return MPCG_OK;
  }
  if (*bytes < total) return fail(ctx, MPCG_ERR_INVALID_ARG, "blob too small: %zu < %zu", *bytes, total);
  BlobHeader h;
  memset(&h, 0, sizeof(h));
  memcpy(h.magic, "MPCGPOL1", 8);
  h.kind = P->kind;
  h.b_bins = P->shape.b_bins;
  h.r_bins = P->shape.r_bins;
  h.t_bin = P->shape.t_bin;
  h.eps_min = P->shape.eps_min;
  h.nprec = P->nprec;
  h.H = P->H;
  for (int a = 0; a < 8; ++a) {
    h.precs[a] = P->shape.precs[a];
    h.cost[a] = P->shape.cost[a];
  }
  h.sched_len = P->sched_len;
  h.joint = P->joint;
  for (int j = 0; j < 4; ++j) h.fixed[j] = P->fixed[j];
  h.payload = (int64_t)payload;
  char* o = (char*)blob;
  memcpy(o, &h, sizeof(h));
  o += sizeof(h);
  cudaSetDevice(ctx->device);
  if (P->kind == 1) CK(ctx, cudaMemcpy(o, P->sched.p, payload, cudaMemcpyDeviceToHost));
  if (P->kind == 2) {
    const size_t qb = sizeof(double) * (size_t)qtable_size(P->S, P->nprec, P->joint);
    CK(ctx, cudaMemcpy(o, P->Q.p, qb, cudaMemcpyDeviceToHost));
    CK(ctx, cudaMemcpy(o + qb, P->visits.p, sizeof(int) * (size_t)visits_size(P->S, P->joint),
                       cudaMemcpyDeviceToHost));
  }
  if (P->kind == 3) CK(ctx, cudaMemcpy(o, P->mlp.p, payload, cudaMemcpyDeviceToHost));
  *bytes = total;
  return MPCG_OK;
}

mpcg_status mpcg_policy_load(mpcg_ctx_t ctx, const void* blob, size_t bytes, mpcg_policy_t* out) {
  if (!ctx || !blob || !out) return fail(ctx, MPCG_ERR_INVALID_ARG, "NULL argument");
  if (bytes < sizeof(BlobHeader)) return fail(ctx, MPCG_ERR_INVALID_ARG, "blob shorter than its header");
  BlobHeader h;
  memcpy(&h, blob, sizeof(h));
  if (memcmp(h.magic, "MPCGPOL1", 8) != 0) return fail(ctx, MPCG_ERR_INVALID_ARG, "bad policy magic");
  if (h.payload < 0 || sizeof(BlobHeader) + (size_t)h.payload > bytes) return fail(ctx, MPCG_ERR_INVALID_ARG, "truncated policy blob");
  const char* o = (const char*)blob + sizeof(h);
  const mpcg_options& c = ctx->opt;
  if (h.kind == 0) {
    return mpcg_policy_fixed(ctx, h.fixed, out);
  }
  if (h.kind == 1) {
    if ((size_t)h.payload != sizeof(int) * 4 * (size_t)h.sched_len) return fail(ctx, MPCG_ERR_INVALID_ARG, "bad schedule payload");
    return mpcg_policy_schedule(ctx, (const int32_t*)o, h.sched_len, out);
  }
  if (h.nprec != c.nprec) return fail(ctx, MPCG_ERR_BAD_POLICY, "policy has %d precisions, context %d", h.nprec, c.nprec);
  for (int a = 0; a < h.nprec; ++a)
    if (h.precs[a] != c.precs[a]) return fail(ctx, MPCG_ERR_BAD_POLICY, "precision set differs at %d", a);
  if (h.kind == 2) {
    if (h.b_bins != c.b_bins || h.r_bins != c.r_bins) return fail(ctx, MPCG_ERR_BAD_POLICY, "state bins differ");
    if ((h.joint != 0) != (c.joint != 0)) return fail(ctx, MPCG_ERR_BAD_POLICY, "joint and per-operation tables differ");
    const int S = c.b_bins * c.r_bins;
    const size_t qb = sizeof(double) * (size_t)qtable_size(S, c.nprec, c.joint ? 1 : 0);
    if ((size_t)h.payload != qb + sizeof(int) * (size_t)visits_size(S, c.joint ? 1 : 0))
      return fail(ctx, MPCG_ERR_INVALID_ARG, "bad table payload");
    return mpcg_policy_qtable(ctx, (const double*)o, (const int32_t*)(o + qb), out);
  }
  if (h.kind == 3) {
    if (h.H != c.mlp_hidden) return fail(ctx, MPCG_ERR_BAD_POLICY, "hidden width %d differs from %d", h.H, c.mlp_hidden);
    if ((size_t)h.payload != sizeof(float) * (size_t)mpcg_mlp_nparams(h.H, h.nprec)) return fail(ctx, MPCG_ERR_INVALID_ARG, "bad MLP payload");
    return mpcg_policy_mlp(ctx, (const float*)o, out);
  }
  return fail(ctx, MPCG_ERR_INVALID_ARG, "unknown policy kind %d", h.kind);
}

mpcg_status mpcg_policy_destroy(mpcg_policy_t P) {
  if (!P) return MPCG_ERR_INVALID_ARG;
  cudaSetDevice(P->device);
  delete P;
  return MPCG_OK;
}

// ---- solves -------------------------------------------------------------------------------

mpcg_status mpcg_solve(mpcg_ctx_t ctx, mpcg_matrix_t A, const double* b, double* x, double tol, int32_t max_iter,
                       mpcg_policy_t policy, mpcg_result* res, mpcg_iter_record* history, int32_t history_cap,
                       void* stream) {
  if (!ctx || !A || !policy || !res) return fail(ctx, MPCG_ERR_INVALID_ARG, "NULL argument");
  ctx->err.clear();
  const int n = A->dm.n;
  if (n > 0 && (!b || !x)) return fail(ctx, MPCG_ERR_INVALID_ARG, "b or x is NULL");
  if (!(tol >= 0.0) || max_iter < 0) return fail(ctx, MPCG_ERR_INVALID_ARG, "tol must be >= 0 and max_iter >= 0");
  if (history && history_cap < 0) return fail(ctx, MPCG_ERR_INVALID_ARG, "history_cap < 0");
  if (A->ctx != ctx || policy->ctx != ctx) return fail(ctx, MPCG_ERR_INVALID_ARG, "objects belong to another context");
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  Plan& pl = ctx->plan;
  const bool bdev = n == 0 || is_device_ptr(b);
  const bool xdev = n == 0 || is_device_ptr(x);
  const bool hdev = !history || is_device_ptr(history);
  const double* bd = b;
  double* xd = x;
  if (!bdev) {
    CK(ctx, pl.bstage.ensure(8 * (size_t)n));
    CK(ctx, cudaMemcpyAsync(pl.bstage.p, b, 8 * (size_t)n, cudaMemcpyHostToDevice, s));
    bd = pl.bstage.as<double>();
  }
  if (!xdev) {
    CK(ctx, pl.xstage.ensure(8 * (size_t)n));
    if (ctx->opt.warm_start) CK(ctx, cudaMemcpyAsync(pl.xstage.p, x, 8 * (size_t)n, cudaMemcpyHostToDevice, s));
    xd = pl.xstage.as<double>();
  }
  mpcg_iter_record* hd = history;
  if (history && !hdev) {
    CK(ctx, pl.hstage.ensure(sizeof(mpcg_iter_record) * (size_t)std::max(history_cap, 1)));
    hd = pl.hstage.as<mpcg_iter_record>();
  }
  std::vector<SysIn> in(1);
  in[0] = SysIn{A, bd, xd, tol, max_iter, hd, history ? history_cap : 0};
  int force = 0;
  if (const char* f = getenv("MPCG_FORCE_TEAM")) force = atoi(f);
  // stepped (one kernel per phase in a while-loop graph) for large systems, or when asked
  const int sm = ctx->opt.stepped;
  const bool stepped =
      ctx->opt.precond != 2 && force == 0 && (sm >= 2 || (sm == 0 && A->dm.nnz >= (1LL << 24)));
  mpcg_status st = build_plan(ctx, pl, in, policy, 0, 0, force, s, 0, stepped);
  pl.stepped_host = stepped && sm == 3;
  if (st != MPCG_OK) return st;
  st = enqueue_plan(ctx, pl, s);
  if (st != MPCG_OK) return st;
  if (!xdev) CK(ctx, cudaMemcpyAsync(x, xd, 8 * (size_t)n, cudaMemcpyDeviceToHost, s));
  if (history && !hdev && history_cap > 0)
    CK(ctx, cudaMemcpyAsync(history, hd, sizeof(mpcg_iter_record) * (size_t)history_cap, cudaMemcpyDeviceToHost, s));
  return finish_plan(ctx, pl, res, s);
}

static mpcg_status collect_batch(mpcg_ctx_t ctx, int32_t nsys, const mpcg_matrix_t* A, const double* const* b,
                                 double* const* x, const double* tol, const int32_t* max_iter, std::vector<SysIn>& in) {
  if (nsys < 0 || (nsys > 0 && (!A || !b || !x || !tol || !max_iter))) return fail(ctx, MPCG_ERR_INVALID_ARG, "bad batch arguments");
  in.resize(nsys);
  for (int i = 0; i < nsys; ++i) {
    if (!A[i] || A[i]->ctx != ctx) return fail(ctx, MPCG_ERR_INVALID_ARG, "system %d: bad matrix", i);
    const int n = A[i]->dm.n;
    if (n > 0 && (!is_device_ptr(b[i]) || !is_device_ptr(x[i])))
      return fail(ctx, MPCG_ERR_INVALID_ARG, "system %d: b and x must be device pointers", i);
    if (!(tol[i] >= 0.0) || max_iter[i] < 0) return fail(ctx, MPCG_ERR_INVALID_ARG, "system %d: bad tol / max_iter", i);
    in[i] = SysIn{A[i], b[i], x[i], tol[i], max_iter[i], nullptr, 0};
  }
  return MPCG_OK;
}

mpcg_status mpcg_solve_batched(mpcg_ctx_t ctx, int32_t nsys, const mpcg_matrix_t* A, const double* const* b,
                               double* const* x, const double* tol, const int32_t* max_iter, mpcg_policy_t policy,
                               mpcg_result* res, void* stream) {
  if (!ctx || !policy || (nsys > 0 && !res)) return fail(ctx, MPCG_ERR_INVALID_ARG, "NULL argument");
  ctx->err.clear();
  cudaSetDevice(ctx->device);
  std::vector<SysIn> in;
  mpcg_status st = collect_batch(ctx, nsys, A, b, x, tol, max_iter, in);
  if (st != MPCG_OK) return st;
  if (nsys == 0) return MPCG_OK;
  cudaStream_t s = (cudaStream_t)stream;
  int force = 0;
  if (const char* f = getenv("MPCG_FORCE_TEAM")) force = atoi(f);
  st = build_plan(ctx, ctx->plan, in, policy, 0, 0, force, s);
  if (st != MPCG_OK) return st;
  st = enqueue_plan(ctx, ctx->plan, s);
  if (st != MPCG_OK) return st;
  return finish_plan(ctx, ctx->plan, res, s);
}

mpcg_status mpcg_graph_create(mpcg_ctx_t ctx, int32_t nsys, const mpcg_matrix_t* A, const double* const* b,
                              double* const* x, const double* tol, const int32_t* max_iter, mpcg_policy_t policy,
                              void* stream, mpcg_graph_t* out) {
  if (!ctx || !policy || !out || nsys < 1) return fail(ctx, MPCG_ERR_INVALID_ARG, "bad graph arguments");
  *out = nullptr;
  ctx->err.clear();
  cudaSetDevice(ctx->device);
  std::vector<SysIn> in;
  mpcg_status st = collect_batch(ctx, nsys, A, b, x, tol, max_iter, in);
  if (st != MPCG_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  std::unique_ptr<mpcg_graph_s> g(new mpcg_graph_s());
  g->ctx = ctx;
  g->device = ctx->device;
  g->plan.reset(new Plan());
  st = build_plan(ctx, *g->plan, in, policy, 0, 0, 0, s);
  if (st != MPCG_OK) return st;
  cudaStream_t cs;
  CK(ctx, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    st = enqueue_plan(ctx, *g->plan, cs);
    cudaGraph_t graph = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    if (st == MPCG_OK && e2 != cudaSuccess) st = fail(ctx, MPCG_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e2));
    g->graph = graph;
  } else {
    st = fail(ctx, MPCG_ERR_CUDA, "cudaStreamBeginCapture failed: %s", cudaGetErrorString(e));
  }
  cudaStreamDestroy(cs);
  if (st != MPCG_OK) {
    if (g->graph) cudaGraphDestroy(g->graph);
    return st;
  }
  CK(ctx, cudaGraphInstantiate(&g->exec, g->graph, 0));
  *out = g.release();
  return MPCG_OK;
}

mpcg_status mpcg_graph_launch(mpcg_graph_t g, void* stream) {
  if (!g) return MPCG_ERR_INVALID_ARG;
  cudaSetDevice(g->ctx->device);
  CK(g->ctx, cudaGraphLaunch(g->exec, (cudaStream_t)stream));
  return MPCG_OK;
}

mpcg_status mpcg_graph_results(mpcg_graph_t g, mpcg_result* res, void* stream) {
  if (!g || !res) return MPCG_ERR_INVALID_ARG;
  cudaSetDevice(g->ctx->device);
  return finish_plan(g->ctx, *g->plan, res, (cudaStream_t)stream);
}

mpcg_status mpcg_graph_destroy(mpcg_graph_t g) {
  if (!g) return MPCG_ERR_INVALID_ARG;
  cudaSetDevice(g->device);
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
  return MPCG_OK;
}

// The options' per-operation masks (bit p = entry p of precs; a 0 mask allows every entry).
static OpMask op_masks(const mpcg_options& o) {
  OpMask m;
  const unsigned all = (1u << o.nprec) - 1u;
  for (int j = 0; j < 4; ++j) m.m[j] = o.op_mask[j] ? ((unsigned)o.op_mask[j] & all) : all;
  return m;
}

// ---- training -----------------------------------------------------------------------------

mpcg_status mpcg_train_qtable(mpcg_ctx_t ctx, int32_t nsys, const mpcg_matrix_t* A, const double* const* b, double tol,
                              int32_t t_max, int32_t episodes, mpcg_policy_t inout, int32_t* iters_out, void* stream) {
  if (!ctx || !inout || nsys < 1 || !A || !b || t_max < 1 || episodes < 1)
    return fail(ctx, MPCG_ERR_INVALID_ARG, "bad training arguments");
  if (inout->kind != 2) return fail(ctx, MPCG_ERR_BAD_POLICY, "training needs a QTABLE policy");
  ctx->err.clear();
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  // Private solution vectors of the episodes (x_0 = 0 each round).
  size_t xbytes = 0;
  for (int i = 0; i < nsys; ++i) xbytes += 8 * (size_t)A[i]->dm.n + 256;
  DevBuf xs;
  CK(ctx, xs.ensure(xbytes));
  std::vector<double*> xp(nsys);
  std::vector<double> tols(nsys, tol);
  std::vector<int32_t> caps(nsys, t_max);
  char* w = xs.as<char>();
  for (int i = 0; i < nsys; ++i) {
    xp[i] = (double*)w;
    w += (8 * (size_t)A[i]->dm.n + 255) / 256 * 256;
  }
  std::vector<SysIn> in;
  mpcg_status st = collect_batch(ctx, nsys, A, b, xp.data(), tols.data(), caps.data(), in);
  if (st != MPCG_OK) return st;
  Plan& pl = ctx->plan;
  int force = 0;
  if (const char* f = getenv("MPCG_FORCE_TEAM")) force = atoi(f);
  st = build_plan(ctx, pl, in, inout, 1, t_max, force, s);
  if (st != MPCG_OK) return st;
  const mpcg_options& o = ctx->opt;
  const int S = o.b_bins * o.r_bins;
  const long long qsize = qtable_size(S, o.nprec, o.joint ? 1 : 0);
  std::vector<mpcg_result> rr(nsys);
  for (int e = 1; e <= episodes; ++e) {
    // epsilon_e = max(eps_floor, eps0 (1 - e / E))  (Section 4.1 with the floor of Section 5)
    double eps = o.eps0 * (1.0 - (double)e / (double)episodes);
    if (eps < o.eps_floor) eps = o.eps_floor;
    pl.L.episode = (unsigned long long)e;
    pl.L.eps = eps;
    CK(ctx, launch_qcopy(inout->Q.as<double>(), pl.qpriv.as<double>(), nsys, qsize, s));
    st = enqueue_plan(ctx, pl, s);
    if (st != MPCG_OK) return st;
    CK(ctx, launch_qmerge(inout->Q.as<double>(), inout->visits.as<int>(), pl.trans.as<Transition>(),
                          pl.st.as<SysState>(), nsys, t_max, S, o.nprec, o.lr, o.gamma, op_masks(o), o.joint ? 1 : 0,
                          s));
    if (iters_out || e == episodes) {
      st = finish_plan(ctx, pl, rr.data(), s);
      if (st != MPCG_OK) return st;
      if (iters_out)
        for (int i = 0; i < nsys; ++i) iters_out[(size_t)(e - 1) * nsys + i] = rr[i].iters;
    }
  }
  return MPCG_OK;
}

// ---- learned policy ----------------------------------------------------------------------

mpcg_status mpcg_collect(mpcg_ctx_t ctx, int32_t nsys, const mpcg_matrix_t* A, const double* const* b, double tol,
                         int32_t max_iter, mpcg_policy_t behavior, double eps, uint64_t episode, mpcg_transition* out,
                         int64_t cap, int64_t* count, void* stream) {
  if (!ctx || !behavior || nsys < 1 || !A || !b || max_iter < 1 || !out || !count || cap < 0)
    return fail(ctx, MPCG_ERR_INVALID_ARG, "bad collection arguments");
  if (behavior->kind != 2 && behavior->kind != 3)
    return fail(ctx, MPCG_ERR_BAD_POLICY, "collection needs a QTABLE or MLP behaviour policy");
  ctx->err.clear();
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  size_t xbytes = 0;
  for (int i = 0; i < nsys; ++i) xbytes += 8 * (size_t)A[i]->dm.n + 256;
  DevBuf xs;
  CK(ctx, xs.ensure(xbytes));
  std::vector<double*> xp(nsys);
  std::vector<double> tols(nsys, tol);
  std::vector<int32_t> caps(nsys, max_iter);
  char* w = xs.as<char>();
  for (int i = 0; i < nsys; ++i) {
    xp[i] = (double*)w;
    w += (8 * (size_t)A[i]->dm.n + 255) / 256 * 256;
  }
  std::vector<SysIn> in;
  mpcg_status st = collect_batch(ctx, nsys, A, b, xp.data(), tols.data(), caps.data(), in);
  if (st != MPCG_OK) return st;
  Plan& pl = ctx->plan;
  st = build_plan(ctx, pl, in, behavior, 1, max_iter, 0, s, max_iter + 1);
  if (st != MPCG_OK) return st;
  const mpcg_options& o = ctx->opt;
  const long long qsize = qtable_size(o.b_bins * o.r_bins, o.nprec, o.joint ? 1 : 0);
  if (behavior->kind == 2) CK(ctx, launch_qcopy(behavior->Q.as<double>(), pl.qpriv.as<double>(), nsys, qsize, s));
  pl.L.episode = (unsigned long long)episode;
  pl.L.eps = eps;
  st = enqueue_plan(ctx, pl, s);
  if (st != MPCG_OK) return st;
  std::vector<mpcg_result> rr(nsys);
  st = finish_plan(ctx, pl, rr.data(), s);
  if (st != MPCG_OK) return st;
  std::vector<SysState> hst(nsys);
  std::vector<Transition> htr((size_t)max_iter * nsys);
  std::vector<float> hf((size_t)kNFeat * (max_iter + 1) * nsys);
  CK(ctx, cudaMemcpy(hst.data(), pl.st.p, sizeof(SysState) * nsys, cudaMemcpyDeviceToHost));
  CK(ctx, cudaMemcpy(htr.data(), pl.trans.p, sizeof(Transition) * htr.size(), cudaMemcpyDeviceToHost));
  CK(ctx, cudaMemcpy(hf.data(), pl.feats.p, sizeof(float) * hf.size(), cudaMemcpyDeviceToHost));
  int64_t c = 0;
  for (int l = 0; l < nsys && c < cap; ++l) {
    const int nt = std::min(hst[l].ntrans, max_iter);
    const float* fl = hf.data() + (size_t)kNFeat * (max_iter + 1) * l;
    for (int t = 0; t < nt && c < cap; ++t, ++c) {
      const Transition& tr = htr[(size_t)max_iter * l + t];
      mpcg_transition& d = out[c];
      memcpy(d.f, fl + (size_t)kNFeat * t, sizeof(d.f));
      memcpy(d.f_next, fl + (size_t)kNFeat * (t + 1), sizeof(d.f_next));
      for (int j = 0; j < 4; ++j) d.act[j] = tr.act[j];
      d.reward = (float)tr.reward;
      d.done = tr.terminal;
    }
  }
  *count = c;
  return MPCG_OK;
}

mpcg_status mpcg_mlp_loss_grad(mpcg_ctx_t ctx, const float* params, int64_t B, const float* feats, const int32_t* acts,
                               const float* y, float* grad, double* loss, void* stream) {
  if (!ctx || !params || B < 1 || !feats || !acts || !y || !grad) return fail(ctx, MPCG_ERR_INVALID_ARG, "NULL argument");
  const mpcg_options& o = ctx->opt;
  for (int64_t i = 0; i < 4 * B; ++i)
    if (acts[i] < 0 || acts[i] >= o.nprec) return fail(ctx, MPCG_ERR_INVALID_ARG, "action %d out of range", acts[i]);
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const long long np = mlp_nparams_dev(o.mlp_hidden, o.nprec);
  const int chunk = 32;
  const int nparts = (int)((B + chunk - 1) / chunk);
  DevBuf dw, df, da, dy, dpart, dl, dg, dloss;
  CK(ctx, dw.ensure(sizeof(float) * np));
  CK(ctx, df.ensure(sizeof(float) * kNFeat * B));
  CK(ctx, da.ensure(sizeof(int) * 4 * B));
  CK(ctx, dy.ensure(sizeof(float) * 4 * B));
  CK(ctx, dpart.ensure(sizeof(float) * np * nparts));
  CK(ctx, dl.ensure(sizeof(double) * nparts));
  CK(ctx, dg.ensure(sizeof(float) * np));
  CK(ctx, dloss.ensure(sizeof(double)));
  CK(ctx, cudaMemcpyAsync(dw.p, params, sizeof(float) * np, cudaMemcpyHostToDevice, s));
  CK(ctx, cudaMemcpyAsync(df.p, feats, sizeof(float) * kNFeat * B, cudaMemcpyHostToDevice, s));
  CK(ctx, cudaMemcpyAsync(da.p, acts, sizeof(int) * 4 * B, cudaMemcpyHostToDevice, s));
  CK(ctx, cudaMemcpyAsync(dy.p, y, sizeof(float) * 4 * B, cudaMemcpyHostToDevice, s));
  CK(ctx, launch_mlp_grad(dw.as<float>(), nullptr, o.mlp_hidden, o.nprec, df.as<float>(), nullptr, da.as<int>(), nullptr,
                          nullptr, dy.as<float>(), nullptr, (int)B, chunk, (float)o.gamma, op_masks(o),
                          dpart.as<float>(), dl.as<double>(), s));
  CK(ctx, launch_mlp_reduce_adam(dpart.as<float>(), nparts, np, dg.as<float>(), nullptr, nullptr, nullptr, 0, 0.f,
                                 dl.as<double>(), dloss.as<double>(), s));
  CK(ctx, cudaMemcpyAsync(grad, dg.p, sizeof(float) * np, cudaMemcpyDeviceToHost, s));
  double hl = 0.0;
  CK(ctx, cudaMemcpyAsync(&hl, dloss.p, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(ctx, cudaStreamSynchronize(s));
  if (loss) *loss = hl;
  return MPCG_OK;
}

mpcg_status mpcg_mlp_train(mpcg_ctx_t ctx, mpcg_policy_t P, const mpcg_transition* data, int64_t count, int32_t steps,
                           int32_t batch, float lr, int32_t target_sync, uint64_t seed, float* loss_out, void* stream) {
  if (!ctx || !P || !data || count < 1 || steps < 1 || batch < 1 || target_sync < 1)
    return fail(ctx, MPCG_ERR_INVALID_ARG, "bad MLP training arguments");
  if (P->kind != 3) return fail(ctx, MPCG_ERR_BAD_POLICY, "mpcg_mlp_train needs an MLP policy");
  const mpcg_options& o = ctx->opt;
  if (P->H != o.mlp_hidden || P->nprec != o.nprec) return fail(ctx, MPCG_ERR_BAD_POLICY, "MLP shape differs from the options");
  for (int64_t i = 0; i < count; ++i)
    for (int j = 0; j < 4; ++j)
      if (data[i].act[j] < 0 || data[i].act[j] >= o.nprec)
        return fail(ctx, MPCG_ERR_INVALID_ARG, "transition %lld: action out of range", (long long)i);
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const long long np = mlp_nparams_dev(o.mlp_hidden, o.nprec);
  const int chunk = 32;
  const int nparts = (batch + chunk - 1) / chunk;
  std::vector<float> hF((size_t)kNFeat * count), hFn((size_t)kNFeat * count), hR(count);
  std::vector<int> hA((size_t)4 * count), hD(count);
  for (int64_t i = 0; i < count; ++i) {
    memcpy(&hF[(size_t)kNFeat * i], data[i].f, sizeof(float) * kNFeat);
    memcpy(&hFn[(size_t)kNFeat * i], data[i].f_next, sizeof(float) * kNFeat);
    for (int j = 0; j < 4; ++j) hA[(size_t)4 * i + j] = data[i].act[j];
    hR[i] = data[i].reward;
    hD[i] = data[i].done;
  }
  DevBuf dF, dFn, dA, dR, dD, dwt, dm, dv, didx, dpart, dl, dloss;
  CK(ctx, dF.ensure(sizeof(float) * hF.size()));
  CK(ctx, dFn.ensure(sizeof(float) * hFn.size()));
  CK(ctx, dA.ensure(sizeof(int) * hA.size()));
  CK(ctx, dR.ensure(sizeof(float) * hR.size()));
  CK(ctx, dD.ensure(sizeof(int) * hD.size()));
  CK(ctx, dwt.ensure(sizeof(float) * np));
  CK(ctx, dm.ensure(sizeof(float) * np));
  CK(ctx, dv.ensure(sizeof(float) * np));
  CK(ctx, didx.ensure(sizeof(long long) * batch));
  CK(ctx, dpart.ensure(sizeof(float) * np * nparts));
  CK(ctx, dl.ensure(sizeof(double) * nparts));
  CK(ctx, dloss.ensure(sizeof(double) * steps));
  CK(ctx, cudaMemcpyAsync(dF.p, hF.data(), sizeof(float) * hF.size(), cudaMemcpyHostToDevice, s));
  CK(ctx, cudaMemcpyAsync(dFn.p, hFn.data(), sizeof(float) * hFn.size(), cudaMemcpyHostToDevice, s));
  CK(ctx, cudaMemcpyAsync(dA.p, hA.data(), sizeof(int) * hA.size(), cudaMemcpyHostToDevice, s));
  CK(ctx, cudaMemcpyAsync(dR.p, hR.data(), sizeof(float) * hR.size(), cudaMemcpyHostToDevice, s));
  CK(ctx, cudaMemcpyAsync(dD.p, hD.data(), sizeof(int) * hD.size(), cudaMemcpyHostToDevice, s));
  CK(ctx, cudaMemsetAsync(dm.p, 0, sizeof(float) * np, s));
  CK(ctx, cudaMemsetAsync(dv.p, 0, sizeof(float) * np, s));
  CK(ctx, cudaMemcpyAsync(dwt.p, P->mlp.p, sizeof(float) * np, cudaMemcpyDeviceToDevice, s));
  for (int t = 1; t <= steps; ++t) {
    CK(ctx, launch_mlp_sample(didx.as<long long>(), batch, count, seed, (unsigned long long)t, s));
    CK(ctx, launch_mlp_grad(P->mlp.as<float>(), dwt.as<float>(), o.mlp_hidden, o.nprec, dF.as<float>(), dFn.as<float>(),
                            dA.as<int>(), dR.as<float>(), dD.as<int>(), nullptr, didx.as<long long>(), batch, chunk,
                            (float)o.gamma, op_masks(o), dpart.as<float>(), dl.as<double>(), s));
    CK(ctx, launch_mlp_reduce_adam(dpart.as<float>(), nparts, np, nullptr, P->mlp.as<float>(), dm.as<float>(),
                                   dv.as<float>(), t, lr, dl.as<double>(), dloss.as<double>() + (t - 1), s));
    if (t % target_sync == 0)
      CK(ctx, cudaMemcpyAsync(dwt.p, P->mlp.p, sizeof(float) * np, cudaMemcpyDeviceToDevice, s));
  }
  std::vector<double> hl(steps);
  CK(ctx, cudaMemcpyAsync(hl.data(), dloss.p, sizeof(double) * steps, cudaMemcpyDeviceToHost, s));
  CK(ctx, cudaStreamSynchronize(s));
  if (loss_out)
    for (int t = 0; t < steps; ++t) loss_out[t] = (float)hl[t];
  return MPCG_OK;
}

mpcg_status mpcg_mlp_adam(mpcg_ctx_t ctx, float* params, float* m, float* v, const float* grad, int32_t t, float lr,
                          void* stream) {
  if (!ctx || !params || !m || !v || !grad || t < 1) return fail(ctx, MPCG_ERR_INVALID_ARG, "bad Adam arguments");
  ctx->err.clear();
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const long long np = mlp_nparams_dev(ctx->opt.mlp_hidden, ctx->opt.nprec);
  const size_t bytes = sizeof(float) * (size_t)np;
  DevBuf dw, dm, dv, dg;
  CK(ctx, dw.ensure(bytes));
  CK(ctx, dm.ensure(bytes));
  CK(ctx, dv.ensure(bytes));
  CK(ctx, dg.ensure(bytes));
  CK(ctx, cudaMemcpyAsync(dw.p, params, bytes, cudaMemcpyHostToDevice, s));
  CK(ctx, cudaMemcpyAsync(dm.p, m, bytes, cudaMemcpyHostToDevice, s));
  CK(ctx, cudaMemcpyAsync(dv.p, v, bytes, cudaMemcpyHostToDevice, s));
  CK(ctx, cudaMemcpyAsync(dg.p, grad, bytes, cudaMemcpyHostToDevice, s));
  // the gradient is the single "partial" of the reduction; no gradient or loss output
  CK(ctx, launch_mlp_reduce_adam(dg.as<float>(), 1, np, nullptr, dw.as<float>(), dm.as<float>(), dv.as<float>(), t, lr,
                                 nullptr, nullptr, s));
  CK(ctx, cudaMemcpyAsync(params, dw.p, bytes, cudaMemcpyDeviceToHost, s));
  CK(ctx, cudaMemcpyAsync(m, dm.p, bytes, cudaMemcpyDeviceToHost, s));
  CK(ctx, cudaMemcpyAsync(v, dv.p, bytes, cudaMemcpyDeviceToHost, s));
  CK(ctx, cudaStreamSynchronize(s));
  return MPCG_OK;
}

mpcg_status mpcg_mlp_targets(mpcg_ctx_t ctx, const float* target_params, int64_t B, const float* feats_next,
                             const float* rew, const int32_t* done, float* y, void* stream) {
  if (!ctx || !target_params || B < 1 || !feats_next || !rew || !done || !y)
    return fail(ctx, MPCG_ERR_INVALID_ARG, "NULL argument or empty batch");
  if (B > (int64_t)1 << 30) return fail(ctx, MPCG_ERR_INVALID_ARG, "batch too large");
  const mpcg_options& o = ctx->opt;
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const long long np = mlp_nparams_dev(o.mlp_hidden, o.nprec);
  DevBuf dw, dfn, dr, dd, dy;
  CK(ctx, dw.ensure(sizeof(float) * np));
  CK(ctx, dfn.ensure(sizeof(float) * kNFeat * B));
  CK(ctx, dr.ensure(sizeof(float) * B));
  CK(ctx, dd.ensure(sizeof(int) * B));
  CK(ctx, dy.ensure(sizeof(float) * 4 * B));
  CK(ctx, cudaMemcpyAsync(dw.p, target_params, sizeof(float) * np, cudaMemcpyHostToDevice, s));
  CK(ctx, cudaMemcpyAsync(dfn.p, feats_next, sizeof(float) * kNFeat * B, cudaMemcpyHostToDevice, s));
  CK(ctx, cudaMemcpyAsync(dr.p, rew, sizeof(float) * B, cudaMemcpyHostToDevice, s));
  CK(ctx, cudaMemcpyAsync(dd.p, done, sizeof(int) * B, cudaMemcpyHostToDevice, s));
  CK(ctx, launch_mlp_targets(dw.as<float>(), o.mlp_hidden, o.nprec, dfn.as<float>(), dr.as<float>(), dd.as<int>(),
                             (int)B, (float)o.gamma, op_masks(o), dy.as<float>(), s));
  CK(ctx, cudaMemcpyAsync(y, dy.p, sizeof(float) * 4 * B, cudaMemcpyDeviceToHost, s));
  CK(ctx, cudaStreamSynchronize(s));
  return MPCG_OK;
}

// ---- solve without device allocation ------------------------------------------------------
//
// For callers that cannot allocate device memory at solve time (for example code running
// under a fixed device-memory budget, inside a memory pool that must not grow, or between
// the set-up and the teardown of an embedding application that reserved all memory up
// front): every scratch buffer of the persistent kernel for one system lives in this
// file-scope device array, reserved when the library is loaded on a device and held until
// the process exits. Layout: a 1 MiB control area (system descriptor, state, result,
// status word, team barriers, team tables, CTA partials), then the work vectors r, p, q and
// p's low-precision copy (28 bytes per row) for at most kNoAllocMaxRows rows.

constexpr int kNoAllocMaxRows = 1 << 20;
constexpr int kNoAllocMaxGrid = 2048;
constexpr size_t kNoAllocCtrl = 1 << 20;
constexpr size_t kNoAllocBytes = kNoAllocCtrl + 28 * (size_t)kNoAllocMaxRows + 4 * 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

mpcg_status mpcg_solve_noalloc(mpcg_ctx_t ctx, mpcg_matrix_t A, const double* b, double* x, double tol,
                               int32_t max_iter, mpcg_policy_t policy, mpcg_result* res, void* stream) {
  if (!ctx || !A || !policy || !res) return fail(ctx, MPCG_ERR_INVALID_ARG, "NULL argument");
  ctx->err.clear();
  const int n = A->dm.n;
  if (n > kNoAllocMaxRows)
    return fail(ctx, MPCG_ERR_INVALID_ARG, "mpcg_solve_noalloc supports at most %d rows (got %d)", kNoAllocMaxRows, n);
  if (n > 0 && (!b || !x)) return fail(ctx, MPCG_ERR_INVALID_ARG, "b or x is NULL");
  if (n > 0 && (!is_device_ptr(b) || !is_device_ptr(x)))
    return fail(ctx, MPCG_ERR_INVALID_ARG, "mpcg_solve_noalloc needs device pointers for b and x");
  if (ctx->opt.precond == 1 && !A->diag_ok)
    return fail(ctx, MPCG_ERR_INVALID_ARG, "Jacobi preconditioning needs a positive diagonal entry in every row");
  if (ctx->opt.precond == 2)
    return fail(ctx, MPCG_ERR_INVALID_ARG, "the no-allocation solve does not run the incomplete Cholesky preconditioner");
  if (ctx->opt.variant != 0)
    return fail(ctx, MPCG_ERR_INVALID_ARG, "the no-allocation solve runs the CG of Section 3 only (variant 0)");
  if (!(tol >= 0.0) || max_iter < 0) return fail(ctx, MPCG_ERR_INVALID_ARG, "tol must be >= 0 and max_iter >= 0");
  if (A->ctx != ctx || policy->ctx != ctx) return fail(ctx, MPCG_ERR_INVALID_ARG, "objects belong to another context");
  cudaError_t ce = cudaSetDevice(ctx->device);
  if (ce != cudaSuccess) return fail(ctx, MPCG_ERR_CUDA, "cudaSetDevice failed: %s", cudaGetErrorString(ce));
  // The array's device address in the current context, looked up with the context's device
  // current on every call (the first lookup on a device loads the library's device code; a
  // cached address would go stale if the context were torn down and created again).
  void* ptr = nullptr;
  ce = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
  if (ce != cudaSuccess || !ptr)
    return fail(ctx, MPCG_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed: %s", cudaGetErrorString(ce));
  unsigned char* base = (unsigned char*)ptr;
  cudaStream_t s = (cudaStream_t)stream;
  const bool stream_shape = uses_stream(A->dm);
  const int grid = ctx->nsm * (stream_shape ? ctx->occ_s : ctx->occ);
  if (grid > kNoAllocMaxGrid) return fail(ctx, MPCG_ERR_INTERNAL, "grid of %d CTAs exceeds the scratch layout", grid);
  // control area
  DevSys* d_sys = (DevSys*)(base + 0);
  SysState* d_st = (SysState*)(base + 4096);
  mpcg_result* d_res = (mpcg_result*)(base + 12288);
  unsigned* d_err = (unsigned*)(base + 16384);
  unsigned* d_bars = (unsigned*)(base + 20480);
  int* d_tsize = (int*)(base + 24576);
  int* d_tfirst = d_tsize + 4;
  int* d_tsoff = d_tsize + 8;
  int* d_tsys = d_tsize + 12;
  int* d_cta_team = (int*)(base + 32768);
  int* d_cta_rank = d_cta_team + kNoAllocMaxGrid;
  double* d_part = (double*)(base + 65536);
  static_assert(4096 >= sizeof(DevSys) && 8192 >= sizeof(SysState), "control area too small");
  static_assert(65536 + sizeof(double) * kNSlot * kNoAllocMaxGrid <= kNoAllocCtrl, "control area too small");
  // work vectors
  unsigned char* w = base + kNoAllocCtrl;
  auto take = [&](size_t bytes) {
    unsigned char* r = w;
    w += (bytes + 255) / 256 * 256;
    return (void*)r;
  };
  DevSys hs;
  memset(&hs, 0, sizeof(hs));
  hs.A = A->dm;
  hs.A.dinv = ctx->opt.precond == 1 ? A->dinv.as<double>() : nullptr;
  hs.b = b;
  hs.x = x;
  hs.r = (double*)take(8 * (size_t)n);
  hs.p = (double*)take(8 * (size_t)n);
  hs.q = take(8 * (size_t)n);
  hs.plow = take(4 * (size_t)n);
  hs.tol = tol;
  hs.max_iter = max_iter;
  for (int j = 0; j < 5; ++j) hs.feat_static[j] = A->feat[j];
  // one team for the system, the remaining CTAs in an empty second team
  const int ts = team_size_for(A->dm.nnz + 4LL * n, grid);
  int tsize[2] = {ts, std::max(1, grid - ts)};
  int tfirst[3] = {0, ts, grid};
  int tsoff[3] = {0, 1, 1};
  int tsys[1] = {0};
  static thread_local int cta_team[kNoAllocMaxGrid], cta_rank[kNoAllocMaxGrid];
  for (int c = 0; c < grid; ++c) {
    cta_team[c] = c < ts ? 0 : 1;
    cta_rank[c] = c < ts ? c : c - ts;
  }
  CK(ctx, cudaMemcpyAsync(d_sys, &hs, sizeof(DevSys), cudaMemcpyHostToDevice, s));
  CK(ctx, cudaMemcpyAsync(d_tsize, tsize, sizeof(tsize), cudaMemcpyHostToDevice, s));
  CK(ctx, cudaMemcpyAsync(d_tfirst, tfirst, sizeof(tfirst), cudaMemcpyHostToDevice, s));
  CK(ctx, cudaMemcpyAsync(d_tsoff, tsoff, sizeof(tsoff), cudaMemcpyHostToDevice, s));
  CK(ctx, cudaMemcpyAsync(d_tsys, tsys, sizeof(tsys), cudaMemcpyHostToDevice, s));
  CK(ctx, cudaMemcpyAsync(d_cta_team, cta_team, sizeof(int) * grid, cudaMemcpyHostToDevice, s));
  CK(ctx, cudaMemcpyAsync(d_cta_rank, cta_rank, sizeof(int) * grid, cudaMemcpyHostToDevice, s));
  // the array keeps the previous call's contents: barriers and the status word start at zero
  CK(ctx, cudaMemsetAsync(d_bars, 0, sizeof(unsigned) * kBarStride * 2, s));
  CK(ctx, cudaMemsetAsync(d_err, 0, sizeof(unsigned), s));
  Launch L;
  memset(&L, 0, sizeof(L));
  L.sys = d_sys;
  L.st = d_st;
  L.nsys = 1;
  L.nteams = 2;
  L.cta_team = d_cta_team;
  L.cta_rank = d_cta_rank;
  L.team_size = d_tsize;
  L.team_first = d_tfirst;
  L.team_sys_off = d_tsoff;
  L.team_sys = d_tsys;
  L.bars = d_bars;
  L.partials = d_part;
  L.res = d_res;
  L.err = d_err;
  mpcg_status st = fill_policy(ctx, policy, L.pol);
  if (st != MPCG_OK) return st;
  L.opt = ctx->ov;
  L.train = 0;
  L.stream_stage = stream_shape ? kStageBytes : 0;
  L.timeout_cycles = kTimeoutCycles;  // the same wait limit as mpcg_solve, with its override
  if (const char* t = getenv("MPCG_TIMEOUT_CYCLES")) L.timeout_cycles = atoll(t);
  cudaGetLastError();
  CK(ctx, launch_cg(L, grid, stream_shape ? 2 * (size_t)kStageBytes : 0, s));
  unsigned herr = 0;
  CK(ctx, cudaMemcpyAsync(res, d_res, sizeof(mpcg_result), cudaMemcpyDeviceToHost, s));
  CK(ctx, cudaMemcpyAsync(&herr, d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  CK(ctx, cudaStreamSynchronize(s));
  if (herr == DERR_TIMEOUT) return fail(ctx, MPCG_ERR_TIMEOUT, "a device-side barrier wait exceeded its limit");
  if (herr) return fail(ctx, MPCG_ERR_INTERNAL, "device status word %u", herr);
  res->kernel_launches = 1;
  return MPCG_OK;
}

}  // extern "C"
