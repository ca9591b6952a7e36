// Setup and auxiliary kernels: CSR validation, the value copies of every format (one
// rounding from fp64 each), the standalone product used for timing and autotuning, and
// the Q-table copy and end-of-round merge of the batched training reading of Algorithm 1.
#include "internal.h"
#include "spmv.cuh"
#include "ic0.cuh"

#include <algorithm>

namespace mpcg {

namespace {

enum : unsigned {
  VF_ROWPTR = 1u,   // row_ptr[0] != 0, row_ptr[n] != nnz, or an entry outside [0, nnz]
  VF_ORDER = 2u,    // row_ptr decreasing
  VF_COL = 4u,      // column index outside [0, n)
  VF_VALUE = 8u,    // non-finite value
  VF_DIAG = 16u,    // diagonal entry missing or not positive
  VF_UNSORTED = 32u // (not an error) some row's column indices do not strictly increase
};

__global__ void validate_rowptr(int n, long long nnz, const int* __restrict__ rp, unsigned* flags, int* bad_row) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i <= n; i += (long long)gridDim.x * blockDim.x) {
    const int v = rp[i];
    unsigned f = 0;
    if (v < 0 || (long long)v > nnz) f |= VF_ROWPTR;
    if (i == 0 && v != 0) f |= VF_ROWPTR;
    if (i == n && (long long)v != nnz) f |= VF_ROWPTR;
    if (i < n && rp[i + 1] < v) f |= VF_ORDER;
    if (f) {
      atomicOr(flags, f);
      atomicMin(bad_row, (int)i);
    }
  }
}

// One warp per row; runs only after validate_rowptr found row_ptr consistent.
__global__ void validate_rows(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                              const double* __restrict__ v, unsigned* flags, int* bad_row) {
  const int lane = threadIdx.x & 31;
  for (long long row = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; row < n;
       row += ((long long)gridDim.x * blockDim.x) >> 5) {
    const int e0 = rp[row], e1 = rp[row + 1];
    unsigned f = 0;
    int diag_ok = 0, unsorted = 0;
    for (int e = e0 + lane; e < e1; e += 32) {
      const int c = ci[e];
      const double a = v[e];
      if (c < 0 || c >= n) f |= VF_COL;
      if (!isfinite(a)) f |= VF_VALUE;
      if (c == row && a > 0.0) diag_ok = 1;
      if (e > e0 && ci[e - 1] >= c) unsorted = 1;
    }
    diag_ok = __any_sync(kFull, diag_ok);
    unsorted = __any_sync(kFull, unsorted);
    f = __reduce_or_sync(kFull, f);
    if (!diag_ok) f |= VF_DIAG;
    if (f && lane == 0) {
      atomicOr(flags, f);
      atomicMin(bad_row, (int)row);
    }
    if (unsorted && lane == 0) atomicOr(flags, (unsigned)VF_UNSORTED);
  }
}

// One warp per row: row scale s_i = 2^e_i with e_i = floor(log2 max_j |a_ij|) (rows whose
// largest entry is below the fp64 normal range use e_i = -1022), then every copy rounded
// once from fp64.
__global__ void convert_values(int n, const int* __restrict__ rp, const double* __restrict__ v64, float* v32,
                               float* vtf, __half* v16, __nv_bfloat16* vbf, __half* v16r, __nv_bfloat16* vbfr,
                               q52_t* v8, short* rexp) {
  const int lane = threadIdx.x & 31;
  for (long long row = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; row < n;
       row += ((long long)gridDim.x * blockDim.x) >> 5) {
    const int e0 = rp[row], e1 = rp[row + 1];
    double m = 0.0;
    for (int e = e0 + lane; e < e1; e += 32) m = fmax(m, fabs(v64[e]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(kFull, m, o));
    int ex = 0;
    if (m > 0.0) ex = (int)(((unsigned long long)__double_as_longlong(m) >> 52) & 0x7ff) - 1023;
    if (ex < -1022) ex = -1022;
    // 2^-ex, split in two factors so that it stays representable for every ex
    const double s1 = pow2(-ex / 2), s2 = pow2(-ex - (-ex / 2));
    if (lane == 0) rexp[row] = (short)ex;
    for (int e = e0 + lane; e < e1; e += 32) {
      const double a = v64[e];
      v32[e] = (float)round_to<24, -126, 127>(a);
      vtf[e] = (float)round_to<11, -126, 127>(a);
      v16[e] = __double2half(round_to<11, -14, 15>(a));
      vbf[e] = __double2bfloat16(round_to<8, -126, 127>(a));
      v8[e] = q52_from_exact((float)round_to<3, -14, 15>(a));
      const double as = (a * s1) * s2;
      v16r[e] = __double2half(round_to<11, -14, 15>(as));
      vbfr[e] = __double2bfloat16(round_to<8, -126, 127>(as));
    }
  }
}

// Row statistics behind the MLP policy's static features: largest and smallest diagonal,
// largest Gershgorin ratio sum_j |a_ij| / a_ii, and the count of entries outside the fp16
// normal range [2^-14, 65504]. Positive doubles order like their bit patterns, so the
// maxima and minima use integer atomics. out: [0] max diag, [1] min diag, [2] max ratio
// (as bit patterns), [3] count.
__global__ void row_features(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                             const double* __restrict__ v, unsigned long long* out) {
  const int lane = threadIdx.x & 31;
  for (long long row = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; row < n;
       row += ((long long)gridDim.x * blockDim.x) >> 5) {
    const int e0 = rp[row], e1 = rp[row + 1];
    double d = 0.0, rs = 0.0;
    unsigned long long cnt = 0;
    for (int e = e0 + lane; e < e1; e += 32) {
      const double a = fabs(v[e]);
      rs += a;
      if (ci[e] == row) d = v[e];
      if (a != 0.0 && (a < 0x1.0p-14 || a > 65504.0)) ++cnt;
    }
    for (int o = 16; o > 0; o >>= 1) {
      rs += __shfl_xor_sync(kFull, rs, o);
      d += __shfl_xor_sync(kFull, d, o);
      cnt += __shfl_xor_sync(kFull, cnt, o);
    }
    if (lane == 0) {
      if (d > 0.0) {
        atomicMax(out + 0, (unsigned long long)__double_as_longlong(d));
        atomicMin(out + 1, (unsigned long long)__double_as_longlong(d));
        atomicMax(out + 2, (unsigned long long)__double_as_longlong(rs / d));
      }
      if (cnt) atomicAdd(out + 3, cnt);
    }
  }
}

// x (fp64) -> fl_f(x) stored in format f.
__global__ void to_format(const double* __restrict__ x, void* xlow, int n, int f) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float r = round_d2f(x[i], f);
    switch (store_of(f)) {
      case ST_Q52: ((q52_t*)xlow)[i] = q52_from_exact(r); break;
      case ST_HALF: ((__half*)xlow)[i] = __float2half_rn(r); break;
      case ST_BF16: ((__nv_bfloat16*)xlow)[i] = __float2bfloat16_rn(r); break;
      default: ((float*)xlow)[i] = r; break;
    }
  }
}

// y = q (stored in format f) as fp64, times the row scale for the row-scaled formats.
__global__ void from_q(const void* q, const short* __restrict__ rexp, double* y, int n, int f) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double v = load_fmt(q, i, f);
    if (row_scaled(f)) v *= pow2(rexp[i]);
    y[i] = v;
  }
}

// Standalone product with the same per-CTA row split and row code as the solver.
__global__ void __launch_bounds__(kThreads) spmv_standalone(const DevSys S, int fmt, int stream_stage, unsigned* err) {
  __shared__ int r01[2];
  __shared__ unsigned long long mbar[2];
  __shared__ unsigned phase;
  extern __shared__ __align__(128) unsigned char dyn[];
  if (threadIdx.x == 0) {
    r01[0] = part_row(S.A.rp, S.A.n, S.A.nnz, blockIdx.x, gridDim.x);
    r01[1] = part_row(S.A.rp, S.A.n, S.A.nnz, blockIdx.x + 1, gridDim.x);
    if (stream_stage > 0) {
      mbar_init(mbar + 0, 1);
      mbar_init(mbar + 1, 1);
      mbar_fence_init();
      phase = 0;
    }
  }
  __syncthreads();
  StreamCtx scx{dyn, mbar, &phase, err, stream_stage};
  DotAcc nu{0.0, 0.f, 0.f};
  spmv_rows(S, Rows{r01[0], r01[1]}, fmt, -1, nu, stream_stage > 0 ? &scx : nullptr);
}

// Jacobi preconditioner: dinv[i] = 1 / a_ii in fp64 (one thread per row); a row without a
// positive diagonal entry sets *bad and gets dinv = 0.
__global__ void jacobi_diag(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                            const double* __restrict__ v, double* dinv, unsigned* bad) {
  for (long long row = blockIdx.x * (long long)blockDim.x + threadIdx.x; row < n;
       row += (long long)gridDim.x * blockDim.x) {
    double d = 0.0;
    for (int e = rp[row]; e < rp[row + 1]; ++e)
      if (ci[e] == row) d = v[e];
    if (d > 0.0) {
      dinv[row] = 1.0 / d;
    } else {
      dinv[row] = 0.0;
      atomicOr(bad, 1u);
    }
  }
}

// Position of column k in the sorted columns ci[lo..hi), or -1.
__device__ __forceinline__ int find_col(const int* __restrict__ ci, int lo, int hi, int k) {
  --hi;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    const int c = ci[mid];
    if (c == k) return mid;
    if (c < k) lo = mid + 1;
    else hi = mid - 1;
  }
  return -1;
}

// IC(0) in fp32 (the SPD reading of Section 5's fp32 incomplete factorization), row by row:
//   l_ij = (fl32(a_ij) - sum_{k<j} l_ik l_jk) / l_jj   for the stored j < i,
//   l_ii = sqrt(fl32(a_ii) - sum_{k<i} l_ik^2),
// each sum over the columns k stored in both rows, in increasing k (a merge of the two sorted
// rows), every operation a single correctly rounded fp32 one. One thread per row, each
// thread's rows in increasing order (grid stride), all CTAs resident: row i waits on the
// completion marks of the rows j < i it reads. A broken row (columns not strictly
// increasing, no diagonal) sets err bit 2 and a non-positive or non-finite pivot bit 1; such
// rows are still marked complete so that no wait is left hanging. Writes F at (i, j <= i)
// and icd[i].
__global__ void __launch_bounds__(kThreads) ic0_factor(int n, const int* __restrict__ rp,
                                                       const int* __restrict__ ci, const double* __restrict__ v,
                                                       float* F, int* icd, unsigned* done, unsigned* err,
                                                       long long limit) {
  bool ok = true;
  for (long long row = blockIdx.x * (long long)blockDim.x + threadIdx.x; row < n;
       row += (long long)gridDim.x * blockDim.x) {
    const int i = (int)row;
    const int e0 = rp[i], e1 = rp[i + 1];
    int di = -1;
    bool broken = false;
    for (int e = e0; e < e1; ++e) {
      const int c = ci[e];
      if (e > e0 && c <= ci[e - 1]) broken = true;
      if (c == i) di = e;
    }
    if (broken || di < 0) {
      atomicOr(err, 2u);
      icd[i] = e0;
      if (e1 > e0) F[e0] = 1.0f;
      st_release(done + i, 1u);
      continue;
    }
    icd[i] = di;
    for (int e = e0; e < di; ++e) {
      const int j = ci[e];
      if (ok && ld_acquire(done + j) < 1u) ok = ic_wait_slow(done + j, 1u, err, 4u, limit);
      const int jb = rp[j], jd = __ldcg(icd + j);
      float s = __double2float_rn(v[e]);
      const int la = e - e0, lc = jd - jb;
      if (la > 8 * lc || lc > 8 * la) {
        // lengths far apart (a hub row against short ones): walk the shorter list and bisect
        // the longer; the matches come in the same increasing order as in the merge
        if (la <= lc) {
          for (int a = e0; a < e; ++a) {
            const int c = find_col(ci, jb, jd, ci[a]);
            if (c >= 0) s = __fsub_rn(s, __fmul_rn(F[a], __ldcg(F + c)));
          }
        } else {
          for (int c = jb; c < jd; ++c) {
            const int a = find_col(ci, e0, e, ci[c]);
            if (a >= 0) s = __fsub_rn(s, __fmul_rn(F[a], __ldcg(F + c)));
          }
        }
      } else {
        int a = e0, c = jb;
        while (a < e && c < jd) {
          const int ka = ci[a], kc = ci[c];
          if (ka < kc) {
            ++a;
          } else if (ka > kc) {
            ++c;
          } else {
            s = __fsub_rn(s, __fmul_rn(F[a], __ldcg(F + c)));
            ++a;
            ++c;
          }
        }
      }
      F[e] = __fdiv_rn(s, jd < rp[j + 1] ? __ldcg(F + jd) : 1.0f);
    }
    float s = __double2float_rn(v[di]);
    for (int e = e0; e < di; ++e) s = __fsub_rn(s, __fmul_rn(F[e], F[e]));
    if (!(s > 0.0f) || !isfinite(s)) {
      atomicOr(err, 1u);
      s = 1.0f;
    }
    F[di] = __fsqrt_rn(s);
    st_release(done + i, 1u);
  }
}

// Upper positions of the factor: (i, j), j > i, takes l_ji from row j. Every off-diagonal
// entry needs its transposed partner (found by bisection in the other row's sorted
// columns); a missing one sets err bit 2.
__global__ void ic0_transpose(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                              const int* __restrict__ icd, float* F, unsigned* err) {
  for (long long row = blockIdx.x * (long long)blockDim.x + threadIdx.x; row < n;
       row += (long long)gridDim.x * blockDim.x) {
    const int i = (int)row;
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
      const int j = ci[e];
      if (j == i) continue;
      const int t = find_col(ci, rp[j], rp[j + 1], i);
      if (t < 0) {
        atomicOr(err, 2u);
        continue;
      }
      if (j > i) F[e] = F[t];
    }
  }
}

__global__ void qcopy_kernel(const double* __restrict__ Q, double* Qpriv, int nlanes, long long qsize) {
  const long long total = qsize * nlanes;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x)
    Qpriv[i] = Q[i % qsize];
}

// End-of-round merge: replays every recorded transition (lane 0..B-1, then iteration
// order) onto the shared tables with the Q-learning update of Section 4.1. The four
// operation tables are independent, so one thread per table replays them in that order.
__global__ void qmerge_kernel(double* Q, int* visits, const Transition* __restrict__ trans,
                              const SysState* __restrict__ st, int nlanes, int cap, int S, int nprec, double lr,
                              double gamma, OpMask mask, int joint, int use_smem) {
  extern __shared__ double tab[];
  const long long np4 = (long long)nprec * nprec * nprec * nprec;
  const long long tsize = (long long)S * nprec;
  const long long total = joint ? S * np4 : 4 * tsize;
  double* T = use_smem ? tab : Q;
  if (use_smem) {
    for (long long i = threadIdx.x; i < total; i += blockDim.x) tab[i] = Q[i];
    __syncthreads();
  }
  const int j = threadIdx.x >> 5;
  if (joint && threadIdx.x == 0) {  // one table over the joint actions, one update per transition
    for (int l = 0; l < nlanes; ++l) {
      int nt = st[l].ntrans;
      if (nt > cap) nt = cap;
      for (int t = 0; t < nt; ++t) {
        const Transition tr = trans[(long long)l * cap + t];
        const int a = ((tr.act[0] * nprec + tr.act[1]) * nprec + tr.act[2]) * nprec + tr.act[3];
        double* row = T + tr.s * np4;
        double target = tr.reward;
        if (!tr.terminal) target = __dadd_rn(target, __dmul_rn(gamma, joint_row_max(T + tr.s_next * np4, nprec, mask.m)));
        const double cur = row[a];
        row[a] = __dadd_rn(cur, __dmul_rn(lr, __dsub_rn(target, cur)));
        visits[tr.s] += 1;
      }
    }
  } else if (!joint && j < 4 && (threadIdx.x & 31) == 0) {
    double* Tj = T + j * tsize;
    for (int l = 0; l < nlanes; ++l) {
      int nt = st[l].ntrans;
      if (nt > cap) nt = cap;
      for (int t = 0; t < nt; ++t) {
        const Transition tr = trans[(long long)l * cap + t];
        double* row = Tj + (long long)tr.s * nprec;
        double target = tr.reward;
        if (!tr.terminal)  // max over the operation's allowed entries
          target = __dadd_rn(target, __dmul_rn(gamma, row_max_allowed(Tj + (long long)tr.s_next * nprec, nprec,
                                                                      mask.m[j])));
        const int a = tr.act[j];
        const double cur = row[a];
        row[a] = __dadd_rn(cur, __dmul_rn(lr, __dsub_rn(target, cur)));
        visits[j * S + tr.s] += 1;
      }
    }
  }
  if (use_smem) {
    __syncthreads();
    for (long long i = threadIdx.x; i < total; i += blockDim.x) Q[i] = tab[i];
  }
}

int grid_for(long long work, int per_block) {
  long long g = (work + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > 152 * 32) g = 152 * 32;
  return (int)g;
}

}  // namespace

cudaError_t launch_validate(int n, long long nnz, const int* rp, const int* ci, const double* v, unsigned* flags,
                            int* bad_row, cudaStream_t s) {
  cudaGetLastError();
  validate_rowptr<<<grid_for((long long)n + 1, kThreads), kThreads, 0, s>>>(n, nnz, rp, flags, bad_row);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  unsigned hf = 0;
  e = cudaMemcpyAsync(&hf, flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess || hf) return e;
  if (n > 0) validate_rows<<<grid_for((long long)n * 32, kThreads), kThreads, 0, s>>>(n, rp, ci, v, flags, bad_row);
  return cudaGetLastError();
}

cudaError_t launch_convert(const DevMatrix& A, float* v32, float* vtf, __half* v16, __nv_bfloat16* vbf,
                           __half* v16r, __nv_bfloat16* vbfr, q52_t* v8, short* rexp, cudaStream_t s) {
  if (A.n == 0) return cudaSuccess;
  cudaGetLastError();
  convert_values<<<grid_for((long long)A.n * 32, kThreads), kThreads, 0, s>>>(A.n, A.rp, A.v64, v32, vtf, v16, vbf,
                                                                             v16r, vbfr, v8, rexp);
  return cudaGetLastError();
}

cudaError_t launch_jacobi_diag(int n, const int* rp, const int* ci, const double* v, double* dinv, unsigned* bad,
                               cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  cudaGetLastError();
  jacobi_diag<<<grid_for(n, kThreads), kThreads, 0, s>>>(n, rp, ci, v, dinv, bad);
  return cudaGetLastError();
}

cudaError_t launch_ic0_factor(int n, const int* rp, const int* ci, const double* v, float* F, int* icd,
                              unsigned* done, unsigned* err, long long timeout_cycles, int nsm, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  cudaGetLastError();
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ic0_factor, kThreads, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  long long want = ((long long)n + kThreads - 1) / kThreads;
  const int grid = (int)std::min<long long>(want, (long long)per_sm * nsm);
  void* args[] = {&n, (void*)&rp, (void*)&ci, (void*)&v, &F, &icd, &done, &err, &timeout_cycles};
  e = cudaLaunchCooperativeKernel((const void*)ic0_factor, dim3(grid), dim3(kThreads), args, 0, s);
  if (e != cudaSuccess) return e;
  ic0_transpose<<<grid_for(n, kThreads), kThreads, 0, s>>>(n, rp, ci, icd, F, err);
  return cudaGetLastError();
}

cudaError_t launch_row_features(int n, const int* rp, const int* ci, const double* v, unsigned long long* out,
                                cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  cudaGetLastError();
  row_features<<<grid_for((long long)n * 32, kThreads), kThreads, 0, s>>>(n, rp, ci, v, out);
  return cudaGetLastError();
}

cudaError_t launch_to_format(const double* x, void* xlow, int n, int f, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  cudaGetLastError();
  to_format<<<grid_for(n, kThreads), kThreads, 0, s>>>(x, xlow, n, f);
  return cudaGetLastError();
}

cudaError_t launch_from_q(const void* q, const short* rexp, double* y, int n, int f, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  cudaGetLastError();
  from_q<<<grid_for(n, kThreads), kThreads, 0, s>>>(q, rexp, y, n, f);
  return cudaGetLastError();
}

cudaError_t launch_spmv_only(const DevSys& S, int fmt, int grid, int stream_stage, unsigned* err, cudaStream_t s) {
  if (S.A.n == 0) return cudaSuccess;
  cudaGetLastError();
  spmv_standalone<<<grid, kThreads, stream_stage > 0 ? 2 * (size_t)stream_stage : 0, s>>>(S, fmt, stream_stage, err);
  return cudaGetLastError();
}

cudaError_t spmv_occupancy(int* blocks_per_sm, size_t smem) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, spmv_standalone, kThreads, smem);
}

cudaError_t cg_set_smem_limit(size_t bytes);

cudaError_t set_smem_limits(size_t bytes) {
  cudaError_t e = cudaFuncSetAttribute(spmv_standalone, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  return cg_set_smem_limit(bytes);
}

cudaError_t launch_qcopy(const double* Q, double* Qpriv, int nlanes, long long qsize, cudaStream_t s) {
  cudaGetLastError();
  qcopy_kernel<<<grid_for(qsize * nlanes, kThreads), kThreads, 0, s>>>(Q, Qpriv, nlanes, qsize);
  return cudaGetLastError();
}

cudaError_t launch_qmerge(double* Q, int* visits, const Transition* trans, const SysState* st, int nlanes, int cap,
                          int S, int nprec, double lr, double gamma, OpMask mask, int joint, cudaStream_t s) {
  const size_t bytes = sizeof(double) * (size_t)qtable_size(S, nprec, joint);
  const int use_smem = bytes <= 48 * 1024 ? 1 : 0;
  cudaGetLastError();
  qmerge_kernel<<<1, 128, use_smem ? bytes : 0, s>>>(Q, visits, trans, st, nlanes, cap, S, nprec, lr, gamma, mask,
                                                     joint, use_smem);
  return cudaGetLastError();
}

}  // namespace mpcg
