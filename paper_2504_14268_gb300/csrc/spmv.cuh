// Sparse matrix-vector product of the mixed-precision CG (op 1 of Section 4.2,
// q = fl_p1(A fl_p1(p))), shared by the persistent solver kernel and the standalone product
// kernel used for timing and autotuning.
#pragma once

#include "internal.h"

namespace mpcg {
namespace {

constexpr unsigned kFull = 0xffffffffu;

struct Rows {
  int r0, r1;
};

// First row of part c of S parts of equal nonzero count (rows [part(c), part(c+1)) ).
__device__ __forceinline__ int part_row(const int* rp, int n, long long nnz, int c, int S) {
  if (c <= 0) return 0;
  if (c >= S) return n;
  const long long target = nnz * (long long)c / (long long)S;
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if ((long long)__ldg(rp + mid) < target) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ void nu_term(double pi, double qi, int p3, double& nd, float& nf) {
  if (p3 == F64) nd = fma(pi, qi, nd);
  else nf = fmaf((float)round_fmt(pi, p3), (float)round_fmt(qi, p3), nf);
}

// Rounds the accumulator of row i onto the product's format, stores it in q and returns the
// row's value of q (times the row scale for the row-scaled formats) as fp64.
__device__ __forceinline__ double store_q(void* q, int i, float acc, int p1, float scale) {
  switch (store_of(p1)) {
    case ST_HALF: {
      const __half h = __float2half_rn(acc);
      ((__half*)q)[i] = h;
      return (double)__half2float(h) * (double)scale;
    }
    case ST_BF16: {
      const __nv_bfloat16 h = __float2bfloat16_rn(acc);
      ((__nv_bfloat16*)q)[i] = h;
      return (double)__bfloat162float(h) * (double)scale;
    }
    default: {
      const float v = (base_fmt(p1) == TF32) ? round_tf32(acc) : acc;
      ((float*)q)[i] = v;
      return (double)v;
    }
  }
}
__device__ __forceinline__ double store_q(void* q, int i, double acc, int, float) {
  ((double*)q)[i] = acc;
  return acc;
}

// Sub-warp vector CSR: K lanes per row, rows strided over the CTA, lane sums combined by an
// xor butterfly in the accumulator precision. With nu_fmt < 0 no nu partial is formed.
template <typename VT, int K>
__device__ void spmv_vec(const DevSys& S, const VT* __restrict__ vals, const VT* xin, Rows R, int p1,
                         int nu_fmt, double& nd, float& nf) {
  using Acc = typename AccOf<VT>::type;
  constexpr int NG = kThreads / K;
  const int lane = threadIdx.x & (K - 1);
  const int grp = threadIdx.x / K;
  const unsigned mask = (K == 32) ? kFull : (((1u << K) - 1u) << ((threadIdx.x & 31) & ~(K - 1)));
  const int* __restrict__ rp = S.A.rp;
  const int* __restrict__ ci = S.A.ci;
  const bool scaled = row_scaled(p1);
  for (int row = R.r0 + grp; row < R.r1; row += NG) {
    const int e0 = __ldg(rp + row), e1 = __ldg(rp + row + 1);
    Acc acc = 0;
    for (int e = e0 + lane; e < e1; e += K) acc += to_acc(__ldg(vals + e)) * to_acc(xin[__ldg(ci + e)]);
#pragma unroll
    for (int o = K / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(mask, acc, o);
    if (lane == 0) {
      const double qv = store_q(S.q, row, acc, p1, scaled ? __ldg(S.A.rscale + row) : 1.f);
      if (nu_fmt >= 0) nu_term(S.p[row], qv, nu_fmt, nd, nf);
    }
  }
}

template <typename VT>
__device__ void spmv_dispatch_k(const DevSys& S, const VT* vals, const VT* xin, Rows R, int p1, int nu_fmt,
                                double& nd, float& nf) {
  switch (S.A.lanes[p1]) {
    case 1: spmv_vec<VT, 1>(S, vals, xin, R, p1, nu_fmt, nd, nf); break;
    case 2: spmv_vec<VT, 2>(S, vals, xin, R, p1, nu_fmt, nd, nf); break;
    case 4: spmv_vec<VT, 4>(S, vals, xin, R, p1, nu_fmt, nd, nf); break;
    case 8: spmv_vec<VT, 8>(S, vals, xin, R, p1, nu_fmt, nd, nf); break;
    case 16: spmv_vec<VT, 16>(S, vals, xin, R, p1, nu_fmt, nd, nf); break;
    default: spmv_vec<VT, 32>(S, vals, xin, R, p1, nu_fmt, nd, nf); break;
  }
}

// Phase A: q = fl_p1(A fl_p1(p)) for the CTA's rows, plus nu partials.
__device__ void spmv_rows(const DevSys& S, Rows R, int p1, int nu_fmt, double& nd, float& nf) {
  switch (p1) {
    case F64: spmv_dispatch_k<double>(S, S.A.v64, S.p, R, p1, nu_fmt, nd, nf); break;
    case F32: spmv_dispatch_k<float>(S, S.A.v32, (const float*)S.plow, R, p1, nu_fmt, nd, nf); break;
    case TF32: spmv_dispatch_k<float>(S, S.A.vtf, (const float*)S.plow, R, p1, nu_fmt, nd, nf); break;
    case F16: spmv_dispatch_k<__half>(S, S.A.v16, (const __half*)S.plow, R, p1, nu_fmt, nd, nf); break;
    case BF16: spmv_dispatch_k<__nv_bfloat16>(S, S.A.vbf, (const __nv_bfloat16*)S.plow, R, p1, nu_fmt, nd, nf); break;
    case F16R: spmv_dispatch_k<__half>(S, S.A.v16r, (const __half*)S.plow, R, p1, nu_fmt, nd, nf); break;
    default: spmv_dispatch_k<__nv_bfloat16>(S, S.A.vbfr, (const __nv_bfloat16*)S.plow, R, p1, nu_fmt, nd, nf); break;
  }
}

}  // namespace
}  // namespace mpcg
