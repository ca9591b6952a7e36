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

// nu term of row i: fl_p3(p_i) fl_p3(q_i), products of rounded inputs accumulated in fp64
// (exact for every format of the set), the sum rounded to p3 by the caller.
__device__ __forceinline__ void nu_term(double pi, double qi, int p3, double& nd) {
  nd = fma(round_fmt(pi, p3), round_fmt(qi, p3), nd);
}

// 2^e as fp64 (e in [-1022, 1023]).
__device__ __forceinline__ double pow2(int e) {
  return __longlong_as_double((long long)((unsigned long long)(e + 1023) << 52));
}

// Rounds the row sum onto the product's format p1 (one rounding), stores it in q and
// returns the row's value of q (times 2^e_i for the row-scaled formats) as fp64.
__device__ __forceinline__ double store_q(void* q, int i, double tot, int p1, double scale) {
  const double r = round_fmt(tot, p1);
  switch (store_of(p1)) {
    case ST_HALF: store_exact((__half*)q, i, r); break;
    case ST_BF16: store_exact((__nv_bfloat16*)q, i, r); break;
    case ST_FLOAT: store_exact((float*)q, i, r); break;
    default: store_exact((double*)q, i, r); break;
  }
  return r * scale;
}

// s + t = a + b exactly (Knuth's TwoSum), fp32, without contraction.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& t) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  t = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Sub-warp vector CSR: K lanes per row, rows strided over the CTA.
// fp64 values: fp64 accumulation. Lower formats: the products of the rounded inputs are
// summed with a compensated fp32 accumulator (sum and error term, TwoSum; fp32 products
// carry their FMA error term too), i.e. the dot product "Dot2" of Ogita, Rump and Oishi
// (SIAM J. Sci. Comput. 2005) in fp32, so the row sum is accurate to about 2^-48 and its
// single rounding onto p1 matches a wide-accumulator sum. The K lane results are combined
// by an xor butterfly of (sum, error) pairs. With nu_fmt < 0 no nu partial is formed.
template <typename VT, int K>
__device__ void spmv_vec(const DevSys& S, const VT* __restrict__ vals, const VT* xin, Rows R, int p1,
                         int nu_fmt, double& nd) {
  constexpr int NG = kThreads / K;
  const int lane = threadIdx.x & (K - 1);
  const int grp = threadIdx.x / K;
  const unsigned mask = (K == 32) ? kFull : (((1u << K) - 1u) << ((threadIdx.x & 31) & ~(K - 1)));
  const int* __restrict__ rp = S.A.rp;
  const int* __restrict__ ci = S.A.ci;
  const bool scaled = row_scaled(p1);
  const short* __restrict__ rexp = S.A.rexp;
  for (int row = R.r0 + grp; row < R.r1; row += NG) {
    const int e0 = __ldg(rp + row), e1 = __ldg(rp + row + 1);
    double tot;
    if constexpr (sizeof(VT) == 8) {
      double acc = 0.0;
      for (int e = e0 + lane; e < e1; e += K) acc = fma(__ldg(vals + e), xin[__ldg(ci + e)], acc);
#pragma unroll
      for (int o = K / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(mask, acc, o);
      tot = acc;
    } else {
      float sum = 0.f, err = 0.f;
      for (int e = e0 + lane; e < e1; e += K) {
        const float a = to_acc(__ldg(vals + e)), xv = to_acc(xin[__ldg(ci + e)]);
        const float pr = __fmul_rn(a, xv);
        float t;
        two_sum(sum, pr, sum, t);
        if constexpr (sizeof(VT) == 4) t = __fadd_rn(t, __fmaf_rn(a, xv, -pr));
        err = __fadd_rn(err, t);
      }
#pragma unroll
      for (int o = K / 2; o > 0; o >>= 1) {
        const float s2 = __shfl_xor_sync(mask, sum, o), e2 = __shfl_xor_sync(mask, err, o);
        float t;
        two_sum(sum, s2, sum, t);
        err = __fadd_rn(__fadd_rn(err, e2), t);
      }
      // an infinite or NaN partial (format overflow) makes the error term meaningless
      tot = isfinite(sum) ? (double)sum + (double)err : (double)sum;
    }
    if (lane == 0) {
      const double qv = store_q(S.q, row, tot, p1, scaled ? pow2(__ldg(rexp + row)) : 1.0);
      if (nu_fmt >= 0) nu_term(S.p[row], qv, nu_fmt, nd);
    }
  }
}

template <typename VT>
__device__ void spmv_dispatch_k(const DevSys& S, const VT* vals, const VT* xin, Rows R, int p1, int nu_fmt,
                                double& nd) {
  switch (S.A.lanes[p1]) {
    case 1: spmv_vec<VT, 1>(S, vals, xin, R, p1, nu_fmt, nd); break;
    case 2: spmv_vec<VT, 2>(S, vals, xin, R, p1, nu_fmt, nd); break;
    case 4: spmv_vec<VT, 4>(S, vals, xin, R, p1, nu_fmt, nd); break;
    case 8: spmv_vec<VT, 8>(S, vals, xin, R, p1, nu_fmt, nd); break;
    case 16: spmv_vec<VT, 16>(S, vals, xin, R, p1, nu_fmt, nd); break;
    default: spmv_vec<VT, 32>(S, vals, xin, R, p1, nu_fmt, nd); break;
  }
}

// Phase A: q = fl_p1(A fl_p1(p)) for the CTA's rows, plus nu partials.
__device__ void spmv_rows(const DevSys& S, Rows R, int p1, int nu_fmt, double& nd) {
  switch (p1) {
    case F64: spmv_dispatch_k<double>(S, S.A.v64, S.p, R, p1, nu_fmt, nd); break;
    case F32: spmv_dispatch_k<float>(S, S.A.v32, (const float*)S.plow, R, p1, nu_fmt, nd); break;
    case TF32: spmv_dispatch_k<float>(S, S.A.vtf, (const float*)S.plow, R, p1, nu_fmt, nd); break;
    case F16: spmv_dispatch_k<__half>(S, S.A.v16, (const __half*)S.plow, R, p1, nu_fmt, nd); break;
    case BF16: spmv_dispatch_k<__nv_bfloat16>(S, S.A.vbf, (const __nv_bfloat16*)S.plow, R, p1, nu_fmt, nd); break;
    case F16R: spmv_dispatch_k<__half>(S, S.A.v16r, (const __half*)S.plow, R, p1, nu_fmt, nd); break;
    default: spmv_dispatch_k<__nv_bfloat16>(S, S.A.vbfr, (const __nv_bfloat16*)S.plow, R, p1, nu_fmt, nd); break;
  }
}

}  // namespace
}  // namespace mpcg
