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
  int g = 0, ng = 1;  // IC(0) substitutions: this CTA's index among the CTAs holding the system
};

// Read-only load of a stored value (the q52 byte through its unsigned char form).
template <typename VT>
__device__ __forceinline__ VT ldg_val(const VT* p) { return __ldg(p); }
template <>
__device__ __forceinline__ q52_t ldg_val<q52_t>(const q52_t* p) {
  return q52_t{__ldg(reinterpret_cast<const unsigned char*>(p))};
}

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

// Accumulator of a dot product term by term: fp64 for the fp64 format, otherwise a
// compensated fp32 pair of the products of rounded inputs (exact products for the 16-bit
// formats and tf32, FMA-corrected for fp32), i.e. the "Dot2" scheme of Ogita, Rump and
// Oishi (SIAM J. Sci. Comput. 26(6), 2005) carried out in fp32.
struct DotAcc {
  double d;
  float s, c;
};

__device__ __forceinline__ void dot_low(DotAcc& a, float x, float y, int f) {
  acc2(x, y, base_fmt(f) != F32, a.s, a.c);
}

// 2^e as fp64 (e in [-1022, 1023]).
__device__ __forceinline__ double pow2(int e) {
  return __longlong_as_double((long long)((unsigned long long)(e + 1023) << 52));
}

// p_i for the row's nu term: when nu's format is the product's (not row-scaled), fl_p3(p_i) is
// the element of p's low copy that the product reads anyway (fl_p1(p_i)), so the fp64 p is not
// read; otherwise p_i in fp64.
template <typename VT>
__device__ __forceinline__ double nu_input(const DevSys& S, const VT* xin, int row, int p1, int nu_fmt) {
  if (nu_fmt < 0) return 0.0;
  if constexpr (sizeof(VT) < 8) {
    if (nu_fmt != F64 && base_fmt(nu_fmt) == base_fmt(p1) && !row_scaled(p1)) return f2d(to_acc(xin[row]));
  }
  return S.p[row];
}

// Row finished with q_i = qf already rounded onto p1: stored in p1's storage; then the row's
// nu term fl_p3(p_i) fl_p3(q_i) (q_i includes the row scale 2^e_i of the row-scaled formats).
// `pi` = p_i in fp64 (read by the caller, ahead of the row when it can).
__device__ __forceinline__ void finish_row_low(const DevSys& S, int row, float qf, int p1, int nu_fmt, double pi,
                                               DotAcc& nu) {
  switch (store_of(p1)) {
    case ST_Q52: ((q52_t*)S.q)[row] = q52_from_exact(qf); break;
    case ST_HALF: ((__half*)S.q)[row] = __float2half_rn(qf); break;
    case ST_BF16: ((__nv_bfloat16*)S.q)[row] = __float2bfloat16_rn(qf); break;
    default: ((float*)S.q)[row] = qf; break;
  }
  if (nu_fmt < 0) return;
  const bool scaled = row_scaled(p1);
  if (nu_fmt == F64) {
    double qd = f2d(qf);
    if (scaled) qd = scale2(qd, __ldg(S.A.rexp + row));
    nu.d = fma(pi, qd, nu.d);
  } else {
    float b;
    if (scaled) b = round_d2f(scale2(f2d(qf), __ldg(S.A.rexp + row)), nu_fmt);
    else b = contains_fmt(nu_fmt, p1) ? qf : round_f2f(qf, nu_fmt);
    dot_low(nu, round_d2f(pi, nu_fmt), b, nu_fmt);
  }
}

// Row finished with an fp64 sum (fp64 product).
__device__ __forceinline__ void finish_row_64(const DevSys& S, int row, double tot, int nu_fmt, double pi,
                                              DotAcc& nu) {
  ((double*)S.q)[row] = tot;
  if (nu_fmt < 0) return;
  if (nu_fmt == F64) nu.d = fma(pi, tot, nu.d);
  else dot_low(nu, round_d2f(pi, nu_fmt), round_d2f(tot, nu_fmt), nu_fmt);
}

// Half the distance from fl_f(v) = r to its neighbours in format f, below and above
// (conservative at binade edges), as fp32; f is fp16, bf16, tf32 or q52.
__device__ __forceinline__ void half_gaps(float r, int f, float& below, float& above) {
  const int t = base_fmt(f) == BF16 ? 8 : base_fmt(f) == Q52 ? 3 : 11;
  const int emin = (base_fmt(f) == F16 || base_fmt(f) == Q52) ? -14 : -126;
  int e = (int)((__float_as_uint(r) >> 23) & 0xff) - 127;
  if (r == 0.f || e < emin) e = emin;
  const float ulp = __uint_as_float((unsigned)(e - t + 1 + 127) << 23);
  const float low = (fabsf(r) == __uint_as_float((unsigned)(e + 127) << 23) && e > emin) ? 0.5f * ulp : ulp;
  // moving toward zero from a power of two the spacing halves
  above = 0.5f * (r >= 0.f ? ulp : low);
  below = 0.5f * (r >= 0.f ? low : ulp);
}

// Products of one row slice accumulated by one lane.
// fp64 values: fp64 accumulation. fp32 (COMP = false): fp32 accumulation (the output format
// is fp32, so the accumulation error stays at its last place). fp16, bf16, tf32 and the
// row-scaled formats (COMP = true): the products are exact in fp32 and are summed with
// Knuth's TwoSum, so s + (the exact sum of the rounding errors t_i) equals the exact row sum;
// c accumulates the t_i in fp32 and a the |t_i|, which bounds the error of c by
// gamma_n a (Higham, "Accuracy and Stability of Numerical Algorithms", Sections 4.2 and 4.3).
// The pair (s, c) is rounded once onto the output format; only when the residual error
// bound reaches a rounding midpoint (about n u^2 sum |a_ij x_j| away, essentially never) is
// the row summed again in fp64 by lane 0.
template <typename VT, bool COMP>
struct RowAcc {
  float s = 0.f, c = 0.f, a = 0.f;
  __device__ __forceinline__ void add(VT av, VT xv) {
    const float af = to_acc(av), xf = to_acc(xv);
    if constexpr (COMP) {
      const float p = __fmul_rn(af, xf);
      float t;
      two_sum(s, p, s, t);
      c = __fadd_rn(c, t);
      a = __fadd_rn(a, fabsf(t));
    } else {
      s = fmaf(af, xf, s);
    }
  }
  template <int K>
  __device__ __forceinline__ void reduce(unsigned mask) {
#pragma unroll
    for (int o = K / 2; o > 0; o >>= 1) {
      const float so = __shfl_xor_sync(mask, s, o);
      if constexpr (COMP) {
        const float co = __shfl_xor_sync(mask, c, o), ao = __shfl_xor_sync(mask, a, o);
        float t;
        two_sum(s, so, s, t);
        c = __fadd_rn(__fadd_rn(c, co), t);
        a = __fadd_rn(__fadd_rn(a, ao), fabsf(t));
      } else {
        s += so;
      }
    }
  }
  // Adds another partial accumulation of the same row (the cross-warp step of a row summed
  // by the whole CTA).
  __device__ __forceinline__ void merge(double os, double oc, double oa) {
    if constexpr (COMP) {
      float t;
      two_sum(s, (float)os, s, t);
      c = __fadd_rn(__fadd_rn(c, (float)oc), t);
      a = __fadd_rn(__fadd_rn(a, (float)oa), fabsf(t));
    } else {
      s += (float)os;
    }
  }
  // Row sum rounded onto p1 (fp32 result). `exact` recomputes the row in fp64 when needed.
  template <class Exact>
  __device__ __forceinline__ float rounded(int p1, int len, Exact&& exact) const {
    if constexpr (!COMP) {
      return s;
    } else {
      // s is the plain fp32 sum: an infinite or NaN product leaves it infinite or NaN as the
      // fp64 sum would be (c, formed from infinite differences, is NaN then)
      if (!isfinite(s)) return s;
      float hi, lo;
      two_sum(s, c, hi, lo);  // hi + lo = s + c exactly
      if (!isfinite(hi)) return hi;
      const float r = round_pair(hi, lo, p1);
      if (!isfinite(r)) return r;
      float below, above;
      half_gaps(r, p1, below, above);
      // |exact - (s + c)| <= gamma_m a with m <= len + 2 log2(K) + 2 additions into c (plus
      // the cross-warp merges of a row summed by the whole CTA), inflated for the roundings of
      // a and d
      const float err = __fmul_rn(a, (float)(len + 32) * 1.2e-7f);
      const float d = __fadd_rn(__fsub_rn(hi, r), lo);
      const float slack = fabsf(d) * 1.2e-7f;
      if (d + err + slack < above && -d + err + slack < below) return r;
      return slow_round(p1, exact());
    }
  }
  __device__ static __noinline__ float slow_round(int p1, double v) { return round_d2f(v, p1); }
};

template <>
struct RowAcc<double, false> {
  double s = 0.0, c = 0.0, a = 0.0;  // c and a unused (fp64 accumulation)
  __device__ __forceinline__ void add(double av, double x) { s = fma(av, x, s); }
  __device__ __forceinline__ void merge(double os, double, double) { s += os; }
  template <int K>
  __device__ __forceinline__ void reduce(unsigned mask) {
#pragma unroll
    for (int o = K / 2; o > 0; o >>= 1) s += __shfl_xor_sync(mask, s, o);
  }
};

// fp64 sum of a row from value and column accessors (the exact fallback).
template <typename VT, class V, class Cf>
__device__ __forceinline__ double row_sum64(int rs, int re, V&& val, Cf&& col, const VT* xin) {
  double acc = 0.0;
  for (int e = rs; e < re; ++e) acc = fma(f2d(to_acc(val(e))), f2d(to_acc(xin[col(e)])), acc);
  return acc;
}

// Finishes a row of the product from its accumulator (lane 0 of the row's lanes). `extra`:
// additions into the accumulator beyond the row's own (partials merged from other threads).
template <typename VT, bool COMP, class V, class Cf>
__device__ __forceinline__ void finish_row(const DevSys& S, int row, int rs, int re, const RowAcc<VT, COMP>& acc, int p1,
                                           int nu_fmt, double pi, DotAcc& nu, V&& val, Cf&& col, const VT* xin,
                                           int extra = 0) {
  if constexpr (sizeof(VT) == 8) {
    finish_row_64(S, row, acc.s, nu_fmt, pi, nu);
  } else {
    const float qf = acc.rounded(p1, re - rs + extra, [&] { return row_sum64<VT>(rs, re, val, col, xin); });
    finish_row_low(S, row, qf, p1, nu_fmt, pi, nu);
  }
}

// ---- bulk copies into shared memory (cp.async.bulk + mbarrier) ------------------------

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// Global -> shared copy of `bytes` (multiple of 16, both addresses 16-byte aligned),
// completing on the mbarrier.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Shared-memory ring of the stream schedule: two stages of `stage_bytes`; in a stage the
// value region comes first (DevMatrix::tile_bytes[format] bytes), then the column region.
// `phase` (shared memory) holds the parity bit each stage's mbarrier waits for next; it
// persists across calls.
struct StreamCtx {
  unsigned char* buf;
  unsigned long long* bar;
  unsigned* phase;
  unsigned* err;
  int stage_bytes;
};

// Bounded wait on a stage's mbarrier; on timeout the device status word is set.
// (about two seconds at 2 GHz; a tile arrives within microseconds)
__device__ __forceinline__ void stage_wait(const StreamCtx& sc, int stage) {
  const unsigned par = (*sc.phase >> stage) & 1u;
  if (mbar_try_wait(sc.bar + stage, par)) return;
  const long long t0 = clock64();
  while (!mbar_try_wait(sc.bar + stage, par)) {
    if (clock64() - t0 > 4000000000ll) {
      if (sc.err) atomicCAS(sc.err, 0u, 1u);
      break;
    }
  }
}

// Rows longer than kLongRow nonzeros (power-law hubs) are summed by the whole CTA after its
// other rows: up to kLongMax of them per CTA range are queued in shared memory; beyond that
// the row's own lane group sums it as any other row.
constexpr int kLongRow = 1024;
constexpr int kLongMax = 32;
struct LongRows {
  int n;
  int rows[kLongMax];
  double part[3][kThreads / 32];
};
// Partial accumulations that the merge-path schedule hands from thread to thread.
struct MergeTails {
  int row[kThreads];
  double s[kThreads];
  float c[kThreads], a[kThreads];
};
// The product's shared memory: the long-row queue of schedules 0 and 2, or the partials of
// the merge-path schedule (never both in one call).
union SpmvShared {
  LongRows lr;
  MergeTails mt;
};
__device__ __forceinline__ SpmvShared& spmv_shared() {
  __shared__ SpmvShared u;
  return u;
}
__device__ __forceinline__ LongRows& long_rows() { return spmv_shared().lr; }
// Empties the CTA's queue (all threads of the CTA call it).
__device__ __forceinline__ void long_begin(LongRows& lr) {
  if (threadIdx.x == 0) lr.n = 0;
  __syncthreads();
}
// Queues a long row (one thread per row); false when the queue is full.
__device__ __forceinline__ bool long_queue(LongRows& lr, int row) {
  const int slot = atomicAdd(&lr.n, 1);
  if (slot < kLongMax) lr.rows[slot] = row;
  return slot < kLongMax;
}
// Sums the queued rows, each by all kThreads threads: a strided pass per thread, a warp
// butterfly, then thread 0 merges the warps' partials and finishes the row.
template <typename VT, bool COMP>
__device__ void long_pass(LongRows& lr, const DevSys& S, const VT* __restrict__ vals, const VT* xin, int p1,
                          int nu_fmt, DotAcc& nu) {
  const int* __restrict__ rp = S.A.rp;
  const int* __restrict__ ci = S.A.ci;
  __syncthreads();
  const int nl = lr.n < kLongMax ? lr.n : kLongMax;
  for (int i = 0; i < nl; ++i) {
    const int row = lr.rows[i];
    const int e0 = __ldg(rp + row), e1 = __ldg(rp + row + 1);
    RowAcc<VT, COMP> acc;
    for (int e = e0 + threadIdx.x; e < e1; e += kThreads) acc.add(ldg_val(vals + e), xin[__ldg(ci + e)]);
    acc.template reduce<32>(kFull);
    if ((threadIdx.x & 31) == 0) {
      lr.part[0][threadIdx.x >> 5] = acc.s;
      lr.part[1][threadIdx.x >> 5] = acc.c;
      lr.part[2][threadIdx.x >> 5] = acc.a;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < kThreads / 32; ++w) acc.merge(lr.part[0][w], lr.part[1][w], lr.part[2][w]);
      finish_row<VT, COMP>(S, row, e0, e1, acc, p1, nu_fmt, nu_input(S, xin, row, p1, nu_fmt), nu,
                           [&](int e) { return ldg_val(vals + e); }, [&](int e) { return __ldg(ci + e); }, xin);
    }
    __syncthreads();
  }
}

// Sub-warp vector CSR: K lanes per row, rows strided over the CTA, operands read from
// global memory. The K lane accumulators are combined by an xor butterfly. With nu_fmt < 0
// no nu partial is formed.
template <typename VT, bool COMP, int K>
__device__ void spmv_vec(const DevSys& S, const VT* __restrict__ vals, const VT* xin, Rows R, int p1,
                         int nu_fmt, DotAcc& nu) {
  constexpr int NG = kThreads / K;
  const int lane = threadIdx.x & (K - 1);
  const int grp = threadIdx.x / K;
  const unsigned mask = (K == 32) ? kFull : (((1u << K) - 1u) << ((threadIdx.x & 31) & ~(K - 1)));
  const int* __restrict__ rp = S.A.rp;
  const int* __restrict__ ci = S.A.ci;
  LongRows& lr = long_rows();
  long_begin(lr);
  for (int row = R.r0 + grp; row < R.r1; row += NG) {
    const int e0 = __ldg(rp + row), e1 = __ldg(rp + row + 1);
    if (e1 - e0 > kLongRow) {
      const bool queued = lane == 0 ? long_queue(lr, row) : false;
      if (__shfl_sync(mask, queued, (threadIdx.x & 31) & ~(K - 1))) continue;
    }
    RowAcc<VT, COMP> acc;
    for (int e = e0 + lane; e < e1; e += K) acc.add(ldg_val(vals + e), xin[__ldg(ci + e)]);
    acc.template reduce<K>(mask);
    if (lane == 0)
      finish_row<VT, COMP>(S, row, e0, e1, acc, p1, nu_fmt, nu_input(S, xin, row, p1, nu_fmt), nu,
                           [&](int e) { return ldg_val(vals + e); }, [&](int e) { return __ldg(ci + e); }, xin);
  }
  long_pass<VT, COMP>(lr, S, vals, xin, p1, nu_fmt, nu);
}

// Element k of a 16-byte word holding 16 / sizeof(VT) values (k known at compile time after
// unrolling, so the values stay in registers).
__device__ __forceinline__ unsigned word_of(const int4& q, int w) {
  return (unsigned)(w == 0 ? q.x : w == 1 ? q.y : w == 2 ? q.z : q.w);
}
template <typename VT>
__device__ __forceinline__ VT lane_of(const int4& q, int k);
template <>
__device__ __forceinline__ q52_t lane_of<q52_t>(const int4& q, int k) {
  return q52_t{(unsigned char)(word_of(q, k >> 2) >> (8 * (k & 3)))};
}
template <>
__device__ __forceinline__ __half lane_of<__half>(const int4& q, int k) {
  return __ushort_as_half((unsigned short)(word_of(q, k >> 1) >> (16 * (k & 1))));
}
template <>
__device__ __forceinline__ __nv_bfloat16 lane_of<__nv_bfloat16>(const int4& q, int k) {
  return __ushort_as_bfloat16((unsigned short)(word_of(q, k >> 1) >> (16 * (k & 1))));
}
template <>
__device__ __forceinline__ float lane_of<float>(const int4& q, int k) {
  return __uint_as_float(word_of(q, k));
}
template <>
__device__ __forceinline__ double lane_of<double>(const int4& q, int k) {
  return __hiloint2double((int)word_of(q, 2 * k + 1), (int)word_of(q, 2 * k));
}

// One thread per row with 16-byte loads: the row's column indices and values are read in
// aligned groups of G elements (G = 8 for 8- and 16-bit values, the 8-bit ones in one 8-byte
// load; 4 otherwise; group starts rounded
// down to a multiple of G, the arrays are padded so the last group stays in bounds), so a
// thread issues one load per 4 columns and per 16 bytes of values instead of one per
// element; elements of a group outside the row are skipped. Long rows go to the CTA queue.
// xs, xoff: where the gathers read x (element c at xs[c - xoff]): x itself, or its staged
// window in shared memory.
template <typename VT, bool COMP>
__device__ void spmv_vload(const DevSys& S, const VT* __restrict__ vals, const VT* xin, Rows R, int p1, int nu_fmt,
                           DotAcc& nu, const VT* xs = nullptr, int xoff = 0) {
  if (xs == nullptr) xs = xin;
  constexpr int G = sizeof(VT) <= 2 ? 8 : 4;
  constexpr int NV = G * (int)sizeof(VT) / 16;  // 16-byte value loads per group (0: one 8-byte load)
  const int* __restrict__ rp = S.A.rp;
  const int* __restrict__ ci = S.A.ci;
  // the row pointers and p_i of a thread's next row are loaded one row ahead
  int row = R.r0 + threadIdx.x;
  int ne0 = 0, ne1 = 0;
  double npi = 0.0;
  if (row < R.r1) {
    ne0 = __ldg(rp + row);
    ne1 = __ldg(rp + row + 1);
    npi = nu_input(S, xin, row, p1, nu_fmt);
  }
  LongRows& lr = long_rows();
  long_begin(lr);
  for (; row < R.r1; row += kThreads) {
    const int e0 = ne0, e1 = ne1;
    const double pi = npi;
    if (row + kThreads < R.r1) {
      ne0 = __ldg(rp + row + kThreads);
      ne1 = __ldg(rp + row + kThreads + 1);
      npi = nu_input(S, xin, row + kThreads, p1, nu_fmt);
    }
    if (e1 - e0 > kLongRow && long_queue(lr, row)) continue;
    RowAcc<VT, COMP> acc;
    for (int g = e0 & ~(G - 1); g < e1; g += G) {
      int c[G];
      VT v[G];
#pragma unroll
      for (int h = 0; h < G / 4; ++h) {
        const int4 cc = __ldg(reinterpret_cast<const int4*>(ci + g) + h);
        c[4 * h] = cc.x;
        c[4 * h + 1] = cc.y;
        c[4 * h + 2] = cc.z;
        c[4 * h + 3] = cc.w;
      }
      if constexpr (NV == 0) {  // eight one-byte values
        const int2 v2 = __ldg(reinterpret_cast<const int2*>(vals + g));
        const int4 vv = make_int4(v2.x, v2.y, 0, 0);
#pragma unroll
        for (int k = 0; k < G; ++k) v[k] = lane_of<VT>(vv, k);
      }
#pragma unroll
      for (int h = 0; h < NV; ++h) {
        const int4 vv = __ldg(reinterpret_cast<const int4*>(vals + g) + h);
        constexpr int PER = 16 / (int)sizeof(VT);
#pragma unroll
        for (int k = 0; k < PER; ++k) v[h * PER + k] = lane_of<VT>(vv, k);
      }
      VT xv[G];
#pragma unroll
      for (int j = 0; j < G; ++j)
        if (g + j >= e0 && g + j < e1) xv[j] = xs[c[j] - xoff];
#pragma unroll
      for (int j = 0; j < G; ++j)
        if (g + j >= e0 && g + j < e1) acc.add(v[j], xv[j]);
    }
    finish_row<VT, COMP>(S, row, e0, e1, acc, p1, nu_fmt, pi, nu, [&](int e) { return ldg_val(vals + e); },
                         [&](int e) { return __ldg(ci + e); }, xin);
  }
  long_pass<VT, COMP>(lr, S, vals, xin, p1, nu_fmt, nu);
}

// Staged stream CSR: the CTA's rows are cut into tiles of kThreads / K rows; the tile's
// contiguous value and column ranges are fetched into a two-stage shared-memory ring with
// bulk copies (16-byte aligned by rounding the byte ranges out; the matrix arrays are
// padded so the rounded ranges stay in bounds) while the previous tile is processed. K lanes
// per row read the row from shared memory (strided, conflict-free) and gather x.
template <typename VT, bool COMP, int K>
__device__ void spmv_stream(const DevSys& S, const VT* __restrict__ vals, const VT* xin, Rows R, int p1,
                            int nu_fmt, DotAcc& nu, const StreamCtx& sc) {
  constexpr int TR = kThreads / K;
  const int nrows = R.r1 - R.r0;
  const int ntiles = nrows > 0 ? (nrows + TR - 1) / TR : 0;
  if (ntiles == 0) return;
  const int lane = threadIdx.x & (K - 1);
  const int grp = threadIdx.x / K;
  const unsigned mask = (K == 32) ? kFull : (((1u << K) - 1u) << ((threadIdx.x & 31) & ~(K - 1)));
  const int* __restrict__ rp = S.A.rp;
  const int* __restrict__ ci = S.A.ci;
  const int vreg = S.A.tile_bytes[p1];
  auto issue = [&](int t, int stage) {
    const int ra = R.r0 + t * TR;
    const int rb = min(ra + TR, R.r1);
    const long long e0 = __ldg(rp + ra), e1 = __ldg(rp + rb);
    const long long vlo = (e0 * (long long)sizeof(VT)) & ~15ll, vhi = (e1 * (long long)sizeof(VT) + 15) & ~15ll;
    const long long clo = (e0 * 4) & ~15ll, chi = (e1 * 4 + 15) & ~15ll;
    unsigned char* base = sc.buf + (size_t)stage * sc.stage_bytes;
    fence_proxy_async();
    mbar_expect_tx(sc.bar + stage, (unsigned)((vhi - vlo) + (chi - clo)));
    bulk_g2s(base, (const char*)vals + vlo, (unsigned)(vhi - vlo), sc.bar + stage);
    bulk_g2s(base + vreg, (const char*)ci + clo, (unsigned)(chi - clo), sc.bar + stage);
  };
  if (threadIdx.x == 0) {
    issue(0, 0);
    if (ntiles > 1) issue(1, 1);
  }
  for (int t = 0; t < ntiles; ++t) {
    const int stage = t & 1;
    stage_wait(sc, stage);
    const int ra = R.r0 + t * TR;
    const int rb = min(ra + TR, R.r1);
    const int e0 = __ldg(rp + ra);
    const unsigned char* base = sc.buf + (size_t)stage * sc.stage_bytes;
    // element index of the first copied value (64-bit: e0 * 8 exceeds 2^31 for large matrices)
    const long long ev0 = (((long long)e0 * (long long)sizeof(VT)) & ~15ll) / (long long)sizeof(VT);
    const long long ec0 = (long long)(e0 & ~3);
    const VT* sv = (const VT*)base - ev0;
    const int* scol = (const int*)(base + vreg) - ec0;
    const int row = ra + grp;
    if (row < rb) {
      const int rs = __ldg(rp + row), re = __ldg(rp + row + 1);
      RowAcc<VT, COMP> acc;
      for (int e = rs + lane; e < re; e += K) acc.add(sv[e], xin[scol[e]]);
      acc.template reduce<K>(mask);
      if (lane == 0)
        finish_row<VT, COMP>(S, row, rs, re, acc, p1, nu_fmt, nu_input(S, xin, row, p1, nu_fmt), nu,
                             [&](int e) { return sv[e]; }, [&](int e) { return scol[e]; }, xin);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      *sc.phase ^= (1u << stage);
      if (t + 2 < ntiles) issue(t + 2, stage);
    }
    __syncthreads();
  }
}

// Merge-path CSR (Merrill and Garland, SC 2016): the CTA's rows and nonzeros form one merged
// list of row ends and products, and every thread takes an equal share of it, so a thread's
// work does not depend on row lengths (a power-law row is split over consecutive threads). A
// thread finds its start by a binary search along its diagonal of the merge, walks its share
// and finishes every row that begins and ends inside it; the partial accumulation of the row
// it leaves unfinished goes to shared memory, and the thread that ends a row begun before its
// share merges the partials of the threads before it, in thread order, with its own before
// rounding once (TwoSum pairs merge exactly, so the 16-bit, tf32 and q52 row sums stay
// correctly rounded).
template <typename VT, bool COMP>
__device__ void spmv_merge(const DevSys& S, const VT* __restrict__ vals, const VT* xin, Rows R, int p1, int nu_fmt,
                           DotAcc& nu) {
  const int* __restrict__ rp = S.A.rp;
  const int* __restrict__ ci = S.A.ci;
  MergeTails& mt = spmv_shared().mt;
  const int nrows = R.r1 - R.r0;
  if (nrows <= 0) return;  // the same for the whole CTA
  const int t = threadIdx.x;
  const int E0 = __ldg(rp + R.r0);
  const int nnz = __ldg(rp + R.r1) - E0;
  const long long total = (long long)nrows + nnz;
  const long long ipt = (total + kThreads - 1) / kThreads;
  const long long d0 = min((long long)t * ipt, total), d1 = min(d0 + ipt, total);
  // the point of the merge path on diagonal d0: lo row ends and d0 - lo products passed
  int lo = (int)max(d0 - (long long)nnz, 0ll), hi = (int)min(d0, (long long)nrows);
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if ((long long)(__ldg(rp + R.r0 + mid + 1) - E0) <= d0 - mid - 1) lo = mid + 1;
    else hi = mid;
  }
  int row = R.r0 + lo;
  int e = E0 + (int)(d0 - lo);
  int rs = row < R.r1 ? __ldg(rp + row) : 0, re = row < R.r1 ? __ldg(rp + row + 1) : 0;
  bool begun_here = e == rs;  // the row's first product (or its end, if empty) is in this share
  bool touched = false;       // products of the current row accumulated by this thread
  RowAcc<VT, COMP> acc, head;
  int head_row = -1;
  __syncthreads();  // the shared union may hold the long-row queue of an earlier product
  mt.row[t] = -1;
  for (long long d = d0; d < d1; ++d) {
    if (e < re) {
      acc.add(ldg_val(vals + e), xin[__ldg(ci + e)]);
      ++e;
      touched = true;
    } else {  // row `row` ends in this share
      if (begun_here) {
        finish_row<VT, COMP>(S, row, rs, re, acc, p1, nu_fmt, nu_input(S, xin, row, p1, nu_fmt), nu,
                             [&](int k) { return ldg_val(vals + k); }, [&](int k) { return __ldg(ci + k); }, xin);
      } else {
        head = acc;
        head_row = row;
      }
      acc = RowAcc<VT, COMP>();
      ++row;
      begun_here = true;
      touched = false;
      rs = re;
      if (row < R.r1) re = __ldg(rp + row + 1);
    }
  }
  if (touched) {  // the current row continues in the next share
    mt.row[t] = row;
    mt.s[t] = (double)acc.s;
    mt.c[t] = (float)acc.c;
    mt.a[t] = (float)acc.a;
  }
  __syncthreads();
  if (head_row >= 0) {
    int tf = t;
    while (tf > 0 && mt.row[tf - 1] == head_row) --tf;
    RowAcc<VT, COMP> m;
    int merged = 0;
    for (int u = tf; u < t; ++u, ++merged) m.merge(mt.s[u], mt.c[u], mt.a[u]);
    m.merge((double)head.s, (double)head.c, (double)head.a);
    const int hs = __ldg(rp + head_row), he = __ldg(rp + head_row + 1);
    finish_row<VT, COMP>(S, head_row, hs, he, m, p1, nu_fmt, nu_input(S, xin, head_row, p1, nu_fmt), nu,
                         [&](int k) { return ldg_val(vals + k); }, [&](int k) { return __ldg(ci + k); }, xin,
                         merged + 1);
  }
  __syncthreads();
}

// Staged x: the CTA's rows read x only within [lo, hi], the smallest and largest column of its
// rows (columns increase in every row); when that window fits the launch's shared-memory
// buffer, the CTA first copies it there with coalesced loads and the one-thread-per-row
// product gathers from shared memory; otherwise it gathers from x as the vector-load schedule.
template <typename VT, bool COMP>
__device__ void spmv_xstage(const DevSys& S, const VT* __restrict__ vals, const VT* xin, Rows R, int p1, int nu_fmt,
                            DotAcc& nu, const StreamCtx& sc) {
  __shared__ int win[2];
  const int* __restrict__ rp = S.A.rp;
  const int* __restrict__ ci = S.A.ci;
  if (threadIdx.x == 0) {
    win[0] = 0x7fffffff;
    win[1] = -1;
  }
  __syncthreads();
  int lo = 0x7fffffff, hi = -1;
  for (int r = R.r0 + (int)threadIdx.x; r < R.r1; r += kThreads) {
    const int e0 = __ldg(rp + r), e1 = __ldg(rp + r + 1);
    if (e1 > e0) {
      lo = min(lo, __ldg(ci + e0));
      hi = max(hi, __ldg(ci + e1 - 1));
    }
  }
  if (hi >= 0) {
    atomicMin(&win[0], lo);
    atomicMax(&win[1], hi);
  }
  __syncthreads();
  const int wlo = win[0], whi = win[1];
  const long long cap = 2LL * sc.stage_bytes / (long long)sizeof(VT);
  if (whi < 0 || (long long)whi - wlo + 1 > cap) {
    __syncthreads();  // win is read by every thread before the next call resets it
    spmv_vload<VT, COMP>(S, vals, xin, R, p1, nu_fmt, nu);
    return;
  }
  VT* sx = reinterpret_cast<VT*>(sc.buf);
  for (int k = threadIdx.x; k <= whi - wlo; k += kThreads) sx[k] = xin[wlo + k];
  __syncthreads();
  spmv_vload<VT, COMP>(S, vals, xin, R, p1, nu_fmt, nu, sx, wlo);
  __syncthreads();  // the buffer and win are reused by the next call
}

template <typename VT, bool COMP>
__device__ void spmv_dispatch_k(const DevSys& S, const VT* vals, const VT* xin, Rows R, int p1, int nu_fmt,
                                DotAcc& nu, const StreamCtx* sc) {
  if (S.A.sched[p1] == SCHED_VLOAD) {
    spmv_vload<VT, COMP>(S, vals, xin, R, p1, nu_fmt, nu);
    return;
  }
  if (S.A.sched[p1] == SCHED_MERGE) {
    spmv_merge<VT, COMP>(S, vals, xin, R, p1, nu_fmt, nu);
    return;
  }
  if (S.A.sched[p1] == SCHED_XSTAGE) {
    if (sc) spmv_xstage<VT, COMP>(S, vals, xin, R, p1, nu_fmt, nu, *sc);
    else spmv_vload<VT, COMP>(S, vals, xin, R, p1, nu_fmt, nu);
    return;
  }
  if (sc && S.A.sched[p1] == SCHED_STREAM) {
    switch (S.A.lanes[p1]) {
      case 1: spmv_stream<VT, COMP, 1>(S, vals, xin, R, p1, nu_fmt, nu, *sc); return;
      case 2: spmv_stream<VT, COMP, 2>(S, vals, xin, R, p1, nu_fmt, nu, *sc); return;
      default: spmv_stream<VT, COMP, 4>(S, vals, xin, R, p1, nu_fmt, nu, *sc); return;
    }
  }
  switch (S.A.lanes[p1]) {
    case 1: spmv_vec<VT, COMP, 1>(S, vals, xin, R, p1, nu_fmt, nu); break;
    case 2: spmv_vec<VT, COMP, 2>(S, vals, xin, R, p1, nu_fmt, nu); break;
    case 4: spmv_vec<VT, COMP, 4>(S, vals, xin, R, p1, nu_fmt, nu); break;
    case 8: spmv_vec<VT, COMP, 8>(S, vals, xin, R, p1, nu_fmt, nu); break;
    case 16: spmv_vec<VT, COMP, 16>(S, vals, xin, R, p1, nu_fmt, nu); break;
    default: spmv_vec<VT, COMP, 32>(S, vals, xin, R, p1, nu_fmt, nu); break;
  }
}

// Phase A: q = fl_p1(A fl_p1(p)) for the CTA's rows, plus nu partials. `sc` is the
// shared-memory ring of the stream schedule (nullptr when the launch has none).
__device__ void spmv_rows(const DevSys& S, Rows R, int p1, int nu_fmt, DotAcc& nu, const StreamCtx* sc) {
  switch (p1) {
    case F64:  // the single-reduction iteration multiplies u, kept in plow in fp64
      spmv_dispatch_k<double, false>(S, S.A.v64, S.sv ? (const double*)S.plow : S.p, R, p1, nu_fmt, nu, sc);
      break;
    case F32: spmv_dispatch_k<float, false>(S, S.A.v32, (const float*)S.plow, R, p1, nu_fmt, nu, sc); break;
    case TF32: spmv_dispatch_k<float, true>(S, S.A.vtf, (const float*)S.plow, R, p1, nu_fmt, nu, sc); break;
    case F16: spmv_dispatch_k<__half, true>(S, S.A.v16, (const __half*)S.plow, R, p1, nu_fmt, nu, sc); break;
    case BF16: spmv_dispatch_k<__nv_bfloat16, true>(S, S.A.vbf, (const __nv_bfloat16*)S.plow, R, p1, nu_fmt, nu, sc);
      break;
    case F16R: spmv_dispatch_k<__half, true>(S, S.A.v16r, (const __half*)S.plow, R, p1, nu_fmt, nu, sc); break;
    case Q52: spmv_dispatch_k<q52_t, true>(S, S.A.v8, (const q52_t*)S.plow, R, p1, nu_fmt, nu, sc); break;
    default: spmv_dispatch_k<__nv_bfloat16, true>(S, S.A.vbfr, (const __nv_bfloat16*)S.plow, R, p1, nu_fmt, nu, sc);
      break;
  }
}

}  // namespace
}  // namespace mpcg
