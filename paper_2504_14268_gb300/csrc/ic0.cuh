// Incomplete Cholesky IC(0) in fp32: the level-ordered substitutions.
//
// Section 5 preconditions with an incomplete factorization held in fp32 (the paper's
// p_fixed); for SPD matrices its symmetric zero-fill form is M = L L^T with L on the
// pattern of A's lower triangle. Applying M^-1 is two triangular substitutions, each a
// chain of row-to-row dependencies. They run inside the solver kernels without grid
// barriers: rows are taken in the level order of each substitution (computed with the
// factor), every row publishes its value with a mark in one 64-bit word, and a row waits until
// the rows it reads are marked. Systems whose levels are narrow are substituted by one CTA,
// level by level with CTA barriers. Every wait is bounded in time and gives up when the
// launch's status word reports an error.
#pragma once
#include "internal.h"
#include "spmv.cuh"

namespace mpcg {

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned ld_relaxed(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// Waits until *mark >= target. False when the wait exceeded `limit` clock cycles (the
// timeout bit is set in *err) or *err was already non-zero.
static __device__ __noinline__ bool ic_wait_slow(const unsigned* mark, unsigned target, unsigned* err, unsigned tbit,
                                          long long limit) {
  const long long t0 = clock64();
  unsigned spins = 0;
  while (ld_acquire(mark) < target) {
    if ((++spins & 63u) == 0u) {
      if (*(volatile unsigned*)err != 0u) return false;
      if (clock64() - t0 > limit) {
        atomicOr(err, tbit);
        return false;
      }
    }
    __nanosleep(32);
  }
  return true;
}

__device__ __forceinline__ unsigned long long ld_relaxed64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_relaxed64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// A row's published value: the fp32 bits in the low word, its mark in the high word. One
// 64-bit access carries both, so a reader that sees the mark has the value with it: no
// fences, no second load.
__device__ __forceinline__ unsigned long long ic_word(float v, unsigned mark) {
  return ((unsigned long long)mark << 32) | __float_as_uint(v);
}
__device__ __forceinline__ float ic_value(unsigned long long w) { return __uint_as_float((unsigned)w); }
__device__ __forceinline__ unsigned ic_mark(unsigned long long w) { return (unsigned)(w >> 32); }

// Both substitutions by one CTA, level by level (ic_apply for systems whose levels hold at
// most half a CTA's threads' worth of rows). Row i of a level waits (bounded) only for the mark
// of its own fl32(r_i), published by the CTA holding the row; the values of earlier levels were
// stored by this CTA before the barrier that ends their level.
template <class F>
__device__ __noinline__ void ic_levels_cta(const DevSys& S, unsigned ep, unsigned* err, unsigned tbit,
                                           long long limit, bool bad, F&& consume) {
  const int* __restrict__ rp = S.A.rp;
  const int* __restrict__ ci = S.A.ci;
  const float* __restrict__ Lf = S.A.icf;
  const int* __restrict__ dp = S.A.icd;
  unsigned long long* W = S.icw;
  const unsigned tr = 3u * ep + 1u, tf = 3u * ep + 2u, tb = 3u * ep + 3u;
  for (int l = 0; l < S.A.nlevf; ++l) {
    const int a = __ldg(S.A.icof + l), b = __ldg(S.A.icof + l + 1);
    for (int x = a + (int)threadIdx.x; x < b; x += kThreads) {
      const int i = __ldg(S.A.icpf + x);
      unsigned long long w = ld_relaxed64(W + i);
      if (ic_mark(w) < tr && !bad) {
        const long long t0 = clock64();
        unsigned spins = 0;
        while (ic_mark(w = ld_relaxed64(W + i)) < tr) {
          __nanosleep(64);
          if ((++spins & 63u) == 0u) {
            if (*(volatile unsigned*)err != 0u) break;
            if (clock64() - t0 > limit) {
              atomicOr(err, tbit);
              break;
            }
          }
        }
      }
      float s = ic_value(w);
      const int e1 = __ldg(dp + i);
      for (int e = __ldg(rp + i); e < e1; ++e)
        s = __fsub_rn(s, __fmul_rn(__ldg(Lf + e), ic_value(W[__ldg(ci + e)])));
      W[i] = ic_word(__fdiv_rn(s, __ldg(Lf + e1)), tf);
    }
    __syncthreads();
  }
  for (int l = 0; l < S.A.nlevb; ++l) {
    const int a = __ldg(S.A.icob + l), b = __ldg(S.A.icob + l + 1);
    for (int x = a + (int)threadIdx.x; x < b; x += kThreads) {
      const int i = __ldg(S.A.icpb + x);
      const int di = __ldg(dp + i), e1 = __ldg(rp + i + 1);
      float s = ic_value(W[i]);  // y_i
      for (int e = di + 1; e < e1; ++e) s = __fsub_rn(s, __fmul_rn(__ldg(Lf + e), ic_value(W[__ldg(ci + e)])));
      const float wv = __fdiv_rn(s, __ldg(Lf + di));
      W[i] = ic_word(wv, tb);
      consume(i, __ldcg(S.r + i), (double)wv);
    }
    __syncthreads();
  }
}

// Threads of a substitution: about two levels' worth of rows (whole warps), at most the
// group's threads. Thread t of the group takes the positions t, t + T, t + 2T, ... of the
// level order, so that every thread works within a few levels of the front.
__device__ __forceinline__ int ic_threads(int width, int ng) {
  const int want = ((2 * width + 31) / 32) * 32;
  const int have = ng * kThreads;
  return want < 32 ? 32 : (want < have ? want : have);
}

// Row bounds of a substitution: the entries [ea, eb) the row's sum reads and the diagonal's
// position (forward: the lower entries, the diagonal after them; backward: the upper ones,
// the diagonal before them).
template <bool BACK>
__device__ __forceinline__ void ic_bounds(const DevSys& S, int i, int& ea, int& eb, int& diag) {
  if constexpr (BACK) {
    diag = __ldg(S.A.icd + i);
    ea = diag + 1;
    eb = __ldg(S.A.rp + i + 1);
  } else {
    ea = __ldg(S.A.rp + i);
    eb = __ldg(S.A.icd + i);
    diag = eb;
  }
}

// One substitution (BACK: L^T w = y, else L y = fl32(r)) by threads 0..T-1 of the group, thread
// gt taking the positions gt, gt + T, ... of the level order `order`. A row waits for its own
// word to carry own_mark (fl32(r_i), or y_i), for the words it reads to carry in_mark, and
// publishes its value with in_mark (forward) or its w with in_mark (backward; both the mark of
// this sweep's outputs). The warp advances in rounds; in a round every lane issues at most one
// batch of independent loads (the next row's bounds two rows ahead, its own word, eight columns
// and factor values, or the eight words those columns name) and uses what it loaded in the round
// before, so a round lasts about one memory round trip whatever the lanes are doing.
template <bool BACK, class F>
__device__ __forceinline__ void ic_sweep(const DevSys& S, int gt, int T, const int* __restrict__ order,
                                         unsigned own_mark, unsigned in_mark, unsigned* err, unsigned tbit,
                                         long long limit, bool& bad, F&& consume) {
  const int* __restrict__ ci = S.A.ci;
  const float* __restrict__ Lf = S.A.icf;
  unsigned long long* W = S.icw;
  const int n = S.A.n;
  const int cnt = gt < T ? (n - gt + T - 1) / T : 0;
  int m = 0;
  int i = 0, ea = 0, eb = 0, diag = 0;  // the current row
  int i1 = 0, a1 = 0, b1 = 0, d1 = 0;   // the next row (its bounds loaded while the current one runs)
  int i2 = 0;                           // the row after it (its index)
  if (cnt > 0) {
    i = __ldg(order + gt);
    ic_bounds<BACK>(S, i, ea, eb, diag);
  }
  if (cnt > 1) i1 = __ldg(order + gt + T);
  if (cnt > 2) i2 = __ldg(order + gt + 2 * T);
  int stage = 0;  // 0: start the row, 1: own word loaded, 2: words loaded, 3: columns loaded
  unsigned long long w0 = 0ull;
  unsigned long long wv[8];
  int c[8];
  float lv[8];
  int nb = 0, kd = 0;  // entries in the batch, entries of it already summed
  float s = 0.f, ldiag = 1.f;
  double rv = 0.0;
  unsigned rounds = 0, nap = 0;
  long long t_last = clock64();
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    wv[k] = 0ull;
    c[k] = 0;
    lv[k] = 0.f;
  }
  while (__any_sync(kFull, m < cnt)) {
    bool moved = false;
    if (m < cnt) {
      if (stage == 0) {  // the row's own word, its first columns and factor values, its diagonal
        w0 = ld_relaxed64(W + i);
        nb = min(8, eb - ea);
        kd = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k)
          if (k < nb) {
            c[k] = __ldg(ci + ea + k);
            lv[k] = __ldg(Lf + ea + k);
          }
        ldiag = __ldg(Lf + diag);
        if (m + 1 < cnt) ic_bounds<BACK>(S, i1, a1, b1, d1);
        stage = 1;
        moved = true;
      } else if (stage == 1) {  // own word: start the sum, or look again
        if (bad || ic_mark(w0) >= own_mark) {
          s = ic_value(w0);
          // backward: r_i was written before fl32(r_i) was published, which came before y_i
          if constexpr (BACK) rv = __ldcg(S.r + i);
#pragma unroll
          for (int k = 0; k < 8; ++k)
            if (k < nb) wv[k] = ld_relaxed64(W + c[k]);
          stage = 2;
          moved = true;
        } else {
          w0 = ld_relaxed64(W + i);
        }
      } else if (stage == 3) {  // columns of the next batch loaded: load their words
#pragma unroll
        for (int k = 0; k < 8; ++k)
          if (k < nb) wv[k] = ld_relaxed64(W + c[k]);
        stage = 2;
        moved = true;
      } else {  // stage 2: sum the ready words in order
        bool stop = false;
#pragma unroll
        for (int k = 0; k < 8; ++k)
          if (k >= kd && k < nb && !stop) {
            if (bad || ic_mark(wv[k]) >= in_mark) {
              s = __fsub_rn(s, __fmul_rn(lv[k], ic_value(wv[k])));
              kd = k + 1;
              moved = true;
            } else {
              stop = true;
            }
          }
        if (kd == nb) {
          ea += nb;
          if (ea == eb) {  // the row is done
            const float v = __fdiv_rn(s, ldiag);
            st_relaxed64(W + i, ic_word(v, in_mark));
            if constexpr (BACK) consume(i, rv, (double)v);
            ++m;
            i = i1;
            ea = a1;
            eb = b1;
            diag = d1;
            i1 = i2;
            if (m + 2 < cnt) i2 = __ldg(order + gt + (m + 2) * T);
            stage = 0;
            moved = true;
          } else {  // the next batch of columns and factor values
            nb = min(8, eb - ea);
            kd = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k)
              if (k < nb) {
                c[k] = __ldg(ci + ea + k);
                lv[k] = __ldg(Lf + ea + k);
              }
            stage = 3;
            moved = true;
          }
        } else {  // look again at the words not ready yet
#pragma unroll
          for (int k = 0; k < 8; ++k)
            if (k >= kd && k < nb) wv[k] = ld_relaxed64(W + c[k]);
        }
      }
    }
    if (__any_sync(kFull, moved)) {
      t_last = clock64();
      nap = 0;
    } else {
      // a round without progress in the whole warp: back off briefly, check the status word
      // now and then, and the time since the warp last moved
      nap = nap ? min(2u * nap, 256u) : 32u;
      __nanosleep(nap);
      if ((++rounds & 63u) == 0u) {
        if (*(volatile unsigned*)err != 0u) {
          bad = true;
        } else if (clock64() - t_last > limit) {
          atomicOr(err, tbit);
          bad = true;
        }
      }
    }
  }
}

// w = M^-1 fl32(r) for one application with epoch `ep`, run by the ng CTAs that hold rows of
// the system (this CTA is number R.g; R is its own row range). Marks in the high word of each
// row's 64-bit word: 3 ep + 1 when fl32(r_i) is published (by the CTA holding row i, which
// wrote r_i), 3 ep + 2 when y_i is, 3 ep + 3 when w_i is; the words start at 0 for a launch and
// the marks only grow. Both substitutions run in fp32 with each row's sum over its stored
// columns in increasing order and one correctly rounded division by l_ii, so the result
// equals a sequential evaluation bit for bit. The rows are taken in level order (icpf for
// L y = r, icpb for L^T w = y): a row's inputs lie in lower levels, hence at earlier
// positions, so the earliest unfinished position always has its inputs and the group, resident
// by the cooperative launch, makes progress; the threads near the front are the only ones
// waiting, which keeps the polling small. y and w share the word: row i overwrites y_i with
// w_i only after every row that reads y_i has published its w (they are exactly the rows its
// backward step waits on, the pattern being symmetric). consume(i, r_i, w_i) runs once per row
// on the thread that finishes w_i. Starts and ends with a CTA barrier.
//
// Waiting never diverges inside a warp: a warp loops as a whole; in each round every lane
// extends its current row's sum over the inputs that are ready, finishing the row when all
// are, and the others try again in the next round. (A lane spinning alone would hold its
// warp at the reconvergence point while the rows it waits for may belong to lanes of that
// same warp.) A warp that sees no progress for `limit` cycles sets the timeout bit; after
// any error the rows are finished without waiting and the host reports the error.
template <class F>
__device__ __forceinline__ void ic_apply(const DevSys& S, Rows R, unsigned ep, unsigned* err, unsigned tbit,
                                         long long limit, F&& consume) {
  unsigned long long* W = S.icw;
  const unsigned tr = 3u * ep + 1u, tf = 3u * ep + 2u, tb = 3u * ep + 3u;
  // publish fl32(r_i) of this CTA's rows (r written by this CTA's threads before the barrier)
  __threadfence();
  __syncthreads();
  for (int i = R.r0 + (int)threadIdx.x; i < R.r1; i += kThreads)
    st_relaxed64(W + i, ic_word(__double2float_rn(S.r[i]), tr));
  bool bad = *(volatile unsigned*)err != 0u;
  if (ic_threads(S.A.icwf, R.ng) <= kThreads && ic_threads(S.A.icwb, R.ng) <= kThreads) {
    // levels of at most half a CTA: the group's first CTA alone runs both substitutions,
    // level by level with a CTA barrier between levels (the values of earlier levels come from
    // this CTA's own stores); only fl32(r_i) of other CTAs' rows is waited for
    __syncthreads();
    if (R.g == 0) ic_levels_cta(S, ep, err, tbit, limit, bad, consume);
    __syncthreads();
    return;
  }
  const int gt = R.g * kThreads + (int)threadIdx.x;  // this thread in the group
  ic_sweep<false>(S, gt, ic_threads(S.A.icwf, R.ng), S.A.icpf, tr, tf, err, tbit, limit, bad, consume);
  ic_sweep<true>(S, gt, ic_threads(S.A.icwb, R.ng), S.A.icpb, tf, tb, err, tbit, limit, bad, consume);
  __syncthreads();
}

}  // namespace mpcg
