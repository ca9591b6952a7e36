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

// Continues the row sum s -= l_e v_col(e) over e = ea, ea + 1, ... < eb in order, eight
// words per memory round trip, as long as the rows read carry a mark >= target. True when
// the sum is complete; otherwise ea and s hold the progress for the next attempt (the order
// of the terms never changes). A retry first reads only the word it stopped at, so that
// waiting rows add one load per round to the lines being polled.
__device__ __forceinline__ bool ic_accumulate(const int* __restrict__ ci, const float* __restrict__ Lf,
                                              const unsigned long long* W, int& ea, int eb, unsigned target,
                                              float& s, bool retry) {
  if (retry && ea < eb) {
    const unsigned long long w = ld_relaxed64(W + __ldg(ci + ea));
    if (ic_mark(w) < target) return false;
    s = __fsub_rn(s, __fmul_rn(__ldg(Lf + ea), ic_value(w)));
    ++ea;
  }
  while (ea < eb) {
    unsigned long long w[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) w[u] = ea + u < eb ? ld_relaxed64(W + __ldg(ci + ea + u)) : 0ull;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      if (ea >= eb) return true;
      if (ic_mark(w[u]) < target) return false;
      s = __fsub_rn(s, __fmul_rn(__ldg(Lf + ea), ic_value(w[u])));
      ++ea;
    }
  }
  return true;
}

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
  const int* __restrict__ rp = S.A.rp;
  const int* __restrict__ ci = S.A.ci;
  const float* __restrict__ Lf = S.A.icf;
  const int* __restrict__ dp = S.A.icd;
  unsigned long long* W = S.icw;
  const int n = S.A.n;
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
  unsigned rounds = 0, nap = 0;
  long long t_last = clock64();
  // a round without progress in the whole warp: back off briefly, check the status word now
  // and then, and the time since the warp last moved
  auto idle = [&]() {
    nap = nap ? min(2u * nap, 256u) : 32u;
    __nanosleep(nap);
    if ((++rounds & 63u) != 0u) return;
    if (*(volatile unsigned*)err != 0u) {
      bad = true;
    } else if (clock64() - t_last > limit) {
      atomicOr(err, tbit);
      bad = true;
    }
  };
  // forward: L y = fl32(r), positions gt, gt + T, ... of the forward level order
  {
    const int T = ic_threads(S.A.icwf, R.ng);
    const int cnt = gt < T ? (n - gt + T - 1) / T : 0;
    int m = 0, ea = 0, eb = 0, i = 0;
    float s = 0.f;
    int stage = 0;  // 0: new row, 1: waiting for fl32(r_i), 2: summing
    while (__any_sync(kFull, m < cnt)) {
      bool moved = false;
      if (m < cnt) {
        if (stage == 0) {
          i = __ldg(S.A.icpf + gt + m * T);
          ea = __ldg(rp + i);
          eb = __ldg(dp + i);
          stage = 1;
        }
        if (stage == 1) {
          const unsigned long long w = ld_relaxed64(W + i);
          if (bad || ic_mark(w) >= tr) {
            s = ic_value(w);
            stage = 2;
            moved = true;
          }
        }
        if (stage == 2) {
          const int e_before = ea;
          if (ic_accumulate(ci, Lf, W, ea, eb, bad ? 0u : tf, s, !moved)) {
            st_relaxed64(W + i, ic_word(__fdiv_rn(s, __ldg(Lf + eb)), tf));
            ++m;
            stage = 0;
            moved = true;
          } else {
            moved = moved || ea != e_before;
          }
        }
      }
      if (__any_sync(kFull, moved)) {
        t_last = clock64();
        nap = 0;
      } else {
        idle();
      }
    }
  }
  // backward: L^T w = y, positions gt, gt + T, ... of the backward level order
  {
    const int T = ic_threads(S.A.icwb, R.ng);
    const int cnt = gt < T ? (n - gt + T - 1) / T : 0;
    int m = 0, ea = 0, eb = 0, di = 0, i = 0;
    float s = 0.f;
    int stage = 0;  // 0: new row, 1: waiting for y_i, 2: summing
    while (__any_sync(kFull, m < cnt)) {
      bool moved = false;
      if (m < cnt) {
        if (stage == 0) {
          i = __ldg(S.A.icpb + gt + m * T);
          di = __ldg(dp + i);
          ea = di + 1;
          eb = __ldg(rp + i + 1);
          stage = 1;
        }
        if (stage == 1) {
          const unsigned long long w = ld_relaxed64(W + i);
          if (bad || ic_mark(w) >= tf) {
            s = ic_value(w);
            stage = 2;
            moved = true;
          }
        }
        if (stage == 2) {
          const int e_before = ea;
          if (ic_accumulate(ci, Lf, W, ea, eb, bad ? 0u : tb, s, !moved)) {
            const float w = __fdiv_rn(s, __ldg(Lf + di));
            st_relaxed64(W + i, ic_word(w, tb));
            consume(i, __ldcg(S.r + i), (double)w);
            ++m;
            stage = 0;
            moved = true;
          } else {
            moved = moved || ea != e_before;
          }
        }
      }
      if (__any_sync(kFull, moved)) {
        t_last = clock64();
        nap = 0;
      } else {
        idle();
      }
    }
  }
  __syncthreads();
}

}  // namespace mpcg
