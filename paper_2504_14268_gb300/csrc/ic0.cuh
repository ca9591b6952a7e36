// Incomplete Cholesky IC(0) in fp32: completion marks and the sync-free substitutions.
//
// Section 5 preconditions with an incomplete factorization held in fp32 (the paper's
// p_fixed); for SPD matrices its symmetric zero-fill form is M = L L^T with L on the
// pattern of A's lower triangle. Applying M^-1 is two triangular substitutions, each a
// chain of row-to-row dependencies. They run inside the solver kernels without grid
// barriers: every row has a completion mark in global memory, a thread handles its rows in
// order (increasing for L y = r, decreasing for L^T w = y) and waits, row by row, until the
// rows it reads are marked. Because every wait is on a row earlier in that order, the
// earliest unfinished row always has its inputs ready, so all threads being resident (a
// cooperative launch) is enough for progress. Every wait is bounded in time and gives up
// when the launch's status word reports an error.
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

// w = M^-1 fl32(r) over the rows of R for one application with epoch `ep` (marks 2 ep + 1
// on y_i after the forward row, 2 ep + 2 on w_i after the backward row; the words start at
// 0 for a launch and the marks only grow). Both substitutions run in fp32 with each row's
// sum over its stored columns in increasing order and one correctly rounded division by
// l_ii, so the result equals a sequential evaluation bit for bit. y and w share the work
// vector: row i overwrites y_i only after every row that reads y_i has finished its own
// backward step. consume(i, r_i, w_i) runs for every row of R once w_i is final. Starts
// and ends with a CTA barrier (r written by other threads of the CTA is read here).
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
  const unsigned tf = 2u * ep + 1u, tb = 2u * ep + 2u;
  __syncthreads();
  bool bad = *(volatile unsigned*)err != 0u;
  const int cnt = R.r1 - R.r0 > (int)threadIdx.x ? (R.r1 - R.r0 - (int)threadIdx.x + kThreads - 1) / kThreads : 0;
  unsigned rounds = 0, nap = 0;
  long long t_last = clock64();
  // a round without progress in the whole warp: back off (up to about a microsecond, so that
  // waiting warps leave the memory system to the rows being finished), check the status
  // word now and then, and the time since the warp last moved
  auto idle = [&]() {
    nap = nap ? min(2u * nap, 1024u) : 32u;
    __nanosleep(nap);
    if ((++rounds & 63u) != 0u) return;
    if (*(volatile unsigned*)err != 0u) {
      bad = true;
    } else if (clock64() - t_last > limit) {
      atomicOr(err, tbit);
      bad = true;
    }
  };
  // forward: L y = fl32(r), this thread's rows in increasing order
  {
    int m = 0, ea = 0, eb = 0;
    float s = 0.f;
    bool fresh = true;
    while (__any_sync(kFull, m < cnt)) {
      bool moved = false;
      if (m < cnt) {
        const int i = R.r0 + (int)threadIdx.x + m * kThreads;
        const bool fresh_row = fresh;
        if (fresh) {
          ea = __ldg(rp + i);
          eb = __ldg(dp + i);
          s = __double2float_rn(S.r[i]);
          fresh = false;
        }
        const int e_before = ea;
        if (ic_accumulate(ci, Lf, W, ea, eb, bad ? 0u : tf, s, !fresh_row)) {
          st_relaxed64(W + i, ic_word(__fdiv_rn(s, __ldg(Lf + eb)), tf));
          ++m;
          fresh = true;
          moved = true;
        } else {
          moved = ea != e_before;
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
  // backward: L^T w = y, this thread's rows in decreasing order
  {
    int m = cnt - 1, ea = 0, eb = 0, di = 0;
    float s = 0.f;
    bool fresh = true;
    while (__any_sync(kFull, m >= 0)) {
      bool moved = false;
      if (m >= 0) {
        const int i = R.r0 + (int)threadIdx.x + m * kThreads;
        const bool fresh_row = fresh;
        if (fresh) {
          di = __ldg(dp + i);
          ea = di + 1;
          eb = __ldg(rp + i + 1);
          s = ic_value(ld_relaxed64(W + i));  // y_i, written by this thread
          fresh = false;
        }
        const int e_before = ea;
        if (ic_accumulate(ci, Lf, W, ea, eb, bad ? 0u : tb, s, !fresh_row)) {
          const float w = __fdiv_rn(s, __ldg(Lf + di));
          st_relaxed64(W + i, ic_word(w, tb));
          consume(i, S.r[i], (double)w);
          --m;
          fresh = true;
          moved = true;
        } else {
          moved = ea != e_before;
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
