// Number formats of the mixed-precision CG on the device: rounding onto each format
// (the fl_p of Section 4 with the Table 1 parameters), storage types, and the
// Philox4x64-10 generator used for the exploration draws of Algorithm 1.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace mpcg {

enum Fmt : int { F16 = 0, BF16 = 1, TF32 = 2, F32 = 3, F64 = 4, BF16R = 5, F16R = 6, NFMT = 7 };

// Storage of a format's value and vector arrays.
enum Store : int { ST_HALF = 0, ST_BF16 = 1, ST_FLOAT = 2, ST_DOUBLE = 3 };

__host__ __device__ constexpr int store_of(int f) {
  return (f == F16 || f == F16R) ? ST_HALF
         : (f == BF16 || f == BF16R) ? ST_BF16
         : (f == F64) ? ST_DOUBLE
                      : ST_FLOAT;
}
__host__ __device__ constexpr int bytes_of(int f) {
  return store_of(f) == ST_DOUBLE ? 8 : store_of(f) == ST_FLOAT ? 4 : 2;
}
__host__ __device__ constexpr bool row_scaled(int f) { return f == BF16R || f == F16R; }
// The row-scaled formats round vectors like their base format.
__host__ __device__ constexpr int base_fmt(int f) { return f == BF16R ? BF16 : f == F16R ? F16 : f; }

// Round-to-nearest-even of x onto a binary format with T significand digits, minimum
// normal exponent EMIN (gradual underflow below) and maximum exponent EMAX, computed on the
// IEEE-754 binary64 bit pattern. Zero, infinities and NaN pass through; results above the
// largest finite value of the format become infinities, as IEEE overflow under
// round-to-nearest does.
template <int T, int EMIN, int EMAX>
__device__ __forceinline__ double round_to(double x) {
  constexpr int DROP = 53 - T;  // fraction bits removed in the format's normal range
  constexpr unsigned long long FMASK = (1ull << DROP) - 1ull;
  constexpr unsigned long long MAXB =
      ((unsigned long long)(EMAX + 1023) << 52) | (((1ull << (T - 1)) - 1ull) << DROP);
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned long long sgn = u & 0x8000000000000000ull;
  const unsigned long long a = u ^ sgn;
  if (a == 0ull || a >= 0x7ff0000000000000ull) return x;
  const int e = (int)(a >> 52) - 1023;
  if (e >= EMIN) {
    // Normal range: add just under half a unit (plus the kept lsb, for ties to even) and
    // clear the removed bits; a carry moves into the exponent field as it should.
    unsigned long long r = (a + (FMASK >> 1) + ((a >> DROP) & 1ull)) & ~FMASK;
    if (r > MAXB) r = 0x7ff0000000000000ull;
    return __longlong_as_double((long long)(r | sgn));
  }
  // Subnormal range of the format: the quantum stays 2^(EMIN - T + 1). With the 53-bit
  // significand m, x / quantum = m 2^-d.
  const int d = DROP + (EMIN - e);
  if (d > 53) return __longlong_as_double((long long)sgn);  // below half a quantum
  const unsigned long long m = (a & 0x000fffffffffffffull) | 0x0010000000000000ull;
  unsigned long long k = m >> d;
  const unsigned long long rem = m & ((1ull << d) - 1ull);
  const unsigned long long half = 1ull << (d - 1);
  if (rem > half || (rem == half && (k & 1ull))) ++k;
  const double y = (double)k * __longlong_as_double((long long)((unsigned long long)(EMIN - T + 1 + 1023) << 52));
  return sgn ? -y : y;
}

// fl_p(x) for a format code; fp64 is the identity.
__device__ __forceinline__ double round_fmt(double x, int f) {
  switch (base_fmt(f)) {
    case F16: return round_to<11, -14, 15>(x);
    case BF16: return round_to<8, -126, 127>(x);
    case TF32: return round_to<11, -126, 127>(x);
    case F32: return round_to<24, -126, 127>(x);
    default: return x;
  }
}

// Rounding of an fp32 accumulator onto tf32 (10 fraction bits, fp32 exponent range),
// round-to-nearest-even on the bit pattern; valid through the subnormal range because
// both formats share the exponent field.
__device__ __forceinline__ float round_tf32(float v) {
  unsigned u = __float_as_uint(v);
  if ((u & 0x7f800000u) == 0x7f800000u) return v;
  u = (u + 0xfffu + ((u >> 13) & 1u)) & ~0x1fffu;
  return __uint_as_float(u);
}

// Rounding of an fp32 accumulator onto the output format of the product (op 1). The fp16
// and bf16 conversions are the CUDA round-to-nearest-even intrinsics (one rounding).
__device__ __forceinline__ float round_acc(float acc, int f) {
  switch (base_fmt(f)) {
    case F16: return __half2float(__float2half_rn(acc));
    case BF16: return __bfloat162float(__float2bfloat16_rn(acc));
    case TF32: return round_tf32(acc);
    default: return acc;
  }
}

// Loads of stored values as the accumulator type.
__device__ __forceinline__ float to_acc(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_acc(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_acc(float v) { return v; }
__device__ __forceinline__ double to_acc(double v) { return v; }

template <typename VT> struct AccOf { using type = float; };
template <> struct AccOf<double> { using type = double; };

// Stores an exactly representable double into storage type VT (the conversion is exact).
__device__ __forceinline__ void store_exact(__half* p, long long i, double v) { p[i] = __double2half(v); }
__device__ __forceinline__ void store_exact(__nv_bfloat16* p, long long i, double v) { p[i] = __double2bfloat16(v); }
__device__ __forceinline__ void store_exact(float* p, long long i, double v) { p[i] = (float)v; }
__device__ __forceinline__ void store_exact(double* p, long long i, double v) { p[i] = v; }

// Reads element i of a vector stored in format f, as fp64 (exact).
__device__ __forceinline__ double load_fmt(const void* p, long long i, int f) {
  switch (store_of(f)) {
    case ST_HALF: return (double)__half2float(((const __half*)p)[i]);
    case ST_BF16: return (double)__bfloat162float(((const __nv_bfloat16*)p)[i]);
    case ST_FLOAT: return (double)((const float*)p)[i];
    default: return ((const double*)p)[i];
  }
}

// Writes fl_f(v) into a vector stored in format f.
__device__ __forceinline__ void store_fmt(void* p, long long i, double v, int f) {
  const double r = round_fmt(v, f);
  switch (store_of(f)) {
    case ST_HALF: store_exact((__half*)p, i, r); break;
    case ST_BF16: store_exact((__nv_bfloat16*)p, i, r); break;
    case ST_FLOAT: store_exact((float*)p, i, r); break;
    default: store_exact((double*)p, i, r); break;
  }
}

// Philox4x64-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as easy as 1, 2, 3",
// SC'11): ten rounds of two 64x64->128-bit multiplications with a Weyl-sequence key schedule.
struct U64x4 { unsigned long long v[4]; };
__device__ __forceinline__ U64x4 philox4x64_10(U64x4 c, unsigned long long k0, unsigned long long k1) {
  const unsigned long long M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const unsigned long long W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned long long hi0 = __umul64hi(M0, c.v[0]), lo0 = M0 * c.v[0];
    const unsigned long long hi1 = __umul64hi(M1, c.v[2]), lo1 = M1 * c.v[2];
    U64x4 n;
    n.v[0] = hi1 ^ c.v[1] ^ k0;
    n.v[1] = lo1;
    n.v[2] = hi0 ^ c.v[3] ^ k1;
    n.v[3] = lo0;
    c = n;
    k0 += W0;
    k1 += W1;
  }
  return c;
}

}  // namespace mpcg
