// Number formats of the mixed-precision CG on the device: rounding onto each format
// (the fl_p of Section 4 with the Table 1 parameters), storage types, and the
// Philox4x64-10 generator used for the exploration draws of Algorithm 1.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace mpcg {

// Q52: Table 1's quarter precision, 3 significand digits with the fp16 exponent range
// (e_min = -14, e_max = 15; the fp8 E5M2 layout).
enum Fmt : int { F16 = 0, BF16 = 1, TF32 = 2, F32 = 3, F64 = 4, BF16R = 5, F16R = 6, Q52 = 7, NFMT = 8 };

// Storage of a format's value and vector arrays.
enum Store : int { ST_HALF = 0, ST_BF16 = 1, ST_FLOAT = 2, ST_DOUBLE = 3, ST_Q52 = 4 };

__host__ __device__ constexpr int store_of(int f) {
  return (f == F16 || f == F16R) ? ST_HALF
         : (f == BF16 || f == BF16R) ? ST_BF16
         : (f == F64) ? ST_DOUBLE
         : (f == Q52) ? ST_Q52
                      : ST_FLOAT;
}
__host__ __device__ constexpr int bytes_of(int f) {
  return store_of(f) == ST_DOUBLE ? 8 : store_of(f) == ST_FLOAT ? 4 : store_of(f) == ST_Q52 ? 1 : 2;
}

// One stored q52 value: sign, 5 exponent bits and 2 fraction bits, the same fields as the
// upper byte of an fp16 number (same exponent bias), so a q52 value is exactly the fp16
// number whose lower byte is zero.
struct q52_t {
  unsigned char b;
};
struct q52x2_t {
  q52_t x, y;
};
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
    case Q52: return round_to<3, -14, 15>(x);
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

// Loads of stored values as the accumulator type.
__device__ __forceinline__ float to_acc(q52_t v) { return __half2float(__ushort_as_half((unsigned short)(v.b << 8))); }
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

// A q52 value given as fp32 (exact) in storage: the upper byte of its fp16 pattern.
__device__ __forceinline__ q52_t q52_from_exact(float v) {
  return q52_t{(unsigned char)(__half_as_ushort(__float2half_rn(v)) >> 8)};
}

// Reads element i of a vector stored in format f, as fp64 (exact).
__device__ __forceinline__ double load_fmt(const void* p, long long i, int f) {
  switch (store_of(f)) {
    case ST_Q52: return (double)to_acc(((const q52_t*)p)[i]);
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
    case ST_Q52: ((q52_t*)p)[i] = q52_from_exact((float)r); break;
    case ST_HALF: store_exact((__half*)p, i, r); break;
    case ST_BF16: store_exact((__nv_bfloat16*)p, i, r); break;
    case ST_FLOAT: store_exact((float*)p, i, r); break;
    default: store_exact((double*)p, i, r); break;
  }
}

// ---- fp32-domain conversions (no fp64 instruction on the common path) ---------------
// GB300 executes fp64 arithmetic and fp64 conversions at a small fraction of the fp32 rate,
// so the per-row work converts between fp32 and fp64 by assembling bit patterns and rounds
// fp64 values onto the 16-bit formats through fp32.

// Exact fp32 -> fp64 from the bit pattern (normal, zero, subnormal, infinite, NaN). Integer
// instructions only: GB300 runs fp64 conversions on its narrow fp64 pipe, and a call to an
// out-of-line slow path in a per-row loop makes the compiler save registers around it.
__device__ __forceinline__ double f2d(float v) {
  const unsigned u = __float_as_uint(v);
  const unsigned sgn = u & 0x80000000u;
  const unsigned a = u & 0x7fffffffu;
  unsigned hi, lo;
  if (a - 0x00800000u < 0x7f000000u) {  // normal
    hi = sgn | ((a >> 3) + (896u << 20));
    lo = a << 29;
  } else if (a == 0u) {
    hi = sgn;
    lo = 0u;
  } else if (a >= 0x7f800000u) {  // infinite or NaN: same fraction bits, top of the exponent
    hi = sgn | 0x7ff00000u | ((a & 0x7fffffu) >> 3);
    lo = a << 29;
  } else {  // subnormal: a 2^-149 with the leading one at bit p
    const int p = 31 - __clz((int)a);
    const unsigned long long bits =
        ((unsigned long long)(p - 149 + 1023) << 52) | (((unsigned long long)a << (52 - p)) & 0xfffffffffffffull);
    hi = sgn | (unsigned)(bits >> 32);
    lo = (unsigned)bits;
  }
  return __hiloint2double((int)hi, (int)lo);
}

// x * 2^e for an fp64 x whose result stays in the normal range (exponent-field add);
// otherwise a multiplication.
__device__ __forceinline__ double scale2(double x, int e) {
  const int hi = __double2hiint(x);
  const int ex = (hi >> 20) & 0x7ff;
  if (e == 0 || x == 0.0) return x;
  if (ex > 0 && ex < 0x7ff && ex + e > 0 && ex + e < 0x7ff) return __hiloint2double(hi + (e << 20), __double2loint(x));
  // subnormal operand or result (rare): two exact power-of-two factors
  const int e1 = e / 2, e2 = e - e1;
  return x * __longlong_as_double((long long)((unsigned long long)(e1 + 1023) << 52)) *
         __longlong_as_double((long long)((unsigned long long)(e2 + 1023) << 52));
}

// Truncation of x onto fp32 with the last bit set when bits were dropped ("round to odd").
// Valid when |x| lies in the fp32 normal range or x = 0; returns false otherwise. Rounding
// the result to nearest onto a format with at most 22 significand digits gives the correctly
// rounded value of x (Boldo and Melquiond, "Emulation of FMA and correctly rounded sums:
// proved algorithms using rounding to odd", IEEE Trans. Computers 57(4), 2008).
__device__ __forceinline__ bool d2f_odd(double x, float& out) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned ex = (hi >> 20) & 0x7ffu;
  if (ex >= 897u && ex <= 1150u) {  // 2^-126 <= |x| < 2^128
    unsigned f = (hi & 0x80000000u) | ((ex - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
    f |= (lo & 0x1fffffffu) ? 1u : 0u;
    out = __uint_as_float(f);
    return true;
  }
  if ((hi & 0x7fffffffu) == 0u && lo == 0u) {
    out = __uint_as_float(hi);
    return true;
  }
  return false;
}

// fl_fp32(x), round to nearest even, for |x| in the fp32 normal range (false otherwise).
__device__ __forceinline__ bool d2f_rn(double x, float& out) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned ex = (hi >> 20) & 0x7ffu;
  if (ex >= 897u && ex <= 1150u) {
    unsigned f = (hi & 0x80000000u) | ((ex - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned rest = lo & 0x1fffffffu;  // dropped bits; half = 0x10000000
    if (rest > 0x10000000u || (rest == 0x10000000u && (f & 1u))) ++f;  // carries into the exponent
    out = __uint_as_float(f);
    return true;
  }
  if ((hi & 0x7fffffffu) == 0u && lo == 0u) {
    out = __uint_as_float(hi);
    return true;
  }
  return false;
}

// fl_q52(v) of an fp32 value: the exact fp64 form rounded on its bit pattern (round to
// nearest even, gradual underflow below 2^-14, overflow beyond 57344 to infinity).
__device__ __forceinline__ float round_q52(float v) { return (float)round_to<3, -14, 15>(f2d(v)); }

// fl_f(v) of an fp32 value (one rounding) for f in {fp16, bf16, tf32, fp32, q52} (and the
// row-scaled variants).
__device__ __forceinline__ float round_f2f(float v, int f) {
  switch (base_fmt(f)) {
    case F16: return __half2float(__float2half_rn(v));
    case BF16: return __bfloat162float(__float2bfloat16_rn(v));
    case TF32: return round_tf32(v);
    case Q52: return round_q52(v);
    default: return v;
  }
}

static __device__ __noinline__ float round_d2f_slow(double x, int f) { return (float)round_fmt(x, f); }

// fl_f(x) of an fp64 value, returned as fp32 (exact), for f other than fp64.
__device__ __forceinline__ float round_d2f(double x, int f) {
  float o;
  if (base_fmt(f) == F32) {
    if (d2f_rn(x, o)) return o;
  } else if (d2f_odd(x, o)) {
    return round_f2f(o, f);
  }
  return round_d2f_slow(x, f);  // outside the fp32 normal range: exact bit-level rounding
}

// Value set of format a contains that of format b (so rounding onto a is the identity on b).
__host__ __device__ constexpr bool contains_fmt(int a, int b) {
  return base_fmt(a) == F64 || base_fmt(a) == base_fmt(b) ||
         (base_fmt(a) == F32 && base_fmt(b) != F64) ||
         (base_fmt(a) == TF32 && (base_fmt(b) == F16 || base_fmt(b) == BF16 || base_fmt(b) == Q52)) ||
         ((base_fmt(a) == F16 || base_fmt(a) == BF16) && base_fmt(b) == Q52);
}

// s + t = a + b exactly (Knuth's TwoSum), fp32, without contraction.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& t) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  t = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Rounds the exact value s + e of a compensated fp32 pair onto format f (fp32 result):
// fp32 takes fl(s + e); the coarser formats round the round-to-odd value of s + e.
__device__ __forceinline__ float round_pair(float s, float e, int f) {
  float hi, lo;
  two_sum(s, e, hi, lo);
  if (base_fmt(f) == F32 || !isfinite(hi)) return hi;
  unsigned b = __float_as_uint(hi);
  if (lo != 0.f && !(b & 1u)) b += ((lo > 0.f) == (hi > 0.f)) ? 1u : 0xffffffffu;
  return round_f2f(__uint_as_float(b), f);
}

// Compensated fp32 accumulation of the product a * b (exact for inputs of at most 12
// significand digits; for fp32 inputs the FMA error of the product is carried too).
__device__ __forceinline__ void acc2(float a, float b, bool exact_product, float& s, float& c) {
  const float p = __fmul_rn(a, b);
  float t;
  two_sum(s, p, s, t);
  if (!exact_product) t = __fadd_rn(t, __fmaf_rn(a, b, -p));
  c = __fadd_rn(c, t);
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
