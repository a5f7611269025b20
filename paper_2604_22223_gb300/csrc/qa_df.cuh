// Double-float arithmetic for the accurate mixed-precision path.
//
// A real number is carried as the unevaluated sum hi + lo of two FP32 values
// (|lo| <= ulp(hi) / 2 after every operation), which gives about 48
// significant bits from FP32 instructions alone.  The building blocks are the
// classical error-free transformations: Knuth's TwoSum (the rounding error of
// a + b as an FP32 value), Dekker's FastTwoSum (the same when |a| >= |b|) and
// TwoProd through a fused multiply-add (the rounding error of a * b).
// Additions use the "sloppy" double-float sum (one TwoSum of the high parts,
// the low parts added in FP32, one renormalisation), whose absolute error is
// of order 2^-44 (|a| + |b|): what linear maps such as FFTs and matrix
// products need.  Every step that must not be contracted or reassociated is
// written with the _rn intrinsics.
//
// On GB300 the FP64 rate is a small fraction of the FP32 rate, so this is the
// fast way to FP64-level accuracy for the GW iteration's pointwise, FFT and
// small-matrix stages; the DLR contractions use the tensor cores instead
// (qa_dlr_oz.cu).
#pragma once

#include <cuda_runtime.h>

namespace qa {

struct dfl {
  float hi, lo;
  dfl() = default;
  __host__ __device__ constexpr dfl(float h, float l) : hi(h), lo(l) {}
  // nearest double-float of a double (constants and table entries)
  __host__ __device__ dfl(double d)
      : hi(static_cast<float>(d)),
        lo(static_cast<float>(d - static_cast<double>(static_cast<float>(d)))) {}
  __host__ __device__ explicit operator double() const {
    return static_cast<double>(hi) + static_cast<double>(lo);
  }
};

// complex double-float: (re.hi, re.lo, im.hi, im.lo), one 16-byte access
struct __align__(16) dfc {
  dfl x, y;
};

// d as hi + lo from its bit pattern with FP32-rate integer and float operations
// (GB300 runs FP64 conversions at the FP64 rate): hi = d truncated to 24
// significant bits, lo = the remaining 29 mantissa bits rounded to 24, so
// |hi + lo - d| <= 2^-47 |d| and 0 <= lo/hi < 2^-23.  Zero takes (0, 0); other
// magnitudes outside [2^-74, 2^100) and non-finite values take the FP64 conversion.
__device__ __forceinline__ dfl df_from_bits(double d) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(d));
  const int e = static_cast<int>((b >> 52) & 0x7ffu);
  if (e < 1023 - 74 || e >= 1023 + 100) {
    if ((b << 1) == 0ull) return dfl(0.0f, 0.0f);
    return dfl(d);
  }
  const unsigned sign = static_cast<unsigned>(b >> 32) & 0x80000000u;
  const float hi = __uint_as_float(sign | (static_cast<unsigned>(e - 1023 + 127) << 23) |
                                   static_cast<unsigned>((b >> 29) & 0x7fffffu));
  // the low 29 bits weigh 2^(e - 1075): as a float, biased exponent e - 948 (>= 1 here)
  const float sc = __uint_as_float(static_cast<unsigned>(e - 948) << 23);
  const float lo = __fmul_rn(__uint2float_rn(static_cast<unsigned>(b & 0x1fffffffu)), sc);
  return dfl(hi, sign ? -lo : lo);
}

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// renormalise s + e with |e| small against |s| (Dekker's FastTwoSum)
__device__ __forceinline__ dfl df_norm(float s, float e) {
  const float h = __fadd_rn(s, e);
  return dfl(h, __fsub_rn(e, __fsub_rn(h, s)));
}

__device__ __forceinline__ dfl operator+(dfl a, dfl b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return df_norm(s, e);
}
__device__ __forceinline__ dfl operator-(dfl a) { return dfl(-a.hi, -a.lo); }
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }
__device__ __forceinline__ dfl operator*(dfl a, dfl b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_norm(p, e);
}
__device__ __forceinline__ dfl& operator+=(dfl& a, dfl b) { a = a + b; return a; }
__device__ __forceinline__ dfl& operator-=(dfl& a, dfl b) { a = a - b; return a; }
__device__ __forceinline__ dfl& operator*=(dfl& a, dfl b) { a = a * b; return a; }

// 1/a: FP32 reciprocal and one Newton step in double-float
__device__ __forceinline__ dfl df_rcp(dfl a) {
  const float q = __frcp_rn(a.hi);
  const dfl r = dfl(1.0f, 0.0f) - a * dfl(q, 0.0f);
  return dfl(q, 0.0f) + dfl(q, 0.0f) * r;
}
__device__ __forceinline__ dfl operator/(dfl a, dfl b) { return a * df_rcp(b); }

__device__ __forceinline__ bool operator<(dfl a, dfl b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool operator>(dfl a, dfl b) { return b < a; }
__device__ __forceinline__ bool operator<=(dfl a, dfl b) { return !(b < a); }
__device__ __forceinline__ bool operator>=(dfl a, dfl b) { return !(a < b); }
__device__ __forceinline__ bool operator==(dfl a, dfl b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ bool operator!=(dfl a, dfl b) { return !(a == b); }

// the overloads below join (do not hide) the global float and double ones
using ::fmax;
using ::sqrt;
using ::__shfl_xor_sync;

__device__ __forceinline__ dfl fmax(dfl a, dfl b) { return a < b ? b : a; }
// square root to double-float accuracy: FP32 root and one correction
__device__ __forceinline__ dfl sqrt(dfl a) {
  if (!(a.hi > 0.0f)) return dfl(0.0f, 0.0f);
  const float s = sqrtf(a.hi);
  const dfl d = a - dfl(s, 0.0f) * dfl(s, 0.0f);
  return df_norm(s, __fdiv_rn(d.hi, 2.0f * s));
}
__device__ __forceinline__ dfl __shfl_xor_sync(unsigned mask, dfl v, int o) {
  return dfl(::__shfl_xor_sync(mask, v.hi, o), ::__shfl_xor_sync(mask, v.lo, o));
}

// ---- complex
// re or im of a*b + c*d (one TwoSum of the two leading products, the rest in
// the error term; each leading product split exactly by an FMA)
__device__ __forceinline__ dfl dot2(dfl a, dfl b, dfl c, dfl d) {
  const float p1 = __fmul_rn(a.hi, b.hi);
  const float p2 = __fmul_rn(c.hi, d.hi);
  float e1 = __fmaf_rn(a.hi, b.hi, -p1);
  float e2 = __fmaf_rn(c.hi, d.hi, -p2);
  float s, e;
  two_sum(p1, p2, s, e);
  e1 = __fmaf_rn(a.hi, b.lo, e1);
  e1 = __fmaf_rn(a.lo, b.hi, e1);
  e2 = __fmaf_rn(c.hi, d.lo, e2);
  e2 = __fmaf_rn(c.lo, d.hi, e2);
  e = __fadd_rn(e, __fadd_rn(e1, e2));
  return df_norm(s, e);
}
// z + a*b + c*d
__device__ __forceinline__ dfl dot2_acc(dfl z, dfl a, dfl b, dfl c, dfl d) {
  const float p1 = __fmul_rn(a.hi, b.hi);
  const float p2 = __fmul_rn(c.hi, d.hi);
  float e1 = __fmaf_rn(a.hi, b.hi, -p1);
  float e2 = __fmaf_rn(c.hi, d.hi, -p2);
  float s1, t1, s2, t2;
  two_sum(z.hi, p1, s1, t1);
  two_sum(s1, p2, s2, t2);
  e1 = __fmaf_rn(a.hi, b.lo, e1);
  e1 = __fmaf_rn(a.lo, b.hi, e1);
  e2 = __fmaf_rn(c.hi, d.lo, e2);
  e2 = __fmaf_rn(c.lo, d.hi, e2);
  const float e = __fadd_rn(__fadd_rn(t1, t2), __fadd_rn(__fadd_rn(e1, e2), z.lo));
  return df_norm(s2, e);
}

__device__ __forceinline__ dfc cadd(dfc a, dfc b) { return dfc{a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ dfc csub(dfc a, dfc b) { return dfc{a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ dfc cmul(dfc a, dfc b) {
  return dfc{dot2(a.x, b.x, -a.y, b.y), dot2(a.x, b.y, a.y, b.x)};
}
// c + a*b
__device__ __forceinline__ dfc cfma(dfc a, dfc b, dfc c) {
  return dfc{dot2_acc(c.x, a.x, b.x, -a.y, b.y), dot2_acc(c.y, a.x, b.y, a.y, b.x)};
}
// c - a*b
__device__ __forceinline__ dfc cfms(dfc a, dfc b, dfc c) {
  return dfc{dot2_acc(c.x, -a.x, b.x, a.y, b.y), dot2_acc(c.y, -a.x, b.y, -a.y, b.x)};
}
__device__ __forceinline__ dfl cabs2(dfc a) { return dot2(a.x, a.x, a.y, a.y); }
__device__ __forceinline__ dfc cconj(dfc a) { return dfc{a.x, -a.y}; }
__device__ __forceinline__ dfc cscale(dfc a, dfl s) { return dfc{a.x * s, a.y * s}; }
__device__ __forceinline__ dfc cinv(dfc a) {
  const dfl d = df_rcp(cabs2(a));
  return dfc{a.x * d, -(a.y * d)};
}
__device__ __forceinline__ double2 to_c64d(dfc a) {
  return make_double2(static_cast<double>(a.x), static_cast<double>(a.y));
}

// Slice-grid code of one double-float complex value for the tensor-core DLR maps:
// 0 for a zero value, else max(e, -100) + 101, where e is the binary exponent of
// x = 2.000004 max(|re.hi|, |im.hi|) in frexp's convention (2^(e-1) <= x < 2^e;
// for a normal x, its biased exponent - 126; a subnormal x clamps to -100).  The
// scaling and the exponent are both monotone in the magnitude, so the largest
// code over a column decodes to the exponent of the column's largest value.
__device__ __forceinline__ unsigned oz_grid_code(dfc v) {
  const float m = fmaxf(fabsf(v.x.hi), fabsf(v.y.hi));
  if (m == 0.0f) return 0u;
  const int be = static_cast<int>((__float_as_uint(m * 2.000004f) >> 23) & 0xffu);
  return static_cast<unsigned>(max(be - 126, -100) + 101);
}

}  // namespace qa
