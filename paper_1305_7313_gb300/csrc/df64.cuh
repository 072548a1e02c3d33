// df64.cuh — double-float arithmetic on the FP32 pipe.
//
// A df64 holds a real number as the unevaluated sum hi + lo of two floats with
// |lo| <= ulp(hi) / 2: about 48 significant bits (unit roundoff ~ 2^-48), the
// exponent range of float.  The operations are built from the error-free
// transformations of the literature:
//   TwoSum (Knuth, TAOCP vol. 2, 4.2.2):  s + e == a + b exactly, 6 flops;
//   FastTwoSum (Dekker 1971, "A floating-point technique for extending the
//   available precision"), valid for |a| >= |b|:  s + e == a + b, 3 flops;
//   TwoProd with a fused multiply-add: p + e == a * b exactly, 2 flops.
// Addition is the "sloppy" double-float sum (TwoSum of the high parts, the low
// parts added in float, one renormalisation): its error is bounded by a small
// multiple of 2^-48 (|a| + |b|), which is the norm-wise bound an FFT needs.
// Multiplication drops lo * lo (below the format's precision).
//
// GB300 issues FP32 at 64 times its FP64 rate, so a transform in df64 — about
// ten FP32 instructions per FP64 one — runs several times faster than the
// same transform in FP64, at an accuracy (~1e-14 relative) far inside the
// 1e-10 the FP64 form promises.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

// The operations compile for the host too, so that they can be checked on a
// CPU (with floating-point contraction off); the kernels use them on the device.
#define DF_HD __host__ __device__ __forceinline__

namespace fockx {

// a * b + c with one rounding, in float
DF_HD float df_fmaf(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return std::fma(a, b, c);
#endif
}
DF_HD unsigned df_float_bits(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  unsigned u;
  std::memcpy(&u, &f, sizeof u);
  return u;
#endif
}
DF_HD double df_double_from_bits(unsigned long long b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double d;
  std::memcpy(&d, &b, sizeof d);
  return d;
#endif
}

struct df64 {
  float hi, lo;
  df64() = default;
  __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr df64(double d)
      : hi(static_cast<float>(d)), lo(static_cast<float>(d - static_cast<double>(static_cast<float>(d)))) {}
  __host__ __device__ constexpr df64(float f) : hi(f), lo(0.0f) {}
  __host__ __device__ constexpr df64(int i) : df64(static_cast<double>(i)) {}
};

struct __align__(16) cdf64 {
  df64 x, y;
};

DF_HD df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }

DF_HD df64 operator+(df64 a, df64 b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  float e = (a.hi - (s - bb)) + (b.hi - bb);  // TwoSum error of the high parts
  e += a.lo + b.lo;
  const float h = s + e;  // FastTwoSum renormalisation
  return df64(h, e - (h - s));
}

DF_HD df64 operator-(df64 a, df64 b) { return a + (-b); }

DF_HD df64 operator*(df64 a, df64 b) {
  const float p = a.hi * b.hi;
  float e = df_fmaf(a.hi, b.hi, -p);  // TwoProd error
  e = df_fmaf(a.hi, b.lo, e);
  e = df_fmaf(a.lo, b.hi, e);
  const float h = p + e;
  return df64(h, e - (h - p));
}

// equal values (a normalised pair represents a value in one way only)
DF_HD bool operator==(df64 a, df64 b) { return a.hi == b.hi && a.lo == b.lo; }
DF_HD df64& operator+=(df64& a, df64 b) { return a = a + b; }
DF_HD df64& operator-=(df64& a, df64 b) { return a = a - b; }
DF_HD df64& operator*=(df64& a, df64 b) { return a = a * b; }

// Exact scaling by a power of two.
DF_HD df64 ldexp_pow2(df64 a, float p2) { return df64(a.hi * p2, a.lo * p2); }

// The double nearest hi + lo (FP64 instructions: for O(nb) work and reductions).
DF_HD double to_double(df64 a) { return (double)a.hi + (double)a.lo; }
DF_HD double to_double(double a) { return a; }
DF_HD double to_double(float a) { return (double)a; }

// The double equal to a normal float, formed with integer instructions only
// (the sign, the rebiased exponent and the mantissa moved into place); zeros
// and subnormals (|f| < 2^-126) give 0.
DF_HD double float_bits_to_double(float f) {
  const unsigned u = df_float_bits(f);
  const unsigned ex = (u >> 23) & 0xffu;
  const unsigned long long bits = ((unsigned long long)(u & 0x80000000u) << 32) |
                                  ((unsigned long long)(ex + 896u) << 52) |
                                  ((unsigned long long)(u & 0x7fffffu) << 29);
  return ex == 0u ? 0.0 : df_double_from_bits(bits);
}

}  // namespace fockx
