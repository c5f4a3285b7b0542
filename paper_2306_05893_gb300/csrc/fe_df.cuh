// Double-float arithmetic for the solve's FP64-accurate sums.
//
// A double-float value is the unevaluated sum hi + lo of two floats (about
// 48 significant bits), updated with Knuth's TwoSum and Dekker's TwoProduct
// (through FMA).  GB300's FP64 pipe issues a warp instruction every ~64
// cycles per SM sub-partition (1.25 TFLOP/s for the GPU), so a gather loop
// with one FP64 multiply-add or conversion per value is bound by that pipe,
// not by HBM; the same sums in double-float run on the FP32 pipe (128 lanes
// per SM per cycle) at a dozen instructions per term.
//
// The FP64 copy of A in the mixed path and the refinement iterate's mirror
// are stored as float2 pairs (x = hi, y = lo, hi = fl32(v), lo = fl32(v - hi)):
// the same 8 bytes as a double, exact to ~2^-48 relative.
#pragma once

#include <cuda_runtime.h>

namespace fe {

// (hi, lo) += (ph, pl), ph the larger part of the addend (TwoSum on the high parts)
__device__ __forceinline__ void df_add_to(float &hi, float &lo, float ph, float pl) {
  const float s = hi + ph, bb = s - hi;
  lo += ((hi - (s - bb)) + (ph - bb)) + pl;
  hi = s;
}

// (hi, lo) += (a.x + a.y)(b.x + b.y) (the lo * lo term, ~2^-48 of the product, dropped)
__device__ __forceinline__ void df_fma_to(float &hi, float &lo, float2 a, float2 b) {
  const float p = a.x * b.x;
  df_add_to(hi, lo, p, fmaf(a.x, b.y, fmaf(a.y, b.x, fmaf(a.x, b.x, -p))));
}

// a double as a float pair (three FP64-pipe instructions: meant for
// element-wise, lane-parallel use, not inside a gather loop)
__device__ __forceinline__ float2 df_split(double v) {
  const float h = float(v);
  return make_float2(h, float(v - double(h)));
}

__device__ __forceinline__ double df_value(float hi, float lo) { return double(hi) + double(lo); }
__device__ __forceinline__ double df_value(float2 v) { return double(v.x) + double(v.y); }

// (hi, lo) of a lane plus that of lane ^ o in a group of W lanes (every lane
// of the group ends with the same bits: TwoSum is exact and symmetric)
template <int W>
__device__ __forceinline__ void df_shfl_add(float &hi, float &lo, int o) {
  const float oh = __shfl_xor_sync(0xffffffffu, hi, o, W), ol = __shfl_xor_sync(0xffffffffu, lo, o, W);
  const float s = hi + oh, bb = s - hi;
  lo = (lo + ol) + ((hi - (s - bb)) + (oh - bb));
  hi = s;
}

// A lane's running dot product, in FP64 for both vector types.  Not in
// double-float: the product of two FP32 vector entries leaves FP32's range
// long before the entries do (a Newton correction's late inner solves carry
// entries near 1e-20, whose squares underflow FP32), while the FP64 product
// of two floats is exact.
template <typename TV>
struct DotAcc {
  double s = 0.0;
  __device__ __forceinline__ void add(TV a, TV b) { s += double(a) * double(b); }
  __device__ __forceinline__ double value() const { return s; }
};

// A double-float number for the element kernels' force path (the material
// laws are templates on their number type).  Sums and products follow the
// error-free transformations above with one renormalisation each: relative
// error about 2^-46 per operation (2^-53 in FP64), exponent range that of
// FP32.  Division: the FP32 quotient corrected by one remainder step.
// Constants convert from double at compile time (constexpr); conversions
// from run-time doubles (three FP64-pipe instructions) belong outside the
// hot loops.
struct dfloat {
  float hi, lo;
  dfloat() = default;
  __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr dfloat(double v) : hi(float(v)), lo(float(v - double(float(v)))) {}
  __host__ __device__ constexpr dfloat(int v) : dfloat(double(v)) {}
  __device__ __forceinline__ explicit dfloat(float2 p) : hi(p.x), lo(p.y) {}
  __device__ __forceinline__ explicit operator float() const { return hi + lo; }
  __device__ __forceinline__ explicit operator double() const { return double(hi) + double(lo); }
  __device__ __forceinline__ float2 pair() const { return make_float2(hi, lo); }
};

__device__ __forceinline__ dfloat df_renorm(float s, float e) {
  const float h = s + e;
  return dfloat(h, e - (h - s));
}
__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
  const float s = a.hi + b.hi, bb = s - a.hi;
  const float e = ((a.hi - (s - bb)) + (b.hi - bb)) + (a.lo + b.lo);
  return df_renorm(s, e);
}
__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }
__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) {
  const float p = a.hi * b.hi;
  const float e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, fmaf(a.hi, b.hi, -p)));
  return df_renorm(p, e);
}
__device__ __forceinline__ dfloat operator/(dfloat a, dfloat b) {
  const float q1 = a.hi / b.hi;
  const dfloat r = a - b * dfloat(q1, 0.f);  // the remainder, in double-float
  const float q2 = r.hi / b.hi;
  return df_renorm(q1, q2);
}
__device__ __forceinline__ dfloat &operator+=(dfloat &a, dfloat b) { return a = a + b; }
__device__ __forceinline__ dfloat &operator-=(dfloat &a, dfloat b) { return a = a - b; }
__device__ __forceinline__ dfloat &operator*=(dfloat &a, dfloat b) { return a = a * b; }
__device__ __forceinline__ dfloat &operator/=(dfloat &a, dfloat b) { return a = a / b; }
__device__ __forceinline__ bool operator>(dfloat a, dfloat b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
__device__ __forceinline__ bool operator<(dfloat a, dfloat b) { return b > a; }

}  // namespace fe
