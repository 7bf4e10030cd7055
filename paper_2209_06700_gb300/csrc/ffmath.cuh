// Device arithmetic shared by the operator and vector kernels of libirk (sm_103a).
//
// Float-float (ff): a value hi + lo with |lo| <= ulp(hi) / 2, about 48 significant bits, computed
// with FP32 instructions only.  On this part FP64 instructions issue at a small fraction of the
// FP32 rate, so the FP64-accurate parts of the solver (the stage operator of Eq. (irk:A) and the
// Krylov vector work) keep their vectors in ff form (8 bytes per value, like FP64) and never touch
// the FP64 pipe on the hot path.  The error-free transformations are Knuth's two-sum (with the
// round-to-nearest intrinsics, never contracted into FMA) and the FMA-based exact product.
#pragma once
#include "kernels.h"

namespace irk {
namespace dev {

template <typename T> __device__ __forceinline__ T zero() { return T(0); }
template <> __device__ __forceinline__ ff zero<ff>() { return ff{0.f, 0.f}; }

__device__ __forceinline__ ff ff_renorm(float s, float e) {
  const float hi = __fadd_rn(s, e);
  return ff{hi, __fsub_rn(e, __fsub_rn(hi, s))};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return ff_renorm(s, e);
}
// a + c v: the product c.hi v.hi is split exactly by an FMA, the cross terms are plain FP32
__device__ __forceinline__ ff ff_mad(ff a, ff c, ff v) {
  const float p = __fmul_rn(c.hi, v.hi);
  float pe = __fmaf_rn(c.hi, v.hi, -p);
  pe = __fmaf_rn(c.hi, v.lo, pe);
  pe = __fmaf_rn(c.lo, v.hi, pe);
  const float s = __fadd_rn(a.hi, p);
  const float bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  e = __fadd_rn(e, __fadd_rn(a.lo, pe));
  return ff_renorm(s, e);
}
__device__ __forceinline__ ff ff_mul(ff c, ff v) {
  const float p = __fmul_rn(c.hi, v.hi);
  float pe = __fmaf_rn(c.hi, v.hi, -p);
  pe = __fmaf_rn(c.hi, v.lo, pe);
  pe = __fmaf_rn(c.lo, v.hi, pe);
  return ff_renorm(p, pe);
}
__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.hi, -a.lo}; }

__device__ __forceinline__ float mad(float a, float c, float v) { return fmaf(c, v, a); }
__device__ __forceinline__ double mad(double a, double c, double v) { return fma(c, v, a); }
__device__ __forceinline__ ff mad(ff a, ff c, ff v) { return ff_mad(a, c, v); }
__device__ __forceinline__ float mul(float c, float v) { return c * v; }
__device__ __forceinline__ double mul(double c, double v) { return c * v; }
__device__ __forceinline__ ff mul(ff c, ff v) { return ff_mul(c, v); }
__device__ __forceinline__ float add(float a, float b) { return a + b; }
__device__ __forceinline__ double add(double a, double b) { return a + b; }
__device__ __forceinline__ ff add(ff a, ff b) { return ff_add(a, b); }
__device__ __forceinline__ float neg(float a) { return -a; }
__device__ __forceinline__ double neg(double a) { return -a; }
__device__ __forceinline__ ff neg(ff a) { return ff_neg(a); }

// Two independent multiply-adds (a, b) <- (a + ca va, b + cb vb).  FP32 and float-float issue
// them as packed pairs (the f32x2 add / sub / mul / fma instructions of sm_100 and later): each
// lane of a packed instruction rounds exactly like the scalar instruction, so the pair equals
// two calls of mad bit for bit, in about half the issued instructions.
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;"
      : "=l"(r)
      : "l"(*reinterpret_cast<const unsigned long long*>(&a)), "l"(*reinterpret_cast<const unsigned long long*>(&b)));
  return *reinterpret_cast<const float2*>(&r);
}
__device__ __forceinline__ void mad2(float& a, float& b, float ca, float cb, float va, float vb) {
  const float2 r = f2fma(make_float2(ca, cb), make_float2(va, vb), make_float2(a, b));
  a = r.x;
  b = r.y;
}
__device__ __forceinline__ void mad2(double& a, double& b, double ca, double cb, double va, double vb) {
  a = fma(ca, va, a);
  b = fma(cb, vb, b);
}
// the steps of ff_mad, lane by lane
__device__ __forceinline__ void mad2(ff& a, ff& b, ff ca, ff cb, ff va, ff vb) {
  const float2 ah = make_float2(a.hi, b.hi), al = make_float2(a.lo, b.lo);
  const float2 ch = make_float2(ca.hi, cb.hi), cl = make_float2(ca.lo, cb.lo);
  const float2 vh = make_float2(va.hi, vb.hi), vl = make_float2(va.lo, vb.lo);
  const float2 p = f2mul(ch, vh);
  float2 pe = f2fma(ch, vh, make_float2(-p.x, -p.y));
  pe = f2fma(ch, vl, pe);
  pe = f2fma(cl, vh, pe);
  const float2 s = f2add(ah, p);
  const float2 bb = f2sub(s, ah);
  float2 e = f2add(f2sub(ah, f2sub(s, bb)), f2sub(p, bb));
  e = f2add(e, f2add(al, pe));
  const float2 hi = f2add(s, e);
  const float2 lo = f2sub(e, f2sub(hi, s));
  a = ff{hi.x, lo.x};
  b = ff{hi.y, lo.y};
}

// conversions (the double <-> ff ones use the FP64 pipe: coefficients and boundary copies only)
template <typename T> __device__ __forceinline__ T from_double(double d) { return (T)d; }
template <> __device__ __forceinline__ ff from_double<ff>(double d) {
  const float hi = __double2float_rn(d);
  return ff{hi, __double2float_rn(d - (double)hi)};
}
__device__ __forceinline__ double to_double(float v) { return (double)v; }
__device__ __forceinline__ double to_double(double v) { return v; }
__device__ __forceinline__ double to_double(ff v) { return (double)v.hi + (double)v.lo; }
// between vector element types: float <-> ff exact one way, rounded to FP32 the other
template <typename To, typename From> __device__ __forceinline__ To convert(From v) { return (To)v; }
template <> __device__ __forceinline__ ff convert<ff, float>(float v) { return ff{v, 0.f}; }
template <> __device__ __forceinline__ float convert<float, ff>(ff v) { return __fadd_rn(v.hi, v.lo); }
template <> __device__ __forceinline__ ff convert<ff, ff>(ff v) { return v; }
template <> __device__ __forceinline__ ff convert<ff, double>(double v) { return from_double<ff>(v); }
template <> __device__ __forceinline__ double convert<double, ff>(ff v) { return to_double(v); }

// vector element loads: read-only path (ld.global.nc) for inputs not written by the same launch
template <typename T> __device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }
template <> __device__ __forceinline__ ff ldg<ff>(const ff* p) {
  const float2 t = __ldg(reinterpret_cast<const float2*>(p));
  return ff{t.x, t.y};
}

__device__ __forceinline__ float shfl_down(float v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double shfl_down(double v, int o) { return __shfl_down_sync(0xffffffffu, v, o); }
__device__ __forceinline__ ff shfl_down(ff v, int o) {
  return ff{__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)};
}
__device__ __forceinline__ float shfl_up(float v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ double shfl_up(double v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ ff shfl_up(ff v) {
  return ff{__shfl_up_sync(0xffffffffu, v.hi, 1), __shfl_up_sync(0xffffffffu, v.lo, 1)};
}

}  // namespace dev
}  // namespace irk
