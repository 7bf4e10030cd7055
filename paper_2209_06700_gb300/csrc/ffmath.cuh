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
__device__ __forceinline__ double to_double(double v) { return v; }
__device__ __forceinline__ double to_double(ff v) { return (double)v.hi + (double)v.lo; }
// binary32 <-> binary64 on the integer pipe.  On a GPU whose FP64 pipe is a small fraction of its
// FP32 and integer pipes, the conversion instructions (which run on the FP64 pipe) bound the basis
// changes between the FP64 outer solver and the FP32 multigrid as much as their multiply-adds; the
// IEEE 754 definitions below give the same results from bit operations.
// float -> double is exact: sign kept, exponent rebiased by 1023 - 127 = 896, fraction moved up by
// 29 bits; a subnormal float is normalised (its leading one becomes the implicit bit); infinities
// keep the all-ones exponent, NaNs come out quiet.
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned sign = u & 0x80000000u, e = (u >> 23) & 0xFFu, frac = u & 0x7FFFFFu;
  unsigned hi, lo;
  if (e - 1u < 0xFEu) {  // normal: 1 <= e <= 254
    hi = sign | ((e + 896u) << 20) | (frac >> 3);
    lo = frac << 29;
  } else if (e == 0xFFu) {  // infinity (frac 0) or NaN (quiet bit set)
    hi = sign | 0x7FF00000u | (frac >> 3) | (frac != 0u ? 0x80000u : 0u);
    lo = frac << 29;
  } else if (frac == 0u) {  // signed zero
    hi = sign;
    lo = 0u;
  } else {  // subnormal: frac 2^-149 with its highest set bit p (0..22) as the implicit one
    const int p = 31 - __clz(frac);
    const unsigned long long f52 = ((unsigned long long)(frac ^ (1u << p))) << (52 - p);
    hi = sign | ((unsigned)(p + 874) << 20) | (unsigned)(f52 >> 32);
    lo = (unsigned)f52;
  }
  return __hiloint2double((int)hi, (int)lo);
}
__device__ __forceinline__ double to_double(float v) { return f32_to_f64(v); }
// double -> float, rounded to nearest with ties to even: the top 23 of the 52 fraction bits are
// kept and the 29 below decide; a carry out of the fraction moves into the exponent (and to
// infinity above the largest float) by itself.  Results below the float's normal range (and
// zeros' signs aside, which are kept directly) go through the hardware conversion: rare.
__device__ __forceinline__ float f64_to_f32_rn(double d) {
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FFu);
  if (e == 0x7FF) return __uint_as_float(sign | 0x7F800000u | ((((hi & 0xFFFFFu) | lo) != 0u) ? 0x400000u : 0u));
  if (e == 0 && (hi & 0xFFFFFu) == 0u && lo == 0u) return __uint_as_float(sign);
  const int fe = e - 896;
  if (fe >= 0xFF) return __uint_as_float(sign | 0x7F800000u);
  if (fe <= 0) return __double2float_rn(d);
  const unsigned keep = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  const unsigned rest = lo & 0x1FFFFFFFu;
  unsigned r = sign | ((unsigned)fe << 23) | keep;
  if (rest > 0x10000000u || (rest == 0x10000000u && (keep & 1u))) r += 1u;
  return __uint_as_float(r);
}

// between vector element types: float <-> ff exact one way, rounded to FP32 the other; float <->
// double through the integer-pipe conversions above
template <typename To, typename From> __device__ __forceinline__ To convert(From v) { return (To)v; }
template <> __device__ __forceinline__ double convert<double, float>(float v) { return f32_to_f64(v); }
template <> __device__ __forceinline__ float convert<float, double>(double v) { return f64_to_f32_rn(v); }
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
