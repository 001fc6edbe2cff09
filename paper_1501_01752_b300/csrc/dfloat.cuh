// Double-float arithmetic: a real number carried as the unevaluated sum
// hi + lo of two FP32 values (|lo| <= ulp(hi) / 2), about 48 significand
// bits, computed entirely on the FP32 pipes.
//
// The outer residual of the mixed-precision solve needs the Eq. 4 product
// to ~1e-12 relative; B300's FP64 rate is a small fraction of its FP32
// rate, so that product runs in this arithmetic instead of FP64.  The
// building blocks are the classical error-free transformations: Knuth's
// two-sum (the exact rounding error of a + b), Dekker's fast two-sum for
// |a| >= |b|, and the FMA-based exact product error a b - fl(a b).  The
// addition is the "sloppy" double-float sum (error within a few units of
// 2^-46 (|a| + |b|)), which is the right error model for an FFT, whose
// rounding analysis is in norm.
//
// Every FP32 operation below goes through an __f*_rn intrinsic so that the
// compiler can neither contract it into an FMA nor reassociate it, either
// of which would break the error-free transformations.
#pragma once
#include "common.cuh"

namespace gsm {

struct __align__(8) dfl {
  float hi, lo;
  dfl() = default;
  __host__ __device__ constexpr dfl(float h, float l) : hi(h), lo(l) {}
  // nearest double-float of a double (exact for |v| in the FP32 range)
  __host__ __device__ constexpr dfl(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
  __host__ __device__ constexpr dfl(int v) : hi((float)v), lo(0.f) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

struct __align__(16) dcx {
  dfl x, y;
};

template <> struct Cx<dfl> { using T = dcx; };
template <> struct Io<dfl> { using T = double2; };   // product input/output stay complex128

__host__ __device__ __forceinline__ dcx mk(dfl a, dfl b) {
  dcx r;
  r.x = a;
  r.y = b;
  return r;
}

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ dfl df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return dfl(s, e);
}

// s + e = a + b exactly when |a| >= |b| (Dekker)
__device__ __forceinline__ dfl df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return dfl(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ dfl operator+(dfl a, dfl b) {
  const dfl s = df_two_sum(a.hi, b.hi);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dfl operator-(dfl a) { return dfl(-a.hi, -a.lo); }
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }

// product: p = fl(a.hi b.hi) plus the exact error of that rounding and the
// two cross terms, accumulated by FMA
__device__ __forceinline__ dfl operator*(dfl a, dfl b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}
// small integer factors (the +-1 direction signs of the FFT kernels)
__device__ __forceinline__ dfl operator*(int s, dfl a) {
  if (s == 1) return a;
  if (s == -1) return -a;
  return dfl(__int2float_rn(s), 0.f) * a;
}
__device__ __forceinline__ dfl &operator+=(dfl &a, dfl b) { return a = a + b; }
__device__ __forceinline__ dfl &operator-=(dfl &a, dfl b) { return a = a - b; }
__device__ __forceinline__ dfl &operator*=(dfl &a, dfl b) { return a = a * b; }

// Complex double-float addition, subtraction and products with the packed
// FP32 instructions of sm_100+ (common.cuh, namespace f2): the real part in
// lane 0 and the imaginary part in lane 1 of every pair go through the same
// error-free steps as the scalar operators above, in the same order, so the
// results are bit-identical to the scalar code with half the instructions.
// These overloads take precedence over the generic complex templates of
// common.cuh wherever the complex type is dcx.
namespace dpk {
struct P {
  float2 hi, lo;   // (re.hi, im.hi), (re.lo, im.lo)
};
__device__ __forceinline__ P pk(dcx a) { return {make_float2(a.x.hi, a.y.hi), make_float2(a.x.lo, a.y.lo)}; }
__device__ __forceinline__ dcx un(P p) { return mk(dfl(p.hi.x, p.lo.x), dfl(p.hi.y, p.lo.y)); }
__device__ __forceinline__ P fast_two_sum(float2 a, float2 b) {
  const float2 s = f2::add(a, b);
  return {s, f2::sub(b, f2::sub(s, a))};
}
// (a.hi + b.hi) error-free, then the low parts: the scalar operator+
__device__ __forceinline__ P add(P a, P b) {
  const float2 s = f2::add(a.hi, b.hi);
  const float2 bb = f2::sub(s, a.hi);
  const float2 e = f2::add(f2::sub(a.hi, f2::sub(s, bb)), f2::sub(b.hi, bb));
  return fast_two_sum(s, f2::add(e, f2::add(a.lo, b.lo)));
}
// a + (-b) of the scalar operators, written with subtractions: x + (-y) and
// x - y round identically, and so do (-y) - z and -(y + z)
__device__ __forceinline__ P sub(P a, P b) {
  const float2 s = f2::sub(a.hi, b.hi);
  const float2 bb = f2::sub(s, a.hi);
  const float2 e = f2::sub(f2::sub(a.hi, f2::sub(s, bb)), f2::add(b.hi, bb));
  return fast_two_sum(s, f2::add(e, f2::sub(a.lo, b.lo)));
}
// lane-wise double-float products (the scalar operator*)
__device__ __forceinline__ P mul(P a, P b) {
  const float2 p = f2::mul(a.hi, b.hi);
  float2 e = f2::fma(a.hi, b.hi, f2::mul(p, make_float2(-1.f, -1.f)));
  e = f2::fma(a.hi, b.lo, e);
  e = f2::fma(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}
}  // namespace dpk

__device__ __forceinline__ dcx cadd(dcx a, dcx b) { return dpk::un(dpk::add(dpk::pk(a), dpk::pk(b))); }
__device__ __forceinline__ dcx csub(dcx a, dcx b) { return dpk::un(dpk::sub(dpk::pk(a), dpk::pk(b))); }
// (a.x b.x - a.y b.y, a.x b.y + a.y b.x): both products of each part in one
// packed product, the real part's second product negated (exact) before the
// packed sum, as the scalar t1 + (-t2)
__device__ __forceinline__ dcx cmul(dcx a, dcx b) {
  const dpk::P ax = {make_float2(a.x.hi, a.x.hi), make_float2(a.x.lo, a.x.lo)};
  const dpk::P ay = {make_float2(a.y.hi, a.y.hi), make_float2(a.y.lo, a.y.lo)};
  const dpk::P bxy = dpk::pk(b);
  const dpk::P byx = {make_float2(b.y.hi, b.x.hi), make_float2(b.y.lo, b.x.lo)};
  const dpk::P t13 = dpk::mul(ax, bxy);
  dpk::P t24 = dpk::mul(ay, byx);
  const float2 sg = make_float2(-1.f, 1.f);
  t24.hi = f2::mul(t24.hi, sg);
  t24.lo = f2::mul(t24.lo, sg);
  return dpk::un(dpk::add(t13, t24));
}
// (a.x s, a.y s)
__device__ __forceinline__ dcx cscale(dcx a, dfl s) {
  const dpk::P ss = {make_float2(s.hi, s.hi), make_float2(s.lo, s.lo)};
  return dpk::un(dpk::mul(dpk::pk(a), ss));
}

// the radix-8 rotations (fft.cuh) for dcx: the same sums and products as
// the generic versions, both parts in one packed pass
template <int S> __device__ __forceinline__ dcx rot8(dcx a) {
  const dfl h(0.70710678118654752440);
  const dpk::P sw = S > 0 ? dpk::P{make_float2(-a.y.hi, a.x.hi), make_float2(-a.y.lo, a.x.lo)}
                          : dpk::P{make_float2(a.y.hi, -a.x.hi), make_float2(a.y.lo, -a.x.lo)};
  const dpk::P hh = {make_float2(h.hi, h.hi), make_float2(h.lo, h.lo)};
  return dpk::un(dpk::mul(dpk::add(dpk::pk(a), sw), hh));
}
template <int S> __device__ __forceinline__ dcx rot8_3(dcx a) {
  const dfl h(0.70710678118654752440);
  const dpk::P na = {make_float2(-a.x.hi, -a.y.hi), make_float2(-a.x.lo, -a.y.lo)};
  const dpk::P sw = S > 0 ? dpk::P{make_float2(-a.y.hi, a.x.hi), make_float2(-a.y.lo, a.x.lo)}
                          : dpk::P{make_float2(a.y.hi, -a.x.hi), make_float2(a.y.lo, -a.x.lo)};
  const dpk::P hh = {make_float2(h.hi, h.hi), make_float2(h.lo, h.lo)};
  return dpk::un(dpk::mul(dpk::add(na, sw), hh));
}

__device__ __forceinline__ dcx shfl_xor1(dcx v, unsigned mask) {
  return mk(dfl(__shfl_xor_sync(mask, v.x.hi, 1), __shfl_xor_sync(mask, v.x.lo, 1)),
            dfl(__shfl_xor_sync(mask, v.y.hi, 1), __shfl_xor_sync(mask, v.y.lo, 1)));
}

// twiddle-table load through the read-only path
__device__ __forceinline__ dcx ldg_c(const dcx *p) {
  const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
  return mk(dfl(t.x, t.y), dfl(t.z, t.w));
}

// complex128 <-> complex double-float at the edges of the product (the
// iterate and the residual stay complex128 in memory)
template <> __device__ __forceinline__ dcx io_in<dcx, double2>(double2 v) { return mk(dfl(v.x), dfl(v.y)); }
template <> __device__ __forceinline__ double2 io_out<double2, dcx>(dcx v) {
  return make_double2((double)v.x, (double)v.y);
}

}  // namespace gsm
