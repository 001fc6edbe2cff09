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
