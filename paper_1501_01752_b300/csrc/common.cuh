// Shared device/host helpers for the GSM kernels: complex arithmetic on
// float2/double2, the per-instance parameter block and the geometry of one
// truncation level.  All kernels are written for sm_103a.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace gsm {

template <typename R> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };

__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { return mk(a.x + b.x, a.y + b.y); }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { return mk(a.x - b.x, a.y - b.y); }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
template <typename C> __host__ __device__ __forceinline__ C cmulc(C a, C b) {
  return mk(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
template <typename C, typename R> __host__ __device__ __forceinline__ C cscale(C a, R s) { return mk(a.x * s, a.y * s); }

// Element type of the product's input and output vectors in memory (X, Y):
// the working complex type, except for the double-float product, whose
// vectors stay complex128 (dfloat.cuh).
template <typename R> struct Io { using T = typename Cx<R>::T; };
// conversions at the edges of the product (identity unless specialised)
template <typename C, typename IO> __device__ __forceinline__ C io_in(IO v) { return v; }
template <typename IO, typename C> __device__ __forceinline__ IO io_out(C v) { return v; }

// the value of the neighbouring lane (lane ^ 1) within the lanes of mask
__device__ __forceinline__ float2 shfl_xor1(float2 v, unsigned mask) {
  return make_float2(__shfl_xor_sync(mask, v.x, 1), __shfl_xor_sync(mask, v.y, 1));
}
__device__ __forceinline__ double2 shfl_xor1(double2 v, unsigned mask) {
  return make_double2(__shfl_xor_sync(mask, v.x, 1), __shfl_xor_sync(mask, v.y, 1));
}

// reciprocal in the working precision (the preconditioner's alpha and 1/k^2:
// FP32 through the correctly rounded reciprocal intrinsic, cheaper than a
// division; every kernel that applies M^{-1} uses the same call)
__device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }

// packed FP32 pair arithmetic of sm_100+ (one add/sub/mul/fma .f32x2
// instruction per call, both lanes rounded to nearest)
namespace f2 {
__device__ __forceinline__ unsigned long long u(float2 a) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
  return r;
}
__device__ __forceinline__ float2 f(unsigned long long r) {
  float2 a;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
  return a;
}
__device__ __forceinline__ float2 add(float2 a, float2 b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(u(a)), "l"(u(b)));
  return f(d);
}
__device__ __forceinline__ float2 sub(float2 a, float2 b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(u(a)), "l"(u(b)));
  return f(d);
}
__device__ __forceinline__ float2 mul(float2 a, float2 b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(u(a)), "l"(u(b)));
  return f(d);
}
// a * b + c
__device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(u(a)), "l"(u(b)), "l"(u(c)));
  return f(d);
}
}  // namespace f2

// read-only loads of twiddle-table entries
__device__ __forceinline__ float2 ldg_c(const float2 *p) { return __ldg(p); }
__device__ __forceinline__ double2 ldg_c(const double2 *p) { return __ldg(p); }

// Per-instance parameters of one incident point (text after Eq. 4).
struct Inst {
  double kinc[3];  // k_inc = kappa * kdir
  double kb2;      // k_b^2 = k0^2 eps_b
  double a[6];     // polarisation (complex, interleaved): E^inc_{m=0}
  // right preconditioner M = I - s Delta_0 G(m) (Delta_0 = (Delta eps/eps_b)_0,
  // the averaged medium): M^{-1} = alpha P_T + beta P_L per harmonic with
  // alpha = 1 / (1 - pc_c / (k_m^2 - k_b^2)), pc_c = s Delta_0 k_b^2, and
  // beta = 1 / (1 + s Delta_0).  pc_c = 0, pc_beta = 1 is the identity.
  double pc_c;
  double pc_beta;
};

// Geometry of one truncation level, passed by value to every kernel.
struct Geo {
  int N[3];        // harmonics per axis (odd)
  int n[3];        // (N - 1) / 2
  int L[3];        // FFT points per axis (2^p or 3 * 2^p, >= 2N - 1)
  double K[3];     // reciprocal vectors 2 pi / Lambda
  long long Nh;    // N0 N1 N2
  long long U;     // 3 Nh complex unknowns per instance
  long long Tsz;   // 3 L0 N1 N2: per-instance intermediate of the matvec
  // per-instance strides of the intermediate T and of the per-harmonic
  // arrays (1/(k_m^2 - k_b^2)): Tsz and Nh for a batch of one truncation, the
  // largest box's sizes when truncations share a batch
  long long Tst;
  long long ist;
};

// cyclic position of harmonic index i (0..N-1, m = i - n) on an L-point grid
__device__ __forceinline__ int wrap(int i, int n, int L) {
  int m = i - n;
  return m < 0 ? m + L : m;
}

}  // namespace gsm
