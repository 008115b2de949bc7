// FP32 pair arithmetic shared by the pair kernels: packed two-lane (f32x2) helpers and the
// Ewald real-space factors.
#pragma once
#include "mop_internal.cuh"

namespace mop {
namespace {

// packed f32x2 arithmetic (fma/add/mul.rn.f32x2, sm_100 family): one instruction for the two
// beads a lane holds; only rsqrt, exp2 and the reciprocal stay per half
__device__ __forceinline__ float2 dup2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 rsq2(float2 a) { return make_float2(rsqrtf(a.x), rsqrtf(a.y)); }

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Ewald real space: erfc(x) = exp(-x^2) erfcx(x), with the scaled complementary error function
// erfcx(x) ~ P(x) / Q(x), a rational least-squares fit of degrees 3 / 4 on [0, 6] written by
// fit_erfcx.py of this package (relative error 2.5e-7 for these FP32 coefficients in exact
// arithmetic, about 5e-7 as evaluated here).  Q(x) >= 1, so the approximate reciprocal
// (relative error ~1 ulp) serves.
__constant__ float kErfcxP[4] = {9.999999234e-01f, 9.697673345e-01f, 4.351839909e-01f, 8.235789757e-02f};
__constant__ float kErfcxQ[5] = {1.000000000e+00f, 2.098139719e+00f, 1.802774676e+00f, 7.701872587e-01f, 1.460288291e-01f};

__device__ __forceinline__ float erfcx_rational(float x) {
  float p = kErfcxP[3], q = kErfcxQ[4];
#pragma unroll
  for (int i = 2; i >= 0; --i) p = fmaf(p, x, kErfcxP[i]);
#pragma unroll
  for (int i = 3; i >= 0; --i) q = fmaf(q, x, kErfcxQ[i]);
  return p * rcp_approx(q);
}

// ec = erfc(beta r) and c2e = 2 beta / sqrt(pi) exp(-beta^2 r^2) for both halves; one Gaussian
// serves both terms.  ewb = beta, ewb2 = beta^2, ewc2 = 2 beta / sqrt(pi).
__device__ __forceinline__ void ewald_terms2(float ewb, float ewb2, float ewc2, float2 r2, float2 rinv, float2* ec,
                                             float2* c2e) {
  const float2 y = mul2(r2, dup2(-ewb2 * 1.4426950408889634f));   // -beta^2 r^2 log2(e)
  const float2 G = make_float2(ex2_approx(y.x), ex2_approx(y.y));
  const float2 x = mul2(dup2(ewb), mul2(r2, rinv));
  float2 p = dup2(kErfcxP[3]), q = dup2(kErfcxQ[4]);
#pragma unroll
  for (int i = 2; i >= 0; --i) p = fma2(p, x, dup2(kErfcxP[i]));
#pragma unroll
  for (int i = 3; i >= 0; --i) q = fma2(q, x, dup2(kErfcxQ[i]));
  *ec = mul2(G, mul2(p, make_float2(rcp_approx(q.x), rcp_approx(q.y))));
  *c2e = mul2(dup2(ewc2), G);
}

}  // namespace
}  // namespace mop
