// Per-site arithmetic of the forward-Euler step, shared by every kernel of the library so
// that the plain, temporally blocked, TMA and batched paths give bitwise-identical
// results.  Every operation is an explicitly rounded intrinsic (__fadd_rn, __fmaf_rn,
// ...), so the compiler cannot contract or reorder differently in different kernels.
//
// Equations (arxiv 2109.02598, Sec. 3; Gray-Scott in its standard form, named in Sec. 1):
//   Model A (AC):  f = lap phi + c1 phi - c2 phi^3
//   Model B (CH):  mu = c2 phi^3 - c1 phi - lap phi,   f = M lap mu
//   Gray-Scott:    f_u = Du lap u - u v^2 + F (1 - u),  f_v = Dv lap v + u v^2 - (F + k) v
//   Model C:       f_psi = lap psi + c1 psi - c2 psi^3 + 2 c5 psi m,
//                  mu_m = c4 m^3 - c3 m - c5 psi^2 - lap m,  f_m = lap mu_m
// Forward Euler (Sec. 2.4.1): x_new = x + dt f(x).
// Laplacian (Sec. 2.2.2): second-order central, 5 points in 2D and 7 in 3D, evaluated as
// fma(-2d, c, ((x- + x+) + (y- + y+)) [+ (z- + z+)]) times 1/h^2: six operations in 3D
// instead of the twelve of the paired-difference form, which matters because the 3D
// kernels are bound by instruction issue.  Each neighbour pair is one commutative
// addition, so the streaming direction does not change the result, and a constant field
// gives exactly zero.
#pragma once

#include <cuda_runtime.h>

#include "pfgpu.h"

namespace pf {

// Coefficients as the kernels use them (float32, rounded once on the host).
//   AC: a0 = c1, a1 = c2
//   CH: a0 = c1, a1 = c2, a2 = dt * M
//   GS: a0 = Du s, a1 = Dv s, a2 = F, a3 = F + k (s = the stencil factor; lap_scale = 1)
//   C:  a0 = c1, a1 = c2, a2 = c3, a3 = c4, a4 = c5, a5 = 2 c5
// lap_scale: the stencil's overall factor, 1/h^2 for the standard 5/7-point stencils,
// 1/(6 h^2) for the isotropic 9/19-point ones, 1/(12 h^2) for the fourth-order 9-point one,
// 1/(30 h^2) for the isotropic 27-point one.
struct ModelParams {
  float a0, a1, a2, a3, a4, a5;
  float dt;
  float lap_scale;
};

// Laplacian stencils (Sec. 2.2.2).
#define PF_ST_STD 0  // 5-point (2D) / 7-point (3D), second order
#define PF_ST_ISO 1  // isotropic 9-point (2D) / 19-point (3D), second order
#define PF_ST_O4 2   // fourth-order 9-point (2D): +-1 and +-2 along each axis
#define PF_ST_ISO27 3  // isotropic 27-point (3D), second order

static_assert(PF_ST_STD == PF_STENCIL_STD && PF_ST_ISO == PF_STENCIL_ISO &&
                  PF_ST_O4 == PF_STENCIL_4TH && PF_ST_ISO27 == PF_STENCIL_ISO27,
              "internal stencil ids follow the public ones");

template <int ST>
struct StencilTraits {
  static constexpr int R = (ST == PF_ST_O4) ? 2 : 1;  // radius in sites
};

template <int MODEL>
struct ModelTraits;
template <>
struct ModelTraits<PF_MODEL_AC> {
  static constexpr int NF = 1;  // fields
  static constexpr int R = 1;   // stencil radius of one step
};
template <>
struct ModelTraits<PF_MODEL_CH> {
  static constexpr int NF = 1;
  static constexpr int R = 2;  // Laplacian of the Laplacian
};
template <>
struct ModelTraits<PF_MODEL_GS> {
  static constexpr int NF = 2;
  static constexpr int R = 1;
};
template <>
struct ModelTraits<PF_MODEL_C> {
  static constexpr int NF = 2;
  static constexpr int R = 2;  // m needs the Laplacian of its chemical potential
};

// 5-/7-point stencil sums before the factor 1/h^2.
__device__ __forceinline__ float lap2d_sum(float c, float xm, float xp, float ym, float yp) {
  const float s = __fadd_rn(__fadd_rn(xm, xp), __fadd_rn(ym, yp));
  return __fmaf_rn(-4.0f, c, s);
}

__device__ __forceinline__ float lap3d_sum(float c, float xm, float xp, float ym, float yp,
                                           float zm, float zp) {
  const float s = __fadd_rn(__fadd_rn(__fadd_rn(xm, xp), __fadd_rn(ym, yp)), __fadd_rn(zm, zp));
  return __fmaf_rn(-6.0f, c, s);
}

__device__ __forceinline__ float lap2d(float c, float xm, float xp, float ym, float yp,
                                       float lap_scale) {
  return __fmul_rn(lap2d_sum(c, xm, xp, ym, yp), lap_scale);
}

__device__ __forceinline__ float lap3d(float c, float xm, float xp, float ym, float yp,
                                       float zm, float zp, float lap_scale) {
  return __fmul_rn(lap3d_sum(c, xm, xp, ym, yp, zm, zp), lap_scale);
}

// Gray-Scott's parameters carry the stencil factor in D_u and D_v, and its lap_scale is 1
// (make_params). x * 1 is exact, so a Gray-Scott kernel may leave the Laplacian's final
// multiply out and still give the bits of one that does it.
template <int MODEL>
__device__ __forceinline__ float lap_scaled(float sum, float lap_scale) {
  if constexpr (MODEL == PF_MODEL_GS)
    return sum;
  else
    return __fmul_rn(sum, lap_scale);
}

// Isotropic 9-point: (4 (axial) + (diagonal) - 20 c) / (6 h^2)
__device__ __forceinline__ float lap2d_iso(float c, float xm, float xp, float ym, float yp,
                                           float d0, float d1, float d2, float d3, float scale) {
  const float ax = __fadd_rn(__fadd_rn(xm, xp), __fadd_rn(ym, yp));
  const float dg = __fadd_rn(__fadd_rn(d0, d1), __fadd_rn(d2, d3));
  return __fmul_rn(__fmaf_rn(-20.0f, c, __fmaf_rn(4.0f, ax, dg)), scale);
}

// Fourth-order 9-point: sum over axes of (16 (x[+1] + x[-1]) - (x[+2] + x[-2])) - 60 c,
// over 12 h^2
__device__ __forceinline__ float lap2d_o4(float c, float xm, float xp, float xm2, float xp2,
                                          float ym, float yp, float ym2, float yp2, float scale) {
  const float ax = __fmaf_rn(16.0f, __fadd_rn(xm, xp), -__fadd_rn(xm2, xp2));
  const float ay = __fmaf_rn(16.0f, __fadd_rn(ym, yp), -__fadd_rn(ym2, yp2));
  return __fmul_rn(__fmaf_rn(-60.0f, c, __fadd_rn(ax, ay)), scale);
}

// Isotropic 19-point: (2 (6 faces) + (12 edges) - 24 c) / (6 h^2); callers pass the sums.
__device__ __forceinline__ float lap3d_iso(float c, float faces, float edges, float scale) {
  return __fmul_rn(__fmaf_rn(-24.0f, c, __fmaf_rn(2.0f, faces, edges)), scale);
}

// Isotropic 27-point: (14 (6 faces) + 3 (12 edges) + (8 corners) - 128 c) / (30 h^2).
__device__ __forceinline__ float lap3d_iso27(float c, float faces, float edges, float corners,
                                             float scale) {
  const float s = __fmaf_rn(14.0f, faces, __fmaf_rn(3.0f, edges, corners));
  return __fmul_rn(__fmaf_rn(-128.0f, c, s), scale);
}

// Model A: phi + dt (lap + c1 phi - c2 phi^3)
__device__ __forceinline__ float ac_update(float p, float lap, const ModelParams& m) {
  const float p3 = __fmul_rn(__fmul_rn(p, p), p);
  float f = __fmaf_rn(m.a0, p, lap);
  f = __fmaf_rn(-m.a1, p3, f);
  return __fmaf_rn(m.dt, f, p);
}

// Model B chemical potential: c2 phi^3 - c1 phi - lap
__device__ __forceinline__ float ch_mu(float p, float lap, const ModelParams& m) {
  const float p3 = __fmul_rn(__fmul_rn(p, p), p);
  const float mu = __fmaf_rn(m.a1, p3, -lap);
  return __fmaf_rn(-m.a0, p, mu);
}

// Model B update: phi + (dt M) lap mu
__device__ __forceinline__ float ch_update(float p, float lap_mu, const ModelParams& m) {
  return __fmaf_rn(m.a2, lap_mu, p);
}

// Gray-Scott update of (u, v) from their Laplacians.
__device__ __forceinline__ void gs_update(float u, float v, float lu, float lv,
                                          const ModelParams& m, float& un, float& vn) {
  const float uvv = __fmul_rn(__fmul_rn(u, v), v);
  float fu = __fmaf_rn(m.a0, lu, -uvv);
  fu = __fmaf_rn(m.a2, __fsub_rn(1.0f, u), fu);
  float fv = __fmaf_rn(m.a1, lv, uvv);
  fv = __fmaf_rn(-m.a3, v, fv);
  un = __fmaf_rn(m.dt, fu, u);
  vn = __fmaf_rn(m.dt, fv, v);
}

// Model C chemical potential of m: c4 m^3 - c3 m - c5 psi^2 - lap m
__device__ __forceinline__ float mc_mu(float psi, float m, float lap_m, const ModelParams& p) {
  const float m3 = __fmul_rn(__fmul_rn(m, m), m);
  float mu = __fmaf_rn(p.a3, m3, -lap_m);
  mu = __fmaf_rn(-p.a2, m, mu);
  return __fmaf_rn(-p.a4, __fmul_rn(psi, psi), mu);
}

// Model C update: psi + dt (lap psi + c1 psi - c2 psi^3 + 2 c5 psi m),  m + dt lap mu_m
__device__ __forceinline__ void mc_update(float psi, float m, float lap_psi, float lap_mu,
                                          const ModelParams& p, float& psi_n, float& m_n) {
  const float p3 = __fmul_rn(__fmul_rn(psi, psi), psi);
  float f = __fmaf_rn(p.a0, psi, lap_psi);
  f = __fmaf_rn(-p.a1, p3, f);
  f = __fmaf_rn(p.a5, __fmul_rn(psi, m), f);
  psi_n = __fmaf_rn(p.dt, f, psi);
  m_n = __fmaf_rn(p.dt, lap_mu, m);
}

// ---- four sites at once with packed FP32 pairs ------------------------------------------
// The sm_100 family executes FP32 add, multiply and fma on register pairs: one instruction
// updates two sites, and per lane the result is the IEEE-rounded result of the scalar
// intrinsic (__fadd2_rn is two __fadd_rn, and so on). The functions below apply the per-site
// arithmetic above to the four sites of a float4 as two pairs, with the same operations in
// the same order, so a kernel that uses them gives the bits of one that uses the scalar
// functions, with about half the arithmetic instructions. Negated operands and x - y = x + (-y)
// are exact, so writing a subtraction as an addition of the negation keeps the bits too.
__device__ __forceinline__ float2 lo2(const float4& v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(const float4& v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float4 cat4(const float2& a, const float2& b) {
  return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ float4 add4(const float4& a, const float4& b) {
  return cat4(__fadd2_rn(lo2(a), lo2(b)), __fadd2_rn(hi2(a), hi2(b)));
}
__device__ __forceinline__ float4 mul4(const float4& a, const float4& b) {
  return cat4(__fmul2_rn(lo2(a), lo2(b)), __fmul2_rn(hi2(a), hi2(b)));
}
__device__ __forceinline__ float4 mul4(float a, const float4& b) {
  const float2 aa = make_float2(a, a);
  return cat4(__fmul2_rn(aa, lo2(b)), __fmul2_rn(aa, hi2(b)));
}
__device__ __forceinline__ float4 fma4(const float4& a, const float4& b, const float4& c) {
  return cat4(__ffma2_rn(lo2(a), lo2(b), lo2(c)), __ffma2_rn(hi2(a), hi2(b), hi2(c)));
}
__device__ __forceinline__ float4 fma4(float a, const float4& b, const float4& c) {
  const float2 aa = make_float2(a, a);
  return cat4(__ffma2_rn(aa, lo2(b), lo2(c)), __ffma2_rn(aa, hi2(b), hi2(c)));
}
__device__ __forceinline__ float4 neg4(const float4& a) {
  return make_float4(-a.x, -a.y, -a.z, -a.w);
}

// lap3d_sum of the four sites of c (x-neighbours: the scalar xm left of c.x, xp right of c.w)
__device__ __forceinline__ float4 lap3d_sum4(const float4& c, float xm, float xp,
                                             const float4& ym, const float4& yp,
                                             const float4& zm, const float4& zp) {
  const float4 sx = make_float4(__fadd_rn(xm, c.y), __fadd_rn(c.x, c.z), __fadd_rn(c.y, c.w),
                                __fadd_rn(c.z, xp));
  const float4 s = add4(add4(sx, add4(ym, yp)), add4(zm, zp));
  return fma4(-6.0f, c, s);
}

// lap2d_sum of the four sites of c
__device__ __forceinline__ float4 lap2d_sum4(const float4& c, float xm, float xp,
                                             const float4& ym, const float4& yp) {
  const float4 sx = make_float4(__fadd_rn(xm, c.y), __fadd_rn(c.x, c.z), __fadd_rn(c.y, c.w),
                                __fadd_rn(c.z, xp));
  return fma4(-4.0f, c, add4(sx, add4(ym, yp)));
}

// ac_update of four sites
__device__ __forceinline__ float4 ac_update4(const float4& p, const float4& lap,
                                             const ModelParams& m) {
  const float4 p3 = mul4(mul4(p, p), p);
  float4 f = fma4(m.a0, p, lap);
  f = fma4(-m.a1, p3, f);
  return fma4(m.dt, f, p);
}

// ch_mu of four sites
__device__ __forceinline__ float4 ch_mu4(const float4& p, const float4& lap,
                                         const ModelParams& m) {
  const float4 p3 = mul4(mul4(p, p), p);
  const float4 mu = fma4(m.a1, p3, neg4(lap));
  return fma4(-m.a0, p, mu);
}

// ch_update of four sites
__device__ __forceinline__ float4 ch_update4(const float4& p, const float4& lap_mu,
                                             const ModelParams& m) {
  return fma4(m.a2, lap_mu, p);
}

// gs_update of four sites
__device__ __forceinline__ void gs_update4(const float4& u, const float4& v, const float4& lu,
                                           const float4& lv, const ModelParams& m, float4& un,
                                           float4& vn) {
  const float4 uvv = mul4(mul4(u, v), v);
  float4 fu = fma4(m.a0, lu, neg4(uvv));
  fu = fma4(m.a2, add4(make_float4(1.0f, 1.0f, 1.0f, 1.0f), neg4(u)), fu);
  float4 fv = fma4(m.a1, lv, uvv);
  fv = fma4(-m.a3, v, fv);
  un = fma4(m.dt, fu, u);
  vn = fma4(m.dt, fv, v);
}

// mc_mu of four sites
__device__ __forceinline__ float4 mc_mu4(const float4& psi, const float4& m4,
                                         const float4& lap_m, const ModelParams& p) {
  const float4 m3 = mul4(mul4(m4, m4), m4);
  float4 mu = fma4(p.a3, m3, neg4(lap_m));
  mu = fma4(-p.a2, m4, mu);
  return fma4(-p.a4, mul4(psi, psi), mu);
}

// mc_update of four sites
__device__ __forceinline__ void mc_update4(const float4& psi, const float4& m4,
                                           const float4& lap_psi, const float4& lap_mu,
                                           const ModelParams& p, float4& psi_n, float4& m_n) {
  const float4 p3 = mul4(mul4(psi, psi), psi);
  float4 f = fma4(p.a0, psi, lap_psi);
  f = fma4(-p.a1, p3, f);
  f = fma4(p.a5, mul4(psi, m4), f);
  psi_n = fma4(p.dt, f, psi);
  m_n = fma4(p.dt, lap_mu, m4);
}

// Checked builds (PF_CHECK): fill n floats of shared memory with NaN before they are staged,
// so a read of a slot that staging or an earlier sub-step did not write turns results into
// NaN, which the parity tests see. Every thread of the CTA calls it; it ends with a CTA
// barrier. A no-op in normal builds.
__device__ __forceinline__ void canary_fill(float* p, size_t n) {
#ifdef PF_CHECK
  for (size_t i = threadIdx.x; i < n; i += blockDim.x) p[i] = __int_as_float(0x7fc00000);
  __syncthreads();
#else
  (void)p;
  (void)n;
#endif
}

// Periodic index: i in [-n, 2n) maps into [0, n); anything else takes the slow modulo
// (only tiles larger than the grid reach it).
__device__ __forceinline__ int wrap_index(int i, int n) {
  if (i < 0) i += n;
  if (i >= n) i -= n;
  if ((unsigned)i >= (unsigned)n) {
    i %= n;
    if (i < 0) i += n;
  }
  return i;
}

}  // namespace pf
