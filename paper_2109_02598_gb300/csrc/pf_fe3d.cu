// 3D forward-Euler step, z-streaming (Sec. 2.4.1 solver, Sec. 2.2.2 7-point stencil,
// Sec. 3 models).  General kernel for any grid size: a CTA owns a TX x TY column of the
// xy plane and a chunk of tz planes; it streams through z keeping a ring of three
// planes (z-1, z, z+1) with a periodic xy halo in shared memory, so every input value is
// fetched from HBM once per CTA plus the halo.  Model B keeps three phi planes (halo 2)
// and three mu planes (halo 1); mu is computed on chip and never stored.  Model C keeps
// both of its fields in the phi planes and the chemical potential of m in the mu planes.
#include "pf_internal.h"
#include "pf_tma.cuh"

namespace pf {

namespace {

constexpr int kNT3 = 256;

template <int MODEL, int TX, int TY>
struct Cfg3 {
  static constexpr int NF = ModelTraits<MODEL>::NF;
  static constexpr int R = ModelTraits<MODEL>::R;
  // phi planes (halo R)
  static constexpr int W = TX + 2 * R;
  static constexpr int HT = TY + 2 * R;
  static constexpr int PL = W * HT;
  // mu planes (Model B only, halo 1)
  static constexpr int W1 = TX + 2;
  static constexpr int HT1 = TY + 2;
  static constexpr int PL1 = W1 * HT1;
  // ring of phi planes: three (z-1, z, z+1), four for Model C, whose psi needs plane z-1
  // while plane z+2 is already staged for the chemical potential of m
  static constexpr int NPH = (MODEL == PF_MODEL_C) ? 4 : 3;
  static constexpr int SMEM_FLOATS = NPH * NF * PL + (R == 2 ? 3 * PL1 : 0);
};

// Stage plane z (periodic) of every field into ring slot `slot`: 4-byte cp.async copies (the
// rows start at x0 - R, so they are not 16-byte aligned), all of a thread's copies issued
// before one wait; the caller's barrier then makes every thread's visible.
template <class C>
__device__ __forceinline__ void load_plane3d(const FieldPtrs& in, const Geom& g, int x0,
                                             int y0, int z, int slot, float* sm) {
  const int64_t zoff = (int64_t)wrap_index(z, g.nz) * g.plane;
  for (int i = threadIdx.x; i < C::PL; i += kNT3) {
    const int r = i / C::W;
    const int c = i - r * C::W;
    const int gy = wrap_index(y0 - C::R + r, g.ny);
    const int gx = wrap_index(x0 - C::R + c, g.nx);
    const int64_t off = zoff + (int64_t)gy * g.pitch + gx;
#pragma unroll
    for (int f = 0; f < C::NF; ++f) cp_async4(sm + (slot * C::NF + f) * C::PL + i, in.f[f] + off);
  }
  cp_async_wait_all();
}

// 3D Laplacian at position p of a staged plane c (row width W) with the planes b below and
// a above: 7-point (ST = PF_ST_STD), isotropic 19-point (faces and edges, PF_ST_ISO) or
// isotropic 27-point (faces, edges and corners, PF_ST_ISO27).
template <int ST>
__device__ __forceinline__ float lap3d_planes(const float* b, const float* c, const float* a,
                                              int p, int W, float scale) {
  if constexpr (ST == PF_ST_STD) {
    return lap3d(c[p], c[p - 1], c[p + 1], c[p - W], c[p + W], b[p], a[p], scale);
  } else {
    const float faces = __fadd_rn(__fadd_rn(__fadd_rn(c[p - 1], c[p + 1]),
                                            __fadd_rn(c[p - W], c[p + W])),
                                  __fadd_rn(b[p], a[p]));
    const float exy = __fadd_rn(__fadd_rn(c[p - W - 1], c[p - W + 1]),
                                __fadd_rn(c[p + W - 1], c[p + W + 1]));
    const float eb = __fadd_rn(__fadd_rn(b[p - 1], b[p + 1]), __fadd_rn(b[p - W], b[p + W]));
    const float ea = __fadd_rn(__fadd_rn(a[p - 1], a[p + 1]), __fadd_rn(a[p - W], a[p + W]));
    const float edges = __fadd_rn(exy, __fadd_rn(eb, ea));
    if constexpr (ST == PF_ST_ISO) {
      return lap3d_iso(c[p], faces, edges, scale);
    } else {
      const float cb = __fadd_rn(__fadd_rn(b[p - W - 1], b[p - W + 1]),
                                 __fadd_rn(b[p + W - 1], b[p + W + 1]));
      const float ca = __fadd_rn(__fadd_rn(a[p - W - 1], a[p - W + 1]),
                                 __fadd_rn(a[p + W - 1], a[p + W + 1]));
      return lap3d_iso27(c[p], faces, edges, __fadd_rn(cb, ca), scale);
    }
  }
}

// AC and Gray-Scott (stencil radius 1).
template <int MODEL, int TX, int TY, int ST>
__global__ void __launch_bounds__(kNT3) fe3d_r1_kernel(FieldPtrs in, FieldOut out, Geom g,
                                                       ModelParams m, int tz) {
  using C = Cfg3<MODEL, TX, TY>;
  constexpr int W = C::W;
  constexpr int PL = C::PL;
  extern __shared__ __align__(16) float sm[];
  const int x0 = blockIdx.x * TX;
  const int y0 = blockIdx.y * TY;
  const int z0 = blockIdx.z * tz;
  const int z1 = min(z0 + tz, g.nz);
  canary_fill(sm, C::SMEM_FLOATS);
  load_plane3d<C>(in, g, x0, y0, z0 - 1, 0, sm);
  load_plane3d<C>(in, g, x0, y0, z0, 1, sm);
  int sb = 0, sc = 1, sa = 2;
  for (int z = z0; z < z1; ++z) {
    load_plane3d<C>(in, g, x0, y0, z + 1, sa, sm);
    __syncthreads();
    const int64_t zoff = (int64_t)z * g.plane;
    for (int i = threadIdx.x; i < TX * TY; i += kNT3) {
      const int rr = i / TX;
      const int r = 1 + rr;
      const int c = 1 + (i - rr * TX);
      const int p = r * W + c;
      const int gx = x0 + c - 1;
      const int gy = y0 + r - 1;
      float val[C::NF];
      if constexpr (MODEL == PF_MODEL_AC) {
        const float* cp = sm + sc * PL;
        const float l = lap3d_planes<ST>(sm + sb * PL, cp, sm + sa * PL, p, W, m.lap_scale);
        val[0] = ac_update(cp[p], l, m);
      } else {
        const float* cu = sm + (sc * 2) * PL;
        const float* cv = cu + PL;
        const float lu = lap3d_planes<ST>(sm + (sb * 2) * PL, cu, sm + (sa * 2) * PL, p, W,
                                          m.lap_scale);
        const float lv = lap3d_planes<ST>(sm + (sb * 2 + 1) * PL, cv, sm + (sa * 2 + 1) * PL, p,
                                          W, m.lap_scale);
        gs_update(cu[p], cv[p], lu, lv, m, val[0], val[1]);
      }
      if (gx < g.nx && gy < g.ny) {
        const int64_t off = zoff + (int64_t)gy * g.pitch + gx;
#pragma unroll
        for (int f = 0; f < C::NF; ++f) out.f[f][off] = val[f];
      }
    }
    __syncthreads();
    const int t = sb;
    sb = sc;
    sc = sa;
    sa = t;
  }
}

// Model B and Model C: mu planes computed on chip from the staged phi planes (halo 2).
// Model B: mu = c2 phi^3 - c1 phi - lap phi of its one field.  Model C: the chemical
// potential of m (field 1), coupled to psi (field 0).
template <int MODEL, int TX, int TY, int ST>
__device__ __forceinline__ void r2_mu_plane(const float* pb, const float* pc, const float* pa,
                                            float* mu, const ModelParams& m) {
  using C = Cfg3<MODEL, TX, TY>;
  constexpr int W = C::W;
  constexpr int PL = C::PL;
  constexpr int F = C::NF - 1;  // the field whose chemical potential is needed
  for (int i = threadIdx.x; i < C::PL1; i += kNT3) {
    const int r1 = i / C::W1;
    const int c1 = i - r1 * C::W1;
    const int p = (r1 + 1) * W + (c1 + 1);  // position in the phi plane (halo 2)
    const float v = pc[F * PL + p];
    const float l = lap3d_planes<ST>(pb + F * PL, pc + F * PL, pa + F * PL, p, W, m.lap_scale);
    if constexpr (MODEL == PF_MODEL_CH)
      mu[i] = ch_mu(v, l, m);
    else
      mu[i] = mc_mu(pc[p], v, l, m);
  }
}

template <int MODEL, int TX, int TY, int ST>
__global__ void __launch_bounds__(kNT3) fe3d_r2_kernel(FieldPtrs in, FieldOut out, Geom g,
                                                       ModelParams m, int tz) {
  using C = Cfg3<MODEL, TX, TY>;
  constexpr int NF = C::NF;
  constexpr int W = C::W;
  constexpr int PL = C::PL;
  constexpr int W1 = C::W1;
  constexpr int PL1 = C::PL1;
  extern __shared__ __align__(16) float sm[];
  constexpr int NPH = C::NPH;
  float* ph = sm;                  // NPH slots of NF phi planes, pslot(p) = (p - z0 + 8) % NPH
  float* mu = sm + NPH * NF * PL;  // 3 mu slots, slot(p) = (p - z0 + 6) % 3
  const int x0 = blockIdx.x * TX;
  const int y0 = blockIdx.y * TY;
  const int z0 = blockIdx.z * tz;
  const int z1 = min(z0 + tz, g.nz);
  auto slot = [&](int p) { return (p - z0 + 6) % 3; };
  auto pslot = [&](int p) { return (p - z0 + 8) % NPH; };
  auto plane = [&](int p) { return ph + pslot(p) * NF * PL; };
  // prologue: mu(z0-1) from phi(z0-2..z0), then mu(z0) from phi(z0-1..z0+1)
  canary_fill(sm, C::SMEM_FLOATS);
  load_plane3d<C>(in, g, x0, y0, z0 - 2, pslot(z0 - 2), ph);
  load_plane3d<C>(in, g, x0, y0, z0 - 1, pslot(z0 - 1), ph);
  load_plane3d<C>(in, g, x0, y0, z0, pslot(z0), ph);
  __syncthreads();
  r2_mu_plane<MODEL, TX, TY, ST>(plane(z0 - 2), plane(z0 - 1), plane(z0), mu + slot(z0 - 1) * PL1, m);
  __syncthreads();
  load_plane3d<C>(in, g, x0, y0, z0 + 1, pslot(z0 + 1), ph);
  __syncthreads();
  r2_mu_plane<MODEL, TX, TY, ST>(plane(z0 - 1), plane(z0), plane(z0 + 1), mu + slot(z0) * PL1, m);
  __syncthreads();
  for (int z = z0; z < z1; ++z) {
    load_plane3d<C>(in, g, x0, y0, z + 2, pslot(z + 2), ph);
    __syncthreads();
    r2_mu_plane<MODEL, TX, TY, ST>(plane(z), plane(z + 1), plane(z + 2), mu + slot(z + 1) * PL1, m);
    __syncthreads();
    const float* mb = mu + slot(z - 1) * PL1;
    const float* mc = mu + slot(z) * PL1;
    const float* ma = mu + slot(z + 1) * PL1;
    const float* pb = plane(z - 1);
    const float* pc = plane(z);
    const float* pa = plane(z + 1);
    const int64_t zoff = (int64_t)z * g.plane;
    for (int i = threadIdx.x; i < TX * TY; i += kNT3) {
      const int rr = i / TX;
      const int cc = i - rr * TX;
      const int q = (rr + 1) * W1 + (cc + 1);  // mu plane position
      const int p = (rr + 2) * W + (cc + 2);   // phi plane position
      const float l = lap3d_planes<ST>(mb, mc, ma, q, W1, m.lap_scale);
      const int gx = x0 + cc;
      const int gy = y0 + rr;
      if (gx >= g.nx || gy >= g.ny) continue;
      const int64_t off = zoff + (int64_t)gy * g.pitch + gx;
      if constexpr (MODEL == PF_MODEL_CH) {
        out.f[0][off] = ch_update(pc[p], l, m);
      } else {
        const float ps = pc[p];
        const float lp = lap3d_planes<ST>(pb, pc, pa, p, W, m.lap_scale);
        float psn, mn;
        mc_update(ps, pc[PL + p], lp, l, m, psn, mn);
        out.f[0][off] = psn;
        out.f[1][off] = mn;
      }
    }
    __syncthreads();
  }
}

int choose_tz(const Geom& g, int tiles_xy) {
  // enough CTAs for several waves on 152 SMs; small grids take short chunks (down to 4
  // planes) and accept the prologue planes they re-read, large grids keep long chunks
  int tz = g.nz;
  while (tz > 4 && (int64_t)tiles_xy * ((g.nz + tz - 1) / tz) < 4 * 152) tz = (tz + 1) / 2;
  return tz;
}

template <int MODEL, int TX, int TY, int ST>
cudaError_t launch3(const Geom& g, FieldPtrs in, FieldOut out, const ModelParams& m,
                    cudaStream_t s) {
  using C = Cfg3<MODEL, TX, TY>;
  const size_t smem = sizeof(float) * C::SMEM_FLOATS;
  static unsigned long long attr_mask = 0;  // per instantiation and device
  const int bx = (g.nx + TX - 1) / TX, by = (g.ny + TY - 1) / TY;
  const int tz = choose_tz(g, bx * by);
  dim3 grid(bx, by, (g.nz + tz - 1) / tz);
  if constexpr (ModelTraits<MODEL>::R == 2) {
    cudaError_t e = ensure_smem_attr(fe3d_r2_kernel<MODEL, TX, TY, ST>, smem, &attr_mask);
    if (e != cudaSuccess) return e;
    fe3d_r2_kernel<MODEL, TX, TY, ST><<<grid, kNT3, smem, s>>>(in, out, g, m, tz);
  } else {
    cudaError_t e = ensure_smem_attr(fe3d_r1_kernel<MODEL, TX, TY, ST>, smem, &attr_mask);
    if (e != cudaSuccess) return e;
    fe3d_r1_kernel<MODEL, TX, TY, ST><<<grid, kNT3, smem, s>>>(in, out, g, m, tz);
  }
  return cudaGetLastError();
}

template <int MODEL>
cudaError_t launch3_tile(int tile_id, const Geom& g, FieldPtrs in, FieldOut out,
                         const ModelParams& m, cudaStream_t s, int stencil) {
  if (stencil == PF_ST_ISO) {
    if (tile_id == 0) return launch3<MODEL, 32, 16, PF_ST_ISO>(g, in, out, m, s);
    return launch3<MODEL, 64, 8, PF_ST_ISO>(g, in, out, m, s);
  }
  if (stencil == PF_ST_ISO27) {
    if (tile_id == 0) return launch3<MODEL, 32, 16, PF_ST_ISO27>(g, in, out, m, s);
    return launch3<MODEL, 64, 8, PF_ST_ISO27>(g, in, out, m, s);
  }
  if (stencil != PF_ST_STD) return cudaErrorInvalidValue;
  if (tile_id == 0) return launch3<MODEL, 32, 16, PF_ST_STD>(g, in, out, m, s);
  return launch3<MODEL, 64, 8, PF_ST_STD>(g, in, out, m, s);
}

}  // namespace

void tile3d_shape(int tile_id, int* tx, int* ty) {
  static const int s[kNumTiles3D][2] = {{32, 16}, {64, 8},   {64, 16}, {128, 8},
                                        {128, 16}, {256, 8}, {32, 8}};
  *tx = s[tile_id][0];
  *ty = s[tile_id][1];
}

int tile3d_id(int tx, int ty) {
  for (int i = 0; i < kNumTiles3D; ++i) {
    int a, b;
    tile3d_shape(i, &a, &b);
    if (a == tx && b == ty) return i;
  }
  return -1;
}

cudaError_t launch_fe3d(int model, int tile_id, const Geom& g, FieldPtrs in, FieldOut out,
                        const ModelParams& m, cudaStream_t s, int stencil) {
  if (tile_id < 0 || tile_id >= kFirstTmaTile3D) return cudaErrorInvalidValue;
  switch (model) {
    case PF_MODEL_AC: return launch3_tile<PF_MODEL_AC>(tile_id, g, in, out, m, s, stencil);
    case PF_MODEL_CH: return launch3_tile<PF_MODEL_CH>(tile_id, g, in, out, m, s, stencil);
    case PF_MODEL_GS: return launch3_tile<PF_MODEL_GS>(tile_id, g, in, out, m, s, stencil);
    case PF_MODEL_C: return launch3_tile<PF_MODEL_C>(tile_id, g, in, out, m, s, stencil);
  }
  return cudaErrorInvalidValue;
}

}  // namespace pf
