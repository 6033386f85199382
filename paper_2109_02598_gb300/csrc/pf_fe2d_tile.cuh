// Tile body of the 2D forward-Euler kernel with temporal blocking; used by the plain
// 2D kernel, the batched runner and the adjoint's recompute, so all execute identical
// arithmetic.
//
// Shared-memory layout per field: HT rows of WS floats.  Staged column s of row r holds
// the periodic value at (x0 - HP + s, y0 - H + r), where H = k R is the halo the k
// sub-steps consume and HP = H rounded up to 4, so columns come in 16-byte-aligned groups
// of four that match aligned groups in HBM.  Staging moves float4s (scalar loads with
// periodic wrap only where a group crosses the grid edge), and every sub-step computes
// four consecutive sites per thread from float4 rows: centre and y-neighbours as float4,
// the two outer x-neighbours as scalars.
#pragma once

#include "pf_internal.h"

namespace pf {

constexpr int kNT2 = 256;  // threads per CTA of every 2D kernel

template <int MODEL, int K, int TX, int TY, int ST = PF_ST_STD>
struct Cfg2 {
  static constexpr int NF = ModelTraits<MODEL>::NF;
  static constexpr int RS = StencilTraits<ST>::R;       // one Laplacian's radius
  static constexpr int R = ModelTraits<MODEL>::R * RS;  // one step's radius
  static constexpr int H = K * R;              // halo the k sub-steps consume (sites)
  static constexpr int HP = (H + 3) / 4 * 4;   // staged halo, 16-byte aligned
  static constexpr int WS = TX + 2 * HP;       // staged row width (floats)
  static constexpr int HT = TY + 2 * H;        // staged rows
  static constexpr int PL = WS * HT;           // floats per staged field
  static constexpr int NBUF = (K > 1) ? 2 : 1;
  static constexpr int MU = (MODEL == PF_MODEL_CH || MODEL == PF_MODEL_C) ? PL : 0;
  static constexpr int SMEM_FLOATS = NF * NBUF * PL + MU;
  static_assert(TX % 4 == 0, "tile width must be a multiple of 4");
};

// Stage rows [y0-H, y0+TY+H) x columns [x0-HP, x0+TX+HP) of every field into buffer 0.
template <class C>
__device__ __forceinline__ void load_region2d(const FieldPtrs& in, int nx, int ny,
                                              int64_t pitch, int x0, int y0, float* sm) {
  constexpr int CH4 = C::WS / 4;  // float4 groups per staged row
  for (int i = threadIdx.x; i < C::HT * CH4; i += kNT2) {
    const int r = i / CH4;
    const int j = i - r * CH4;
    const int gy = wrap_index(y0 - C::H + r, ny);
    const int gx = x0 - C::HP + 4 * j;
    const int64_t row = (int64_t)gy * pitch;
    float* dst = sm + r * C::WS + 4 * j;
    if (gx >= 0 && gx + 3 < nx) {
#pragma unroll
      for (int f = 0; f < C::NF; ++f)
        *reinterpret_cast<float4*>(dst + f * C::PL) =
            __ldg(reinterpret_cast<const float4*>(in.f[f] + row + gx));
    } else {
      const int64_t o0 = row + wrap_index(gx, nx), o1 = row + wrap_index(gx + 1, nx);
      const int64_t o2 = row + wrap_index(gx + 2, nx), o3 = row + wrap_index(gx + 3, nx);
#pragma unroll
      for (int f = 0; f < C::NF; ++f) {
        const float* p = in.f[f];
        *reinterpret_cast<float4*>(dst + f * C::PL) =
            make_float4(__ldg(p + o0), __ldg(p + o1), __ldg(p + o2), __ldg(p + o3));
      }
    }
  }
}

// 2D Laplacians of four consecutive sites from a float4 row and its neighbours, with the
// stencil ST (its neighbours beyond the float4 come from scalars of the same rows).
template <int ST = PF_ST_STD>
__device__ __forceinline__ float4 lap2d_x4(const float* s, int p, int ws, float scale) {
  const float4 c = *reinterpret_cast<const float4*>(s + p);
  const float4 u = *reinterpret_cast<const float4*>(s + p - ws);
  const float4 d = *reinterpret_cast<const float4*>(s + p + ws);
  const float l = s[p - 1], r = s[p + 4];
  float4 o;
  if constexpr (ST == PF_ST_STD) {
    o.x = lap2d(c.x, l, c.y, u.x, d.x, scale);
    o.y = lap2d(c.y, c.x, c.z, u.y, d.y, scale);
    o.z = lap2d(c.z, c.y, c.w, u.z, d.z, scale);
    o.w = lap2d(c.w, c.z, r, u.w, d.w, scale);
  } else if constexpr (ST == PF_ST_ISO) {
    const float ul = s[p - ws - 1], ur = s[p - ws + 4], dl = s[p + ws - 1], dr = s[p + ws + 4];
    o.x = lap2d_iso(c.x, l, c.y, u.x, d.x, ul, u.y, dl, d.y, scale);
    o.y = lap2d_iso(c.y, c.x, c.z, u.y, d.y, u.x, u.z, d.x, d.z, scale);
    o.z = lap2d_iso(c.z, c.y, c.w, u.z, d.z, u.y, u.w, d.y, d.w, scale);
    o.w = lap2d_iso(c.w, c.z, r, u.w, d.w, u.z, ur, d.z, dr, scale);
  } else {
    const float l2 = s[p - 2], r2 = s[p + 5];
    const float4 u2 = *reinterpret_cast<const float4*>(s + p - 2 * ws);
    const float4 d2 = *reinterpret_cast<const float4*>(s + p + 2 * ws);
    o.x = lap2d_o4(c.x, l, c.y, l2, c.z, u.x, d.x, u2.x, d2.x, scale);
    o.y = lap2d_o4(c.y, c.x, c.z, l, c.w, u.y, d.y, u2.y, d2.y, scale);
    o.z = lap2d_o4(c.z, c.y, c.w, c.x, r, u.z, d.z, u2.z, d2.z, scale);
    o.w = lap2d_o4(c.w, c.z, r, c.y, r2, u.w, d.w, u2.w, d2.w, scale);
  }
  return o;
}

// Chemical potential of four sites at p of a staged region (Model B: of field 0; Model C:
// of m, field 1, coupled to psi, field 0), into mu at p. Rows are ws floats apart and
// fields pl floats apart. Shared by every 2D kernel, so all compute identical arithmetic.
template <int MODEL, int ST>
__device__ __forceinline__ void site4_mu(const float* src, int p, int ws, int pl,
                                         const ModelParams& m, float* mu) {
  if constexpr (MODEL == PF_MODEL_CH) {
    const float4 c = *reinterpret_cast<const float4*>(src + p);
    const float4 l = lap2d_x4<ST>(src, p, ws, m.lap_scale);
    *reinterpret_cast<float4*>(mu + p) =
        make_float4(ch_mu(c.x, l.x, m), ch_mu(c.y, l.y, m), ch_mu(c.z, l.z, m),
                    ch_mu(c.w, l.w, m));
  } else {  // Model C: chemical potential of m (field 1), coupled to psi (field 0)
    const float4 ps = *reinterpret_cast<const float4*>(src + p);
    const float4 c = *reinterpret_cast<const float4*>(src + pl + p);
    const float4 l = lap2d_x4<ST>(src + pl, p, ws, m.lap_scale);
    *reinterpret_cast<float4*>(mu + p) =
        make_float4(mc_mu(ps.x, c.x, l.x, m), mc_mu(ps.y, c.y, l.y, m),
                    mc_mu(ps.z, c.z, l.z, m), mc_mu(ps.w, c.w, l.w, m));
  }
}

// One forward-Euler update of four sites at p for every field: val[f] receives field f.
template <int MODEL, int ST>
__device__ __forceinline__ void site4_update(const float* src, const float* mu, int p, int ws,
                                             int pl, const ModelParams& m, float4* val) {
  if constexpr (MODEL == PF_MODEL_AC) {
    const float4 c = *reinterpret_cast<const float4*>(src + p);
    const float4 l = lap2d_x4<ST>(src, p, ws, m.lap_scale);
    val[0] = make_float4(ac_update(c.x, l.x, m), ac_update(c.y, l.y, m),
                         ac_update(c.z, l.z, m), ac_update(c.w, l.w, m));
  } else if constexpr (MODEL == PF_MODEL_CH) {
    const float4 c = *reinterpret_cast<const float4*>(src + p);
    const float4 l = lap2d_x4<ST>(mu, p, ws, m.lap_scale);
    val[0] = make_float4(ch_update(c.x, l.x, m), ch_update(c.y, l.y, m),
                         ch_update(c.z, l.z, m), ch_update(c.w, l.w, m));
  } else if constexpr (MODEL == PF_MODEL_C) {
    const float4 ps = *reinterpret_cast<const float4*>(src + p);
    const float4 c = *reinterpret_cast<const float4*>(src + pl + p);
    const float4 lp = lap2d_x4<ST>(src, p, ws, m.lap_scale);
    const float4 lm = lap2d_x4<ST>(mu, p, ws, m.lap_scale);
    mc_update(ps.x, c.x, lp.x, lm.x, m, val[0].x, val[1].x);
    mc_update(ps.y, c.y, lp.y, lm.y, m, val[0].y, val[1].y);
    mc_update(ps.z, c.z, lp.z, lm.z, m, val[0].z, val[1].z);
    mc_update(ps.w, c.w, lp.w, lm.w, m, val[0].w, val[1].w);
  } else {
    const float4 u = *reinterpret_cast<const float4*>(src + p);
    const float4 v = *reinterpret_cast<const float4*>(src + pl + p);
    const float4 lu = lap2d_x4<ST>(src, p, ws, m.lap_scale);
    const float4 lv = lap2d_x4<ST>(src + pl, p, ws, m.lap_scale);
    gs_update(u.x, v.x, lu.x, lv.x, m, val[0].x, val[1].x);
    gs_update(u.y, v.y, lu.y, lv.y, m, val[0].y, val[1].y);
    gs_update(u.z, v.z, lu.z, lv.z, m, val[0].z, val[1].z);
    gs_update(u.w, v.w, lu.w, lv.w, m, val[0].w, val[1].w);
  }
}

// k forward-Euler sub-steps of one tile; the last one is written to `out` (sites beyond
// nx, ny are computed on periodic images and not stored).
template <int MODEL, int K, int TX, int TY, int ST = PF_ST_STD>
__device__ __forceinline__ void fe2d_tile(const FieldPtrs& in, const FieldOut& out, int nx,
                                          int ny, int64_t pitch, int x0, int y0,
                                          const ModelParams& m, float* sm) {
  using C = Cfg2<MODEL, K, TX, TY, ST>;
  constexpr int WS = C::WS;
  constexpr int PL = C::PL;
  load_region2d<C>(in, nx, ny, pitch, x0, y0, sm);
  __syncthreads();
#pragma unroll
  for (int s = 0; s < K; ++s) {
    const float* src = sm + (s & 1) * C::NF * PL;
    float* dst = sm + ((s + 1) & 1) * C::NF * PL;
    float* mu = sm + C::NF * C::NBUF * PL;
    if constexpr (MODEL == PF_MODEL_CH || MODEL == PF_MODEL_C) {
      // mu on the region one stencil radius wider than this sub-step's update
      const int rlo = C::R * s + C::RS, rhi = C::HT - rlo;
      const int clo = (C::HP - C::H + C::R * s + C::RS) / 4;
      const int chi = (WS - (C::HP - C::H + C::R * s + C::RS) + 3) / 4;
      const int nch = chi - clo;
      auto mu_rows = [&](const int nrows, const int ncols) {
        for (int i = threadIdx.x; i < nrows * ncols; i += kNT2) {
          const int rr = i / ncols;
          const int p = (rlo + rr) * WS + 4 * (clo + i - rr * ncols);
          site4_mu<MODEL, ST>(src, p, WS, PL, m, mu);
        }
      };
      // mu is needed R (K-1-s) + RS past the grid's last row and column, no further
      const int marg = C::R * (K - 1 - s) + C::RS;
      const int rhi_e = min(rhi, C::H + (ny - y0) + marg);
      const int chi_e = min(chi, (C::HP + (nx - x0) + marg + 3) / 4);
      if (rhi_e == rhi && chi_e == chi) mu_rows(rhi - rlo, nch);  // compile-time bounds
      else if (rhi_e > rlo && chi_e > clo) mu_rows(rhi_e - rlo, chi_e - clo);
      __syncthreads();
    }
    const bool last = (s == K - 1);
    const int rlo = C::R * (s + 1), rhi = C::HT - rlo;
    const int clo = last ? C::HP / 4 : (C::HP - C::H + C::R * (s + 1)) / 4;
    const int chi = last ? (C::HP + TX) / 4 : (WS - (C::HP - C::H + C::R * (s + 1)) + 3) / 4;
    const int nch = chi - clo;
    // A tile that reaches past the grid's last row or column (small or ragged grids, batch
    // instances) skips the sites more than R (K-1-s) past it: they never reach a stored
    // value. Tiles inside the grid keep the compile-time bounds.
    const int marg = C::R * (K - 1 - s);
    const int rhi_e = min(rhi, C::H + (ny - y0) + marg);
    const int chi_e = min(chi, (C::HP + (nx - x0) + marg + 3) / 4);
    auto update_rows = [&](const int nrows, const int ncols) {
    for (int i = threadIdx.x; i < nrows * ncols; i += kNT2) {
      const int rr = i / ncols;
      const int r = rlo + rr;
      const int j = clo + i - rr * ncols;
      const int p = r * WS + 4 * j;
      float4 val[C::NF];
      site4_update<MODEL, ST>(src, mu, p, WS, PL, m, val);
      if (last) {
        const int gx = x0 + 4 * j - C::HP;
        const int gy = y0 + r - C::H;
        if (gy < ny) {
          const int64_t off = (int64_t)gy * pitch + gx;
          if (gx + 3 < nx) {
#pragma unroll
            for (int f = 0; f < C::NF; ++f) *reinterpret_cast<float4*>(out.f[f] + off) = val[f];
          } else {
#pragma unroll
            for (int f = 0; f < C::NF; ++f) {
              if (gx < nx) out.f[f][off] = val[f].x;
              if (gx + 1 < nx) out.f[f][off + 1] = val[f].y;
              if (gx + 2 < nx) out.f[f][off + 2] = val[f].z;
            }
          }
        }
      } else {
#pragma unroll
        for (int f = 0; f < C::NF; ++f) *reinterpret_cast<float4*>(dst + f * PL + p) = val[f];
      }
    }
    };
    if (rhi_e == rhi && chi_e == chi) update_rows(rhi - rlo, nch);  // compile-time bounds
    else if (rhi_e > rlo && chi_e > clo) update_rows(rhi_e - rlo, chi_e - clo);
    if (!last) __syncthreads();
  }
}

}  // namespace pf
