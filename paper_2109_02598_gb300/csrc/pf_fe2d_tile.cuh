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
#include "pf_tma.cuh"

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

// Stage rows [y0-H, y0+TY+H) x columns [x0-HP, x0+TX+HP) of every field into buffer 0:
// 16-byte copies where the four columns lie inside the grid (x0, HP and the row pitch are
// multiples of 4, so those are 16-byte aligned), four periodic 4-byte copies elsewhere. The
// calling thread's copies are complete when this returns (WAIT; otherwise at the next
// cp_async_wait_all); the caller's barrier then makes every thread's visible.
template <class C, bool WAIT = true>
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
      for (int f = 0; f < C::NF; ++f) cp_async16(dst + f * C::PL, in.f[f] + row + gx);
    } else {
      const int64_t o0 = row + wrap_index(gx, nx), o1 = row + wrap_index(gx + 1, nx);
      const int64_t o2 = row + wrap_index(gx + 2, nx), o3 = row + wrap_index(gx + 3, nx);
#pragma unroll
      for (int f = 0; f < C::NF; ++f) {
        const float* p = in.f[f];
        float* d = dst + f * C::PL;
        cp_async4(d, p + o0);
        cp_async4(d + 1, p + o1);
        cp_async4(d + 2, p + o2);
        cp_async4(d + 3, p + o3);
      }
    }
  }
  if (WAIT) cp_async_wait_all();
}

// 2D Laplacians of four consecutive sites from a float4 row and its neighbours, with the
// stencil ST (its neighbours beyond the float4 come from scalars of the same rows). MODEL
// only matters for Gray-Scott with the standard stencil, whose factor is 1 (lap_scaled).
template <int ST = PF_ST_STD, int MODEL = PF_MODEL_AC>
__device__ __forceinline__ float4 lap2d_x4(const float* s, int p, int ws, float scale) {
  const float4 c = *reinterpret_cast<const float4*>(s + p);
  const float4 u = *reinterpret_cast<const float4*>(s + p - ws);
  const float4 d = *reinterpret_cast<const float4*>(s + p + ws);
  const float l = s[p - 1], r = s[p + 4];
  float4 o;
  if constexpr (ST == PF_ST_STD) {
    o.x = lap_scaled<MODEL>(lap2d_sum(c.x, l, c.y, u.x, d.x), scale);
    o.y = lap_scaled<MODEL>(lap2d_sum(c.y, c.x, c.z, u.y, d.y), scale);
    o.z = lap_scaled<MODEL>(lap2d_sum(c.z, c.y, c.w, u.z, d.z), scale);
    o.w = lap_scaled<MODEL>(lap2d_sum(c.w, c.z, r, u.w, d.w), scale);
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
    const float4 lu = lap2d_x4<ST, MODEL>(src, p, ws, m.lap_scale);
    const float4 lv = lap2d_x4<ST, MODEL>(src + pl, p, ws, m.lap_scale);
    gs_update(u.x, v.x, lu.x, lv.x, m, val[0].x, val[1].x);
    gs_update(u.y, v.y, lu.y, lv.y, m, val[0].y, val[1].y);
    gs_update(u.z, v.z, lu.z, lv.z, m, val[0].z, val[1].z);
    gs_update(u.w, v.w, lu.w, lv.w, m, val[0].w, val[1].w);
  }
}

// ---- row strips (standard 5-point stencil) ----------------------------------------
// A thread walks a vertical strip of one column group and keeps the rows above, at and below
// the current site in registers: one float4 row load per site group and Laplacian instead of
// three. The per-site arithmetic is that of lap2d_x4, site4_mu and site4_update, bit for bit.

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }

// Strips are taken once each holds at least this many rows (ceil(nrows / S) >= 3, i.e.
// nrows > 2 S): shorter ones lengthen a thread's dependent chain more than they save loads
// (measured: 64x16 tiles at k = 4 with 2-row strips, 10 % slower; 128x16 tiles at k = 4 with
// 3-4-row strips, 1-2 % faster).
constexpr int kMinStripRows = 3;

// Laplacians of a float4 group from its row (c), the rows above (u) and below (d) and its two
// x-edge scalars: lap2d_x4<PF_ST_STD, MODEL>'s arithmetic.
template <int MODEL = PF_MODEL_AC>
__device__ __forceinline__ float4 lap4_rows(const float4& c, const float4& u, const float4& d,
                                            float l, float r, float scale) {
  float4 o;
  o.x = lap_scaled<MODEL>(lap2d_sum(c.x, l, c.y, u.x, d.x), scale);
  o.y = lap_scaled<MODEL>(lap2d_sum(c.y, c.x, c.z, u.y, d.y), scale);
  o.z = lap_scaled<MODEL>(lap2d_sum(c.z, c.y, c.w, u.z, d.z), scale);
  o.w = lap_scaled<MODEL>(lap2d_sum(c.w, c.z, r, u.w, d.w), scale);
  return o;
}

// Thread t's strip of a region of nrows rows from rlo and ncols column groups from clo:
// column group clo + t % ncols, rows [r0, r1) of strip t / ncols (S = kNT2 / ncols strips of
// ceil(nrows / S) rows; threads beyond S ncols get none).
struct Strip {
  int j, r0, r1;
};

__device__ __forceinline__ Strip strip_of(int rlo, int nrows, int clo, int ncols) {
  Strip st;
  const int S = kNT2 / ncols;
  const int q = threadIdx.x / ncols;
  st.j = clo + (threadIdx.x - q * ncols);
  if (q >= S) {
    st.r0 = st.r1 = 0;
    return st;
  }
  const int L = (nrows + S - 1) / S;
  st.r0 = rlo + q * L;
  st.r1 = min(rlo + nrows, st.r0 + L);
  return st;
}

// site4_mu down a strip.
template <int MODEL>
__device__ __forceinline__ void mu_strip(const float* src, int ws, int pl, const Strip& st,
                                         const ModelParams& m, float* mu) {
  if (st.r0 >= st.r1) return;
  const float* A = MODEL == PF_MODEL_CH ? src : src + pl;  // the field under the Laplacian
  int p = st.r0 * ws + 4 * st.j;
  float4 u = ld4(A + p - ws), c = ld4(A + p);
  for (int r = st.r0; r < st.r1; ++r, p += ws) {
    const float4 d = ld4(A + p + ws);
    const float4 l = lap4_rows(c, u, d, A[p - 1], A[p + 4], m.lap_scale);
    if constexpr (MODEL == PF_MODEL_CH) {
      *reinterpret_cast<float4*>(mu + p) = make_float4(ch_mu(c.x, l.x, m), ch_mu(c.y, l.y, m),
                                                       ch_mu(c.z, l.z, m), ch_mu(c.w, l.w, m));
    } else {
      const float4 ps = ld4(src + p);
      *reinterpret_cast<float4*>(mu + p) =
          make_float4(mc_mu(ps.x, c.x, l.x, m), mc_mu(ps.y, c.y, l.y, m),
                      mc_mu(ps.z, c.z, l.z, m), mc_mu(ps.w, c.w, l.w, m));
    }
    u = c;
    c = d;
  }
}

// site4_update down a strip; emit(r, j, p, val) stores each group's new values.
template <int MODEL, class Emit>
__device__ __forceinline__ void update_strip(const float* src, const float* mu, int ws, int pl,
                                             const Strip& st, const ModelParams& m, Emit&& emit) {
  if (st.r0 >= st.r1) return;
  constexpr int NF = ModelTraits<MODEL>::NF;
  constexpr bool TWO = MODEL == PF_MODEL_GS || MODEL == PF_MODEL_C;  // two Laplacians
  const float* A0 = MODEL == PF_MODEL_CH ? mu : src;        // AC, GS: phi / u; C: psi
  const float* A1 = MODEL == PF_MODEL_GS ? src + pl : mu;   // GS: v; C: mu
  int p = st.r0 * ws + 4 * st.j;
  float4 u0 = ld4(A0 + p - ws), c0 = ld4(A0 + p);
  float4 u1 = make_float4(0.f, 0.f, 0.f, 0.f), c1 = u1;
  if constexpr (TWO) {
    u1 = ld4(A1 + p - ws);
    c1 = ld4(A1 + p);
  }
  for (int r = st.r0; r < st.r1; ++r, p += ws) {
    const float4 d0 = ld4(A0 + p + ws);
    const float4 l0 = lap4_rows<MODEL>(c0, u0, d0, A0[p - 1], A0[p + 4], m.lap_scale);
    float4 d1 = d0, l1 = l0;
    if constexpr (TWO) {
      d1 = ld4(A1 + p + ws);
      l1 = lap4_rows<MODEL>(c1, u1, d1, A1[p - 1], A1[p + 4], m.lap_scale);
    }
    float4 val[NF];
    if constexpr (MODEL == PF_MODEL_AC) {
      val[0] = make_float4(ac_update(c0.x, l0.x, m), ac_update(c0.y, l0.y, m),
                           ac_update(c0.z, l0.z, m), ac_update(c0.w, l0.w, m));
    } else if constexpr (MODEL == PF_MODEL_CH) {
      const float4 c = ld4(src + p);
      val[0] = make_float4(ch_update(c.x, l0.x, m), ch_update(c.y, l0.y, m),
                           ch_update(c.z, l0.z, m), ch_update(c.w, l0.w, m));
    } else if constexpr (MODEL == PF_MODEL_C) {
      const float4 cm = ld4(src + pl + p);
      mc_update(c0.x, cm.x, l0.x, l1.x, m, val[0].x, val[1].x);
      mc_update(c0.y, cm.y, l0.y, l1.y, m, val[0].y, val[1].y);
      mc_update(c0.z, cm.z, l0.z, l1.z, m, val[0].z, val[1].z);
      mc_update(c0.w, cm.w, l0.w, l1.w, m, val[0].w, val[1].w);
    } else {
      gs_update(c0.x, c1.x, l0.x, l1.x, m, val[0].x, val[1].x);
      gs_update(c0.y, c1.y, l0.y, l1.y, m, val[0].y, val[1].y);
      gs_update(c0.z, c1.z, l0.z, l1.z, m, val[0].z, val[1].z);
      gs_update(c0.w, c1.w, l0.w, l1.w, m, val[0].w, val[1].w);
    }
    emit(r, st.j, p, val);
    u0 = c0;
    c0 = d0;
    if constexpr (TWO) {
      u1 = c1;
      c1 = d1;
    }
  }
}

// ---- full rows with periodic halo columns (the on-chip kernels) ---------------------
// A staged full row holds nx values from column HP on, with HP halo columns per side that
// are periodic copies of the row's other end.

// Store the float4 at staged column 4j + HP of a row, and its periodic copy when the column
// lies within HP of either row end.
template <int HP>
__device__ __forceinline__ void put_row4(float* row, int j, int nx, float4 v) {
  const int c = 4 * j;
  *reinterpret_cast<float4*>(row + HP + c) = v;
  if (c < HP) *reinterpret_cast<float4*>(row + HP + nx + c) = v;
  if (c >= nx - HP) *reinterpret_cast<float4*>(row + c - (nx - HP)) = v;
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
  static_assert(WS / 4 <= kNT2, "a row's column groups must fit the CTA (row strips)");
  canary_fill(sm, C::SMEM_FLOATS);
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
        if (ST == PF_ST_STD && nrows > (kMinStripRows - 1) * (kNT2 / ncols)) {
          mu_strip<MODEL>(src, WS, PL, strip_of(rlo, nrows, clo, ncols), m, mu);
        } else {
          for (int i = threadIdx.x; i < nrows * ncols; i += kNT2) {
            const int rr = i / ncols;
            const int p = (rlo + rr) * WS + 4 * (clo + i - rr * ncols);
            site4_mu<MODEL, ST>(src, p, WS, PL, m, mu);
          }
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
    auto emit = [&](const int r, const int j, const int p, const float4* val) {
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
    };
    auto update_rows = [&](const int nrows, const int ncols) {
      if (ST == PF_ST_STD && nrows > (kMinStripRows - 1) * (kNT2 / ncols)) {
        update_strip<MODEL>(src, mu, WS, PL, strip_of(rlo, nrows, clo, ncols), m, emit);
      } else {
        for (int i = threadIdx.x; i < nrows * ncols; i += kNT2) {
          const int rr = i / ncols;
          const int j = clo + i - rr * ncols;
          const int p = (rlo + rr) * WS + 4 * j;
          float4 val[C::NF];
          site4_update<MODEL, ST>(src, mu, p, WS, PL, m, val);
          emit(rlo + rr, j, p, val);
        }
      }
    };
    if (rhi_e == rhi && chi_e == chi) update_rows(rhi - rlo, nch);  // compile-time bounds
    else if (rhi_e > rlo && chi_e > clo) update_rows(rhi_e - rlo, chi_e - clo);
    if (!last) __syncthreads();
  }
}

}  // namespace pf
