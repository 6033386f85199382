// 3D forward-Euler step for the radius-2 models, Model B (Cahn-Hilliard) and Model C (the
// eutectic model: psi coupled to a conserved m), with TMA plane staging (Sec. 2.4.1 solver,
// Sec. 2.2.2 7-point Laplacian, Sec. 3 models).
//
// The right-hand side needs the Laplacian of a chemical potential mu (of phi in Model B, of m
// in Model C), which itself holds a Laplacian, so a site's update reads the field two sites
// away. mu is computed on chip and never stored: on the tile plus a one-site ring (without
// its corners, which no 7-point Laplacian reads), from the staged planes.
//
// Work: TX x TY columns of the xy plane times z-chunks, one CTA per (column, chunk) item,
// chunks alternating up and down in z (as the radius-1 TMA kernel). Per input plane and field,
// TMA brings into an NS-stage ring: rows y0-2 .. y0+TY+1 of the tile's columns (a 2-row box,
// the TX x TY interior, a 2-row box), the 4-wide column boxes left and right of rows
// y0 .. y0+TY-1, and four 4 x 1 corner boxes (columns left and right, rows y0-1 and y0+TY),
// every box at wrapped coordinates and in its own 128-byte aligned slot. One thread issues
// them NS planes ahead; consumers wait on the stage's mbarrier (bounded).
//
// Per output plane z (one CTA barrier): mu(z+1) on the tile and its ring into one of two mu
// planes in shared memory (the other holds mu(z), written the iteration before), then the
// update of plane z: the Laplacian of mu(z) with its in-plane neighbours from shared memory
// and its z-neighbours mu(z-1), mu(z+1) from this thread's registers, and for Model C the
// Laplacian of psi from the staged planes z-1, z, z+1. Each thread owns a float4 of x in one
// row; x-neighbours come from the lanes on either side (warp shuffle) and from the column
// boxes (or the mu ring) at the tile edge. The per-site functions are those of every other
// kernel, in the same operand order, so the result is the general 3D kernel's bit for bit.
//
// Requires nx % TX == 0 and ny % TY == 0 (the host falls back to the general kernel).
#include "pf_grid.h"
#include "pf_internal.h"
#include "pf_tma.cuh"

#include <cudaTypedefs.h>

namespace pf {

namespace {

template <int MODEL, int TX, int TY, int NS>
struct CfgR2 {
  static constexpr int NF = ModelTraits<MODEL>::NF;
  static constexpr int LX = TX / 4;                 // threads per row
  static constexpr int NT = LX * TY;                // threads per CTA
  static constexpr int MAIN = (TY + 4) * TX;        // rows y0-2 .. y0+TY+1
  static constexpr int SIDE = TY * 4;               // a 4-wide column box, rows y0 .. y0+TY-1
  static constexpr int CORNER = 32;                 // a 4 x 1 box in a 128-byte slot
  static constexpr int SL = MAIN, SR = MAIN + SIDE;  // left and right column boxes
  static constexpr int CLT = MAIN + 2 * SIDE;        // corners: left/right of row y0-1,
  static constexpr int CRT = CLT + CORNER;           //          left/right of row y0+TY
  static constexpr int CLB = CRT + CORNER;
  static constexpr int CRB = CLB + CORNER;
  static constexpr int FIELD = MAIN + 2 * SIDE + 4 * CORNER;  // floats per field per stage
  static constexpr int STAGE = NF * FIELD;
  static constexpr uint32_t TX_BYTES = NF * (MAIN + 2 * SIDE + 4 * 4) * 4;  // bytes landed
  static constexpr int MW = TX + 8;        // mu row: ring column at 3, tile at 4 .. TX+3, ring at TX+4
  static constexpr int MPL = (TY + 2) * MW;  // mu plane: ring row, TY rows, ring row
  static constexpr size_t SMEM = (size_t)(NS * STAGE + 2 * MPL) * 4 + NS * 8 + 128;
  static_assert(TX % 32 == 0 && (TY * 16) % 128 == 0, "every box starts 128-byte aligned");
  static_assert(MODEL == PF_MODEL_CH || MODEL == PF_MODEL_C, "radius-2 models");
};

// Chemical potential of four sites (Model B: of phi; Model C: of m, coupled to psi).
template <int MODEL>
__device__ __forceinline__ float4 mu4(const float4& psi, const float4& f, const float4& l,
                                      const ModelParams& m) {
  if constexpr (MODEL == PF_MODEL_CH) {
    return make_float4(ch_mu(f.x, l.x, m), ch_mu(f.y, l.y, m), ch_mu(f.z, l.z, m),
                       ch_mu(f.w, l.w, m));
  } else {
    return make_float4(mc_mu(psi.x, f.x, l.x, m), mc_mu(psi.y, f.y, l.y, m),
                       mc_mu(psi.z, f.z, l.z, m), mc_mu(psi.w, f.w, l.w, m));
  }
}

template <int MODEL>
__device__ __forceinline__ float mu1(float psi, float f, float l, const ModelParams& m) {
  if constexpr (MODEL == PF_MODEL_CH)
    return ch_mu(f, l, m);
  else
    return mc_mu(psi, f, l, m);
}

// 7-point Laplacians of four sites (operand order of lap3d: centre, x-, x+, y-, y+, z-, z+).
__device__ __forceinline__ float4 lap4(const float4& c, float xm, float xp, const float4& ym,
                                       const float4& yp, const float4& zm, const float4& zp,
                                       float s) {
  return make_float4(lap3d(c.x, xm, c.y, ym.x, yp.x, zm.x, zp.x, s),
                     lap3d(c.y, c.x, c.z, ym.y, yp.y, zm.y, zp.y, s),
                     lap3d(c.z, c.y, c.w, ym.z, yp.z, zm.z, zp.z, s),
                     lap3d(c.w, c.z, xp, ym.w, yp.w, zm.w, zp.w, s));
}

__device__ __forceinline__ float4 ld4s(const float* p) {
  return *reinterpret_cast<const float4*>(p);
}

template <int MODEL, int TX, int TY, int NS>
__global__ void __launch_bounds__(CfgR2<MODEL, TX, TY, NS>::NT)
    fe3d_tma_r2_kernel(const __grid_constant__ Tma2Maps maps, FieldOut out, Geom g,
                       ModelParams m, int tiles_x, int nchunks, int chunk_len, int* err_flag) {
  using C = CfgR2<MODEL, TX, TY, NS>;
  constexpr int NF = C::NF;
  constexpr int LX = C::LX;
  constexpr int FM = NF - 1;  // the field under mu: phi (Model B) or m (Model C)
  constexpr int MW = C::MW;
  extern __shared__ unsigned char smem_raw[];
  const uint32_t base_sa = smem_addr(smem_raw);
  float* ring = reinterpret_cast<float*>(smem_raw + ((128 - (base_sa & 127)) & 127));
  float* mupl = ring + NS * C::STAGE;  // two mu planes
  uint64_t* bars = reinterpret_cast<uint64_t*>(mupl + 2 * C::MPL);

  const int tid = threadIdx.x;
  const int tx4 = tid % LX;
  const int ty = tid / LX;
  canary_fill(ring, (size_t)NS * C::STAGE + 2 * C::MPL);  // TMA issues follow a proxy fence
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) mbar_init(&bars[s], 1);
    mbar_fence_init();
  }
  __syncthreads();

  uint32_t q_base = 0, q_issued = 0;
  bool err = false;
  auto stage_ptr = [&](uint32_t q) { return ring + (q % NS) * C::STAGE; };
  auto issue = [&](uint32_t q, int x0, int y0, int p) {
    float* st = stage_ptr(q);
    uint64_t* bar = &bars[q % NS];
    const int z = wrap_index(p, g.nz);
    const int ym2 = wrap_index(y0 - 2, g.ny), ym1 = wrap_index(y0 - 1, g.ny);
    const int yb = wrap_index(y0 + TY, g.ny);
    const int xl = wrap_index(x0 - 4, g.nx), xr = wrap_index(x0 + TX, g.nx);
    mbar_arrive_expect_tx(bar, C::TX_BYTES);
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      float* fs = st + f * C::FIELD;
      tma_load_3d(fs, &maps.row2[f], x0, ym2, z, bar);
      tma_load_3d(fs + 2 * TX, &maps.inner[f], x0, y0, z, bar);
      tma_load_3d(fs + (TY + 2) * TX, &maps.row2[f], x0, yb, z, bar);
      tma_load_3d(fs + C::SL, &maps.side[f], xl, y0, z, bar);
      tma_load_3d(fs + C::SR, &maps.side[f], xr, y0, z, bar);
      tma_load_3d(fs + C::CLT, &maps.corner[f], xl, ym1, z, bar);
      tma_load_3d(fs + C::CRT, &maps.corner[f], xr, ym1, z, bar);
      tma_load_3d(fs + C::CLB, &maps.corner[f], xl, yb, z, bar);
      tma_load_3d(fs + C::CRB, &maps.corner[f], xr, yb, z, bar);
    }
  };
  auto wait = [&](uint32_t q) -> bool {
    return mbar_wait_bounded(&bars[q % NS], (q / NS) & 1u, kWaitBudgetCycles);
  };
  // staged value of a field at tile-relative (x, y): main block for 0 <= x < TX, y in
  // [-2, TY+1]; left column x = -1 or -2 and right column x = TX or TX+1 for y in [0, TY),
  // and x = -1 or TX at y = -1 and y = TY from the corner boxes
  auto mainp = [](const float* F, int y, int x) { return F + (y + 2) * TX + x; };
  auto left = [](const float* F, int y, int c) -> float {  // c = 3: x0-1, c = 2: x0-2
    if (y < 0) return F[C::CLT + c];
    if (y >= TY) return F[C::CLB + c];
    return F[C::SL + y * 4 + c];
  };
  auto right = [](const float* F, int y, int c) -> float {  // c = 0: x0+TX, c = 1: x0+TX+1
    if (y < 0) return F[C::CRT + c];
    if (y >= TY) return F[C::CRB + c];
    return F[C::SR + y * 4 + c];
  };

  // mu of the plane staged at zc (neighbours zb, za) into mu plane `dst`: every thread its
  // interior float4 (returned), and the ring items spread over the first threads.
  auto mu_plane = [&](const float* zb, const float* zc, const float* za, float* dst) -> float4 {
    const float* Fb = zb + FM * C::FIELD;
    const float* Fc = zc + FM * C::FIELD;
    const float* Fa = za + FM * C::FIELD;
    const float* Pc = zc;  // psi (Model C)
    const float4 c = ld4s(mainp(Fc, ty, 4 * tx4));
    float xm = __shfl_up_sync(0xffffffffu, c.w, 1, LX);
    float xp = __shfl_down_sync(0xffffffffu, c.x, 1, LX);
    if (tx4 == 0) xm = left(Fc, ty, 3);
    if (tx4 == LX - 1) xp = right(Fc, ty, 0);
    const float4 l = lap4(c, xm, xp, ld4s(mainp(Fc, ty - 1, 4 * tx4)),
                          ld4s(mainp(Fc, ty + 1, 4 * tx4)), ld4s(mainp(Fb, ty, 4 * tx4)),
                          ld4s(mainp(Fa, ty, 4 * tx4)), m.lap_scale);
    float4 psi = c;
    if constexpr (MODEL == PF_MODEL_C) psi = ld4s(mainp(Pc, ty, 4 * tx4));
    const float4 mu = mu4<MODEL>(psi, c, l, m);
    *reinterpret_cast<float4*>(dst + (ty + 1) * MW + 4 + 4 * tx4) = mu;
    // ring: rows y = -1 and y = TY as float4 groups, columns x = -1 and x = TX as scalars
    constexpr int NRING = 2 * LX + 2 * TY;
    for (int it = tid; it < NRING; it += C::NT) {
      if (it < 2 * LX) {
        const int y = it < LX ? -1 : TY;
        const int j = it < LX ? it : it - LX;
        const float4 rc = ld4s(mainp(Fc, y, 4 * j));
        const float rxm = j == 0 ? left(Fc, y, 3) : *mainp(Fc, y, 4 * j - 1);
        const float rxp = j == LX - 1 ? right(Fc, y, 0) : *mainp(Fc, y, 4 * j + 4);
        const float4 rl = lap4(rc, rxm, rxp, ld4s(mainp(Fc, y - 1, 4 * j)),
                               ld4s(mainp(Fc, y + 1, 4 * j)), ld4s(mainp(Fb, y, 4 * j)),
                               ld4s(mainp(Fa, y, 4 * j)), m.lap_scale);
        float4 rpsi = rc;
        if constexpr (MODEL == PF_MODEL_C) rpsi = ld4s(mainp(Pc, y, 4 * j));
        *reinterpret_cast<float4*>(dst + (y + 1) * MW + 4 + 4 * j) = mu4<MODEL>(rpsi, rc, rl, m);
      } else {
        const int k = it - 2 * LX;
        const int y = k < TY ? k : k - TY;
        float v, vxm, vxp, vym, vyp, vzm, vza, vpsi;
        if (k < TY) {  // x = -1
          v = left(Fc, y, 3);
          vxm = left(Fc, y, 2);
          vxp = *mainp(Fc, y, 0);
          vym = left(Fc, y - 1, 3);
          vyp = left(Fc, y + 1, 3);
          vzm = left(Fb, y, 3);
          vza = left(Fa, y, 3);
          vpsi = MODEL == PF_MODEL_C ? left(Pc, y, 3) : v;
        } else {  // x = TX
          v = right(Fc, y, 0);
          vxm = *mainp(Fc, y, TX - 1);
          vxp = right(Fc, y, 1);
          vym = right(Fc, y - 1, 0);
          vyp = right(Fc, y + 1, 0);
          vzm = right(Fb, y, 0);
          vza = right(Fa, y, 0);
          vpsi = MODEL == PF_MODEL_C ? right(Pc, y, 0) : v;
        }
        const float rl = lap3d(v, vxm, vxp, vym, vyp, vzm, vza, m.lap_scale);
        dst[(y + 1) * MW + (k < TY ? 3 : TX + 4)] = mu1<MODEL>(vpsi, v, rl, m);
      }
    }
    return mu;
  };

  const int ncols = tiles_x * (g.ny / TY);
  const int nitems = ncols * nchunks;
  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int col = item % ncols;
    const int chunk = item / ncols;
    const int zlo = chunk * chunk_len;
    const int zhi = min(g.nz, zlo + chunk_len);
    if (zlo >= zhi) continue;  // uniform over the CTA
    const int dir = (chunk & 1) ? -1 : 1;
    const int n = zhi - zlo;
    const int zfirst = dir > 0 ? zlo : zhi - 1;
    const int x0 = (col % tiles_x) * TX;
    const int y0 = (col / tiles_x) * TY;
    const int nin = n + 4;  // input planes zfirst - 2 dir .. zlast + 2 dir
    auto in_plane = [&](int i) { return zfirst + (i - 2) * dir; };

    if (__syncthreads_or(err)) break;
    if (tid == 0) {
      fence_proxy_async_smem();
      const int n0 = nin < NS ? nin : NS;
      for (int i = 0; i < n0; ++i) issue(q_base + i, x0, y0, in_plane(i));
      q_issued = q_base + n0;
    }
    // prologue: mu of planes zfirst - dir (this thread's float4 only) and zfirst (the tile
    // and its ring, into mu plane 0)
    float4 mu_m = make_float4(0.f, 0.f, 0.f, 0.f), mu_c = mu_m;
    err = !wait(q_base);
    if (!err) err = !wait(q_base + 1);
    if (!err) err = !wait(q_base + 2);
    err = __any_sync(0xffffffffu, err);  // warp-uniform before the shuffles
    if (!err) mu_m = mu_plane(stage_ptr(q_base), stage_ptr(q_base + 1), stage_ptr(q_base + 2),
                              mupl + C::MPL);  // ring written to plane 1, overwritten below
    if (__syncthreads_or(err)) break;
    err = !wait(q_base + 3);
    err = __any_sync(0xffffffffu, err);
    if (!err) mu_c = mu_plane(stage_ptr(q_base + 1), stage_ptr(q_base + 2), stage_ptr(q_base + 3),
                              mupl);
    const int gy = y0 + ty;
    const int gx = x0 + 4 * tx4;
    for (int o = 0; o < n; ++o) {
      // output plane z (input o + 2); mu(z + dir) from inputs o + 2 .. o + 4 into plane
      // (o + 1) % 2; mu(z) in plane o % 2
      if (__syncthreads_or(err)) break;
      if (tid == 0 && o + NS < nin) {
        fence_proxy_async_smem();
        issue(q_base + o + NS, x0, y0, in_plane(o + NS));
        q_issued = q_base + o + NS + 1;
      }
      err = !wait(q_base + o + 4);
      err = __any_sync(0xffffffffu, err);
      if (err) continue;
      const float* s1 = stage_ptr(q_base + o + 1);
      const float* s2 = stage_ptr(q_base + o + 2);
      const float* s3 = stage_ptr(q_base + o + 3);
      const float* s4 = stage_ptr(q_base + o + 4);
      float* mu_next = mupl + ((o + 1) & 1) * C::MPL;
      const float* mu_cur = mupl + (o & 1) * C::MPL;
      const float4 mu_p = mu_plane(s2, s3, s4, mu_next);
      // Laplacian of mu(z)
      float lxm = __shfl_up_sync(0xffffffffu, mu_c.w, 1, LX);
      float lxp = __shfl_down_sync(0xffffffffu, mu_c.x, 1, LX);
      if (tx4 == 0) lxm = mu_cur[(ty + 1) * MW + 3];
      if (tx4 == LX - 1) lxp = mu_cur[(ty + 1) * MW + TX + 4];
      const float4 lmu = lap4(mu_c, lxm, lxp, ld4s(mu_cur + ty * MW + 4 + 4 * tx4),
                              ld4s(mu_cur + (ty + 2) * MW + 4 + 4 * tx4), mu_m, mu_p,
                              m.lap_scale);
      const int z = zfirst + o * dir;
      const int64_t off = (int64_t)z * g.plane + (int64_t)gy * g.pitch + gx;
      if constexpr (MODEL == PF_MODEL_CH) {
        const float4 p = ld4s(mainp(s2, ty, 4 * tx4));
        *reinterpret_cast<float4*>(out.f[0] + off) =
            make_float4(ch_update(p.x, lmu.x, m), ch_update(p.y, lmu.y, m),
                        ch_update(p.z, lmu.z, m), ch_update(p.w, lmu.w, m));
      } else {
        // Laplacian of psi at plane z from the staged planes z - dir, z, z + dir
        const float4 pc = ld4s(mainp(s2, ty, 4 * tx4));
        float pxm = __shfl_up_sync(0xffffffffu, pc.w, 1, LX);
        float pxp = __shfl_down_sync(0xffffffffu, pc.x, 1, LX);
        if (tx4 == 0) pxm = left(s2, ty, 3);
        if (tx4 == LX - 1) pxp = right(s2, ty, 0);
        const float4 lpsi = lap4(pc, pxm, pxp, ld4s(mainp(s2, ty - 1, 4 * tx4)),
                                 ld4s(mainp(s2, ty + 1, 4 * tx4)), ld4s(mainp(s1, ty, 4 * tx4)),
                                 ld4s(mainp(s3, ty, 4 * tx4)), m.lap_scale);
        const float4 mc = ld4s(mainp(s2 + C::FIELD, ty, 4 * tx4));
        float4 pn, mn;
        mc_update(pc.x, mc.x, lpsi.x, lmu.x, m, pn.x, mn.x);
        mc_update(pc.y, mc.y, lpsi.y, lmu.y, m, pn.y, mn.y);
        mc_update(pc.z, mc.z, lpsi.z, lmu.z, m, pn.z, mn.z);
        mc_update(pc.w, mc.w, lpsi.w, lmu.w, m, pn.w, mn.w);
        *reinterpret_cast<float4*>(out.f[0] + off) = pn;
        *reinterpret_cast<float4*>(out.f[1] + off) = mn;
      }
      mu_m = mu_c;
      mu_c = mu_p;
    }
    q_base += nin;
  }

  if (__syncthreads_or(err)) {
    // A wait ran out: record it, let this CTA's copies in flight land (bounded), return.
    if (tid == 0) {
      atomicExch(err_flag, 1);
      for (uint32_t q = (q_issued > NS ? q_issued - NS : 0); q < q_issued; ++q)
        (void)mbar_wait_bounded(&bars[q % NS], (q / NS) & 1u, kWaitBudgetCycles);
    }
  }
}

template <int MODEL, int TX, int TY, int NS>
cudaError_t launch_r2(pf_grid_s* gr, const Tma2Maps& maps, FieldOut out, cudaStream_t st) {
  using C = CfgR2<MODEL, TX, TY, NS>;
  auto kern = fe3d_tma_r2_kernel<MODEL, TX, TY, NS>;
  static unsigned long long attr_mask = 0;  // per instantiation and device
  cudaError_t e = ensure_smem_attr(kern, C::SMEM, &attr_mask);
  if (e != cudaSuccess) return e;
  static int occ_by_dev[64] = {};  // resident CTAs per SM, per device
  int occ = gr->device < 64 ? occ_by_dev[gr->device] : 0;
  if (occ == 0) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, C::NT, C::SMEM);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    if (gr->device < 64) occ_by_dev[gr->device] = occ;
  }
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, gr->device);
  if (e != cudaSuccess) return e;
  const Geom g = grid_geom(gr);
  const int tiles_x = g.nx / TX;
  const long long ncols = (long long)tiles_x * (g.ny / TY);
  const long long slots = (long long)sms * occ;
  // as many z-chunks as keep every column of a chunk resident at once; a chunk streams 4
  // planes besides its own, so chunks keep at least 4 planes where the grid has them
  // (measured: two-plane chunks and issuing the boxes from all lanes of warp 0 made Model B
  // 256^3 drop from 393 to 247 GLUPS and Model C 64^3 from 9.5 to 12.5 us per step)
  long long nchunks = slots / ncols;
  if (nchunks > g.nz / 4) nchunks = g.nz / 4;
  if (nchunks < 1) nchunks = 1;
  const int chunk_len = (int)((g.nz + nchunks - 1) / nchunks);
  nchunks = (g.nz + chunk_len - 1) / chunk_len;
  const long long items = ncols * nchunks;
  const long long grid = items < slots ? items : slots;
  kern<<<(unsigned)grid, C::NT, C::SMEM, st>>>(maps, out, g, gr->params, tiles_x,
                                                 (int)nchunks, chunk_len, gr->d_err);
  return cudaGetLastError();
}

}  // namespace

// Tensor maps of one ping-pong buffer for the given tile (cached until the tile changes).
cudaError_t tma2_maps(pf_grid_s* gr, int tma_tile, int buf) {
  Tma2Cache& tc = gr->tma2;
  if (tc.tile == tma_tile && tc.valid[buf]) return cudaSuccess;
  if (tc.tile != tma_tile) {
    tc.valid[0] = tc.valid[1] = false;
    tc.tile = tma_tile;
  }
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (encode == nullptr) {
    cudaDriverEntryPointQueryResult qr;
    void* fn = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &qr);
    if (e != cudaSuccess) return e;
    if (qr != cudaDriverEntryPointSuccess || fn == nullptr) return cudaErrorNotSupported;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  int tx, ty;
  tma3d_tile_shape(tma_tile, &tx, &ty);
  const cuuint64_t dims[3] = {(cuuint64_t)gr->nx, (cuuint64_t)gr->ny, (cuuint64_t)gr->nz};
  const cuuint64_t strides[2] = {(cuuint64_t)gr->pitch * 4, (cuuint64_t)gr->plane * 4};
  const cuuint32_t estr[3] = {1, 1, 1};
  const cuuint32_t box_inner[3] = {(cuuint32_t)tx, (cuuint32_t)ty, 1};
  const cuuint32_t box_row2[3] = {(cuuint32_t)tx, 2, 1};
  const cuuint32_t box_side[3] = {4, (cuuint32_t)ty, 1};
  const cuuint32_t box_corner[3] = {4, 1, 1};
  for (int f = 0; f < gr->nf; ++f) {
    void* base = gr->buf[buf][f];
    Tma2Maps& mp = tc.maps[buf];
    struct {
      CUtensorMap* map;
      const cuuint32_t* box;
      CUtensorMapL2promotion promo;
    } list[4] = {{&mp.inner[f], box_inner, CU_TENSOR_MAP_L2_PROMOTION_L2_256B},
                 {&mp.row2[f], box_row2, CU_TENSOR_MAP_L2_PROMOTION_L2_256B},
                 {&mp.side[f], box_side, CU_TENSOR_MAP_L2_PROMOTION_NONE},
                 {&mp.corner[f], box_corner, CU_TENSOR_MAP_L2_PROMOTION_NONE}};
    for (auto& it : list) {
      CUresult r = encode(it.map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides,
                          it.box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, it.promo, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
  }
  tc.valid[buf] = true;
  return cudaSuccess;
}

cudaError_t launch_fe3d_tma_r2(pf_grid_s* gr, int tma_tile, int src, int dst, cudaStream_t st) {
  cudaError_t e = tma2_maps(gr, tma_tile, src);
  if (e != cudaSuccess) return e;
  FieldOut out{};
  for (int f = 0; f < gr->nf; ++f) out.f[f] = gr->buf[dst][f];
  const Tma2Maps& maps = gr->tma2.maps[src];
  if (gr->model == PF_MODEL_CH) {
    switch (tma_tile) {
      case 0: return launch_r2<PF_MODEL_CH, 64, 16, 6>(gr, maps, out, st);
      case 1: return launch_r2<PF_MODEL_CH, 128, 8, 6>(gr, maps, out, st);
      case 2: return launch_r2<PF_MODEL_CH, 128, 16, 6>(gr, maps, out, st);
    }
  } else if (gr->model == PF_MODEL_C) {
    switch (tma_tile) {
      case 0: return launch_r2<PF_MODEL_C, 64, 16, 6>(gr, maps, out, st);
      case 1: return launch_r2<PF_MODEL_C, 128, 8, 6>(gr, maps, out, st);
      case 2: return launch_r2<PF_MODEL_C, 128, 16, 6>(gr, maps, out, st);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace pf
