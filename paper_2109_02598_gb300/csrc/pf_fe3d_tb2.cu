// 3D forward-Euler with temporal blocking of depth 2 for the radius-1 models (Allen-Cahn,
// Gray-Scott): two time steps per pass over HBM (Sec. 2.4.1 solver, Sec. 2.2.2 7-point
// Laplacian), so HBM traffic per lattice-site update halves to 4 NF bytes.
//
// Tiles span whole x-rows (W = nx, 128 or 256), so the periodic wrap in x is an index wrap
// inside shared memory; a CTA owns TY rows and streams a z-chunk (even chunks up, odd
// chunks down, as in the depth-1 kernel).  Per input plane, TMA brings rows
// y0-2 .. y0+TY+1 of every field (three boxes: two rows above, the TY rows, two rows
// below, wrapped in y) into an NS-stage ring.  Thread (x4, r), r = 0 .. TY+1, computes the
// first time level on row y0-1+r (one ring wider than the tile in y) and stores it to a
// three-plane ring in shared memory; threads r = 1 .. TY then compute the second level on
// row y0-1+r from that ring and write it to HBM.  Both levels keep their z-neighbours in
// registers (each thread reads the planes of its own column), and the same per-site
// functions as every other kernel make the result bitwise identical to two depth-1 steps.
//
// Requires nx == W, ny % TY == 0 and ny >= 2.
#include "pf_grid.h"
#include "pf_internal.h"
#include "pf_tma.cuh"

#include <cudaTypedefs.h>

namespace pf {

namespace {

template <int MODEL, int W, int TY, int NS>
struct CfgB {
  static constexpr int NF = ModelTraits<MODEL>::NF;
  static constexpr int LX = W / 4;              // float4 columns per row
  static constexpr int NT = LX * (TY + 2);      // one thread per first-level column
  static constexpr int IN_ROWS = TY + 4;        // staged input rows (halo 2)
  static constexpr int IN_FIELD = IN_ROWS * W;  // floats per field per input stage
  static constexpr int IN_STAGE = NF * IN_FIELD;
  static constexpr int L1_ROWS = TY + 2;
  static constexpr int L1_FIELD = L1_ROWS * W;
  static constexpr int L1_PLANE = NF * L1_FIELD;
  static constexpr uint32_t TX_BYTES = IN_STAGE * 4;
  static constexpr size_t SMEM =
      (size_t)(NS * IN_STAGE + 3 * L1_PLANE) * 4 + NS * 8 + 128;  // + barriers + align
  static_assert(W % 32 == 0, "rows must be 128-byte multiples");
};

// x-neighbour scalars of the float4 at column 4*x4 in a row of W floats (periodic).
template <int W>
__device__ __forceinline__ void x_edges(const float* row, int x4, float& xm, float& xp) {
  xm = row[x4 == 0 ? W - 1 : 4 * x4 - 1];
  xp = row[x4 == W / 4 - 1 ? 0 : 4 * x4 + 4];
}

template <int MODEL>
__device__ __forceinline__ void update4(const float4* c, const float4* lap, float4* res,
                                        const ModelParams& m) {
  if constexpr (MODEL == PF_MODEL_AC) {
    res[0].x = ac_update(c[0].x, lap[0].x, m);
    res[0].y = ac_update(c[0].y, lap[0].y, m);
    res[0].z = ac_update(c[0].z, lap[0].z, m);
    res[0].w = ac_update(c[0].w, lap[0].w, m);
  } else {
    gs_update(c[0].x, c[1].x, lap[0].x, lap[1].x, m, res[0].x, res[1].x);
    gs_update(c[0].y, c[1].y, lap[0].y, lap[1].y, m, res[0].y, res[1].y);
    gs_update(c[0].z, c[1].z, lap[0].z, lap[1].z, m, res[0].z, res[1].z);
    gs_update(c[0].w, c[1].w, lap[0].w, lap[1].w, m, res[0].w, res[1].w);
  }
}

// 7-point Laplacians of four sites: centre c, z-neighbours zm/zp, rows above/below and the
// two x-edge scalars of the centre row. The multiply by lap_scale stays even for Gray-Scott
// (whose factor is 1, so the bits are those of lap_scaled): leaving it out measured 1.3 %
// slower in this kernel (476 against 482 GLUPS on GS 256^3).
__device__ __forceinline__ float4 lap3d_x4(const float4& c, const float4& ym, const float4& yp,
                                           const float4& zm, const float4& zp, float xm,
                                           float xp, float lap_scale) {
  float4 l;
  l.x = lap3d(c.x, xm, c.y, ym.x, yp.x, zm.x, zp.x, lap_scale);
  l.y = lap3d(c.y, c.x, c.z, ym.y, yp.y, zm.y, zp.y, lap_scale);
  l.z = lap3d(c.z, c.y, c.w, ym.z, yp.z, zm.z, zp.z, lap_scale);
  l.w = lap3d(c.w, c.z, xp, ym.w, yp.w, zm.w, zp.w, lap_scale);
  return l;
}

template <int MODEL, int W, int TY, int NS>
__global__ void __launch_bounds__(CfgB<MODEL, W, TY, NS>::NT, 1)
    fe3d_tb2_kernel(const __grid_constant__ Tb2Maps maps, FieldOut out, Geom g, ModelParams m,
                    int nchunks, int chunk_len, int balanced, int* err_flag) {
  using C = CfgB<MODEL, W, TY, NS>;
  constexpr int NF = C::NF;
  constexpr int LX = C::LX;
  extern __shared__ unsigned char smem_raw[];
  const uint32_t base_sa = smem_addr(smem_raw);
  float* ring = reinterpret_cast<float*>(smem_raw + ((128 - (base_sa & 127)) & 127));
  float* l1 = ring + NS * C::IN_STAGE;  // three first-level planes
  uint64_t* bars = reinterpret_cast<uint64_t*>(l1 + 3 * C::L1_PLANE);

  const int tid = threadIdx.x;
  const int x4 = tid % LX;
  const int r = tid / LX;  // first-level row y0 - 1 + r; input row r + 1
  const bool second = (r >= 1 && r <= TY);
  canary_fill(ring, (size_t)NS * C::IN_STAGE + 3 * C::L1_PLANE);  // TMA issues follow a proxy fence
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) mbar_init(&bars[s], 1);
    mbar_fence_init();
  }
  __syncthreads();

  uint32_t q_base = 0, q_issued = 0;
  bool err = false;
  auto stage_ptr = [&](uint32_t q) { return ring + (q % NS) * C::IN_STAGE; };
  auto issue = [&](uint32_t q, int y0, int p) {
    float* st = stage_ptr(q);
    uint64_t* bar = &bars[q % NS];
    const int z = wrap_index(p, g.nz);
    const int ytop = wrap_index(y0 - 2, g.ny);
    const int ybot = wrap_index(y0 + TY, g.ny);
    mbar_arrive_expect_tx(bar, C::TX_BYTES);
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      float* fs = st + f * C::IN_FIELD;
      tma_load_3d(fs, &maps.row2[f], 0, ytop, z, bar);
      tma_load_3d(fs + 2 * W, &maps.inner[f], 0, y0, z, bar);
      tma_load_3d(fs + (TY + 2) * W, &maps.row2[f], 0, ybot, z, bar);
    }
  };
  auto wait = [&](uint32_t q) -> bool {
    return mbar_wait_bounded(&bars[q % NS], (q / NS) & 1u, kWaitBudgetCycles);
  };

  const int ncols = g.ny / TY;
  const int nitems = ncols * nchunks;
  // Work: (row tile, z-range) segments. Item mode: item = (tile, chunk of chunk_len planes),
  // items dealt round-robin over the CTAs, chunks alternating up and down. Balanced mode:
  // the (tile, plane) units in tile-major order cut into gridDim.x equal ranges, one per CTA
  // (a range crossing a tile boundary makes two segments), direction alternating by CTA.
  // units = ny nz / TY < 2^31 for every grid this kernel takes (nx = W, at most 2^36 sites)
  const int units = ncols * g.nz;
  int pos = (int)((int64_t)units * blockIdx.x / gridDim.x);
  const int pos_end = (int)((int64_t)units * (blockIdx.x + 1) / gridDim.x);
  int item = blockIdx.x;
  for (;;) {
    int col, zlo, zhi, dir;
    if (balanced) {
      if (pos >= pos_end) break;
      col = pos / g.nz;
      zlo = pos - col * g.nz;
      zhi = min(g.nz, zlo + (pos_end - pos));
      dir = (blockIdx.x & 1) ? -1 : 1;
      pos += zhi - zlo;
    } else {
      if (item >= nitems) break;
      col = item % ncols;
      const int chunk = item / ncols;
      zlo = chunk * chunk_len;
      zhi = min(g.nz, zlo + chunk_len);
      dir = (chunk & 1) ? -1 : 1;
      item += gridDim.x;
      if (zlo >= zhi) continue;  // uniform over the CTA
    }
    const int n = zhi - zlo;                  // output planes
    const int zfirst = dir > 0 ? zlo : zhi - 1;
    const int y0 = col * TY;
    const int nin = n + 4;                    // input planes zfirst-2dir .. zlast+2dir
    auto in_plane = [&](int i) { return zfirst + (i - 2) * dir; };

    if (__syncthreads_or(err)) break;
    if (tid == 0) {
      fence_proxy_async_smem();
      const int n0 = nin < NS ? nin : NS;
      for (int i = 0; i < n0; ++i) issue(q_base + i, y0, in_plane(i));
      q_issued = q_base + n0;
    }
    // prologue: centre values of input planes 0 and 1 for this thread's column
    float4 izm[NF], ic[NF], lzm[NF], lc[NF];
    err = !wait(q_base);
    if (!err) {
      const float* st = stage_ptr(q_base);
#pragma unroll
      for (int f = 0; f < NF; ++f)
        izm[f] = *reinterpret_cast<const float4*>(st + f * C::IN_FIELD + (r + 1) * W + 4 * x4);
      err = !wait(q_base + 1);
    }
    if (!err) {
      const float* st = stage_ptr(q_base + 1);
#pragma unroll
      for (int f = 0; f < NF; ++f)
        ic[f] = *reinterpret_cast<const float4*>(st + f * C::IN_FIELD + (r + 1) * W + 4 * x4);
    }
    // first-level index j = 0 .. n+1 is plane zfirst + (j-1) dir, from input planes j, j+1,
    // j+2; second-level output o = j - 2 uses first-level planes o, o+1, o+2. The stages of
    // input planes j+1, j+2, the mbarrier phase of j+2 and the first-level ring planes
    // j % 3, (j-1) % 3 advance incrementally instead of by division.
    uint32_t s1 = (q_base + 1) % NS, s2 = (q_base + 2) % NS;
    uint32_t ph2 = ((q_base + 2) / NS) & 1u;
    float* l1w = l1;                       // first-level ring plane j % 3
    float* l1r = l1 + 2 * C::L1_PLANE;     // and (j - 1) % 3
    for (int j = 0; j < n + 2; ++j) {
      if (__syncthreads_or(err)) break;
      if (tid == 0 && j + NS < nin) {
        fence_proxy_async_smem();
        issue(q_base + j + NS, y0, in_plane(j + NS));
        q_issued = q_base + j + NS + 1;
      }
      err = !mbar_wait_bounded(&bars[s2], ph2, kWaitBudgetCycles);
      if (err) continue;
      // ---- first level on row r of plane j (input centre plane j+1)
      const float* sc = ring + s1 * C::IN_STAGE;
      const float* sp = ring + s2 * C::IN_STAGE;
      s1 = s2;
      if (++s2 == NS) {
        s2 = 0;
        ph2 ^= 1u;
      }
      float4 izp[NF], lap[NF], l1v[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const float* F = sc + f * C::IN_FIELD;
        const float4 ym = *reinterpret_cast<const float4*>(F + r * W + 4 * x4);
        const float4 yp = *reinterpret_cast<const float4*>(F + (r + 2) * W + 4 * x4);
        izp[f] = *reinterpret_cast<const float4*>(sp + f * C::IN_FIELD + (r + 1) * W + 4 * x4);
        float xm, xp;
        x_edges<W>(F + (r + 1) * W, x4, xm, xp);
        lap[f] = lap3d_x4(ic[f], ym, yp, izm[f], izp[f], xm, xp, m.lap_scale);
      }
      update4<MODEL>(ic, lap, l1v, m);
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        *reinterpret_cast<float4*>(l1w + f * C::L1_FIELD + r * W + 4 * x4) = l1v[f];
        izm[f] = ic[f];
        ic[f] = izp[f];
      }
      // ---- second level for output o = j - 2: centre is first-level plane j-1, whose
      // rows were completed before this iteration's barrier
      if (j >= 2 && second) {
        const float* lp = l1r;
        float4 lap2[NF], res[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          const float* F = lp + f * C::L1_FIELD;
          const float4 ym = *reinterpret_cast<const float4*>(F + (r - 1) * W + 4 * x4);
          const float4 yp = *reinterpret_cast<const float4*>(F + (r + 1) * W + 4 * x4);
          float xm, xp;
          x_edges<W>(F + r * W, x4, xm, xp);
          lap2[f] = lap3d_x4(lc[f], ym, yp, lzm[f], l1v[f], xm, xp, m.lap_scale);
        }
        update4<MODEL>(lc, lap2, res, m);
        const int z = zfirst + (j - 2) * dir;
        const int64_t off = (int64_t)z * g.plane + (int64_t)(y0 + r - 1) * g.pitch + 4 * x4;
#pragma unroll
        for (int f = 0; f < NF; ++f) *reinterpret_cast<float4*>(out.f[f] + off) = res[f];
      }
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        lzm[f] = lc[f];
        lc[f] = l1v[f];
      }
      l1r = l1w;
      l1w = l1w == l1 + 2 * C::L1_PLANE ? l1 : l1w + C::L1_PLANE;
    }
    q_base += nin;
  }

  if (__syncthreads_or(err)) {
    if (tid == 0) {
      atomicExch(err_flag, 1);
      for (uint32_t q = (q_issued > NS ? q_issued - NS : 0); q < q_issued; ++q)
        (void)mbar_wait_bounded(&bars[q % NS], (q / NS) & 1u, kWaitBudgetCycles);
    }
  }
}

template <int MODEL, int W, int TY, int NS>
cudaError_t launch_tb2(pf_grid_s* gr, const Tb2Maps& maps, FieldOut out, cudaStream_t st) {
  using C = CfgB<MODEL, W, TY, NS>;
  auto kern = fe3d_tb2_kernel<MODEL, W, TY, NS>;
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
  const long long ncols = g.ny / TY;
  const long long slots = (long long)sms * occ;
  long long nchunks = slots / ncols;
  if (nchunks > g.nz / 4) nchunks = g.nz / 4;
  if (nchunks < 1) nchunks = 1;
  const int chunk_len = (int)((g.nz + nchunks - 1) / nchunks);
  nchunks = (g.nz + chunk_len - 1) / chunk_len;
  const long long items = ncols * nchunks;
  long long grid = items < slots ? items : slots;
  // Balanced mode when it shortens the longest CTA's plane count (each segment also streams
  // 4 halo planes): item mode runs ceil(items / grid) items of chunk_len + 4 planes, balanced
  // mode about units / slots + 8 planes (two segments at most when a range is under nz).
  const long long units = ncols * (long long)g.nz;
  const long long item_span = (items + grid - 1) / grid * (chunk_len + 4);
  const long long per = (units + slots - 1) / slots;
  const long long bal_span = per + (per < g.nz ? 8 : 4 * ((per + g.nz - 1) / g.nz + 1));
  int balanced = 0;
  if (bal_span < item_span && slots > grid) {
    balanced = 1;
    grid = slots < units ? slots : units;
  }
  kern<<<(unsigned)grid, C::NT, C::SMEM, st>>>(maps, out, g, gr->params, (int)nchunks, chunk_len,
                                               balanced, gr->d_err);
  return cudaGetLastError();
}

}  // namespace

bool fe3d_tb2_supported(int model, int tx, int ty, const Geom& g) {
  if (model != PF_MODEL_AC && model != PF_MODEL_GS) return false;
  if (ty != 8 || (tx != 128 && tx != 256)) return false;
  return g.nx == tx && g.ny % ty == 0 && g.ny >= 2;
}

cudaError_t tb2_maps(pf_grid_s* gr, int tx, int buf) {
  Tb2Cache& tc = gr->tb2;
  if (tc.width == tx && tc.valid[buf]) return cudaSuccess;
  if (tc.width != tx) {
    tc.valid[0] = tc.valid[1] = false;
    tc.width = tx;
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
  const cuuint64_t dims[3] = {(cuuint64_t)gr->nx, (cuuint64_t)gr->ny, (cuuint64_t)gr->nz};
  const cuuint64_t strides[2] = {(cuuint64_t)gr->pitch * 4, (cuuint64_t)gr->plane * 4};
  const cuuint32_t estr[3] = {1, 1, 1};
  const cuuint32_t box_row2[3] = {(cuuint32_t)tx, 2, 1};
  const cuuint32_t box_inner[3] = {(cuuint32_t)tx, 8, 1};
  for (int f = 0; f < gr->nf; ++f) {
    void* base = gr->buf[buf][f];
    Tb2Maps& mp = tc.maps[buf];
    CUresult r = encode(&mp.row2[f], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides,
                        box_row2, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r == CUDA_SUCCESS)
      r = encode(&mp.inner[f], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box_inner,
                 estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  }
  tc.valid[buf] = true;
  return cudaSuccess;
}

cudaError_t launch_fe3d_tb2(pf_grid_s* gr, int tx, int src, int dst, cudaStream_t st) {
  cudaError_t e = tb2_maps(gr, tx, src);
  if (e != cudaSuccess) return e;
  FieldOut out{};
  for (int f = 0; f < gr->nf; ++f) out.f[f] = gr->buf[dst][f];
  const Tb2Maps& maps = gr->tb2.maps[src];
  if (gr->model == PF_MODEL_GS) {
    if (tx == 256) return launch_tb2<PF_MODEL_GS, 256, 8, 5>(gr, maps, out, st);
    return launch_tb2<PF_MODEL_GS, 128, 8, 6>(gr, maps, out, st);
  }
  if (gr->model == PF_MODEL_AC) {
    if (tx == 256) return launch_tb2<PF_MODEL_AC, 256, 8, 6>(gr, maps, out, st);
    return launch_tb2<PF_MODEL_AC, 128, 8, 6>(gr, maps, out, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace pf
