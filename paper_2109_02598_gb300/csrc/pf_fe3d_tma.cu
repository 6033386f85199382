// 3D forward-Euler step for the radius-1 models (Allen-Cahn, Gray-Scott) with TMA plane
// staging (Sec. 2.4.1 solver, Sec. 2.2.2 7-point Laplacian, Sec. 3 / Sec. 1 models).
//
// Work: the grid is cut into TX x TY columns in the xy plane and every column into
// nchunks z-chunks; one CTA streams one (column, chunk) item at a time, all columns of a
// chunk side by side, so the halo rows and columns a tile shares with its neighbours are
// fetched from HBM once and served from L2 to the second reader.  Even chunks stream up
// in z and odd chunks down, so the plane two chunks share at their boundary is read by
// both CTAs at the same moment too.  Streaming keeps the z-neighbours in registers: the
// values of one plane become the "previous" values of the next (the 7-point sum pairs the
// two z-neighbours in one addition, which is commutative, so the direction does not
// change the result).
//
// Staging: per plane and field, five TMA boxes land in a ring of NS shared-memory stages:
// the TX x TY interior, the rows above and below (wrapped in y), and 4-wide column boxes
// left and right (wrapped in x; only their inner column is used).  No thread spends an
// instruction on loading or wrapping; the producer thread issues the boxes NS-2 planes
// ahead and the consumers wait on the stage's mbarrier (bounded).
//
// Compute: each thread owns a float4 of x in one row; x-neighbours come from the lanes
// on either side (warp shuffle), from the column boxes at the tile edge; y-neighbours from
// shared memory; z-neighbours from registers.  Results go straight to HBM as float4.
//
// Requires nx % TX == 0 and ny % TY == 0 (the host falls back to the general kernel).
#include "pf_grid.h"
#include "pf_internal.h"
#include "pf_tma.cuh"

#include <cudaTypedefs.h>

namespace pf {

namespace {

template <int MODEL, int TX, int TY, int NS>
struct CfgT {
  static constexpr int NF = ModelTraits<MODEL>::NF;
  static constexpr int LX = TX / 4;                 // threads per row
  static constexpr int NT = LX * TY;                // threads per CTA
  static constexpr int MAIN = (TY + 2) * TX;        // floats: halo row, TY rows, halo row
  static constexpr int SIDE = TY * 4;               // floats per 4-wide column box
  static constexpr int FIELD = MAIN + 2 * SIDE;     // floats per field per stage
  static constexpr int STAGE = NF * FIELD;          // floats per stage
  static constexpr uint32_t TX_BYTES = STAGE * 4;   // bytes one plane brings in
  static constexpr size_t SMEM = (size_t)NS * STAGE * 4 + NS * 8 + 128;  // + barriers + align
  static_assert(TX % 32 == 0, "row boxes must start 128-byte aligned");
  static_assert((TY * 16) % 128 == 0 || TY * 16 == 128, "column boxes 128-byte aligned");
};

template <int MODEL, int TX, int TY, int NS>
__global__ void __launch_bounds__(CfgT<MODEL, TX, TY, NS>::NT)
    fe3d_tma_kernel(const __grid_constant__ Tma3dMaps maps, FieldOut out, Geom g,
                    ModelParams m, int tiles_x, int nchunks, int chunk_len, int* err_flag) {
  using C = CfgT<MODEL, TX, TY, NS>;
  constexpr int NF = C::NF;
  constexpr int LX = C::LX;
  extern __shared__ unsigned char smem_raw[];
  // 128-byte aligned stage ring, barriers after it
  const uint32_t base_sa = smem_addr(smem_raw);
  float* ring = reinterpret_cast<float*>(smem_raw + ((128 - (base_sa & 127)) & 127));
  uint64_t* bars = reinterpret_cast<uint64_t*>(ring + NS * C::STAGE);

  const int tid = threadIdx.x;
  const int tx4 = tid % LX;
  const int ty = tid / LX;
  canary_fill(ring, (size_t)NS * C::STAGE);  // TMA issues follow a proxy fence
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) mbar_init(&bars[s], 1);
    mbar_fence_init();
  }
  __syncthreads();

  uint32_t q_base = 0;     // sequence number of the next plane load of this CTA
  uint32_t q_issued = 0;   // (thread 0) loads issued so far
  bool err = false;

  auto stage_ptr = [&](uint32_t q) { return ring + (q % NS) * C::STAGE; };
  // Producer: plane p (any integer, wrapped) of column (x0, y0) as load number q.
  auto issue = [&](uint32_t q, int x0, int y0, int p) {
    float* st = stage_ptr(q);
    uint64_t* bar = &bars[q % NS];
    const int z = wrap_index(p, g.nz);
    const int ytop = wrap_index(y0 - 1, g.ny);
    const int ybot = wrap_index(y0 + TY, g.ny);
    const int xl = wrap_index(x0 - 4, g.nx);
    const int xr = wrap_index(x0 + TX, g.nx);
    mbar_arrive_expect_tx(bar, C::TX_BYTES);
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      float* fs = st + f * C::FIELD;
      tma_load_3d(fs, &maps.row[f], x0, ytop, z, bar);
      tma_load_3d(fs + TX, &maps.inner[f], x0, y0, z, bar);
      tma_load_3d(fs + (TY + 1) * TX, &maps.row[f], x0, ybot, z, bar);
      tma_load_3d(fs + C::MAIN, &maps.side[f], xl, y0, z, bar);
      tma_load_3d(fs + C::MAIN + C::SIDE, &maps.side[f], xr, y0, z, bar);
    }
  };
  auto wait = [&](uint32_t q) -> bool {
    return mbar_wait_bounded(&bars[q % NS], (q / NS) & 1u, kWaitBudgetCycles);
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
    const int np = n + 2;  // planes zfirst - dir, zfirst, ..., zfirst + n*dir

    if (__syncthreads_or(err)) break;
    if (tid == 0) {
      fence_proxy_async_smem();
      const int n0 = np < NS ? np : NS;
      for (int i = 0; i < n0; ++i) issue(q_base + i, x0, y0, zfirst + (i - 1) * dir);
      q_issued = q_base + n0;
    }
    // prologue: centre values of the planes before and at zfirst
    float4 zm[NF], c[NF];
    err = !wait(q_base);
    if (!err) {
      const float* st = stage_ptr(q_base);
#pragma unroll
      for (int f = 0; f < NF; ++f)
        zm[f] = *reinterpret_cast<const float4*>(st + f * C::FIELD + (ty + 1) * TX + 4 * tx4);
      err = !wait(q_base + 1);
    }
    if (!err) {
      const float* st = stage_ptr(q_base + 1);
#pragma unroll
      for (int f = 0; f < NF; ++f)
        c[f] = *reinterpret_cast<const float4*>(st + f * C::FIELD + (ty + 1) * TX + 4 * tx4);
    }

    const int gy = y0 + ty;
    const int gx = x0 + 4 * tx4;
    for (int i = 0; i < n; ++i) {
      const int z = zfirst + i * dir;  // output plane; its load index is i + 1
      if (__syncthreads_or(err)) break;
      if (tid == 0 && i + NS < np) {
        fence_proxy_async_smem();
        issue(q_base + i + NS, x0, y0, zfirst + (i + NS - 1) * dir);
        q_issued = q_base + i + NS + 1;
      }
      err = !wait(q_base + i + 2);  // the plane after z in streaming order
      err = __any_sync(0xffffffffu, err);  // warp-uniform before the shuffles below
      if (err) continue;
      const float* sz = stage_ptr(q_base + i + 1);
      const float* sp = stage_ptr(q_base + i + 2);
      float4 res[NF], zp[NF], lap[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const float* M = sz + f * C::FIELD;
        const float4 ym = *reinterpret_cast<const float4*>(M + ty * TX + 4 * tx4);
        const float4 yp = *reinterpret_cast<const float4*>(M + (ty + 2) * TX + 4 * tx4);
        zp[f] = *reinterpret_cast<const float4*>(sp + f * C::FIELD + (ty + 1) * TX + 4 * tx4);
        float xm = __shfl_up_sync(0xffffffffu, c[f].w, 1, LX);
        float xp = __shfl_down_sync(0xffffffffu, c[f].x, 1, LX);
        if (tx4 == 0) xm = M[C::MAIN + ty * 4 + 3];
        if (tx4 == LX - 1) xp = M[C::MAIN + C::SIDE + ty * 4 + 0];
        lap[f].x = lap_scaled<MODEL>(
            lap3d_sum(c[f].x, xm, c[f].y, ym.x, yp.x, zm[f].x, zp[f].x), m.lap_scale);
        lap[f].y = lap_scaled<MODEL>(
            lap3d_sum(c[f].y, c[f].x, c[f].z, ym.y, yp.y, zm[f].y, zp[f].y), m.lap_scale);
        lap[f].z = lap_scaled<MODEL>(
            lap3d_sum(c[f].z, c[f].y, c[f].w, ym.z, yp.z, zm[f].z, zp[f].z), m.lap_scale);
        lap[f].w = lap_scaled<MODEL>(
            lap3d_sum(c[f].w, c[f].z, xp, ym.w, yp.w, zm[f].w, zp[f].w), m.lap_scale);
      }
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
      const int64_t off = (int64_t)z * g.plane + (int64_t)gy * g.pitch + gx;
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        *reinterpret_cast<float4*>(out.f[f] + off) = res[f];
        zm[f] = c[f];
        c[f] = zp[f];
      }
    }
    q_base += np;
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
cudaError_t launch_tma(pf_grid_s* gr, const Tma3dMaps& maps, FieldOut out, cudaStream_t st) {
  using C = CfgT<MODEL, TX, TY, NS>;
  auto kern = fe3d_tma_kernel<MODEL, TX, TY, NS>;
  static unsigned long long attr_mask = 0;  // per instantiation and device
  cudaError_t e0 = ensure_smem_attr(kern, C::SMEM, &attr_mask);
  if (e0 != cudaSuccess) return e0;
  static int occ_by_dev[64] = {};  // resident CTAs per SM, per device
  int occ = gr->device < 64 ? occ_by_dev[gr->device] : 0;
  if (occ == 0) {
    e0 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, C::NT, C::SMEM);
    if (e0 != cudaSuccess) return e0;
    if (occ < 1) occ = 1;
    if (gr->device < 64) occ_by_dev[gr->device] = occ;
  }
  int sms = 0;
  cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, gr->device);
  if (e != cudaSuccess) return e;
  const Geom g = grid_geom(gr);
  const int tiles_x = g.nx / TX;
  const int tiles_y = g.ny / TY;
  const long long ncols = (long long)tiles_x * tiles_y;
  const long long slots = (long long)sms * occ;
  // as many z-chunks as keep every column of a chunk resident at once, chunks >= 2 planes
  long long nchunks = slots / ncols;
  if (nchunks > g.nz / 2) nchunks = g.nz / 2;
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

bool fe3d_tma_supported(int model, int tma_tile, const Geom& g) {
  if (model != PF_MODEL_AC && model != PF_MODEL_GS && model != PF_MODEL_CH &&
      model != PF_MODEL_C)
    return false;
  if (tma_tile < 0 || tma_tile >= kNumTmaTiles3D) return false;
  int tx, ty;
  tma3d_tile_shape(tma_tile, &tx, &ty);
  return g.nx % tx == 0 && g.ny % ty == 0;
}

void tma3d_tile_shape(int tma_tile, int* tx, int* ty) {
  static const int s[kNumTmaTiles3D][2] = {{64, 16}, {128, 8}, {128, 16}};
  *tx = s[tma_tile][0];
  *ty = s[tma_tile][1];
}

cudaError_t launch_fe3d_tma(pf_grid_s* gr, int tma_tile, int src, int dst, cudaStream_t st) {
  if (gr->model == PF_MODEL_CH || gr->model == PF_MODEL_C)
    return launch_fe3d_tma_r2(gr, tma_tile, src, dst, st);
  cudaError_t e = tma3d_maps(gr, tma_tile, src);
  if (e != cudaSuccess) return e;
  FieldOut out{};
  for (int f = 0; f < gr->nf; ++f) out.f[f] = gr->buf[dst][f];
  const Tma3dMaps& maps = gr->tma.maps[src];
  if (gr->model == PF_MODEL_GS) {
    switch (tma_tile) {
      case 0: return launch_tma<PF_MODEL_GS, 64, 16, 5>(gr, maps, out, st);
      case 1: return launch_tma<PF_MODEL_GS, 128, 8, 5>(gr, maps, out, st);
      case 2: return launch_tma<PF_MODEL_GS, 128, 16, 5>(gr, maps, out, st);
    }
  } else if (gr->model == PF_MODEL_AC) {
    switch (tma_tile) {
      case 0: return launch_tma<PF_MODEL_AC, 64, 16, 6>(gr, maps, out, st);
      case 1: return launch_tma<PF_MODEL_AC, 128, 8, 6>(gr, maps, out, st);
      case 2: return launch_tma<PF_MODEL_AC, 128, 16, 5>(gr, maps, out, st);
    }
  }
  return cudaErrorInvalidValue;
}

// Tensor maps of one ping-pong buffer for the given tile (cached until the tile changes).
cudaError_t tma3d_maps(pf_grid_s* gr, int tma_tile, int buf) {
  TmaCache& tc = gr->tma;
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
  const cuuint32_t box_row[3] = {(cuuint32_t)tx, 1, 1};
  const cuuint32_t box_side[3] = {4, (cuuint32_t)ty, 1};
  for (int f = 0; f < gr->nf; ++f) {
    void* base = gr->buf[buf][f];
    Tma3dMaps& mp = tc.maps[buf];
    CUresult r = encode(&mp.inner[f], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides,
                        box_inner, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r == CUDA_SUCCESS)
      r = encode(&mp.row[f], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box_row,
                 estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r == CUDA_SUCCESS)
      r = encode(&mp.side[f], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box_side,
                 estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                 CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  }
  tc.valid[buf] = true;
  return cudaSuccess;
}

}  // namespace pf
