// 2D forward-Euler step with temporal blocking (Sec. 2.4.1 solver, Sec. 2.2.2 stencils,
// Sec. 3 models) — one fused kernel per k steps.
//
// A CTA owns a TX x TY output tile.  It stages the tile plus a periodic halo of
// H = k * R sites (R = 1 for AC/GS, 2 for CH) in shared memory, runs k forward-Euler
// sub-steps there on a region that shrinks by R per sub-step (halo sites are recomputed
// redundantly instead of exchanged), and writes only the last sub-step to HBM.  HBM
// traffic per site and step is therefore 2 * NF * 4 / k bytes.  Model B computes the
// chemical potential mu on the region one ring wider than the phi update and never
// stores it to HBM (the paper's provisional variable, Sec. 2.3.2, kept on chip).
//
// The tile body is a device function so the batched runner (many grids, one launch)
// executes exactly the same arithmetic.
#include "pf_fe2d_tile.cuh"
#include "pf_internal.h"

namespace pf {

namespace {

template <int MODEL, int K, int TX, int TY>
__global__ void __launch_bounds__(kNT2) fe2d_kernel(FieldPtrs in, FieldOut out, Geom g,
                                                    ModelParams m) {
  extern __shared__ __align__(16) float sm[];
  const int x0 = blockIdx.x * TX;
  const int y0 = blockIdx.y * TY;
  fe2d_tile<MODEL, K, TX, TY>(in, out, g.nx, g.ny, g.pitch, x0, y0, m, sm);
}

// Batched Gray-Scott: CTA b runs the same tile body on work-list entry b.
template <int K, int TX, int TY>
__global__ void __launch_bounds__(kNT2) batch_gs2d_kernel(const BatchInst* __restrict__ insts,
                                                          const BatchTile* __restrict__ tiles,
                                                          const float* in_base, float* out_base) {
  extern __shared__ __align__(16) float sm[];
  const BatchTile t = tiles[blockIdx.x];
  const BatchInst I = insts[t.inst];
  const int64_t plane = I.pitch * I.ny;
  FieldPtrs in{};
  FieldOut out{};
  in.f[0] = in_base + I.off;
  in.f[1] = in_base + I.off + plane;
  out.f[0] = out_base + I.off;
  out.f[1] = out_base + I.off + plane;
  fe2d_tile<PF_MODEL_GS, K, TX, TY>(in, out, I.nx, I.ny, I.pitch, t.x0, t.y0, I.m, sm);
}

template <int K, int TX, int TY>
cudaError_t launch_batch_one(const BatchInst* d_insts, const BatchTile* d_tiles, int ntiles,
                             const float* in_base, float* out_base, cudaStream_t s) {
  using C = Cfg2<PF_MODEL_GS, K, TX, TY>;
  const size_t smem = sizeof(float) * C::SMEM_FLOATS;
  static unsigned long long attr_mask = 0;
  cudaError_t e = ensure_smem_attr(batch_gs2d_kernel<K, TX, TY>, smem, &attr_mask);
  if (e != cudaSuccess) return e;
  batch_gs2d_kernel<K, TX, TY><<<ntiles, kNT2, smem, s>>>(d_insts, d_tiles, in_base, out_base);
  return cudaGetLastError();
}

template <int K>
cudaError_t launch_batch_tile(int tile_id, const BatchInst* d_insts, const BatchTile* d_tiles,
                              int ntiles, const float* in_base, float* out_base, cudaStream_t s) {
  switch (tile_id) {
    case 0: return launch_batch_one<K, 64, 16>(d_insts, d_tiles, ntiles, in_base, out_base, s);
    case 1: return launch_batch_one<K, 128, 16>(d_insts, d_tiles, ntiles, in_base, out_base, s);
    case 2: return launch_batch_one<K, 32, 32>(d_insts, d_tiles, ntiles, in_base, out_base, s);
    case 3: return launch_batch_one<K, 128, 32>(d_insts, d_tiles, ntiles, in_base, out_base, s);
  }
  return cudaErrorInvalidValue;
}

template <int MODEL, int K, int TX, int TY>
cudaError_t launch_one(const Geom& g, FieldPtrs in, FieldOut out, const ModelParams& m,
                       cudaStream_t s) {
  using C = Cfg2<MODEL, K, TX, TY>;
  const size_t smem = sizeof(float) * C::SMEM_FLOATS;
  static unsigned long long attr_mask = 0;  // per instantiation and device
  cudaError_t e = ensure_smem_attr(fe2d_kernel<MODEL, K, TX, TY>, smem, &attr_mask);
  if (e != cudaSuccess) return e;
  dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, 1);
  fe2d_kernel<MODEL, K, TX, TY><<<grid, kNT2, smem, s>>>(in, out, g, m);
  return cudaGetLastError();
}

template <int MODEL, int K>
cudaError_t launch_tile(int tile_id, const Geom& g, FieldPtrs in, FieldOut out,
                        const ModelParams& m, cudaStream_t s) {
  switch (tile_id) {
    case 0: return launch_one<MODEL, K, 64, 16>(g, in, out, m, s);
    case 1: return launch_one<MODEL, K, 128, 16>(g, in, out, m, s);
    case 2: return launch_one<MODEL, K, 32, 32>(g, in, out, m, s);
    case 3: return launch_one<MODEL, K, 128, 32>(g, in, out, m, s);
  }
  return cudaErrorInvalidValue;
}

template <int K, int TX, int TY>
cudaError_t prepare_one() {
  using C = Cfg2<PF_MODEL_GS, K, TX, TY>;
  return cudaFuncSetAttribute(batch_gs2d_kernel<K, TX, TY>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(sizeof(float) * C::SMEM_FLOATS));
}

template <int K>
cudaError_t prepare_k() {
  cudaError_t e = prepare_one<K, 64, 16>();
  if (e == cudaSuccess) e = prepare_one<K, 128, 16>();
  if (e == cudaSuccess) e = prepare_one<K, 32, 32>();
  if (e == cudaSuccess) e = prepare_one<K, 128, 32>();
  return e;
}

}  // namespace

cudaError_t prepare_batch_gs2d() {
  cudaError_t e = prepare_k<1>();
  if (e == cudaSuccess) e = prepare_k<2>();
  if (e == cudaSuccess) e = prepare_k<4>();
  return e;
}

cudaError_t launch_batch_gs2d(int tile_id, int k, const BatchInst* d_insts,
                              const BatchTile* d_tiles, int ntiles, const float* in_base,
                              float* out_base, cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  if (k == 1) return launch_batch_tile<1>(tile_id, d_insts, d_tiles, ntiles, in_base, out_base, s);
  if (k == 2) return launch_batch_tile<2>(tile_id, d_insts, d_tiles, ntiles, in_base, out_base, s);
  if (k == 4) return launch_batch_tile<4>(tile_id, d_insts, d_tiles, ntiles, in_base, out_base, s);
  return cudaErrorInvalidValue;
}

void tile2d_shape(int tile_id, int* tx, int* ty) {
  static const int s[kNumTiles2D][2] = {{64, 16}, {128, 16}, {32, 32}, {128, 32}};
  *tx = s[tile_id][0];
  *ty = s[tile_id][1];
}

int tile2d_id(int tx, int ty) {
  for (int i = 0; i < kNumTiles2D; ++i) {
    int a, b;
    tile2d_shape(i, &a, &b);
    if (a == tx && b == ty) return i;
  }
  return -1;
}

bool fe2d_supported(int model, int k) {
  if (model == PF_MODEL_CH || model == PF_MODEL_C) return k == 1 || k == 2;
  return k == 1 || k == 2 || k == 4;
}

cudaError_t launch_fe2d(int model, int tile_id, int k, const Geom& g, FieldPtrs in,
                        FieldOut out, const ModelParams& m, cudaStream_t s) {
  if (tile_id < 0 || tile_id >= kNumTiles2D || !fe2d_supported(model, k))
    return cudaErrorInvalidValue;
  switch (model) {
    case PF_MODEL_AC:
      if (k == 1) return launch_tile<PF_MODEL_AC, 1>(tile_id, g, in, out, m, s);
      if (k == 2) return launch_tile<PF_MODEL_AC, 2>(tile_id, g, in, out, m, s);
      return launch_tile<PF_MODEL_AC, 4>(tile_id, g, in, out, m, s);
    case PF_MODEL_GS:
      if (k == 1) return launch_tile<PF_MODEL_GS, 1>(tile_id, g, in, out, m, s);
      if (k == 2) return launch_tile<PF_MODEL_GS, 2>(tile_id, g, in, out, m, s);
      return launch_tile<PF_MODEL_GS, 4>(tile_id, g, in, out, m, s);
    case PF_MODEL_CH:
      if (k == 1) return launch_tile<PF_MODEL_CH, 1>(tile_id, g, in, out, m, s);
      return launch_tile<PF_MODEL_CH, 2>(tile_id, g, in, out, m, s);
    case PF_MODEL_C:
      if (k == 1) return launch_tile<PF_MODEL_C, 1>(tile_id, g, in, out, m, s);
      return launch_tile<PF_MODEL_C, 2>(tile_id, g, in, out, m, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace pf
