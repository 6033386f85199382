// 2D forward-Euler step with the isotropic 9-point or the fourth-order 9-point Laplacian
// (Sec. 2.2.2): the same tile body as pf_fe2d.cu instantiated for those stencils, in a
// translation unit of its own so that the build compiles the two in parallel.  Tiles 64x16
// and 128x32, temporal depth 1 or 2, every model.
#include "pf_fe2d_tile.cuh"
#include "pf_internal.h"

namespace pf {

namespace {

template <int MODEL, int K, int TX, int TY, int ST>
__global__ void __launch_bounds__(kNT2) fe2d_st_kernel(FieldPtrs in, FieldOut out, Geom g,
                                                       ModelParams m) {
  extern __shared__ __align__(16) float sm[];
  fe2d_tile<MODEL, K, TX, TY, ST>(in, out, g.nx, g.ny, g.pitch, blockIdx.x * TX, blockIdx.y * TY,
                                  m, sm);
}

template <int MODEL, int K, int TX, int TY, int ST>
cudaError_t launch_st(const Geom& g, FieldPtrs in, FieldOut out, const ModelParams& m,
                      cudaStream_t s) {
  using C = Cfg2<MODEL, K, TX, TY, ST>;
  const size_t smem = sizeof(float) * C::SMEM_FLOATS;
  static unsigned long long attr_mask = 0;
  cudaError_t e = ensure_smem_attr(fe2d_st_kernel<MODEL, K, TX, TY, ST>, smem, &attr_mask);
  if (e != cudaSuccess) return e;
  dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, 1);
  fe2d_st_kernel<MODEL, K, TX, TY, ST><<<grid, kNT2, smem, s>>>(in, out, g, m);
  return cudaGetLastError();
}

template <int MODEL, int ST>
cudaError_t launch_model_st(int tile_id, int k, const Geom& g, FieldPtrs in, FieldOut out,
                            const ModelParams& m, cudaStream_t s) {
  if (tile_id == 0 && k == 1) return launch_st<MODEL, 1, 64, 16, ST>(g, in, out, m, s);
  if (tile_id == 0 && k == 2) return launch_st<MODEL, 2, 64, 16, ST>(g, in, out, m, s);
  if (tile_id == 3 && k == 1) return launch_st<MODEL, 1, 128, 32, ST>(g, in, out, m, s);
  if (tile_id == 3 && k == 2) return launch_st<MODEL, 2, 128, 32, ST>(g, in, out, m, s);
  return cudaErrorInvalidValue;
}

template <int ST>
cudaError_t launch_stencil(int model, int tile_id, int k, const Geom& g, FieldPtrs in,
                           FieldOut out, const ModelParams& m, cudaStream_t s) {
  switch (model) {
    case PF_MODEL_AC: return launch_model_st<PF_MODEL_AC, ST>(tile_id, k, g, in, out, m, s);
    case PF_MODEL_CH: return launch_model_st<PF_MODEL_CH, ST>(tile_id, k, g, in, out, m, s);
    case PF_MODEL_GS: return launch_model_st<PF_MODEL_GS, ST>(tile_id, k, g, in, out, m, s);
    case PF_MODEL_C: return launch_model_st<PF_MODEL_C, ST>(tile_id, k, g, in, out, m, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

bool fe2d_stencil_supported(int stencil, int tile_id, int k) {
  if (stencil == PF_ST_STD) return true;
  return (stencil == PF_ST_ISO || stencil == PF_ST_O4) && (tile_id == 0 || tile_id == 3) &&
         (k == 1 || k == 2);
}

cudaError_t launch_fe2d_stencil(int stencil, int model, int tile_id, int k, const Geom& g,
                                FieldPtrs in, FieldOut out, const ModelParams& m,
                                cudaStream_t s) {
  if (stencil == PF_ST_STD) return launch_fe2d(model, tile_id, k, g, in, out, m, s);
  if (stencil == PF_ST_ISO) return launch_stencil<PF_ST_ISO>(model, tile_id, k, g, in, out, m, s);
  if (stencil == PF_ST_O4) return launch_stencil<PF_ST_O4>(model, tile_id, k, g, in, out, m, s);
  return cudaErrorInvalidValue;
}

}  // namespace pf
