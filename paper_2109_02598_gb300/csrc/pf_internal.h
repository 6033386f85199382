// Host-side declarations shared by the translation units of libpfgpu (not installed).
#pragma once

#include <nvtx3/nvToolsExt.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>

#include "pf_model.cuh"
#include "pfgpu.h"

#define PF_MAX_FIELDS 4  // fields of a grid: 1 or 2 for Models A-C and Gray-Scott, up to 4 for N species

namespace pf {

// Geometry of one field in the padded device layout: [nz][ny][pitch] floats, x fastest,
// pitch = nx rounded up to a multiple of 4 (16-byte rows); padding is never read as data.
struct Geom {
  int dim;
  int nx, ny, nz;  // nz == 1 for 2D
  int64_t pitch;   // floats per row
  int64_t plane;   // floats per z-plane (pitch * ny)
};

struct FieldPtrs {
  const float* f[PF_MAX_FIELDS];
};
struct FieldOut {
  float* f[PF_MAX_FIELDS];
};

// N coupled species (PF_MODEL_RD): du_i/dt = D_i lap u_i + sum_m K[i][m] prod_j u_j^E[m][j],
// as the kernel takes it (pf_rdn.cu): D_i times the stencil factor 1/h^2 and the rates rounded
// once to float32; monomial m's exponents packed two bits per field (field j at bits 2j).
constexpr int kRdMonomials = 8;
struct RdParams {
  int nmono;
  int E[kRdMonomials];
  float D[PF_MAX_FIELDS];
  float K[PF_MAX_FIELDS][kRdMonomials];
  float dt;
};
cudaError_t launch_rd(const Geom& g, int nf, FieldPtrs in, FieldOut out, const RdParams& p,
                      cudaStream_t s);

// Set a kernel's dynamic shared-memory limit once per device (the attribute is per device;
// `mask` has one bit per device ordinal below 64, set after success).
template <class KernelT>
cudaError_t ensure_smem_attr(KernelT kernel, size_t bytes, unsigned long long* mask) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = dev < 64 ? (1ull << dev) : 0ull;
  if (bit != 0 && (*mask & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) *mask |= bit;
  return e;
}

// A named range on the host timeline of a profiler that reads NVTX (header-only NVTX3; without
// such a tool attached a push or pop is a call through a null-checked pointer).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Thread-local error reporting (pf_last_error).
void set_error(const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);

#define PF_CUDA_TRY(call)                                  \
  do {                                                     \
    cudaError_t pf_e_ = (call);                            \
    if (pf_e_ != cudaSuccess) return pf::cuda_fail(pf_e_, #call); \
  } while (0)

// ---- 2D tiled forward-Euler kernel (temporal blocking depth k) -------------------
// Tile ids: 0 = 64x16, 1 = 128x16, 2 = 32x32, 3 = 128x32.
constexpr int kNumTiles2D = 4;
void tile2d_shape(int tile_id, int* tx, int* ty);
int tile2d_id(int tx, int ty);  // -1 if unsupported
bool fe2d_supported(int model, int k);
cudaError_t launch_fe2d(int model, int tile_id, int k, const Geom& g, FieldPtrs in,
                        FieldOut out, const ModelParams& m, cudaStream_t s);

// Other Laplacian stencils in 2D (PF_ST_ISO, PF_ST_O4): tiles 0 (64x16) and 3 (128x32),
// k in {1, 2}; PF_ST_STD forwards to launch_fe2d.
bool fe2d_stencil_supported(int stencil, int tile_id, int k);
cudaError_t launch_fe2d_stencil(int stencil, int model, int tile_id, int k, const Geom& g,
                                FieldPtrs in, FieldOut out, const ModelParams& m,
                                cudaStream_t s);

// ---- 2D grids held on chip by one thread-block cluster (pf_fe2d_cluster.cu) --------
// Tile id kTileCluster2D: each CTA of a cluster of fe2d_cluster_size() CTAs keeps a band of
// full rows in shared memory; one launch runs all n_steps (k steps per halo exchange).
constexpr int kTileCluster2D = kNumTiles2D;
int fe2d_cluster_size();
bool fe2d_cluster_supported(int model, int k, const Geom& q);
cudaError_t launch_fe2d_cluster(int model, int k, const Geom& q, FieldPtrs in, FieldOut out,
                                const ModelParams& m, int64_t n_steps, cudaStream_t st);

// ---- 2D grids held in the shared memory of all SMs (pf_fe2d_bands.cu) ---------------
// Tile id kTileBands2D (tile_y = PF_TILE_BANDS): one band of full rows per SM, neighbouring
// bands exchange edge rows through global memory every step; AC and CH, k = 1.
constexpr int kTileBands2D = kNumTiles2D + 1;
bool fe2d_bands_supported(int model, const Geom& q);

// ---- 2D register-streaming kernel: one warp per strip of 32 C columns (pf_fe2d_strips.cu) --
// tile ids kTileStrips2D (128 columns per warp, C = 4) and kTileStrips2D + 1 (64, C = 2)
constexpr int kTileStrips2D = kNumTiles2D + 2;
constexpr int kNumStrips2D = 2;
// stencil: PF_ST_STD for every model, PF_ST_ISO (9-point) for Allen-Cahn and Gray-Scott
bool fe2d_strips_supported(int model, int k, int stencil);
cudaError_t launch_fe2d_strips(int model, int stencil, int lanes_cols, int k, const Geom& g,
                               FieldPtrs in, FieldOut out, const ModelParams& m, cudaStream_t s);

// ---- 3D z-streaming forward-Euler kernels (k = 1) -------------------------------
// Tile ids: 0 = 32x16, 1 = 64x8 (general kernel, any size, all models);
//           2 = 64x16, 3 = 128x8, 4 = 128x16 (TMA kernel, AC/GS, nx % TX == ny % TY == 0);
//           with k = 2: 3 = 128x8 and 5 = 256x8 (depth-2 TMA kernel, AC/GS, nx == TX).
//           6 = 32x8: the box kernel (Models B and C, nx % 4 == 0, k = 1 or 2; whole
//           32x8x8 boxes per CTA).
constexpr int kNumTiles3D = 7;
constexpr int kFirstTmaTile3D = 2;
constexpr int kTileBox3D = 6;
bool fe3d_box_supported(int model, int k, const Geom& g);
cudaError_t launch_fe3d_box(int model, int k, const Geom& g, FieldPtrs in, FieldOut out,
                            const ModelParams& m, cudaStream_t s);
void tile3d_shape(int tile_id, int* tx, int* ty);
int tile3d_id(int tx, int ty);
cudaError_t launch_fe3d(int model, int tile_id, const Geom& g, FieldPtrs in, FieldOut out,
                        const ModelParams& m, cudaStream_t s, int stencil = PF_ST_STD);

// ---- batched 2D Gray-Scott (many independent grids, one launch per k steps) -------
// Instance i: fields at buffer base + off (u) and base + off + pitch * ny (v).
struct BatchInst {
  int nx, ny;
  int64_t pitch;  // floats per row
  int64_t off;    // floats from the buffer base to field u
  ModelParams m;  // per-instance coefficients
};
struct BatchTile {
  int inst, x0, y0;
};
// A strip task of the batch (strip kernel of 32 c lanes' columns, c = 4 or 2 for the whole
// launch): output columns [x0, x0 + wo) and rows [y0, y0 + hy) of instance inst; x0 is a
// multiple of 4 and wo too unless the strip ends at the instance's last column.
struct BatchStrip {
  int inst, x0, y0;
  short hy, wo;
};
int strip_out_cols(int model, int k, int c);  // output columns of a strip of 32 c columns
int strip_task_rows(int model, int k);        // fewest rows per batch strip task
int batch_gs2d_strips_resident(int k, int c);  // warps of the batch strip kernel on the device
cudaError_t launch_batch_gs2d_strips(int c, int k, const BatchInst* d_insts,
                                     const BatchStrip* d_tasks, int ntasks, const float* in_base,
                                     float* out_base, cudaStream_t s);
cudaError_t prepare_batch_gs2d();  // set kernel attributes (call before any capture)
cudaError_t launch_batch_gs2d(int tile_id, int k, const BatchInst* d_insts,
                              const BatchTile* d_tiles, int ntiles, const float* in_base,
                              float* out_base, cudaStream_t s);

// ---- reductions -------------------------------------------------------------------
// Writes one double to d_out. d_partials must hold kReduceBlocks doubles.
constexpr int kReduceBlocks = 512;
cudaError_t launch_reduce(int what, const Geom& g, const float* field, double c1, double c2,
                          double h, double* d_partials, double* d_out, cudaStream_t s);
// Model C free energy of (psi, m) with coefficients c[0..4] = c1..c5.
cudaError_t launch_reduce_energy_c(const Geom& g, const float* psi, const float* m,
                                   const double* c, double h, double* d_partials,
                                   double* d_out, cudaStream_t s);

}  // namespace pf
