// The grid handle behind pf_grid_t (the paper's Grid + System + Model state,
// Sec. 2.2.1 and 2.2.5): geometry, the two ping-pong copies of every field in the padded
// device layout, the model coefficients and the kernel tuning.
#pragma once

#include <cuda.h>

#include "pf_internal.h"

namespace pf {

// TMA descriptors of one ping-pong buffer for the 3D kernel: the tile interior box, the
// one-row halo box and the 4-wide column box, per field.
struct Tma3dMaps {
  CUtensorMap inner[PF_MAX_FIELDS];
  CUtensorMap row[PF_MAX_FIELDS];
  CUtensorMap side[PF_MAX_FIELDS];
};

struct TmaCache {
  int tile = -1;  // TMA tile the maps were encoded for
  bool valid[2] = {false, false};
  Tma3dMaps maps[2];
};

// TMA descriptors of the radius-2 3D kernel (Models B and C): the tile interior box, a
// two-row halo box, the 4-wide column box and a 4 x 1 corner box, per field.
struct Tma2Maps {
  CUtensorMap inner[PF_MAX_FIELDS];
  CUtensorMap row2[PF_MAX_FIELDS];
  CUtensorMap side[PF_MAX_FIELDS];
  CUtensorMap corner[PF_MAX_FIELDS];
};

struct Tma2Cache {
  int tile = -1;
  bool valid[2] = {false, false};
  Tma2Maps maps[2];
};

// TMA descriptors of the depth-2 3D kernel: a two-row halo box and the 8-row interior box,
// both spanning the whole x-row, per field.
struct Tb2Maps {
  CUtensorMap row2[PF_MAX_FIELDS];
  CUtensorMap inner[PF_MAX_FIELDS];
};

struct Tb2Cache {
  int width = -1;
  bool valid[2] = {false, false};
  Tb2Maps maps[2];
};

constexpr uint32_t kGridMagic = 0x50464744u;  // "PFGD"

struct AdjointState {
  int64_t n_steps = 0;       // steps of the recorded forward pass
  int64_t interval = 0;      // checkpoint interval C
  int64_t n_ckpt = 0;        // checkpoints stored (states 0, C, 2C, ...)
  float* ckpt = nullptr;     // n_ckpt * nf * field_elems floats
  float* seg = nullptr;      // seg_bufs * (C - 1) * nf * field_elems floats: recomputed
                             // segments (two buffers: one is recomputed while the reverse
                             // steps read the other)
  int seg_bufs = 0;          // 2, or 1 where the second buffer could not be allocated
  float* lam = nullptr;      // 2 * nf * field_elems floats: adjoint ping-pong
  double* gpart = nullptr;   // per-CTA parameter-gradient partials (4 per CTA)
  double* gout = nullptr;    // 4 final sums (device)
  double* ghost = nullptr;   // 4 final sums (pinned host)
  int64_t gpart_cap = 0;     // CTAs the partial buffer holds
  double coeffs[4] = {0, 0, 0, 0};
  double dt = 0;
  int ready = 0;             // a forward pass is recorded
};

}  // namespace pf

struct pf_grid_s {
  uint32_t magic = 0;
  int dim = 0;
  int nx = 0, ny = 0, nz = 1;
  int nf = 0;
  double h = 1.0;
  cudaStream_t stream = nullptr;
  int device = 0;
  int64_t pitch = 0, plane = 0, field_elems = 0;
  float* base = nullptr;
  float* buf[2][PF_MAX_FIELDS] = {};
  int cur = 0;
  int model = 0;
  double coeffs[5] = {0, 0, 0, 0, 0};
  double dt = 0;
  int model_set = 0;
  int stencil = 0;  // PF_STENCIL_* (Laplacian stencil of the step)
  pf::ModelParams params{};
  // N coupled species (PF_MODEL_RD): the coefficient list as given and the kernel's form
  static constexpr int kMaxRdCoeffs = PF_MAX_FIELDS + 1 + 2 * PF_MAX_FIELDS * pf::kRdMonomials;
  double rd_coeffs[kMaxRdCoeffs] = {};
  int rd_ncoeffs = 0;
  pf::RdParams rd{};
  int tile = -1;      // kernel tile id in effect (2D or 3D table)
  int k = 0;          // temporal-blocking depth in effect
  int req_tile = -1;  // tile asked for by pf_set_tuning (-1 = library default)
  int req_k = 0;      // depth asked for (0 = library default)
  double* red_partials = nullptr;  // kReduceBlocks partials + 1 result
  double* red_host = nullptr;      // pinned
  pf::AdjointState adj;
  pf::TmaCache tma;
  pf::Tma2Cache tma2;
  pf::Tb2Cache tb2;
  int* d_err = nullptr;  // set by a kernel whose bounded wait ran out
  // band kernel (2D grid resident in the SMs' shared memory): exchange slots of the bands'
  // edge rows as tagged 64-bit words, allocated at its first launch, and the last tag used
  unsigned long long* band_x = nullptr;
  size_t band_x_words = 0;
  unsigned int band_tag = 0;
  // CUDA-graph cache of pf_step: a few recorded launch sequences, keyed by
  // (steps, tile, k, starting buffer), least recently used replaced first
  cudaStream_t capture = nullptr;  // private stream used only to record graphs
  cudaStream_t capture2 = nullptr;  // second branch of the adjoint's reverse-pass graph
  struct StepGraph {
    cudaGraphExec_t exec = nullptr;
    int64_t steps = -1;
    int tile = -1, k = -1, start = -1, flip = 0;
    uint64_t used = 0;
  } step_graphs[4];
  uint64_t graph_clock = 0;
  // CUDA-graph cache of the adjoint's reverse pass
  cudaGraphExec_t adj_exec = nullptr;
  int64_t adj_exec_steps = -1, adj_exec_interval = -1;
  int adj_exec_lb = 0;  // lambda buffer holding lambda^0 after the graph
};

namespace pf {
void adjoint_release(pf_grid_s* g);
void drop_graphs(pf_grid_s* g);
int invalid(const char* fmt, ...);
int check_grid(pf_grid_s* g);
Geom grid_geom(const pf_grid_s* g);
ModelParams make_params(int model, const double* c, double dt, double h, int stencil = 0);
cudaError_t launch_step(pf_grid_s* g, int tile, int k, int src, int dst, cudaStream_t st);

// ---- 3D TMA kernels (AC, GS; Models B and C in pf_fe3d_tma2.cu): TMA tile ids 0 = 64x16,
// 1 = 128x8, 2 = 128x16
constexpr int kNumTmaTiles3D = 3;
void tma3d_tile_shape(int tma_tile, int* tx, int* ty);
bool fe3d_tma_supported(int model, int tma_tile, const Geom& g);
cudaError_t tma3d_maps(pf_grid_s* g, int tma_tile, int buf);
cudaError_t launch_fe3d_tma(pf_grid_s* g, int tma_tile, int src, int dst, cudaStream_t st);
// Models B and C on the same tiles (pf_fe3d_tma2.cu)
cudaError_t launch_fe3d_tma_r2(pf_grid_s* g, int tma_tile, int src, int dst, cudaStream_t st);

// ---- 2D band kernel (AC, CH; k = 1): one band of full rows per SM, all steps in one
// cooperative launch (pf_fe2d_bands.cu)
cudaError_t launch_fe2d_bands(pf_grid_s* g, int src, int dst, int64_t n_steps, cudaStream_t st);
void fe2d_bands_release(pf_grid_s* g);

// ---- 3D depth-2 kernel (AC, GS; full x-rows of 128 or 256, 8-row tiles)
bool fe3d_tb2_supported(int model, int tx, int ty, const Geom& g);
cudaError_t launch_fe3d_tb2(pf_grid_s* g, int tx, int src, int dst, cudaStream_t st);
}  // namespace pf
