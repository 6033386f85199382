// Batched 2D Gray-Scott runner: many independent periodic grids of uneven sizes and
// coefficients advance together, one launch per k steps over a flat (instance, tile) work
// list, the whole run captured once as a CUDA graph and replayed.  This is the GPU form of
// the paper's multi-model driver (Sec. 2.4, "simultaneous-configs"), which runs a list of
// models one after another on the CPU.
//
// Every instance runs the same tile body (or strip body) as the single-grid 2D kernels, so
// each instance's state is bitwise identical to running it alone through pf_step with any
// tuning.
#include <algorithm>
#include <functional>
#include <cmath>
#include <new>
#include <vector>

#include "pf_grid.h"
#include "pf_internal.h"

namespace pf {
double stable_dt_limit(int model, int dim, double h, const double* c, int stencil);
}

struct pf_batch_s {
  uint32_t magic = 0;
  int n = 0;
  double dt = 0, h = 1;
  cudaStream_t stream = nullptr;
  cudaStream_t capture = nullptr;  // private stream used only to record graphs
  std::vector<pf::BatchInst> insts;
  std::vector<int64_t> nx, ny;
  float* base[2] = {nullptr, nullptr};
  float* mem = nullptr;
  int64_t total_floats = 0;  // per buffer
  pf::BatchInst* d_insts = nullptr;
  pf::BatchTile* d_tiles[pf::kNumTiles2D] = {};
  int ntiles[pf::kNumTiles2D] = {};
  pf::BatchStrip* d_strips[6] = {};  // strip kernel work lists: (c = 4, 2) x (k = 1, 2, 4)
  int nstrips[6] = {};
  int cur = 0;
  int tile = 0;  // tile id in the 2D table, or pf::kTileStrips2D (+ 1): the strip kernel
  int k = 1;
  // graph cache: one executable per starting buffer for the current (steps, tile, k)
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  int64_t g_steps = -1;
  int g_tile = -1, g_k = -1;
  int g_flip = 0;
};

namespace pf {

constexpr uint32_t kBatchMagic = 0x50464254u;  // "PFBT"

static int check_batch(pf_batch_s* b) {
  if (b == nullptr || b->magic != kBatchMagic) return invalid("invalid batch handle");
  return PF_OK;
}

// Work list of every instance's tiles for tile id t (largest instances first).
static cudaError_t batch_tiles(pf_batch_s* b, int t) {
  if (b->d_tiles[t] != nullptr) return cudaSuccess;
  int tx, ty;
  tile2d_shape(t, &tx, &ty);
  std::vector<int> order(b->n);
  for (int i = 0; i < b->n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
    return b->nx[a] * b->ny[a] > b->nx[c] * b->ny[c];
  });
  std::vector<BatchTile> list;
  for (int i : order)
    for (int64_t y = 0; y < b->ny[i]; y += ty)
      for (int64_t x = 0; x < b->nx[i]; x += tx) list.push_back(BatchTile{i, (int)x, (int)y});
  if (list.size() > (size_t)INT32_MAX) return cudaErrorInvalidValue;
  cudaError_t e = cudaMalloc(&b->d_tiles[t], sizeof(BatchTile) * list.size());
  if (e != cudaSuccess) return e;
  e = cudaMemcpy(b->d_tiles[t], list.data(), sizeof(BatchTile) * list.size(),
                 cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  b->ntiles[t] = (int)list.size();
  return cudaSuccess;
}

static int kslot(int k) { return k == 4 ? 2 : k == 2 ? 1 : 0; }

// Strip kernel work list for strips of 32 c columns (c = 4 or 2) and depth k: per instance
// (largest first), its width split evenly over the fewest strips that cover it, each cut
// into tasks of hy rows; the strips of one band of rows are consecutive, so neighbouring
// warps share halo columns. One width for every strip: a narrower strip for an instance's
// remainder columns takes about as long per row as a full one (its warp waits on its row
// loads instead of sharing the issue slots), so remainder strips cost a whole strip each
// (measured: 512 instances of sides a multiple of 120, 682 GLUPS; the same sides plus one
// column, each with a 32-column remainder strip, 449).
//
// Split: s = ceil(nx / W) strips (W = the strip's output columns rounded down to a multiple
// of 4), boundaries b_j = 4 ceil(j nx / 4 s), b_s = nx. Then b_j - j nx / s lies in [0, 4), so
// an inner strip's width is a multiple of 4 below nx / s + 4 <= W + 4, i.e. at most W, and
// the last one is at most nx / s <= W; every width is positive once nx >= 4 s (for s >= 2,
// nx > W >= 24). The boundaries keep every strip's vector loads aligned.
//
// The task height hy is chosen for the launch as a whole. The device starts the one-warp
// tasks in list order as warps finish, so a list a little longer than a whole number of
// waves leaves most warps idle while the last tasks run (one 4096^2 instance: 3010 tasks of
// 48 rows on 2432 resident warps ran 46 % slower than 2415 tasks of 60 rows). Each
// candidate height's list is played through that dispatch on the resident warps, with a
// task costing its iterations (rows + the levels' start-up), and the shortest makespan wins
// (the taller height on a tie).
static std::vector<int> strip_bounds(int nx, int w) {
  const int s = (nx + w - 1) / w;
  std::vector<int> b(s + 1);
  for (int j = 0; j < s; ++j) b[j] = 4 * (int)(((int64_t)j * nx + 4 * s - 1) / (4 * s));
  b[s] = nx;
  return b;
}

static double strip_makespan(const pf_batch_s* b, const std::vector<int>& order,
                             const std::vector<int>& nstrips, int hy, int k, int resident,
                             std::vector<double>& slots) {
  slots.assign((size_t)resident, 0.0);
  std::make_heap(slots.begin(), slots.end(), std::greater<double>());
  double span = 0;
  for (int i : order) {
    const int ny = (int)b->ny[i];
    for (int y = 0; y < ny; y += hy) {
      const double cost = std::min(hy, ny - y) + 3.0 * k;
      for (int j = 0; j < nstrips[i]; ++j) {
        std::pop_heap(slots.begin(), slots.end(), std::greater<double>());
        slots.back() += cost;
        span = std::max(span, slots.back());
        std::push_heap(slots.begin(), slots.end(), std::greater<double>());
      }
    }
  }
  return span;
}

static int strip_c(int t) { return t == kTileStrips2D ? 4 : 2; }
static int strip_slot(int t, int k) { return (t - kTileStrips2D) * 3 + kslot(k); }

static cudaError_t batch_strips(pf_batch_s* b, int t, int k) {
  const int c = strip_c(t), slot = strip_slot(t, k);
  if (b->d_strips[slot] != nullptr) return cudaSuccess;
  const int w = strip_out_cols(PF_MODEL_GS, k, c) / 4 * 4;
  if (w <= 0) return cudaErrorInvalidValue;
  std::vector<int> order(b->n), nstrips(b->n);
  for (int i = 0; i < b->n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int q) {
    return b->nx[a] * b->ny[a] > b->nx[q] * b->ny[q];
  });
  int64_t strip_rows_total = 0;  // rows of every strip: the task count at hy = 1
  for (int i = 0; i < b->n; ++i) {
    nstrips[i] = (int)((b->nx[i] + w - 1) / w);
    strip_rows_total += (int64_t)nstrips[i] * b->ny[i];
  }
  // candidate heights: from the floor up, skipping those whose lists would be too long to
  // play through cheaply (a list of a few million tasks is past every tail effect anyway)
  const int resident = batch_gs2d_strips_resident(k, c);
  const int floor_rows = strip_task_rows(PF_MODEL_GS, k);
  int hy = 0;
  double best = 0;
  std::vector<double> slots;
  for (int h = floor_rows; h <= 192; h += 4) {
    if (strip_rows_total / h > (int64_t)1 << 22 && h < 192) continue;
    const double span = strip_makespan(b, order, nstrips, h, k, resident, slots);
    if (hy == 0 || span <= best) {
      best = span;
      hy = h;
    }
  }
  std::vector<BatchStrip> list;
  for (int i : order) {
    const int ny = (int)b->ny[i];
    const std::vector<int> xb = strip_bounds((int)b->nx[i], w);
    for (int y = 0; y < ny; y += hy)
      for (size_t j = 0; j + 1 < xb.size(); ++j) {
        const int wo = xb[j + 1] - xb[j];
        if (wo <= 0 || wo > w) return cudaErrorInvalidValue;  // excluded by the split's bound
        list.push_back(BatchStrip{i, xb[j], y, (short)std::min(hy, ny - y), (short)wo});
      }
  }
  if (list.size() > (size_t)INT32_MAX) return cudaErrorInvalidValue;
  cudaError_t e = cudaMalloc(&b->d_strips[slot], sizeof(BatchStrip) * list.size());
  if (e != cudaSuccess) return e;
  e = cudaMemcpy(b->d_strips[slot], list.data(), sizeof(BatchStrip) * list.size(),
                 cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  b->nstrips[slot] = (int)list.size();
  return cudaSuccess;
}

static cudaError_t batch_launch(pf_batch_s* b, int t, int k, int src, cudaStream_t s) {
  if (t == kTileStrips2D || t == kTileStrips2D + 1) {
    cudaError_t e = batch_strips(b, t, k);
    if (e != cudaSuccess) return e;
    const int slot = strip_slot(t, k);
    return launch_batch_gs2d_strips(strip_c(t), k, b->d_insts, b->d_strips[slot],
                                    b->nstrips[slot], b->base[src], b->base[1 - src], s);
  }
  cudaError_t e = batch_tiles(b, t);
  if (e != cudaSuccess) return e;
  return launch_batch_gs2d(t, k, b->d_insts, b->d_tiles[t], b->ntiles[t], b->base[src],
                           b->base[1 - src], s);
}

static void drop_graphs(pf_batch_s* b) {
  for (int i = 0; i < 2; ++i) {
    if (b->exec[i]) cudaGraphExecDestroy(b->exec[i]);
    b->exec[i] = nullptr;
  }
  b->g_steps = -1;
}

}  // namespace pf

using namespace pf;

extern "C" {

int pf_batch_create(int n, const pf_gs2d_spec* specs, double dt, double h, void* stream,
                    pf_batch_t* out) {
  if (out == nullptr) return invalid("out is NULL");
  *out = nullptr;
  if (n < 1 || specs == nullptr) return invalid("need n >= 1 instance specs");
  if (!(dt > 0) || !(h > 0) || !std::isfinite(dt) || !std::isfinite(h))
    return invalid("dt and h must be finite and > 0");
  const int64_t lim = (int64_t)1 << 20;
  int64_t total = 0;
  for (int i = 0; i < n; ++i) {
    const pf_gs2d_spec& s = specs[i];
    if (s.nx < 1 || s.ny < 1 || s.nx > lim || s.ny > lim)
      return invalid("instance %d: sizes must be in [1, 2^20]", i);
    const double c[4] = {s.Du, s.Dv, s.F, s.k};
    for (double v : c)
      if (!std::isfinite(v)) return invalid("instance %d: non-finite coefficient", i);
    if (dt > stable_dt_limit(PF_MODEL_GS, 2, h, c, PF_ST_STD)) {
      set_error("instance %d: dt = %g exceeds the forward-Euler stability limit %g", i, dt,
                stable_dt_limit(PF_MODEL_GS, 2, h, c, PF_ST_STD));
      return PF_ERR_UNSTABLE_DT;
    }
    const int64_t pitch = (s.nx + 3) / 4 * 4;
    total += (2 * pitch * s.ny + 63) / 64 * 64;  // u and v, 256-byte aligned
  }
  pf_batch_s* b = new (std::nothrow) pf_batch_s();
  if (b == nullptr) return PF_ERR_OOM;
  b->magic = kBatchMagic;
  b->n = n;
  b->dt = dt;
  b->h = h;
  b->stream = (cudaStream_t)stream;
  b->insts.resize(n);
  b->nx.resize(n);
  b->ny.resize(n);
  int64_t off = 0;
  for (int i = 0; i < n; ++i) {
    const pf_gs2d_spec& s = specs[i];
    const double c[4] = {s.Du, s.Dv, s.F, s.k};
    BatchInst& I = b->insts[i];
    I.nx = (int)s.nx;
    I.ny = (int)s.ny;
    I.pitch = (s.nx + 3) / 4 * 4;
    I.off = off;
    I.m = make_params(PF_MODEL_GS, c, dt, h);
    b->nx[i] = s.nx;
    b->ny[i] = s.ny;
    off += (2 * I.pitch * s.ny + 63) / 64 * 64;
  }
  b->total_floats = total;
  cudaError_t e = cudaMalloc(&b->mem, sizeof(float) * total * 2);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->mem, 0, sizeof(float) * total * 2, b->stream);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_insts, sizeof(BatchInst) * n);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_insts, b->insts.data(), sizeof(BatchInst) * n,
                        cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = prepare_batch_gs2d();
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    int rc = cuda_fail(e, "pf_batch_create");
    pf_batch_destroy(b);
    return rc;
  }
  b->base[0] = b->mem;
  b->base[1] = b->mem + total;
  b->tile = 0;  // 64 x 16
  b->k = 1;
  *out = b;
  return PF_OK;
}

void pf_batch_destroy(pf_batch_t b) {
  if (b == nullptr || b->magic != kBatchMagic) return;
  cudaStreamSynchronize(b->stream);
  drop_graphs(b);
  for (int t = 0; t < kNumTiles2D; ++t)
    if (b->d_tiles[t]) cudaFree(b->d_tiles[t]);
  for (int i = 0; i < 6; ++i)
    if (b->d_strips[i]) cudaFree(b->d_strips[i]);
  if (b->d_insts) cudaFree(b->d_insts);
  if (b->mem) cudaFree(b->mem);
  if (b->capture) cudaStreamDestroy(b->capture);
  b->magic = 0;
  delete b;
}

int pf_batch_write_field(pf_batch_t b, int inst, int field, const float* src, int on_device) {
  if (int rc = check_batch(b)) return rc;
  if (inst < 0 || inst >= b->n || field < 0 || field > 1 || src == nullptr)
    return invalid("bad instance %d / field %d / src", inst, field);
  const BatchInst& I = b->insts[inst];
  float* dst = b->base[b->cur] + I.off + field * I.pitch * I.ny;
  const size_t w = sizeof(float) * I.nx;
  PF_CUDA_TRY(cudaMemcpy2DAsync(dst, sizeof(float) * I.pitch, src, w, w, I.ny,
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                b->stream));
  if (!on_device) PF_CUDA_TRY(cudaStreamSynchronize(b->stream));
  return PF_OK;
}

int pf_batch_read_field(pf_batch_t b, int inst, int field, float* dst, int on_device) {
  if (int rc = check_batch(b)) return rc;
  if (inst < 0 || inst >= b->n || field < 0 || field > 1 || dst == nullptr)
    return invalid("bad instance %d / field %d / dst", inst, field);
  const BatchInst& I = b->insts[inst];
  const float* src = b->base[b->cur] + I.off + field * I.pitch * I.ny;
  const size_t w = sizeof(float) * I.nx;
  PF_CUDA_TRY(cudaMemcpy2DAsync(dst, w, src, sizeof(float) * I.pitch, w, I.ny,
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                b->stream));
  if (!on_device) PF_CUDA_TRY(cudaStreamSynchronize(b->stream));
  return PF_OK;
}

int pf_batch_set_tuning(pf_batch_t b, int tile_x, int tile_y, int k_steps) {
  if (int rc = check_batch(b)) return rc;
  int t = b->tile;
  if (tile_y == PF_TILE_STRIPS) {
    if (tile_x != 128 && tile_x != 64)
      return invalid("the batch's strip kernel takes tile 128 or 64 x PF_TILE_STRIPS");
    t = tile_x == 128 ? kTileStrips2D : kTileStrips2D + 1;
  } else if (tile_x != 0 || tile_y != 0) {
    t = tile2d_id(tile_x, tile_y);
    if (t < 0) return invalid("unsupported 2D tile %dx%d", tile_x, tile_y);
  }
  int k = k_steps == 0 ? b->k : k_steps;
  if (!fe2d_supported(PF_MODEL_GS, k)) return invalid("unsupported temporal depth %d", k);
  b->tile = t;
  b->k = k;
  return PF_OK;
}

int pf_batch_get_tuning(pf_batch_t b, int* tile_x, int* tile_y, int* k_steps) {
  if (int rc = check_batch(b)) return rc;
  int tx = b->tile == kTileStrips2D ? 128 : 64, ty = PF_TILE_STRIPS;
  if (b->tile < kTileStrips2D) tile2d_shape(b->tile, &tx, &ty);
  if (tile_x) *tile_x = tx;
  if (tile_y) *tile_y = ty;
  if (k_steps) *k_steps = b->k;
  return PF_OK;
}

int pf_batch_autotune(pf_batch_t b, int probe_launches, int* tile_x, int* tile_y,
                      int* k_steps) {
  NvtxRange nvtx_("pf_batch_autotune");
  if (int rc = check_batch(b)) return rc;
  if (probe_launches < 1) probe_launches = 3;
  cudaEvent_t e0, e1;
  PF_CUDA_TRY(cudaEventCreate(&e0));
  PF_CUDA_TRY(cudaEventCreate(&e1));
  float best = INFINITY;
  int bt = b->tile, bk = b->k;
  static const int ks[3] = {1, 2, 4};
  cudaError_t e = cudaSuccess;
  for (int ti = 0; ti < kNumTiles2D + 2 && e == cudaSuccess; ++ti) {
    // the tiles, then the strip kernel with 128- and 64-column strips
    const int t = ti < kNumTiles2D ? ti : kTileStrips2D + (ti - kNumTiles2D);
    for (int ki = 0; ki < 3 && e == cudaSuccess; ++ki) {
      const int k = ks[ki];
      e = batch_launch(b, t, k, b->cur, b->stream);  // warm-up (state unchanged)
      if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
      for (int i = 0; i < probe_launches && e == cudaSuccess; ++i)
        e = batch_launch(b, t, k, b->cur, b->stream);
      if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e == cudaSuccess && ms / (probe_launches * k) < best) {
        best = ms / (probe_launches * k);
        bt = t;
        bk = k;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(e, "pf_batch_autotune");
  b->tile = bt;
  b->k = bk;
  return pf_batch_get_tuning(b, tile_x, tile_y, k_steps);
}

int pf_batch_run(pf_batch_t b, int64_t n_steps) {
  NvtxRange nvtx_("pf_batch_run");
  if (int rc = check_batch(b)) return rc;
  if (n_steps < 0) return invalid("n_steps must be >= 0");
  if (n_steps == 0) return PF_OK;
  if (b->g_steps != n_steps || b->g_tile != b->tile || b->g_k != b->k) drop_graphs(b);
  if (b->exec[b->cur] == nullptr) {
    const bool strips = b->tile >= kTileStrips2D;
    cudaError_t e = strips ? cudaSuccess : batch_tiles(b, b->tile);
    for (int k = b->k; k >= 1 && e == cudaSuccess && strips; k >>= 1)
      e = batch_strips(b, b->tile, k);  // allocate outside the capture (every depth used)
    if (e != cudaSuccess) return cuda_fail(e, "pf_batch_run work list");
    PF_CUDA_TRY(cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal));
    int src = b->cur;
    int64_t left = n_steps;
    int launches = 0;
    while (left > 0 && e == cudaSuccess) {
      int k = b->k;
      while (k > left) k >>= 1;
      e = batch_launch(b, b->tile, k, src, b->capture);
      src = 1 - src;
      left -= k;
      ++launches;
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(b->capture, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return cuda_fail(e != cudaSuccess ? e : e2, "pf_batch_run capture");
    }
    e = cudaGraphInstantiate(&b->exec[b->cur], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      b->exec[b->cur] = nullptr;
      return cuda_fail(e, "cudaGraphInstantiate");
    }
    b->g_steps = n_steps;
    b->g_tile = b->tile;
    b->g_k = b->k;
    b->g_flip = launches & 1;
  }
  PF_CUDA_TRY(cudaGraphLaunch(b->exec[b->cur], b->stream));
  if (b->g_flip) b->cur = 1 - b->cur;
  return PF_OK;
}

int pf_batch_synchronize(pf_batch_t b) {
  if (int rc = check_batch(b)) return rc;
  PF_CUDA_TRY(cudaStreamSynchronize(b->stream));
  return PF_OK;
}

int pf_batch_info(pf_batch_t b, int64_t* sites, int64_t* bytes_per_copy) {
  if (int rc = check_batch(b)) return rc;
  int64_t s = 0;
  for (int i = 0; i < b->n; ++i) s += b->nx[i] * b->ny[i];
  if (sites) *sites = s;
  if (bytes_per_copy) *bytes_per_copy = b->total_floats * (int64_t)sizeof(float);
  return PF_OK;
}

}  // extern "C"
