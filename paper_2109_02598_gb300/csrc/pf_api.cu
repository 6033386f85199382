// C ABI of libpfgpu: grid handles, model selection, field I/O, stepping, reductions and
// tuning.  Declarations and contracts are in include/pfgpu.h.
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <new>

#include "pf_grid.h"
#include "pf_internal.h"

namespace pf {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

int cuda_fail(cudaError_t e, const char* what) {
  set_error("CUDA error %d (%s) in %s: %s", (int)e, cudaGetErrorName(e), what,
            cudaGetErrorString(e));
  // reset the runtime's last error, so a failed launch that left the context usable (a
  // grid too large to co-schedule, a bad configuration) is not reported again by the next
  // launch's check; an error that poisons the context keeps failing every later call anyway
  (void)cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? PF_ERR_OOM : PF_ERR_CUDA;
}

int invalid(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return PF_ERR_INVALID_ARG;
}

int model_fields(int model) {
  switch (model) {
    case PF_MODEL_AC: return 1;
    case PF_MODEL_CH: return 1;
    case PF_MODEL_GS: return 2;
    case PF_MODEL_C: return 2;
    case PF_MODEL_RD: return -1;  // the grid's field count, 1 .. PF_MAX_FIELDS
  }
  return 0;
}

int model_ncoeffs(int model) {
  switch (model) {
    case PF_MODEL_AC: return 2;
    case PF_MODEL_CH: return 3;
    case PF_MODEL_GS: return 4;
    case PF_MODEL_C: return 5;
  }
  return 0;
}

// Linear forward-Euler stability: dt * |largest eigenvalue of the linearised right-hand
// side| <= 2, with the periodic Laplacian's spectrum in [-4d/h^2, 0] and, for AC/CH, the
// cubic term linearised about |phi| <= 1 (slope between -c1 and 3 c2 - c1).
// Largest magnitude of the Laplacian stencil's Fourier symbol, times h^2.
double stencil_lmax(int dim, int stencil) {
  if (stencil == PF_ST_ISO) return 16.0 / 3.0;               // 9-point (pi,pi); 19-point (pi,pi,0)
  if (stencil == PF_ST_O4) return 32.0 / 3.0;                // fourth order, both axes at pi
  if (stencil == PF_ST_ISO27) return 92.0 / 15.0;            // 27-point (pi,pi,pi): 184/30
  return 4.0 * dim;                                          // 5- / 7-point
}

double stable_dt_limit(int model, int dim, double h, const double* c, int stencil = PF_ST_STD) {
  const double lmax = stencil_lmax(dim, stencil) / (h * h);
  switch (model) {
    case PF_MODEL_AC: {
      const double s = lmax + std::fmax(0.0, 3.0 * c[1] - c[0]);
      return s > 0 ? 2.0 / s : INFINITY;
    }
    case PF_MODEL_CH: {
      const double s = c[2] * lmax * (lmax + std::fmax(0.0, 3.0 * c[1] - c[0]));
      return s > 0 ? 2.0 / s : INFINITY;
    }
    case PF_MODEL_GS: {
      const double s = std::fmax(c[0], c[1]) * lmax + c[2] + c[3];
      return s > 0 ? 2.0 / s : INFINITY;
    }
    case PF_MODEL_C: {  // the stiffer of the psi (Model A-like) and m (Model B-like) parts
      const double sa = lmax + std::fmax(0.0, 3.0 * c[1] - c[0]) + 2.0 * std::fabs(c[4]);
      const double sb = lmax * (lmax + std::fmax(0.0, 3.0 * c[3] - c[2]));
      const double s = std::fmax(sa, sb);
      return s > 0 ? 2.0 / s : INFINITY;
    }
  }
  return 0.0;
}

ModelParams make_params(int model, const double* c, double dt, double h, int stencil) {
  ModelParams m{};
  m.dt = (float)dt;
  const double denom = stencil == PF_ST_ISO     ? 6.0
                       : stencil == PF_ST_O4    ? 12.0
                       : stencil == PF_ST_ISO27 ? 30.0
                                                : 1.0;
  m.lap_scale = (float)(1.0 / (denom * h * h));
  switch (model) {
    case PF_MODEL_AC:
      m.a0 = (float)c[0];
      m.a1 = (float)c[1];
      break;
    case PF_MODEL_CH:
      m.a0 = (float)c[0];
      m.a1 = (float)c[1];
      m.a2 = (float)(dt * c[2]);
      break;
    case PF_MODEL_GS:
      // the stencil factor goes into the diffusion coefficients (the only terms with a
      // Laplacian), so Gray-Scott kernels may skip the multiply by lap_scale = 1
      m.a0 = (float)(c[0] * (double)m.lap_scale);
      m.a1 = (float)(c[1] * (double)m.lap_scale);
      m.a2 = (float)c[2];
      m.a3 = (float)(c[2] + c[3]);
      m.lap_scale = 1.0f;
      break;
    case PF_MODEL_C:
      m.a0 = (float)c[0];
      m.a1 = (float)c[1];
      m.a2 = (float)c[2];
      m.a3 = (float)c[3];
      m.a4 = (float)c[4];
      m.a5 = (float)(2.0 * c[4]);
      break;
  }
  return m;
}

Geom grid_geom(const pf_grid_s* g) {
  Geom q{};
  q.dim = g->dim;
  q.nx = g->nx;
  q.ny = g->ny;
  q.nz = g->nz;
  q.pitch = g->pitch;
  q.plane = g->plane;
  return q;
}

bool tile_supported(pf_grid_s* g, int tile, int k);

// Turn the requested tuning (or the defaults) into the tuning in effect for the current
// model and grid.
int resolve_tuning(pf_grid_s* g) {
  if (g->model_set && g->model == PF_MODEL_RD) {  // one kernel per dimension (pf_rdn.cu)
    g->tile = 0;
    g->k = 1;
    return PF_OK;
  }
  if (g->dim == 2) {
    const int def = g->stencil == PF_ST_STD ? 1 : 0;  // 128 x 16; other stencils 64 x 16
    g->tile = g->req_tile >= 0 ? g->req_tile : def;
    g->k = g->req_k > 0 ? g->req_k : 1;
    const bool on_chip = g->tile == kTileCluster2D || g->tile == kTileBands2D;
    const bool strips = g->tile >= kTileStrips2D && g->tile < kTileStrips2D + kNumStrips2D;
    if (!on_chip && !strips && g->model_set && !fe2d_supported(g->model, g->k)) g->k = 1;
    if (strips) {
      if (!(g->model_set && tile_supported(g, g->tile, g->k))) {
        g->tile = def;
        g->k = 1;
      }
    } else if (on_chip) {
      if (!(g->model_set && tile_supported(g, g->tile, g->k))) {
        g->tile = def;
        g->k = 1;
      }
    } else if (!fe2d_stencil_supported(g->stencil, g->tile, g->k)) {
      g->tile = def;
      g->k = 1;
    }
  } else if (g->stencil != PF_ST_STD) {
    g->tile = (g->req_tile == 0 || g->req_tile == 1) ? g->req_tile : 0;  // general kernel
    g->k = 1;
  } else {
    // default: the fastest TMA tile that divides the grid (measured on GS 256^3:
    // 128x16 > 64x16 = 128x8), else the general kernel
    int def = 0;
    if (g->model_set) {
      static const int pref[3] = {2, 0, 1};  // TMA tile ids 128x16, 64x16, 128x8
      for (int i = 0; i < 3 && def == 0; ++i)
        if (fe3d_tma_supported(g->model, pref[i], grid_geom(g))) def = kFirstTmaTile3D + pref[i];
    }
    g->tile = g->req_tile >= 0 ? g->req_tile : def;
    g->k = g->req_k > 0 ? g->req_k : 1;
    if (!(g->model_set && tile_supported(g, g->tile, g->k))) {
      g->tile = def;
      g->k = 1;
    }
  }
  return PF_OK;
}

bool tile_supported(pf_grid_s* g, int tile, int k) {
  if (g->model == PF_MODEL_RD) return tile == 0 && k == 1;
  if (g->dim == 2 && tile == kTileCluster2D)
    return g->stencil == PF_ST_STD && fe2d_cluster_supported(g->model, k, grid_geom(g));
  if (g->dim == 2 && tile == kTileBands2D)
    return g->stencil == PF_ST_STD && k == 1 && fe2d_bands_supported(g->model, grid_geom(g));
  if (g->dim == 2 && tile >= kTileStrips2D && tile < kTileStrips2D + kNumStrips2D)
    return fe2d_strips_supported(g->model, k, g->stencil);
  if (g->dim == 2) return fe2d_supported(g->model, k) && fe2d_stencil_supported(g->stencil, tile, k);
  if (g->stencil != PF_ST_STD) return (tile == 0 || tile == 1) && k == 1;
  if (tile == kTileBox3D) return fe3d_box_supported(g->model, k, grid_geom(g));
  int tx, ty;
  tile3d_shape(tile, &tx, &ty);
  if (k == 2) return fe3d_tb2_supported(g->model, tx, ty, grid_geom(g));
  if (k != 1) return false;
  if (tile < kFirstTmaTile3D) return true;
  return fe3d_tma_supported(g->model, tile - kFirstTmaTile3D, grid_geom(g));
}

// The depth-1 kernel used for the remainder of a depth-2 launch plan: the tile itself if it
// has a depth-1 form, else the fastest depth-1 TMA tile that divides the grid, else the
// general kernel (every path gives the same result bit for bit).
int k1_tile(pf_grid_s* g, int tile) {
  if (tile_supported(g, tile, 1)) return tile;
  static const int pref[3] = {2, 0, 1};
  for (int i = 0; i < 3; ++i)
    if (fe3d_tma_supported(g->model, pref[i], grid_geom(g))) return kFirstTmaTile3D + pref[i];
  return 0;
}

// A kernel that gave up on a bounded wait leaves a flag; report it (and clear it).
int check_device_error(pf_grid_s* g) {
  int flag = 0;
  PF_CUDA_TRY(cudaMemcpyAsync(&flag, g->d_err, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
  PF_CUDA_TRY(cudaStreamSynchronize(g->stream));
  if (flag != 0) {
    PF_CUDA_TRY(cudaMemsetAsync(g->d_err, 0, sizeof(int), g->stream));
    set_error("a kernel's bounded wait (for a TMA copy or a neighbouring band) ran out; the "
              "state is invalid");
    return PF_ERR_TIMEOUT;
  }
  return PF_OK;
}

int k1_tile(pf_grid_s* g, int tile);

// One launch advancing `k` steps from buffer `src` into buffer `dst`.
cudaError_t launch_step(pf_grid_s* g, int tile, int k, int src, int dst, cudaStream_t st) {
  FieldPtrs in{};
  FieldOut out{};
  for (int f = 0; f < g->nf; ++f) {
    in.f[f] = g->buf[src][f];
    out.f[f] = g->buf[dst][f];
  }
  const Geom q = grid_geom(g);
  if (g->model == PF_MODEL_RD) return launch_rd(q, g->nf, in, out, g->rd, st);
  if (g->dim == 2 && tile == kTileCluster2D)
    return launch_fe2d_cluster(g->model, k, q, in, out, g->params, k, st);
  if (g->dim == 2 && tile == kTileBands2D) return launch_fe2d_bands(g, src, dst, k, st);
  if (g->dim == 2 && tile >= kTileStrips2D && tile < kTileStrips2D + kNumStrips2D)
    return launch_fe2d_strips(g->model, g->stencil, tile == kTileStrips2D ? 128 : 64, k, q, in,
                              out, g->params, st);
  if (g->dim == 2) return launch_fe2d_stencil(g->stencil, g->model, tile, k, q, in, out, g->params, st);
  if (g->stencil != PF_ST_STD) return launch_fe3d(g->model, tile, q, in, out, g->params, st, g->stencil);
  if (tile == kTileBox3D) return launch_fe3d_box(g->model, k, q, in, out, g->params, st);
  if (k == 2) {
    int tx, ty;
    tile3d_shape(tile, &tx, &ty);
    return launch_fe3d_tb2(g, tx, src, dst, st);
  }
  tile = k1_tile(g, tile);
  if (tile >= kFirstTmaTile3D) return launch_fe3d_tma(g, tile - kFirstTmaTile3D, src, dst, st);
  return launch_fe3d(g->model, tile, q, in, out, g->params, st);
}

// Forget every recorded graph (their kernel parameters carry coefficients and tuning).
void drop_graphs(pf_grid_s* g) {
  for (auto& sg : g->step_graphs) {
    if (sg.exec) cudaGraphExecDestroy(sg.exec);
    sg = pf_grid_s::StepGraph();
  }
  if (g->adj_exec) cudaGraphExecDestroy(g->adj_exec);
  g->adj_exec = nullptr;
  g->adj_exec_steps = -1;
}

// Launch plan of pf_step: depths k, k, ..., then smaller ones for the remainder.
static int count_launches(int64_t n, int kmax) {
  int c = 0;
  while (n > 0) {
    int k = kmax;
    while (k > n) k >>= 1;
    n -= k;
    ++c;
  }
  return c;
}

// Record the launches of pf_step(n) from buffer g->cur into a graph on the private stream.
static int record_step_graph(pf_grid_s* g, int64_t n, cudaGraphExec_t* exec, int* flip) {
  if (g->capture == nullptr)
    PF_CUDA_TRY(cudaStreamCreateWithFlags(&g->capture, cudaStreamNonBlocking));
  PF_CUDA_TRY(cudaStreamBeginCapture(g->capture, cudaStreamCaptureModeRelaxed));
  cudaError_t e = cudaSuccess;
  int src = g->cur, launches = 0;
  int64_t left = n;
  while (left > 0 && e == cudaSuccess) {
    int k = g->k;
    while (k > left) k >>= 1;
    e = launch_step(g, g->tile, k, src, 1 - src, g->capture);
    src = 1 - src;
    left -= k;
    ++launches;
  }
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(g->capture, &graph);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cuda_fail(e != cudaSuccess ? e : e2, "pf_step graph capture");
  }
  e = cudaGraphInstantiate(exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    *exec = nullptr;
    return cuda_fail(e, "pf_step cudaGraphInstantiate");
  }
  *flip = launches & 1;
  return PF_OK;
}

constexpr int kGraphMinLaunches = 8;

int check_grid(pf_grid_s* g) {
  if (g == nullptr || g->magic != kGridMagic) return invalid("invalid grid handle");
  return PF_OK;
}

}  // namespace pf

using namespace pf;

extern "C" {

int pf_version(void) { return 10100; }

const char* pf_last_error(void) { return g_err; }

int pf_create_grid(int dim, const int64_t* n, int n_fields, double h, void* stream,
                   pf_grid_t* out) {
  if (out == nullptr) return invalid("out is NULL");
  *out = nullptr;
  if (dim != 2 && dim != 3) return invalid("dim must be 2 or 3 (got %d)", dim);
  if (n == nullptr) return invalid("n is NULL");
  const int64_t nz = dim == 3 ? n[2] : 1;
  const int64_t lim = (int64_t)1 << 30;
  if (n[0] < 1 || n[1] < 1 || nz < 1 || n[0] > lim || n[1] > lim || nz > lim)
    return invalid("grid sizes must be in [1, 2^30] (got %lld x %lld x %lld)",
                   (long long)n[0], (long long)n[1], (long long)nz);
  if (n_fields < 1 || n_fields > PF_MAX_FIELDS)
    return invalid("n_fields must be in [1, %d] (got %d)", PF_MAX_FIELDS, n_fields);
  if (!(h > 0.0) || !std::isfinite(h)) return invalid("h must be finite and > 0");
  const int64_t pitch = (n[0] + 3) / 4 * 4;
  const int64_t plane = pitch * n[1];  // <= (2^30 + 3) 2^30: no overflow
  const int64_t max_elems = (int64_t)1 << 36;
  if (plane > max_elems || nz > max_elems / plane)  // by division: plane * nz may overflow
    return invalid("grid too large: %lld x %lld x %lld floats exceed 2^36", (long long)pitch,
                   (long long)n[1], (long long)nz);
  const int64_t elems = plane * nz;
  pf_grid_s* g = new (std::nothrow) pf_grid_s();
  if (g == nullptr) return PF_ERR_OOM;
  g->magic = kGridMagic;
  g->dim = dim;
  g->nx = (int)n[0];
  g->ny = (int)n[1];
  g->nz = (int)nz;
  g->nf = n_fields;
  g->h = h;
  g->stream = (cudaStream_t)stream;
  g->pitch = pitch;
  g->plane = plane;
  g->field_elems = elems;
  cudaError_t e = cudaGetDevice(&g->device);
  if (e == cudaSuccess) e = cudaMalloc(&g->base, sizeof(float) * elems * 2 * n_fields);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->base, 0, sizeof(float) * elems * 2 * n_fields, g->stream);
  if (e == cudaSuccess) e = cudaMalloc(&g->red_partials, sizeof(double) * (kReduceBlocks + 1));
  if (e == cudaSuccess) e = cudaMallocHost(&g->red_host, sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&g->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(g->d_err, 0, sizeof(int), g->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess) {
    int rc = cuda_fail(e, "pf_create_grid allocation");
    pf_destroy(g);
    return rc;
  }
  for (int b = 0; b < 2; ++b)
    for (int f = 0; f < n_fields; ++f) g->buf[b][f] = g->base + (b * n_fields + f) * elems;
  g->cur = 0;
  g->req_tile = -1;
  g->req_k = 0;
  resolve_tuning(g);
  *out = g;
  return PF_OK;
}

void pf_destroy(pf_grid_t g) {
  if (g == nullptr || g->magic != kGridMagic) return;
  cudaStreamSynchronize(g->stream);
  pf::adjoint_release(g);
  pf::fe2d_bands_release(g);
  drop_graphs(g);
  if (g->capture) cudaStreamDestroy(g->capture);
  if (g->capture2) cudaStreamDestroy(g->capture2);
  if (g->base) cudaFree(g->base);
  if (g->red_partials) cudaFree(g->red_partials);
  if (g->red_host) cudaFreeHost(g->red_host);
  if (g->d_err) cudaFree(g->d_err);
  g->magic = 0;
  delete g;
}

// N coupled species: coefficients D_0 .. D_{N-1}, M, the M x N exponents (row by row), the
// N x M rates (row by row), N = the grid's field count.
int set_model_rd(pf_grid_s* g, const double* c, int n_coeffs, double dt, int force) {
  const int N = g->nf;
  if (c == nullptr || n_coeffs < N + 1) return invalid("N-species model: coefficient list too short");
  for (int i = 0; i < n_coeffs; ++i)
    if (!std::isfinite(c[i])) return invalid("coefficient %d is not finite", i);
  const double mm = c[N];
  if (!(mm >= 0 && mm <= kRdMonomials && mm == std::floor(mm)))
    return invalid("N-species model: the monomial count (coefficient %d) must be an integer "
                   "in [0, %d]", N, kRdMonomials);
  const int M = (int)mm;
  if (n_coeffs != N + 1 + 2 * N * M)
    return invalid("N-species model with %d fields and %d monomials takes %d coefficients "
                   "(got %d)", N, M, N + 1 + 2 * N * M, n_coeffs);
  for (int i = 0; i < N; ++i)
    if (c[i] < 0) return invalid("diffusion coefficient D_%d must be >= 0", i);
  const double* E = c + N + 1;
  const double* K = E + M * N;
  for (int i = 0; i < M * N; ++i)
    if (!(E[i] >= 0 && E[i] <= 3 && E[i] == std::floor(E[i])))
      return invalid("exponents must be integers in [0, 3] (coefficient %d)", N + 1 + i);
  if (g->stencil != PF_ST_STD) return invalid("the N-species model runs with the 5-/7-point stencil");
  if (!(dt > 0.0) || !std::isfinite(dt)) return invalid("dt must be finite and > 0");
  // stability of the diffusion part (the reaction terms depend on the state): dt max D
  // (4 d / h^2) <= 2
  double dmax = 0;
  for (int i = 0; i < N; ++i) dmax = std::fmax(dmax, c[i]);
  const double lim = dmax > 0 ? 2.0 * g->h * g->h / (dmax * 4.0 * g->dim) : INFINITY;
  if (dt > lim && !force) {
    set_error("dt = %g exceeds the forward-Euler stability limit %g of the diffusion terms "
              "(pass force=1 to accept)", dt, lim);
    return PF_ERR_UNSTABLE_DT;
  }
  RdParams p{};
  p.nmono = M;
  for (int m = 0; m < M; ++m) {
    int packed = 0;
    for (int j = 0; j < N; ++j) packed |= ((int)E[m * N + j]) << (2 * j);
    p.E[m] = packed;
  }
  for (int i = 0; i < N; ++i) {
    p.D[i] = (float)(c[i] / (g->h * g->h));
    for (int m = 0; m < M; ++m) p.K[i][m] = (float)K[i * M + m];
  }
  p.dt = (float)dt;
  g->model = PF_MODEL_RD;
  g->rd = p;
  g->rd_ncoeffs = n_coeffs;
  for (int i = 0; i < n_coeffs; ++i) g->rd_coeffs[i] = c[i];
  g->dt = dt;
  g->model_set = 1;
  drop_graphs(g);
  resolve_tuning(g);
  return PF_OK;
}

int pf_set_model(pf_grid_t g, int model, const double* coeffs, int n_coeffs, double dt,
                 int force) {
  if (int rc = check_grid(g)) return rc;
  if (model == PF_MODEL_RD) return set_model_rd(g, coeffs, n_coeffs, dt, force);
  if (model_fields(model) == 0) return invalid("unknown model %d", model);
  if (model_fields(model) != g->nf)
    return invalid("model %d needs %d field(s); grid has %d", model, model_fields(model), g->nf);
  if (coeffs == nullptr || n_coeffs != model_ncoeffs(model))
    return invalid("model %d takes exactly %d coefficients (got %d)", model,
                   model_ncoeffs(model), n_coeffs);
  for (int i = 0; i < n_coeffs; ++i)
    if (!std::isfinite(coeffs[i])) return invalid("coefficient %d is not finite", i);
  if (!(dt > 0.0) || !std::isfinite(dt)) return invalid("dt must be finite and > 0");
  const double lim = stable_dt_limit(model, g->dim, g->h, coeffs, g->stencil);
  if (dt > lim && !force) {
    set_error("dt = %g exceeds the forward-Euler stability limit %g for this model and grid "
              "(pass force=1 to accept)", dt, lim);
    return PF_ERR_UNSTABLE_DT;
  }
  g->model = model;
  for (int i = 0; i < n_coeffs; ++i) g->coeffs[i] = coeffs[i];
  g->dt = dt;
  g->params = make_params(model, coeffs, dt, g->h, g->stencil);
  g->model_set = 1;
  drop_graphs(g);  // recorded graphs carry the old coefficients
  resolve_tuning(g);
  return PF_OK;
}

int pf_write_field(pf_grid_t g, int field, const float* src, int src_on_device) {
  if (int rc = check_grid(g)) return rc;
  if (field < 0 || field >= g->nf) return invalid("field %d out of range", field);
  if (src == nullptr) return invalid("src is NULL");
  const size_t w = sizeof(float) * g->nx;
  PF_CUDA_TRY(cudaMemcpy2DAsync(g->buf[g->cur][field], sizeof(float) * g->pitch, src, w, w,
                                (size_t)g->ny * g->nz,
                                src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                g->stream));
  if (!src_on_device) PF_CUDA_TRY(cudaStreamSynchronize(g->stream));
  return PF_OK;
}

int pf_read_field(pf_grid_t g, int field, float* dst, int dst_on_device) {
  if (int rc = check_grid(g)) return rc;
  if (field < 0 || field >= g->nf) return invalid("field %d out of range", field);
  if (dst == nullptr) return invalid("dst is NULL");
  const size_t w = sizeof(float) * g->nx;
  PF_CUDA_TRY(cudaMemcpy2DAsync(dst, w, g->buf[g->cur][field], sizeof(float) * g->pitch, w,
                                (size_t)g->ny * g->nz,
                                dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                g->stream));
  if (!dst_on_device) return check_device_error(g);
  return PF_OK;
}

int pf_write_field_host_async(pf_grid_t g, int field, const float* src) {
  if (int rc = check_grid(g)) return rc;
  if (field < 0 || field >= g->nf) return invalid("field %d out of range", field);
  if (src == nullptr) return invalid("src is NULL");
  const size_t w = sizeof(float) * g->nx;
  PF_CUDA_TRY(cudaMemcpy2DAsync(g->buf[g->cur][field], sizeof(float) * g->pitch, src, w, w,
                                (size_t)g->ny * g->nz, cudaMemcpyHostToDevice, g->stream));
  return PF_OK;
}

int pf_read_field_host_async(pf_grid_t g, int field, float* dst) {
  if (int rc = check_grid(g)) return rc;
  if (field < 0 || field >= g->nf) return invalid("field %d out of range", field);
  if (dst == nullptr) return invalid("dst is NULL");
  const size_t w = sizeof(float) * g->nx;
  PF_CUDA_TRY(cudaMemcpy2DAsync(dst, w, g->buf[g->cur][field], sizeof(float) * g->pitch, w,
                                (size_t)g->ny * g->nz, cudaMemcpyDeviceToHost, g->stream));
  return PF_OK;
}

int pf_step(pf_grid_t g, int64_t n_steps) {
  NvtxRange nvtx_("pf_step");
  if (int rc = check_grid(g)) return rc;
  if (!g->model_set) {
    set_error("pf_step: no model set (call pf_set_model first)");
    return PF_ERR_STATE;
  }
  if (n_steps < 0) return invalid("n_steps must be >= 0");
  if (n_steps == 0) return PF_OK;
  if (g->dim == 2 && g->tile == kTileCluster2D) {
    // the whole run in one launch of the on-chip cluster kernel
    FieldPtrs in{};
    FieldOut out{};
    for (int f = 0; f < g->nf; ++f) {
      in.f[f] = g->buf[g->cur][f];
      out.f[f] = g->buf[1 - g->cur][f];
    }
    PF_CUDA_TRY(launch_fe2d_cluster(g->model, g->k, grid_geom(g), in, out, g->params, n_steps,
                                    g->stream));
    g->cur = 1 - g->cur;
    return PF_OK;
  }
  if (g->dim == 2 && g->tile == kTileBands2D) {
    // the whole run in one cooperative launch of the band kernel
    PF_CUDA_TRY(launch_fe2d_bands(g, g->cur, 1 - g->cur, n_steps, g->stream));
    g->cur = 1 - g->cur;
    return PF_OK;
  }
  if (count_launches(n_steps, g->k) >= kGraphMinLaunches) {
    // replay a recorded graph of the whole launch sequence (one host call)
    pf_grid_s::StepGraph* hit = nullptr;
    pf_grid_s::StepGraph* victim = &g->step_graphs[0];
    for (auto& sg : g->step_graphs) {
      if (sg.exec && sg.steps == n_steps && sg.tile == g->tile && sg.k == g->k &&
          sg.start == g->cur)
        hit = &sg;
      if (sg.used < victim->used) victim = &sg;
    }
    if (hit == nullptr) {
      if (victim->exec) cudaGraphExecDestroy(victim->exec);
      *victim = pf_grid_s::StepGraph();
      if (int rc = record_step_graph(g, n_steps, &victim->exec, &victim->flip)) return rc;
      victim->steps = n_steps;
      victim->tile = g->tile;
      victim->k = g->k;
      victim->start = g->cur;
      hit = victim;
    }
    hit->used = ++g->graph_clock;
    PF_CUDA_TRY(cudaGraphLaunch(hit->exec, g->stream));
    if (hit->flip) g->cur = 1 - g->cur;
    return PF_OK;
  }
  int64_t left = n_steps;
  while (left > 0) {
    int k = g->k;
    while (k > left) k >>= 1;  // k in {4, 2, 1}
    PF_CUDA_TRY(launch_step(g, g->tile, k, g->cur, 1 - g->cur, g->stream));
    g->cur = 1 - g->cur;
    left -= k;
  }
  return PF_OK;
}

int pf_reduce(pf_grid_t g, int what, int field, double* out) {
  NvtxRange nvtx_("pf_reduce");
  if (int rc = check_grid(g)) return rc;
  if (out == nullptr) return invalid("out is NULL");
  if (what != PF_REDUCE_MASS && what != PF_REDUCE_ENERGY) return invalid("unknown reduction %d", what);
  if (field < 0 || field >= g->nf) return invalid("field %d out of range", field);
  double c1 = 0, c2 = 0;
  if (what == PF_REDUCE_ENERGY) {
    if (!g->model_set ||
        (g->model != PF_MODEL_AC && g->model != PF_MODEL_CH && g->model != PF_MODEL_C)) {
      set_error("energy needs an Allen-Cahn, Cahn-Hilliard or Model C model");
      return PF_ERR_STATE;
    }
    c1 = g->coeffs[0];
    c2 = g->coeffs[1];
  }
  if (what == PF_REDUCE_ENERGY && g->model == PF_MODEL_C) {
    PF_CUDA_TRY(launch_reduce_energy_c(grid_geom(g), g->buf[g->cur][0], g->buf[g->cur][1],
                                       g->coeffs, g->h, g->red_partials,
                                       g->red_partials + kReduceBlocks, g->stream));
  } else {
    PF_CUDA_TRY(launch_reduce(what, grid_geom(g), g->buf[g->cur][field], c1, c2, g->h,
                              g->red_partials, g->red_partials + kReduceBlocks, g->stream));
  }
  PF_CUDA_TRY(cudaMemcpyAsync(g->red_host, g->red_partials + kReduceBlocks, sizeof(double),
                              cudaMemcpyDeviceToHost, g->stream));
  if (int rc = check_device_error(g)) return rc;
  *out = *g->red_host;
  if (!std::isfinite(*out)) {
    set_error("reduction is not finite (%g): the state has blown up", *out);
    return PF_ERR_NONFINITE;
  }
  return PF_OK;
}

int pf_set_stencil(pf_grid_t g, int stencil) {
  if (int rc = check_grid(g)) return rc;
  if (stencil != PF_STENCIL_STD && stencil != PF_STENCIL_ISO && stencil != PF_STENCIL_4TH &&
      stencil != PF_STENCIL_ISO27)
    return invalid("unknown stencil %d", stencil);
  if (stencil == PF_STENCIL_ISO27 && g->dim != 3)
    return invalid("the 27-point stencil is defined for 3D grids only");
  if (stencil == PF_STENCIL_4TH && g->dim != 2)
    return invalid("the fourth-order stencil is defined for 2D grids only");
  if (g->model_set && g->model == PF_MODEL_RD && stencil != PF_STENCIL_STD)
    return invalid("the N-species model runs with the 5-/7-point stencil");
  if (g->model_set && g->model != PF_MODEL_RD && stencil != g->stencil) {
    const double lim = stable_dt_limit(g->model, g->dim, g->h, g->coeffs, stencil);
    if (g->dt > lim) {
      set_error("dt = %g exceeds the forward-Euler stability limit %g with this stencil "
                "(set a smaller dt first)", g->dt, lim);
      return PF_ERR_UNSTABLE_DT;
    }
  }
  g->stencil = stencil;
  if (g->model_set && g->model != PF_MODEL_RD)
    g->params = make_params(g->model, g->coeffs, g->dt, g->h, stencil);
  g->req_tile = -1;
  g->req_k = 0;
  drop_graphs(g);
  return resolve_tuning(g);
}

int pf_set_tuning(pf_grid_t g, int tile_x, int tile_y, int k_steps) {
  if (int rc = check_grid(g)) return rc;
  if (g->model_set && g->model == PF_MODEL_RD) {  // one kernel: the tile request is not used
    if (k_steps < 0 || k_steps > 1)
      return invalid("the N-species model runs one step per launch (k_steps 0 or 1)");
    (void)tile_x;
    (void)tile_y;
    return resolve_tuning(g);
  }
  int tile = -1;
  if (tile_x == 0 && tile_y == 0) {
    tile = -1;
  } else if (g->dim == 2) {
    const int cs = fe2d_cluster_size();
    if (tile_x == g->nx && tile_y == PF_TILE_BANDS) {
      tile = kTileBands2D;  // the band kernel: one band of full rows per SM
      if (g->stencil != PF_ST_STD || (k_steps != 0 && k_steps != 1) ||
          !(g->model_set && fe2d_bands_supported(g->model, grid_geom(g))))
        return invalid("the band kernel (tile %d x PF_TILE_BANDS) needs an Allen-Cahn or "
                       "Cahn-Hilliard model, the standard stencil, k = 1, nx %% 4 == 0 with "
                       "64 <= nx <= 4096, and a band of the grid in each SM's shared memory",
                       tile_x);
    } else if (tile_y == PF_TILE_STRIPS) {
      tile = tile_x == 128 ? kTileStrips2D : tile_x == 64 ? kTileStrips2D + 1 : -1;
      const int kk = k_steps > 0 ? k_steps : 1;
      if (tile < 0 || !(g->model_set && fe2d_strips_supported(g->model, kk, g->stencil)))
        return invalid("the strip kernel (tile 128 or 64 x PF_TILE_STRIPS) needs a model set "
                       "and k = 1, 2 or 4 (Models A, Gray-Scott: the 5- or 9-point stencil) or "
                       "k = 1 or 2 (Models B, C: the 5-point stencil)");
    } else if (tile_x == g->nx && g->ny % cs == 0 && tile_y == g->ny / cs) {
      tile = kTileCluster2D;  // the on-chip cluster kernel: full rows, ny / CS rows per CTA
      const int kk = k_steps > 0 ? k_steps : 1;
      if (g->stencil != PF_ST_STD ||
          !(g->model_set && fe2d_cluster_supported(g->model, kk, grid_geom(g))))
        return invalid("the on-chip cluster kernel (tile %dx%d) needs a model set, the standard "
                       "stencil, nx %% 4 == 0 and the grid in %d CTAs' shared memory with "
                       "k %d", tile_x, tile_y, cs, kk);
    } else {
      tile = tile2d_id(tile_x, tile_y);
    }
    if (tile < 0) return invalid("unsupported 2D tile %dx%d", tile_x, tile_y);
  } else {
    tile = tile3d_id(tile_x, tile_y);
    if (tile < 0) return invalid("unsupported 3D tile %dx%d", tile_x, tile_y);
  }
  if (k_steps < 0) return invalid("k_steps must be >= 0");
  if (g->dim == 3 && k_steps > 2) return invalid("3D grids support k = 1 and 2");
  if (g->dim == 3 && k_steps == 2 && tile != kTileBox3D) {
    int tx = tile_x, ty = tile_y;
    if (tile < 0) return invalid("k = 2 in 3D needs an explicit tile (nx x 8, nx = 128 or 256)");
    if (!(g->model_set && fe3d_tb2_supported(g->model, tx, ty, grid_geom(g))))
      return invalid("3D k = 2 needs an AC/GS model, tile nx x 8 with nx = 128 or 256, ny %% 8 == 0");
  }
  const bool strip_tile = g->dim == 2 && tile >= kTileStrips2D && tile < kTileStrips2D + kNumStrips2D;
  if (k_steps > 0 && g->dim == 2 && tile != kTileCluster2D && tile != kTileBands2D && !strip_tile) {
    const int model = g->model_set ? g->model : PF_MODEL_AC;
    if (!fe2d_supported(model, k_steps))
      return invalid("temporal blocking depth %d unsupported for this model", k_steps);
  }
  if (g->stencil != PF_ST_STD && tile != kTileCluster2D && tile != kTileBands2D && !strip_tile) {
    const int t = tile >= 0 ? tile : 0;
    const int kk = k_steps > 0 ? k_steps : 1;
    const bool ok = g->dim == 2 ? fe2d_stencil_supported(g->stencil, t, kk)
                                : ((t == 0 || t == 1) && kk == 1);
    if (!ok)
      return invalid("this stencil runs with 2D tiles 64x16 or 128x32 and k <= 2 (the 9-point "
                     "one also on the strip kernel), or 3D tiles 32x16 or 64x8 and k = 1");
  }
  if (g->dim == 3 && tile == kTileBox3D) {
    if (!(g->model_set && fe3d_box_supported(g->model, k_steps > 0 ? k_steps : 1, grid_geom(g))))
      return invalid("3D tile 32x8 (the box kernel) needs Model B or C, k = 1 or 2 and "
                     "nx %% 4 == 0");
  } else if (g->dim == 3 && k_steps != 2 && tile >= kFirstTmaTile3D &&
             !(g->model_set && fe3d_tma_supported(g->model, tile - kFirstTmaTile3D, grid_geom(g)))) {
    return invalid("3D tile %dx%d needs nx %% %d == 0 and ny %% %d == 0", tile_x, tile_y,
                   tile_x, tile_y);
  }
  g->req_tile = tile;
  g->req_k = k_steps;
  drop_graphs(g);
  return resolve_tuning(g);
}

int pf_get_tuning(pf_grid_t g, int* tile_x, int* tile_y, int* k_steps) {
  if (int rc = check_grid(g)) return rc;
  int tx, ty;
  if (g->dim == 2 && g->tile == kTileCluster2D) {
    tx = g->nx;
    ty = g->ny / fe2d_cluster_size();
  } else if (g->dim == 2 && g->tile == kTileBands2D) {
    tx = g->nx;
    ty = PF_TILE_BANDS;
  } else if (g->dim == 2 && g->tile >= kTileStrips2D && g->tile < kTileStrips2D + kNumStrips2D) {
    tx = g->tile == kTileStrips2D ? 128 : 64;
    ty = PF_TILE_STRIPS;
  } else if (g->dim == 2) {
    tile2d_shape(g->tile, &tx, &ty);
  } else {
    tile3d_shape(g->tile, &tx, &ty);
  }
  if (tile_x) *tile_x = tx;
  if (tile_y) *tile_y = ty;
  if (k_steps) *k_steps = g->k;
  return PF_OK;
}

int pf_autotune(pf_grid_t g, int probe_launches, int* tile_x, int* tile_y, int* k_steps) {
  NvtxRange nvtx_("pf_autotune");
  if (int rc = check_grid(g)) return rc;
  if (!g->model_set) {
    set_error("pf_autotune: no model set");
    return PF_ERR_STATE;
  }
  if (probe_launches < 1) probe_launches = 3;
  cudaEvent_t e0, e1;
  PF_CUDA_TRY(cudaEventCreate(&e0));
  PF_CUDA_TRY(cudaEventCreate(&e1));
  float best = INFINITY;
  int best_tile = g->tile, best_k = g->k;
  // 2D: + the cluster kernel, the band kernel and the two strip widths
  const int ntiles = g->dim == 2 ? kTileStrips2D + kNumStrips2D : kNumTiles3D;
  static const int ks[4] = {1, 2, 4, 8};  // 8: the cluster kernel only
  int rc = PF_OK;
  for (int t = 0; t < ntiles && rc == PF_OK; ++t) {
    for (int ki = 0; ki < 4 && rc == PF_OK; ++ki) {
      const int k = ks[ki];
      if (!tile_supported(g, t, k)) continue;
      // the cluster and band kernels run a whole pf_step in one launch: probe them that way
      const bool cluster = g->dim == 2 && (t == kTileCluster2D || t == kTileBands2D);
      const int64_t probe_steps = cluster ? (int64_t)probe_launches * k * 16 : 0;
      // Every probe reads buffer cur and writes 1 - cur, so the state is left as it was.
      // Tiled candidates run as a replayed graph of n_l launches, as pf_step runs them.
      const int n_l = probe_launches > 8 ? probe_launches : 8;
      cudaGraphExec_t probe = nullptr;
      cudaError_t e = launch_step(g, t, k, g->cur, 1 - g->cur, g->stream);  // warm-up
      if (cluster && (e == cudaErrorCooperativeLaunchTooLarge || e == cudaErrorLaunchOutOfResources)) {
        // the on-chip kernels need all their CTAs resident at once; where the device cannot
        // host them now (other work, a restricted context), they are not candidates
        cudaGetLastError();
        continue;
      }
      if (!cluster && e == cudaSuccess) {
        if (g->capture == nullptr)
          e = cudaStreamCreateWithFlags(&g->capture, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(g->capture, cudaStreamCaptureModeRelaxed);
        if (e == cudaSuccess) {
          cudaError_t el = cudaSuccess;
          for (int i = 0; i < n_l && el == cudaSuccess; ++i)
            el = launch_step(g, t, k, g->cur, 1 - g->cur, g->capture);
          cudaGraph_t graph = nullptr;
          e = cudaStreamEndCapture(g->capture, &graph);
          if (e == cudaSuccess) e = el;
          if (e == cudaSuccess) e = cudaGraphInstantiate(&probe, graph, 0);
          if (graph) cudaGraphDestroy(graph);
        }
        if (e == cudaSuccess) e = cudaGraphLaunch(probe, g->stream);  // warm-up replay
      }
      if (e == cudaSuccess) e = cudaEventRecord(e0, g->stream);
      if (cluster && t == kTileBands2D && e == cudaSuccess) {
        e = launch_fe2d_bands(g, g->cur, 1 - g->cur, probe_steps, g->stream);
      } else if (cluster && e == cudaSuccess) {
        FieldPtrs in{};
        FieldOut out{};
        for (int f = 0; f < g->nf; ++f) {
          in.f[f] = g->buf[g->cur][f];
          out.f[f] = g->buf[1 - g->cur][f];
        }
        e = launch_fe2d_cluster(g->model, k, grid_geom(g), in, out, g->params, probe_steps,
                                g->stream);
      }
      if (!cluster && e == cudaSuccess) e = cudaGraphLaunch(probe, g->stream);
      if (e == cudaSuccess) e = cudaEventRecord(e1, g->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (probe) cudaGraphExecDestroy(probe);
      float ms = 0;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) {
        rc = cuda_fail(e, "pf_autotune probe");
        break;
      }
      const float per_step = cluster ? ms / probe_steps : ms / ((float)n_l * k);
      if (per_step < best) {
        best = per_step;
        best_tile = t;
        best_k = k;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != PF_OK) return rc;
  g->req_tile = best_tile;
  g->req_k = best_k;
  drop_graphs(g);
  resolve_tuning(g);
  return pf_get_tuning(g, tile_x, tile_y, k_steps);
}

int pf_synchronize(pf_grid_t g) {
  if (int rc = check_grid(g)) return rc;
  return check_device_error(g);
}

int pf_copy_planes(pf_grid_t g, int field, int64_t first, int64_t count, float* buf,
                   int to_buf, int buf_on_device) {
  if (int rc = check_grid(g)) return rc;
  if (field < 0 || field >= g->nf) return invalid("field %d out of range", field);
  const int64_t nslow = g->dim == 3 ? g->nz : g->ny;  // planes (3D) or rows (2D)
  if (first < 0 || count < 0 || first > nslow || count > nslow - first)
    return invalid("planes [%lld, %lld) outside [0, %lld)", (long long)first,
                   (long long)(first + count), (long long)nslow);
  if (count > 0 && buf == nullptr) return invalid("buf is NULL");
  if (count == 0) return PF_OK;
  // a plane (3D) is ny rows of nx floats; a 2D "plane" is one row
  const int64_t rows_per = g->dim == 3 ? g->ny : 1;
  const size_t w = sizeof(float) * g->nx;
  float* dev = g->buf[g->cur][field] + first * (g->dim == 3 ? g->plane : g->pitch);
  const cudaMemcpyKind kind = buf_on_device ? cudaMemcpyDeviceToDevice
                              : to_buf      ? cudaMemcpyDeviceToHost
                                            : cudaMemcpyHostToDevice;
  if (to_buf)
    PF_CUDA_TRY(cudaMemcpy2DAsync(buf, w, dev, sizeof(float) * g->pitch, w,
                                  (size_t)(count * rows_per), kind, g->stream));
  else
    PF_CUDA_TRY(cudaMemcpy2DAsync(dev, sizeof(float) * g->pitch, buf, w, w,
                                  (size_t)(count * rows_per), kind, g->stream));
  if (!buf_on_device) return check_device_error(g);  // synchronizes the stream
  return PF_OK;
}

int pf_field_view(pf_grid_t g, int field, float** dev_ptr, int64_t* pitch, int64_t* plane) {
  if (int rc = check_grid(g)) return rc;
  if (field < 0 || field >= g->nf) return invalid("field %d out of range", field);
  if (dev_ptr) *dev_ptr = g->buf[g->cur][field];
  if (pitch) *pitch = g->pitch;
  if (plane) *plane = g->plane;
  return PF_OK;
}

}  // extern "C"
