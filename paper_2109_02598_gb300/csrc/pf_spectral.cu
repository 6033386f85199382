// Semi-implicit Fourier spectral solver (Sec. 2.4.2) for Models A, B and C (Sec. 3).
//
// Buffers (nk modes and nsite sites per field; cs = nk rounded up to 32 and rs = nsite
// rounded up to 64, so that every slice starts on 256 bytes):
//   spec  float2 [2 nf][cs]: the state psi_hat (slices 0..nf-1) and f_hat (nf..2nf-1);
//   work  float2 [nf][cs]:   psi_hat / N, the input of the next inverse transform;
//   real  float  [nf][rs]:   the fields in real space, then their nonlinear terms.
// One step:
//   1. inverse transform work -> real (cuFFT's complex-to-real transform overwrites work);
//   2. nonlinear terms f(psi) in place on real (all fields of a site at once);
//   3. forward transform real -> spec[nf..2nf) = f_hat;
//   4. psi_hat <- A psi_hat + (B N) f_hat and work <- psi_hat / N.
// The state stays in Fourier space: two transforms per field and step, and no round-trip
// rounding on it. The spectrum of a real field is Hermitian, psi_hat(-k) = conj psi_hat(k);
// on the planes kx = 0 and kx = nx/2 (even nx) the half spectrum holds both k and -k, and
// the forward transform meets this only to rounding. Step 4 therefore uses, on those
// planes, the Hermitian part (f_hat(k) + conj f_hat(-k)) / 2. With A and B N even in k and
// the products rounded symmetrically, the state then stays exactly Hermitian; the
// rounding-level remainder would otherwise build up unseen (the inverse transform ignores
// it) and grow wherever A > 1, e.g. |k|^2 < c1 in Model A. A and B N are computed once,
// in float64, and stored as float2 per mode. Padding is zero and stays zero: the
// transforms neither read nor write it and the kernels map zero to zero.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>

#include "pf_cufft.h"
#include "pf_internal.h"
#include "pf_spectral.h"

namespace pf {
int invalid(const char* fmt, ...);
}

namespace pf {
namespace {

constexpr uint32_t kSpectralMagic = 0x53504543u;
constexpr int kChunkSteps = 32;
constexpr int kThreads = 256;
constexpr int kMaxBlocks = 152 * 8;

struct SpecGeom {
  int rank;
  int64_t d[3];
  int64_t nxh;  // d[rank-1] / 2 + 1
  int64_t nk, cs;
};

// np.fft.fftfreq numerator of index i on an axis of n points: i, or i - n past the middle.
__device__ __forceinline__ double fft_index(int64_t i, int64_t n) {
  return (double)(i <= (n - 1) / 2 ? i : i - n);
}

// 2 pi f / (n h), as 2 pi * (f * (1 / (n h))).
__device__ __forceinline__ double wavenumber(double f, int64_t n, double h) {
  const double val = __ddiv_rn(1.0, __dmul_rn((double)n, h));
  return __dmul_rn(2.0 * 3.141592653589793, __dmul_rn(f, val));
}

// |k|^2 of half-spectrum mode i (x the halved, fastest axis).
__device__ double mode_k2(const SpecGeom& g, int64_t i, double h) {
  const int64_t ix = i % g.nxh;
  const int64_t rest = i / g.nxh;
  const double kx = wavenumber((double)ix, g.d[g.rank - 1], h);
  const int64_t ny = g.d[g.rank - 2];
  const double ky = wavenumber(fft_index(rest % ny, ny), ny, h);
  double s = __dmul_rn(ky, ky);
  if (g.rank == 3) {
    const double kz = wavenumber(fft_index(rest / ny, g.d[0]), g.d[0], h);
    s = __dadd_rn(__dmul_rn(kz, kz), s);
  }
  return __dadd_rn(s, __dmul_rn(kx, kx));
}

// (A, B N) per mode and field, in float64, rounded to float32 (Sec. 2.4.2).
__global__ void spectral_table_kernel(int model, SpecGeom g, double h, double dt, double c1,
                                      double c3, double M, int nf, float2* __restrict__ table) {
  const int64_t total = g.nk * nf;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int f = (int)(t / g.nk);
    const int64_t i = t % g.nk;
    const double k2 = mode_k2(g, i, h);
    double L, N;
    if (model == PF_MODEL_AC || (model == PF_MODEL_C && f == 0)) {
      L = c1 - k2;
      N = 1.0;
    } else if (model == PF_MODEL_CH) {
      L = M * (c1 * k2 - k2 * k2);
      N = -M * k2;
    } else {  // Model C, m
      L = c3 * k2 - k2 * k2;
      N = -k2;
    }
    const double Ldt = L * dt;
    const double A = exp(Ldt);
    const double B = fabs(Ldt) < 1e-12 ? dt * (1.0 + 0.5 * Ldt) : expm1(Ldt) / (Ldt / dt);
    table[f * g.cs + i] = make_float2((float)A, (float)(B * N));
  }
}


// In place over rs / 4 float4 groups of every field (padding included: zero in, zero out).
template <int MODEL>
__global__ void spectral_nonlinear_kernel(float* __restrict__ real, int64_t rs, NlCoeffs k) {
  float4* p4 = reinterpret_cast<float4*>(real);
  float4* m4 = reinterpret_cast<float4*>(real + rs);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rs / 4;
       i += (int64_t)gridDim.x * blockDim.x) {
    float4 p = p4[i];
    float4 m = make_float4(0.f, 0.f, 0.f, 0.f);
    if (MODEL == PF_MODEL_C) m = m4[i];
    nonlinear_site<MODEL>(p.x, m.x, k.c);
    nonlinear_site<MODEL>(p.y, m.y, k.c);
    nonlinear_site<MODEL>(p.z, m.z, k.c);
    nonlinear_site<MODEL>(p.w, m.w, k.c);
    p4[i] = p;
    if (MODEL == PF_MODEL_C) m4[i] = m;
  }
}

// Half-spectrum index of -k for mode i on a self-conjugate plane (same kx).
__device__ __forceinline__ int64_t mirror_mode(const SpecGeom& g, int64_t i) {
  const int64_t ix = i % g.nxh, rest = i / g.nxh;
  const int64_t ny = g.d[g.rank - 2];
  const int64_t iy = rest % ny, iz = rest / ny;
  const int64_t nz = g.rank == 3 ? g.d[0] : 1;
  const int64_t my = iy == 0 ? 0 : ny - iy, mz = iz == 0 ? 0 : nz - iz;
  return (mz * ny + my) * g.nxh + ix;
}

__device__ __forceinline__ bool self_conjugate_plane(const SpecGeom& g, int64_t i) {
  const int64_t ix = i % g.nxh;
  return ix == 0 || 2 * ix == g.d[g.rank - 1];
}

// The Hermitian part of v on the self-conjugate planes: (v(k) + conj v(-k)) / 2, with the
// sums taken in an order that gives exactly conjugate values at k and -k.
__device__ __forceinline__ float2 hermitian_part(const SpecGeom& g, const float2* v, int64_t i,
                                                 float2 vi) {
  if (i >= g.nk || !self_conjugate_plane(g, i)) return vi;
  const float2 vm = v[mirror_mode(g, i)];
  return make_float2(__fmul_rn(0.5f, __fadd_rn(vi.x, vm.x)), __fmul_rn(0.5f, __fsub_rn(vi.y, vm.y)));
}

__device__ __forceinline__ float2 update_mode(float2 s, float2 f, float A, float BN) {
  return make_float2(__fmaf_rn(A, s.x, __fmul_rn(BN, f.x)), __fmaf_rn(A, s.y, __fmul_rn(BN, f.y)));
}

// psi_hat <- A psi_hat + (B N) f_hat and work <- psi_hat / N, over modes t < total = nf cs
// (field t / cs, mode t % cs); psi_hat at spec[t], f_hat at spec[total + t]. Modes are taken
// two at a time (16-byte accesses); total and cs are even, so a pair never spans two fields.
__global__ void spectral_update_kernel(float2* __restrict__ spec, float2* __restrict__ work,
                                       const float2* __restrict__ table, SpecGeom g,
                                       int64_t total, float inv_n) {
  float4* s4 = reinterpret_cast<float4*>(spec);
  const float4* f4 = reinterpret_cast<const float4*>(spec + total);
  const float4* t4 = reinterpret_cast<const float4*>(table);
  float4* w4 = reinterpret_cast<float4*>(work);
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < total / 2;
       j += (int64_t)gridDim.x * blockDim.x) {
    const float4 tb = t4[j];
    const float4 sv = s4[j];
    const float4 fv = f4[j];
    const int64_t f = (2 * j) / g.cs, i = (2 * j) % g.cs;
    const float2* fh = reinterpret_cast<const float2*>(f4) + f * g.cs;
    const float2 fa = hermitian_part(g, fh, i, make_float2(fv.x, fv.y));
    const float2 fb = hermitian_part(g, fh, i + 1, make_float2(fv.z, fv.w));
    const float2 a = update_mode(make_float2(sv.x, sv.y), fa, tb.x, tb.y);
    const float2 b = update_mode(make_float2(sv.z, sv.w), fb, tb.z, tb.w);
    s4[j] = make_float4(a.x, a.y, b.x, b.y);
    w4[j] = make_float4(__fmul_rn(a.x, inv_n), __fmul_rn(a.y, inv_n), __fmul_rn(b.x, inv_n),
                        __fmul_rn(b.y, inv_n));
  }
}

// A freshly transformed field: state <- the Hermitian part of raw, work <- state / N.
__global__ void spectral_load_kernel(const float2* __restrict__ raw, float2* __restrict__ state,
                                     float2* __restrict__ work, SpecGeom g, float inv_n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.nk;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = hermitian_part(g, raw, i, raw[i]);
    state[i] = v;
    work[i] = make_float2(__fmul_rn(v.x, inv_n), __fmul_rn(v.y, inv_n));
  }
}

int blocks_for(int64_t work_items) {
  int64_t b = (work_items + kThreads - 1) / kThreads;
  if (b < 1) b = 1;
  return (int)(b < kMaxBlocks ? b : kMaxBlocks);
}

float inv_sites(const pf_spectral_s* s) { return (float)(1.0 / (double)s->nsite); }

SpecGeom spec_geom(const pf_spectral_s* s) {
  SpecGeom g{};
  g.rank = s->dim;
  for (int i = 0; i < s->dim; ++i) g.d[i] = s->d[i];
  g.nxh = s->d[s->dim - 1] / 2 + 1;
  g.nk = s->nk;
  g.cs = s->cs;
  return g;
}

cudaError_t launch_nonlinear(const pf_spectral_s* s, cudaStream_t st) {
  const NlCoeffs k = nl_coeffs(s);
  const int blocks = blocks_for(s->rs / 4);
  if (s->model == PF_MODEL_AC)
    spectral_nonlinear_kernel<PF_MODEL_AC><<<blocks, kThreads, 0, st>>>(s->real, s->rs, k);
  else if (s->model == PF_MODEL_CH)
    spectral_nonlinear_kernel<PF_MODEL_CH><<<blocks, kThreads, 0, st>>>(s->real, s->rs, k);
  else
    spectral_nonlinear_kernel<PF_MODEL_C><<<blocks, kThreads, 0, st>>>(s->real, s->rs, k);
  return cudaGetLastError();
}

// AUTO takes the fused engine where it was measured faster than cuFFT on GB300: every grid
// it takes except two-field (Model C) 2D grids with a 1024 side (per step, fused vs cuFFT:
// 64^2 Model A 9.2 vs 10.1 us, 128^2 A 10.9 vs 13.3 and C 11.1 vs 13.7, 256^2 A 12.8 vs 13.2,
// 512^2 A 13.5 vs 16.3 and C 17.3 vs 18.4, 1024^2 A 28.2 vs 32.4 but C 67.7 vs 37.9, 64^3 A
// 17.4 vs 18.2 and C 18.3 vs 21.7).
bool auto_prefers_fused(const pf_spectral_s* s) {
  if (!s->fused_ok) return false;
  if (s->dim == 3) return true;
  const int64_t nmax = s->d[0] > s->d[1] ? s->d[0] : s->d[1];
  return s->nf == 1 || nmax < 1024;
}

bool use_fused(const pf_spectral_s* s) {
  if (s->engine == PF_SPECTRAL_ENGINE_FUSED) return true;
  return s->engine == PF_SPECTRAL_ENGINE_AUTO && auto_prefers_fused(s);
}

// Enqueue one step on stream st.
int enqueue_step(pf_spectral_s* s, cudaStream_t st) {
  const CufftApi* api = s->api;
  cufftResult r = api->set_stream(s->c2r_all, st);
  if (r == CUFFT_SUCCESS)
    r = api->exec_c2r(s->c2r_all, reinterpret_cast<cufftComplex*>(s->work), s->real);
  if (r != CUFFT_SUCCESS) return cufft_fail(r, "pf_spectral_step inverse transform");
  PF_CUDA_TRY(launch_nonlinear(s, st));
  const int64_t total = s->cs * s->nf;
  r = api->set_stream(s->r2c_all, st);
  if (r == CUFFT_SUCCESS)
    r = api->exec_r2c(s->r2c_all, s->real, reinterpret_cast<cufftComplex*>(s->spec + total));
  if (r != CUFFT_SUCCESS) return cufft_fail(r, "pf_spectral_step forward transform");
  spectral_update_kernel<<<blocks_for(total / 2), kThreads, 0, st>>>(
      s->spec, s->work, s->table, spec_geom(s), total, inv_sites(s));
  PF_CUDA_TRY(cudaGetLastError());
  return PF_OK;
}

// Record kChunkSteps steps into a graph (once). A capture that fails leaves the solver on
// direct launches (same kernels, same results).
void ensure_chunk_graph(pf_spectral_s* s) {
  if (s->chunk != nullptr || s->graph_failed) return;
  if (s->capture == nullptr &&
      cudaStreamCreateWithFlags(&s->capture, cudaStreamNonBlocking) != cudaSuccess) {
    s->graph_failed = true;
    cudaGetLastError();
    return;
  }
  if (cudaStreamBeginCapture(s->capture, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    s->graph_failed = true;
    cudaGetLastError();
    return;
  }
  int rc = PF_OK;
  for (int i = 0; i < kChunkSteps && rc == PF_OK; ++i) rc = enqueue_step(s, s->capture);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(s->capture, &graph);
  if (rc == PF_OK && e == cudaSuccess) e = cudaGraphInstantiate(&s->chunk, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (rc != PF_OK || e != cudaSuccess) {
    s->chunk = nullptr;
    s->graph_failed = true;
    cudaGetLastError();
  }
}

int check_spectral(pf_spectral_s* s) {
  if (s == nullptr || s->magic != kSpectralMagic) return invalid("invalid spectral handle");
  return PF_OK;
}

void release(pf_spectral_s* s) {
  spectral_fused_release(s);
  if (s->chunk) cudaGraphExecDestroy(s->chunk);
  if (s->api) {
    for (cufftHandle p : {s->c2r_all, s->r2c_all, s->r2c_one, s->c2r_one})
      if (p != -1) s->api->destroy(p);
  }
  cudaFree(s->spec);
  cudaFree(s->work);
  cudaFree(s->table);
  cudaFree(s->real);
  cudaFree(s->fft_work);
  if (s->capture) cudaStreamDestroy(s->capture);
  s->magic = 0;
  delete s;
}

}  // namespace
}  // namespace pf

using namespace pf;

extern "C" {

int pf_spectral_create(int dim, const int64_t* n, double h, int model, const double* coeffs,
                       int n_coeffs, double dt, void* stream, pf_spectral_t* out) {
  if (out == nullptr || n == nullptr) return invalid("pf_spectral_create: NULL argument");
  *out = nullptr;
  if (dim != 2 && dim != 3) return invalid("dim must be 2 or 3 (got %d)", dim);
  const int64_t nx = n[0], ny = n[1], nz = dim == 3 ? n[2] : 1;
  const int64_t lim = (int64_t)1 << 30;
  if (nx < 2 || ny < 1 || nz < 1 || nx > lim || ny > lim || nz > lim || nx * ny > lim ||
      nx * ny * nz > lim)
    return invalid("sizes must be nx >= 2, ny, nz >= 1, with at most 2^30 sites (got %lld x "
                   "%lld x %lld)", (long long)nx, (long long)ny, (long long)nz);
  if (!(h > 0.0) || !std::isfinite(h)) return invalid("h must be finite and > 0");
  if (!(dt > 0.0) || !std::isfinite(dt)) return invalid("dt must be finite and > 0");
  int want = 0, nf = 1;
  if (model == PF_MODEL_AC) want = 2;
  else if (model == PF_MODEL_CH) want = 3;
  else if (model == PF_MODEL_C) want = 5, nf = 2;
  else return invalid("the spectral solver takes Models A, B and C (got model %d)", model);
  if (coeffs == nullptr || n_coeffs != want)
    return invalid("model %d takes %d coefficients (got %d)", model, want, n_coeffs);
  for (int i = 0; i < want; ++i)
    if (!std::isfinite(coeffs[i])) return invalid("coefficient %d is not finite", i);
  if (model == PF_MODEL_CH && !(coeffs[2] > 0.0)) return invalid("mobility M must be > 0");

  const CufftApi* api = cufft_api();
  if (api == nullptr) return PF_ERR_CUDA;

  pf_spectral_s* s = new (std::nothrow) pf_spectral_s();
  if (s == nullptr) return invalid("host allocation failed");
  s->magic = kSpectralMagic;
  s->dim = dim;
  s->model = model;
  s->nf = nf;
  if (dim == 2) {
    s->d[0] = ny;
    s->d[1] = nx;
  } else {
    s->d[0] = nz;
    s->d[1] = ny;
    s->d[2] = nx;
  }
  s->nsite = nx * ny * nz;
  s->nk = (nx / 2 + 1) * ny * nz;
  s->rs = (s->nsite + 63) / 64 * 64;
  s->cs = (s->nk + 31) / 32 * 32;
  s->h = h;
  s->dt = dt;
  for (int i = 0; i < 5; ++i) s->coeffs[i] = i < want ? coeffs[i] : 0.0;
  for (int i = 0; i < 5; ++i) s->cf[i] = (float)s->coeffs[i];
  s->stream = (cudaStream_t)stream;
  s->api = api;

  const size_t tbytes = sizeof(float2) * (size_t)(s->cs * nf);
  const size_t cbytes = 2 * tbytes;
  const size_t rbytes = sizeof(float) * (size_t)(s->rs * nf);
  cudaError_t e = cudaMalloc(&s->spec, cbytes);
  if (e == cudaSuccess) e = cudaMalloc(&s->work, tbytes);
  if (e == cudaSuccess) e = cudaMalloc(&s->table, tbytes);
  if (e == cudaSuccess) e = cudaMalloc(&s->real, rbytes);
  if (e != cudaSuccess) {
    int rc = e == cudaErrorMemoryAllocation ? (set_error("pf_spectral_create: out of device memory"), PF_ERR_OOM)
                                            : cuda_fail(e, "pf_spectral_create allocation");
    cudaGetLastError();
    release(s);
    return rc;
  }
  // Plans: all fields at once for the steps, one field for reads and writes; one shared
  // work area (every transform runs on the solver's stream, one after another).
  size_t w[4] = {0, 0, 0, 0};
  int rc = cufft_plan(api, &s->c2r_all, dim, s->d, CUFFT_C2R, nf, s->rs, s->cs, 0, &w[0]);
  if (rc == PF_OK)
    rc = cufft_plan(api, &s->r2c_all, dim, s->d, CUFFT_R2C, nf, s->rs, s->cs, 0, &w[1]);
  if (rc == PF_OK && nf > 1)
    rc = cufft_plan(api, &s->r2c_one, dim, s->d, CUFFT_R2C, 1, s->rs, s->cs, 0, &w[2]);
  if (rc == PF_OK && nf > 1)
    rc = cufft_plan(api, &s->c2r_one, dim, s->d, CUFFT_C2R, 1, s->rs, s->cs, 0, &w[3]);
  if (rc != PF_OK) {
    release(s);
    return rc;
  }
  size_t wmax = 0;
  for (size_t x : w) wmax = x > wmax ? x : wmax;
  if (wmax > 0) {
    e = cudaMalloc(&s->fft_work, wmax);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("pf_spectral_create: out of device memory (transform work area)");
      release(s);
      return PF_ERR_OOM;
    }
  }
  for (cufftHandle p : {s->c2r_all, s->r2c_all, s->r2c_one, s->c2r_one}) {
    if (p == -1) continue;
    cufftResult r = api->set_work_area(p, s->fft_work);
    if (r != CUFFT_SUCCESS) {
      rc = cufft_fail(r, "cufftSetWorkArea");
      release(s);
      return rc;
    }
  }
  // Tables, zero state.
  const SpecGeom g = spec_geom(s);
  const double M = model == PF_MODEL_CH ? s->coeffs[2] : 1.0;
  e = cudaMemsetAsync(s->table, 0, tbytes, s->stream);
  if (e != cudaSuccess) {
    rc = cuda_fail(e, "pf_spectral_create tables");
    release(s);
    return rc;
  }
  spectral_table_kernel<<<blocks_for(s->nk * nf), kThreads, 0, s->stream>>>(
      model, g, h, dt, s->coeffs[0], model == PF_MODEL_C ? s->coeffs[2] : 0.0, M, nf, s->table);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemsetAsync(s->spec, 0, cbytes, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->work, 0, tbytes, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->real, 0, rbytes, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) {
    rc = cuda_fail(e, "pf_spectral_create tables");
    release(s);
    return rc;
  }
  s->fused_ok = spectral_fused_supported(s);
  *out = s;
  return PF_OK;
}

void pf_spectral_destroy(pf_spectral_t s) {
  if (s == nullptr || s->magic != kSpectralMagic) return;
  cudaStreamSynchronize(s->stream);
  release(s);
}

int pf_spectral_write_field(pf_spectral_t s, int field, const float* src, int src_on_device) {
  if (int rc = check_spectral(s)) return rc;
  if (field < 0 || field >= s->nf) return invalid("field %d out of range [0, %d)", field, s->nf);
  if (src == nullptr) return invalid("src is NULL");
  float* real = s->real + field * s->rs;
  float2* raw = s->spec + (s->nf + field) * s->cs;  // the f_hat slice, free between steps
  PF_CUDA_TRY(cudaMemcpyAsync(real, src, sizeof(float) * (size_t)s->nsite,
                              src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                              s->stream));
  const cufftHandle plan = s->nf > 1 ? s->r2c_one : s->r2c_all;
  cufftResult r = s->api->set_stream(plan, s->stream);
  if (r == CUFFT_SUCCESS) r = s->api->exec_r2c(plan, real, reinterpret_cast<cufftComplex*>(raw));
  if (r != CUFFT_SUCCESS) return cufft_fail(r, "pf_spectral_write_field transform");
  spectral_load_kernel<<<blocks_for(s->nk), kThreads, 0, s->stream>>>(
      raw, s->spec + field * s->cs, s->work + field * s->cs, spec_geom(s), inv_sites(s));
  PF_CUDA_TRY(cudaGetLastError());
  if (!src_on_device) PF_CUDA_TRY(cudaStreamSynchronize(s->stream));
  return PF_OK;
}

int pf_spectral_read_field(pf_spectral_t s, int field, float* dst, int dst_on_device) {
  if (int rc = check_spectral(s)) return rc;
  if (field < 0 || field >= s->nf) return invalid("field %d out of range [0, %d)", field, s->nf);
  if (dst == nullptr) return invalid("dst is NULL");
  // the inverse transform overwrites its input: transform a copy of psi_hat / N, made in
  // the field's f_hat slice (free between steps)
  float2* copy = s->spec + (s->nf + field) * s->cs;
  float* real = s->real + field * s->rs;
  PF_CUDA_TRY(cudaMemcpyAsync(copy, s->work + field * s->cs, sizeof(float2) * (size_t)s->nk,
                              cudaMemcpyDeviceToDevice, s->stream));
  const cufftHandle plan = s->nf > 1 ? s->c2r_one : s->c2r_all;
  cufftResult r = s->api->set_stream(plan, s->stream);
  if (r == CUFFT_SUCCESS) r = s->api->exec_c2r(plan, reinterpret_cast<cufftComplex*>(copy), real);
  if (r != CUFFT_SUCCESS) return cufft_fail(r, "pf_spectral_read_field transform");
  PF_CUDA_TRY(cudaMemcpyAsync(dst, real, sizeof(float) * (size_t)s->nsite,
                              dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                              s->stream));
  if (!dst_on_device) {
    PF_CUDA_TRY(cudaStreamSynchronize(s->stream));
    if (int rc = spectral_fused_check(s)) return rc;
  }
  return PF_OK;
}

int pf_spectral_step(pf_spectral_t s, int64_t n_steps) {
  NvtxRange nvtx_("pf_spectral_step");
  if (int rc = check_spectral(s)) return rc;
  if (n_steps < 0) return invalid("n_steps must be >= 0");
  if (use_fused(s)) return spectral_fused_run(s, n_steps);
  int64_t left = n_steps;
  if (left >= kChunkSteps) ensure_chunk_graph(s);
  if (s->chunk != nullptr) {
    for (; left >= kChunkSteps; left -= kChunkSteps)
      PF_CUDA_TRY(cudaGraphLaunch(s->chunk, s->stream));
  }
  for (; left > 0; --left)
    if (int rc = enqueue_step(s, s->stream)) return rc;
  return PF_OK;
}

int pf_spectral_synchronize(pf_spectral_t s) {
  if (int rc = check_spectral(s)) return rc;
  PF_CUDA_TRY(cudaStreamSynchronize(s->stream));
  return spectral_fused_check(s);
}

int pf_spectral_set_engine(pf_spectral_t s, int engine) {
  if (int rc = check_spectral(s)) return rc;
  if (engine != PF_SPECTRAL_ENGINE_AUTO && engine != PF_SPECTRAL_ENGINE_CUFFT &&
      engine != PF_SPECTRAL_ENGINE_FUSED)
    return invalid("unknown spectral engine %d", engine);
  if (engine == PF_SPECTRAL_ENGINE_FUSED && !s->fused_ok)
    return invalid("the fused engine takes power-of-two sides (nx in [4, 1024]) whose (y, z) "
                   "slab fits in a CTA's shared memory");
  s->engine = engine;
  return PF_OK;
}

int pf_spectral_get_engine(pf_spectral_t s, int* engine) {
  if (int rc = check_spectral(s)) return rc;
  if (engine == nullptr) return invalid("engine is NULL");
  *engine = use_fused(s) ? PF_SPECTRAL_ENGINE_FUSED : PF_SPECTRAL_ENGINE_CUFFT;
  return PF_OK;
}

}  // extern "C"
