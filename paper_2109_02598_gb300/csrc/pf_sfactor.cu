// Radially averaged structure factor of a phase indicator (analysis of the phase-separated
// systems of Sec. 3): rho = [psi > 0], rho_hat by a float64 transform, S = |rho_hat|^2 / N,
// binned by |k| with per-bin sums taken in a fixed order.
//
// The half spectrum holds each mode k with kx in (0, nx/2) once for itself and once for its
// mirror -k (equal |k|, equal S for a real rho), so those modes count twice; kx = 0 and the
// Nyquist plane of an even nx count once.  |k| and the bin index are float64, evaluated with
// the correctly rounded operations of the definition in a fixed order.
#include <cuda_runtime.h>

#include <cmath>

#include "pf_cufft.h"
#include "pf_internal.h"

namespace pf {
int invalid(const char* fmt, ...);
}

namespace pf {
namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kMaxBins = 1024;
constexpr int kMaxBinBlocks = 2 * 152;

struct SfGeom {
  int rank;
  int64_t d[3];  // C order, x last
  int64_t nxh, nk, nsite;
  double h, kmax;
  int n_bins;
};

__device__ __forceinline__ double fft_index(int64_t i, int64_t n) {
  return (double)(i <= (n - 1) / 2 ? i : i - n);
}

__device__ __forceinline__ double wavenumber(double f, int64_t n, double h) {
  const double val = __ddiv_rn(1.0, __dmul_rn((double)n, h));
  return __dmul_rn(2.0 * 3.141592653589793, __dmul_rn(f, val));
}

__global__ void indicator_kernel(const float* __restrict__ psi, int64_t pitch, int64_t nx,
                                 int64_t ny, int64_t nsite, double* __restrict__ rho) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nsite;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = i % nx, row = i / nx;  // row = z * ny + y
    rho[i] = psi[row * pitch + x] > 0.f ? 1.0 : 0.0;
  }
}

// Each block takes a contiguous range of modes, split into one contiguous range per warp.
// A warp computes 32 modes at a time; lane 0 adds them into the warp's own histogram in
// lane order. The block then sums its warps' histograms in warp order.
__global__ void __launch_bounds__(kThreads)
    sf_bin_kernel(const double2* __restrict__ rhat, SfGeom g, int64_t per_block,
                  double* __restrict__ part_sum, unsigned long long* __restrict__ part_cnt) {
  extern __shared__ unsigned char smem_raw[];
  double* wsum = reinterpret_cast<double*>(smem_raw);
  unsigned long long* wcnt =
      reinterpret_cast<unsigned long long*>(wsum + (size_t)kWarps * g.n_bins);
  for (int i = threadIdx.x; i < kWarps * g.n_bins; i += kThreads) {
    wsum[i] = 0.0;
    wcnt[i] = 0ull;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t b0 = (int64_t)blockIdx.x * per_block;
  const int64_t b1 = min(g.nk, b0 + per_block);
  const int64_t per_warp = (b1 - b0 + kWarps - 1) / kWarps;
  const int64_t w0 = min(b1, b0 + warp * per_warp);
  const int64_t w1 = min(b1, w0 + per_warp);
  const int64_t nx = g.d[g.rank - 1], ny = g.d[g.rank - 2];
  const double nbins = (double)g.n_bins;
  double* my_sum = wsum + (size_t)warp * g.n_bins;
  unsigned long long* my_cnt = wcnt + (size_t)warp * g.n_bins;
  for (int64_t base = w0; base < w1; base += 32) {
    const int64_t i = base + lane;
    int bin = 0, weight = 0;
    double S = 0.0;
    if (i < w1) {
      const int64_t ix = i % g.nxh, rest = i / g.nxh;
      const double kx = wavenumber(fft_index(ix, nx), nx, g.h);
      const double ky = wavenumber(fft_index(rest % ny, ny), ny, g.h);
      double s2;
      if (g.rank == 3) {
        const double kz = wavenumber(fft_index(rest / ny, g.d[0]), g.d[0], g.h);
        s2 = __dadd_rn(__dadd_rn(__dmul_rn(kz, kz), __dmul_rn(ky, ky)), __dmul_rn(kx, kx));
      } else {
        s2 = __dadd_rn(__dmul_rn(ky, ky), __dmul_rn(kx, kx));
      }
      const double kmag = __dsqrt_rn(s2);
      if (kmag > 0.0) {
        const double q = __dmul_rn(__ddiv_rn(kmag, g.kmax), nbins);
        const double fq = floor(q);
        bin = fq >= (double)(g.n_bins - 1) ? g.n_bins - 1 : (int)fq;
        weight = (ix == 0 || 2 * ix == nx) ? 1 : 2;
        const double2 r = rhat[i];
        S = __ddiv_rn(__dadd_rn(__dmul_rn(r.x, r.x), __dmul_rn(r.y, r.y)), (double)g.nsite);
      }
    }
    for (int src = 0; src < 32; ++src) {
      const int b = __shfl_sync(0xffffffffu, bin, src);
      const int w = __shfl_sync(0xffffffffu, weight, src);
      const double v = __shfl_sync(0xffffffffu, S, src);
      if (lane == 0 && w > 0) {
        my_sum[b] = __dadd_rn(my_sum[b], v);
        if (w == 2) my_sum[b] = __dadd_rn(my_sum[b], v);
        my_cnt[b] += (unsigned long long)w;
      }
    }
  }
  __syncthreads();
  for (int b = threadIdx.x; b < g.n_bins; b += kThreads) {
    double s = 0.0;
    unsigned long long c = 0ull;
    for (int w = 0; w < kWarps; ++w) {
      s = __dadd_rn(s, wsum[(size_t)w * g.n_bins + b]);
      c += wcnt[(size_t)w * g.n_bins + b];
    }
    part_sum[(size_t)blockIdx.x * g.n_bins + b] = s;
    part_cnt[(size_t)blockIdx.x * g.n_bins + b] = c;
  }
}

__global__ void sf_final_kernel(const double* __restrict__ part_sum,
                                const unsigned long long* __restrict__ part_cnt, int nblocks,
                                int n_bins, double* __restrict__ mean,
                                long long* __restrict__ counts) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < n_bins; b += gridDim.x * blockDim.x) {
    double s = 0.0;
    unsigned long long c = 0ull;
    for (int k = 0; k < nblocks; ++k) {
      s = __dadd_rn(s, part_sum[(size_t)k * n_bins + b]);
      c += part_cnt[(size_t)k * n_bins + b];
    }
    mean[b] = c > 0 ? __ddiv_rn(s, (double)c) : 0.0;
    counts[b] = (long long)c;
  }
}

unsigned long long g_bin_smem_mask = 0;

}  // namespace
}  // namespace pf

using namespace pf;

extern "C" int pf_structure_factor(int dim, const int64_t* n, int64_t pitch, const float* psi,
                                   double h, int n_bins, double* centres, double* mean,
                                   int64_t* counts, void* stream) {
  if (n == nullptr || psi == nullptr || centres == nullptr || mean == nullptr ||
      counts == nullptr)
    return invalid("pf_structure_factor: NULL argument");
  if (dim != 2 && dim != 3) return invalid("dim must be 2 or 3 (got %d)", dim);
  const int64_t nx = n[0], ny = n[1], nz = dim == 3 ? n[2] : 1;
  const int64_t lim = (int64_t)1 << 30;
  if (nx < 2 || ny < 1 || nz < 1 || nx > lim || ny > lim || nz > lim || nx * ny > lim ||
      nx * ny * nz > lim)
    return invalid("sizes must be nx >= 2, ny, nz >= 1, with at most 2^30 sites (got %lld x "
                   "%lld x %lld)", (long long)nx, (long long)ny, (long long)nz);
  if (pitch < nx || pitch > lim) return invalid("pitch %lld must be in [nx, 2^30]", (long long)pitch);
  if (!(h > 0.0) || !std::isfinite(h)) return invalid("h must be finite and > 0");
  if (n_bins < 1 || n_bins > kMaxBins) return invalid("n_bins must be in [1, %d]", kMaxBins);
  const CufftApi* api = cufft_api();
  if (api == nullptr) return PF_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;

  SfGeom g{};
  g.rank = dim;
  if (dim == 2) {
    g.d[0] = ny;
    g.d[1] = nx;
  } else {
    g.d[0] = nz;
    g.d[1] = ny;
    g.d[2] = nx;
  }
  g.nxh = nx / 2 + 1;
  g.nk = g.nxh * ny * nz;
  g.nsite = nx * ny * nz;
  g.h = h;
  g.kmax = (3.141592653589793 / h) * std::sqrt((double)dim);
  g.n_bins = n_bins;

  int64_t nblocks = (g.nk + 4095) / 4096;
  if (nblocks > kMaxBinBlocks) nblocks = kMaxBinBlocks;
  const int64_t per_block = (g.nk + nblocks - 1) / nblocks;

  // One allocation: rho, rho_hat, partial sums and counts, results.
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t b_rho = up(sizeof(double) * (size_t)g.nsite);
  const size_t b_hat = up(sizeof(double2) * (size_t)g.nk);
  const size_t b_part = up(sizeof(double) * (size_t)(nblocks * n_bins));
  const size_t b_res = up(sizeof(double) * (size_t)n_bins);
  unsigned char* mem = nullptr;
  cudaError_t e = cudaMalloc(&mem, b_rho + b_hat + 2 * b_part + 2 * b_res);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("pf_structure_factor: out of device memory");
    return PF_ERR_OOM;
  }
  double* rho = reinterpret_cast<double*>(mem);
  double2* rhat = reinterpret_cast<double2*>(mem + b_rho);
  double* psum = reinterpret_cast<double*>(mem + b_rho + b_hat);
  unsigned long long* pcnt = reinterpret_cast<unsigned long long*>(mem + b_rho + b_hat + b_part);
  double* d_mean = reinterpret_cast<double*>(mem + b_rho + b_hat + 2 * b_part);
  long long* d_cnt = reinterpret_cast<long long*>(mem + b_rho + b_hat + 2 * b_part + b_res);

  cufftHandle plan = -1;
  int rc = cufft_plan(api, &plan, dim, g.d, CUFFT_D2Z, 1, 0, 0, 1, nullptr);
  if (rc == PF_OK) {
    int64_t blocks = (g.nsite + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    indicator_kernel<<<(int)blocks, 256, 0, st>>>(psi, pitch, nx, ny, g.nsite, rho);
    e = cudaGetLastError();
    cufftResult r = CUFFT_SUCCESS;
    if (e == cudaSuccess) {
      r = api->set_stream(plan, st);
      if (r == CUFFT_SUCCESS) r = api->exec_d2z(plan, rho, reinterpret_cast<cufftDoubleComplex*>(rhat));
    }
    if (r != CUFFT_SUCCESS) {
      rc = cufft_fail(r, "pf_structure_factor transform");
    } else {
      const size_t smem = (size_t)kWarps * n_bins * (sizeof(double) + sizeof(unsigned long long));
      if (e == cudaSuccess)
        e = ensure_smem_attr(sf_bin_kernel, (size_t)kWarps * kMaxBins * 16, &g_bin_smem_mask);
      if (e == cudaSuccess) {
        sf_bin_kernel<<<(int)nblocks, kThreads, smem, st>>>(rhat, g, per_block, psum, pcnt);
        e = cudaGetLastError();
      }
      if (e == cudaSuccess) {
        sf_final_kernel<<<(n_bins + 255) / 256, 256, 0, st>>>(psum, pcnt, (int)nblocks, n_bins,
                                                              d_mean, d_cnt);
        e = cudaGetLastError();
      }
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(mean, d_mean, sizeof(double) * n_bins, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(counts, d_cnt, sizeof(int64_t) * n_bins, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) rc = cuda_fail(e, "pf_structure_factor");
    }
  }
  if (plan != -1) api->destroy(plan);
  cudaStreamSynchronize(st);
  cudaFree(mem);
  if (rc != PF_OK) return rc;
  for (int b = 0; b < n_bins; ++b) centres[b] = ((double)b + 0.5) * g.kmax / (double)n_bins;
  return PF_OK;
}

extern "C" int pf_porod_fit(int n_bins, const double* centres, const double* mean,
                            const int64_t* counts, double k_lo, double k_hi, double* slope,
                            double* intercept, int* n_used) {
  if (centres == nullptr || mean == nullptr || counts == nullptr || slope == nullptr ||
      intercept == nullptr || n_used == nullptr)
    return invalid("pf_porod_fit: NULL argument");
  if (n_bins < 1) return invalid("n_bins must be >= 1");
  if (!(k_lo < k_hi)) return invalid("the window needs k_lo < k_hi");
  // two passes over the usable bins in bin order: the means, then the centred sums
  int n = 0;
  double sx = 0.0, sy = 0.0;
  auto usable = [&](int b) {
    return centres[b] >= k_lo && centres[b] <= k_hi && counts[b] > 0 && mean[b] > 0.0;
  };
  for (int b = 0; b < n_bins; ++b) {
    if (!usable(b)) continue;
    sx += std::log(centres[b]);
    sy += std::log(mean[b]);
    ++n;
  }
  if (n < 2) return invalid("fewer than two usable bins in [%g, %g]", k_lo, k_hi);
  const double xbar = sx / n, ybar = sy / n;
  double sxy = 0.0, sxx = 0.0;
  for (int b = 0; b < n_bins; ++b) {
    if (!usable(b)) continue;
    const double dx = std::log(centres[b]) - xbar;
    const double dy = std::log(mean[b]) - ybar;
    sxy += dx * dy;
    sxx += dx * dx;
  }
  if (!(sxx > 0.0)) return invalid("the usable bins share one centre");
  *slope = sxy / sxx;
  *intercept = ybar - *slope * xbar;
  *n_used = n;
  return PF_OK;
}
