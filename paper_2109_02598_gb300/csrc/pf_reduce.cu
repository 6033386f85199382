// Deterministic reductions of a field: mass h^d sum(phi) and the discrete free energy
//   E = h^d sum_x [ 1/2 sum_i ((phi_{x+e_i} - phi_x)/h)^2 - c1/2 phi^2 + c2/4 phi^4 ],
// the energy whose discrete gradient flow is Model A (Sec. 3) with forward differences on
// the periodic grid.  Each CTA sums a fixed range of rows in FP64 (per-thread sums, then
// warp shuffles, then shared memory) into one partial; one CTA adds the partials in a fixed
// tree order.  The result depends only on the grid shape, not on timing.
#include "pf_internal.h"

namespace pf {

namespace {

constexpr int kNTR = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

template <int NT>
__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (wid == 0) {
    t = (lane < NT / 32) ? red[lane] : 0.0;
    t = warp_sum(t);
  }
  return t;  // valid in thread 0
}

__global__ void __launch_bounds__(kNTR) reduce_rows_kernel(int what, Geom g, const float* f,
                                                           double c1, double c2, double inv_h2,
                                                           double* partials) {
  __shared__ double red[kNTR / 32];
  const int64_t rows = (int64_t)g.ny * g.nz;
  const int64_t r0 = rows * blockIdx.x / gridDim.x;
  const int64_t r1 = rows * (blockIdx.x + 1) / gridDim.x;
  double acc = 0.0;
  for (int64_t row = r0; row < r1; ++row) {
    const int y = (int)(row % g.ny);
    const int z = (int)(row / g.ny);
    const float* rp = f + (int64_t)z * g.plane + (int64_t)y * g.pitch;
    if (what == PF_REDUCE_MASS) {
      for (int x = threadIdx.x; x < g.nx; x += kNTR) acc += (double)rp[x];
    } else {
      const float* ry = f + (int64_t)z * g.plane + (int64_t)((y + 1) % g.ny) * g.pitch;
      const float* rz = f + (int64_t)((z + 1) % g.nz) * g.plane + (int64_t)y * g.pitch;
      for (int x = threadIdx.x; x < g.nx; x += kNTR) {
        const double p = rp[x];
        const double dx = (double)rp[(x + 1) % g.nx] - p;
        const double dy = (double)ry[x] - p;
        double grad2 = dx * dx + dy * dy;
        if (g.dim == 3) {
          const double dz = (double)rz[x] - p;
          grad2 += dz * dz;
        }
        const double p2 = p * p;
        acc += 0.5 * grad2 * inv_h2 - 0.5 * c1 * p2 + 0.25 * c2 * p2 * p2;
      }
    }
  }
  const double t = block_sum<kNTR>(acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// Model C: 1/2 |grad psi|^2 - c1/2 psi^2 + c2/4 psi^4 + 1/2 |grad m|^2 - c3/2 m^2
// + c4/4 m^4 - c5 psi^2 m, forward differences, summed like reduce_rows_kernel.
__global__ void __launch_bounds__(kNTR) reduce_energy_c_kernel(Geom g, const float* fp,
                                                               const float* fm, double c1,
                                                               double c2, double c3, double c4,
                                                               double c5, double inv_h2,
                                                               double* partials) {
  __shared__ double red[kNTR / 32];
  const int64_t rows = (int64_t)g.ny * g.nz;
  const int64_t r0 = rows * blockIdx.x / gridDim.x;
  const int64_t r1 = rows * (blockIdx.x + 1) / gridDim.x;
  double acc = 0.0;
  for (int64_t row = r0; row < r1; ++row) {
    const int y = (int)(row % g.ny);
    const int z = (int)(row / g.ny);
    const int64_t o = (int64_t)z * g.plane + (int64_t)y * g.pitch;
    const int64_t oy = (int64_t)z * g.plane + (int64_t)((y + 1) % g.ny) * g.pitch;
    const int64_t oz = (int64_t)((z + 1) % g.nz) * g.plane + (int64_t)y * g.pitch;
    for (int x = threadIdx.x; x < g.nx; x += kNTR) {
      const int xp = (x + 1) % g.nx;
      const double p = fp[o + x], q = fm[o + x];
      double d, gsum = 0.0;
      d = (double)fp[o + xp] - p; gsum += d * d;
      d = (double)fp[oy + x] - p; gsum += d * d;
      d = (double)fm[o + xp] - q; gsum += d * d;
      d = (double)fm[oy + x] - q; gsum += d * d;
      if (g.dim == 3) {
        d = (double)fp[oz + x] - p; gsum += d * d;
        d = (double)fm[oz + x] - q; gsum += d * d;
      }
      const double p2 = p * p, q2 = q * q;
      acc += 0.5 * gsum * inv_h2 - 0.5 * c1 * p2 + 0.25 * c2 * p2 * p2 - 0.5 * c3 * q2 +
             0.25 * c4 * q2 * q2 - c5 * p2 * q;
    }
  }
  const double t = block_sum<kNTR>(acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kReduceBlocks) reduce_final_kernel(const double* partials,
                                                                     double scale, double* out) {
  __shared__ double red[kReduceBlocks / 32];
  const double t = block_sum<kReduceBlocks>(partials[threadIdx.x], red);
  if (threadIdx.x == 0) *out = t * scale;
}

}  // namespace

cudaError_t launch_reduce(int what, const Geom& g, const float* field, double c1, double c2,
                          double h, double* d_partials, double* d_out, cudaStream_t s) {
  const double inv_h2 = 1.0 / (h * h);
  reduce_rows_kernel<<<kReduceBlocks, kNTR, 0, s>>>(what, g, field, c1, c2, inv_h2, d_partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  double scale = h * h;
  if (g.dim == 3) scale *= h;
  reduce_final_kernel<<<1, kReduceBlocks, 0, s>>>(d_partials, scale, d_out);
  return cudaGetLastError();
}

cudaError_t launch_reduce_energy_c(const Geom& g, const float* psi, const float* m,
                                   const double* c, double h, double* d_partials,
                                   double* d_out, cudaStream_t s) {
  reduce_energy_c_kernel<<<kReduceBlocks, kNTR, 0, s>>>(g, psi, m, c[0], c[1], c[2], c[3], c[4],
                                                        1.0 / (h * h), d_partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  double scale = h * h;
  if (g.dim == 3) scale *= h;
  reduce_final_kernel<<<1, kReduceBlocks, 0, s>>>(d_partials, scale, d_out);
  return cudaGetLastError();
}

}  // namespace pf
