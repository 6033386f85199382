// Deterministic reductions of a field: mass h^d sum(phi) and the discrete free energy
//   E = h^d sum_x [ 1/2 sum_i ((phi_{x+e_i} - phi_x)/h)^2 - c1/2 phi^2 + c2/4 phi^4 ],
// the energy whose discrete gradient flow is Model A (Sec. 3) with forward differences on
// the periodic grid.  Each CTA sums a fixed range of rows in FP64 (per-thread sums over float4
// groups of a row, then warp shuffles, then shared memory) into one partial; one CTA adds the
// partials in a fixed tree order.  The result depends only on the grid shape, not on timing.
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

// Rows of a CTA: the range [r0, r1) of the ny nz rows, walked with (y, z) advanced
// incrementally. A thread takes float4 groups of a row (rows start 16-byte aligned: the pitch
// is a multiple of 4); the group past nx - 1 masks its padding lanes.
struct RowWalk {
  int64_t row, end;
  int y, z;
  __device__ RowWalk(const Geom& g) {
    const int64_t rows = (int64_t)g.ny * g.nz;
    row = rows * blockIdx.x / gridDim.x;
    end = rows * (blockIdx.x + 1) / gridDim.x;
    z = (int)(row / g.ny);
    y = (int)(row - (int64_t)z * g.ny);
  }
  __device__ void next(const Geom& g) {
    ++row;
    if (++y == g.ny) {
      y = 0;
      ++z;
    }
  }
};

__device__ __forceinline__ float lane4(const float4& v, int i) {
  return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}

// Forward-difference energy density of one site: p its value, dx, dy, dz the differences to
// its x+1, y+1 and z+1 neighbours (dz unused in 2D).
__device__ __forceinline__ double ac_energy_site(double p, double dx, double dy, double dz,
                                                 int dim, double c1, double c2, double inv_h2) {
  double grad2 = dx * dx + dy * dy;
  if (dim == 3) grad2 += dz * dz;
  const double p2 = p * p;
  return 0.5 * grad2 * inv_h2 - 0.5 * c1 * p2 + 0.25 * c2 * p2 * p2;
}

__global__ void __launch_bounds__(kNTR) reduce_rows_kernel(int what, Geom g, const float* f,
                                                           double c1, double c2, double inv_h2,
                                                           double* partials) {
  __shared__ double red[kNTR / 32];
  double acc = 0.0;
  const int ng = (g.nx + 3) / 4;  // float4 groups per row
  for (RowWalk w(g); w.row < w.end; w.next(g)) {
    const float* rp = f + (int64_t)w.z * g.plane + (int64_t)w.y * g.pitch;
    if (what == PF_REDUCE_MASS) {
      for (int j = threadIdx.x; j < ng; j += kNTR) {
        const float4 v = *reinterpret_cast<const float4*>(rp + 4 * j);
        const int n = min(4, g.nx - 4 * j);
        double s = (double)v.x;
        if (n > 1) s += (double)v.y;
        if (n > 2) s += (double)v.z;
        if (n > 3) s += (double)v.w;
        acc += s;
      }
    } else {
      const int yn = w.y + 1 == g.ny ? 0 : w.y + 1;
      const int zn = w.z + 1 == g.nz ? 0 : w.z + 1;
      const float* ry = f + (int64_t)w.z * g.plane + (int64_t)yn * g.pitch;
      const float* rz = f + (int64_t)zn * g.plane + (int64_t)w.y * g.pitch;
      for (int j = threadIdx.x; j < ng; j += kNTR) {
        const int x = 4 * j;
        const float4 v = *reinterpret_cast<const float4*>(rp + x);
        const float4 vy = *reinterpret_cast<const float4*>(ry + x);
        const float4 vz = g.dim == 3 ? *reinterpret_cast<const float4*>(rz + x) : v;
        const int n = min(4, g.nx - x);
        const float after = rp[x + 4 >= g.nx ? x + 4 - g.nx : x + 4];  // x+4 (periodic)
        for (int i = 0; i < n; ++i) {
          const double p = lane4(v, i);
          // the x+1 neighbour: in this group, or the row's first value past its last
          const double xn = i + 1 < n ? (double)lane4(v, i + 1) : (x + i + 1 == g.nx ? (double)rp[0] : (double)after);
          acc += ac_energy_site(p, xn - p, (double)lane4(vy, i) - p, (double)lane4(vz, i) - p,
                                g.dim, c1, c2, inv_h2);
        }
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
  double acc = 0.0;
  const int ng = (g.nx + 3) / 4;
  for (RowWalk w(g); w.row < w.end; w.next(g)) {
    const int yn = w.y + 1 == g.ny ? 0 : w.y + 1;
    const int zn = w.z + 1 == g.nz ? 0 : w.z + 1;
    const int64_t o = (int64_t)w.z * g.plane + (int64_t)w.y * g.pitch;
    const int64_t oy = (int64_t)w.z * g.plane + (int64_t)yn * g.pitch;
    const int64_t oz = (int64_t)zn * g.plane + (int64_t)w.y * g.pitch;
    for (int j = threadIdx.x; j < ng; j += kNTR) {
      const int x = 4 * j;
      const int n = min(4, g.nx - x);
      const float4 p4 = *reinterpret_cast<const float4*>(fp + o + x);
      const float4 q4 = *reinterpret_cast<const float4*>(fm + o + x);
      const float4 py = *reinterpret_cast<const float4*>(fp + oy + x);
      const float4 qy = *reinterpret_cast<const float4*>(fm + oy + x);
      const float4 pz = g.dim == 3 ? *reinterpret_cast<const float4*>(fp + oz + x) : p4;
      const float4 qz = g.dim == 3 ? *reinterpret_cast<const float4*>(fm + oz + x) : q4;
      const int xa = x + 4 >= g.nx ? x + 4 - g.nx : x + 4;
      const float pa = fp[o + xa], qa = fm[o + xa];
      for (int i = 0; i < n; ++i) {
        const double p = lane4(p4, i), q = lane4(q4, i);
        const bool wrap = x + i + 1 == g.nx;
        const double pxn = i + 1 < n ? (double)lane4(p4, i + 1) : (wrap ? (double)fp[o] : (double)pa);
        const double qxn = i + 1 < n ? (double)lane4(q4, i + 1) : (wrap ? (double)fm[o] : (double)qa);
        double d, gsum = 0.0;
        d = pxn - p; gsum += d * d;
        d = (double)lane4(py, i) - p; gsum += d * d;
        d = qxn - q; gsum += d * d;
        d = (double)lane4(qy, i) - q; gsum += d * d;
        if (g.dim == 3) {
          d = (double)lane4(pz, i) - p; gsum += d * d;
          d = (double)lane4(qz, i) - q; gsum += d * d;
        }
        const double p2 = p * p, q2 = q * q;
        acc += 0.5 * gsum * inv_h2 - 0.5 * c1 * p2 + 0.25 * c2 * p2 * p2 - 0.5 * c3 * q2 +
               0.25 * c4 * q2 * q2 - c5 * p2 * q;
      }
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
