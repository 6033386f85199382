// N coupled species of reaction-diffusion type (any number of fields up to PF_MAX_FIELDS,
// Sec. 2.3's coupled equations of motion; Gray-Scott of Sec. 1 is the two-species case):
//   du_i/dt = D_i lap u_i + sum_m K[i][m] prod_j u_j^E[m][j]
// with up to kRdMonomials monomials of integer exponents 0..3, advanced by forward Euler
// (Sec. 2.4.1) with the 5-/7-point Laplacian (Sec. 2.2.2), every field from the same state.
//
// One fused kernel per step: a CTA stages its tile plus a one-site periodic halo of every
// field in shared memory (2D: 16-byte cp.async groups; 3D: a three-plane ring streamed
// through z), then evaluates every field's Laplacian and the reaction polynomial in registers
// and writes the new state. Per site, in a fixed order: the monomials prod_j u_j^e by repeated
// multiplication (j ascending), then for each field acc = (D_i h^-2) * (neighbour sum - 2d u_i),
// acc += K[i][m] * monomial_m (fma, m ascending), u_i + dt acc (fma). The 2D and 3D kernels
// share this arithmetic.
#include "pf_internal.h"
#include "pf_tma.cuh"

namespace pf {

namespace {

constexpr int kRdThreads = 256;

// The reaction and the Euler update of one site: u[NF] in, lsum[NF] the Laplacians' neighbour
// sums (before the factor), res[NF] out.
template <int NF>
__device__ __forceinline__ void rd_site(const float* u, const float* lsum, const RdParams& p,
                                        float* res) {
  float mono[kRdMonomials];
#pragma unroll
  for (int m = 0; m < kRdMonomials; ++m) {
    float v = 1.0f;
    if (m < p.nmono) {
#pragma unroll
      for (int j = 0; j < NF; ++j) {
        const int e = (p.E[m] >> (2 * j)) & 3;
#pragma unroll
        for (int t = 0; t < 3; ++t)
          if (t < e) v = __fmul_rn(v, u[j]);
      }
    }
    mono[m] = v;
  }
#pragma unroll
  for (int i = 0; i < NF; ++i) {
    float acc = __fmul_rn(p.D[i], lsum[i]);
#pragma unroll
    for (int m = 0; m < kRdMonomials; ++m)
      if (m < p.nmono) acc = __fmaf_rn(p.K[i][m], mono[m], acc);
    res[i] = __fmaf_rn(p.dt, acc, u[i]);
  }
}

// ---- 2D: TX x TY tiles, rows staged with 4 halo columns each side (16-byte groups)
template <int NF, int TX, int TY>
struct CfgRd2 {
  static constexpr int WS = TX + 8;      // staged row: columns x0-4 .. x0+TX+3
  static constexpr int HT = TY + 2;      // rows y0-1 .. y0+TY
  static constexpr int PL = WS * HT;     // floats per field
  static constexpr int GROUPS = (TX / 4) * TY;
};

template <int NF, int TX, int TY>
__global__ void __launch_bounds__(kRdThreads) rd2d_kernel(FieldPtrs in, FieldOut out, Geom g,
                                                          RdParams p) {
  using C = CfgRd2<NF, TX, TY>;
  extern __shared__ __align__(16) float sm[];
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  canary_fill(sm, (size_t)NF * C::PL);
  constexpr int CH4 = C::WS / 4;
  for (int i = threadIdx.x; i < C::HT * CH4; i += kRdThreads) {
    const int r = i / CH4, j = i - r * CH4;
    const int gy = wrap_index(y0 - 1 + r, g.ny);
    const int gx = x0 - 4 + 4 * j;
    const int64_t row = (int64_t)gy * g.pitch;
    float* dst = sm + r * C::WS + 4 * j;
    if (gx >= 0 && gx + 3 < g.nx) {
#pragma unroll
      for (int f = 0; f < NF; ++f) cp_async16(dst + f * C::PL, in.f[f] + row + gx);
    } else {
#pragma unroll
      for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int c = 0; c < 4; ++c)
          cp_async4(dst + f * C::PL + c, in.f[f] + row + wrap_index(gx + c, g.nx));
    }
  }
  cp_async_wait_all();
  __syncthreads();
  for (int q = threadIdx.x; q < C::GROUPS; q += kRdThreads) {
    const int rr = q / (TX / 4), j = q - rr * (TX / 4);
    const int gy = y0 + rr, gx = x0 + 4 * j;
    if (gy >= g.ny || gx >= g.nx) continue;
    const int pc = (rr + 1) * C::WS + 4 + 4 * j;
    float4 c[NF], ls[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const float* s = sm + f * C::PL;
      c[f] = *reinterpret_cast<const float4*>(s + pc);
      const float4 ym = *reinterpret_cast<const float4*>(s + pc - C::WS);
      const float4 yp = *reinterpret_cast<const float4*>(s + pc + C::WS);
      const float xm = s[pc - 1], xp = s[pc + 4];
      ls[f] = make_float4(lap2d_sum(c[f].x, xm, c[f].y, ym.x, yp.x),
                          lap2d_sum(c[f].y, c[f].x, c[f].z, ym.y, yp.y),
                          lap2d_sum(c[f].z, c[f].y, c[f].w, ym.z, yp.z),
                          lap2d_sum(c[f].w, c[f].z, xp, ym.w, yp.w));
    }
    float4 res[NF];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      float u[NF], l[NF], r[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        u[f] = reinterpret_cast<const float*>(&c[f])[e];
        l[f] = reinterpret_cast<const float*>(&ls[f])[e];
      }
      rd_site<NF>(u, l, p, r);
#pragma unroll
      for (int f = 0; f < NF; ++f) reinterpret_cast<float*>(&res[f])[e] = r[f];
    }
    const int64_t off = (int64_t)gy * g.pitch + gx;
    if (gx + 3 < g.nx) {
#pragma unroll
      for (int f = 0; f < NF; ++f) *reinterpret_cast<float4*>(out.f[f] + off) = res[f];
    } else {
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const float* v = reinterpret_cast<const float*>(&res[f]);
        for (int e = 0; e < 4 && gx + e < g.nx; ++e) out.f[f][off + e] = v[e];
      }
    }
  }
}

// ---- 3D: TX x TY columns streaming a z-chunk through a ring of three planes per field
template <int NF, int TX, int TY>
struct CfgRd3 {
  static constexpr int W = TX + 2, HT = TY + 2;  // plane with a one-site halo
  static constexpr int PL = W * HT;
};

template <int NF, int TX, int TY>
__device__ __forceinline__ void rd_load_plane(const FieldPtrs& in, const Geom& g, int x0,
                                              int y0, int z, float* slot) {
  using C = CfgRd3<NF, TX, TY>;
  const int64_t zoff = (int64_t)wrap_index(z, g.nz) * g.plane;
  for (int i = threadIdx.x; i < C::PL; i += kRdThreads) {
    const int r = i / C::W, c = i - r * C::W;
    const int64_t off = zoff + (int64_t)wrap_index(y0 - 1 + r, g.ny) * g.pitch +
                        wrap_index(x0 - 1 + c, g.nx);
#pragma unroll
    for (int f = 0; f < NF; ++f) cp_async4(slot + f * C::PL + i, in.f[f] + off);
  }
  cp_async_wait_all();
}

template <int NF, int TX, int TY>
__global__ void __launch_bounds__(kRdThreads) rd3d_kernel(FieldPtrs in, FieldOut out, Geom g,
                                                          RdParams p, int tz) {
  using C = CfgRd3<NF, TX, TY>;
  constexpr int W = C::W, PL = C::PL, SLOT = NF * PL;
  extern __shared__ __align__(16) float sm[];
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int z0 = blockIdx.z * tz, z1 = min(z0 + tz, g.nz);
  canary_fill(sm, (size_t)3 * SLOT);
  rd_load_plane<NF, TX, TY>(in, g, x0, y0, z0 - 1, sm);
  rd_load_plane<NF, TX, TY>(in, g, x0, y0, z0, sm + SLOT);
  int sb = 0, sc = 1, sa = 2;
  for (int z = z0; z < z1; ++z) {
    rd_load_plane<NF, TX, TY>(in, g, x0, y0, z + 1, sm + sa * SLOT);
    __syncthreads();
    for (int i = threadIdx.x; i < TX * TY; i += kRdThreads) {
      const int rr = i / TX, cc = i - rr * TX;
      const int gx = x0 + cc, gy = y0 + rr;
      if (gx >= g.nx || gy >= g.ny) continue;
      const int q = (rr + 1) * W + cc + 1;
      float u[NF], l[NF], r[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const float* b = sm + sb * SLOT + f * PL;
        const float* c = sm + sc * SLOT + f * PL;
        const float* a = sm + sa * SLOT + f * PL;
        u[f] = c[q];
        l[f] = lap3d_sum(c[q], c[q - 1], c[q + 1], c[q - W], c[q + W], b[q], a[q]);
      }
      rd_site<NF>(u, l, p, r);
      const int64_t off = (int64_t)z * g.plane + (int64_t)gy * g.pitch + gx;
#pragma unroll
      for (int f = 0; f < NF; ++f) out.f[f][off] = r[f];
    }
    __syncthreads();
    const int t = sb;
    sb = sc;
    sc = sa;
    sa = t;
  }
}

template <int NF>
cudaError_t launch_rd_nf(const Geom& g, FieldPtrs in, FieldOut out, const RdParams& p,
                         cudaStream_t s) {
  if (g.dim == 2) {
    constexpr int TX = 64, TY = 16;
    using C = CfgRd2<NF, TX, TY>;
    const size_t smem = sizeof(float) * NF * C::PL;
    static unsigned long long attr_mask = 0;  // per instantiation and device
    cudaError_t e = ensure_smem_attr(rd2d_kernel<NF, TX, TY>, smem, &attr_mask);
    if (e != cudaSuccess) return e;
    const dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY);
    rd2d_kernel<NF, TX, TY><<<grid, kRdThreads, smem, s>>>(in, out, g, p);
    return cudaGetLastError();
  }
  constexpr int TX = 32, TY = 16;
  using C = CfgRd3<NF, TX, TY>;
  const size_t smem = sizeof(float) * 3 * NF * C::PL;
  static unsigned long long attr_mask = 0;
  cudaError_t e = ensure_smem_attr(rd3d_kernel<NF, TX, TY>, smem, &attr_mask);
  if (e != cudaSuccess) return e;
  const int bx = (g.nx + TX - 1) / TX, by = (g.ny + TY - 1) / TY;
  // z-chunks: enough CTAs for several waves on the SMs, at least 4 planes each
  int tz = g.nz;
  while (tz > 4 && (int64_t)bx * by * ((g.nz + tz - 1) / tz) < 4 * 152) tz = (tz + 1) / 2;
  const dim3 grid(bx, by, (g.nz + tz - 1) / tz);
  rd3d_kernel<NF, TX, TY><<<grid, kRdThreads, smem, s>>>(in, out, g, p, tz);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_rd(const Geom& g, int nf, FieldPtrs in, FieldOut out, const RdParams& p,
                      cudaStream_t s) {
  switch (nf) {
    case 1: return launch_rd_nf<1>(g, in, out, p, s);
    case 2: return launch_rd_nf<2>(g, in, out, p, s);
    case 3: return launch_rd_nf<3>(g, in, out, p, s);
    case 4: return launch_rd_nf<4>(g, in, out, p, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace pf
