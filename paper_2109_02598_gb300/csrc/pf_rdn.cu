// N coupled species of reaction-diffusion type (any number of fields up to PF_MAX_FIELDS,
// Sec. 2.3's coupled equations of motion; Gray-Scott of Sec. 1 is the two-species case):
//   du_i/dt = D_i lap u_i + sum_m K[i][m] prod_j u_j^E[m][j]
// with up to kRdMonomials monomials of integer exponents 0..3, advanced by forward Euler
// (Sec. 2.4.1) with the 5-/7-point Laplacian (Sec. 2.2.2), every field from the same state.
//
// One fused kernel per step: a CTA stages its tile plus a one-site periodic halo of every
// field in shared memory (2D: rows with four halo columns a side as 16-byte cp.async groups;
// 3D: the same rows for each plane of a z-chunk, streamed through a four-plane ring with the
// plane after next in flight while a plane is computed), then each thread takes four
// consecutive sites: every field's Laplacian, the reaction polynomial and the Euler update in
// registers, and one 16-byte store per field. Per site, in a fixed order: for each field
// acc = (D_i h^-2) * (neighbour sum - 2d u_i); for each monomial m (ascending) its value
// prod_j u_j^e by repeated multiplication from 1 (j ascending), then acc_i += K[i][m] * value
// (fma); finally u_i + dt acc_i (fma). The 2D and 3D kernels share this arithmetic.
//
// The exponents are data, the same for every site: a monomial's multiplications run as loops
// whose trip counts are uniform across the warp, each step multiplying a thread's four sites,
// so a site pays only for the multiplications its monomials have (no predicated slots for
// the absent ones), and the rates K[i][m] are constant-bank operands (m is unrolled).
#include "pf_stage.cuh"

namespace pf {

namespace {

// The reaction and the Euler update of four sites: u[f][s] the state, ls[f][s] the
// Laplacians' neighbour sums (before the factor), res[f][s] the new state.
template <int NF>
__device__ __forceinline__ void rd_sites4(const float (&u)[NF][4], const float (&ls)[NF][4],
                                          const RdParams& p, float (&res)[NF][4]) {
  float acc[NF][4];
#pragma unroll
  for (int i = 0; i < NF; ++i)
#pragma unroll
    for (int s = 0; s < 4; ++s) acc[i][s] = __fmul_rn(p.D[i], ls[i][s]);
#pragma unroll
  for (int m = 0; m < kRdMonomials; ++m) {
    if (m >= p.nmono) break;  // uniform
    float v[4] = {1.0f, 1.0f, 1.0f, 1.0f};
#pragma unroll
    for (int j = 0; j < NF; ++j) {
      const int e = (p.E[m] >> (2 * j)) & 3;
#pragma unroll 1
      for (int t = 0; t < e; ++t)
#pragma unroll
        for (int s = 0; s < 4; ++s) v[s] = __fmul_rn(v[s], u[j][s]);
    }
#pragma unroll
    for (int i = 0; i < NF; ++i)
#pragma unroll
      for (int s = 0; s < 4; ++s) acc[i][s] = __fmaf_rn(p.K[i][m], v[s], acc[i][s]);
  }
#pragma unroll
  for (int i = 0; i < NF; ++i)
#pragma unroll
    for (int s = 0; s < 4; ++s) res[i][s] = __fmaf_rn(p.dt, acc[i][s], u[i][s]);
}

// Store four sites of every field at off (gx = their first column).
template <int NF>
__device__ __forceinline__ void rd_store4(const FieldOut& out, int64_t off, int gx, int nx,
                                          const float (&res)[NF][4]) {
  if (gx + 3 < nx) {
#pragma unroll
    for (int f = 0; f < NF; ++f)
      *reinterpret_cast<float4*>(out.f[f] + off) =
          make_float4(res[f][0], res[f][1], res[f][2], res[f][3]);
  } else {
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (gx + e < nx) out.f[f][off + e] = res[f][e];
  }
}

// ---- 2D: TX x TY tiles, rows staged with 4 halo columns each side (16-byte groups)
constexpr int kRd2Threads = 256;

template <int NF, int TX, int TY>
struct CfgRd2 {
  static constexpr int WS = TX + 8;      // staged row: columns x0-4 .. x0+TX+3
  static constexpr int HT = TY + 2;      // rows y0-1 .. y0+TY
  static constexpr int PL = WS * HT;     // floats per field
  static constexpr int GROUPS = (TX / 4) * TY;
};

template <int NF, int TX, int TY>
__global__ void __launch_bounds__(kRd2Threads) rd2d_kernel(FieldPtrs in, FieldOut out, Geom g,
                                                           RdParams p) {
  using C = CfgRd2<NF, TX, TY>;
  extern __shared__ __align__(16) float sm[];
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  canary_fill(sm, (size_t)NF * C::PL);
  stage_rows4<NF>(in, g, x0, y0, 0, C::WS, C::HT, C::PL, sm, kRd2Threads);
  cp_async_wait_all();
  __syncthreads();
  for (int q = threadIdx.x; q < C::GROUPS; q += kRd2Threads) {
    const int rr = q / (TX / 4), j = q - rr * (TX / 4);
    const int gy = y0 + rr, gx = x0 + 4 * j;
    if (gy >= g.ny || gx >= g.nx) continue;
    const int pc = (rr + 1) * C::WS + 4 + 4 * j;
    float u[NF][4], ls[NF][4];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const float* s = sm + f * C::PL;
      const float4 c = *reinterpret_cast<const float4*>(s + pc);
      const float4 ym = *reinterpret_cast<const float4*>(s + pc - C::WS);
      const float4 yp = *reinterpret_cast<const float4*>(s + pc + C::WS);
      const float xm = s[pc - 1], xp = s[pc + 4];
      u[f][0] = c.x;
      u[f][1] = c.y;
      u[f][2] = c.z;
      u[f][3] = c.w;
      ls[f][0] = lap2d_sum(c.x, xm, c.y, ym.x, yp.x);
      ls[f][1] = lap2d_sum(c.y, c.x, c.z, ym.y, yp.y);
      ls[f][2] = lap2d_sum(c.z, c.y, c.w, ym.z, yp.z);
      ls[f][3] = lap2d_sum(c.w, c.z, xp, ym.w, yp.w);
    }
    float res[NF][4];
    rd_sites4<NF>(u, ls, p, res);
    rd_store4<NF>(out, (int64_t)gy * g.pitch + gx, gx, g.nx, res);
  }
}

// ---- 3D: TX x TY columns streaming a z-chunk through a ring of four planes per field
constexpr int kRd3Threads = 128;

template <int NF, int TX, int TY>
struct CfgRd3 {
  static constexpr int WS = TX + 8, HT = TY + 2;  // staged plane: as the 2D tile
  static constexpr int PL = WS * HT;               // floats per field and plane
  static constexpr int SLOT = NF * PL;
  static constexpr int GROUPS = (TX / 4) * TY;
  static_assert(GROUPS == kRd3Threads, "one group of four sites per thread and plane");
};

template <int NF, int TX, int TY>
__global__ void __launch_bounds__(kRd3Threads) rd3d_kernel(FieldPtrs in, FieldOut out, Geom g,
                                                           RdParams p, int tz) {
  using C = CfgRd3<NF, TX, TY>;
  constexpr int WS = C::WS, PL = C::PL, SLOT = C::SLOT;
  extern __shared__ __align__(16) float sm[];
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int z0 = blockIdx.z * tz, z1 = min(z0 + tz, g.nz);
  canary_fill(sm, (size_t)4 * SLOT);
  // plane p sits in slot (p - z0 + 1) % 4; planes z0 - 1, z0, z0 + 1 first, one group each
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    stage_rows4<NF>(in, g, x0, y0, (int64_t)wrap_index(z0 - 1 + k, g.nz) * g.plane, WS, C::HT, PL,
                 sm + k * SLOT, kRd3Threads);
    cp_async_commit();
  }
  const int rr = threadIdx.x / (TX / 4), j = threadIdx.x - rr * (TX / 4);
  const int gy = y0 + rr, gx = x0 + 4 * j;
  const bool active = gy < g.ny && gx < g.nx;
  const int pc = (rr + 1) * WS + 4 + 4 * j;
  for (int z = z0; z < z1; ++z) {
    const int i = z - z0;
    // plane z + 2 into the slot of plane z - 2 (free since the barrier closing the last
    // iteration); it is the next iteration's z + 1 plane
    if (z + 2 <= z1)
      stage_rows4<NF>(in, g, x0, y0, (int64_t)wrap_index(z + 2, g.nz) * g.plane, WS, C::HT, PL,
                   sm + ((i + 3) & 3) * SLOT, kRd3Threads);
    cp_async_commit();         // possibly empty: the group count stays one per iteration
    cp_async_wait_group<1>();  // all but the newest group: plane z + 1 has landed
    __syncthreads();
    if (active) {
      const float* b = sm + (i & 3) * SLOT;        // plane z - 1
      const float* c = sm + ((i + 1) & 3) * SLOT;  // plane z
      const float* a = sm + ((i + 2) & 3) * SLOT;  // plane z + 1
      float u[NF][4], ls[NF][4];
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const float* cf = c + f * PL;
        const float4 q = *reinterpret_cast<const float4*>(cf + pc);
        const float4 ym = *reinterpret_cast<const float4*>(cf + pc - WS);
        const float4 yp = *reinterpret_cast<const float4*>(cf + pc + WS);
        const float4 zm = *reinterpret_cast<const float4*>(b + f * PL + pc);
        const float4 zp = *reinterpret_cast<const float4*>(a + f * PL + pc);
        const float xm = cf[pc - 1], xp = cf[pc + 4];
        u[f][0] = q.x;
        u[f][1] = q.y;
        u[f][2] = q.z;
        u[f][3] = q.w;
        ls[f][0] = lap3d_sum(q.x, xm, q.y, ym.x, yp.x, zm.x, zp.x);
        ls[f][1] = lap3d_sum(q.y, q.x, q.z, ym.y, yp.y, zm.y, zp.y);
        ls[f][2] = lap3d_sum(q.z, q.y, q.w, ym.z, yp.z, zm.z, zp.z);
        ls[f][3] = lap3d_sum(q.w, q.z, xp, ym.w, yp.w, zm.w, zp.w);
      }
      float res[NF][4];
      rd_sites4<NF>(u, ls, p, res);
      rd_store4<NF>(out, (int64_t)z * g.plane + (int64_t)gy * g.pitch + gx, gx, g.nx, res);
    }
    __syncthreads();  // every thread is done with plane z - 1 before its slot is refilled
  }
  cp_async_wait_all();  // nothing in flight at exit (the last groups are empty)
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
    rd2d_kernel<NF, TX, TY><<<grid, kRd2Threads, smem, s>>>(in, out, g, p);
    return cudaGetLastError();
  }
  constexpr int TX = 32, TY = 16;
  using C = CfgRd3<NF, TX, TY>;
  const size_t smem = sizeof(float) * 4 * C::SLOT;
  static unsigned long long attr_mask = 0;
  cudaError_t e = ensure_smem_attr(rd3d_kernel<NF, TX, TY>, smem, &attr_mask);
  if (e != cudaSuccess) return e;
  static int resident[64] = {};  // per device
  const int bx = (g.nx + TX - 1) / TX, by = (g.ny + TY - 1) / TY;
  const int tz = one_wave_tz(g.nz, bx * by,
                             resident_ctas(rd3d_kernel<NF, TX, TY>, kRd3Threads, smem, resident));
  const dim3 grid(bx, by, (g.nz + tz - 1) / tz);
  rd3d_kernel<NF, TX, TY><<<grid, kRd3Threads, smem, s>>>(in, out, g, p, tz);
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
