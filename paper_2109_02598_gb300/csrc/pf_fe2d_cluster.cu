// 2D forward-Euler step for grids small enough to live on chip: one thread-block cluster
// holds the whole grid in shared memory and runs every step of a pf_step call in one launch.
//
// CTA `rank` of the cluster (CS CTAs) owns the band of rows [rank B, (rank+1) B), B = ny/CS,
// kept in the tile layout of the 2D tile body with full rows: WS = nx + 2 HP floats per row
// (HP halo columns per side, which hold periodic copies of the row's other end) and
// HT = B + 2H rows (H = K R halo rows per side). A super-step advances K steps:
//   1. the halo rows are copied from this CTA's receive buffer, into which the neighbouring
//      bands stored their H edge rows at the end of the previous super-step (the first
//      super-step stages everything from global memory instead);
//   2. K sub-steps on shrinking regions, exactly as the tiled kernels do them (the same
//      per-site functions, so every path gives the same bits);
//   3. the band's top H rows are stored into the receive buffer of the band above, its
//      bottom H rows into that of the band below (remote stores to distributed shared
//      memory), and the cluster synchronises (barrier.cluster with release / acquire: all
//      CTAs of a cluster are co-scheduled and run the same number of super-steps, so it
//      always completes, and the stores are visible after it).
// Receive buffers are double-buffered by parity, so one cluster barrier per super-step
// suffices: a CTA reads parity p during super-step s while its neighbours store parity
// 1 - p. The halo columns are never refreshed in a pass of their own: every write of a value
// whose column lies within HP of a row end (staging, halo rows, the last sub-step) also
// writes its periodic copy. After the last super-step each CTA writes its band to global
// memory; no distributed shared memory access follows the last barrier.
#include <cooperative_groups.h>

#include "pf_fe2d_tile.cuh"
#include "pf_internal.h"

namespace cg = cooperative_groups;

namespace pf {

namespace {

struct ClGeom {
  int nx, ny, band;  // band = ny / CS rows per CTA
  int ws, ht;        // staged row width (floats) and rows
  int pl;            // floats per staged field
  int64_t pitch;     // global row pitch (floats)
};

template <int MODEL, int K>
struct CfgCl {
  static constexpr int NF = ModelTraits<MODEL>::NF;
  static constexpr int RS = 1;  // standard 5-point stencil
  static constexpr int R = ModelTraits<MODEL>::R;
  static constexpr int H = K * R;
  static constexpr int HP = (H + 3) / 4 * 4;
  static constexpr bool MU = MODEL == PF_MODEL_CH || MODEL == PF_MODEL_C;
};

constexpr int kNTC = 512;  // threads per CTA

// Floats of shared memory: two work buffers of NF fields, the chemical potential, and the
// receive buffers [2 parities][2 sides][NF][H rows][nx] (side 0: the rows above the band).
template <int MODEL, int K>
size_t cluster_smem_floats(const ClGeom& g) {
  using C = CfgCl<MODEL, K>;
  return (size_t)2 * C::NF * g.pl + (C::MU ? g.pl : 0) + (size_t)4 * C::NF * C::H * g.nx;
}

template <int MODEL, int K>
__global__ void __launch_bounds__(kNTC, 1)
    fe2d_cluster_kernel(FieldPtrs in, FieldOut out, ClGeom g, ModelParams m, int64_t n_steps) {
  using C = CfgCl<MODEL, K>;
  constexpr int NF = C::NF, R = C::R, RS = C::RS, H = C::H, HP = C::HP;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int cs = (int)cluster.num_blocks();
  extern __shared__ float4 smem4[];
  float* sm = reinterpret_cast<float*>(smem4);
  const int WS = g.ws, HT = g.ht, PL = g.pl, NX = g.nx, B = g.band;
  float* cur = sm;
  float* alt = sm + NF * PL;
  float* mu = sm + 2 * NF * PL;
  float* recv = mu + (C::MU ? PL : 0);  // [parity][side][f][r][x]
  const int EXF = H * NX;                // floats per (parity, side, field)
  const int y0 = rank * B;
  const int nx4 = NX / 4;
  // sub-step work: thread (tr, tj) takes column groups tj, tj + ngl, ... of rows
  // rlo + tr, rlo + tr + rstep, ... (no per-item division)
  const int ngl = WS / 4 < kNTC ? WS / 4 : kNTC;
  const int tj = threadIdx.x % ngl, tr = threadIdx.x / ngl, rstep = kNTC / ngl;

#ifdef PF_CHECK
  canary_fill(sm, (size_t)2 * NF * PL + (C::MU ? PL : 0) + (size_t)4 * NF * H * NX);
  cluster.sync();  // no neighbour stores into this CTA's receive buffers before the fill
#endif
  // stage rows y0 - H .. y0 + B + H - 1 (periodic in y) with their halo columns
  for (int i = threadIdx.x; i < HT * nx4; i += kNTC) {
    const int r = i / nx4, j = i - r * nx4;
    const int gy = wrap_index(y0 - H + r, g.ny);
#pragma unroll
    for (int f = 0; f < NF; ++f)
      put_row4<HP>(cur + f * PL + r * WS, j, NX,
                   __ldg(reinterpret_cast<const float4*>(in.f[f] + gy * g.pitch + 4 * j)));
  }
  __syncthreads();

  int par = 0;
  bool first = true;
  for (int64_t left = n_steps; left > 0;) {
    const int keff = left >= K ? K : (int)left;
    if (!first) {
      // 1. halo rows from the receive buffer (parity par), with their periodic copies
      for (int i = threadIdx.x; i < NF * H * nx4; i += kNTC) {
        const int f = i / (H * nx4);
        const int rem = i - f * H * nx4;
        const int r = rem / nx4, j = rem - r * nx4;
        const int eo = f * EXF + r * NX + 4 * j;
        put_row4<HP>(cur + f * PL + r * WS, j, NX,
                     *reinterpret_cast<const float4*>(recv + (par * 2 + 0) * NF * EXF + eo));
        put_row4<HP>(cur + f * PL + (H + B + r) * WS, j, NX,
                     *reinterpret_cast<const float4*>(recv + (par * 2 + 1) * NF * EXF + eo));
      }
      __syncthreads();
    }
    first = false;
    // 2. keff sub-steps; with keff < K the regions start as if K - keff sub-steps had run
    for (int s = 0; s < keff; ++s) {
      const int e = s + (K - keff);
      const bool last = (s == keff - 1);
      if constexpr (C::MU) {
        const int rlo = R * e + RS, rhi = HT - rlo;
        const int clo = (HP - H + R * e + RS) / 4;
        const int chi = (WS - (HP - H + R * e + RS) + 3) / 4;
        if (tr < rstep)
          for (int r = rlo + tr; r < rhi; r += rstep)
            for (int j = tj; j < chi; j += ngl)
              if (j >= clo) site4_mu<MODEL, PF_ST_STD>(cur, r * WS + 4 * j, WS, PL, m, mu);
        __syncthreads();
      }
      const int rlo = R * (e + 1), rhi = HT - rlo;
      const int clo = last ? HP / 4 : (HP - H + R * (e + 1)) / 4;
      const int chi = last ? (HP + NX) / 4 : (WS - (HP - H + R * (e + 1)) + 3) / 4;
      if (tr < rstep) {
        for (int r = rlo + tr; r < rhi; r += rstep) {
          for (int j = tj; j < chi; j += ngl) {
            if (j < clo) continue;
            const int p = r * WS + 4 * j;
            float4 val[NF];
            site4_update<MODEL, PF_ST_STD>(cur, mu, p, WS, PL, m, val);
            if (last) {  // band interior: also the periodic copies, for the next super-step
#pragma unroll
              for (int f = 0; f < NF; ++f)
                put_row4<HP>(alt + f * PL + r * WS, j - HP / 4, NX, val[f]);
            } else {
#pragma unroll
              for (int f = 0; f < NF; ++f) *reinterpret_cast<float4*>(alt + f * PL + p) = val[f];
            }
          }
        }
      }
      __syncthreads();
      float* t = cur;
      cur = alt;
      alt = t;
    }
    left -= keff;
    if (left > 0) {
      // 3. the band's top H rows into the receive buffer of the band above (its side 1),
      // the bottom H rows into that of the band below (its side 0), parity par ^ 1
      const int np = par ^ 1;
      float* rv_up = cluster.map_shared_rank(recv, (rank + cs - 1) % cs);
      float* rv_dn = cluster.map_shared_rank(recv, (rank + 1) % cs);
      for (int i = threadIdx.x; i < NF * H * nx4; i += kNTC) {
        const int f = i / (H * nx4);
        const int rem = i - f * H * nx4;
        const int r = rem / nx4, j = rem - r * nx4;
        const int eo = f * EXF + r * NX + 4 * j;
        *reinterpret_cast<float4*>(rv_up + (np * 2 + 1) * NF * EXF + eo) =
            *reinterpret_cast<const float4*>(cur + f * PL + (H + r) * WS + HP + 4 * j);
        *reinterpret_cast<float4*>(rv_dn + (np * 2 + 0) * NF * EXF + eo) =
            *reinterpret_cast<const float4*>(cur + f * PL + (B + r) * WS + HP + 4 * j);
      }
      par = np;
      cluster.sync();
    }
  }
  // the band's rows to global memory
  for (int i = threadIdx.x; i < B * nx4; i += kNTC) {
    const int r = i / nx4, j = i - r * nx4;
#pragma unroll
    for (int f = 0; f < NF; ++f)
      *reinterpret_cast<float4*>(out.f[f] + (int64_t)(y0 + r) * g.pitch + 4 * j) =
          *reinterpret_cast<const float4*>(cur + f * PL + (H + r) * WS + HP + 4 * j);
  }
}

template <int MODEL, int K>
ClGeom cluster_geom(const Geom& q, int cs) {
  using C = CfgCl<MODEL, K>;
  ClGeom g{};
  g.nx = q.nx;
  g.ny = q.ny;
  g.band = q.ny / cs;
  g.ws = q.nx + 2 * C::HP;
  g.ht = g.band + 2 * C::H;
  g.pl = g.ws * g.ht;
  g.pitch = q.pitch;
  return g;
}

int g_cluster_size[64] = {};  // per device: 16 if non-portable clusters of 16 are allowed, else 8

int cluster_size_for_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 8;
  }
  if (dev < 64 && g_cluster_size[dev]) return g_cluster_size[dev];
  int cs = 8;
  auto kern = fe2d_cluster_kernel<PF_MODEL_AC, 1>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
      cudaSuccess) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(16);
    cfg.blockDim = dim3(kNTC);
    cfg.dynamicSmemBytes = 0;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = 16;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int ok = 0;
    if (cudaOccupancyMaxPotentialClusterSize(&ok, kern, &cfg) == cudaSuccess && ok >= 16) cs = 16;
  }
  cudaGetLastError();
  if (dev < 64) g_cluster_size[dev] = cs;
  return cs;
}

template <int MODEL, int K>
bool cluster_fits(const Geom& q, int cs) {
  using C = CfgCl<MODEL, K>;
  if (q.dim != 2 || q.nx % 4 != 0 || q.nx < C::HP || q.ny % cs != 0) return false;
  const ClGeom g = cluster_geom<MODEL, K>(q, cs);
  if (g.band < C::H || g.band < 1) return false;
  return cluster_smem_floats<MODEL, K>(g) * sizeof(float) <= 220 * 1024;
}

template <int MODEL, int K>
cudaError_t launch_cluster(const Geom& q, FieldPtrs in, FieldOut out, const ModelParams& m,
                           int64_t n_steps, cudaStream_t st) {
  const int cs = cluster_size_for_device();
  const ClGeom g = cluster_geom<MODEL, K>(q, cs);
  const size_t smem = cluster_smem_floats<MODEL, K>(g) * sizeof(float);
  auto kern = fe2d_cluster_kernel<MODEL, K>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && cs > 8)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(cs);
  cfg.blockDim = dim3(kNTC);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = cs;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, in, out, g, m, n_steps);
}

}  // namespace

int fe2d_cluster_size() { return cluster_size_for_device(); }

bool fe2d_cluster_supported(int model, int k, const Geom& q) {
  const int cs = cluster_size_for_device();
  switch (model) {
    case PF_MODEL_AC:
      return k == 1   ? cluster_fits<PF_MODEL_AC, 1>(q, cs)
             : k == 2 ? cluster_fits<PF_MODEL_AC, 2>(q, cs)
             : k == 4 ? cluster_fits<PF_MODEL_AC, 4>(q, cs)
                      : k == 8 && cluster_fits<PF_MODEL_AC, 8>(q, cs);
    case PF_MODEL_GS:
      return k == 1   ? cluster_fits<PF_MODEL_GS, 1>(q, cs)
             : k == 2 ? cluster_fits<PF_MODEL_GS, 2>(q, cs)
             : k == 4 ? cluster_fits<PF_MODEL_GS, 4>(q, cs)
                      : k == 8 && cluster_fits<PF_MODEL_GS, 8>(q, cs);
    case PF_MODEL_CH:
      return k == 1 ? cluster_fits<PF_MODEL_CH, 1>(q, cs)
                    : k == 2 && cluster_fits<PF_MODEL_CH, 2>(q, cs);
    case PF_MODEL_C:
      return k == 1 ? cluster_fits<PF_MODEL_C, 1>(q, cs)
                    : k == 2 && cluster_fits<PF_MODEL_C, 2>(q, cs);
  }
  return false;
}

cudaError_t launch_fe2d_cluster(int model, int k, const Geom& q, FieldPtrs in, FieldOut out,
                                const ModelParams& m, int64_t n_steps, cudaStream_t st) {
  if (!fe2d_cluster_supported(model, k, q)) return cudaErrorInvalidValue;
  switch (model) {
    case PF_MODEL_AC:
      if (k == 1) return launch_cluster<PF_MODEL_AC, 1>(q, in, out, m, n_steps, st);
      if (k == 2) return launch_cluster<PF_MODEL_AC, 2>(q, in, out, m, n_steps, st);
      if (k == 4) return launch_cluster<PF_MODEL_AC, 4>(q, in, out, m, n_steps, st);
      return launch_cluster<PF_MODEL_AC, 8>(q, in, out, m, n_steps, st);
    case PF_MODEL_GS:
      if (k == 1) return launch_cluster<PF_MODEL_GS, 1>(q, in, out, m, n_steps, st);
      if (k == 2) return launch_cluster<PF_MODEL_GS, 2>(q, in, out, m, n_steps, st);
      if (k == 4) return launch_cluster<PF_MODEL_GS, 4>(q, in, out, m, n_steps, st);
      return launch_cluster<PF_MODEL_GS, 8>(q, in, out, m, n_steps, st);
    case PF_MODEL_CH:
      if (k == 1) return launch_cluster<PF_MODEL_CH, 1>(q, in, out, m, n_steps, st);
      return launch_cluster<PF_MODEL_CH, 2>(q, in, out, m, n_steps, st);
    case PF_MODEL_C:
      if (k == 1) return launch_cluster<PF_MODEL_C, 1>(q, in, out, m, n_steps, st);
      return launch_cluster<PF_MODEL_C, 2>(q, in, out, m, n_steps, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace pf
