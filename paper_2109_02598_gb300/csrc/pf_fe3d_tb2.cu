// 3D forward-Euler with temporal blocking of depth 2 for the radius-1 models (Allen-Cahn,
// Gray-Scott): two time steps per pass over HBM (Sec. 2.4.1 solver, Sec. 2.2.2 7-point
// Laplacian), so HBM traffic per lattice-site update halves to 4 NF bytes.
//
// Tiles span whole x-rows (W = nx, 128 or 256), so the periodic wrap in x is an index wrap
// inside shared memory; a CTA owns TY rows and streams z-ranges of them (the split over the
// CTAs is Tb2Sched below).  Per input plane, TMA brings rows y0-2 .. y0+TY+1 of every field
// (three boxes: two rows above, the TY rows, two rows below, wrapped in y) into an NS-stage
// ring.  Thread (x4, r), r = 0 .. TY+1, computes the first time level on row y0-1+r (one
// row wider than the tile in y) and stores it to a two-plane buffer in shared memory;
// threads r = 1 .. TY then compute the second level on row y0-1+r from it and write it to
// HBM.  Both levels keep their z-neighbours in registers (each thread reads the planes of
// its own column), and the same per-site functions as every other kernel make the result
// bitwise identical to two depth-1 steps.
//
// Requires nx == W, ny % TY == 0 and ny >= 2.
#include "pf_grid.h"
#include "pf_internal.h"
#include "pf_tma.cuh"

#include <cudaTypedefs.h>

#include <algorithm>
#include <type_traits>

namespace pf {

namespace {

template <int MODEL, int W, int TY, int NS, int V_ = 1>
struct CfgB {
  static constexpr int NF = ModelTraits<MODEL>::NF;
  static constexpr int LX = W / 4;              // float4 columns per row
  static constexpr int V = V_;                  // float4 columns per thread
  static constexpr int TPR = LX / V;            // threads per row: one warp or two
  static constexpr int NT = TPR * (TY + 2);     // one thread per first-level column group
  static constexpr int IN_ROWS = TY + 4;        // staged input rows (halo 2)
  static constexpr int IN_FIELD = IN_ROWS * W;  // floats per field per input stage
  static constexpr int IN_STAGE = NF * IN_FIELD;
  static constexpr int L1_ROWS = TY + 2;
  static constexpr int L1_FIELD = L1_ROWS * W;
  static constexpr int L1_PLANE = NF * L1_FIELD;
  static constexpr uint32_t TX_BYTES = IN_STAGE * 4;
  static constexpr size_t SMEM =
      (size_t)(NS * IN_STAGE + 2 * L1_PLANE) * 4 + NS * 8 + 128;  // + barriers + align
  static_assert(TPR == 32 || TPR == 64, "a row is one warp or two");
};

// x-neighbour scalars of a thread's V float4 columns 4 V lane .. 4 V lane + 4 V - 1 of a row
// that one warp holds whole (the grid's full periodic row): the left neighbour of the first
// column is the previous lane's last value, the right neighbour of the last column the next
// lane's first value, lane 0 and lane 31 wrapping to each other. No shared-memory load: the
// earlier layout (one float4 per thread, two warps per 256-wide row) took the values at the
// warps' ends from shared memory, two loads per field and level.
template <int V>
__device__ __forceinline__ void x_edges_row(const float4 (&c)[V], float& xm, float& xp) {
  const int lane = threadIdx.x & 31;
  xm = __shfl_sync(0xffffffffu, c[V - 1].w, (lane + 31) & 31);
  xp = __shfl_sync(0xffffffffu, c[0].x, (lane + 1) & 31);
}

// The same for a row that two warps share (one float4 column per thread, 256-wide rows):
// the neighbouring lanes' c.w and c.x by warp shuffle, and at the warp's two ends one load
// from the shared row whose address is the same for every lane (a broadcast). Plain scalar
// loads of the two neighbours, four floats apart across the lanes, cost four shared-memory
// wavefronts each (four lanes per bank); this costs two.
template <int W>
__device__ __forceinline__ void x_edges_c(const float* row, int x4, const float4& c, float& xm,
                                          float& xp) {
  const int lane = threadIdx.x & 31;
  const int xb = x4 - lane;  // first float4 column of this warp
  const float em = row[xb == 0 ? W - 1 : 4 * xb - 1];
  const float ep = row[xb + 32 == W / 4 ? 0 : 4 * (xb + 32)];
  const float wm = __shfl_up_sync(0xffffffffu, c.w, 1);
  const float wp = __shfl_down_sync(0xffffffffu, c.x, 1);
  xm = lane == 0 ? em : wm;
  xp = lane == 31 ? ep : wp;
}

template <int MODEL>
__device__ __forceinline__ void update4(const float4* c, const float4* lap, float4* res,
                                        const ModelParams& m) {
  if constexpr (MODEL == PF_MODEL_AC) {
    res[0].x = ac_update(c[0].x, lap[0].x, m);
    res[0].y = ac_update(c[0].y, lap[0].y, m);
    res[0].z = ac_update(c[0].z, lap[0].z, m);
    res[0].w = ac_update(c[0].w, lap[0].w, m);
  } else {
    gs_update(c[0].x, c[1].x, lap[0].x, lap[1].x, m, res[0].x, res[1].x);
    gs_update(c[0].y, c[1].y, lap[0].y, lap[1].y, m, res[0].y, res[1].y);
    gs_update(c[0].z, c[1].z, lap[0].z, lap[1].z, m, res[0].z, res[1].z);
    gs_update(c[0].w, c[1].w, lap[0].w, lap[1].w, m, res[0].w, res[1].w);
  }
}

// 7-point Laplacians of four sites: centre c, z-neighbours zm/zp, rows above/below and the
// two x-edge scalars of the centre row. Gray-Scott's stencil factor is carried in D_u and D_v
// (its lap_scale is 1), so its final multiply is left out, as lap_scaled does: the same bits,
// eight instructions fewer per float4 and level (GS 256^3: 503 -> 521 GLUPS). The sums run as
// packed FP32 pairs (lap3d_sum4: lap3d_sum's operations in its order, each lane's bits
// unchanged) while the update stays scalar, which splits the arithmetic between the heavy FMA
// pipe (the pairs) and both pipes (the scalars): GS 256^3 558 -> 596 GLUPS. Packing the
// update too loads the heavy pipe alone (measured slower before this change).
template <int MODEL>
__device__ __forceinline__ float4 lap3d_x4(const float4& c, const float4& ym, const float4& yp,
                                           const float4& zm, const float4& zp, float xm,
                                           float xp, float lap_scale) {
  float4 l = lap3d_sum4(c, xm, xp, ym, yp, zm, zp);
  if constexpr (MODEL != PF_MODEL_GS) l = mul4(lap_scale, l);  // lap_scaled
  return l;
}

// How the (row tile, plane) work is split over the CTAs (chosen on the host, tb2_schedule).
//   ITEMS:    item = (tile, chunk of chunk_len planes), items dealt round-robin over the CTAs,
//             chunks alternating up and down in z.
//   BALANCED: the (tile, plane) units in tile-major order cut into gridDim.x equal ranges,
//             one per CTA (a range crossing a tile boundary makes two segments), direction
//             alternating by CTA.
//   ROWS:     full_rows rows of one CTA per tile, row c streaming planes [c L, (c+1) L) in
//             the direction of chunk c; the remaining CTAs split the top row [full_rows L, nz)
//             of every tile in tile-major order. CTAs of neighbouring tiles in a full row work
//             on the same plane at the same time, so the halo rows they share come from L2.
struct Tb2Sched {
  int mode;
  int nchunks, chunk_len;    // ITEMS
  int full_rows, L, pdir;    // ROWS: rows of ncols CTAs, their chunk length, partial direction
};
constexpr int kTb2Items = 0, kTb2Balanced = 1, kTb2Rows = 2;

// Per-thread state of one z-stream: z-windows of the input planes (level 1's z-neighbours and
// centre) and of the first-level planes (level 2's), three slots each, slot = plane mod 3, so
// the plane loop, unrolled by three, renames them instead of moving them.
template <int MODEL, int W, int TY, int NS, int V_>
struct Tb2Stream {
  using C = CfgB<MODEL, W, TY, NS, V_>;
  static constexpr int NF = C::NF;
  static constexpr int V = C::V;
  float4 iw[NF][3][V];  // input planes
  float4 lw[NF][3][V];  // first-level planes

  // Laplacians of the thread's V float4 columns: centre c (row `row` of a shared plane, read
  // only where two warps share the row), rows above / below, z-neighbours.
  __device__ __forceinline__ static void laps(const float4 (&c)[V], const float* row, int col0,
                                              const float4 (&ym)[V], const float4 (&yp)[V],
                                              const float4 (&zm)[V], const float4 (&zp)[V],
                                              float lap_scale, float4 (&l)[V]) {
    float xm, xp;
    if constexpr (C::TPR == 32)
      x_edges_row<V>(c, xm, xp);
    else
      x_edges_c<W>(row, col0 / 4, c[0], xm, xp);
#pragma unroll
    for (int i = 0; i < V; ++i)
      l[i] = lap3d_x4<MODEL>(c[i], ym[i], yp[i], zm[i], zp[i], i == 0 ? xm : c[i - 1].w,
                             i == V - 1 ? xp : c[i + 1].x, lap_scale);
  }

  // Plane iteration j (phase P = j mod 3): level 1 on row r of first-level plane j from
  // input planes j (slot P), j + 1 (P + 1, centre) and j + 2 (P + 2, read from stage sp
  // now), into lw slot P and the shared plane l1w; then, for j >= 2 on rows 1 .. TY, level 2
  // of output plane j - 2 from first-level planes j - 2 (P + 1), j - 1 (P + 2, with its
  // y-neighbours from the shared plane l1r) and j (P), stored to HBM at off.
  template <int P>
  __device__ __forceinline__ void step(const float* sc, const float* sp, float* l1w,
                                       const float* l1r, int r, int col0, bool level2,
                                       const FieldOut& out, int64_t off, const ModelParams& m) {
    constexpr int S0 = P, S1 = (P + 1) % 3, S2 = (P + 2) % 3;
    float4 lap[NF][V];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const float* F = sc + f * C::IN_FIELD;
      float4 ym[V], yp[V];
#pragma unroll
      for (int i = 0; i < V; ++i) {
        ym[i] = *reinterpret_cast<const float4*>(F + r * W + col0 + 4 * i);
        yp[i] = *reinterpret_cast<const float4*>(F + (r + 2) * W + col0 + 4 * i);
        iw[f][S2][i] = *reinterpret_cast<const float4*>(sp + f * C::IN_FIELD + (r + 1) * W +
                                                        col0 + 4 * i);
      }
      laps(iw[f][S1], F + (r + 1) * W, col0, ym, yp, iw[f][S0], iw[f][S2], m.lap_scale, lap[f]);
    }
#pragma unroll
    for (int i = 0; i < V; ++i) {
      float4 c[NF], l[NF], res[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        c[f] = iw[f][S1][i];
        l[f] = lap[f][i];
      }
      update4<MODEL>(c, l, res, m);
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        lw[f][S0][i] = res[f];
        *reinterpret_cast<float4*>(l1w + f * C::L1_FIELD + r * W + col0 + 4 * i) = res[f];
      }
    }
    if (!level2) return;
    float4 lap2[NF][V];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const float* F = l1r + f * C::L1_FIELD;
      float4 ym[V], yp[V];
#pragma unroll
      for (int i = 0; i < V; ++i) {
        ym[i] = *reinterpret_cast<const float4*>(F + (r - 1) * W + col0 + 4 * i);
        yp[i] = *reinterpret_cast<const float4*>(F + (r + 1) * W + col0 + 4 * i);
      }
      laps(lw[f][S2], F + r * W, col0, ym, yp, lw[f][S1], lw[f][S0], m.lap_scale, lap2[f]);
    }
#pragma unroll
    for (int i = 0; i < V; ++i) {
      float4 c[NF], l[NF], res[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        c[f] = lw[f][S2][i];
        l[f] = lap2[f][i];
      }
      update4<MODEL>(c, l, res, m);
#pragma unroll
      for (int f = 0; f < NF; ++f) *reinterpret_cast<float4*>(out.f[f] + off + 4 * i) = res[f];
    }
  }
};

template <int MODEL, int W, int TY, int NS, int V_>
__global__ void __launch_bounds__(CfgB<MODEL, W, TY, NS, V_>::NT, 1)
    fe3d_tb2_kernel(const __grid_constant__ Tb2Maps maps, FieldOut out, Geom g, ModelParams m,
                    Tb2Sched sc_, int* err_flag) {
  using C = CfgB<MODEL, W, TY, NS, V_>;
  constexpr int NF = C::NF;
  constexpr int V = C::V;
  extern __shared__ unsigned char smem_raw[];
  const uint32_t base_sa = smem_addr(smem_raw);
  float* ring = reinterpret_cast<float*>(smem_raw + ((128 - (base_sa & 127)) & 127));
  float* l1 = ring + NS * C::IN_STAGE;  // two first-level planes
  uint64_t* bars = reinterpret_cast<uint64_t*>(l1 + 2 * C::L1_PLANE);

  const int tid = threadIdx.x;
  const int r = tid / C::TPR;             // first-level row y0 - 1 + r; input row r + 1
  const int col0 = 4 * V * (tid % C::TPR);  // first column of this thread's V float4 columns
  const bool second = (r >= 1 && r <= TY);  // the same in the whole warp
  canary_fill(ring, (size_t)NS * C::IN_STAGE + 2 * C::L1_PLANE);  // TMA issues follow a proxy fence
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) mbar_init(&bars[s], 1);
    mbar_fence_init();
  }
  __syncthreads();

  uint32_t q_base = 0, q_issued = 0;
  bool err = false;
  auto stage_ptr = [&](uint32_t q) { return ring + (q % NS) * C::IN_STAGE; };
  auto issue = [&](uint32_t q, int y0, int p) {
    float* st = stage_ptr(q);
    uint64_t* bar = &bars[q % NS];
    const int z = wrap_index(p, g.nz);
    const int ytop = wrap_index(y0 - 2, g.ny);
    const int ybot = wrap_index(y0 + TY, g.ny);
    mbar_arrive_expect_tx(bar, C::TX_BYTES);
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      float* fs = st + f * C::IN_FIELD;
      tma_load_3d(fs, &maps.row2[f], 0, ytop, z, bar);
      tma_load_3d(fs + 2 * W, &maps.inner[f], 0, y0, z, bar);
      tma_load_3d(fs + (TY + 2) * W, &maps.row2[f], 0, ybot, z, bar);
    }
  };
  auto wait = [&](uint32_t q) -> bool {
    return mbar_wait_bounded(&bars[q % NS], (q / NS) & 1u, kWaitBudgetCycles);
  };

  const int ncols = g.ny / TY;
  // Work: (row tile, z-range) segments, per the schedule's mode (Tb2Sched).
  // units = ny nz / TY < 2^31 for every grid this kernel takes (nx = W, at most 2^36 sites)
  // Live across a segment: pos, pos_end (BALANCED, the ROWS top row) or item; the rest is
  // recomputed from the launch parameters when a segment starts.
  int pos = 0, pos_end = 0, item = blockIdx.x;
  const int nfull = sc_.full_rows * ncols;
  if (sc_.mode == kTb2Balanced) {
    const int units = ncols * g.nz;
    pos = (int)((int64_t)units * blockIdx.x / gridDim.x);
    pos_end = (int)((int64_t)units * (blockIdx.x + 1) / gridDim.x);
  } else if (sc_.mode == kTb2Rows && (int)blockIdx.x >= nfull) {
    const int units = ncols * (g.nz - sc_.full_rows * sc_.L);
    const int p = blockIdx.x - nfull, np = gridDim.x - nfull;
    pos = (int)((int64_t)units * p / np);
    pos_end = (int)((int64_t)units * (p + 1) / np);
  }
  Tb2Stream<MODEL, W, TY, NS, V_> zs;
  for (;;) {
    int col, zlo, zhi, dir;
    if (sc_.mode == kTb2Items || (sc_.mode == kTb2Rows && (int)blockIdx.x < nfull)) {
      const bool rows = sc_.mode == kTb2Rows;
      if (item >= (rows ? nfull : ncols * sc_.nchunks)) break;
      col = item % ncols;
      const int chunk = item / ncols;
      const int len = rows ? sc_.L : sc_.chunk_len;
      zlo = chunk * len;
      zhi = min(g.nz, zlo + len);
      dir = (chunk & 1) ? -1 : 1;
      item += rows ? nfull : gridDim.x;
      if (zlo >= zhi) continue;  // uniform over the CTA
    } else {
      if (pos >= pos_end) break;
      const bool rows = sc_.mode == kTb2Rows;
      const int zbase = rows ? sc_.full_rows * sc_.L : 0;
      const int zlen = g.nz - zbase;
      col = pos / zlen;
      zlo = pos - col * zlen;
      zhi = min(zlen, zlo + (pos_end - pos));
      pos += zhi - zlo;
      zlo += zbase;
      zhi += zbase;
      dir = rows ? sc_.pdir : ((blockIdx.x & 1) ? -1 : 1);
    }
    const int n = zhi - zlo;                  // output planes
    const int zfirst = dir > 0 ? zlo : zhi - 1;
    const int y0 = col * TY;
    const int nin = n + 4;                    // input planes zfirst-2dir .. zlast+2dir
    auto in_plane = [&](int i) { return zfirst + (i - 2) * dir; };

    if (__syncthreads_or(err)) break;
    if (tid == 0) {
      fence_proxy_async_smem();
      const int n0 = nin < NS ? nin : NS;
      for (int i = 0; i < n0; ++i) issue(q_base + i, y0, in_plane(i));
      q_issued = q_base + n0;
    }
    // prologue: this thread's columns of input planes 0 and 1 (window slots 0 and 1)
    err = !wait(q_base);
    if (!err) {
      const float* st = stage_ptr(q_base);
#pragma unroll
      for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int i = 0; i < V; ++i)
          zs.iw[f][0][i] = *reinterpret_cast<const float4*>(st + f * C::IN_FIELD + (r + 1) * W +
                                                            col0 + 4 * i);
    }
    if (!err) err = !wait(q_base + 1);
    if (!err) {
      const float* st = stage_ptr(q_base + 1);
#pragma unroll
      for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int i = 0; i < V; ++i)
          zs.iw[f][1][i] = *reinterpret_cast<const float4*>(st + f * C::IN_FIELD + (r + 1) * W +
                                                            col0 + 4 * i);
    }
    // first-level plane j = 0 .. n+1 is plane zfirst + (j-1) dir, from input planes j, j+1,
    // j+2; second-level output o = j - 2 uses first-level planes o, o+1, o+2 (in registers,
    // o+1's rows above and below from shared memory). The stages of input planes j+1, j+2 and
    // the mbarrier phase of j+2 advance incrementally instead of by division. Two first-level
    // planes in shared memory suffice: iteration j writes plane j into the slot of plane
    // j - 2, which iteration j - 1 read last, and the barrier at the top of iteration j
    // separates the two.
    uint32_t s1 = (q_base + 1) % NS, s2 = (q_base + 2) % NS;
    uint32_t ph2 = ((q_base + 2) / NS) & 1u;
    // one plane iteration of phase P; false: stop (a wait ran out somewhere in the CTA)
    auto plane = [&](auto phase, int j) -> bool {
      constexpr int P = decltype(phase)::value;
      if (__syncthreads_or(err)) return false;
      if (tid == 0 && j + NS < nin) {
        fence_proxy_async_smem();
        issue(q_base + j + NS, y0, in_plane(j + NS));
        q_issued = q_base + j + NS + 1;
      }
      err = !mbar_wait_bounded(&bars[s2], ph2, kWaitBudgetCycles);
      err = __any_sync(0xffffffffu, err);  // the shuffles need the whole warp
      if (err) return true;                // the next barrier stops the CTA
      const float* sc = ring + s1 * C::IN_STAGE;
      const float* sp = ring + s2 * C::IN_STAGE;
      s1 = s2;
      if (++s2 == NS) {
        s2 = 0;
        ph2 ^= 1u;
      }
      float* l1w = l1 + (j & 1) * C::L1_PLANE;        // first-level plane j
      const float* l1r = l1 + ((j + 1) & 1) * C::L1_PLANE;  // and j - 1
      const int z = zfirst + (j - 2) * dir;
      const int64_t off = (int64_t)z * g.plane + (int64_t)(y0 + r - 1) * g.pitch + col0;
      zs.template step<P>(sc, sp, l1w, l1r, r, col0, j >= 2 && second, out, off, m);
      return true;
    };
    const int nj = n + 2;
    for (int j = 0; j < nj; j += 3) {
      if (!plane(std::integral_constant<int, 0>(), j)) break;
      if (j + 1 >= nj || !plane(std::integral_constant<int, 1>(), j + 1)) break;
      if (j + 2 >= nj || !plane(std::integral_constant<int, 2>(), j + 2)) break;
    }
    q_base += nin;
  }

  if (__syncthreads_or(err)) {
    if (tid == 0) {
      atomicExch(err_flag, 1);
      for (uint32_t q = (q_issued > NS ? q_issued - NS : 0); q < q_issued; ++q)
        (void)mbar_wait_bounded(&bars[q % NS], (q / NS) & 1u, kWaitBudgetCycles);
    }
  }
}

// The work split with the shortest longest-CTA plane count (each segment streams 4 halo
// planes besides its own), ROWS preferred when it is within one plane of the best, since it
// keeps neighbouring tiles in step over z.
Tb2Sched tb2_schedule(int ncols, int nz, long long slots, long long* grid_out) {
  Tb2Sched s{};
  // ITEMS
  long long nchunks = slots / ncols;
  if (nchunks > nz / 4) nchunks = nz / 4;
  if (nchunks < 1) nchunks = 1;
  const int chunk_len = (int)((nz + nchunks - 1) / nchunks);
  nchunks = (nz + chunk_len - 1) / chunk_len;
  const long long items = (long long)ncols * nchunks;
  const long long item_grid = items < slots ? items : slots;
  const long long item_span = (items + item_grid - 1) / item_grid * (chunk_len + 4);
  // BALANCED: about units / slots + 8 planes (two segments at most when a range is under nz)
  const long long units = (long long)ncols * nz;
  const long long per = (units + slots - 1) / slots;
  const long long bal_span = per + (per < nz ? 8 : 4 * ((per + nz - 1) / nz + 1));
  const long long bal_grid = slots < units ? slots : units;
  // ROWS
  long long rows_span = -1, rows_L = 0;
  const long long F = slots / ncols, R = slots - F * ncols;
  for (long long L = 4; F >= 1 && L * F <= nz; ++L) {
    const long long Lp = nz - F * L;  // planes of the top row
    long long span = L + 4;
    if (Lp > 0) {
      if (R == 0) continue;
      const long long pu = ((long long)ncols * Lp + R - 1) / R;
      const long long segs = (pu + Lp - 1) / Lp + 1;
      span = std::max(span, pu + 4 * segs);
    }
    if (rows_span < 0 || span < rows_span) {
      rows_span = span;
      rows_L = L;
    }
  }
  const long long best = std::min(item_span, slots > item_grid ? bal_span : item_span);
  if (rows_span > 0 && rows_span <= best + 1) {
    s.mode = kTb2Rows;
    s.full_rows = (int)F;
    s.L = (int)rows_L;
    s.pdir = ((F - 1) & 1) ? 1 : -1;  // meet the last full row's chunk at its end
    *grid_out = (nz - F * rows_L) > 0 ? slots : F * ncols;
  } else if (bal_span < item_span && slots > item_grid) {
    s.mode = kTb2Balanced;
    *grid_out = bal_grid;
  } else {
    s.mode = kTb2Items;
    *grid_out = item_grid;
  }
  s.nchunks = (int)nchunks;
  s.chunk_len = chunk_len;
  return s;
}

template <int MODEL, int W, int TY, int NS, int V = 1>
cudaError_t launch_tb2(pf_grid_s* gr, const Tb2Maps& maps, FieldOut out, cudaStream_t st) {
  using C = CfgB<MODEL, W, TY, NS, V>;
  auto kern = fe3d_tb2_kernel<MODEL, W, TY, NS, V>;
  static unsigned long long attr_mask = 0;  // per instantiation and device
  cudaError_t e = ensure_smem_attr(kern, C::SMEM, &attr_mask);
  if (e != cudaSuccess) return e;
  static int occ_by_dev[64] = {};  // resident CTAs per SM, per device
  int occ = gr->device < 64 ? occ_by_dev[gr->device] : 0;
  if (occ == 0) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, C::NT, C::SMEM);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    if (gr->device < 64) occ_by_dev[gr->device] = occ;
  }
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, gr->device);
  if (e != cudaSuccess) return e;
  const Geom g = grid_geom(gr);
  long long grid = 0;
  const Tb2Sched sc = tb2_schedule(g.ny / TY, g.nz, (long long)sms * occ, &grid);
  kern<<<(unsigned)grid, C::NT, C::SMEM, st>>>(maps, out, g, gr->params, sc, gr->d_err);
  return cudaGetLastError();
}

}  // namespace

bool fe3d_tb2_supported(int model, int tx, int ty, const Geom& g) {
  if (model != PF_MODEL_AC && model != PF_MODEL_GS) return false;
  if (ty != 8 || (tx != 128 && tx != 256)) return false;
  return g.nx == tx && g.ny % ty == 0 && g.ny >= 2;
}

cudaError_t tb2_maps(pf_grid_s* gr, int tx, int buf) {
  Tb2Cache& tc = gr->tb2;
  if (tc.width == tx && tc.valid[buf]) return cudaSuccess;
  if (tc.width != tx) {
    tc.valid[0] = tc.valid[1] = false;
    tc.width = tx;
  }
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (encode == nullptr) {
    cudaDriverEntryPointQueryResult qr;
    void* fn = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &qr);
    if (e != cudaSuccess) return e;
    if (qr != cudaDriverEntryPointSuccess || fn == nullptr) return cudaErrorNotSupported;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const cuuint64_t dims[3] = {(cuuint64_t)gr->nx, (cuuint64_t)gr->ny, (cuuint64_t)gr->nz};
  const cuuint64_t strides[2] = {(cuuint64_t)gr->pitch * 4, (cuuint64_t)gr->plane * 4};
  const cuuint32_t estr[3] = {1, 1, 1};
  const cuuint32_t box_row2[3] = {(cuuint32_t)tx, 2, 1};
  const cuuint32_t box_inner[3] = {(cuuint32_t)tx, 8, 1};
  for (int f = 0; f < gr->nf; ++f) {
    void* base = gr->buf[buf][f];
    Tb2Maps& mp = tc.maps[buf];
    CUresult r = encode(&mp.row2[f], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides,
                        box_row2, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r == CUDA_SUCCESS)
      r = encode(&mp.inner[f], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box_inner,
                 estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  }
  tc.valid[buf] = true;
  return cudaSuccess;
}

cudaError_t launch_fe3d_tb2(pf_grid_s* gr, int tx, int src, int dst, cudaStream_t st) {
  cudaError_t e = tb2_maps(gr, tx, src);
  if (e != cudaSuccess) return e;
  FieldOut out{};
  for (int f = 0; f < gr->nf; ++f) out.f[f] = gr->buf[dst][f];
  const Tb2Maps& maps = gr->tb2.maps[src];
  if (gr->model == PF_MODEL_GS) {
    // seven ring stages (213 KB of shared memory): 559 GLUPS on 256^3 against 553 with 4-6
    if (tx == 256) return launch_tb2<PF_MODEL_GS, 256, 8, 7>(gr, maps, out, st);
    return launch_tb2<PF_MODEL_GS, 128, 8, 6>(gr, maps, out, st);
  }
  if (gr->model == PF_MODEL_AC) {
    if (tx == 256) return launch_tb2<PF_MODEL_AC, 256, 8, 6>(gr, maps, out, st);
    return launch_tb2<PF_MODEL_AC, 128, 8, 6>(gr, maps, out, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace pf
