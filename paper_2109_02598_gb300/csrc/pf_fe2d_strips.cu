// 2D forward-Euler steps streamed through registers (Sec. 2.4.1 solver with the 5-point
// stencil of Sec. 2.2.2; Models A, B, C and Gray-Scott, Sec. 3).
//
// A warp owns a strip of 32 C consecutive columns: lane i holds columns xs + C i .. + C - 1.
// It walks down the strip one row per iteration and runs K forward-Euler levels at once, all
// in registers: level s keeps the last three rows it produced (a three-slot window per
// field, slot = iteration mod 3), the level above reads them, and the row neighbours across
// lanes come by warp shuffle. Nothing goes through shared memory and no barrier is needed: a
// warp is a self-contained task. The strip's outer HXP columns on either side are halo whose
// values go wrong by one column per stencil application (the shuffle has no neighbour there),
// so after K levels only the middle WO = 32 C - 2 HXP columns are stored.
//
// Levels run from K down to 1 within an iteration, each from the windows as the previous
// iteration left them, so no level waits on another in the same iteration, and the input row
// is loaded last (it is first read one iteration later). Radius-1 models (A, Gray-Scott):
// level s of iteration t computes row ys + t - 2 s (ys = y0 - K is the first row loaded).
// Radius-2 models (B, C): level s first computes the chemical potential of level s - 1 on the
// centre row of that level's window, then its own row one above from the potential window
// (whose newest row it has just written) and the state row kept in the window's oldest slot;
// Model C also keeps lap psi beside mu, computed from the same centre row. Level s then
// trails level s - 1 by three rows per iteration: row ys + t - 3 s, ys = y0 - 2 K.
//
// The per-site arithmetic is that of the tile body (lap2d_sum with the same operands in the
// same order, ac_update, ch_mu, ch_update, gs_update, mc_mu, mc_update), so every path gives
// the same bits.
//
// Allen-Cahn and Gray-Scott also run with the isotropic 9-point Laplacian (Sec. 2.2.2): its
// diagonal neighbours lie in the rows above and below, which the windows hold already, and
// the ones beyond a lane come by two more shuffles per row. Its radius is still one site, so
// the halo columns and the level schedule are those of the 5-point stencil.
#include "pf_internal.h"
#include "pf_model.cuh"

namespace pf {

template <int MODEL, int K, int C>
struct StripCfg {
  static constexpr int NF = ModelTraits<MODEL>::NF;
  static constexpr int R = ModelTraits<MODEL>::R;   // 1 (A, Gray-Scott) or 2 (B, C)
  static constexpr int HX = K * R;                  // halo columns the K levels consume
  static constexpr int HXP = (HX + C - 1) / C * C;  // ... rounded up to whole lanes
  static constexpr int WO = 32 * C - 2 * HXP;       // output columns per strip
  static constexpr int NM = MODEL == PF_MODEL_C ? 2 : 1;  // mu (and Model C's lap psi)
  // Floats a lane holds in windows: the warps per SM the register allocation must allow
  // follow from it (65536 / (32 x MINW) registers per thread). The kernels wait mostly on
  // their row loads, so more resident warps pay until spills cost more than they hide: with
  // fewer than 96 floats of windows, 32 warps (64 registers, the most one-warp CTAs can
  // reach: 32 CTAs per SM) with at most a few spilled words (measured: Model B 8192^2 at
  // K = 2, C = 4 843 -> 1107 GLUPS, Gray-Scott 4096^2 at K = 4, C = 2 870 -> 907, Model C
  // 4096^2 at K = 2, C = 2 381 -> 487, against 20 warps); with 96 or more, 16 or 12 warps
  // (Gray-Scott 4096^2 at K = 4, C = 4: 16 warps of 128 registers 681 GLUPS, 12 of 154
  // registers 550, 32 of 64 registers 378 with kilobytes of spills).
  static constexpr int WIN = K * 3 * C * (NF + (R == 2 ? NM : 0));
  static constexpr int MINW = (WIN > 96 || (MODEL == PF_MODEL_C && WIN == 96)) ? 12
                              : WIN >= 96 ? 16 : 32;
  static_assert(WO > 0, "strip too narrow for this depth");
};

namespace {

// One warp per CTA: every value a task derives from its index (strip origin, rows, and in
// the batch the instance's pointers, sizes and coefficients) is then the same across the
// CTA, which lets the compiler keep it in uniform registers and leaves the vector registers
// to the windows (measured: Gray-Scott 4096^2 at K = 4, 741 GLUPS with four warps per CTA,
// 785 with one).
constexpr int kStripWarps = 1;
constexpr int kStripThreads = 32 * kStripWarps;

// A lane's C values of one row. xin (the same in every lane of the warp): every lane's
// columns lie inside the row, so each takes one vector load (gx is a multiple of C and rows
// start 16-byte aligned); otherwise every lane takes C periodic scalar loads, so the warp
// never splits between the two paths.
template <int C>
__device__ __forceinline__ void load_lane(const float* __restrict__ row, int gx, int nx,
                                          bool xin, float (&v)[C]) {
  if (xin) {
    if constexpr (C == 4) {
      const float4 q = __ldg(reinterpret_cast<const float4*>(row + gx));
      v[0] = q.x;
      v[1] = q.y;
      v[2] = q.z;
      v[3] = q.w;
    } else if constexpr (C == 2) {
      const float2 q = __ldg(reinterpret_cast<const float2*>(row + gx));
      v[0] = q.x;
      v[1] = q.y;
    } else {
      v[0] = __ldg(row + gx);
    }
  } else {
#pragma unroll
    for (int j = 0; j < C; ++j) v[j] = __ldg(row + wrap_index(gx + j, nx));
  }
}

// Store a lane's C values; xout (the same in every lane of the warp): every storing lane's
// columns lie inside the row, else each column is stored only if it does.
template <int C>
__device__ __forceinline__ void store_lane(float* row, int gx, int nx, bool xout,
                                           const float (&v)[C]) {
  if (xout) {
    if constexpr (C == 4) {
      *reinterpret_cast<float4*>(row + gx) = make_float4(v[0], v[1], v[2], v[3]);
    } else if constexpr (C == 2) {
      *reinterpret_cast<float2*>(row + gx) = make_float2(v[0], v[1]);
    } else {
      row[gx] = v[0];
    }
  } else {
#pragma unroll
    for (int j = 0; j < C; ++j)
      if (gx + j < nx) row[gx + j] = v[j];
  }
}

// Packed FP32 pairs (one instruction updates two sites, each lane's result the scalar
// operation's bits; the *4 helpers of pf_model.cuh). A packed pair issues to the heavy FMA pipe
// only, so packing everything can be slower than scalar code that spreads over both pipes;
// the choices below are the measured ones. Laplacian sums (kStripPackedLap): packed for 2 and
// 4 columns a lane except Gray-Scott with 128-column strips (787 -> 775 GLUPS at 4096^2);
// Model B 8192^2 823 -> 858, Model C 4096^2 383 -> 388, Allen-Cahn with 64-column strips 1296
// -> 1307. Updates (kStripPacked): Gray-Scott with 64-column strips (Gray-Scott 4096^2: 808 ->
// 879 GLUPS) and Allen-Cahn with 128-column strips (Allen-Cahn 4096^2: 1340 -> 1483);
// Gray-Scott with 128-column strips measured slower with them (791 -> 731), Allen-Cahn with
// 64-column strips the same.
template <int MODEL, int C>
constexpr bool kStripPacked = (MODEL == PF_MODEL_GS && C == 2) || (MODEL == PF_MODEL_AC && C == 4);
template <int MODEL, int C>
constexpr bool kStripPackedLap = (C == 2 || C == 4) && !(MODEL == PF_MODEL_GS && C == 4);

// Laplacians of a lane's C sites from the rows above (u), at (c) and below (d); the x
// neighbours beyond the lane come from the adjacent lanes. ST: PF_ST_STD (5-point) or
// PF_ST_ISO (9-point, lap2d_iso with the tile body's operands in its order: the axial
// neighbours, then up-left, up-right, down-left, down-right).
template <int MODEL, int C, int ST>
__device__ __forceinline__ void lap_lane(const float (&u)[C], const float (&c)[C],
                                         const float (&d)[C], float scale, float (&l)[C]) {
  static_assert(ST == PF_ST_STD || ST == PF_ST_ISO, "radius-1 stencils only");
  const float xl = __shfl_up_sync(0xffffffffu, c[C - 1], 1);
  const float xr = __shfl_down_sync(0xffffffffu, c[0], 1);
  if constexpr (ST == PF_ST_ISO) {
    const float ul = __shfl_up_sync(0xffffffffu, u[C - 1], 1);
    const float ur = __shfl_down_sync(0xffffffffu, u[0], 1);
    const float dl = __shfl_up_sync(0xffffffffu, d[C - 1], 1);
    const float dr = __shfl_down_sync(0xffffffffu, d[0], 1);
#pragma unroll
    for (int j = 0; j < C; ++j) {
      const float left = j == 0 ? xl : c[j - 1];
      const float right = j == C - 1 ? xr : c[j + 1];
      const float up_l = j == 0 ? ul : u[j - 1];
      const float up_r = j == C - 1 ? ur : u[j + 1];
      const float dn_l = j == 0 ? dl : d[j - 1];
      const float dn_r = j == C - 1 ? dr : d[j + 1];
      l[j] = lap2d_iso(c[j], left, right, u[j], d[j], up_l, up_r, dn_l, dn_r, scale);
    }
  } else if constexpr (kStripPackedLap<MODEL, C> && C == 4) {
    float4 r = lap2d_sum4(make_float4(c[0], c[1], c[2], c[3]), xl, xr,
                          make_float4(u[0], u[1], u[2], u[3]),
                          make_float4(d[0], d[1], d[2], d[3]));
    if constexpr (MODEL != PF_MODEL_GS) r = mul4(scale, r);
    l[0] = r.x;
    l[1] = r.y;
    l[2] = r.z;
    l[3] = r.w;
  } else if constexpr (kStripPackedLap<MODEL, C> && C == 2) {
    // lap2d_sum of two sites: (xm + xp) + (ym + yp), then -4 c + that
    const float2 sx = make_float2(__fadd_rn(xl, c[1]), __fadd_rn(c[0], xr));
    const float2 sy = __fadd2_rn(make_float2(u[0], u[1]), make_float2(d[0], d[1]));
    float2 r = __ffma2_rn(make_float2(-4.0f, -4.0f), make_float2(c[0], c[1]), __fadd2_rn(sx, sy));
    if constexpr (MODEL != PF_MODEL_GS) r = __fmul2_rn(make_float2(scale, scale), r);
    l[0] = r.x;
    l[1] = r.y;
  } else {
#pragma unroll
    for (int j = 0; j < C; ++j) {
      const float left = j == 0 ? xl : c[j - 1];
      const float right = j == C - 1 ? xr : c[j + 1];
      l[j] = lap_scaled<MODEL>(lap2d_sum(c[j], left, right, u[j], d[j]), scale);
    }
  }
}

template <int MODEL, int K, int C, int ST = PF_ST_STD>
struct StripRun {
  static_assert(ST == PF_ST_STD || ModelTraits<MODEL>::R == 1,
                "the 9-point stencil runs on the radius-1 models");
  using S = StripCfg<MODEL, K, C>;
  static constexpr int NF = S::NF;
  static constexpr int R = S::R;
  static constexpr int NM = S::NM;
  float w[K][NF][3][C];                     // state of level s = 0..K-1
  float mw[R == 2 ? K : 1][NM][3][C];       // radius 2: mu (and lap psi) of level s's state

  // the task
  FieldPtrs in;
  FieldOut out;
  int nx, ny, y0, hy, gx;
  int64_t pitch;
  bool st_lane, xin, xout;

  // Level s (1..K) at an iteration of phase P; its new row goes to o.
  template <int P, int s>
  __device__ __forceinline__ void level(const ModelParams& m, float (&o)[NF][C]) {
    constexpr int su = P, sc = (P + 1) % 3, sd = (P + 2) % 3;
    if constexpr (MODEL == PF_MODEL_AC) {
      float l[C];
      lap_lane<MODEL, C, ST>(w[s - 1][0][su], w[s - 1][0][sc], w[s - 1][0][sd], m.lap_scale, l);
      if constexpr (kStripPacked<MODEL, C> && C == 4) {
        const float(&p)[C] = w[s - 1][0][sc];
        const float4 r = ac_update4(make_float4(p[0], p[1], p[2], p[3]),
                                    make_float4(l[0], l[1], l[2], l[3]), m);
        o[0][0] = r.x;
        o[0][1] = r.y;
        o[0][2] = r.z;
        o[0][3] = r.w;
      } else {
#pragma unroll
        for (int j = 0; j < C; ++j) o[0][j] = ac_update(w[s - 1][0][sc][j], l[j], m);
      }
    } else if constexpr (MODEL == PF_MODEL_GS) {
      float lu[C], lv[C];
      lap_lane<MODEL, C, ST>(w[s - 1][0][su], w[s - 1][0][sc], w[s - 1][0][sd], m.lap_scale, lu);
      lap_lane<MODEL, C, ST>(w[s - 1][1][su], w[s - 1][1][sc], w[s - 1][1][sd], m.lap_scale, lv);
      if constexpr (kStripPacked<MODEL, C> && C == 2) {
        // the pair twice over in a float4 (gs_update4), the copy discarded
        const float(&u)[C] = w[s - 1][0][sc];
        const float(&v)[C] = w[s - 1][1][sc];
        float4 un, vn;
        gs_update4(make_float4(u[0], u[1], u[0], u[1]), make_float4(v[0], v[1], v[0], v[1]),
                   make_float4(lu[0], lu[1], lu[0], lu[1]), make_float4(lv[0], lv[1], lv[0], lv[1]),
                   m, un, vn);
        o[0][0] = un.x;
        o[0][1] = un.y;
        o[1][0] = vn.x;
        o[1][1] = vn.y;
      } else {
#pragma unroll
        for (int j = 0; j < C; ++j)
          gs_update(w[s - 1][0][sc][j], w[s - 1][1][sc][j], lu[j], lv[j], m, o[0][j], o[1][j]);
      }
    } else {
      // chemical potential (Model C: and lap psi) of level s - 1's centre row, into slot P
      float(&mu)[3][C] = mw[s - 1][0];
      if constexpr (MODEL == PF_MODEL_CH) {
        float l[C];
        lap_lane<MODEL, C, ST>(w[s - 1][0][su], w[s - 1][0][sc], w[s - 1][0][sd], m.lap_scale, l);
#pragma unroll
        for (int j = 0; j < C; ++j) mu[P][j] = ch_mu(w[s - 1][0][sc][j], l[j], m);
      } else {
        float lm[C];
        lap_lane<MODEL, C, ST>(w[s - 1][1][su], w[s - 1][1][sc], w[s - 1][1][sd], m.lap_scale, lm);
        lap_lane<MODEL, C, ST>(w[s - 1][0][su], w[s - 1][0][sc], w[s - 1][0][sd], m.lap_scale,
                           mw[s - 1][1][P]);
#pragma unroll
        for (int j = 0; j < C; ++j)
          mu[P][j] = mc_mu(w[s - 1][0][sc][j], w[s - 1][1][sc][j], lm[j], m);
      }
      // the row one above: its mu rows sit in slots P + 1, P + 2, P, its state in level
      // s - 1's oldest slot P, and (Model C) its lap psi in slot P + 2
      float lmu[C];
      lap_lane<MODEL, C, ST>(mu[sc], mu[sd], mu[su], m.lap_scale, lmu);
      if constexpr (MODEL == PF_MODEL_CH) {
#pragma unroll
        for (int j = 0; j < C; ++j) o[0][j] = ch_update(w[s - 1][0][su][j], lmu[j], m);
      } else {
#pragma unroll
        for (int j = 0; j < C; ++j)
          mc_update(w[s - 1][0][su][j], w[s - 1][1][su][j], mw[s - 1][1][sd][j], lmu[j], m,
                    o[0][j], o[1][j]);
      }
    }
  }

  // Iterations in which level s runs: [lo(s), hi(s)). Radius 1: level s is valid from
  // t = 3 s, and the output needs it until t = hy + 2 K + s - 1. Radius 2: its chemical
  // potential is valid from t = 5 s - 2, its state from 5 s, and the output needs it until
  // t = hy + 4 K + s - 1.
  static __device__ __forceinline__ int lo(int s) { return R == 1 ? 3 * s : 5 * s - 2; }
  __device__ __forceinline__ int hi(int s) const { return hy + 2 * R * K + s; }
  __device__ __forceinline__ int rows_in() const { return hy + 2 * R * K; }

  // Levels K-1 .. 1 at an iteration t of phase P (with G, levels outside their range are
  // skipped; without, every level is known to be in range).
  template <int P, bool G, int s>
  __device__ __forceinline__ void inner_levels(int t, const ModelParams& m) {
    if constexpr (s >= 1) {
      if (!G || (unsigned)(t - lo(s)) < (unsigned)(hi(s) - lo(s))) {
        float o[NF][C];
        level<P, s>(m, o);
#pragma unroll
        for (int f = 0; f < NF; ++f)
#pragma unroll
          for (int j = 0; j < C; ++j) w[s][f][P][j] = o[f][j];
      }
      inner_levels<P, G, s - 1>(t, m);
    }
  }

  // First iteration that stores an output row (every level runs from here until the input
  // rows end).
  static constexpr int T0 = (2 * R + 1) * K;

  template <int P, bool G>
  __device__ __forceinline__ void iteration(int t, const ModelParams& m) {
    // level K: output row y0 + t - T0 (radius 2: its chemical potential starts two
    // iterations before the first output row)
    if (!G || (unsigned)(t - lo(K)) < (unsigned)(T0 + hy - lo(K))) {
      float o[NF][C];
      level<P, K>(m, o);
      if (st_lane && (!G || t >= T0)) {
        const int64_t row = (int64_t)(y0 + t - T0) * pitch;
#pragma unroll
        for (int f = 0; f < NF; ++f) store_lane<C>(out.f[f] + row, gx, nx, xout, o[f]);
      }
    }
    inner_levels<P, G, K - 1>(t, m);
    // level 0: input row ys + t, first read in the next iteration
    if (!G || t < rows_in()) {
      const int64_t row = (int64_t)wrap_index(y0 - R * K + t, ny) * pitch;
#pragma unroll
      for (int f = 0; f < NF; ++f) load_lane<C>(in.f[f] + row, gx, nx, xin, w[0][f][P]);
    }
  }

  // Output rows [y0, y0 + hy) and columns [x0, x0 + wo) of the strip whose output columns
  // start at x0 (wo <= WO, a multiple of C unless the strip ends at the row's end).
  __device__ __forceinline__ void run(const FieldPtrs& in_, const FieldOut& out_, int nx_,
                                      int ny_, int64_t pitch_, int x0, int wo, int y0_, int hy_,
                                      const ModelParams& m) {
    in = in_;
    out = out_;
    nx = nx_;
    ny = ny_;
    pitch = pitch_;
    y0 = y0_;
    hy = hy_;
    const int lane = threadIdx.x & 31;
    gx = x0 - S::HXP + C * lane;
    st_lane = lane >= S::HXP / C && lane < (S::HXP + wo + C - 1) / C;
    // strips that reach past either end of the row (every strip of a narrow grid or batch
    // instance) take the periodic paths with the whole warp
    xin = __all_sync(0xffffffffu, gx >= 0 && gx + C <= nx);
    xout = __all_sync(0xffffffffu, !st_lane || gx + C <= nx);
    const int t_main = rows_in();  // the input rows end here
    int t = 0;
    for (; t < T0; t += 3) {  // start-up: levels begin one after another
      iteration<0, true>(t, m);
      iteration<1, true>(t + 1, m);
      iteration<2, true>(t + 2, m);
    }
    for (; t + 3 <= t_main; t += 3) {  // steady state: every level, no range checks
      iteration<0, false>(t, m);
      iteration<1, false>(t + 1, m);
      iteration<2, false>(t + 2, m);
    }
    for (; t < T0 + hy; t += 3) {  // drain: levels finish one after another
      iteration<0, true>(t, m);
      iteration<1, true>(t + 1, m);
      iteration<2, true>(t + 2, m);
    }
  }
};

// One warp per task: strips of WO output columns by rows of hy (the last row of tasks is
// shorter); consecutive warps take neighbouring strips of the same rows.
template <int MODEL, int K, int C, int ST>
__global__ void __launch_bounds__(kStripThreads, (StripCfg<MODEL, K, C>::MINW / kStripWarps))
    fe2d_strip_kernel(FieldPtrs in, FieldOut out, Geom g, ModelParams m, int hy, int tasks_x,
                      int ntasks) {
  using S = StripCfg<MODEL, K, C>;
  const int task = blockIdx.x * kStripWarps + (threadIdx.x >> 5);
  if (task >= ntasks) return;  // the whole warp
  const int ty = task / tasks_x;
  const int tx = task - ty * tasks_x;
  const int y0 = ty * hy;
  StripRun<MODEL, K, C, ST> r;
  r.run(in, out, g.nx, g.ny, g.pitch, tx * S::WO, S::WO, y0, min(hy, g.ny - y0), m);
}

// Batched Gray-Scott: warp w runs strip task w of the list, a strip of 32 C columns whose
// output width the task gives (every instance's width is split evenly over its strips).
template <int K, int C>
__global__ void __launch_bounds__(kStripThreads, (StripCfg<PF_MODEL_GS, K, C>::MINW / kStripWarps))
    batch_gs2d_strip_kernel(const BatchInst* __restrict__ insts,
                            const BatchStrip* __restrict__ tasks, int ntasks,
                            const float* in_base, float* out_base) {
  const int task = blockIdx.x * kStripWarps + (threadIdx.x >> 5);
  if (task >= ntasks) return;  // the whole warp
  const BatchStrip t = tasks[task];
  const BatchInst I = insts[t.inst];
  const int64_t plane = I.pitch * I.ny;
  FieldPtrs in{};
  FieldOut out{};
  in.f[0] = in_base + I.off;
  in.f[1] = in_base + I.off + plane;
  out.f[0] = out_base + I.off;
  out.f[1] = out_base + I.off + plane;
  StripRun<PF_MODEL_GS, K, C> r;
  r.run(in, out, I.nx, I.ny, I.pitch, t.x0, t.wo, t.y0, t.hy, I.m);
}

// Rows per task. A task's first and last rows carry the levels' start-up and drain, which
// argues for long tasks, and every warp slot should stay busy: so as many tasks as the
// device holds warps at once (one wave, rows split evenly), unless that makes them shorter
// than min_rows; then tasks of min_rows rows in several waves.
int strip_rows(int tasks_x, int ny, int resident_warps, int min_rows) {
  const int per_col = resident_warps / tasks_x;
  if (per_col >= 1) {
    const int hy = (ny + per_col - 1) / per_col;
    if (hy >= min_rows || hy >= ny) return hy;
  }
  return min_rows < ny ? min_rows : ny;
}

template <int MODEL, int K, int C, int ST>
cudaError_t launch_strip(const Geom& g, FieldPtrs in, FieldOut out, const ModelParams& m,
                         cudaStream_t s) {
  using S = StripCfg<MODEL, K, C>;
  using Run = StripRun<MODEL, K, C, ST>;
  static int resident[64] = {};  // resident warps of this kernel on the whole device
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 64) return cudaErrorInvalidDevice;
  if (resident[dev] == 0) {
    int b = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fe2d_strip_kernel<MODEL, K, C, ST>,
                                                      kStripThreads, 0);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    resident[dev] = (b > 0 ? b : 1) * (sms > 0 ? sms : 1) * kStripWarps;
  }
  const int tasks_x = (g.nx + S::WO - 1) / S::WO;
  const int hy = strip_rows(tasks_x, g.ny, resident[dev], 4 * Run::T0);
  const int ntasks = tasks_x * ((g.ny + hy - 1) / hy);
  const int blocks = (ntasks + kStripWarps - 1) / kStripWarps;
  fe2d_strip_kernel<MODEL, K, C, ST><<<blocks, kStripThreads, 0, s>>>(in, out, g, m, hy,
                                                                      tasks_x, ntasks);
  return cudaGetLastError();
}

template <int MODEL, int C, int ST>
cudaError_t launch_strip_k(int k, const Geom& g, FieldPtrs in, FieldOut out,
                           const ModelParams& m, cudaStream_t s) {
  if (k == 1) return launch_strip<MODEL, 1, C, ST>(g, in, out, m, s);
  if (k == 2) return launch_strip<MODEL, 2, C, ST>(g, in, out, m, s);
  if constexpr (ModelTraits<MODEL>::R == 1) {
    if (k == 4) return launch_strip<MODEL, 4, C, ST>(g, in, out, m, s);
  }
  return cudaErrorInvalidValue;
}

template <int MODEL, int ST = PF_ST_STD>
cudaError_t launch_strip_c(int lanes_cols, int k, const Geom& g, FieldPtrs in, FieldOut out,
                           const ModelParams& m, cudaStream_t s) {
  if (lanes_cols == 128) return launch_strip_k<MODEL, 4, ST>(k, g, in, out, m, s);
  if (lanes_cols == 64) return launch_strip_k<MODEL, 2, ST>(k, g, in, out, m, s);
  return cudaErrorInvalidValue;
}

template <int K, int C>
cudaError_t launch_batch_k(const BatchInst* d_insts, const BatchStrip* d_tasks, int ntasks,
                           const float* in_base, float* out_base, cudaStream_t s) {
  const int blocks = (ntasks + kStripWarps - 1) / kStripWarps;
  batch_gs2d_strip_kernel<K, C><<<blocks, kStripThreads, 0, s>>>(d_insts, d_tasks, ntasks,
                                                                 in_base, out_base);
  return cudaGetLastError();
}

template <int K, int C>
int batch_resident_kc() {
  int b = 0, sms = 0, dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, batch_gs2d_strip_kernel<K, C>,
                                                      kStripThreads, 0);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return (b > 0 ? b : 1) * (sms > 0 ? sms : 1) * kStripWarps;
}

template <int MODEL, int K>
int out_cols_k(int c) {
  if (c == 4) return StripCfg<MODEL, K, 4>::WO;
  if (c == 2) return StripCfg<MODEL, K, 2>::WO;
  return StripCfg<MODEL, K, 1>::WO;
}

}  // namespace

int strip_out_cols(int model, int k, int c) {
  const bool r2 = model == PF_MODEL_CH || model == PF_MODEL_C;
  if (k == 1) return r2 ? out_cols_k<PF_MODEL_CH, 1>(c) : out_cols_k<PF_MODEL_AC, 1>(c);
  if (k == 2) return r2 ? out_cols_k<PF_MODEL_CH, 2>(c) : out_cols_k<PF_MODEL_AC, 2>(c);
  if (k == 4 && !r2) return out_cols_k<PF_MODEL_AC, 4>(c);
  return 0;
}

// The shortest batch task considered: twice the levels' start-up.
int strip_task_rows(int model, int k) {
  const int r = (model == PF_MODEL_CH || model == PF_MODEL_C) ? 2 : 1;
  return 2 * (2 * r + 1) * k;
}

int batch_gs2d_strips_resident(int k, int c) {
  static int resident[2][3][64] = {};  // c = 4, 2; k = 1, 2, 4; per device
  const int ci = c == 2 ? 1 : 0, ki = k == 4 ? 2 : k == 2 ? 1 : 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev >= 64) {
    cudaGetLastError();
    return 1;
  }
  int& r = resident[ci][ki][dev];
  if (r == 0) {
    if (c == 2)
      r = k == 4 ? batch_resident_kc<4, 2>() : k == 2 ? batch_resident_kc<2, 2>()
                                                      : batch_resident_kc<1, 2>();
    else
      r = k == 4 ? batch_resident_kc<4, 4>() : k == 2 ? batch_resident_kc<2, 4>()
                                                      : batch_resident_kc<1, 4>();
    if (r == 0) return 1;  // not cached: asked again next time
  }
  return r;
}

cudaError_t launch_batch_gs2d_strips(int c, int k, const BatchInst* d_insts,
                                     const BatchStrip* d_tasks, int ntasks, const float* in_base,
                                     float* out_base, cudaStream_t s) {
  if (ntasks <= 0) return cudaSuccess;
  if (c == 4) {
    if (k == 1) return launch_batch_k<1, 4>(d_insts, d_tasks, ntasks, in_base, out_base, s);
    if (k == 2) return launch_batch_k<2, 4>(d_insts, d_tasks, ntasks, in_base, out_base, s);
    if (k == 4) return launch_batch_k<4, 4>(d_insts, d_tasks, ntasks, in_base, out_base, s);
  } else if (c == 2) {
    if (k == 1) return launch_batch_k<1, 2>(d_insts, d_tasks, ntasks, in_base, out_base, s);
    if (k == 2) return launch_batch_k<2, 2>(d_insts, d_tasks, ntasks, in_base, out_base, s);
    if (k == 4) return launch_batch_k<4, 2>(d_insts, d_tasks, ntasks, in_base, out_base, s);
  }
  return cudaErrorInvalidValue;
}

bool fe2d_strips_supported(int model, int k, int stencil) {
  if (stencil == PF_ST_ISO) return (model == PF_MODEL_AC || model == PF_MODEL_GS) &&
                                   (k == 1 || k == 2 || k == 4);
  if (stencil != PF_ST_STD) return false;
  if (model == PF_MODEL_AC || model == PF_MODEL_GS) return k == 1 || k == 2 || k == 4;
  if (model == PF_MODEL_CH || model == PF_MODEL_C) return k == 1 || k == 2;
  return false;
}

cudaError_t launch_fe2d_strips(int model, int stencil, int lanes_cols, int k, const Geom& g,
                               FieldPtrs in, FieldOut out, const ModelParams& m, cudaStream_t s) {
  if (!fe2d_strips_supported(model, k, stencil)) return cudaErrorInvalidValue;
  if (stencil == PF_ST_ISO) {
    if (model == PF_MODEL_AC)
      return launch_strip_c<PF_MODEL_AC, PF_ST_ISO>(lanes_cols, k, g, in, out, m, s);
    return launch_strip_c<PF_MODEL_GS, PF_ST_ISO>(lanes_cols, k, g, in, out, m, s);
  }
  switch (model) {
    case PF_MODEL_AC: return launch_strip_c<PF_MODEL_AC>(lanes_cols, k, g, in, out, m, s);
    case PF_MODEL_GS: return launch_strip_c<PF_MODEL_GS>(lanes_cols, k, g, in, out, m, s);
    case PF_MODEL_CH: return launch_strip_c<PF_MODEL_CH>(lanes_cols, k, g, in, out, m, s);
    case PF_MODEL_C: return launch_strip_c<PF_MODEL_C>(lanes_cols, k, g, in, out, m, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace pf
