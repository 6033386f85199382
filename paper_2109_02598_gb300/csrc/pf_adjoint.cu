// Discrete adjoint of the forward-Euler Gray-Scott time loop with sqrt(N) checkpointing.
//
// Forward map (Sec. 2.4.1 solver; Gray-Scott in its standard form, Sec. 1):
//   x^{n+1} = x^n + dt f(x^n; theta),  theta = (Du, Dv, F, k).
// For a loss L(x^N) with lambda^N = dL/dx^N, reverse-mode differentiation of the loop gives
//   lambda^n = lambda^{n+1} + dt J(x^n)^T lambda^{n+1},
//   dL/dtheta = sum_n dt (df/dtheta)(x^n)^T lambda^{n+1},   dL/dx^0 = lambda^0.
// With (u, v) = x^n and (a, b) = lambda^{n+1}, and the periodic Laplacian symmetric:
//   a' = a + dt [Du lap a - (v^2 + F) a + v^2 b]
//   b' = b + dt [Dv lap b - 2uv a + (2uv - F - k) b]
//   dL/dDu += dt sum a lap u,  dL/dDv += dt sum b lap v,
//   dL/dF  += dt sum [(1 - u) a - v b],  dL/dk += -dt sum v b.
//
// Model A (x' = x + dt (lap x + c1 x - c2 x^3)) and Model B (x' = x + dt M lap mu(x),
// mu = c2 x^3 - c1 x - lap x) take the same loop with their own reverse steps:
//   A: lambda^n = lambda + dt [lap lambda + (c1 - 3 c2 x^2) lambda];
//      sums S = (sum lambda x, sum lambda x^3), dL/d(c1, c2) = dt (S0, -S1).
//   B: w = lap lambda, lambda^n = lambda + dt M [(3 c2 x^2 - c1) w - lap w];
//      sums S = (sum w x, sum w x^3, sum w mu), dL/d(c1, c2, M) = dt (-M S0, M S1, S2).
//
// Memory/recompute: the forward pass stores x at every C-th step (C ~ sqrt(N)); the
// backward pass walks the segments from last to first, recomputes the segment's states
// from its checkpoint with the forward kernel, then runs the segment's adjoint steps.
// Parameter-gradient partials are summed per CTA in FP64 (each CTA owns one slot, so the
// order is fixed and the result deterministic) and added up in a fixed order at the end.
#include <cmath>
#include <vector>

#include "pf_fe2d_tile.cuh"
#include "pf_grid.h"
#include "pf_internal.h"

namespace pf {

namespace {

constexpr int kATX = 64, kATY = 16;  // adjoint tile
constexpr int kAW = kATX + 2, kAH = kATY + 2, kAPL = kAW * kAH;

// Warp sum of per-thread float partials, in float (a fixed tree, so the same bits on every
// run), widened to double for the per-warp and per-CTA sums. FP64 arithmetic is a small
// fraction of FP32 throughput on this GPU: a double-precision shuffle tree in every CTA of
// every reverse step took most of the kernel's time.
__device__ __forceinline__ double warp_sum_f(double v) {
  float f = (float)v;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) f = __fadd_rn(f, __shfl_down_sync(0xffffffffu, f, o));
  return (double)f;
}

// Double-precision warp sum, for the final fixed-order sum over the CTAs' slots (once per
// reverse pass).
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// One reverse step on a 64 x TY tile: stage u, v (the state x^n) and a, b (lambda^{n+1})
// with a periodic halo of 1 as aligned float4 groups (the forward tile body's staging), then
// four sites per thread: update (a, b) and add the parameter-gradient terms to per-thread
// sums, which go to this tile's FP64 slot in a fixed order.
// TY = 8 on grids too small to give every SM several 16-row tiles (more CTAs in flight hide
// the L2 latency of the staging: 512^2 reverse step 8.4 -> 7.6 us), else 16 (2048^2: 49.5 us
// with 16 rows, 58.8 with 8).
template <int TY>
__global__ void __launch_bounds__(kNT2) adj_gs2d_kernel(FieldPtrs x, FieldPtrs lam,
                                                        FieldOut lam_out, Geom g,
                                                        ModelParams m, double* gpart) {
  using AdjCfg = Cfg2<PF_MODEL_GS, 1, kATX, TY>;
  constexpr int WS = AdjCfg::WS, PL = AdjCfg::PL, HP = AdjCfg::HP, H = AdjCfg::H;
  __shared__ __align__(16) float sm[4 * PL];  // u, v, a, b
  __shared__ double red[4][kNT2 / 32];
  const int x0 = blockIdx.x * kATX;
  const int y0 = blockIdx.y * TY;
  canary_fill(sm, 4 * PL);
  load_region2d<AdjCfg, false>(x, g.nx, g.ny, g.pitch, x0, y0, sm);  // waits with the next
  load_region2d<AdjCfg>(lam, g.nx, g.ny, g.pitch, x0, y0, sm + 2 * PL);
  __syncthreads();
  const float* su = sm;
  const float* sv = sm + PL;
  const float* sa = sm + 2 * PL;
  const float* sb = sm + 3 * PL;
  float pDu = 0.f, pDv = 0.f, pF = 0.f, pk = 0.f;
  constexpr int NG = kATX / 4;  // float4 groups per tile row
  for (int i = threadIdx.x; i < TY * NG; i += kNT2) {
    const int rr = i / NG, j = i - rr * NG;
    const int gy = y0 + rr;
    const int gx = x0 + 4 * j;
    if (gy >= g.ny || gx >= g.nx) continue;
    const int p = (rr + H) * WS + HP + 4 * j;
    const float4 u4 = *reinterpret_cast<const float4*>(su + p);
    const float4 v4 = *reinterpret_cast<const float4*>(sv + p);
    const float4 a4 = *reinterpret_cast<const float4*>(sa + p);
    const float4 b4 = *reinterpret_cast<const float4*>(sb + p);
    const float4 la4 = lap2d_x4(sa, p, WS, m.lap_scale);
    const float4 lb4 = lap2d_x4(sb, p, WS, m.lap_scale);
    const float4 lu4 = lap2d_x4(su, p, WS, m.lap_scale);
    const float4 lv4 = lap2d_x4(sv, p, WS, m.lap_scale);
    const float uu[4] = {u4.x, u4.y, u4.z, u4.w}, vv_[4] = {v4.x, v4.y, v4.z, v4.w};
    const float aa[4] = {a4.x, a4.y, a4.z, a4.w}, bb[4] = {b4.x, b4.y, b4.z, b4.w};
    const float la[4] = {la4.x, la4.y, la4.z, la4.w}, lb[4] = {lb4.x, lb4.y, lb4.z, lb4.w};
    const float lu[4] = {lu4.x, lu4.y, lu4.z, lu4.w}, lv[4] = {lv4.x, lv4.y, lv4.z, lv4.w};
    float na[4], nb[4];
    const int nvalid = g.nx - gx < 4 ? g.nx - gx : 4;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float u = uu[e], v = vv_[e], a = aa[e], b = bb[e];
      const float vv = __fmul_rn(v, v);
      const float uv2 = __fmul_rn(2.0f, __fmul_rn(u, v));
      // a' = a + dt [Du la - (v^2 + F) a + v^2 b]
      float fa = __fmaf_rn(-__fadd_rn(vv, m.a2), a, __fmul_rn(vv, b));
      fa = __fmaf_rn(m.a0, la[e], fa);
      // b' = b + dt [Dv lb - 2uv a + (2uv - F - k) b]
      float fb = __fmaf_rn(__fsub_rn(uv2, m.a3), b, -__fmul_rn(uv2, a));
      fb = __fmaf_rn(m.a1, lb[e], fb);
      na[e] = __fmaf_rn(m.dt, fa, a);
      nb[e] = __fmaf_rn(m.dt, fb, b);
      if (e < nvalid) {
        pDu = __fmaf_rn(a, lu[e], pDu);
        pDv = __fmaf_rn(b, lv[e], pDv);
        pF = __fadd_rn(pF, __fsub_rn(__fmul_rn(__fsub_rn(1.0f, u), a), __fmul_rn(v, b)));
        pk = __fsub_rn(pk, __fmul_rn(v, b));
      }
    }
    const int64_t off = (int64_t)gy * g.pitch + gx;
    if (nvalid == 4) {
      *reinterpret_cast<float4*>(lam_out.f[0] + off) = make_float4(na[0], na[1], na[2], na[3]);
      *reinterpret_cast<float4*>(lam_out.f[1] + off) = make_float4(nb[0], nb[1], nb[2], nb[3]);
    } else {
      for (int e = 0; e < nvalid; ++e) {
        lam_out.f[0][off + e] = na[e];
        lam_out.f[1][off + e] = nb[e];
      }
    }
  }
  double t[4] = {pDu, pDv, pF, pk};
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    t[q] = warp_sum_f(t[q]);
    if (lane == 0) red[q][wid] = t[q];
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double s = 0.0;
    for (int w = 0; w < kNT2 / 32; ++w) s += red[threadIdx.x][w];
    double* slot = gpart + 4 * ((int64_t)blockIdx.y * gridDim.x + blockIdx.x);
    slot[threadIdx.x] += s;
  }
}

// Add this CTA's per-thread sums t[0..NG) into its FP64 slot (fixed order).
template <int NG>
__device__ __forceinline__ void add_to_slot(double (&t)[4], double (&red)[4][kNT2 / 32],
                                            double* gpart) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NG; ++q) {
    t[q] = warp_sum_f(t[q]);
    if (lane == 0) red[q][wid] = t[q];
  }
  __syncthreads();
  if (threadIdx.x < NG) {
    double s = 0.0;
    for (int w = 0; w < kNT2 / 32; ++w) s += red[threadIdx.x][w];
    gpart[4 * ((int64_t)blockIdx.y * gridDim.x + blockIdx.x) + threadIdx.x] += s;
  }
}

// Model A reverse step on a tile (halo 1 of x = phi^n and lambda^{n+1}).
__global__ void __launch_bounds__(kNT2) adj_ac2d_kernel(FieldPtrs x, FieldPtrs lam,
                                                        FieldOut lam_out, Geom g,
                                                        ModelParams m, double* gpart) {
  __shared__ float sp[kAPL], sl[kAPL];
  __shared__ double red[4][kNT2 / 32];
  const int x0 = blockIdx.x * kATX;
  const int y0 = blockIdx.y * kATY;
  canary_fill(sp, kAPL);
  canary_fill(sl, kAPL);
  for (int i = threadIdx.x; i < kAPL; i += kNT2) {
    const int r = i / kAW;
    const int c = i - r * kAW;
    const int64_t off =
        (int64_t)wrap_index(y0 - 1 + r, g.ny) * g.pitch + wrap_index(x0 - 1 + c, g.nx);
    cp_async4(&sp[i], x.f[0] + off);
    cp_async4(&sl[i], lam.f[0] + off);
  }
  cp_async_wait_all();
  __syncthreads();
  const float c2x3 = __fmul_rn(3.0f, m.a1);
  float s0 = 0.f, s1 = 0.f;
  for (int i = threadIdx.x; i < kATX * kATY; i += kNT2) {
    const int rr = i / kATX;
    const int cc = i - rr * kATX;
    const int gx = x0 + cc, gy = y0 + rr;
    if (gx >= g.nx || gy >= g.ny) continue;
    const int p = (rr + 1) * kAW + (cc + 1);
    const float ph = sp[p], l = sl[p];
    const float ll = lap2d(l, sl[p - 1], sl[p + 1], sl[p - kAW], sl[p + kAW], m.lap_scale);
    const float sfac = __fmaf_rn(-c2x3, __fmul_rn(ph, ph), m.a0);  // c1 - 3 c2 phi^2
    const float f = __fmaf_rn(sfac, l, ll);
    lam_out.f[0][(int64_t)gy * g.pitch + gx] = __fmaf_rn(m.dt, f, l);
    const float lp = __fmul_rn(l, ph);
    s0 = __fadd_rn(s0, lp);
    s1 = __fmaf_rn(lp, __fmul_rn(ph, ph), s1);
  }
  double t[4] = {s0, s1, 0.0, 0.0};
  add_to_slot<2>(t, red, gpart);
}

// Model B reverse step on a tile: stage phi^n and lambda^{n+1} with a halo of 2, form
// w = lap lambda on the tile plus one ring, then lambda^n on the tile.
constexpr int kBW = kATX + 4, kBH = kATY + 4, kBPL = kBW * kBH;
__global__ void __launch_bounds__(kNT2) adj_ch2d_kernel(FieldPtrs x, FieldPtrs lam,
                                                        FieldOut lam_out, Geom g,
                                                        ModelParams m, double* gpart) {
  __shared__ float sp[kBPL], sl[kBPL], sw[kBPL];
  __shared__ double red[4][kNT2 / 32];
  const int x0 = blockIdx.x * kATX;
  const int y0 = blockIdx.y * kATY;
  canary_fill(sp, kBPL);
  canary_fill(sl, kBPL);
  canary_fill(sw, kBPL);
  for (int i = threadIdx.x; i < kBPL; i += kNT2) {
    const int r = i / kBW;
    const int c = i - r * kBW;
    const int64_t off =
        (int64_t)wrap_index(y0 - 2 + r, g.ny) * g.pitch + wrap_index(x0 - 2 + c, g.nx);
    cp_async4(&sp[i], x.f[0] + off);
    cp_async4(&sl[i], lam.f[0] + off);
  }
  cp_async_wait_all();
  __syncthreads();
  // w on rows/cols 1 .. kBH-2 / kBW-2 (the tile and one ring)
  for (int i = threadIdx.x; i < (kATX + 2) * (kATY + 2); i += kNT2) {
    const int r = 1 + i / (kATX + 2);
    const int c = 1 + i % (kATX + 2);
    const int p = r * kBW + c;
    sw[p] = lap2d(sl[p], sl[p - 1], sl[p + 1], sl[p - kBW], sl[p + kBW], m.lap_scale);
  }
  __syncthreads();
  const float c2x3 = __fmul_rn(3.0f, m.a1);
  float s0 = 0.f, s1 = 0.f, s2 = 0.f;
  for (int i = threadIdx.x; i < kATX * kATY; i += kNT2) {
    const int rr = i / kATX;
    const int cc = i - rr * kATX;
    const int gx = x0 + cc, gy = y0 + rr;
    if (gx >= g.nx || gy >= g.ny) continue;
    const int p = (rr + 2) * kBW + (cc + 2);
    const float ph = sp[p], l = sl[p], w = sw[p];
    const float lw = lap2d(w, sw[p - 1], sw[p + 1], sw[p - kBW], sw[p + kBW], m.lap_scale);
    const float ph2 = __fmul_rn(ph, ph);
    const float sfac = __fmaf_rn(c2x3, ph2, -m.a0);  // 3 c2 phi^2 - c1
    const float f = __fmaf_rn(sfac, w, -lw);
    lam_out.f[0][(int64_t)gy * g.pitch + gx] = __fmaf_rn(m.a2, f, l);  // a2 = dt M
    const float lph = lap2d(ph, sp[p - 1], sp[p + 1], sp[p - kBW], sp[p + kBW], m.lap_scale);
    const float mu = ch_mu(ph, lph, m);
    const float wp = __fmul_rn(w, ph);
    s0 = __fadd_rn(s0, wp);
    s1 = __fmaf_rn(wp, ph2, s1);
    s2 = __fmaf_rn(w, mu, s2);
  }
  double t[4] = {s0, s1, s2, 0.0};
  add_to_slot<3>(t, red, gpart);
}

// out[q] = sum over CTAs of gpart[4 * cta + q], in CTA order split over 256 threads.
__global__ void __launch_bounds__(256) adj_final_kernel(const double* gpart, int64_t nctas,
                                                        double* out) {
  __shared__ double red[4][256 / 32];
  double t[4] = {0, 0, 0, 0};
  const int64_t per = (nctas + 255) / 256;
  const int64_t c0 = per * threadIdx.x;
  const int64_t c1 = c0 + per < nctas ? c0 + per : nctas;
  for (int64_t c = c0; c < c1; ++c)
#pragma unroll
    for (int q = 0; q < 4; ++q) t[q] += gpart[4 * c + q];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    t[q] = warp_sum_d(t[q]);
    if (lane == 0) red[q][wid] = t[q];
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double s = 0.0;
    for (int w = 0; w < 256 / 32; ++w) s += red[threadIdx.x][w];
    out[threadIdx.x] = s;
  }
}

// Tile height of the Gray-Scott reverse step on this grid (see adj_gs2d_kernel): 8 when
// 16-row tiles would give fewer than four per SM, else 16.
int gs_adj_ty(const Geom& q, int device) {
  static int sms_by_dev[64] = {};
  int sms = device >= 0 && device < 64 ? sms_by_dev[device] : 0;
  if (sms == 0) {
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
      cudaGetLastError();
      sms = 1;
    } else if (device >= 0 && device < 64) {
      sms_by_dev[device] = sms;
    }
  }
  const int64_t tiles16 = (int64_t)((q.nx + kATX - 1) / kATX) * ((q.ny + 15) / 16);
  return tiles16 < 4 * (int64_t)sms ? 8 : 16;
}

// Reverse-step launch grid for the grid's model.
dim3 adj_grid(const pf_grid_s* g) {
  const Geom q = grid_geom(g);
  const int ty = g->model == PF_MODEL_GS ? gs_adj_ty(q, g->device) : kATY;
  return dim3((q.nx + kATX - 1) / kATX, (q.ny + ty - 1) / ty, 1);
}

float* ckpt_field(pf_grid_s* g, int64_t i, int f) {
  return g->adj.ckpt + (i * g->nf + f) * g->field_elems;
}
float* seg_field(pf_grid_s* g, int b, int64_t j, int f) {
  return g->adj.seg + (((int64_t)b * (g->adj.interval - 1) + j) * g->nf + f) * g->field_elems;
}
float* lam_field(pf_grid_s* g, int b, int f) {
  return g->adj.lam + (b * g->nf + f) * g->field_elems;
}

int check_gs2d(pf_grid_s* g) {
  if (!g->model_set ||
      (g->model != PF_MODEL_GS && g->model != PF_MODEL_AC && g->model != PF_MODEL_CH)) {
    set_error("the adjoint needs a Gray-Scott, Allen-Cahn or Cahn-Hilliard model");
    return PF_ERR_STATE;
  }
  if (g->dim != 2) return invalid("the adjoint is implemented for 2D grids");
  if (g->stencil != PF_ST_STD) return invalid("the adjoint uses the standard 5-point stencil");
  return PF_OK;
}

}  // namespace

void adjoint_release(pf_grid_s* g) {
  AdjointState& a = g->adj;
  if (a.ckpt) cudaFree(a.ckpt);
  if (a.seg) cudaFree(a.seg);
  if (a.lam) cudaFree(a.lam);
  if (a.gpart) cudaFree(a.gpart);
  if (a.gout) cudaFree(a.gout);
  if (a.ghost) cudaFreeHost(a.ghost);
  a = AdjointState();
}

// Enqueue the whole reverse pass on stream st, which the caller is recording into a graph:
// zero the gradient slots, then per segment from last to first recompute its states and
// run its reverse steps, then sum the slots. *lb_out receives the buffer holding lambda^0.
//
// Two branches: the reverse steps on st, the recomputation on st2 (forked into the same
// capture). With two segment buffers, segment s - 1 is recomputed into one buffer while
// segment s's reverse steps read the other, so the two chains of small launches overlap:
// recomputing segment s waits for its checkpoint only and for the reverse steps of segment
// s + 2 (the last reader of its buffer); the reverse steps of segment s wait for its
// recomputation. Each chain keeps its order, so every kernel sees the same inputs as in a
// serial pass and the result is the same bits.
static cudaError_t enqueue_reverse(pf_grid_s* g, const ModelParams& m, cudaStream_t st,
                                   cudaStream_t st2, int* lb_out) {
  AdjointState& a = g->adj;
  const Geom q = grid_geom(g);
  const dim3 grid = adj_grid(g);
  const int gs_ty = gs_adj_ty(q, g->device);
  const int64_t nctas = (int64_t)grid.x * grid.y;
  const int64_t C = a.interval;
  const int nb = a.seg_bufs > 0 ? a.seg_bufs : 1;
  // per segment: its recomputation done (on st2), its reverse steps done (on st)
  std::vector<cudaEvent_t> rec((size_t)a.n_ckpt, nullptr), rev((size_t)a.n_ckpt, nullptr);
  cudaEvent_t fork = nullptr, join = nullptr;
  cudaError_t e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
  for (int64_t s = 0; s < a.n_ckpt && e == cudaSuccess; ++s) {
    e = cudaEventCreateWithFlags(&rec[(size_t)s], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&rev[(size_t)s], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventRecord(fork, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st2, fork, 0);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.gpart, 0, sizeof(double) * 4 * nctas, st);
  int lb = 0;  // lambda ping-pong buffer holding the current adjoint state
  for (int64_t s = a.n_ckpt - 1; s >= 0 && e == cudaSuccess; --s) {
    const int64_t s0 = s * C;
    const int64_t len = std::min(C, a.n_steps - s0);
    const int b = (int)(s % nb);
    // states x^{s0} .. x^{s0+len-1}: slot 0 is the checkpoint, slots 1.. are recomputed
    auto state = [&](int64_t j, int f) -> float* {
      return j == 0 ? ckpt_field(g, s, f) : seg_field(g, b, j - 1, f);
    };
    // recompute on st2, once the buffer's previous reader (segment s + nb) is done
    if (s + nb < a.n_ckpt) e = cudaStreamWaitEvent(st2, rev[(size_t)(s + nb)], 0);
    for (int64_t j = 1; j < len && e == cudaSuccess; ++j) {
      FieldPtrs in{};
      FieldOut out{};
      for (int f = 0; f < g->nf; ++f) {
        in.f[f] = state(j - 1, f);
        out.f[f] = state(j, f);
      }
      e = launch_fe2d(g->model, 0, 1, q, in, out, m, st2);
    }
    if (e == cudaSuccess) e = cudaEventRecord(rec[(size_t)s], st2);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, rec[(size_t)s], 0);
    for (int64_t j = len - 1; j >= 0 && e == cudaSuccess; --j) {
      FieldPtrs xs{}, li{};
      FieldOut lo{};
      for (int f = 0; f < g->nf; ++f) {
        xs.f[f] = state(j, f);
        li.f[f] = lam_field(g, lb, f);
        lo.f[f] = lam_field(g, 1 - lb, f);
      }
      if (g->model == PF_MODEL_GS)
        if (gs_ty == 8)
          adj_gs2d_kernel<8><<<grid, kNT2, 0, st>>>(xs, li, lo, q, m, a.gpart);
        else
          adj_gs2d_kernel<16><<<grid, kNT2, 0, st>>>(xs, li, lo, q, m, a.gpart);
      else if (g->model == PF_MODEL_AC)
        adj_ac2d_kernel<<<grid, kNT2, 0, st>>>(xs, li, lo, q, m, a.gpart);
      else
        adj_ch2d_kernel<<<grid, kNT2, 0, st>>>(xs, li, lo, q, m, a.gpart);
      e = cudaGetLastError();
      lb = 1 - lb;
    }
    if (e == cudaSuccess) e = cudaEventRecord(rev[(size_t)s], st);
  }
  // join the second branch before the capture ends (also on an error, so that it can end)
  cudaError_t ej = cudaEventRecord(join, st2);
  if (ej == cudaSuccess) ej = cudaStreamWaitEvent(st, join, 0);
  if (e == cudaSuccess) e = ej;
  if (e == cudaSuccess) {
    adj_final_kernel<<<1, 256, 0, st>>>(a.gpart, nctas, a.gout);
    e = cudaGetLastError();
  }
  for (cudaEvent_t ev : rec)
    if (ev) cudaEventDestroy(ev);
  for (cudaEvent_t ev : rev)
    if (ev) cudaEventDestroy(ev);
  if (fork) cudaEventDestroy(fork);
  if (join) cudaEventDestroy(join);
  *lb_out = lb;
  return e;
}

}  // namespace pf

using namespace pf;

extern "C" {

int pf_adj_forward(pf_grid_t g, int64_t n_steps, int64_t ckpt_interval) {
  NvtxRange nvtx_("pf_adj_forward");
  if (int rc = check_grid(g)) return rc;
  if (int rc = check_gs2d(g)) return rc;
  if (n_steps < 1) return invalid("n_steps must be >= 1");
  if (ckpt_interval < 0) return invalid("ckpt_interval must be >= 0");
  int64_t C = ckpt_interval > 0 ? ckpt_interval : (int64_t)std::ceil(std::sqrt((double)n_steps));
  if (C > n_steps) C = n_steps;
  const int64_t n_ckpt = (n_steps + C - 1) / C;
  AdjointState& a = g->adj;
  const size_t state = sizeof(float) * g->nf * g->field_elems;
  if (a.n_ckpt != n_ckpt || a.interval != C) {
    // (re)allocate for this schedule
    if (a.ckpt) cudaFree(a.ckpt);
    if (a.seg) cudaFree(a.seg);
    a.ckpt = nullptr;
    a.seg = nullptr;
    a.seg_bufs = 0;
    PF_CUDA_TRY(cudaMalloc(&a.ckpt, state * n_ckpt));
    if (C > 1) {
      // two segment buffers where there are two segments and the memory allows, else one
      // (the reverse pass then recomputes and reverses one segment after the other)
      if (n_ckpt > 1 && cudaMalloc(&a.seg, 2 * state * (C - 1)) == cudaSuccess) {
        a.seg_bufs = 2;
      } else {
        cudaGetLastError();  // a failed first try leaves no sticky error
        PF_CUDA_TRY(cudaMalloc(&a.seg, state * (C - 1)));
        a.seg_bufs = 1;
      }
    }
    a.n_ckpt = n_ckpt;
    a.interval = C;
  }
  if (a.lam == nullptr) {
    PF_CUDA_TRY(cudaMalloc(&a.lam, 2 * state));
    PF_CUDA_TRY(cudaMemsetAsync(a.lam, 0, 2 * state, g->stream));
  }
  const dim3 grid = adj_grid(g);
  const int64_t nctas = (int64_t)grid.x * grid.y;
  if (a.gpart_cap < nctas) {
    if (a.gpart) cudaFree(a.gpart);
    a.gpart = nullptr;
    PF_CUDA_TRY(cudaMalloc(&a.gpart, sizeof(double) * 4 * nctas));
    a.gpart_cap = nctas;
  }
  if (a.gout == nullptr) PF_CUDA_TRY(cudaMalloc(&a.gout, sizeof(double) * 4));
  if (a.ghost == nullptr) PF_CUDA_TRY(cudaMallocHost(&a.ghost, sizeof(double) * 4));
  for (int64_t s = 0; s < n_ckpt; ++s) {
    for (int f = 0; f < g->nf; ++f)
      PF_CUDA_TRY(cudaMemcpyAsync(ckpt_field(g, s, f), g->buf[g->cur][f],
                                  sizeof(float) * g->field_elems, cudaMemcpyDeviceToDevice,
                                  g->stream));
    const int64_t len = std::min(C, n_steps - s * C);
    if (int rc = pf_step(g, len)) return rc;
  }
  for (int i = 0; i < 4; ++i) a.coeffs[i] = g->coeffs[i];
  a.dt = g->dt;
  a.n_steps = n_steps;
  a.ready = 1;
  return PF_OK;
}

int pf_adj_backward(pf_grid_t g, const float* dLdu_N, const float* dLdv_N, int on_device,
                    float* dLdu0, float* dLdv0, double* dtheta) {
  NvtxRange nvtx_("pf_adj_backward");
  if (int rc = check_grid(g)) return rc;
  if (int rc = check_gs2d(g)) return rc;
  AdjointState& a = g->adj;
  if (!a.ready) {
    set_error("pf_adj_backward: no recorded forward pass (call pf_adj_forward first)");
    return PF_ERR_STATE;
  }
  if (dLdu_N == nullptr || (g->nf == 2 && dLdv_N == nullptr))
    return invalid("dL/dx_N must not be NULL");
  const ModelParams m = make_params(g->model, a.coeffs, a.dt, g->h);
  const size_t w = sizeof(float) * g->nx;
  const cudaMemcpyKind kin = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const cudaMemcpyKind kout = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const float* src[2] = {dLdu_N, dLdv_N};
  for (int f = 0; f < g->nf; ++f)
    PF_CUDA_TRY(cudaMemcpy2DAsync(lam_field(g, 0, f), sizeof(float) * g->pitch, src[f], w, w,
                                  (size_t)g->ny, kin, g->stream));
  if (g->adj_exec == nullptr || g->adj_exec_steps != a.n_steps ||
      g->adj_exec_interval != a.interval) {
    if (g->adj_exec) cudaGraphExecDestroy(g->adj_exec);
    g->adj_exec = nullptr;
    if (g->capture == nullptr)
      PF_CUDA_TRY(cudaStreamCreateWithFlags(&g->capture, cudaStreamNonBlocking));
    if (g->capture2 == nullptr)
      PF_CUDA_TRY(cudaStreamCreateWithFlags(&g->capture2, cudaStreamNonBlocking));
    PF_CUDA_TRY(cudaStreamBeginCapture(g->capture, cudaStreamCaptureModeRelaxed));
    int lb = 0;
    cudaError_t e = enqueue_reverse(g, m, g->capture, g->capture2, &lb);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(g->capture, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return cuda_fail(e != cudaSuccess ? e : e2, "pf_adj_backward graph capture");
    }
    e = cudaGraphInstantiate(&g->adj_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      g->adj_exec = nullptr;
      return cuda_fail(e, "pf_adj_backward cudaGraphInstantiate");
    }
    g->adj_exec_steps = a.n_steps;
    g->adj_exec_interval = a.interval;
    g->adj_exec_lb = lb;
  }
  PF_CUDA_TRY(cudaGraphLaunch(g->adj_exec, g->stream));
  const int lb = g->adj_exec_lb;
  PF_CUDA_TRY(cudaMemcpyAsync(a.ghost, a.gout, sizeof(double) * 4, cudaMemcpyDeviceToHost,
                              g->stream));
  float* dst[2] = {dLdu0, dLdv0};
  for (int f = 0; f < g->nf; ++f)
    if (dst[f] != nullptr)
      PF_CUDA_TRY(cudaMemcpy2DAsync(dst[f], w, lam_field(g, lb, f), sizeof(float) * g->pitch, w,
                                    (size_t)g->ny, kout, g->stream));
  PF_CUDA_TRY(cudaStreamSynchronize(g->stream));
  if (dtheta != nullptr) {
    const double* S = a.ghost;
    if (g->model == PF_MODEL_GS) {
      // the kernel's Laplacians of u and v are unscaled (the parameters carry 1/h^2 in
      // D_u and D_v), so the sums for D_u and D_v take the factor here
      const double s = 1.0 / (g->h * g->h);
      for (int i = 0; i < 4; ++i) dtheta[i] = a.dt * S[i] * (i < 2 ? s : 1.0);
    } else if (g->model == PF_MODEL_AC) {
      dtheta[0] = a.dt * S[0];
      dtheta[1] = -a.dt * S[1];
    } else {
      const double M = a.coeffs[2];
      dtheta[0] = -a.dt * M * S[0];
      dtheta[1] = a.dt * M * S[1];
      dtheta[2] = a.dt * S[2];
    }
  }
  return PF_OK;
}

}  // extern "C"
