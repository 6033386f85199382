// Tile body of the 2D forward-Euler kernel with temporal blocking; used by the plain
// 2D kernel and by the batched runner so both execute identical arithmetic.
#pragma once

#include "pf_internal.h"

namespace pf {

constexpr int kNT2 = 256;  // threads per CTA of every 2D kernel

template <int MODEL, int K, int TX, int TY>
struct Cfg2 {
  static constexpr int NF = ModelTraits<MODEL>::NF;
  static constexpr int R = ModelTraits<MODEL>::R;
  static constexpr int H = K * R;          // halo width in sites
  static constexpr int W = TX + 2 * H;     // staged region width
  static constexpr int HT = TY + 2 * H;    // staged region height
  static constexpr int PL = W * HT;        // floats per staged field
  static constexpr int NBUF = (K > 1) ? 2 : 1;
  static constexpr int MU = (MODEL == PF_MODEL_CH) ? PL : 0;
  static constexpr int SMEM_FLOATS = NF * NBUF * PL + MU;
};

// Stage rows [y0-H, y0+TY+H) x cols [x0-H, x0+TX+H) of every field (periodic wrap) into
// buffer 0 of shared memory: sm[f * PL + r * W + c].
template <class C>
__device__ __forceinline__ void load_region2d(const FieldPtrs& in, int nx, int ny,
                                              int64_t pitch, int x0, int y0, float* sm) {
  for (int i = threadIdx.x; i < C::PL; i += kNT2) {
    const int r = i / C::W;
    const int c = i - r * C::W;
    const int gy = wrap_index(y0 - C::H + r, ny);
    const int gx = wrap_index(x0 - C::H + c, nx);
    const int64_t off = (int64_t)gy * pitch + gx;
#pragma unroll
    for (int f = 0; f < C::NF; ++f) sm[f * C::PL + i] = __ldg(in.f[f] + off);
  }
}

// k forward-Euler sub-steps of one tile; the last one is written to `out` (sites beyond
// nx, ny are computed on periodic images and not stored).
template <int MODEL, int K, int TX, int TY>
__device__ __forceinline__ void fe2d_tile(const FieldPtrs& in, const FieldOut& out, int nx,
                                          int ny, int64_t pitch, int x0, int y0,
                                          const ModelParams& m, float* sm) {
  using C = Cfg2<MODEL, K, TX, TY>;
  constexpr int W = C::W;
  constexpr int PL = C::PL;
  load_region2d<C>(in, nx, ny, pitch, x0, y0, sm);
  __syncthreads();
#pragma unroll
  for (int s = 0; s < K; ++s) {
    const float* src = sm + (s & 1) * C::NF * PL;
    float* dst = sm + ((s + 1) & 1) * C::NF * PL;
    if constexpr (MODEL == PF_MODEL_CH) {
      float* mu = sm + C::NF * C::NBUF * PL;
      const int lm = C::R * s + 1;
      const int mrows = C::HT - 2 * lm;
      const int mcols = W - 2 * lm;
      for (int i = threadIdx.x; i < mrows * mcols; i += kNT2) {
        const int r = lm + i / mcols;
        const int c = lm + (i - (i / mcols) * mcols);
        const int p = r * W + c;
        const float pc = src[p];
        const float l = lap2d(pc, src[p - 1], src[p + 1], src[p - W], src[p + W], m.inv_h2);
        mu[p] = ch_mu(pc, l, m);
      }
      __syncthreads();
    }
    const bool last = (s == K - 1);
    const int lo = C::R * (s + 1);
    const int rows = C::HT - 2 * lo;
    const int cols = W - 2 * lo;
    for (int i = threadIdx.x; i < rows * cols; i += kNT2) {
      const int rr = i / cols;
      const int r = lo + rr;
      const int c = lo + (i - rr * cols);
      const int p = r * W + c;
      float val[C::NF];
      if constexpr (MODEL == PF_MODEL_AC) {
        const float pc = src[p];
        const float l = lap2d(pc, src[p - 1], src[p + 1], src[p - W], src[p + W], m.inv_h2);
        val[0] = ac_update(pc, l, m);
      } else if constexpr (MODEL == PF_MODEL_CH) {
        const float* mu = sm + C::NF * C::NBUF * PL;
        const float l = lap2d(mu[p], mu[p - 1], mu[p + 1], mu[p - W], mu[p + W], m.inv_h2);
        val[0] = ch_update(src[p], l, m);
      } else {
        const float* su = src;
        const float* sv = src + PL;
        const float u = su[p], v = sv[p];
        const float lu = lap2d(u, su[p - 1], su[p + 1], su[p - W], su[p + W], m.inv_h2);
        const float lv = lap2d(v, sv[p - 1], sv[p + 1], sv[p - W], sv[p + W], m.inv_h2);
        gs_update(u, v, lu, lv, m, val[0], val[1]);
      }
      if (last) {
        const int gx = x0 + c - C::H;
        const int gy = y0 + r - C::H;
        if (gx < nx && gy < ny) {
          const int64_t off = (int64_t)gy * pitch + gx;
#pragma unroll
          for (int f = 0; f < C::NF; ++f) out.f[f][off] = val[f];
        }
      } else {
#pragma unroll
        for (int f = 0; f < C::NF; ++f) dst[f * PL + p] = val[f];
      }
    }
    if (!last) __syncthreads();
  }
}

}  // namespace pf
