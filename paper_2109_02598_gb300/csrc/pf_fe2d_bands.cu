// 2D forward-Euler step with the whole grid resident in the shared memory of all SMs: one
// CTA per SM (a cooperative launch, so all CTAs run at once), each holding a band of full
// rows, for grids too large for one thread-block cluster but within the SMs' combined
// shared memory (Model B 2048^2: 13-14 rows of 2048 per SM). All steps of a pf_step call
// run in one launch; the state is read from global memory once and written once.
//
// CTA b of P owns rows [y0, y0 + B), y0 = floor(b ny / P), B >= 2R, staged as full rows with
// kHP periodic halo columns per side plus R halo rows above and below (R = 1 for Model A;
// R = 2 for Model B, whose step takes the Laplacian of the chemical potential). Each thread
// takes V consecutive columns: V = 2 up to 2048 columns (up to 1024 threads, which hides the
// shared-memory and barrier latency better than V = 4), V = 4 beyond. A step from state n
// to n + 1:
//   1. (n > 0) copy the neighbouring bands' edge rows of state n into the halo rows, and
//      commit this band's own edge rows of state n (kept aside during the previous step,
//      because its interior still needed the old values);
//   2. compute the band's top R and bottom R rows of state n + 1 (one phase for both), keep
//      them aside and store them into this CTA's exchange slots of parity (n + 1) & 1;
//   3. compute the interior rows in place, walking down the band two rows per CTA barrier:
//      each thread keeps its own column group's rows around the current ones in registers
//      (Model B: also their chemical potential, whose row-neighbour values sit in a six-row
//      shared ring used as three rotating pairs of rows).
// The exchange is tagged: every float travels in a 64-bit word whose upper half is the step
// it belongs to, written and read with single-copy-atomic 8-byte accesses, so a reader that
// finds the expected tag in all its words has the data, with no flag, fence or barrier across
// CTAs. Each band depends on both neighbours every step, so neighbours stay within one step
// of each other, and double-buffering the slots by parity keeps a slot from being rewritten
// before it has been read. Tags run on across launches (a per-grid counter), so words left
// by an earlier launch never match. Computing the edge rows first lets the interior hide
// the exchange latency. A read that finds stale tags retries for a bounded clock budget; on
// timeout the CTA sets the grid's error word and returns, its neighbours then time out in
// turn, and the host reports PF_ERR_TIMEOUT.
// The per-site arithmetic is that of the tiled kernels (lap4_rows, ch_mu, ch_update,
// ac_update), so the results are bitwise identical to theirs.
#include "pf_fe2d_tile.cuh"
#include "pf_grid.h"
#include "pf_internal.h"
#include "pf_sync.cuh"
#include "pf_tma.cuh"

namespace pf {

namespace {

constexpr int kHP = 4;             // halo columns per side of a staged row
constexpr int kMaxThreads = 1024;  // nx / V threads per CTA

struct BandGeom {
  int nx, ny;
  int ws;    // staged row width (floats): nx + 2 kHP
  int bmax;  // rows of the longest band
  int64_t pitch;
};

template <int MODEL>
struct BandCfg {
  static constexpr int R = ModelTraits<MODEL>::R;
  static constexpr bool MU = MODEL == PF_MODEL_CH;
  static constexpr int RING = MU ? 6 : 0;  // chemical-potential rows in shared memory
};

// Shared memory (floats): the band with its halo rows, the chemical-potential ring (Model B)
// and the 2R rows of new edge values kept aside.
template <int MODEL>
size_t band_smem_floats(const BandGeom& g) {
  using C = BandCfg<MODEL>;
  return (size_t)(g.bmax + 2 * C::R + C::RING) * g.ws + (size_t)2 * C::R * g.nx;
}

// ---- V consecutive columns of a staged row (V = 2 or 4) --------------------------------
template <int V>
struct Vec {
  float v[V];
};

template <int V>
__device__ __forceinline__ Vec<V> ldv(const float* p) {
  Vec<V> a;
  if constexpr (V == 4) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    a.v[0] = t.x;
    a.v[1] = t.y;
    a.v[2] = t.z;
    a.v[3] = t.w;
  } else {
    const float2 t = *reinterpret_cast<const float2*>(p);
    a.v[0] = t.x;
    a.v[1] = t.y;
  }
  return a;
}

template <int V>
__device__ __forceinline__ void stv(float* p, const Vec<V>& a) {
  if constexpr (V == 4)
    *reinterpret_cast<float4*>(p) = make_float4(a.v[0], a.v[1], a.v[2], a.v[3]);
  else
    *reinterpret_cast<float2*>(p) = make_float2(a.v[0], a.v[1]);
}

// Store columns V j .. V j + V - 1 of a staged row (first halo column at `row`), and their
// periodic copies when they lie within kHP of either row end.
template <int V>
__device__ __forceinline__ void put_rowv(float* row, int j, int nx, const Vec<V>& a) {
  const int c0 = V * j;
  stv<V>(row + kHP + c0, a);
  if (c0 < kHP) stv<V>(row + kHP + nx + c0, a);
  if (c0 >= nx - kHP) stv<V>(row + c0 - (nx - kHP), a);
}

// ---- per-row arithmetic (that of the tiled kernels, element by element) -----------------
// Laplacians of V sites from their row (c), the rows above (u) and below (d) and the row
// neighbours l, r of the first and last site.
template <int V>
__device__ __forceinline__ Vec<V> lapv(const Vec<V>& c, const Vec<V>& u, const Vec<V>& d,
                                       float l, float r, float scale) {
  Vec<V> o;
#pragma unroll
  for (int i = 0; i < V; ++i)
    o.v[i] = lap2d(c.v[i], i == 0 ? l : c.v[i - 1], i == V - 1 ? r : c.v[i + 1], u.v[i], d.v[i],
                   scale);
  return o;
}

// `p` points at this thread's first column in a staged row; its row neighbours are p[-1]
// and p[V].
template <int V>
__device__ __forceinline__ Vec<V> mu_at(const float* p, const Vec<V>& c, const Vec<V>& u,
                                        const Vec<V>& d, const ModelParams& m) {
  const Vec<V> l = lapv<V>(c, u, d, p[-1], p[V], m.lap_scale);
  Vec<V> o;
#pragma unroll
  for (int i = 0; i < V; ++i) o.v[i] = ch_mu(c.v[i], l.v[i], m);
  return o;
}

// Model B update of state c from the chemical potential of its row (mc, staged at q), the row
// above (mu) and below (md).
template <int V>
__device__ __forceinline__ Vec<V> ch_at(const Vec<V>& c, const float* q, const Vec<V>& mc,
                                        const Vec<V>& mu, const Vec<V>& md,
                                        const ModelParams& m) {
  const Vec<V> l = lapv<V>(mc, mu, md, q[-1], q[V], m.lap_scale);
  Vec<V> o;
#pragma unroll
  for (int i = 0; i < V; ++i) o.v[i] = ch_update(c.v[i], l.v[i], m);
  return o;
}

template <int V>
__device__ __forceinline__ Vec<V> ac_at(const float* p, const Vec<V>& c, const Vec<V>& u,
                                        const Vec<V>& d, const ModelParams& m) {
  const Vec<V> l = lapv<V>(c, u, d, p[-1], p[V], m.lap_scale);
  Vec<V> o;
#pragma unroll
  for (int i = 0; i < V; ++i) o.v[i] = ac_update(c.v[i], l.v[i], m);
  return o;
}

template <int MODEL, int V, int NT>
__global__ void __launch_bounds__(NT, 1)
    fe2d_bands_kernel(const float* __restrict__ in, float* __restrict__ out, BandGeom g,
                      ModelParams m, int64_t n_steps, unsigned long long* __restrict__ xbuf,
                      unsigned int tag0, int* __restrict__ err, long long budget) {
  using C = BandCfg<MODEL>;
  using VT = Vec<V>;
  constexpr int R = C::R;
  extern __shared__ float4 smem4[];
  float* phi = reinterpret_cast<float*>(smem4);  // staged rows -R .. bmax + R - 1
  float* ring = phi + (size_t)(g.bmax + 2 * R) * g.ws;
  float* aside = ring + C::RING * g.ws;  // new edge rows: top R, then bottom R
  const int ws = g.ws, nx = g.nx, j = threadIdx.x;
  const int c = kHP + V * j;  // this thread's first staged column
  const int P = gridDim.x, b = blockIdx.x;
  const int y0 = (int)((int64_t)b * g.ny / P);
  const int B = (int)((int64_t)(b + 1) * g.ny / P) - y0;
  const int up = b == 0 ? P - 1 : b - 1, dn = b == P - 1 ? 0 : b + 1;
  auto row = [&](int y) { return phi + (y + R) * ws; };     // staged row y (first halo column)
  auto at = [&](int y) { return phi + (y + R) * ws + c; };  // this thread's columns of row y
  // exchange slot (CTA, parity, side) of R rows of nx words; side 0 = top rows, 1 = bottom
  auto slot = [&](int cta, int par, int side) {
    return xbuf + ((size_t)(cta * 2 + par) * 2 + side) * R * nx + V * j;
  };
  auto put_aside = [&](int r, const VT& v) { stv<V>(aside + r * nx + V * j, v); };
  auto get_aside = [&](int r) { return ldv<V>(aside + r * nx + V * j); };

  canary_fill(phi, (size_t)(g.bmax + 2 * R + C::RING) * ws + (size_t)2 * R * nx);
  for (int y = -R; y < B + R; ++y) {
    const int gy = wrap_index(y0 + y, g.ny);
    VT v;
    if constexpr (V == 4) {
      const float4 t = __ldg(reinterpret_cast<const float4*>(in + gy * g.pitch) + j);
      v.v[0] = t.x;
      v.v[1] = t.y;
      v.v[2] = t.z;
      v.v[3] = t.w;
    } else {
      const float2 t = __ldg(reinterpret_cast<const float2*>(in + gy * g.pitch) + j);
      v.v[0] = t.x;
      v.v[1] = t.y;
    }
    put_rowv<V>(row(y), j, nx, v);
  }
  for (int64_t n = 0; n < n_steps; ++n) {
    const int np = (int)((n + 1) & 1);
    const unsigned int ntag = tag0 + (unsigned int)n + 1u;  // tag of state n + 1
    if (n > 0) {
      // 1. this band's edge rows of state n (the halo rows arrived during the last step)
#pragma unroll
      for (int r = 0; r < R; ++r) {
        put_rowv<V>(row(r), j, nx, get_aside(r));
        put_rowv<V>(row(B - R + r), j, nx, get_aside(R + r));
      }
    }
    __syncthreads();  // staging or the halo rows and committed edge rows are complete
    // The neighbours' rows of state n + 1 (the next step's halo): group q of this thread's
    // V words, q < R: row q of the bottom slot of the band above (into staged row q - R);
    // q >= R: row q - R of the top slot of the band below (into staged row B + q - R). Bit q
    // of `pend` marks a group still to fetch. They are read at the end of the step, before
    // its closing barrier (reading them earlier, during the interior, measured slower: the
    // neighbours publish them at about the time this band publishes its own).
    const unsigned long long* hu = slot(up, np, 1);
    const unsigned long long* hd = slot(dn, np, 0);
    unsigned int pend = n + 1 < n_steps ? (1u << (2 * R)) - 1u : 0u;
    unsigned long long* st = slot(b, np, 0);
    unsigned long long* sb = slot(b, np, 1);
    if constexpr (C::MU) {
      // 2. rows 0, 1 and B-2, B-1 of state n + 1 in one phase; ring rows r0..r5 hold the
      // chemical potential of rows 0, 1, 2 and B-2, B-1, B
      float* r0 = ring;
      float* r1 = ring + ws;
      float* r2 = ring + 2 * ws;
      float* r3 = ring + 3 * ws;
      float* r4 = ring + 4 * ws;
      float* r5 = ring + 5 * ws;
      const VT f0 = ldv<V>(at(-2)), f1 = ldv<V>(at(-1)), f2 = ldv<V>(at(0)), f3 = ldv<V>(at(1));
      VT pc = ldv<V>(at(2)), pd = ldv<V>(at(3));  // rows 2, 3: carried into the interior
      const VT tm_1 = mu_at<V>(at(-1), f1, f0, f2, m);
      const VT tm0 = mu_at<V>(at(0), f2, f1, f3, m);
      VT mm = mu_at<V>(at(1), f3, f2, pc, m);  // mu(1), mu(2): carried into the interior
      VT mc = mu_at<V>(at(2), pc, f3, pd, m);
      put_rowv<V>(r0, j, nx, tm0);
      put_rowv<V>(r1, j, nx, mm);
      put_rowv<V>(r2, j, nx, mc);
      const VT g0 = ldv<V>(at(B - 4)), g1 = ldv<V>(at(B - 3)), g2 = ldv<V>(at(B - 2));
      const VT g3 = ldv<V>(at(B - 1)), g4 = ldv<V>(at(B)), g5 = ldv<V>(at(B + 1));
      const VT bm3 = mu_at<V>(at(B - 3), g1, g0, g2, m);
      const VT bm2 = mu_at<V>(at(B - 2), g2, g1, g3, m);
      const VT bm1 = mu_at<V>(at(B - 1), g3, g2, g4, m);
      const VT bm0 = mu_at<V>(at(B), g4, g3, g5, m);
      put_rowv<V>(r3, j, nx, bm2);
      put_rowv<V>(r4, j, nx, bm1);
      put_rowv<V>(r5, j, nx, bm0);
      __syncthreads();
      const VT e0 = ch_at<V>(f2, r0 + c, tm0, tm_1, mm, m);
      const VT e1 = ch_at<V>(f3, r1 + c, mm, tm0, mc, m);
      const VT e2 = ch_at<V>(g2, r3 + c, bm2, bm3, bm1, m);
      const VT e3 = ch_at<V>(g3, r4 + c, bm1, bm2, bm0, m);
      put_aside(0, e0);
      put_aside(1, e1);
      put_aside(2, e2);
      put_aside(3, e3);
      ll_store<V>(st, ntag, e0.v);
      ll_store<V>(st + nx, ntag, e1.v);
      ll_store<V>(sb, ntag, e2.v);
      ll_store<V>(sb + nx, ntag, e3.v);
      // 3. interior rows 2 .. B-3 in place, two per barrier. The ring's pairs of rows
      // (r3, r4), (r5, r0), (r1, r2) take the chemical potential of rows (y+1, y+2) in turn;
      // `prev` is the ring row of mu(y).
      if (B - 2 > 2) {
        const float* prev = r2;
        float *wa = r3, *wb = r4, *na = r5, *nb = r0, *la = r1, *lb = r2;
        __syncthreads();  // the edge phase has read r0, r1, r3, r4
        int y = 2;
        for (; y + 1 < B - 2; y += 2) {
          const float* py = at(y);
          const VT p2 = ldv<V>(py + 2 * ws), p3 = ldv<V>(py + 3 * ws);
          const VT md = mu_at<V>(py + ws, pd, pc, p2, m);
          const VT mdd = mu_at<V>(py + 2 * ws, p2, pd, p3, m);
          put_rowv<V>(wa, j, nx, md);
          put_rowv<V>(wb, j, nx, mdd);
          __syncthreads();
          put_rowv<V>(row(y), j, nx, ch_at<V>(pc, prev + c, mc, mm, md, m));
          put_rowv<V>(row(y + 1), j, nx, ch_at<V>(pd, wa + c, md, mc, mdd, m));
          mm = md;
          mc = mdd;
          pc = p2;
          pd = p3;
          prev = wb;
          float* ta = wa;
          float* tb = wb;
          wa = na;
          wb = nb;
          na = la;
          nb = lb;
          la = ta;
          lb = tb;
        }
        if (y < B - 2) {  // one row left
          const float* py = at(y);
          const VT p2 = ldv<V>(py + 2 * ws);
          const VT md = mu_at<V>(py + ws, pd, pc, p2, m);
          put_rowv<V>(wa, j, nx, md);
          __syncthreads();
          put_rowv<V>(row(y), j, nx, ch_at<V>(pc, prev + c, mc, mm, md, m));
        }
      }
    } else {
      // 2. rows 0 and B-1 of state n + 1
      const VT f0 = ldv<V>(at(-1)), f1 = ldv<V>(at(0));
      VT pu = f1, pc = ldv<V>(at(1));  // rows 0, 1: carried into the interior
      const VT e0 = ac_at<V>(at(0), f1, f0, pc, m);
      const VT g0 = ldv<V>(at(B - 2)), g1 = ldv<V>(at(B - 1)), g2 = ldv<V>(at(B));
      const VT e1 = ac_at<V>(at(B - 1), g1, g0, g2, m);
      put_aside(0, e0);
      put_aside(1, e1);
      ll_store<V>(st, ntag, e0.v);
      ll_store<V>(sb, ntag, e1.v);
      // 3. interior rows 1 .. B-2 in place, two per barrier (the edge phase read only rows
      // 0 and B-1 of other threads, which the interior does not write, and only this
      // thread's own columns of the halo rows)
      int y = 1;
      for (; y + 1 < B - 1; y += 2) {
        const float* py = at(y);
        const VT pd = ldv<V>(py + ws), p2 = ldv<V>(py + 2 * ws);
        const VT v0 = ac_at<V>(py, pc, pu, pd, m);
        const VT v1 = ac_at<V>(py + ws, pd, pc, p2, m);
        __syncthreads();  // every thread has read rows y, y+1 before they are overwritten
        put_rowv<V>(row(y), j, nx, v0);
        put_rowv<V>(row(y + 1), j, nx, v1);
        pu = pd;
        pc = p2;
      }
      if (y < B - 1) {  // one row left
        const float* py = at(y);
        const VT pd = ldv<V>(py + ws);
        const VT v0 = ac_at<V>(py, pc, pu, pd, m);
        __syncthreads();
        put_rowv<V>(row(y), j, nx, v0);
      }
    }
    // 4. the next halo: read until every group is fresh (bounded). The halo rows are not
    // read after the edge phase's first barrier, so they can be filled before this step's end.
    int ok = 1;
    if (pend) {
      const long long t0 = clock64();
      while (pend) {
        LLWords<V> w[2 * R];
#pragma unroll
        for (int q = 0; q < 2 * R; ++q)
          if (pend >> q & 1u) w[q] = ll_load<V>(q < R ? hu + (size_t)q * nx : hd + (size_t)(q - R) * nx);
#pragma unroll
        for (int q = 0; q < 2 * R; ++q) {
          if ((pend >> q & 1u) && ll_fresh<V>(w[q], ntag)) {
            VT v;
            ll_values<V>(w[q], v.v);
            put_rowv<V>(q < R ? row(q - R) : row(B + q - R), j, nx, v);
            pend &= ~(1u << q);
          }
        }
        if (pend && clock64() - t0 > budget) {
          ok = 0;
          atomicExch(err, 1);
          break;
        }
      }
    }
    // the interior has read the rows that the next step's commit overwrites
    if (!__syncthreads_and(ok)) return;
  }
  // the band to global memory (edge rows from the values kept aside)
  for (int y = 0; y < B; ++y) {
    const bool edge = n_steps > 0 && (y < R || y >= B - R);
    const VT v = edge ? get_aside(y < R ? y : y - (B - R) + R) : ldv<V>(at(y));
    stv<V>(out + (int64_t)(y0 + y) * g.pitch + V * j, v);
  }
}

struct DevLimits {
  int sms = 0, smem_optin = 0;
};
DevLimits g_limits[64];

DevLimits device_limits() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return DevLimits{};
  }
  if (dev < 64 && g_limits[dev].sms) return g_limits[dev];
  DevLimits d;
  if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&d.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
          cudaSuccess) {
    cudaGetLastError();
    return DevLimits{};
  }
  if (dev < 64) g_limits[dev] = d;
  return d;
}

// CTAs of the launch: one per SM, fewer where the bands would be shorter than 2R rows.
template <int MODEL>
int band_ctas(const Geom& q, int sms) {
  const int lim = q.ny / (2 * BandCfg<MODEL>::R);
  return lim < sms ? lim : sms;
}

template <int MODEL>
BandGeom band_geom(const Geom& q, int ctas) {
  BandGeom g{};
  g.nx = q.nx;
  g.ny = q.ny;
  g.ws = q.nx + 2 * kHP;
  g.bmax = (q.ny + ctas - 1) / ctas;
  g.pitch = q.pitch;
  return g;
}

template <int MODEL>
bool bands_fit(const Geom& q) {
  if (q.dim != 2 || q.nx % 4 != 0 || q.nx < 64 || q.nx > 4 * kMaxThreads) return false;
  const DevLimits d = device_limits();
  if (d.sms == 0) return false;
  const int ctas = band_ctas<MODEL>(q, d.sms);
  if (ctas < 2) return false;
  return band_smem_floats<MODEL>(band_geom<MODEL>(q, ctas)) * sizeof(float) <=
         (size_t)d.smem_optin;
}

template <int MODEL>
cudaError_t launch_bands(pf_grid_s* gr, int src, int dst, int64_t n_steps, cudaStream_t st) {
  const Geom q = grid_geom(gr);
  const DevLimits d = device_limits();
  const int ctas = band_ctas<MODEL>(q, d.sms);
  const BandGeom g = band_geom<MODEL>(q, ctas);
  const size_t smem = band_smem_floats<MODEL>(g) * sizeof(float);
  const size_t words = (size_t)ctas * 4 * BandCfg<MODEL>::R * q.nx;
  cudaError_t e = cudaSuccess;
  if (gr->band_x == nullptr || gr->band_x_words < words) {
    cudaFree(gr->band_x);
    gr->band_x = nullptr;
    gr->band_x_words = 0;
    e = cudaMalloc(&gr->band_x, words * sizeof(unsigned long long));
    if (e != cudaSuccess) return e;
    gr->band_x_words = words;
    gr->band_tag = 0;  // forces the clearing below
  }
  // tags of this launch: band_tag + 1 .. band_tag + n_steps; words of earlier launches carry
  // smaller tags. Restart from cleared slots before the 32-bit tag would wrap.
  if (gr->band_tag == 0 || (uint64_t)gr->band_tag + (uint64_t)n_steps + 1 > 0xffffffffull) {
    e = cudaMemsetAsync(gr->band_x, 0, gr->band_x_words * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    gr->band_tag = 1;
  }
  unsigned int tag0 = gr->band_tag;
  gr->band_tag = (unsigned int)((uint64_t)gr->band_tag + (uint64_t)n_steps + 1);
  // two columns per thread up to 2048 columns (1024 threads), four beyond
  const int v = q.nx <= 2048 ? 2 : 4;
  const int threads = q.nx / v;
  const void* kern = v == 4          ? (const void*)fe2d_bands_kernel<MODEL, 4, 1024>
                     : threads > 512 ? (const void*)fe2d_bands_kernel<MODEL, 2, 1024>
                                     : (const void*)fe2d_bands_kernel<MODEL, 2, 512>;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const float* in = gr->buf[src][0];
  float* out = gr->buf[dst][0];
  ModelParams m = gr->params;
  unsigned long long* xb = gr->band_x;
  int* err = gr->d_err;
  long long budget = kWaitBudgetCycles;
  void* args[] = {(void*)&in, (void*)&out,  (void*)&g,   (void*)&m,     (void*)&n_steps,
                  (void*)&xb, (void*)&tag0, (void*)&err, (void*)&budget};
  return cudaLaunchCooperativeKernel(kern, dim3(ctas), dim3(threads), args, smem, st);
}

}  // namespace

bool fe2d_bands_supported(int model, const Geom& q) {
  switch (model) {
    case PF_MODEL_AC:
      return bands_fit<PF_MODEL_AC>(q);
    case PF_MODEL_CH:
      return bands_fit<PF_MODEL_CH>(q);
  }
  return false;
}

cudaError_t launch_fe2d_bands(pf_grid_s* g, int src, int dst, int64_t n_steps, cudaStream_t st) {
  if (!fe2d_bands_supported(g->model, grid_geom(g))) return cudaErrorInvalidValue;
  if (g->model == PF_MODEL_AC) return launch_bands<PF_MODEL_AC>(g, src, dst, n_steps, st);
  return launch_bands<PF_MODEL_CH>(g, src, dst, n_steps, st);
}

void fe2d_bands_release(pf_grid_s* g) {
  cudaFree(g->band_x);
  g->band_x = nullptr;
  g->band_x_words = 0;
  g->band_tag = 0;
}

}  // namespace pf
