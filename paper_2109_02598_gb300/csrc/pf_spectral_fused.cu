// Fused engine of the semi-implicit spectral solver (Sec. 2.4.2) for grids whose sides are
// powers of two: 2D with sides 4 .. 1024, and 3D with nx in 4 .. 1024 and ny nz small enough
// for one (y, z) slab to stay in a CTA's shared memory. Every step of a pf_spectral_step call
// runs inside one cooperative launch, with this file's own FFTs in shared memory.
//
// The state psi_hat [nz][ny][nxh] (and the tables) are those of the cuFFT engine; W (the f_hat
// slices of spec, which this engine uses as scratch) carries the data between the two phases
// of a step. In 2D it has the state's layout [y][kx]; in 3D it is held as [kx][z][y], so that
// a slab is contiguous and the strided accesses fall to the row phase, whose tasks spread
// them over many more SMs (the slab phase has one task per kx):
//   row phase   per x-row (z, y): the inverse transform along x of W's half spectrum, the
//               nonlinear terms, the forward transform along x, back into W. Two real rows
//               share one complex FFT: rows r and r+1 of a one-field model, or psi and m of
//               one row in Model C (whose nonlinear terms need both at the same site);
//   slab phase  per column kx (and field): the ny x nz slab of W at that kx, transformed
//               forward along y and then z -> f_hat; on the self-conjugate columns (kx = 0,
//               nx/2) its Hermitian part, pairing (kz, ky) with (-kz, -ky); the update
//               psi_hat <- A psi_hat + (B N) f_hat; and the inverse transform (z, then y) of
//               psi_hat / N back into W for the next row phase. In 2D the slab is one column.
// Each slab team owns fixed slabs for the whole launch and keeps their psi_hat and (A, B N) in
// shared memory: a prologue loads them and fills W from psi_hat; the last step writes
// psi_hat and work = psi_hat / N (as the cuFFT engine leaves them) back to global memory
// instead of the inverse transform. The phases are separated by a grid barrier (release /
// acquire atomics) whose waits are bounded by a clock budget: on timeout a CTA sets the
// error word and returns, so the launch always ends.
//
// A task (a row pair, or a slab) is done by a team of 32 .. 1024 threads of a CTA, chosen
// per phase so that each thread does one radix-8 butterfly per pass where the tasks still fit
// in one round on the SMs; a team synchronises on its own named barrier. The FFTs are
// Stockham passes (radix 8, then one radix-4 or radix-2 pass) between two shared-memory
// buffers: natural order in and out, no bit reversal, and every thread loads all
// of a butterfly's inputs before it computes. A slab's transforms are batched passes: along y
// the slab's nz rows at once, along z its ny columns at once, consecutive lanes on
// consecutive FFTs of the batch; the slab's rows are padded to ny + 1 values in shared memory,
// so those lanes fall on distinct banks in both directions.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "pf_spectral.h"
#include "pf_tma.cuh"

namespace pf {
int invalid(const char* fmt, ...);

namespace {

constexpr int kThreads = 1024;  // the widest CTA (launch bound); see fused_shape
constexpr int kMaxSide = 1024;

struct FusedArgs {
  float2* state;  // [nf][cs]
  float2* W;      // [nf][cs]
  float2* work;   // [nf][cs]
  const float2* table;
  const float2* twx;  // W_nx^j, j < nx
  const float2* twy;  // W_ny^j, j < ny
  const float2* twz;  // W_nz^j, j < nz (3D)
  int nx, ny, nz, nxh, lognx, logny, lognz, nf;
  int nrows;               // x-rows: ny nz
  int wr, wk;              // W: mode kx of x-row r at W + field cs + r wr + kx wk
  int rbuf, cbuf;          // float2s of one row team's / slab team's two FFT buffers
  int row_team, col_team;  // threads per task in the row and slab phases
  int cpt;                 // slabs owned per slab team
  int64_t cs;
  float inv_n;
  NlCoeffs k;
  int64_t steps;
  unsigned int* bar;  // count, generation, error
  long long budget;
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(__fmaf_rn(a.x, b.x, -__fmul_rn(a.y, b.y)),
                     __fmaf_rn(a.x, b.y, __fmul_rn(a.y, b.x)));
}

// The threads that share one task: `size` threads (a power of two from 8) of one CTA, the
// `index`-th such group. Teams wider than a warp synchronise on named barrier index + 1; a
// warp, or a warp's 8- or 16-lane teams, on __syncwarp (the whole warp: its teams run the same
// control flow, see the row phase).
struct Team {
  int size, rank, index;
  __device__ __forceinline__ void sync() const {
    if (size <= 32) __syncwarp();
    else asm volatile("bar.sync %0, %1;" ::"r"(index + 1), "r"(size) : "memory");
  }
};

__device__ __forceinline__ Team make_team(int size) {
  Team t;
  t.size = size;
  t.rank = threadIdx.x % size;
  t.index = threadIdx.x / size;
  return t;
}

// 4-point DFT of (a, b, c, d): out[m] = sum_r x_r W_4^{r m}, W_4 = -i (forward) or +i.
template <bool INV>
__device__ __forceinline__ void dft4(const float2& a, const float2& b, const float2& c,
                                     const float2& d, float2* out) {
  const float2 a0 = make_float2(__fadd_rn(a.x, c.x), __fadd_rn(a.y, c.y));
  const float2 a1 = make_float2(__fsub_rn(a.x, c.x), __fsub_rn(a.y, c.y));
  const float2 a2 = make_float2(__fadd_rn(b.x, d.x), __fadd_rn(b.y, d.y));
  const float2 dd = make_float2(__fsub_rn(b.x, d.x), __fsub_rn(b.y, d.y));
  const float2 a3 = INV ? make_float2(-dd.y, dd.x) : make_float2(dd.y, -dd.x);
  out[0] = make_float2(__fadd_rn(a0.x, a2.x), __fadd_rn(a0.y, a2.y));
  out[1] = make_float2(__fadd_rn(a1.x, a3.x), __fadd_rn(a1.y, a3.y));
  out[2] = make_float2(__fsub_rn(a0.x, a2.x), __fsub_rn(a0.y, a2.y));
  out[3] = make_float2(__fsub_rn(a1.x, a3.x), __fsub_rn(a1.y, a3.y));
}

// One Stockham pass of radix R over `batch` FFTs of n points (stride ns so far). FFT b's
// element i lives at buf[b bs + i es] in both buffers. Butterfly j < n/R of an FFT takes
// in[j + r n/R], twiddles it by W_{ns R}^{(j mod ns) r}, and writes its R-point DFT to
// out[(j - j mod ns) R + j mod ns + r ns]. tw holds W_n^i = exp(-2 pi i i / n), i < n; INV
// conjugates every twiddle (the inverse transform, unnormalised). BF: consecutive lanes take
// consecutive FFTs of the batch (for bs = 1, where the elements are strided), else
// consecutive butterflies of one FFT.
template <int R, bool INV, bool BF>
__device__ __forceinline__ void stockham_pass(const float2* __restrict__ in,
                                              float2* __restrict__ out, int n, int logq, int ns,
                                              int batch, int logb, int bs, int es,
                                              const float2* __restrict__ tw, const Team& tm) {
  const int q = n / R;
  const int tws = n / (ns * R);
  const int total = q * batch;
#pragma unroll 2
  for (int t = tm.rank; t < total; t += tm.size) {
    int b, j;
    if (BF) {
      j = t >> logb;
      b = t - (j << logb);
    } else {
      b = t >> logq;
      j = t - (b << logq);
    }
    const float2* ib = in + b * bs;
    float2* ob = out + b * bs;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = ib[(j + r * q) * es];
    const int k = j & (ns - 1);
#pragma unroll
    for (int r = 1; r < R; ++r) {
      float2 w = tw[(k * r * tws) & (n - 1)];
      if (INV) w.y = -w.y;
      v[r] = cmul(w, v[r]);
    }
    const int base = (j - k) * R + k;
    if (R == 8) {
      // two 4-point DFTs (even and odd inputs), the odd one twiddled by W_8^m, combined
      float2 e[4], o[4];
      dft4<INV>(v[0], v[2], v[4], v[6], e);
      dft4<INV>(v[1], v[3], v[5], v[7], o);
      const float c = 0.70710678118654752f;  // sqrt(1/2)
      const float2 o1 = o[1], o3 = o[3];
      if (!INV) {  // W_8 = c (1 - i), W_8^2 = -i, W_8^3 = -c (1 + i)
        o[1] = make_float2(__fmul_rn(c, __fadd_rn(o1.x, o1.y)), __fmul_rn(c, __fsub_rn(o1.y, o1.x)));
        o[2] = make_float2(o[2].y, -o[2].x);
        o[3] = make_float2(__fmul_rn(c, __fsub_rn(o3.y, o3.x)), -__fmul_rn(c, __fadd_rn(o3.x, o3.y)));
      } else {  // the conjugates: c (1 + i), i, c (-1 + i)
        o[1] = make_float2(__fmul_rn(c, __fsub_rn(o1.x, o1.y)), __fmul_rn(c, __fadd_rn(o1.x, o1.y)));
        o[2] = make_float2(-o[2].y, o[2].x);
        o[3] = make_float2(-__fmul_rn(c, __fadd_rn(o3.x, o3.y)), __fmul_rn(c, __fsub_rn(o3.x, o3.y)));
      }
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        ob[(base + m * ns) * es] = make_float2(__fadd_rn(e[m].x, o[m].x), __fadd_rn(e[m].y, o[m].y));
        ob[(base + (m + 4) * ns) * es] =
            make_float2(__fsub_rn(e[m].x, o[m].x), __fsub_rn(e[m].y, o[m].y));
      }
    } else if (R == 2) {
      ob[base * es] = make_float2(__fadd_rn(v[0].x, v[1].x), __fadd_rn(v[0].y, v[1].y));
      ob[(base + ns) * es] = make_float2(__fsub_rn(v[0].x, v[1].x), __fsub_rn(v[0].y, v[1].y));
    } else {
      float2 x[4];
      dft4<INV>(v[0], v[1], v[2], v[3], x);
#pragma unroll
      for (int m = 0; m < 4; ++m) ob[(base + m * ns) * es] = x[m];
    }
  }
}

// `batch` = 2^logb FFTs of n = 2^logn points in b (layout as stockham_pass) by one team,
// natural order in and out: radix-8 passes, then one radix-4 or radix-2 pass for the rest.
// b and b2 are used in turn and the result is in the returned buffer (the other one is
// free). logn = 0 returns b untouched. Each pass ends with a team barrier and its stores and
// loads make a round trip through shared memory, so fewer, wider passes are faster: radix 8
// takes a 64-point transform in two passes instead of three (radix 4), 512 points in three
// instead of five.
template <bool INV, bool BF>
__device__ __forceinline__ float2* team_fft(float2* b, float2* b2, int n, int logn, int logb,
                                            int bs, int es, const float2* tw, const Team& tm) {
  float2* in = b;
  float2* out = b2;
  int ns = 1;
  const int batch = 1 << logb;
  int left = logn;
  for (; left >= 3; left -= 3) {
    stockham_pass<8, INV, BF>(in, out, n, logn - 3, ns, batch, logb, bs, es, tw, tm);
    tm.sync();
    float2* t = in;
    in = out;
    out = t;
    ns <<= 3;
  }
  if (left == 2) {
    stockham_pass<4, INV, BF>(in, out, n, logn - 2, ns, batch, logb, bs, es, tw, tm);
    tm.sync();
    in = out;
  } else if (left == 1) {
    stockham_pass<2, INV, BF>(in, out, n, logn - 1, ns, batch, logb, bs, es, tw, tm);
    tm.sync();
    in = out;
  }
  return in;
}

// One FFT of n points, contiguous.
template <bool INV>
__device__ __forceinline__ float2* team_fft1(float2* b, float2* b2, int n, int logn,
                                             const float2* tw, const Team& tm) {
  return team_fft<INV, false>(b, b2, n, logn, 0, 0, 1, tw, tm);
}

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier (sense by generation): bar[0] counts arrivals, bar[1] is the generation,
// bar[2] the error word. Bounded: false after budget clocks without a release.
__device__ __forceinline__ bool grid_barrier(unsigned int* bar, unsigned int nblocks,
                                             long long budget) {
  __syncthreads();
  int ok = 1;
  if (threadIdx.x == 0) {
    const unsigned int my_gen = ld_acquire(bar + 1);
    __threadfence();  // the CTA's writes, ordered before this thread by the CTA barrier
    unsigned int old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(bar) : "memory");
    if (old + 1 == nblocks) {
      asm volatile("st.relaxed.gpu.global.u32 [%0], 0;" ::"l"(bar) : "memory");
      asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar + 1) : "memory");
    } else {
      const long long t0 = clock64();
      while (ld_acquire(bar + 1) == my_gen) {
        if (clock64() - t0 > budget) {
          atomicExch(bar + 2, 1u);
          ok = 0;
          break;
        }
      }
    }
  }
  return __syncthreads_and(ok) != 0;
}

template <int MODEL>
__device__ __forceinline__ void nl_pair(float2& z, const NlCoeffs& k) {
  if (MODEL == PF_MODEL_C) {
    nonlinear_site<MODEL>(z.x, z.y, k.c);
  } else {
    float unused = 0.f;
    nonlinear_site<MODEL>(z.x, unused, k.c);
    nonlinear_site<MODEL>(z.y, unused, k.c);
  }
}

// Row task: two real x-rows (field f1 row y1, field f2 row y2; a row index counts (z, y)
// rows, z slowest) whose half spectra are in W. A team with no task (valid false) runs the
// same steps on its own buffers without touching W, so that the warp it shares with other
// teams stays in step.
template <int MODEL>
__device__ __forceinline__ void row_task(const FusedArgs& a, int f1, int y1, int f2, int y2,
                                         bool valid, float2* b, float2* b2, const float2* twx,
                                         const Team& tm) {
  const int nx = a.nx, nh = nx >> 1;
  const int64_t ks = a.wk;  // mode stride of a row in W
  // both half spectra into b2 (X1 at [0, nh], X2 at [nh + 1, 2 nh + 1]; b2 holds nx + 2), all
  // of a thread's copies in flight before one wait
  const float2* X1g = a.W + f1 * a.cs + (int64_t)y1 * a.wr;
  const float2* X2g = a.W + f2 * a.cs + (int64_t)y2 * a.wr;
  for (int k = tm.rank; k <= nh && valid; k += tm.size) {
    cp_async8(b2 + k, X1g + k * ks);
    cp_async8(b2 + nh + 1 + k, X2g + k * ks);
  }
  cp_async_wait_all();
  tm.sync();
  const float2* X1 = b2;
  const float2* X2 = b2 + nh + 1;
  // Z = X1 + i X2 over the full length, each extended by Hermitian symmetry; the imaginary
  // parts at k = 0 and nx/2 are dropped, as a complex-to-real transform does
  for (int k = tm.rank; k < nx; k += tm.size) {
    float2 p, q;
    if (k <= nh) {
      p = X1[k];
      q = X2[k];
      if (k == 0 || k == nh) p.y = q.y = 0.f;
    } else {
      p = X1[nx - k];
      q = X2[nx - k];
      p.y = -p.y;
      q.y = -q.y;
    }
    b[k] = make_float2(__fsub_rn(p.x, q.y), __fadd_rn(p.y, q.x));
  }
  tm.sync();
  float2* z = team_fft1<true>(b, b2, nx, a.lognx, twx, tm);
  float2* other = z == b ? b2 : b;
  for (int k = tm.rank; k < nx; k += tm.size) {
    float2 v = z[k];
    nl_pair<MODEL>(v, a.k);
    z[k] = v;
  }
  tm.sync();
  const float2* Y = team_fft1<false>(z, other, nx, a.lognx, twx, tm);
  float2* F1 = a.W + f1 * a.cs + (int64_t)y1 * a.wr;
  float2* F2 = a.W + f2 * a.cs + (int64_t)y2 * a.wr;
  for (int k = tm.rank; k <= nh && valid; k += tm.size) {
    const float2 y = Y[k];
    const float2 r = Y[(nx - k) & (nx - 1)];  // Y(-k); conj taken below
    const float2 s = make_float2(__fadd_rn(y.x, r.x), __fsub_rn(y.y, r.y));  // Y + conj Y(-k)
    const float2 d = make_float2(__fsub_rn(y.x, r.x), __fadd_rn(y.y, r.y));  // Y - conj Y(-k)
    F1[k * ks] = make_float2(__fmul_rn(0.5f, s.x), __fmul_rn(0.5f, s.y));
    F2[k * ks] = make_float2(__fmul_rn(0.5f, d.y), __fmul_rn(-0.5f, d.x));  // -i d / 2
  }
  tm.sync();
}

// Slab task (field f, column kx): the ny x nz values W[f][z][y][kx], held in shared memory as
// [z][y] with rows of ny + 1 (the pad keeps a batched pass's lanes, one FFT each, on distinct
// banks), with the slab's psi_hat in st and (A, B N) in tb (shared memory, [kz][ky]).
// mode 0: prologue (W <- inverse(psi_hat / N)); mode 1: full step; mode 2: last step (psi_hat
// and work = psi_hat / N to global memory, no inverse transform). In 2D (nz = 1) it is one
// column of ny values.
__device__ __forceinline__ void slab_task(const FusedArgs& a, int f, int kx, int mode,
                                          float2* st, const float2* tb, float2* b, float2* b2,
                                          const float2* twy, const float2* twz, const Team& tm) {
  const int ny = a.ny, nz = a.nz, ns = ny * nz, rp = ny + 1;
  const int64_t base = f * a.cs + kx;  // the state's layout, [z][y][kx]
  const int64_t rstride = a.nxh;
  const float2* Wg = a.W + f * a.cs + (int64_t)kx * a.wk;  // the slab in W (rows wr apart)
  float2* o = b;  // receives psi_hat / N for the inverse transform
  if (mode != 0) {
    for (int i = tm.rank; i < ns; i += tm.size)
      cp_async8(b + i + (i >> a.logny), Wg + (int64_t)i * a.wr);
    cp_async_wait_all();
    tm.sync();
    // forward along y (the nz rows of the slab), then along z (its ny columns); in both,
    // consecutive lanes take consecutive FFTs of the batch
    float2* fy = team_fft<false, true>(b, b2, ny, a.logny, a.lognz, rp, 1, twy, tm);
    float2* fh = team_fft<false, true>(fy, fy == b ? b2 : b, nz, a.lognz, a.logny, 1, rp, twz, tm);
    o = fh == b ? b2 : b;
    if (kx == 0 || 2 * kx == a.nx) {
      // Hermitian part on a self-conjugate column: (kz, ky) pairs with (-kz, -ky)
      for (int i = tm.rank; i < ns; i += tm.size) {
        const int kz = i >> a.logny, ky = i & (ny - 1);
        const int mz = (nz - kz) & (nz - 1), my = (ny - ky) & (ny - 1);
        const int m = mz * ny + my;
        if (i > m) continue;
        float2* pu = fh + kz * rp + ky;
        float2* pv = fh + mz * rp + my;
        const float2 u = *pu, v = *pv;
        const float2 hpart = make_float2(__fmul_rn(0.5f, __fadd_rn(u.x, v.x)),
                                         __fmul_rn(0.5f, __fsub_rn(u.y, v.y)));
        *pu = hpart;
        *pv = make_float2(hpart.x, -hpart.y);
      }
      tm.sync();
    }
    for (int i = tm.rank; i < ns; i += tm.size) {
      const int pi = i + (i >> a.logny);
      const float2 s = st[i];
      const float2 t = tb[i];
      const float2 f_ = fh[pi];
      const float2 sn = make_float2(__fmaf_rn(t.x, s.x, __fmul_rn(t.y, f_.x)),
                                    __fmaf_rn(t.x, s.y, __fmul_rn(t.y, f_.y)));
      st[i] = sn;
      const float2 sc = make_float2(__fmul_rn(sn.x, a.inv_n), __fmul_rn(sn.y, a.inv_n));
      if (mode == 2) {
        a.state[base + i * rstride] = sn;
        a.work[base + i * rstride] = sc;
      } else {
        o[pi] = sc;
      }
    }
  } else {
    for (int i = tm.rank; i < ns; i += tm.size) {
      const float2 s = st[i];
      o[i + (i >> a.logny)] = make_float2(__fmul_rn(s.x, a.inv_n), __fmul_rn(s.y, a.inv_n));
    }
  }
  tm.sync();
  if (mode != 2) {
    float2* gz = team_fft<true, true>(o, o == b ? b2 : b, nz, a.lognz, a.logny, 1, rp, twz, tm);
    const float2* g = team_fft<true, true>(gz, gz == b ? b2 : b, ny, a.logny, a.lognz, rp, 1,
                                           twy, tm);
    float2* Wo = a.W + f * a.cs + (int64_t)kx * a.wk;
    for (int i = tm.rank; i < ns; i += tm.size) Wo[(int64_t)i * a.wr] = g[i + (i >> a.logny)];
  }
  tm.sync();
}

template <int MODEL>
__global__ void __launch_bounds__(kThreads) spectral_fused_kernel(FusedArgs a) {
  extern __shared__ float2 smem[];
  const Team rt = make_team(a.row_team), ct = make_team(a.col_team);
  const int rteams = blockDim.x / a.row_team, cteams = blockDim.x / a.col_team;
  const int ns = a.ny * a.nz;
  float2* twx = smem;
  float2* twy = twx + a.nx;
  float2* twz = twy + a.ny;
  // the two phases' FFT buffers share one region: rteams x rbuf or cteams x cbuf
  float2* bufs = twz + a.nz;
  const int bregion = rteams * a.rbuf > cteams * a.cbuf ? rteams * a.rbuf : cteams * a.cbuf;
  float2* res = bufs + bregion;  // cteams x cpt x (psi_hat, table) slabs
  float2* rb = bufs + (size_t)rt.index * a.rbuf;
  float2* cb = bufs + (size_t)ct.index * a.cbuf;
  float2* st = res + (size_t)ct.index * a.cpt * 2 * ns;
  float2* tb = st + (size_t)a.cpt * ns;
  for (int j = threadIdx.x; j < a.nx; j += blockDim.x) twx[j] = a.twx[j];
  for (int j = threadIdx.x; j < a.ny; j += blockDim.x) twy[j] = a.twy[j];
  for (int j = threadIdx.x; j < a.nz; j += blockDim.x) twz[j] = a.twz[j];
  const int gct = blockIdx.x * cteams + ct.index, nct = gridDim.x * cteams;
  // row tasks: the CTAs' warps (or warp-wide teams) in turn, so that a phase with fewer tasks
  // than teams spreads them over every CTA; a warp of narrower teams takes consecutive tasks
  const int rtpw = a.row_team < 32 ? 32 / a.row_team : 1;  // row teams per warp
  const int nrt = gridDim.x * rteams;
  const int rt0 = ((rt.index / rtpw) * gridDim.x + blockIdx.x) * rtpw;  // this warp's first
  const int col_tasks = a.nf * a.nxh;
  const int row_tasks = MODEL == PF_MODEL_C ? a.nrows : (a.nrows >> 1);
  for (int i = 0; i < a.cpt; ++i) {
    const int t = gct + i * nct;
    if (t >= col_tasks) break;
    const int64_t base = (t / a.nxh) * a.cs + t % a.nxh;
    for (int k = ct.rank; k < ns; k += ct.size) {
      st[(size_t)i * ns + k] = a.state[base + (int64_t)k * a.nxh];
      tb[(size_t)i * ns + k] = a.table[base + (int64_t)k * a.nxh];
    }
  }
  __syncthreads();
  for (int i = 0; i < a.cpt; ++i) {
    const int t = gct + i * nct;
    if (t >= col_tasks) break;
    slab_task(a, t / a.nxh, t % a.nxh, 0, st + (size_t)i * ns, tb + (size_t)i * ns, cb,
              cb + a.cbuf / 2, twy, twz, ct);
  }
  if (!grid_barrier(a.bar, gridDim.x, a.budget)) return;
  for (int64_t step = 0; step < a.steps; ++step) {
    // teams narrower than a warp take their rounds together: the warp's first team decides
    // the trip count, and a team past the last task runs without touching W
    for (int t0 = rt0; t0 < row_tasks; t0 += nrt) {
      const int t = t0 + rt.index % rtpw;
      const bool valid = t < row_tasks;
      if (MODEL == PF_MODEL_C) row_task<MODEL>(a, 0, t, 1, t, valid, rb, rb + a.nx, twx, rt);
      else row_task<MODEL>(a, 0, 2 * t, 0, 2 * t + 1, valid, rb, rb + a.nx, twx, rt);
    }
    if (!grid_barrier(a.bar, gridDim.x, a.budget)) return;
    const int mode = step + 1 == a.steps ? 2 : 1;
    for (int i = 0; i < a.cpt; ++i) {
      const int t = gct + i * nct;
      if (t >= col_tasks) break;
      slab_task(a, t / a.nxh, t % a.nxh, mode, st + (size_t)i * ns, tb + (size_t)i * ns, cb,
                cb + a.cbuf / 2, twy, twz, ct);
    }
    if (mode == 1 && !grid_barrier(a.bar, gridDim.x, a.budget)) return;
  }
}

bool is_pow2(int64_t n) { return n > 0 && (n & (n - 1)) == 0; }

int ilog2(int64_t n) {
  int l = 0;
  while ((int64_t)1 << l < n) ++l;
  return l;
}

// Launch shape. For each CTA width (128 .. 1024 threads): per phase, the team size that gives
// one radix-8 butterfly per thread and pass, halved while that phase's tasks would need more
// than one round on the SMs; CTAs for the larger phase (at most one per SM, which keeps the
// grid barrier short); the slabs each slab team owns; and the shared memory that takes. The
// width whose phases need the fewest butterfly rounds per thread (task rounds times
// butterflies per thread) wins, the narrowest on a tie: warps that share an SM's issue slots
// lengthen every task's dependent chain. Where a width's slab teams do not fit, they are
// widened (fewer per CTA) until they do.
struct FusedShape {
  int threads, blocks, row_team, col_team, cpt, rbuf, cbuf;
  int rounds;  // the longer phase's task rounds per team
  size_t smem;
};

// Teams wider than a warp synchronise on named barriers 1 .. 15 (0 is the CTA's), so a CTA
// holds at most 15 of them: a 64-thread team in a 1024-thread CTA becomes a warp.
int team_for(int64_t n, int64_t tasks, int sms, int threads, int min_size = 32) {
  int64_t size = n / 8;
  if (size < min_size) size = min_size;
  if (size > threads) size = threads;
  while (size > 32 && (tasks + threads / size - 1) / (threads / size) > sms) size >>= 1;
  while (size > 32 && threads / size > 15) size >>= 1;
  return (int)size;
}

struct FusedDims {
  int64_t nx, ny, nz;
};

FusedDims fused_dims(const pf_spectral_s* s) {
  if (s->dim == 3) return {s->d[2], s->d[1], s->d[0]};
  return {s->d[1], s->d[0], 1};
}

FusedShape fused_shape_for(const pf_spectral_s* s, int sms, int threads, int col_team = 0) {
  const FusedDims d = fused_dims(s);
  const int64_t ns = d.ny * d.nz;  // values of a slab, and x-rows of a field
  const int64_t col_tasks = s->nf * (d.nx / 2 + 1);
  const int64_t row_tasks = s->model == PF_MODEL_C ? ns : ns / 2;
  FusedShape f{};
  f.threads = threads;
  // 3D: 8- or 16-lane teams for short rows (measured: Model C 64^3 22.2 -> 18.3 us per step);
  // 2D grids keep warp-wide teams (64^2 and 128^2 measured 0.6-1.0 us faster with them)
  f.row_team = team_for(d.nx, row_tasks, sms, f.threads, s->dim == 3 ? 8 : 32);
  f.col_team = col_team > 0 ? col_team : team_for(ns, col_tasks, sms, f.threads);
  const int64_t rteams = f.threads / f.row_team, cteams = f.threads / f.col_team;
  // row work counted in warps (a narrower team shares its warp's issue slots), so that short
  // rows still spread over as many SMs as warp-wide teams would
  const int64_t rwarps = f.threads / 32;
  const int64_t rtasks_per_warp = f.row_team < 32 ? 32 / f.row_team : 1;
  int64_t blocks = (row_tasks + rwarps * rtasks_per_warp - 1) / (rwarps * rtasks_per_warp);
  if (f.row_team < 32) blocks = std::max(blocks, (row_tasks + rwarps - 1) / rwarps);
  const int64_t cblocks = (col_tasks + cteams - 1) / cteams;
  if (cblocks > blocks) blocks = cblocks;
  if (blocks > sms) blocks = sms;
  f.blocks = (int)blocks;
  f.cpt = (int)((col_tasks + blocks * cteams - 1) / (blocks * cteams));
  f.rbuf = (int)(2 * d.nx + 2);  // b [nx], b2 [nx + 2]: b2 first takes both half spectra
  f.cbuf = (int)(2 * d.nz * (d.ny + 1));  // two padded slabs: rows of ny + 1
  const int64_t region = std::max(rteams * f.rbuf, cteams * f.cbuf);
  f.smem = sizeof(float2) * (size_t)(d.nx + d.ny + d.nz + region + cteams * f.cpt * 2 * ns);
  const int64_t rrounds = (row_tasks + blocks * rteams - 1) / (blocks * rteams);
  const int64_t rb = (d.nx / 8 + f.row_team - 1) / f.row_team;  // butterflies per thread
  const int64_t cb = (ns / 8 + f.col_team - 1) / f.col_team;
  f.rounds = (int)(rrounds * std::max<int64_t>(rb, 1) + f.cpt * std::max<int64_t>(cb, 1));
  return f;
}

FusedShape fused_shape(const pf_spectral_s* s, int sms) {
  int optin = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    optin = 0;
  }
  FusedShape best = fused_shape_for(s, sms, 128);
  for (int threads : {256, 512, kThreads}) {
    FusedShape f = fused_shape_for(s, sms, threads);
    // wider slab teams (fewer per CTA) where their buffers and resident slabs do not fit
    while (f.smem > (size_t)optin && f.col_team < threads)
      f = fused_shape_for(s, sms, threads, 2 * f.col_team);
    const bool fits = f.smem <= (size_t)optin, best_fits = best.smem <= (size_t)optin;
    if ((fits && (!best_fits || f.rounds < best.rounds)) || (!fits && !best_fits && f.smem < best.smem))
      best = f;
  }
  return best;
}

template <int MODEL>
const void* fused_kernel_ptr() {
  return reinterpret_cast<const void*>(&spectral_fused_kernel<MODEL>);
}

const void* kernel_for(int model) {
  if (model == PF_MODEL_AC) return fused_kernel_ptr<PF_MODEL_AC>();
  if (model == PF_MODEL_CH) return fused_kernel_ptr<PF_MODEL_CH>();
  return fused_kernel_ptr<PF_MODEL_C>();
}

unsigned long long g_attr_mask[3] = {0, 0, 0};

}  // namespace

int device_limits(int* sms, int* smem_optin) {
  int dev = 0;
  PF_CUDA_TRY(cudaGetDevice(&dev));
  PF_CUDA_TRY(cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev));
  PF_CUDA_TRY(cudaDeviceGetAttribute(smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  return PF_OK;
}

bool spectral_fused_supported(const pf_spectral_s* s) {
  const FusedDims d = fused_dims(s);
  if (!(is_pow2(d.nx) && is_pow2(d.ny) && is_pow2(d.nz) && d.nx >= 4 && d.nx <= kMaxSide &&
        d.ny >= 2 && d.ny <= kMaxSide && d.nz <= kMaxSide))
    return false;
  if (s->dim == 3 && d.nz < 2) return false;
  int sms = 0, optin = 0;
  if (device_limits(&sms, &optin) != PF_OK) return false;
  return fused_shape(s, sms).smem <= (size_t)optin;
}

int spectral_fused_prepare(pf_spectral_s* s) {
  if (s->fused_blocks > 0) return PF_OK;
  if (!spectral_fused_supported(s))
    return invalid("the fused engine takes power-of-two sides (nx in [4, 1024]) whose (y, z) "
                   "slab fits in a CTA's shared memory");
  const FusedDims d = fused_dims(s);
  std::vector<float2> tw((size_t)(d.nx + d.ny + d.nz));
  size_t o = 0;
  for (int64_t n : {d.nx, d.ny, d.nz}) {
    for (int64_t j = 0; j < n; ++j) {
      const double t = -2.0 * 3.141592653589793 * (double)j / (double)n;
      tw[o++] = make_float2((float)std::cos(t), (float)std::sin(t));
    }
  }
  cudaError_t e = cudaMalloc(&s->twiddle, sizeof(float2) * tw.size());
  if (e == cudaSuccess) e = cudaMalloc(&s->d_bar, 4 * sizeof(unsigned int));
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("fused spectral engine: out of device memory");
    return PF_ERR_OOM;
  }
  PF_CUDA_TRY(cudaMemcpyAsync(s->twiddle, tw.data(), sizeof(float2) * tw.size(),
                              cudaMemcpyHostToDevice, s->stream));
  PF_CUDA_TRY(cudaMemsetAsync(s->d_bar, 0, 4 * sizeof(unsigned int), s->stream));
  PF_CUDA_TRY(cudaStreamSynchronize(s->stream));
  int sms = 0, optin = 0;
  if (int rc = device_limits(&sms, &optin)) return rc;
  const FusedShape f = fused_shape(s, sms);
  const int mi = s->model == PF_MODEL_AC ? 0 : (s->model == PF_MODEL_CH ? 1 : 2);
  const void* kern = kernel_for(s->model);
  int dev = 0;
  PF_CUDA_TRY(cudaGetDevice(&dev));
  // the limit is per kernel and device: set it once, to the device's opt-in maximum
  if (dev >= 64 || !(g_attr_mask[mi] & (1ull << dev))) {
    PF_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    if (dev < 64) g_attr_mask[mi] |= 1ull << dev;
  }
  int per_sm = 0;
  PF_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, f.threads, f.smem));
  if (per_sm < 1) return invalid("fused spectral engine: the kernel does not fit on an SM");
  s->fused_blocks = f.blocks;
  s->fused_threads = f.threads;
  s->fused_row_team = f.row_team;
  s->fused_col_team = f.col_team;
  s->fused_cpt = f.cpt;
  s->fused_rbuf = f.rbuf;
  s->fused_cbuf = f.cbuf;
  s->fused_smem = f.smem;
  return PF_OK;
}

int spectral_fused_run(pf_spectral_s* s, int64_t n_steps) {
  if (n_steps <= 0) return PF_OK;
  if (int rc = spectral_fused_prepare(s)) return rc;
  const FusedDims d = fused_dims(s);
  FusedArgs a{};
  a.state = s->spec;
  a.W = s->spec + s->nf * s->cs;
  a.work = s->work;
  a.table = s->table;
  a.twx = s->twiddle;
  a.twy = s->twiddle + d.nx;
  a.twz = s->twiddle + d.nx + d.ny;
  a.nx = (int)d.nx;
  a.ny = (int)d.ny;
  a.nz = (int)d.nz;
  a.nxh = (int)(d.nx / 2 + 1);
  a.lognx = ilog2(d.nx);
  a.logny = ilog2(d.ny);
  a.lognz = ilog2(d.nz);
  a.nf = s->nf;
  a.nrows = (int)(d.ny * d.nz);
  a.wr = s->dim == 3 ? 1 : a.nxh;
  a.wk = s->dim == 3 ? a.nrows : 1;
  a.rbuf = s->fused_rbuf;
  a.cbuf = s->fused_cbuf;
  a.row_team = s->fused_row_team;
  a.col_team = s->fused_col_team;
  a.cpt = s->fused_cpt;
  a.cs = s->cs;
  a.inv_n = (float)(1.0 / (double)s->nsite);
  a.k = nl_coeffs(s);
  a.steps = n_steps;
  a.bar = s->d_bar;
  a.budget = kWaitBudgetCycles;
  void* args[] = {&a};
  PF_CUDA_TRY(cudaLaunchCooperativeKernel(kernel_for(s->model), dim3(s->fused_blocks),
                                          dim3(s->fused_threads), args, s->fused_smem,
                                          s->stream));
  return PF_OK;
}

int spectral_fused_check(pf_spectral_s* s) {
  if (s->d_bar == nullptr) return PF_OK;
  unsigned int flag = 0;
  PF_CUDA_TRY(cudaMemcpyAsync(&flag, s->d_bar + 2, sizeof(unsigned int), cudaMemcpyDeviceToHost,
                              s->stream));
  PF_CUDA_TRY(cudaStreamSynchronize(s->stream));
  if (flag != 0) {
    PF_CUDA_TRY(cudaMemsetAsync(s->d_bar, 0, 4 * sizeof(unsigned int), s->stream));
    set_error("a grid barrier wait of the fused spectral engine ran out; the state is invalid");
    return PF_ERR_TIMEOUT;
  }
  return PF_OK;
}

void spectral_fused_release(pf_spectral_s* s) {
  cudaFree(s->twiddle);
  cudaFree(s->d_bar);
  s->twiddle = nullptr;
  s->d_bar = nullptr;
}

}  // namespace pf
