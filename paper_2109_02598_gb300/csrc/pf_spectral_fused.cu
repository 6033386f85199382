// Fused engine of the semi-implicit spectral solver (Sec. 2.4.2) for 2D grids whose sides are
// powers of two (4 .. 1024): every step of a pf_spectral_step call runs inside one
// cooperative launch, with this file's own radix-2 FFTs in shared memory.
//
// The state psi_hat [ny][nxh] (and the tables) are those of the cuFFT engine; W [ny][nxh]
// per field (the f_hat slices of spec) carries the data between the two phases of a step:
//   row phase     per row: the inverse transform along x of W's half spectrum, the nonlinear
//                 terms, the forward transform along x, back into W. Two real rows share one
//                 complex FFT: rows y and y+1 of a one-field model, or psi and m of one row in
//                 Model C (whose nonlinear terms need both at the same site);
//   column phase  per column kx: the forward transform along y of W -> f_hat; on the
//                 self-conjugate columns (kx = 0, nx/2) its Hermitian part; the update
//                 psi_hat <- A psi_hat + (B N) f_hat; and the inverse transform along y of
//                 psi_hat / N back into W for the next row phase.
// Each column team owns fixed columns for the whole launch and keeps their psi_hat and (A, B N) in
// shared memory: a prologue loads them and fills W from psi_hat; the last step writes
// psi_hat and work = psi_hat / N (as the cuFFT engine leaves them) back to global memory
// instead of the inverse transform. The phases are separated by a grid barrier (release /
// acquire atomics) whose waits are bounded by a clock budget: on timeout a CTA sets the
// error word and returns, so the launch always ends.
//
// A task (a row pair, or a column) is done by a team of 32, 64, 128 or 256 threads of a
// CTA, chosen per phase so that each thread does one radix-4 butterfly per pass where the
// tasks still fit in one round on the SMs; a team synchronises on its own named barrier.
// The FFTs are Stockham passes (radix 4, then one radix-2 pass for an odd power of two)
// between two shared-memory buffers of max(nx, ny) complex values per team: natural order in
// and out, no bit reversal, and every thread loads all of a butterfly's inputs before it
// computes.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "pf_spectral.h"
#include "pf_tma.cuh"

namespace pf {
int invalid(const char* fmt, ...);

namespace {

constexpr int kThreads = 256;  // the widest CTA; grids of sides <= 256 use 128 threads
constexpr int kMaxSide = 1024;

struct FusedArgs {
  float2* state;  // [nf][cs]
  float2* W;      // [nf][cs]
  float2* work;   // [nf][cs]
  const float2* table;
  const float2* twx;  // W_nx^j, j < nx
  const float2* twy;  // W_ny^j, j < ny
  int nx, ny, nxh, lognx, logny, nf, nmax;
  int row_team, col_team;  // threads per task in the row and column phases
  int cpt;                 // columns owned per column team
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

// The threads that share one task: `size` threads (a multiple of 32) of one CTA, the
// `index`-th such group; teams wider than a warp synchronise on named barrier index + 1.
struct Team {
  int size, rank, index;
  __device__ __forceinline__ void sync() const {
    if (size == 32) __syncwarp();
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

// One Stockham pass of radix R over n points (stride ns so far): butterfly j < n/R takes
// in[j + r n/R], twiddles it by W_{ns R}^{(j mod ns) r}, and writes its R-point DFT to
// out[(j - j mod ns) R + j mod ns + r ns]. tw holds W_n^i = exp(-2 pi i i / n), i < n; INV
// conjugates every twiddle (the inverse transform, unnormalised).
template <int R, bool INV>
__device__ __forceinline__ void stockham_pass(const float2* __restrict__ in,
                                              float2* __restrict__ out, int n, int ns,
                                              const float2* __restrict__ tw, const Team& tm) {
  const int q = n / R;
  const int tws = n / (ns * R);
#pragma unroll 2
  for (int j = tm.rank; j < q; j += tm.size) {
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = in[j + r * q];
    const int k = j & (ns - 1);
#pragma unroll
    for (int r = 1; r < R; ++r) {
      float2 w = tw[(k * r * tws) & (n - 1)];
      if (INV) w.y = -w.y;
      v[r] = cmul(w, v[r]);
    }
    const int base = (j - k) * R + k;
    if (R == 2) {
      out[base] = make_float2(__fadd_rn(v[0].x, v[1].x), __fadd_rn(v[0].y, v[1].y));
      out[base + ns] = make_float2(__fsub_rn(v[0].x, v[1].x), __fsub_rn(v[0].y, v[1].y));
    } else {
      const float2 a0 = make_float2(__fadd_rn(v[0].x, v[2].x), __fadd_rn(v[0].y, v[2].y));
      const float2 a1 = make_float2(__fsub_rn(v[0].x, v[2].x), __fsub_rn(v[0].y, v[2].y));
      const float2 a2 = make_float2(__fadd_rn(v[1].x, v[3].x), __fadd_rn(v[1].y, v[3].y));
      const float2 d = make_float2(__fsub_rn(v[1].x, v[3].x), __fsub_rn(v[1].y, v[3].y));
      // (v1 - v3) times -i (forward) or +i (inverse)
      const float2 a3 = INV ? make_float2(-d.y, d.x) : make_float2(d.y, -d.x);
      out[base] = make_float2(__fadd_rn(a0.x, a2.x), __fadd_rn(a0.y, a2.y));
      out[base + ns] = make_float2(__fadd_rn(a1.x, a3.x), __fadd_rn(a1.y, a3.y));
      out[base + 2 * ns] = make_float2(__fsub_rn(a0.x, a2.x), __fsub_rn(a0.y, a2.y));
      out[base + 3 * ns] = make_float2(__fsub_rn(a1.x, a3.x), __fsub_rn(a1.y, a3.y));
    }
  }
}

// FFT of the n = 2^logn points in b by one team, natural order in and out; b and b2 are
// used in turn and the result is in the returned buffer (the other one is free).
template <bool INV>
__device__ __forceinline__ float2* team_fft(float2* b, float2* b2, int n, int logn,
                                            const float2* tw, const Team& tm) {
  float2* in = b;
  float2* out = b2;
  int ns = 1;
  for (int p = 0; p < (logn >> 1); ++p) {
    stockham_pass<4, INV>(in, out, n, ns, tw, tm);
    tm.sync();
    float2* t = in;
    in = out;
    out = t;
    ns <<= 2;
  }
  if (logn & 1) {
    stockham_pass<2, INV>(in, out, n, ns, tw, tm);
    tm.sync();
    in = out;
  }
  return in;
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

// Row task: two real rows (field f1 row y1, field f2 row y2) whose half spectra are in W.
template <int MODEL>
__device__ __forceinline__ void row_task(const FusedArgs& a, int f1, int y1, int f2, int y2,
                                         float2* b, float2* b2, const float2* twx,
                                         const Team& tm) {
  const int nx = a.nx, nh = nx >> 1;
  const float2* X1 = a.W + f1 * a.cs + (int64_t)y1 * a.nxh;
  const float2* X2 = a.W + f2 * a.cs + (int64_t)y2 * a.nxh;
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
  float2* z = team_fft<true>(b, b2, nx, a.lognx, twx, tm);
  float2* other = z == b ? b2 : b;
  for (int k = tm.rank; k < nx; k += tm.size) {
    float2 v = z[k];
    nl_pair<MODEL>(v, a.k);
    z[k] = v;
  }
  tm.sync();
  const float2* Y = team_fft<false>(z, other, nx, a.lognx, twx, tm);
  float2* F1 = a.W + f1 * a.cs + (int64_t)y1 * a.nxh;
  float2* F2 = a.W + f2 * a.cs + (int64_t)y2 * a.nxh;
  for (int k = tm.rank; k <= nh; k += tm.size) {
    const float2 y = Y[k];
    const float2 r = Y[(nx - k) & (nx - 1)];  // Y(-k); conj taken below
    const float2 s = make_float2(__fadd_rn(y.x, r.x), __fsub_rn(y.y, r.y));  // Y + conj Y(-k)
    const float2 d = make_float2(__fsub_rn(y.x, r.x), __fadd_rn(y.y, r.y));  // Y - conj Y(-k)
    F1[k] = make_float2(__fmul_rn(0.5f, s.x), __fmul_rn(0.5f, s.y));
    F2[k] = make_float2(__fmul_rn(0.5f, d.y), __fmul_rn(-0.5f, d.x));  // -i d / 2
  }
  tm.sync();
}

// Column task (field f, column kx) with the column's psi_hat in st and (A, B N) in tb
// (shared memory, natural order). mode 0: prologue (W <- inverse_y(psi_hat / N)); mode 1:
// full step; mode 2: last step (psi_hat and work = psi_hat / N to global memory, no inverse
// transform).
__device__ __forceinline__ void column_task(const FusedArgs& a, int f, int kx, int mode,
                                            float2* st, const float2* tb, float2* b, float2* b2,
                                            const float2* twy, const Team& tm) {
  const int ny = a.ny;
  const int64_t base = f * a.cs + kx;
  const int64_t rstride = a.nxh;
  float2* o = b;  // receives psi_hat / N for the inverse transform
  if (mode != 0) {
    for (int y = tm.rank; y < ny; y += tm.size) b[y] = a.W[base + y * rstride];
    tm.sync();
    float2* fh = team_fft<false>(b, b2, ny, a.logny, twy, tm);
    o = fh == b ? b2 : b;
    if (kx == 0 || 2 * kx == a.nx) {
      for (int ky = tm.rank; ky <= (ny >> 1); ky += tm.size) {
        const int km = (ny - ky) & (ny - 1);
        const float2 u = fh[ky], v = fh[km];
        const float2 hpart = make_float2(__fmul_rn(0.5f, __fadd_rn(u.x, v.x)),
                                         __fmul_rn(0.5f, __fsub_rn(u.y, v.y)));
        fh[ky] = hpart;
        fh[km] = make_float2(hpart.x, -hpart.y);
      }
      tm.sync();
    }
    for (int ky = tm.rank; ky < ny; ky += tm.size) {
      const float2 s = st[ky];
      const float2 t = tb[ky];
      const float2 f_ = fh[ky];
      const float2 sn = make_float2(__fmaf_rn(t.x, s.x, __fmul_rn(t.y, f_.x)),
                                    __fmaf_rn(t.x, s.y, __fmul_rn(t.y, f_.y)));
      st[ky] = sn;
      const float2 sc = make_float2(__fmul_rn(sn.x, a.inv_n), __fmul_rn(sn.y, a.inv_n));
      if (mode == 2) {
        a.state[base + ky * rstride] = sn;
        a.work[base + ky * rstride] = sc;
      } else {
        o[ky] = sc;
      }
    }
  } else {
    for (int ky = tm.rank; ky < ny; ky += tm.size) {
      const float2 s = st[ky];
      o[ky] = make_float2(__fmul_rn(s.x, a.inv_n), __fmul_rn(s.y, a.inv_n));
    }
  }
  tm.sync();
  if (mode != 2) {
    const float2* g = team_fft<true>(o, o == b ? b2 : b, ny, a.logny, twy, tm);
    for (int y = tm.rank; y < ny; y += tm.size) a.W[base + y * rstride] = g[y];
  }
  tm.sync();
}

template <int MODEL>
__global__ void __launch_bounds__(kThreads) spectral_fused_kernel(FusedArgs a) {
  extern __shared__ float2 smem[];
  const Team rt = make_team(a.row_team), ct = make_team(a.col_team);
  const int rteams = blockDim.x / a.row_team, cteams = blockDim.x / a.col_team;
  const int bteams = rteams > cteams ? rteams : cteams;
  float2* twx = smem;
  float2* twy = twx + a.nx;
  float2* bufs = twy + a.ny;  // bteams x 2 x nmax: each team's FFT buffers (per phase)
  float2* res = bufs + (size_t)bteams * 2 * a.nmax;  // cteams x cpt x (psi_hat, table) columns
  float2* rb = bufs + (size_t)rt.index * 2 * a.nmax;
  float2* cb = bufs + (size_t)ct.index * 2 * a.nmax;
  float2* st = res + (size_t)ct.index * a.cpt * 2 * a.ny;
  float2* tb = st + (size_t)a.cpt * a.ny;
  for (int j = threadIdx.x; j < a.nx; j += blockDim.x) twx[j] = a.twx[j];
  for (int j = threadIdx.x; j < a.ny; j += blockDim.x) twy[j] = a.twy[j];
  const int gct = blockIdx.x * cteams + ct.index, nct = gridDim.x * cteams;
  const int grt = blockIdx.x * rteams + rt.index, nrt = gridDim.x * rteams;
  const int col_tasks = a.nf * a.nxh;
  const int row_tasks = MODEL == PF_MODEL_C ? a.ny : (a.ny >> 1);
  for (int i = 0; i < a.cpt; ++i) {
    const int t = gct + i * nct;
    if (t >= col_tasks) break;
    const int64_t base = (t / a.nxh) * a.cs + t % a.nxh;
    for (int ky = ct.rank; ky < a.ny; ky += ct.size) {
      st[(size_t)i * a.ny + ky] = a.state[base + (int64_t)ky * a.nxh];
      tb[(size_t)i * a.ny + ky] = a.table[base + (int64_t)ky * a.nxh];
    }
  }
  __syncthreads();
  for (int i = 0; i < a.cpt; ++i) {
    const int t = gct + i * nct;
    if (t >= col_tasks) break;
    column_task(a, t / a.nxh, t % a.nxh, 0, st + (size_t)i * a.ny, tb + (size_t)i * a.ny, cb,
                cb + a.nmax, twy, ct);
  }
  if (!grid_barrier(a.bar, gridDim.x, a.budget)) return;
  for (int64_t step = 0; step < a.steps; ++step) {
    for (int t = grt; t < row_tasks; t += nrt) {
      if (MODEL == PF_MODEL_C) row_task<MODEL>(a, 0, t, 1, t, rb, rb + a.nmax, twx, rt);
      else row_task<MODEL>(a, 0, 2 * t, 0, 2 * t + 1, rb, rb + a.nmax, twx, rt);
    }
    if (!grid_barrier(a.bar, gridDim.x, a.budget)) return;
    const int mode = step + 1 == a.steps ? 2 : 1;
    for (int i = 0; i < a.cpt; ++i) {
      const int t = gct + i * nct;
      if (t >= col_tasks) break;
      column_task(a, t / a.nxh, t % a.nxh, mode, st + (size_t)i * a.ny, tb + (size_t)i * a.ny,
                  cb, cb + a.nmax, twy, ct);
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

// Launch shape. The CTA width: 128 threads for grids of sides <= 256 (their teams are one
// warp, and warps that share an SM's issue slots lengthen every task's dependent chain),
// else 256. Per phase, the team size that gives one radix-4 butterfly per thread and pass,
// halved while that phase's tasks would need more than one round on the SMs; CTAs for the
// larger phase (at most one per SM, which keeps the grid barrier short); the columns each
// column team owns; and the shared memory that takes.
struct FusedShape {
  int threads, blocks, row_team, col_team, cpt;
  size_t smem;
};

int team_for(int64_t n, int64_t tasks, int sms, int threads) {
  int64_t size = n / 4;
  if (size < 32) size = 32;
  if (size > threads) size = threads;
  while (size > 32 && (tasks + threads / size - 1) / (threads / size) > sms) size >>= 1;
  return (int)size;
}

FusedShape fused_shape(const pf_spectral_s* s, int sms) {
  const int64_t nx = s->d[1], ny = s->d[0];
  const int64_t nmax = nx > ny ? nx : ny;
  const int64_t col_tasks = s->nf * (nx / 2 + 1);
  const int64_t row_tasks = s->model == PF_MODEL_C ? ny : ny / 2;
  FusedShape f{};
  f.threads = nmax <= 256 ? 128 : kThreads;
  f.row_team = team_for(nx, row_tasks, sms, f.threads);
  f.col_team = team_for(ny, col_tasks, sms, f.threads);
  const int64_t rteams = f.threads / f.row_team, cteams = f.threads / f.col_team;
  int64_t blocks = (row_tasks + rteams - 1) / rteams;
  const int64_t cblocks = (col_tasks + cteams - 1) / cteams;
  if (cblocks > blocks) blocks = cblocks;
  if (blocks > sms) blocks = sms;
  f.blocks = (int)blocks;
  f.cpt = (int)((col_tasks + blocks * cteams - 1) / (blocks * cteams));
  const int64_t bteams = rteams > cteams ? rteams : cteams;
  f.smem = sizeof(float2) * (size_t)(nx + ny + bteams * 2 * nmax + cteams * f.cpt * 2 * ny);
  return f;
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
  if (s->dim != 2) return false;
  const int64_t nx = s->d[1], ny = s->d[0];
  if (!(is_pow2(nx) && is_pow2(ny) && nx >= 4 && ny >= 2 && nx <= kMaxSide && ny <= kMaxSide))
    return false;
  int sms = 0, optin = 0;
  if (device_limits(&sms, &optin) != PF_OK) return false;
  return fused_shape(s, sms).smem <= (size_t)optin;
}

int spectral_fused_prepare(pf_spectral_s* s) {
  if (s->fused_blocks > 0) return PF_OK;
  if (!spectral_fused_supported(s))
    return invalid("the fused engine takes 2D grids with power-of-two sides in [4, 1024]");
  const int64_t nx = s->d[1], ny = s->d[0];
  std::vector<float2> tw((size_t)(nx + ny));
  for (int64_t j = 0; j < nx; ++j) {
    const double t = -2.0 * 3.141592653589793 * (double)j / (double)nx;
    tw[(size_t)j] = make_float2((float)std::cos(t), (float)std::sin(t));
  }
  for (int64_t j = 0; j < ny; ++j) {
    const double t = -2.0 * 3.141592653589793 * (double)j / (double)ny;
    tw[(size_t)(nx + j)] = make_float2((float)std::cos(t), (float)std::sin(t));
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
  s->fused_smem = f.smem;
  return PF_OK;
}

int spectral_fused_run(pf_spectral_s* s, int64_t n_steps) {
  if (n_steps <= 0) return PF_OK;
  if (int rc = spectral_fused_prepare(s)) return rc;
  const int64_t nx = s->d[1], ny = s->d[0];
  FusedArgs a{};
  a.state = s->spec;
  a.W = s->spec + s->nf * s->cs;
  a.work = s->work;
  a.table = s->table;
  a.twx = s->twiddle;
  a.twy = s->twiddle + nx;
  a.nx = (int)nx;
  a.ny = (int)ny;
  a.nxh = (int)(nx / 2 + 1);
  a.lognx = ilog2(nx);
  a.logny = ilog2(ny);
  a.nf = s->nf;
  a.nmax = (int)(nx > ny ? nx : ny);
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
