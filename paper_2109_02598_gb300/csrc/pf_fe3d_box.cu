// 3D forward-Euler steps of the radius-2 models (Models B and C, Sec. 3; Sec. 2.4.1 solver
// with the 7-point Laplacian of Sec. 2.2.2) for small grids: one CTA per box of
// BX x BY x BZ sites and K = 1 or 2 steps per launch, no streaming.
//
// The z-streaming kernels walk a column of planes one at a time, a barrier per plane; on a
// grid as small as 64^3 the columns are short and that serial walk is the step's time. Here a
// CTA stages its whole box with a halo of 2 K (the periodic images included) in shared
// memory and then, per step, computes the chemical potential on a region one site wider than
// the step's result and the step's result on a region that shrinks by two sites per step
// until the box itself is left: one wait for the copies and a barrier per stage. The halo is
// recomputed by neighbouring boxes instead of exchanged. Per site the arithmetic is that of
// the other kernels (lap3d with the same operands in the same order, ch_mu / ch_update,
// mc_mu / mc_update), so the result is the same bits.
//
// Staging: columns x0 - 4 .. x0 + BX + 3 (whole 16-byte groups, x0 a multiple of 4; a halo of
// four covers both depths) of rows y0 - 2K .. y0 + BY + 2K - 1 of planes z0 - 2K .. z0 + BZ +
// 2K - 1, every field, as 16-byte cp.async copies; with nx % 4 == 0 a group wraps as a whole,
// so the periodic images are aligned too.
#include "pf_internal.h"
#include "pf_model.cuh"
#include "pf_tma.cuh"

namespace pf {

namespace {

constexpr int kBX = 32, kBY = 8, kBZ = 8;  // output box

// A region of the box with halo hx in x and h in y and z: sites (x, y, z) relative to the box
// origin, x in [-hx, kBX + hx), y and z in [-h, kB* + h), x fastest.
template <int HX, int H>
struct Region {
  static constexpr int X = kBX + 2 * HX, Y = kBY + 2 * H, Z = kBZ + 2 * H;
  static constexpr int ROW = X, PL = X * Y, SIZE = X * Y * Z;
  static __device__ __forceinline__ int at(int x, int y, int z) {
    return (z + H) * PL + (y + H) * ROW + (x + HX);
  }
};

template <int MODEL, int K>
struct BoxCfg {
  static constexpr int NF = ModelTraits<MODEL>::NF;
  static constexpr int THREADS = K == 1 ? 512 : 1024;
  using S0 = Region<4, 2 * K>;          // staged state
  using M0 = Region<2 * K - 1, 2 * K - 1>;  // chemical potential of the staged state
  using S1 = Region<2, 2>;              // state after one step (K = 2)
  using M1 = Region<1, 1>;              // its chemical potential (K = 2; in M0's space)
  static constexpr int SMEM_FLOATS =
      NF * S0::SIZE + M0::SIZE + (K == 2 ? NF * S1::SIZE : 0);
  static_assert(MODEL == PF_MODEL_CH || MODEL == PF_MODEL_C, "radius-2 models");
  static_assert(K == 1 || K == 2, "depth 1 or 2");
};

// Chemical potential on region RM from the state in region RS (NF fields, field f at f * fs):
// Model B of phi, Model C of m (field 1) coupled to psi (field 0).
template <int MODEL, int THREADS, class RM, class RS>
__device__ __forceinline__ void box_mu(const float* st, int fs, float* mu, const ModelParams& m) {
  constexpr int F = ModelTraits<MODEL>::NF - 1;
  const float* c = st + F * fs;
  for (int i = threadIdx.x; i < RM::SIZE; i += THREADS) {
    const int x = i % RM::X - (RM::X - kBX) / 2;
    const int y = (i / RM::X) % RM::Y - (RM::Y - kBY) / 2;
    const int z = i / RM::PL - (RM::Z - kBZ) / 2;
    const int p = RS::at(x, y, z);
    const float l = lap3d(c[p], c[p - 1], c[p + 1], c[p - RS::ROW], c[p + RS::ROW],
                          c[p - RS::PL], c[p + RS::PL], m.lap_scale);
    if constexpr (MODEL == PF_MODEL_CH)
      mu[i] = ch_mu(c[p], l, m);
    else
      mu[i] = mc_mu(st[p], c[p], l, m);
  }
}

// One step on region RO from the chemical potential in RM and the state in RS; emit(i, x, y,
// z, v) takes site i of RO and its NF new values.
template <int MODEL, int THREADS, class RO, class RM, class RS, class Emit>
__device__ __forceinline__ void box_update(const float* st, int fs, const float* mu,
                                           const ModelParams& m, Emit&& emit) {
  for (int i = threadIdx.x; i < RO::SIZE; i += THREADS) {
    const int x = i % RO::X - (RO::X - kBX) / 2;
    const int y = (i / RO::X) % RO::Y - (RO::Y - kBY) / 2;
    const int z = i / RO::PL - (RO::Z - kBZ) / 2;
    const int q = RM::at(x, y, z);
    const float lm = lap3d(mu[q], mu[q - 1], mu[q + 1], mu[q - RM::ROW], mu[q + RM::ROW],
                           mu[q - RM::PL], mu[q + RM::PL], m.lap_scale);
    const int p = RS::at(x, y, z);
    float v[2];
    if constexpr (MODEL == PF_MODEL_CH) {
      v[0] = ch_update(st[p], lm, m);
    } else {
      const float lp = lap3d(st[p], st[p - 1], st[p + 1], st[p - RS::ROW], st[p + RS::ROW],
                             st[p - RS::PL], st[p + RS::PL], m.lap_scale);
      mc_update(st[p], st[fs + p], lp, lm, m, v[0], v[1]);
    }
    emit(i, x, y, z, v);
  }
}

template <int MODEL, int K>
__global__ void __launch_bounds__(BoxCfg<MODEL, K>::THREADS)
    fe3d_box_kernel(FieldPtrs in, FieldOut out, Geom g, ModelParams m) {
  using B = BoxCfg<MODEL, K>;
  using S0 = typename B::S0;
  using M0 = typename B::M0;
  constexpr int NF = B::NF;
  constexpr int T = B::THREADS;
  extern __shared__ __align__(16) float sm[];
  float* st = sm;                  // staged state, field f at f * S0::SIZE
  float* mu = sm + NF * S0::SIZE;  // chemical potential (of the staged state, then of step 1)
  float* s1 = mu + M0::SIZE;       // K = 2: state after one step, field f at f * S1::SIZE
  const int x0 = blockIdx.x * kBX, y0 = blockIdx.y * kBY, z0 = blockIdx.z * kBZ;
  canary_fill(sm, B::SMEM_FLOATS);

  // stage: (field, plane, row, 16-byte group)
  constexpr int G = S0::X / 4;
  for (int i = threadIdx.x; i < NF * S0::Z * S0::Y * G; i += T) {
    int t = i;
    const int j = t % G;
    t /= G;
    const int r = t % S0::Y;
    t /= S0::Y;
    const int q = t % S0::Z;
    const int f = t / S0::Z;
    const int gx = wrap_index(x0 - 4 + 4 * j, g.nx);  // a multiple of 4: the group wraps whole
    const int gy = wrap_index(y0 - 2 * K + r, g.ny);
    const int gz = wrap_index(z0 - 2 * K + q, g.nz);
    const float* src = (NF == 1 || f == 0) ? in.f[0] : in.f[1];  // no indexed parameter
    cp_async16(st + f * S0::SIZE + q * S0::PL + r * S0::ROW + 4 * j,
               src + (int64_t)gz * g.plane + (int64_t)gy * g.pitch + gx);
  }
  cp_async_wait_all();
  __syncthreads();

  // the last step's result goes to HBM (sites inside the grid)
  auto store = [&](int, int x, int y, int z, const float* v) {
    const int gx = x0 + x, gy = y0 + y, gz = z0 + z;
    if (gx >= g.nx || gy >= g.ny || gz >= g.nz) return;
    const int64_t off = (int64_t)gz * g.plane + (int64_t)gy * g.pitch + gx;
    out.f[0][off] = v[0];
    if constexpr (NF == 2) out.f[1][off] = v[1];
  };
  box_mu<MODEL, T, M0, S0>(st, S0::SIZE, mu, m);
  __syncthreads();
  if constexpr (K == 1) {
    box_update<MODEL, T, Region<0, 0>, M0, S0>(st, S0::SIZE, mu, m, store);
  } else {
    using S1 = typename B::S1;
    using M1 = typename B::M1;
    box_update<MODEL, T, S1, M0, S0>(st, S0::SIZE, mu, m,
                                     [&](int i, int, int, int, const float* v) {
                                       s1[i] = v[0];
                                       if constexpr (NF == 2) s1[S1::SIZE + i] = v[1];
                                     });
    __syncthreads();
    box_mu<MODEL, T, M1, S1>(s1, S1::SIZE, mu, m);
    __syncthreads();
    box_update<MODEL, T, Region<0, 0>, M1, S1>(s1, S1::SIZE, mu, m, store);
  }
}

template <int MODEL, int K>
cudaError_t launch_box(const Geom& g, FieldPtrs in, FieldOut out, const ModelParams& m,
                       cudaStream_t s) {
  using B = BoxCfg<MODEL, K>;
  const size_t smem = sizeof(float) * B::SMEM_FLOATS;
  static unsigned long long attr_mask = 0;  // per instantiation and device
  cudaError_t e = ensure_smem_attr(fe3d_box_kernel<MODEL, K>, smem, &attr_mask);
  if (e != cudaSuccess) return e;
  dim3 grid((g.nx + kBX - 1) / kBX, (g.ny + kBY - 1) / kBY, (g.nz + kBZ - 1) / kBZ);
  fe3d_box_kernel<MODEL, K><<<grid, B::THREADS, smem, s>>>(in, out, g, m);
  return cudaGetLastError();
}

}  // namespace

bool fe3d_box_supported(int model, int k, const Geom& g) {
  return (model == PF_MODEL_CH || model == PF_MODEL_C) && (k == 1 || k == 2) && g.dim == 3 &&
         g.nx % 4 == 0;
}

cudaError_t launch_fe3d_box(int model, int k, const Geom& g, FieldPtrs in, FieldOut out,
                            const ModelParams& m, cudaStream_t s) {
  if (!fe3d_box_supported(model, k, g)) return cudaErrorInvalidValue;
  if (model == PF_MODEL_CH)
    return k == 1 ? launch_box<PF_MODEL_CH, 1>(g, in, out, m, s)
                  : launch_box<PF_MODEL_CH, 2>(g, in, out, m, s);
  return k == 1 ? launch_box<PF_MODEL_C, 1>(g, in, out, m, s)
                : launch_box<PF_MODEL_C, 2>(g, in, out, m, s);
}

}  // namespace pf
