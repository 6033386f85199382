// 3D forward-Euler step, z-streaming (Sec. 2.4.1 solver, Sec. 2.2.2 7-, 19- and 27-point
// stencils, Sec. 3 models).  General kernels for any grid size: a CTA owns a TX x TY column
// of the xy plane and a chunk of tz planes; it streams through z keeping a ring of planes
// with a periodic xy halo in shared memory, so every input value is fetched from HBM once
// per CTA plus the halo.  Allen-Cahn and Gray-Scott: four planes (z-1, z, z+1 and z+2 in
// flight), four sites per thread.  Model B keeps three phi planes (halo 2) and three mu
// planes (halo 1); mu is computed on chip and never stored.  Model C keeps both of its
// fields in the phi planes and the chemical potential of m in the mu planes.
#include "pf_stage.cuh"

namespace pf {

namespace {

constexpr int kNT3 = 256;

template <int MODEL, int TX, int TY>
struct Cfg3 {
  static constexpr int NF = ModelTraits<MODEL>::NF;
  static constexpr int R = ModelTraits<MODEL>::R;
  // phi planes (halo R)
  static constexpr int W = TX + 2 * R;
  static constexpr int HT = TY + 2 * R;
  static constexpr int PL = W * HT;
  // mu planes (Model B only, halo 1)
  static constexpr int W1 = TX + 2;
  static constexpr int HT1 = TY + 2;
  static constexpr int PL1 = W1 * HT1;
  // ring of phi planes: three (z-1, z, z+1), four for Model C, whose psi needs plane z-1
  // while plane z+2 is already staged for the chemical potential of m
  static constexpr int NPH = (MODEL == PF_MODEL_C) ? 4 : 3;
  static constexpr int SMEM_FLOATS = NPH * NF * PL + (R == 2 ? 3 * PL1 : 0);
};

// Stage plane z (periodic) of every field into ring slot `slot`: 4-byte cp.async copies (the
// rows start at x0 - R, so they are not 16-byte aligned), all of a thread's copies issued
// before one wait; the caller's barrier then makes every thread's visible.
template <class C>
__device__ __forceinline__ void load_plane3d(const FieldPtrs& in, const Geom& g, int x0,
                                             int y0, int z, int slot, float* sm) {
  const int64_t zoff = (int64_t)wrap_index(z, g.nz) * g.plane;
  for (int i = threadIdx.x; i < C::PL; i += kNT3) {
    const int r = i / C::W;
    const int c = i - r * C::W;
    const int gy = wrap_index(y0 - C::R + r, g.ny);
    const int gx = wrap_index(x0 - C::R + c, g.nx);
    const int64_t off = zoff + (int64_t)gy * g.pitch + gx;
#pragma unroll
    for (int f = 0; f < C::NF; ++f) cp_async4(sm + (slot * C::NF + f) * C::PL + i, in.f[f] + off);
  }
  cp_async_wait_all();
}

// 3D Laplacian at position p of a staged plane c (row width W) with the planes b below and
// a above: 7-point (ST = PF_ST_STD), isotropic 19-point (faces and edges, PF_ST_ISO) or
// isotropic 27-point (faces, edges and corners, PF_ST_ISO27).
template <int ST>
__device__ __forceinline__ float lap3d_planes(const float* b, const float* c, const float* a,
                                              int p, int W, float scale) {
  if constexpr (ST == PF_ST_STD) {
    return lap3d(c[p], c[p - 1], c[p + 1], c[p - W], c[p + W], b[p], a[p], scale);
  } else {
    const float faces = __fadd_rn(__fadd_rn(__fadd_rn(c[p - 1], c[p + 1]),
                                            __fadd_rn(c[p - W], c[p + W])),
                                  __fadd_rn(b[p], a[p]));
    const float exy = __fadd_rn(__fadd_rn(c[p - W - 1], c[p - W + 1]),
                                __fadd_rn(c[p + W - 1], c[p + W + 1]));
    const float eb = __fadd_rn(__fadd_rn(b[p - 1], b[p + 1]), __fadd_rn(b[p - W], b[p + W]));
    const float ea = __fadd_rn(__fadd_rn(a[p - 1], a[p + 1]), __fadd_rn(a[p - W], a[p + W]));
    const float edges = __fadd_rn(exy, __fadd_rn(eb, ea));
    if constexpr (ST == PF_ST_ISO) {
      return lap3d_iso(c[p], faces, edges, scale);
    } else {
      const float cb = __fadd_rn(__fadd_rn(b[p - W - 1], b[p - W + 1]),
                                 __fadd_rn(b[p + W - 1], b[p + W + 1]));
      const float ca = __fadd_rn(__fadd_rn(a[p - W - 1], a[p - W + 1]),
                                 __fadd_rn(a[p + W - 1], a[p + W + 1]));
      return lap3d_iso27(c[p], faces, edges, __fadd_rn(cb, ca), scale);
    }
  }
}

// AC and Gray-Scott (stencil radius 1): a CTA of 128 threads streams its TX x TY column
// through a four-plane ring in shared memory (rows with four halo columns a side, staged by
// 16-byte copies two planes ahead), and each thread takes four consecutive sites of a row.
// When a plane enters, each thread reads its three rows once and forms, per site and field,
// the plane's sums in the order every stencil uses them: F = the site, E = (x-1 + x+1) +
// (y-1 + y+1) and, for the 19- and 27-point stencils, C = (the four in-plane diagonals).
// The sums of planes z-1, z and z+1 stay in registers, in slots named by plane mod 3 (the
// plane loop unrolled by three, so no register moves), and the Laplacian of plane z is
//   7-point:  E(z) + (F(z-1) + F(z+1)), less 6 c;
//   19-point: faces = E(z) + (F(z-1) + F(z+1)), edges = C(z) + (E(z-1) + E(z+1));
//   27-point: and corners = C(z-1) + C(z+1);
// the operands and order of lap3d_planes, so the bits of every other 3D path.
constexpr int kNT31 = 128;

template <int MODEL, int TX, int TY>
struct Cfg31 {
  static constexpr int NF = ModelTraits<MODEL>::NF;
  static constexpr int WS = TX + 8, HT = TY + 2;  // columns x0-4 .. x0+TX+3, rows y0-1 .. y0+TY
  static constexpr int PL = WS * HT;              // floats per field and plane
  static constexpr int SLOT = NF * PL;
  static_assert((TX / 4) * TY == kNT31, "one group of four sites per thread and plane");
};

// The values of one row around a thread's four sites: v[0] = x - 1, v[1..4] the sites,
// v[5] = x + 4. The x-edges come from the neighbouring lanes of the same row by shuffle and
// from shared memory only at the row's ends (first / last: the thread's group is the first /
// last of its tile row): scalar loads at a stride of four floats would meet four rows of a
// warp in the same eight banks. Every lane of the warp calls it.
__device__ __forceinline__ void row6(const float* r, float (&v)[6], bool first, bool last) {
  const float4 q = *reinterpret_cast<const float4*>(r);
  const float sl = __shfl_up_sync(0xffffffffu, q.w, 1);
  const float sr = __shfl_down_sync(0xffffffffu, q.x, 1);
  v[0] = first ? r[-1] : sl;
  v[1] = q.x;
  v[2] = q.y;
  v[3] = q.z;
  v[4] = q.w;
  v[5] = last ? r[4] : sr;
}
__device__ __forceinline__ void row4(const float* r, float (&v)[6]) {
  const float4 q = *reinterpret_cast<const float4*>(r);
  v[1] = q.x;
  v[2] = q.y;
  v[3] = q.z;
  v[4] = q.w;
}

template <int MODEL, int TX, int TY, int ST>
struct R1Run {
  using Cf = Cfg31<MODEL, TX, TY>;
  static constexpr int NF = Cf::NF, WS = Cf::WS, PL = Cf::PL, SLOT = Cf::SLOT;
  static constexpr bool kDiag = ST != PF_ST_STD;  // the 19- and 27-point stencils need C
  float F[3][NF][4], E[3][NF][4], C[3][NF][kDiag ? 4 : 1];

  const float* sm;
  FieldOut out;
  Geom g;
  int x0, y0, z0, z1, gy, gx, p;
  bool first, last, active;

  // The sums of the plane in ring slot rs into window slot W.
  template <int W>
  __device__ __forceinline__ void enter(int rs) {
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const float* q = sm + rs * SLOT + f * PL + p;
      float r0[6], r1[6], r2[6];  // rows y - 1, y, y + 1
      row6(q, r1, first, last);
      if constexpr (kDiag) {
        row6(q - WS, r0, first, last);
        row6(q + WS, r2, first, last);
      } else {
        row4(q - WS, r0);
        row4(q + WS, r2);
      }
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int x = s + 1;
        F[W][f][s] = r1[x];
        E[W][f][s] = __fadd_rn(__fadd_rn(r1[x - 1], r1[x + 1]), __fadd_rn(r0[x], r2[x]));
        if constexpr (kDiag)
          C[W][f][s] = __fadd_rn(__fadd_rn(r0[x - 1], r0[x + 1]), __fadd_rn(r2[x - 1], r2[x + 1]));
      }
    }
  }

  // Laplacian of site s of field f on plane z from window slots Bs (z-1), Cs (z), As (z+1).
  template <int Bs, int Cs, int As>
  __device__ __forceinline__ float lap(int f, int s, float scale) const {
    const float c = F[Cs][f][s];
    const float faces = __fadd_rn(E[Cs][f][s], __fadd_rn(F[Bs][f][s], F[As][f][s]));
    if constexpr (ST == PF_ST_STD) {
      return __fmul_rn(__fmaf_rn(-6.0f, c, faces), scale);  // lap3d
    } else {
      const float edges = __fadd_rn(C[Cs][f][s], __fadd_rn(E[Bs][f][s], E[As][f][s]));
      if constexpr (ST == PF_ST_ISO)
        return lap3d_iso(c, faces, edges, scale);
      else
        return lap3d_iso27(c, faces, edges, __fadd_rn(C[Bs][f][s], C[As][f][s]), scale);
    }
  }

  // Plane z at phase P (window slot of plane z-1): wait for plane z+1, stage plane z+3, take
  // plane z+1's sums, update plane z.
  template <int P>
  __device__ __forceinline__ void iteration(int z, const FieldPtrs& in, const ModelParams& m) {
    constexpr int Bs = P, Cs = (P + 1) % 3, As = (P + 2) % 3;
    const int i = z - z0;
    cp_async_wait_group<1>();  // plane z + 1 has landed (plane z + 2 may be in flight)
    __syncthreads();           // ... for every thread; and every read of plane z - 1's ring
                               // slot (in the iteration before the last) is done
    if (z + 3 <= z1)
      stage_rows4<NF>(in, g, x0, y0, (int64_t)wrap_index(z + 3, g.nz) * g.plane, WS, Cf::HT, PL,
                      const_cast<float*>(sm) + (i & 3) * SLOT, kNT31);
    cp_async_commit();  // possibly empty: one group per iteration
    enter<As>((i + 2) & 3);
    float res[NF][4];
    if constexpr (MODEL == PF_MODEL_AC) {
#pragma unroll
      for (int s = 0; s < 4; ++s)
        res[0][s] = ac_update(F[Cs][0][s], lap<Bs, Cs, As>(0, s, m.lap_scale), m);
    } else {
#pragma unroll
      for (int s = 0; s < 4; ++s)
        gs_update(F[Cs][0][s], F[Cs][1][s], lap<Bs, Cs, As>(0, s, m.lap_scale),
                  lap<Bs, Cs, As>(1, s, m.lap_scale), m, res[0][s], res[1][s]);
    }
    if (active) {
      const int64_t off = (int64_t)z * g.plane + (int64_t)gy * g.pitch + gx;
      if (gx + 3 < g.nx) {
#pragma unroll
        for (int f = 0; f < NF; ++f)
          *reinterpret_cast<float4*>(out.f[f] + off) =
              make_float4(res[f][0], res[f][1], res[f][2], res[f][3]);
      } else {
#pragma unroll
        for (int f = 0; f < NF; ++f)
#pragma unroll
          for (int e = 0; e < 4; ++e)
            if (gx + e < g.nx) out.f[f][off + e] = res[f][e];
      }
    }
  }
};

template <int MODEL, int TX, int TY, int ST>
__global__ void __launch_bounds__(kNT31) fe3d_r1_kernel(FieldPtrs in, FieldOut out, Geom g,
                                                        ModelParams m, int tz) {
  using Run = R1Run<MODEL, TX, TY, ST>;
  using Cf = typename Run::Cf;
  constexpr int NF = Cf::NF, WS = Cf::WS, PL = Cf::PL, SLOT = Cf::SLOT;
  extern __shared__ __align__(16) float smem[];
  Run r;
  r.sm = smem;
  r.out = out;
  r.g = g;
  r.x0 = blockIdx.x * TX;
  r.y0 = blockIdx.y * TY;
  r.z0 = blockIdx.z * tz;
  r.z1 = min(r.z0 + tz, g.nz);
  const int rr = threadIdx.x / (TX / 4), j = threadIdx.x - rr * (TX / 4);
  r.gy = r.y0 + rr;
  r.gx = r.x0 + 4 * j;
  r.active = r.gy < g.ny && r.gx < g.nx;  // lanes past the grid compute but store nothing
  r.first = j == 0;
  r.last = j == TX / 4 - 1;
  r.p = (rr + 1) * WS + 4 + 4 * j;
  canary_fill(smem, (size_t)4 * SLOT);
  // plane q sits in ring slot (q - z0 + 1) % 4: planes z0 - 1 .. z0 + 2 first, one group each
  // (z0 + 2 is needed only when the chunk has a second plane)
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (k < 3 || r.z0 + 1 < r.z1)
      stage_rows4<NF>(in, g, r.x0, r.y0, (int64_t)wrap_index(r.z0 - 1 + k, g.nz) * g.plane, WS,
                      Cf::HT, PL, smem + k * SLOT, kNT31);
    cp_async_commit();
  }
  cp_async_wait_group<2>();  // planes z0 - 1 and z0
  __syncthreads();
  r.template enter<0>(0);  // window slot of plane q: (q - z0 + 1) % 3
  r.template enter<1>(1);
  int z = r.z0;
  for (; z + 3 <= r.z1; z += 3) {
    r.template iteration<0>(z, in, m);
    r.template iteration<1>(z + 1, in, m);
    r.template iteration<2>(z + 2, in, m);
  }
  if (z < r.z1) r.template iteration<0>(z, in, m);
  if (z + 1 < r.z1) r.template iteration<1>(z + 1, in, m);
  cp_async_wait_all();  // nothing in flight at exit
}

// Model B and Model C: mu planes computed on chip from the staged phi planes (halo 2).
// Model B: mu = c2 phi^3 - c1 phi - lap phi of its one field.  Model C: the chemical
// potential of m (field 1), coupled to psi (field 0).
template <int MODEL, int TX, int TY, int ST>
__device__ __forceinline__ void r2_mu_plane(const float* pb, const float* pc, const float* pa,
                                            float* mu, const ModelParams& m) {
  using C = Cfg3<MODEL, TX, TY>;
  constexpr int W = C::W;
  constexpr int PL = C::PL;
  constexpr int F = C::NF - 1;  // the field whose chemical potential is needed
  for (int i = threadIdx.x; i < C::PL1; i += kNT3) {
    const int r1 = i / C::W1;
    const int c1 = i - r1 * C::W1;
    const int p = (r1 + 1) * W + (c1 + 1);  // position in the phi plane (halo 2)
    const float v = pc[F * PL + p];
    const float l = lap3d_planes<ST>(pb + F * PL, pc + F * PL, pa + F * PL, p, W, m.lap_scale);
    if constexpr (MODEL == PF_MODEL_CH)
      mu[i] = ch_mu(v, l, m);
    else
      mu[i] = mc_mu(pc[p], v, l, m);
  }
}

template <int MODEL, int TX, int TY, int ST>
__global__ void __launch_bounds__(kNT3) fe3d_r2_kernel(FieldPtrs in, FieldOut out, Geom g,
                                                       ModelParams m, int tz) {
  using C = Cfg3<MODEL, TX, TY>;
  constexpr int NF = C::NF;
  constexpr int W = C::W;
  constexpr int PL = C::PL;
  constexpr int W1 = C::W1;
  constexpr int PL1 = C::PL1;
  extern __shared__ __align__(16) float sm[];
  constexpr int NPH = C::NPH;
  float* ph = sm;                  // NPH slots of NF phi planes, pslot(p) = (p - z0 + 8) % NPH
  float* mu = sm + NPH * NF * PL;  // 3 mu slots, slot(p) = (p - z0 + 6) % 3
  const int x0 = blockIdx.x * TX;
  const int y0 = blockIdx.y * TY;
  const int z0 = blockIdx.z * tz;
  const int z1 = min(z0 + tz, g.nz);
  auto slot = [&](int p) { return (p - z0 + 6) % 3; };
  auto pslot = [&](int p) { return (p - z0 + 8) % NPH; };
  auto plane = [&](int p) { return ph + pslot(p) * NF * PL; };
  // prologue: mu(z0-1) from phi(z0-2..z0), then mu(z0) from phi(z0-1..z0+1)
  canary_fill(sm, C::SMEM_FLOATS);
  load_plane3d<C>(in, g, x0, y0, z0 - 2, pslot(z0 - 2), ph);
  load_plane3d<C>(in, g, x0, y0, z0 - 1, pslot(z0 - 1), ph);
  load_plane3d<C>(in, g, x0, y0, z0, pslot(z0), ph);
  __syncthreads();
  r2_mu_plane<MODEL, TX, TY, ST>(plane(z0 - 2), plane(z0 - 1), plane(z0), mu + slot(z0 - 1) * PL1, m);
  __syncthreads();
  load_plane3d<C>(in, g, x0, y0, z0 + 1, pslot(z0 + 1), ph);
  __syncthreads();
  r2_mu_plane<MODEL, TX, TY, ST>(plane(z0 - 1), plane(z0), plane(z0 + 1), mu + slot(z0) * PL1, m);
  __syncthreads();
  for (int z = z0; z < z1; ++z) {
    load_plane3d<C>(in, g, x0, y0, z + 2, pslot(z + 2), ph);
    __syncthreads();
    r2_mu_plane<MODEL, TX, TY, ST>(plane(z), plane(z + 1), plane(z + 2), mu + slot(z + 1) * PL1, m);
    __syncthreads();
    const float* mb = mu + slot(z - 1) * PL1;
    const float* mc = mu + slot(z) * PL1;
    const float* ma = mu + slot(z + 1) * PL1;
    const float* pb = plane(z - 1);
    const float* pc = plane(z);
    const float* pa = plane(z + 1);
    const int64_t zoff = (int64_t)z * g.plane;
    for (int i = threadIdx.x; i < TX * TY; i += kNT3) {
      const int rr = i / TX;
      const int cc = i - rr * TX;
      const int q = (rr + 1) * W1 + (cc + 1);  // mu plane position
      const int p = (rr + 2) * W + (cc + 2);   // phi plane position
      const float l = lap3d_planes<ST>(mb, mc, ma, q, W1, m.lap_scale);
      const int gx = x0 + cc;
      const int gy = y0 + rr;
      if (gx >= g.nx || gy >= g.ny) continue;
      const int64_t off = zoff + (int64_t)gy * g.pitch + gx;
      if constexpr (MODEL == PF_MODEL_CH) {
        out.f[0][off] = ch_update(pc[p], l, m);
      } else {
        const float ps = pc[p];
        const float lp = lap3d_planes<ST>(pb, pc, pa, p, W, m.lap_scale);
        float psn, mn;
        mc_update(ps, pc[PL + p], lp, l, m, psn, mn);
        out.f[0][off] = psn;
        out.f[1][off] = mn;
      }
    }
    __syncthreads();
  }
}

int choose_tz(const Geom& g, int tiles_xy) {
  // enough CTAs for several waves on 152 SMs; small grids take short chunks (down to 4
  // planes) and accept the prologue planes they re-read, large grids keep long chunks
  int tz = g.nz;
  while (tz > 4 && (int64_t)tiles_xy * ((g.nz + tz - 1) / tz) < 4 * 152) tz = (tz + 1) / 2;
  return tz;
}

template <int MODEL, int TX, int TY, int ST>
cudaError_t launch3(const Geom& g, FieldPtrs in, FieldOut out, const ModelParams& m,
                    cudaStream_t s) {
  using C = Cfg3<MODEL, TX, TY>;
  const size_t smem = sizeof(float) * C::SMEM_FLOATS;
  static unsigned long long attr_mask = 0;  // per instantiation and device
  const int bx = (g.nx + TX - 1) / TX, by = (g.ny + TY - 1) / TY;
  const int tz = choose_tz(g, bx * by);
  dim3 grid(bx, by, (g.nz + tz - 1) / tz);
  if constexpr (ModelTraits<MODEL>::R == 2) {
    cudaError_t e = ensure_smem_attr(fe3d_r2_kernel<MODEL, TX, TY, ST>, smem, &attr_mask);
    if (e != cudaSuccess) return e;
    fe3d_r2_kernel<MODEL, TX, TY, ST><<<grid, kNT3, smem, s>>>(in, out, g, m, tz);
  } else {
    using C1 = Cfg31<MODEL, TX, TY>;
    const size_t smem1 = sizeof(float) * 4 * C1::SLOT;
    cudaError_t e = ensure_smem_attr(fe3d_r1_kernel<MODEL, TX, TY, ST>, smem1, &attr_mask);
    if (e != cudaSuccess) return e;
    static int resident[64] = {};  // per device
    const int tz1 = one_wave_tz(
        g.nz, bx * by, resident_ctas(fe3d_r1_kernel<MODEL, TX, TY, ST>, kNT31, smem1, resident));
    const dim3 grid1(bx, by, (g.nz + tz1 - 1) / tz1);
    fe3d_r1_kernel<MODEL, TX, TY, ST><<<grid1, kNT31, smem1, s>>>(in, out, g, m, tz1);
  }
  return cudaGetLastError();
}

template <int MODEL>
cudaError_t launch3_tile(int tile_id, const Geom& g, FieldPtrs in, FieldOut out,
                         const ModelParams& m, cudaStream_t s, int stencil) {
  if (stencil == PF_ST_ISO) {
    if (tile_id == 0) return launch3<MODEL, 32, 16, PF_ST_ISO>(g, in, out, m, s);
    return launch3<MODEL, 64, 8, PF_ST_ISO>(g, in, out, m, s);
  }
  if (stencil == PF_ST_ISO27) {
    if (tile_id == 0) return launch3<MODEL, 32, 16, PF_ST_ISO27>(g, in, out, m, s);
    return launch3<MODEL, 64, 8, PF_ST_ISO27>(g, in, out, m, s);
  }
  if (stencil != PF_ST_STD) return cudaErrorInvalidValue;
  if (tile_id == 0) return launch3<MODEL, 32, 16, PF_ST_STD>(g, in, out, m, s);
  return launch3<MODEL, 64, 8, PF_ST_STD>(g, in, out, m, s);
}

}  // namespace

void tile3d_shape(int tile_id, int* tx, int* ty) {
  static const int s[kNumTiles3D][2] = {{32, 16}, {64, 8},   {64, 16}, {128, 8},
                                        {128, 16}, {256, 8}, {32, 8}};
  *tx = s[tile_id][0];
  *ty = s[tile_id][1];
}

int tile3d_id(int tx, int ty) {
  for (int i = 0; i < kNumTiles3D; ++i) {
    int a, b;
    tile3d_shape(i, &a, &b);
    if (a == tx && b == ty) return i;
  }
  return -1;
}

cudaError_t launch_fe3d(int model, int tile_id, const Geom& g, FieldPtrs in, FieldOut out,
                        const ModelParams& m, cudaStream_t s, int stencil) {
  if (tile_id < 0 || tile_id >= kFirstTmaTile3D) return cudaErrorInvalidValue;
  switch (model) {
    case PF_MODEL_AC: return launch3_tile<PF_MODEL_AC>(tile_id, g, in, out, m, s, stencil);
    case PF_MODEL_CH: return launch3_tile<PF_MODEL_CH>(tile_id, g, in, out, m, s, stencil);
    case PF_MODEL_GS: return launch3_tile<PF_MODEL_GS>(tile_id, g, in, out, m, s, stencil);
    case PF_MODEL_C: return launch3_tile<PF_MODEL_C>(tile_id, g, in, out, m, s, stencil);
  }
  return cudaErrorInvalidValue;
}

}  // namespace pf
