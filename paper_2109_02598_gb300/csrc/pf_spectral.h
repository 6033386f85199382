// Internal state of a spectral solver, shared by its two engines: cuFFT plus this library's
// pointwise kernels (pf_spectral.cu) and the fused engine (pf_spectral_fused.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "pf_cufft.h"
#include "pf_internal.h"

struct pf_spectral_s {
  uint32_t magic;
  int dim, model, nf;
  int64_t d[3];       // C-order dims: (ny, nx) or (nz, ny, nx)
  int64_t nsite, nk;  // real sites and half-spectrum modes per field
  int64_t rs, cs;     // padded per-field strides of the real (floats) and complex arrays
  double h, dt, coeffs[5];
  float cf[5];        // coefficients rounded to float32 once
  cudaStream_t stream = nullptr;
  cudaStream_t capture = nullptr;
  float2* spec = nullptr;
  float2* work = nullptr;
  float2* table = nullptr;
  float* real = nullptr;
  void* fft_work = nullptr;
  cufftHandle c2r_all = -1, r2c_all = -1, r2c_one = -1, c2r_one = -1;
  cudaGraphExec_t chunk = nullptr;
  bool graph_failed = false;
  const pf::CufftApi* api = nullptr;
  // fused engine
  int engine = 0;                   // PF_SPECTRAL_ENGINE_*
  bool fused_ok = false;            // the fused engine takes this grid (set at creation)
  float2* twiddle = nullptr;        // W_nx^j (j < nx), W_ny^j (j < ny), W_nz^j (j < nz)
  unsigned int* d_bar = nullptr;    // grid barrier: count, generation; then the error flag
  int fused_blocks = 0;             // CTAs of the cooperative launch (0: not prepared)
  int fused_threads = 0;            // threads per CTA
  int fused_row_team = 0;           // threads per row task
  int fused_col_team = 0;           // threads per slab task
  int fused_cpt = 0;                // slabs each slab team owns
  int fused_rbuf = 0, fused_cbuf = 0;  // float2s of a row / slab team's FFT buffers
  size_t fused_smem = 0;            // dynamic shared memory per CTA
};


namespace pf {

struct NlCoeffs {
  float c[4];
};

// Nonlinear terms in place (Sec. 3 equations, the part left after the linear split).
template <int MODEL>
__device__ __forceinline__ void nonlinear_site(float& p, float& m, const float* c) {
  if (MODEL == PF_MODEL_AC) {  // -c2 psi^3
    p = __fmul_rn(__fmul_rn(c[0], p), __fmul_rn(p, p));
  } else if (MODEL == PF_MODEL_CH) {  // c2 psi^3
    p = __fmul_rn(__fmul_rn(c[0], p), __fmul_rn(p, p));
  } else {  // psi: psi (2 c5 m - c2 psi^2);  m: c4 m^3 - c5 psi^2
    const float p2 = __fmul_rn(p, p);
    const float fp = __fmul_rn(p, __fmaf_rn(c[1], m, __fmul_rn(c[0], p2)));
    const float fm = __fmaf_rn(__fmul_rn(c[2], __fmul_rn(m, m)), m, __fmul_rn(c[3], p2));
    p = fp;
    m = fm;
  }
}

// Coefficients of nonlinear_site as the kernels take them.
inline NlCoeffs nl_coeffs(const pf_spectral_s* s) {
  NlCoeffs k{};
  if (s->model == PF_MODEL_AC) {
    k.c[0] = -s->cf[1];  // -c2
  } else if (s->model == PF_MODEL_CH) {
    k.c[0] = s->cf[1];  // c2
  } else {
    k.c[0] = -s->cf[1];                    // -c2
    k.c[1] = (float)(2.0 * s->coeffs[4]);  // 2 c5
    k.c[2] = s->cf[3];                     // c4
    k.c[3] = -s->cf[4];                    // -c5
  }
  return k;
}

// The fused engine (pf_spectral_fused.cu).
bool spectral_fused_supported(const pf_spectral_s* s);
int spectral_fused_prepare(pf_spectral_s* s);  // twiddles, barrier words; idempotent
int spectral_fused_run(pf_spectral_s* s, int64_t n_steps);
int spectral_fused_check(pf_spectral_s* s);    // PF_ERR_TIMEOUT if a barrier wait ran out
void spectral_fused_release(pf_spectral_s* s);

}  // namespace pf
