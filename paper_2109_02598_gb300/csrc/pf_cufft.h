// cuFFT, loaded on first use with dlopen so that the rest of the library loads and runs on
// a machine without it. Only the types come from cufft.h; no symbol is linked.
#pragma once

#include <cufft.h>

#include <cstddef>
#include <cstdint>

namespace pf {

struct CufftApi {
  cufftResult (*create)(cufftHandle*);
  cufftResult (*destroy)(cufftHandle);
  cufftResult (*set_stream)(cufftHandle, cudaStream_t);
  cufftResult (*set_auto_allocation)(cufftHandle, int);
  cufftResult (*set_work_area)(cufftHandle, void*);
  cufftResult (*make_plan_many64)(cufftHandle, int, long long*, long long*, long long,
                                  long long, long long*, long long, long long, cufftType,
                                  long long, size_t*);
  cufftResult (*exec_r2c)(cufftHandle, cufftReal*, cufftComplex*);
  cufftResult (*exec_c2r)(cufftHandle, cufftComplex*, cufftReal*);
  cufftResult (*exec_d2z)(cufftHandle, cufftDoubleReal*, cufftDoubleComplex*);
};

// The loaded API, or nullptr after setting the error message (PF_ERR_CUDA to report).
const CufftApi* cufft_api();

// Report a failed cuFFT call; returns PF_ERR_CUDA (or PF_ERR_OOM for an allocation failure).
int cufft_fail(cufftResult r, const char* what);

// A batched real<->complex plan over the C-order dims d[0..rank) (last fastest), each
// transform dense: real arrays of prod(d) values and half spectra of
// prod(d[:-1]) * (d[-1]/2 + 1) values, `batch` of each, real_dist and cplx_dist elements
// apart (0 = back to back). Requires d[rank-1] >= 2. With auto_alloc == 0 the caller sets the work area;
// *work_bytes receives its size. On failure the handle is destroyed and -1 stored.
int cufft_plan(const CufftApi* api, cufftHandle* plan, int rank, const int64_t* d,
               cufftType type, int64_t batch, int64_t real_dist, int64_t cplx_dist,
               int auto_alloc, size_t* work_bytes);

}  // namespace pf
