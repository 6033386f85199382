// dlopen-based cuFFT loader (see pf_cufft.h).
#include <dlfcn.h>

#include <mutex>

#include "pf_cufft.h"
#include "pf_internal.h"

#ifndef PF_CUDA_LIBDIR
#define PF_CUDA_LIBDIR ""
#endif

namespace pf {

namespace {

std::once_flag g_once;
CufftApi g_api{};
bool g_ok = false;
char g_why[256] = "";

template <class F>
bool sym(void* h, const char* name, F* out) {
  *out = reinterpret_cast<F>(dlsym(h, name));
  return *out != nullptr;
}

void load() {
  // The soname of the toolkit's cuFFT, then the toolkit this library was built against,
  // then the unversioned name.
  char built[512];
  snprintf(built, sizeof(built), "%s/libcufft.so.12", PF_CUDA_LIBDIR);
  const char* names[3] = {"libcufft.so.12", built, "libcufft.so"};
  void* h = nullptr;
  for (const char* n : names) {
    if (n[0] == '/' && PF_CUDA_LIBDIR[0] == '\0') continue;
    h = dlopen(n, RTLD_NOW | RTLD_LOCAL);
    if (h != nullptr) break;
  }
  if (h == nullptr) {
    snprintf(g_why, sizeof(g_why), "cuFFT (libcufft.so.12) could not be loaded: %s",
             dlerror());
    return;
  }
  bool ok = sym(h, "cufftCreate", &g_api.create) && sym(h, "cufftDestroy", &g_api.destroy) &&
            sym(h, "cufftSetStream", &g_api.set_stream) &&
            sym(h, "cufftSetAutoAllocation", &g_api.set_auto_allocation) &&
            sym(h, "cufftSetWorkArea", &g_api.set_work_area) &&
            sym(h, "cufftMakePlanMany64", &g_api.make_plan_many64) &&
            sym(h, "cufftExecR2C", &g_api.exec_r2c) && sym(h, "cufftExecC2R", &g_api.exec_c2r) &&
            sym(h, "cufftExecD2Z", &g_api.exec_d2z);
  if (!ok) {
    snprintf(g_why, sizeof(g_why), "cuFFT was loaded but lacks an expected entry point");
    return;
  }
  g_ok = true;
}

}  // namespace

const CufftApi* cufft_api() {
  std::call_once(g_once, load);
  if (!g_ok) {
    set_error("%s", g_why);
    return nullptr;
  }
  return &g_api;
}

int cufft_fail(cufftResult r, const char* what) {
  set_error("cuFFT error %d in %s", (int)r, what);
  return r == CUFFT_ALLOC_FAILED ? PF_ERR_OOM : PF_ERR_CUDA;
}

int cufft_plan(const CufftApi* api, cufftHandle* plan, int rank, const int64_t* d,
               cufftType type, int64_t batch, int64_t real_dist, int64_t cplx_dist,
               int auto_alloc, size_t* work_bytes) {
  // Axes of length 1 other than the last change neither layout nor result: leave them out
  // (the last, halved axis always stays).
  long long n[3], re[3], cx[3];
  long long nre = 1, ncx = 1;
  int r_eff = 0;
  for (int i = 0; i < rank; ++i) {
    if (d[i] == 1 && i != rank - 1) continue;
    n[r_eff] = re[r_eff] = cx[r_eff] = d[i];
    nre *= d[i];
    ++r_eff;
  }
  rank = r_eff;
  cx[rank - 1] = n[rank - 1] / 2 + 1;
  for (int i = 0; i < rank; ++i) ncx *= cx[i];
  if (real_dist > 0) nre = real_dist;
  if (cplx_dist > 0) ncx = cplx_dist;
  const bool forward = type == CUFFT_R2C || type == CUFFT_D2Z;
  *plan = -1;
  cufftResult r = api->create(plan);
  if (r != CUFFT_SUCCESS) {
    *plan = -1;
    return cufft_fail(r, "cufftCreate");
  }
  r = api->set_auto_allocation(*plan, auto_alloc);
  size_t ws = 0;
  if (r == CUFFT_SUCCESS)
    r = api->make_plan_many64(*plan, rank, n, forward ? re : cx, 1, forward ? nre : ncx,
                              forward ? cx : re, 1, forward ? ncx : nre, type, batch, &ws);
  if (r != CUFFT_SUCCESS) {
    api->destroy(*plan);
    *plan = -1;
    return cufft_fail(r, "cufftMakePlanMany64");
  }
  if (work_bytes) *work_bytes = ws;
  return PF_OK;
}

}  // namespace pf
