// Staging of a tile's rows into shared memory with 16-byte cp.async copies, for the kernels
// that take four consecutive sites per thread: rows y0-1 .. y0+ht-2 of columns x0-4 ..
// x0+ws-5 of every field (a row of ws floats; ws - 8 output columns plus four halo columns a
// side, so each row's interior starts 16-byte aligned in shared memory and in the field).
#pragma once

#include "pf_internal.h"
#include "pf_tma.cuh"

namespace pf {

// Copy the rows of every field at plane offset zoff into dst (rows ws floats apart, fields pl
// floats apart): a 16-byte copy where a group of four columns lies inside the row, else four
// periodic 4-byte copies. Issues the copies and returns: the caller commits or waits.
template <int NF>
__device__ __forceinline__ void stage_rows4(const FieldPtrs& in, const Geom& g, int x0, int y0,
                                            int64_t zoff, int ws, int ht, int pl, float* dst,
                                            int nthreads) {
  const int ch4 = ws / 4;
  for (int i = threadIdx.x; i < ht * ch4; i += nthreads) {
    const int r = i / ch4, j = i - r * ch4;
    const int gy = wrap_index(y0 - 1 + r, g.ny);
    const int gx = x0 - 4 + 4 * j;
    const int64_t row = zoff + (int64_t)gy * g.pitch;
    float* d = dst + r * ws + 4 * j;
    if (gx >= 0 && gx + 3 < g.nx) {
#pragma unroll
      for (int f = 0; f < NF; ++f) cp_async16(d + f * pl, in.f[f] + row + gx);
    } else {
#pragma unroll
      for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int c = 0; c < 4; ++c)
          cp_async4(d + f * pl + c, in.f[f] + row + wrap_index(gx + c, g.nx));
    }
  }
}

// CTAs of a kernel that the device holds at once (cached per device; 0 on error).
template <class KernelT>
int resident_ctas(KernelT kernel, int threads, size_t smem, int* cache) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev >= 64) return 0;
  if (cache[dev] == 0) {
    int b = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, threads, smem) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    cache[dev] = (b > 0 ? b : 1) * (sms > 0 ? sms : 1);
  }
  return cache[dev];
}

// Planes per z-chunk for a grid of tiles_xy columns: as many chunks as fit the device in one
// wave beside the other columns (a partial second wave leaves most SMs idle), at least four
// planes each.
inline int one_wave_tz(int nz, int tiles_xy, int resident) {
  int nzc = resident > 0 ? resident / tiles_xy : 1;
  nzc = nzc < 1 ? 1 : nzc;
  const int max_chunks = nz / 4 > 1 ? nz / 4 : 1;
  nzc = nzc > max_chunks ? max_chunks : nzc;
  return (nz + nzc - 1) / nzc;
}

}  // namespace pf
