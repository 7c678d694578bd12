// Adjoint of the boundary integrals (filled in by the adjoint kernels).
#include "sph2d_internal.h"

namespace sph2d {

sph2d_status launch_backward(Ctx* c, int kernel, int mode, const void* d_gamma, void* d_particles,
                             void* d_tris) {
  (void)kernel; (void)mode; (void)d_gamma; (void)d_particles; (void)d_tris;
  return set_err(c, SPH2D_ERR_UNSUPPORTED, "backward not built yet");
}

}  // namespace sph2d
