// FP64 instantiation of the pair-integral kernels (all steps in IEEE double).
#include "integrals_impl.cuh"

namespace sph2d {

sph2d_status integrals_fp64(Ctx* c, int kernel, int md, const IntArgs& a) {
  return dispatch_integrals<double>(c, kernel, md, a);
}

sph2d_status pairs_fp64(Ctx* c, const double* pairs, int64_t P, int kernel, double H, int deg,
                        unsigned long long* nfix, void* out) {
  return dispatch_pairs<double>(c, pairs, P, kernel, H, deg, nfix, out);
}

}  // namespace sph2d
