// FP32 + FP64-fix-up instantiation of the pair-integral kernels (float outputs).
#include "integrals_impl.cuh"

namespace sph2d {

sph2d_status integrals_fp32(Ctx* c, int kernel, int md, const IntArgs& a) {
  return dispatch_integrals<float>(c, kernel, md, a);
}

sph2d_status pairs_fp32(Ctx* c, const double* pairs, int64_t P, int kernel, double H, int deg,
                        unsigned long long* nfix, void* out) {
  return dispatch_pairs<float>(c, pairs, P, kernel, H, deg, nfix, out);
}

}  // namespace sph2d
