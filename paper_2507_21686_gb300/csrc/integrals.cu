// Host side of the forward integral calls: argument packing and precision dispatch.
#include <cuda_runtime.h>

#include "integrals_impl.cuh"

namespace sph2d {

sph2d_status integrals_fp64(Ctx* c, int kernel, int md, const IntArgs& a);
sph2d_status integrals_fp32(Ctx* c, int kernel, int md, const IntArgs& a);
sph2d_status integrals_hybrid(Ctx* c, int kernel, int md, const IntArgs& a);
sph2d_status pairs_fp64(Ctx* c, const double* pairs, int64_t P, int kernel, double H, int deg,
                        unsigned long long* nfix, void* out);
sph2d_status pairs_fp32(Ctx* c, const double* pairs, int64_t P, int kernel, double H, int deg,
                        unsigned long long* nfix, void* out);

sph2d_status launch_integrals(Ctx* c, int kernel, int moment_degree, int mode, void* gamma,
                              void* grad, void* moments) {
  const Cells& cl = c->cells;
  IntArgs a;
  a.parts = reinterpret_cast<const float4*>(cl.particles);
  a.tris = cl.tris;
  a.pair_tri = static_cast<const int32_t*>(c->pair_tri.ptr);
  a.pair_pid = static_cast<const int32_t*>(c->pair_pid.ptr);
  a.pair_off = static_cast<const int64_t*>(c->pair_off.ptr);
  a.P = cl.P;
  a.N = cl.N;
  a.H = cl.H;
  a.invH = 1.0 / cl.H;
  a.C = kernel_C(kernel);
  a.gamma = gamma;
  a.grad = grad;
  a.mom = moments;
  a.nm = num_moments(moment_degree);
  a.slots = nullptr;
  sph2d_status s = ensure(c, c->host_flags_dev, 64);
  if (s != SPH2D_OK) return s;
  a.nfix = static_cast<unsigned long long*>(c->host_flags_dev.ptr);
  a.work = a.nfix + 1;                       // chunk counter of the pair kernels
  cudaError_t e = cudaMemsetAsync(a.nfix, 0, 2 * sizeof(unsigned long long), c->stream);
  if (e != cudaSuccess) return cuda_err(c, e, "memset");
  const int md = md_for(moment_degree);
  s = mode == SPH2D_FP64 ? integrals_fp64(c, kernel, md, a)
                         : (mode == SPH2D_FP32_HYBRID ? integrals_hybrid(c, kernel, md, a)
                                                      : integrals_fp32(c, kernel, md, a));
  if (s != SPH2D_OK) return s;
  e = cudaMemcpyAsync(c->pinned + 8, a.nfix, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                      c->stream);
  if (e != cudaSuccess) return cuda_err(c, e, "fixup count copy");
  c->stats.n_pairs = cl.P;
  c->stats.n_fallback = 0;
  c->fixup_pending = true;
  c->fallback_pending = mode == SPH2D_FP32_HYBRID;   // pinned[10]: pairs left to the closed form
  return SPH2D_OK;
}

sph2d_status launch_pair_integrals(Ctx* c, const double* pairs, int64_t P, int kernel, double H,
                                   int moment_degree, int mode, void* out) {
  sph2d_status s = ensure(c, c->host_flags_dev, 64);
  if (s != SPH2D_OK) return s;
  auto* nfix = static_cast<unsigned long long*>(c->host_flags_dev.ptr);
  cudaError_t e = cudaMemsetAsync(nfix, 0, sizeof(unsigned long long), c->stream);
  if (e != cudaSuccess) return cuda_err(c, e, "memset");
  s = mode == SPH2D_FP64 ? pairs_fp64(c, pairs, P, kernel, H, moment_degree, nfix, out)
                         : pairs_fp32(c, pairs, P, kernel, H, moment_degree, nfix, out);
  if (s != SPH2D_OK) return s;
  e = cudaMemcpyAsync(c->pinned + 8, nfix, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                      c->stream);
  if (e != cudaSuccess) return cuda_err(c, e, "fixup count copy");
  c->stats = sph2d_stats{};
  c->stats.n_pairs = P;
  c->fixup_pending = true;
  c->fallback_pending = false;
  return SPH2D_OK;
}

}  // namespace sph2d
