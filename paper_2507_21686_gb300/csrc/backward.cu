// Adjoint of the boundary integrals for a loss L(gamma).
//
//   dL/dx_i  = dL/dgamma_i * grad gamma_i          (the forward gradient, recomputed)
//   dL/dnu_j = sum_i dL/dgamma_i * d gamma_i / d nu_j
// where d gamma_i / d nu_j is the transport-theorem edge integral of pair_math.cuh.  The
// vertex gradients are summed triangle-major: the particle-major pair list is transposed into
// per-triangle particle lists, each sorted ascending, and one warp walks a triangle's list in
// that order and reduces with a fixed butterfly, so results do not depend on scheduling.
// Nothing from the forward call is stored: pair geometry is recomputed.
#include <cuda_runtime.h>

#include "integrals_impl.cuh"

namespace sph2d {

struct BwdArgs {
  const float4* parts;
  const float* tris;
  const int64_t* tri_off;
  const int32_t* tri_pid;
  int64_t M;
  double invH, C;
  const void* d_gamma;
  void* d_tris;
  unsigned long long* nfix;
};

// d gamma / d vertices of one pair in the mode's precision; returns 1 if FP64 was used
template <typename OT, int KID>
__device__ __forceinline__ int pair_vertex_grad(const BwdArgs& a, int pid, const float* t, OT* g) {
  return vertex_grad_pair<OT, KID>(a.parts[pid], t, a.invH, a.C, g);
}

template <typename OT, int KID>
__global__ void __launch_bounds__(128) vertex_grad_kernel(BwdArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  const OT* dg = static_cast<const OT*>(a.d_gamma);
  unsigned long long fixes = 0;
  for (int64_t t = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; t < a.M; t += nw) {
    OT acc[6] = {OT(0), OT(0), OT(0), OT(0), OT(0), OT(0)};
    const int64_t s0 = __ldg(a.tri_off + t), s1 = __ldg(a.tri_off + t + 1);
    const float* tp = a.tris + 6 * t;
    for (int64_t k = s0 + lane; k < s1; k += 32) {
      const int pid = __ldg(a.tri_pid + k);
      OT g[6];
      fixes += pair_vertex_grad<OT, KID>(a, pid, tp, g);
      const OT w = dg[pid];
#pragma unroll
      for (int i = 0; i < 6; ++i) acc[i] += w * g[i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
      for (int i = 0; i < 6; ++i) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], o);
    }
    if (lane == 0) {
      OT* out = static_cast<OT*>(a.d_tris) + 6 * t;
#pragma unroll
      for (int i = 0; i < 6; ++i) out[i] = acc[i];
    }
  }
  if (fixes) atomicAdd(a.nfix, fixes);
}

__global__ void tri_pair_count_kernel(const int32_t* __restrict__ pair_tri, int64_t P,
                                      unsigned long long* __restrict__ cnt) {
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q < P) atomicAdd(cnt + pair_tri[q], 1ull);
}

__global__ void tri_pair_fill_kernel(const int32_t* __restrict__ pair_tri, const int32_t* __restrict__ pair_pid,
                                     int64_t P, const int64_t* __restrict__ tri_off,
                                     unsigned long long* __restrict__ cursor, int32_t* __restrict__ tri_pid) {
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= P) return;
  const int32_t t = pair_tri[q];
  const unsigned long long k = atomicAdd(cursor + t, 1ull);
  tri_pid[tri_off[t] + int64_t(k)] = pair_pid[q];
}

template <typename OT>
__global__ void particle_grad_kernel(const OT* __restrict__ dg, const OT* __restrict__ grad, int64_t N,
                                     OT* __restrict__ dp) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= N) return;
  dp[2 * i] = dg[i] * grad[2 * i];
  dp[2 * i + 1] = dg[i] * grad[2 * i + 1];
}

template <typename OT>
static sph2d_status run_vertex_grads(Ctx* c, int kernel, const BwdArgs& a) {
  static int grid_blocks[4] = {0, 0, 0, 0};
  const int kk = kernel & 3;
  if (grid_blocks[kk] == 0) {
    int per_sm = 0, sms = 0;
    switch (kk) {
      case 0: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, vertex_grad_kernel<OT, KID_WC2>, 128, 0); break;
      case 1: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, vertex_grad_kernel<OT, KID_WC4>, 128, 0); break;
      case 2: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, vertex_grad_kernel<OT, KID_WC6>, 128, 0); break;
      default: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, vertex_grad_kernel<OT, KID_CUBIC>, 128, 0); break;
    }
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    grid_blocks[kk] = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
  }
  if (a.M == 0) return SPH2D_OK;
  const int64_t want = (a.M + 3) / 4;
  const unsigned blocks = unsigned(want < grid_blocks[kk] ? want : grid_blocks[kk]);
  switch (kk) {
    case 0: SPH2D_LAUNCH(c, (vertex_grad_kernel<OT, KID_WC2>), blocks, 128, a); break;
    case 1: SPH2D_LAUNCH(c, (vertex_grad_kernel<OT, KID_WC4>), blocks, 128, a); break;
    case 2: SPH2D_LAUNCH(c, (vertex_grad_kernel<OT, KID_WC6>), blocks, 128, a); break;
    default: SPH2D_LAUNCH(c, (vertex_grad_kernel<OT, KID_CUBIC>), blocks, 128, a); break;
  }
  return SPH2D_OK;
}

sph2d_status launch_backward(Ctx* c, int kernel, int mode, const void* d_gamma, void* d_particles,
                             void* d_tris) {
  const Cells& cl = c->cells;
  const int64_t N = cl.N, M = cl.M, P = cl.P;
  const size_t elem = mode == SPH2D_FP64 ? sizeof(double) : sizeof(float);
  cudaStream_t st = c->stream;
  cudaError_t e;
  // particle gradients: recompute grad gamma with the forward kernel, scale by dL/dgamma
  sph2d_status s = ensure(c, c->bwd_g, size_t(N) * elem);
  if (s == SPH2D_OK) s = ensure(c, c->bwd_grad, size_t(2 * N) * elem);
  if (s != SPH2D_OK) return s;
  s = launch_integrals(c, kernel, -1, mode, c->bwd_g.ptr, c->bwd_grad.ptr, nullptr);
  if (s != SPH2D_OK) return s;
  if (N > 0) {
    const unsigned b = unsigned((N + 255) / 256);
    if (mode == SPH2D_FP64)
      SPH2D_LAUNCH(c, (particle_grad_kernel<double>), b, 256, static_cast<const double*>(d_gamma),
                   static_cast<const double*>(c->bwd_grad.ptr), N, static_cast<double*>(d_particles));
    else
      SPH2D_LAUNCH(c, (particle_grad_kernel<float>), b, 256, static_cast<const float*>(d_gamma),
                   static_cast<const float*>(c->bwd_grad.ptr), N, static_cast<float*>(d_particles));
  }
  if (M == 0) return SPH2D_OK;
  // transpose the pair list into per-triangle particle lists, sorted ascending
  s = ensure(c, c->tri_cursor, size_t(M) * sizeof(unsigned long long));
  if (s == SPH2D_OK) s = ensure(c, c->tri_off, size_t(M + 1) * sizeof(int64_t));
  if (s == SPH2D_OK) s = ensure(c, c->tri_pid, size_t(P > 0 ? P : 1) * sizeof(int32_t));
  if (s != SPH2D_OK) return s;
  auto* cnt = static_cast<unsigned long long*>(c->tri_cursor.ptr);
  auto* toff = static_cast<int64_t*>(c->tri_off.ptr);
  auto* tpid = static_cast<int32_t*>(c->tri_pid.ptr);
  e = cudaMemsetAsync(cnt, 0, size_t(M) * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return cuda_err(c, e, "memset");
  const unsigned pb = unsigned((P + 255) / 256);
  const int32_t* ptri = static_cast<const int32_t*>(c->pair_tri.ptr);
  const int32_t* ppid = static_cast<const int32_t*>(c->pair_pid.ptr);
  if (P > 0) SPH2D_LAUNCH(c, (tri_pair_count_kernel), pb, 256, ptri, P, cnt);
  s = exclusive_scan_i64(c, reinterpret_cast<const int64_t*>(cnt), toff, M);
  if (s != SPH2D_OK) return s;
  e = cudaMemsetAsync(cnt, 0, size_t(M) * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return cuda_err(c, e, "memset");
  if (P > 0) SPH2D_LAUNCH(c, (tri_pair_fill_kernel), pb, 256, ptri, ppid, P, toff, cnt, tpid);
  launch_sort_segments(c, toff, tpid, M);
  // vertex gradients, one warp per triangle
  s = ensure(c, c->host_flags_dev, 64);
  if (s != SPH2D_OK) return s;
  BwdArgs a;
  a.parts = reinterpret_cast<const float4*>(cl.particles);
  a.tris = cl.tris;
  a.tri_off = toff;
  a.tri_pid = tpid;
  a.M = M;
  a.invH = 1.0 / cl.H;
  a.C = kernel_C(kernel);
  a.d_gamma = d_gamma;
  a.d_tris = d_tris;
  a.nfix = static_cast<unsigned long long*>(c->host_flags_dev.ptr) + 1;
  e = cudaMemsetAsync(a.nfix, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return cuda_err(c, e, "memset");
  s = mode == SPH2D_FP64 ? run_vertex_grads<double>(c, kernel, a) : run_vertex_grads<float>(c, kernel, a);
  if (s != SPH2D_OK) return s;
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(c, e, "backward launch");
  return SPH2D_OK;
}

}  // namespace sph2d
