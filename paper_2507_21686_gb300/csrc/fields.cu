// Piecewise-linear boundary fields (Sec. 3, Eq. taus and basicdiff): for per-vertex values
// A_j of each triangle, interpolated barycentrically (A_T linear on T),
//
//   <A>_i      = sum_T int_T A_T(x') W(x_i - x', H) dx'
//   <grad A>_i = sum_T int_T A_T(x') grad_x W(x_i - x', H) dx'
//
// Per pair, in the local frame p = (x' - x_i)/H where A_T(p) = A_0 + a . (p - p_0) (a the
// local gradient of A_T, p_0 the first vertex):
//   value = A_0 gamma_T + a . ((M10, M01) - p_0 gamma_T)       (the tau form of Eq. taus)
//   grad  = (a / H) gamma_T - sum_j A_j d gamma_T / d nu_j      (integration by parts: the
//           area term of the constant gradient plus the boundary term, whose edge integrals
//           of W lambda_j are the transport-theorem vertex gradients of the adjoint)
// so one pair needs gamma, the first moments and the three vertex gradients, shared by up to
// kMaxFields fields.  Difference and symmetric gradient forms (Sec. 3) are linear in the
// per-vertex values and combine per particle from fields such as rho A and rho.
#include <cuda_runtime.h>

#include "fields_common.cuh"

namespace sph2d {

// field contributions of one pair; returns 1 if any FP64 fix-up was taken
template <typename OT, int KID, bool GRAD>
__device__ __forceinline__ int field_pair(const FieldArgs& f, int pid, int tid, OT* v) {
  const IntArgs& a = f.a;
  OT w[nv_of(1)];                           // gamma, grad gamma, M00, M10, M01
  int fix = eval_pair<OT, KID, 1>(a, pid, tid, w);
  OT g[6];
  const float* t = a.tris + 6 * int64_t(tid);
  const float4 p = a.parts[pid];
  if (GRAD) fix |= vertex_grad_pair<OT, KID>(p, t, a.invH, a.C, g);
  // local frame in the output precision (FP32 path: from the FP32 inputs, as the pair kernel)
  OT l[6];
  if (sizeof(OT) == sizeof(float)) {
    const float ih = float(a.invH);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      l[2 * j] = OT((__ldg(t + 2 * j) - p.x) * ih);
      l[2 * j + 1] = OT((__ldg(t + 2 * j + 1) - p.y) * ih);
    }
  } else {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      l[2 * j] = OT((double(__ldg(t + 2 * j)) - double(p.x)) * a.invH);
      l[2 * j + 1] = OT((double(__ldg(t + 2 * j + 1)) - double(p.y)) * a.invH);
    }
  }
  const OT e1x = l[2] - l[0], e1y = l[3] - l[1], e2x = l[4] - l[0], e2y = l[5] - l[1];
  const OT D = diff_of_products(e1x, e2y, e1y, e2x);   // twice the signed area
  if (D == OT(0)) return fix;                          // zero area: no contribution
  const OT iD = OT(1) / D;
  const float* A = f.values + int64_t(tid) * 3 * f.nf;
#pragma unroll
  for (int k = 0; k < kMaxFields; ++k) {
    if (k < f.nf) {
      const OT a0 = OT(__ldg(A + k)), a1 = OT(__ldg(A + f.nf + k)), a2 = OT(__ldg(A + 2 * f.nf + k));
      const OT d1 = a1 - a0, d2 = a2 - a0;
      // local gradient of the interpolant: a = (d1 (e2y, -e2x) + d2 (-e1y, e1x)) / D
      const OT gx = (d1 * e2y - d2 * e1y) * iD;
      const OT gy = (d2 * e1x - d1 * e2x) * iD;
      // <A> = a0 gamma + a . (M1 - p0 gamma): the interpolant centred at vertex 0
      v[3 * k] = a0 * w[0] + gx * (w[4] - l[0] * w[0]) + gy * (w[5] - l[1] * w[0]);
      if (GRAD) {
        const OT ih = OT(a.invH);
        v[3 * k + 1] = gx * ih * w[0] - (a0 * g[0] + a1 * g[2] + a2 * g[4]);
        v[3 * k + 2] = gy * ih * w[0] - (a0 * g[1] + a1 * g[3] + a2 * g[5]);
      }
    }
  }
  return fix;
}

// one warp per 32 consecutive pairs, segmented per-particle sums and crossing slots as in
// integrals_kernel, for 3 values per field
template <typename OT, int KID, bool GRAD>
__global__ void __launch_bounds__(128, int_minb<OT>()) field_kernel(FieldArgs f) {
  constexpr int NV = 3 * kMaxFields;
  const IntArgs& a = f.a;
  const int lane = threadIdx.x & 31;
  const int64_t nchunks = (a.P + 31) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  unsigned long long fixes = 0;
  for (int64_t ch = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
       ch < nchunks;) {
    const unsigned long long nx = chunk_prefetch(a.work);
    const int64_t q = ch * 32 + lane;
    int pid = -1;
    OT v[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = OT(0);
    int fix = 0;
    if (q < a.P) {
      pid = __ldg(a.pair_pid + q);
      fix = field_pair<OT, KID, GRAD>(f, pid, __ldg(a.pair_tri + q), v);
    }
    fixes += __popc(__ballot_sync(0xffffffffu, fix));
    field_warp_sum<OT>(f, ch, pid, v);
    ch = chunk_next(a.work, ch, nw, nx);
  }
  if (lane == 0 && fixes) atomicAdd(a.nfix, fixes);
}

template <typename OT, int KID, bool GRAD>
static sph2d_status run_fields(Ctx* c, FieldArgs f) {
  constexpr int NV = 3 * kMaxFields;
  const int64_t nchunks = (f.a.P + 31) >> 5;
  sph2d_status s = ensure(c, c->slots, size_t(nchunks * 2 * NV + 1) * sizeof(OT));
  if (s != SPH2D_OK) return s;
  f.a.slots = c->slots.ptr;
  if (f.a.P > 0) {
    int per_sm = 0, sms = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, field_kernel<OT, KID, GRAD>, 128, 0);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    const int64_t cap = int64_t(per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
    const int64_t want = (nchunks + 3) / 4;
    SPH2D_LAUNCH(c, (field_kernel<OT, KID, GRAD>), unsigned(want < cap ? want : cap), 128, f);
  }
  if (f.a.N > 0) SPH2D_LAUNCH(c, (field_finalize_kernel<OT>), unsigned((f.a.N + 255) / 256), 256, f);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(c, e, "field integrals launch");
  return SPH2D_OK;
}

template <typename OT, bool GRAD>
static sph2d_status dispatch_fields(Ctx* c, int kernel, const FieldArgs& f) {
  switch (kernel) {
    case KID_WC2: return run_fields<OT, KID_WC2, GRAD>(c, f);
    case KID_WC4: return run_fields<OT, KID_WC4, GRAD>(c, f);
    case KID_WC6: return run_fields<OT, KID_WC6, GRAD>(c, f);
    default: return run_fields<OT, KID_CUBIC, GRAD>(c, f);
  }
}

sph2d_status launch_fields(Ctx* c, int kernel, int mode, const float* values, int nf, void* value,
                           void* grad) {
  const Cells& cl = c->cells;
  FieldArgs f{};
  IntArgs& a = f.a;
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
  f.values = values;
  f.nf = nf;
  f.value = value;
  f.grad = grad;
  sph2d_status s = ensure(c, c->host_flags_dev, 64);
  if (s != SPH2D_OK) return s;
  a.nfix = static_cast<unsigned long long*>(c->host_flags_dev.ptr);
  a.work = a.nfix + 1;                               // chunk counter
  cudaError_t e = cudaMemsetAsync(a.nfix, 0, 2 * sizeof(unsigned long long), c->stream);
  if (e != cudaSuccess) return cuda_err(c, e, "memset");
  const bool g = grad != nullptr;
  if (mode == SPH2D_FP64) s = g ? dispatch_fields<double, true>(c, kernel, f) : dispatch_fields<double, false>(c, kernel, f);
  else s = g ? dispatch_fields<float, true>(c, kernel, f) : dispatch_fields<float, false>(c, kernel, f);
  if (s != SPH2D_OK) return s;
  e = cudaMemcpyAsync(c->pinned + 8, a.nfix, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return cuda_err(c, e, "fixup count copy");
  c->stats.n_pairs = cl.P;
  c->stats.n_fallback = 0;
  c->fixup_pending = true;
  c->fallback_pending = false;
  return SPH2D_OK;
}

}  // namespace sph2d
