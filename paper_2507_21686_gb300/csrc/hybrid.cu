// Hybrid FP32 mode (the extension Sec. 6.1 suggests: quadrature for triangles entirely inside
// the support, the closed form for every other pair).
//
// A pair is integrated by quadrature when its local triangle lies at least half its longest
// edge away from the particle (the odd powers of r are not smooth only at the particle) and
// either inside the support (|v_j| < 1) or across its edge with one vertex inside and a
// longest edge below a per-kernel size.  The rule is a 6 x 6 conical product of
// Gauss-Legendre rules with its apex at the innermost vertex (s along rays from it, t across
// them); each ray is cut where it leaves the unit disk, so the integrand is smooth along
// the rays and the kernel's truncation shows only across them.  Measured over generic
// triangles up to 1.2 H this reaches ~5e-7 of the output scales inside the support and
// <= 1.5e-6 at the size limits across its edge, for every output including third moments:
// inside the FP32 budget of 1e-5.  The cubic spline's second piece (support H/2) is smooth
// on a triangle inside r < 1/2 (taken with the first), zero on one at least 1/2 away, and
// otherwise left to the closed form of that piece alone.  On the box benchmark this covers
// most pairs at a fifth of the closed form's arithmetic.
//
// Three launches, as the cubic spline's path: quadrature for eligible pairs into a per-pair
// buffer and a warp-aggregated list of the others; the closed form (FP32 + fix-up) over that
// list; per-particle sums of the per-pair values in pair order (deterministic).  The cubic
// spline's closed form takes its two launches over the list (second piece only within H/2).
#include <cuda_runtime.h>

#include <cmath>

#include "integrals_impl.cuh"
#include "quad.cuh"

namespace sph2d {

// quadrature of one pair -> v (gamma, grad, moments), world-scaled like eval_local.
// Conical product with the apex at vertex `apex`: p = v0 + s d(t), d(t) = (v1 - v0) + t (v2 - v1),
// Jacobian s |(v1 - v0) x (v2 - v0)|; along each ray s runs to min(1, s+), s+ the exit from
// the unit disk (|v0| < 1), taken as -c / (b + sqrt(b^2 - a c)) with a = |d|^2, b = v0 . d,
// c = |v0|^2 - 1 (no cancellation: b + sqrt(.) > 0 whenever c < 0).
template <int KID, int MD>
__device__ __forceinline__ void quad_pair(const QuadRule& qr, const float* vin, const QuadClass& qc, double C,
                                          double invH, float* out) {
  const int i0 = qc.apex, i1 = i0 == 2 ? 0 : i0 + 1, i2 = i1 == 2 ? 0 : i1 + 1;
  const float v0x = vin[2 * i0], v0y = vin[2 * i0 + 1];
  const float e1x = vin[2 * i1] - v0x, e1y = vin[2 * i1 + 1] - v0y;
  const float e2x = vin[2 * i2] - vin[2 * i1], e2y = vin[2 * i2 + 1] - vin[2 * i1 + 1];
  const float a2 = fabsf(diff_of_products(e1x, vin[2 * i2 + 1] - v0y, e1y, vin[2 * i2] - v0x));
  const float c0 = v0x * v0x + v0y * v0y - 1.0f;
  float g = 0.0f, gx = 0.0f, gy = 0.0f;
  float m[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll 2
  for (int j = 0; j < kQuadN; ++j) {
    const float dx = e1x + qr.u[j] * e2x, dy = e1y + qr.u[j] * e2y;
    const float aa = dx * dx + dy * dy, bb = v0x * dx + v0y * dy;
    const float sp = -c0 / (bb + sqrtf(fmaxf(bb * bb - aa * c0, 0.0f)));
    const float ss = fminf(1.0f, sp);
    const float wj = qr.w[j] * ss * ss;
#pragma unroll
    for (int i = 0; i < kQuadN; ++i) {
      const float s = ss * qr.u[i];
      const float px = v0x + s * dx, py = v0y + s * dy;
      const float r = sqrtf(px * px + py * py);
      float k, kd;
      kernel_and_slope<KID>(r, qc.inner, k, kd);
      const float w = wj * qr.wu[i];
      const float wk = w * k, wd = w * kd;
      g += wk;
      gx += wd * px;
      gy += wd * py;
      if (MD >= 1) {
        m[1] += wk * px;
        m[2] += wk * py;
      }
      if (MD >= 3) {
        const float xx = px * px, xy = px * py, yy = py * py;
        m[3] += wk * xx;
        m[4] += wk * xy;
        m[5] += wk * yy;
        m[6] += wk * xx * px;
        m[7] += wk * xx * py;
        m[8] += wk * px * yy;
        m[9] += wk * yy * py;
      }
    }
  }
  const float c = float(C) * a2;
  out[0] = c * g;
  out[1] = -c * float(invH) * gx;          // grad gamma = -(C/H) int k'(r) p / r
  out[2] = -c * float(invH) * gy;
  if (MD >= 1) {
    out[3] = c * g;
    out[4] = c * m[1];
    out[5] = c * m[2];
  }
  if (MD >= 3) {
#pragma unroll
    for (int i = 3; i < 10; ++i) out[3 + i] = c * m[i];
  }
}

// quadrature for the pairs that qualify into vals; the others appended to list (closed form);
// cubic spline: quadrature pairs within 1/2 of the particle (not inside r < 1/2) appended to
// near, for the second piece in closed form
template <int KID, int MD>
__global__ void __launch_bounds__(128, int_minb<float>()) hybrid_first_kernel(IntArgs a, QuadRule qr,
                                                                              float* __restrict__ vals,
                                                                              int64_t* __restrict__ list,
                                                                              unsigned long long* __restrict__ count,
                                                                              int64_t* __restrict__ near,
                                                                              unsigned long long* __restrict__ near_count) {
  constexpr int NV = nv_of(MD);
  const int lane = threadIdx.x & 31;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  const float ih = float(a.invH);
  const int64_t nchunks = (a.P + 31) >> 5, nw = stride >> 5;
  for (int64_t ch = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; ch < nchunks;) {
    const unsigned long long nx = chunk_prefetch(a.work);
    const int64_t q = ch * 32 + lane;
    bool analytic = false, piece2 = false;
    if (q < a.P) {
      const float4 p = a.parts[__ldg(a.pair_pid + q)];
      const float* t = a.tris + 6 * int64_t(__ldg(a.pair_tri + q));
      float v[6];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        v[2 * j] = (__ldg(t + 2 * j) - p.x) * ih;
        v[2 * j + 1] = (__ldg(t + 2 * j + 1) - p.y) * ih;
      }
      const QuadClass qc = quad_classify<KID>(v);
      if (qc.quad) {
        float w[13];
        quad_pair<KID, MD>(qr, v, qc, a.C, a.invH, w);
        float* o = vals + q * NV;
#pragma unroll
        for (int i = 0; i < NV; ++i) o[i] = w[i];
        piece2 = qc.near;
      } else {
        analytic = true;
      }
    }
    warp_append(analytic, q, list, count);
    if (KID == KID_CUBIC) warp_append(piece2, q, near, near_count);
    ch = chunk_next(a.work, ch, nw, nx);
  }
}

// the closed form (FP32 + FP64 fix-up) over the list
template <int KID, int MD>
__global__ void __launch_bounds__(128, int_minb<float>()) hybrid_second_kernel(IntArgs a, float* __restrict__ vals,
                                                                               const int64_t* __restrict__ list,
                                                                               const unsigned long long* __restrict__ count) {
  constexpr int NV = nv_of(MD);
  const int64_t n = int64_t(*count);
  const int64_t nchunks = (n + 31) >> 5, nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  unsigned long long fixes = 0;
  for (int64_t ch = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; ch < nchunks;) {
    const unsigned long long nx = chunk_prefetch(a.work);
    const int64_t i = ch * 32 + (threadIdx.x & 31);
    if (i < n) {
      const int64_t q = list[i];
      float v[NV];
      fixes += eval_pair<float, KID, MD>(a, __ldg(a.pair_pid + q), __ldg(a.pair_tri + q), v);
      float* o = vals + q * NV;
#pragma unroll
      for (int k = 0; k < NV; ++k) o[k] = v[k];
    }
    ch = chunk_next(a.work, ch, nw, nx);
  }
  if (fixes) atomicAdd(a.nfix, fixes);
}

template <int KID, int MD>
static sph2d_status run_hybrid(Ctx* c, IntArgs a) {
  constexpr int NV = nv_of(MD);
  constexpr int nlists = KID == KID_CUBIC ? 3 : 1;
  const int64_t nchunks = (a.P + 31) >> 5;
  const int64_t cap = a.P > 0 ? a.P : 1;
  sph2d_status s = ensure(c, c->slots, size_t(nchunks * 2 * NV + 1) * sizeof(float));
  if (s == SPH2D_OK) s = ensure(c, c->pair_vals, size_t(cap) * NV * sizeof(float));
  if (s == SPH2D_OK) s = ensure(c, c->pair_list2, size_t(cap) * nlists * sizeof(int64_t) + 64);
  if (s != SPH2D_OK) return s;
  a.slots = c->slots.ptr;
  float* vals = static_cast<float*>(c->pair_vals.ptr);
  int64_t* list = reinterpret_cast<int64_t*>(static_cast<char*>(c->pair_list2.ptr) + 64);
  int64_t* near = list + cap;                        // cubic: pairs within H/2 whose second piece is pending
  int64_t* fix_list = list + 2 * cap;                // cubic: FP32 pairs for the FP64 fix-up
  auto* count = static_cast<unsigned long long*>(c->pair_list2.ptr);   // [0] list, [1] near, [2] fix-up
  cudaError_t e = cudaMemsetAsync(count, 0, 64, c->stream);
  if (e != cudaSuccess) return cuda_err(c, e, "memset");
  if (a.P > 0) {
    const int64_t blocks = (a.P + 127) / 128;
    IntArgs aq = a, al = a, a2 = a;                  // chunk counters in the zeroed header
    aq.work = count + 4;
    al.work = count + 5;
    a2.work = count + 6;
    SPH2D_LAUNCH(c, (hybrid_first_kernel<KID, MD>), resident_blocks(c, hybrid_first_kernel<KID, MD>, blocks), 128, aq,
                 quad_rule(), vals, list, count, near, count + 1);
    if constexpr (KID == KID_CUBIC) {
      // the cubic spline's pieces over the list, as its closed-form path (the second piece also
      // for the quadrature pairs already in near)
      SPH2D_LAUNCH(c, (cubic_first_kernel<float, MD>), resident_blocks(c, cubic_first_kernel<float, MD>, blocks), 128,
                   al, vals, list, count, near, count + 1, fix_list, count + 2);
      SPH2D_LAUNCH(c, (cubic_fixup_kernel<MD>), resident_blocks(c, cubic_fixup_kernel<MD>, blocks), 128, a, vals,
                   fix_list, count + 2);
      SPH2D_LAUNCH(c, (cubic_second_kernel<float, MD>), resident_blocks(c, cubic_second_kernel<float, MD>, blocks), 128,
                   a2, vals, near, count + 1);
    } else {
      SPH2D_LAUNCH(c, (hybrid_second_kernel<KID, MD>), resident_blocks(c, hybrid_second_kernel<KID, MD>, blocks), 128, al,
                   vals, list, count);
    }
    SPH2D_LAUNCH(c, (reduce_pairs_kernel<float, MD>), resident_blocks(c, reduce_pairs_kernel<float, MD>, (nchunks + 3) / 4),
                 128, a, vals);
  }
  if (a.N > 0) SPH2D_LAUNCH(c, (finalize_kernel<float, MD>), unsigned((a.N + 255) / 256), 256, a);
  // the number of pairs left to the closed form, as the fallback count
  e = cudaMemcpyAsync(c->pinned + 10, count, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return cuda_err(c, e, "fallback count copy");
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(c, e, "hybrid launch");
  return SPH2D_OK;
}

template <int KID>
static sph2d_status run_hybrid_md(Ctx* c, int md, const IntArgs& a) {
  return md == 3 ? run_hybrid<KID, 3>(c, a) : (md == 1 ? run_hybrid<KID, 1>(c, a) : run_hybrid<KID, 0>(c, a));
}

sph2d_status integrals_hybrid(Ctx* c, int kernel, int md, const IntArgs& a) {
  switch (kernel) {
    case KID_WC2: return run_hybrid_md<KID_WC2>(c, md, a);
    case KID_WC4: return run_hybrid_md<KID_WC4>(c, md, a);
    case KID_WC6: return run_hybrid_md<KID_WC6>(c, md, a);
    default: return run_hybrid_md<KID_CUBIC>(c, md, a);
  }
}

}  // namespace sph2d
