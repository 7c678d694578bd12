// Hybrid FP32 mode (the extension Sec. 6.1 suggests: quadrature for triangles entirely inside
// the support, the closed form for every other pair).
//
// A pair is integrated by quadrature when its local triangle lies inside the support
// (|v_j| < 1) and at least half its longest edge away from the particle; for the cubic spline
// the triangle must also stay on one side of the r = 1/2 circle (all of it inside, or at
// least 1/2 away), where the spline switches polynomial.  Then the integrand is smooth on the
// triangle (the odd powers of r are not smooth only at the particle), and a 6 x 6
// conical-product Gauss-Legendre rule (collapsed square s, t in [0, 1]^2, p = v0 + s (v1 - v0)
// + s t (v2 - v1), Jacobian s |v1-v0 x v2-v0|) reaches ~5e-7 of the output scales for every
// output including third moments (measured over generic triangles up to 1.2 H), inside the FP32
// budget of 1e-5.  On the box benchmark this covers about half of the pairs at a fifth of the
// closed form's arithmetic.
//
// Three launches, as the cubic spline's path: quadrature for eligible pairs into a per-pair
// buffer and a warp-aggregated list of the others; the closed form (FP32 + fix-up) over that
// list; per-particle sums of the per-pair values in pair order (deterministic).
#include <cuda_runtime.h>

#include <cmath>

#include "integrals_impl.cuh"

namespace sph2d {

constexpr int kQuadN = 6, kQuadPts = kQuadN * kQuadN;

// rule passed by value (kernel-parameter constant bank): s, s t and weight * s per point
struct QuadRule {
  float s[kQuadPts], st[kQuadPts], ws[kQuadPts];
};

// Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration on P_n (host)
static void gauss_legendre_nodes(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = std::cos(3.141592653589793 * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      const double dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) {
        // final derivative at the converged node
        p0 = 1.0;
        p1 = z;
        for (int k = 2; k <= n; ++k) {
          const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
          p0 = p1;
          p1 = p2;
        }
        const double d = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * d * d);
        break;
      }
    }
  }
}

static const QuadRule& quad_rule() {
  static QuadRule r = [] {
    QuadRule q{};
    double x[kQuadN], w[kQuadN];
    gauss_legendre_nodes(kQuadN, x, w);
    for (int i = 0; i < kQuadN; ++i)
      for (int j = 0; j < kQuadN; ++j) {
        const double s = 0.5 * (x[i] + 1.0), t = 0.5 * (x[j] + 1.0);
        const int k = i * kQuadN + j;
        q.s[k] = float(s);
        q.st[k] = float(s * t);
        q.ws[k] = float(0.25 * w[i] * w[j] * s);
      }
    return q;
  }();
  return r;
}

// polynomial pieces of the kernel seen by a quadrature triangle: k(r) and k'(r)/r
template <int KID>
struct QuadKernel;
template <> struct QuadKernel<KID_WC2> { using P = PolyWC2; };
template <> struct QuadKernel<KID_WC4> { using P = PolyWC4; };
template <> struct QuadKernel<KID_WC6> { using P = PolyWC6; };
template <> struct QuadKernel<KID_CUBIC> { using P = PolyCubeOut; };   // unused: the cubic picks its piece

template <class P>
__device__ __forceinline__ void kernel_and_slope(float r, float& k, float& kd) {
  // k = sum b_q r^q, kd = k'(r)/r = b_1 / r + sum_{q>=0} (q+2) b_{q+2} r^q
  float a = 0.0f, b = 0.0f;
#pragma unroll
  for (int q = P::K; q >= 0; --q) a = a * r + float(P::b(q));
#pragma unroll
  for (int q = P::K - 2; q >= 0; --q) b = b * r + float((q + 2) * P::b(q + 2));
  if (P::b(1) != 0.0) b += float(P::b(1)) / r;
  k = a;
  kd = b;
}

// eligibility for quadrature (FP32 local frame); inner: for the cubic spline, whether the
// triangle lies inside r < 1/2 (else it lies beyond 1/2)
template <int KID>
__device__ __forceinline__ bool quad_eligible(const float* v, bool& inner) {
  float rmax2 = 0.0f, lmax2 = 0.0f, dmin2 = 3.0e38f;
  bool pos = false, neg = false;
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const int b = e == 2 ? 0 : e + 1;
    const float ax = v[2 * e], ay = v[2 * e + 1], bx = v[2 * b], by = v[2 * b + 1];
    const float ex = bx - ax, ey = by - ay;
    const float a2 = ax * ax + ay * ay;
    rmax2 = fmaxf(rmax2, a2);
    const float l2 = ex * ex + ey * ey;
    lmax2 = fmaxf(lmax2, l2);
    const float cr = ax * ey - ay * ex;
    pos = pos || cr > 0.0f;
    neg = neg || cr < 0.0f;
    const float tn = -(ax * ex + ay * ey);
    // squared distance from the particle to the edge segment (the perpendicular case
    // compared as cr^2 / l2 without dividing)
    float d2;
    if (tn <= 0.0f) d2 = a2;
    else if (tn >= l2) d2 = bx * bx + by * by;
    else d2 = l2 > 0.0f ? cr * cr / l2 : a2;
    dmin2 = fminf(dmin2, d2);
  }
  const bool inside = pos != neg;                // the particle lies in the triangle
  inner = rmax2 < 0.25f;
  bool ok = !inside && rmax2 < 1.0f && lmax2 > 0.0f && dmin2 >= 0.25f * lmax2 && (pos || neg);
  if (KID == KID_CUBIC) ok = ok && (inner || dmin2 >= 0.25f);
  return ok;
}

// quadrature of one eligible pair -> v (gamma, grad, moments), world-scaled like eval_local
template <int KID, int MD>
__device__ __forceinline__ void quad_pair(const QuadRule& qr, const float* v, bool inner, double C, double invH,
                                          float* out) {
  const float v0x = v[0], v0y = v[1];
  const float e1x = v[2] - v[0], e1y = v[3] - v[1], e2x = v[4] - v[2], e2y = v[5] - v[3];
  const float a2 = fabsf(diff_of_products(e1x, v[5] - v[1], e1y, v[4] - v[0]));
  float g = 0.0f, gx = 0.0f, gy = 0.0f;
  float m[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll 4
  for (int i = 0; i < kQuadPts; ++i) {
    const float s = qr.s[i], st = qr.st[i];
    const float px = v0x + s * e1x + st * e2x;
    const float py = v0y + s * e1y + st * e2y;
    const float r = sqrtf(px * px + py * py);
    float k, kd;
    if (KID == KID_CUBIC) {
      if (inner) kernel_and_slope<PolyCubeIn>(r, k, kd);
      else kernel_and_slope<PolyCubeOut>(r, k, kd);
    } else {
      kernel_and_slope<typename QuadKernel<KID>::P>(r, k, kd);
    }
    const float w = qr.ws[i];
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

template <int KID, int MD>
__global__ void __launch_bounds__(128, int_minb<float>()) hybrid_first_kernel(IntArgs a, QuadRule qr,
                                                                              float* __restrict__ vals,
                                                                              int64_t* __restrict__ list,
                                                                              unsigned long long* __restrict__ count) {
  constexpr int NV = nv_of(MD);
  const int lane = threadIdx.x & 31;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  const float ih = float(a.invH);
  for (int64_t base = int64_t(blockIdx.x) * blockDim.x + threadIdx.x - lane; base < a.P; base += stride) {
    const int64_t q = base + lane;
    bool analytic = false;
    if (q < a.P) {
      const float4 p = a.parts[__ldg(a.pair_pid + q)];
      const float* t = a.tris + 6 * int64_t(__ldg(a.pair_tri + q));
      float v[6];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        v[2 * j] = (__ldg(t + 2 * j) - p.x) * ih;
        v[2 * j + 1] = (__ldg(t + 2 * j + 1) - p.y) * ih;
      }
      bool inner;
      if (quad_eligible<KID>(v, inner)) {
        float w[13];
        quad_pair<KID, MD>(qr, v, inner, a.C, a.invH, w);
        float* o = vals + q * NV;
#pragma unroll
        for (int i = 0; i < NV; ++i) o[i] = w[i];
      } else {
        analytic = true;
      }
    }
    const unsigned m = __ballot_sync(0xffffffffu, analytic);
    if (m) {
      unsigned long long b = 0;
      const int leader = __ffs(m) - 1;
      if (lane == leader) b = atomicAdd(count, (unsigned long long)__popc(m));
      b = __shfl_sync(0xffffffffu, b, leader);
      if (analytic) list[b + __popc(m & ((1u << lane) - 1u))] = q;
    }
  }
}

// the closed form (FP32 + FP64 fix-up) over the list
template <int KID, int MD>
__global__ void __launch_bounds__(128, int_minb<float>()) hybrid_second_kernel(IntArgs a, float* __restrict__ vals,
                                                                               const int64_t* __restrict__ list,
                                                                               const unsigned long long* __restrict__ count) {
  constexpr int NV = nv_of(MD);
  const int64_t n = int64_t(*count);
  unsigned long long fixes = 0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t q = list[i];
    float v[NV];
    fixes += eval_pair<float, KID, MD>(a, __ldg(a.pair_pid + q), __ldg(a.pair_tri + q), v);
    float* o = vals + q * NV;
#pragma unroll
    for (int k = 0; k < NV; ++k) o[k] = v[k];
  }
  if (fixes) atomicAdd(a.nfix, fixes);
}

template <typename K>
static unsigned blocks_for(Ctx* c, K kern, int64_t wanted) {
  int per_sm = 0, sms = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, 0);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  const int64_t cap = int64_t(per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
  return unsigned(wanted < cap ? (wanted > 0 ? wanted : 1) : cap);
}

template <int KID, int MD>
static sph2d_status run_hybrid(Ctx* c, IntArgs a) {
  constexpr int NV = nv_of(MD);
  const int64_t nchunks = (a.P + 31) >> 5;
  sph2d_status s = ensure(c, c->slots, size_t(nchunks * 2 * NV + 1) * sizeof(float));
  if (s == SPH2D_OK) s = ensure(c, c->pair_vals, size_t(a.P > 0 ? a.P : 1) * NV * sizeof(float));
  if (s == SPH2D_OK) s = ensure(c, c->pair_list2, size_t(a.P > 0 ? a.P : 1) * sizeof(int64_t) + 64);
  if (s != SPH2D_OK) return s;
  a.slots = c->slots.ptr;
  float* vals = static_cast<float*>(c->pair_vals.ptr);
  int64_t* list = reinterpret_cast<int64_t*>(static_cast<char*>(c->pair_list2.ptr) + 64);
  auto* count = static_cast<unsigned long long*>(c->pair_list2.ptr);
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), c->stream);
  if (e != cudaSuccess) return cuda_err(c, e, "memset");
  if (a.P > 0) {
    const int64_t blocks = (a.P + 127) / 128;
    SPH2D_LAUNCH(c, (hybrid_first_kernel<KID, MD>), blocks_for(c, hybrid_first_kernel<KID, MD>, blocks), 128, a,
                 quad_rule(), vals, list, count);
    SPH2D_LAUNCH(c, (hybrid_second_kernel<KID, MD>), blocks_for(c, hybrid_second_kernel<KID, MD>, blocks), 128, a,
                 vals, list, count);
    SPH2D_LAUNCH(c, (reduce_pairs_kernel<float, MD>), blocks_for(c, reduce_pairs_kernel<float, MD>, (nchunks + 3) / 4),
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
