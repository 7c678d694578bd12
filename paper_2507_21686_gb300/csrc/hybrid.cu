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

namespace sph2d {

constexpr int kQuadN = 6;

// rule passed by value (kernel-parameter constant bank): Gauss-Legendre nodes u on [0, 1],
// their weights w, and w u (the collapsed coordinate's Jacobian factor)
struct QuadRule {
  float u[kQuadN], w[kQuadN], wu[kQuadN];
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
    for (int i = 0; i < kQuadN; ++i) {
      q.u[i] = float(0.5 * (x[i] + 1.0));
      q.w[i] = float(0.5 * w[i]);
      q.wu[i] = float(0.25 * w[i] * (x[i] + 1.0));
    }
    return q;
  }();
  return r;
}

// k(r) and k'(r)/r in factored form: (1 - r)^n times a positive polynomial keeps FP32 relative
// accuracy near the support edge, where the expanded polynomials cancel (C4's coefficients
// reach 150 while k(0.9) ~ 1e-6).  Cubic spline: inner (r < 1/2, both pieces)
// 1 - 6 r^2 + 6 r^3, k'/r = -12 + 18 r; otherwise the first piece alone, 2 (1 - r)^3,
// k'/r = -6 (1 - r)^2 / r (r > 0: the particle is away from the triangle).  Beyond r = 1
// every form is clamped to zero (rounding at the support edge).
template <int KID>
__device__ __forceinline__ void kernel_and_slope(float r, bool inner, float& k, float& kd) {
  const float m = fmaxf(1.0f - r, 0.0f), m2 = m * m, m3 = m2 * m;   // zero beyond the support
  if (KID == KID_WC2) {                 // (1-r)^4 (1 + 4r),  k'/r = -20 (1-r)^3
    k = m3 * m * (1.0f + 4.0f * r);
    kd = -20.0f * m3;
  } else if (KID == KID_WC4) {          // (1-r)^6 (1 + 6r + 35/3 r^2),  k'/r = -56/3 (1-r)^5 (1 + 5r)
    const float m5 = m3 * m2;
    k = m5 * m * (1.0f + r * (6.0f + r * (35.0f / 3.0f)));
    kd = (-56.0f / 3.0f) * m5 * (1.0f + 5.0f * r);
  } else if (KID == KID_WC6) {          // (1-r)^8 (1 + 8r + 25r^2 + 32r^3),  k'/r = -22 (1-r)^7 (1 + 7r + 16r^2)
    const float m7 = m3 * m3 * m;
    k = m7 * m * (1.0f + r * (8.0f + r * (25.0f + 32.0f * r)));
    kd = -22.0f * m7 * (1.0f + r * (7.0f + 16.0f * r));
  } else if (inner) {
    k = 1.0f + r * r * (-6.0f + 6.0f * r);
    kd = -12.0f + 18.0f * r;
  } else {
    k = 2.0f * m3;
    kd = -6.0f * m2 / r;
  }
}

// eligibility for quadrature (FP32 local frame).  A triangle crossing the support edge
// r = 1 qualifies when one vertex lies inside (the apex of the rule) and its longest edge
// (squared, local units) stays below a per-kernel size where the 6 x 6 rule with each ray
// cut at the circle keeps within ~1.5e-6 of the output scales: the kernel's last kink
// ((1 - r)^n_+ has n - 1 continuous derivatives) is then only across the rays, not along them.
template <int KID>
__device__ __forceinline__ constexpr float cross_lmax2() {
  return KID == KID_WC2 ? 0.6f * 0.6f : KID == KID_WC4 ? 0.75f * 0.75f : KID == KID_WC6 ? 0.7f * 0.7f : 0.45f * 0.45f;
}

// Classification of a pair for the hybrid mode.  quad: the first (or only) kernel piece by
// quadrature, apex = index of the innermost vertex.  Cubic spline only: inner = the triangle
// lies inside r < 1/2 (one polynomial there, by quadrature too); near = otherwise within 1/2
// of the particle, so the second piece (support 1/2) is left to the closed form.
struct QuadClass {
  bool quad, inner, near;
  int apex;
};

template <int KID>
__device__ __forceinline__ QuadClass quad_classify(const float* v) {
  float rmax2 = 0.0f, rmin2 = 3.0e38f, lmax2 = 0.0f, dmin2 = 3.0e38f;
  int apex = 0;
  bool pos = false, neg = false;
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const int b = e == 2 ? 0 : e + 1;
    const float ax = v[2 * e], ay = v[2 * e + 1], bx = v[2 * b], by = v[2 * b + 1];
    const float ex = bx - ax, ey = by - ay;
    const float a2 = ax * ax + ay * ay;
    rmax2 = fmaxf(rmax2, a2);
    if (a2 < rmin2) {
      rmin2 = a2;
      apex = e;
    }
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
  QuadClass c;
  c.apex = apex;
  c.quad = !inside && (pos || neg) && lmax2 > 0.0f && dmin2 >= 0.25f * lmax2 &&
           (rmax2 < 1.0f || (rmin2 < 1.0f && lmax2 < cross_lmax2<KID>()));
  c.inner = KID == KID_CUBIC && rmax2 < 0.25f;
  c.near = KID == KID_CUBIC && !c.inner && dmin2 < 0.25f;
  return c;
}

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
  for (int64_t base = int64_t(blockIdx.x) * blockDim.x + threadIdx.x - lane; base < a.P; base += stride) {
    const int64_t q = base + lane;
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
  constexpr int nlists = KID == KID_CUBIC ? 2 : 1;
  const int64_t nchunks = (a.P + 31) >> 5;
  const int64_t cap = a.P > 0 ? a.P : 1;
  sph2d_status s = ensure(c, c->slots, size_t(nchunks * 2 * NV + 1) * sizeof(float));
  if (s == SPH2D_OK) s = ensure(c, c->pair_vals, size_t(cap) * NV * sizeof(float));
  if (s == SPH2D_OK) s = ensure(c, c->pair_list2, size_t(cap) * nlists * sizeof(int64_t) + 64);
  if (s != SPH2D_OK) return s;
  a.slots = c->slots.ptr;
  float* vals = static_cast<float*>(c->pair_vals.ptr);
  int64_t* list = reinterpret_cast<int64_t*>(static_cast<char*>(c->pair_list2.ptr) + 64);
  int64_t* near = list + cap;                        // cubic: pairs within H/2 among the list
  auto* count = static_cast<unsigned long long*>(c->pair_list2.ptr);
  cudaError_t e = cudaMemsetAsync(count, 0, 2 * sizeof(unsigned long long), c->stream);
  if (e != cudaSuccess) return cuda_err(c, e, "memset");
  if (a.P > 0) {
    const int64_t blocks = (a.P + 127) / 128;
    SPH2D_LAUNCH(c, (hybrid_first_kernel<KID, MD>), blocks_for(c, hybrid_first_kernel<KID, MD>, blocks), 128, a,
                 quad_rule(), vals, list, count, near, count + 1);
    if constexpr (KID == KID_CUBIC) {
      // the cubic spline's two pieces over the list, as its closed-form path (the second
      // piece also for the quadrature pairs already in near)
      SPH2D_LAUNCH(c, (cubic_first_kernel<float, MD>), blocks_for(c, cubic_first_kernel<float, MD>, blocks), 128,
                   a, vals, list, count, near, count + 1);
      SPH2D_LAUNCH(c, (cubic_second_kernel<float, MD>), blocks_for(c, cubic_second_kernel<float, MD>, blocks), 128,
                   a, vals, near, count + 1);
    } else {
      SPH2D_LAUNCH(c, (hybrid_second_kernel<KID, MD>), blocks_for(c, hybrid_second_kernel<KID, MD>, blocks), 128, a,
                   vals, list, count);
    }
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
