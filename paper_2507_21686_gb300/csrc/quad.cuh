// Gauss-Legendre conical-product rule and the pair classification of the hybrid FP32 mode
// (shared by the integrals and the higher-order fields).  See hybrid.cu for the design.
#pragma once

#include <cmath>

#include "integrals_impl.cuh"

namespace sph2d {

constexpr int kQuadN = 6;

// rule passed by value (kernel-parameter constant bank): Gauss-Legendre nodes u on [0, 1],
// their weights w, and w u (the collapsed coordinate's Jacobian factor)
struct QuadRule {
  static constexpr int N = kQuadN;
  float u[kQuadN], w[kQuadN], wu[kQuadN];
};

// a finer rule across the rays (their directions), for the cubic spline's second piece: nodes
// on [0, 1] and their weights
constexpr int kQuadFineN = 10;
struct QuadRaysFine {
  static constexpr int N = kQuadFineN;
  float u[kQuadFineN], w[kQuadFineN];
};

// Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration on P_n (host)
static inline void gauss_legendre_nodes(int n, double* x, double* w) {
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

static inline const QuadRule& quad_rule() {
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

static inline const QuadRaysFine& quad_rays_fine() {
  static QuadRaysFine r = [] {
    QuadRaysFine q{};
    double x[kQuadFineN], w[kQuadFineN];
    gauss_legendre_nodes(kQuadFineN, x, w);
    for (int i = 0; i < kQuadFineN; ++i) {
      q.u[i] = float(0.5 * (x[i] + 1.0));
      q.w[i] = float(0.5 * w[i]);
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
    kd = div_fast(-6.0f * m2, r);
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

// Longest edge (squared, local units) below which the cubic spline's second piece of a near
// pair is taken by quadrature too: in the doubled frame, where that piece is (1 - r')^3_+, the
// triangle crosses r' = 1 with its apex inside; with 10 rays of 6 nodes each, measured over
// generic triangles within H of the particle, the pair stays within 7.8e-7 of the output scales
// at this size (2.1e-6 with 8 rays, 5.5e-6 with 6).
constexpr float kHalfQuadLmax2 = 0.45f * 0.45f;

// Classification of a pair for the hybrid mode.  quad: the first (or only) kernel piece by
// quadrature, apex = index of the innermost vertex.  Cubic spline only: inner = the triangle
// lies inside r < 1/2 (one polynomial there, by quadrature too); near = otherwise within 1/2
// of the particle, so the second piece (support 1/2) needs its own integral; half = a near
// pair whose apex lies inside r < 1/2 and whose longest edge is below kHalfQuadLmax2, so that
// the second piece can be taken by the finer rule in the doubled frame.
struct QuadClass {
  bool quad, inner, near, half;
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
  c.half = c.near && rmin2 < 0.25f && lmax2 < kHalfQuadLmax2;
  return c;
}

}  // namespace sph2d
