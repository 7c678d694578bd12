// Closed-form integrals of a compact polynomial SPH kernel over one triangle, in the
// normalised frame of Sec. 2 (particle at the origin, support radius 1).
//
// Decomposition.  The paper splits the triangle into sectors, segments and stubs about the
// particle (Sec. 4, Alg. 1-4) and evaluates each piece in closed form (Sec. 5).  Here the
// same integral is written as the signed sum of the three "fans" (origin, v_e, v_{e+1}) over
// the edges -- the signed-area combination of Sec. 4.4, Eq. intermediateWedge, applied to
// every edge at once -- and each fan is cut where its edge leaves the unit disc:
//   * sector pieces (edge beyond r = 1): the cone integrals of Sec. 5.2, radius 1;
//   * the edge piece (r runs to the edge, r <= 1): the segment/stub integrals of
//     Sec. 5.3-5.4.  In the edge's own frame (normal n at distance d, tangent coordinate t),
//     r = rho(t) = sqrt(d^2 + t^2), the angle u obeys du = d dt / rho^2 and the angular
//     factors become algebraic, cos u = d/rho and sin u = t/rho (the role the Chebyshev
//     identities T_a, U_{a-1} of asin/acos play in Sec. 5.1).  Every radial power then
//     reduces to the square-root integrals
//         J_q(t) = int_0^t (d^2 + s^2)^{q/2} ds = t d^q 2F1(-q/2, 1/2; 3/2; -t^2/d^2)
//     of Sec. 5.1, which satisfy the Gauss contiguous relation
//         J_q = (t rho^q + q d^2 J_{q-2}) / (q + 1),   J_0 = t,  J_{-1} = asinh(t/d).
//     On each side of the foot point all terms of the recurrence have one sign, so the
//     upward recurrence is stable as d -> 0 (the particle approaching the edge line, where
//     the paper's 2F1 argument approaches 1 and it resorts to an epsilon shift).
// No branch depends on how many vertices lie inside the support: the paper's case switch
// (Sec. 4.6) becomes clamping of the tangent coordinates to [-sqrt(1-d^2), sqrt(1-d^2)].
//
// Outputs per triangle (raw, without the constant C, the orientation sign or 1/H):
//   g      = int k(|p|) dA
//   gx,gy  = int k'(|p|) p/|p| dA
//   m[10]  = int p_x^a p_y^b k(|p|) dA   in the order 00 10 01 20 11 02 30 21 12 03
#pragma once

#include <math.h>
#include <string.h>

#include "log_table.h"

#if defined(__CUDACC__)
#define SPH2D_HD __host__ __device__ __forceinline__
#else
#define SPH2D_HD inline
#include <cmath>
#endif

// Code shape (measured on GB300): the radial recurrence is unrolled with compile-time
// coefficients (zero terms vanish) -- SPH2D_Q_UNROLL=0 selects a loop over rows of a
// constant-memory table instead, which measured 15-40% slower.  The three fans of a triangle
// are a loop (tri_raw below); the two-piece cubic spline loops over its pieces and their fans
// (six inlined fans overflow the instruction cache: 3.5x slower measured).
#ifndef SPH2D_Q_UNROLL
#define SPH2D_Q_UNROLL 1
#endif
// compensated division of the recurrence by q + 1: exact small-integer division (1) or a
// multiplication by the compensated reciprocal (0)
#ifndef SPH2D_DIVQ
#define SPH2D_DIVQ 1
#endif


namespace sph2d {

#if !defined(__CUDA_ARCH__)
using std::atan2;
using std::fabs;
using std::fmax;
using std::fmin;
using std::log;
using std::sqrt;
#endif

enum : int { KID_WC2 = 0, KID_WC4 = 1, KID_WC6 = 2, KID_CUBIC = 3 };

// ---------------------------------------------------------------------------------------
// kernel polynomials k(q) = sum_k b_k q^k (Sec. 2: integer powers of q); the cubic spline is
// split into compact pieces 2 (1-q)^3_+ - (1-2q)^3_+ so every piece is one polynomial on
// its own support (Sec. 2, piecewise kernels "by careful evaluation of the bounds").
// ---------------------------------------------------------------------------------------
struct PolyWC2 {
  static constexpr int K = 5;
  SPH2D_HD static constexpr double b(int k) {
    return k == 0 ? 1.0 : k == 2 ? -10.0 : k == 3 ? 20.0 : k == 4 ? -15.0 : k == 5 ? 4.0 : 0.0;
  }
};
struct PolyWC4 {
  static constexpr int K = 8;
  SPH2D_HD static constexpr double b(int k) {
    return k == 0 ? 1.0 : k == 2 ? -28.0 / 3.0 : k == 4 ? 70.0 : k == 5 ? -448.0 / 3.0
         : k == 6 ? 140.0 : k == 7 ? -64.0 : k == 8 ? 35.0 / 3.0 : 0.0;
  }
};
struct PolyWC6 {
  static constexpr int K = 11;
  SPH2D_HD static constexpr double b(int k) {
    return k == 0 ? 1.0 : k == 2 ? -11.0 : k == 4 ? 66.0 : k == 6 ? -462.0 : k == 7 ? 1056.0
         : k == 8 ? -1155.0 : k == 9 ? 704.0 : k == 10 ? -231.0 : k == 11 ? 32.0 : 0.0;
  }
};
struct PolyCubeIn {  // cubic spline for q < 1/2: 1 - 6 q^2 + 6 q^3
  static constexpr int K = 3;
  SPH2D_HD static constexpr double b(int k) { return k == 0 ? 1.0 : k == 2 ? -6.0 : k == 3 ? 6.0 : 0.0; }
};
struct PolyCubeOut {  // cubic spline for 1/2 <= q < 1: 2 (1-q)^3
  static constexpr int K = 3;
  SPH2D_HD static constexpr double b(int k) { return k == 0 ? 2.0 : k == 1 ? -6.0 : k == 2 ? 6.0 : k == 3 ? -2.0 : 0.0; }
};
struct PolyCube {  // (1-q)^3
  static constexpr int K = 3;
  SPH2D_HD static constexpr double b(int k) {
    return k == 0 ? 1.0 : k == 1 ? -3.0 : k == 2 ? 3.0 : k == 3 ? -1.0 : 0.0;
  }
};

// sum_k b_k / (k + n)
template <class P>
SPH2D_HD constexpr double kappa(int n) {
  double s = 0.0;
  for (int k = 0; k <= P::K; ++k) s += P::b(k) / double(k + n);
  return s;
}
// sum_k k b_k / (k + 1)   (int_0^1 k'(r) r dr)
template <class P>
SPH2D_HD constexpr double kappa_grad() {
  double s = 0.0;
  for (int k = 1; k <= P::K; ++k) s += double(k) * P::b(k) / double(k + 1);
  return s;
}

// int_0^1 k(q) dq (the cubic spline: 2 int (1-q)^3 - int_0^(1/2) (1-2q)^3 = (2 - 1/2) int_0^1 (1-q)^3)
SPH2D_HD constexpr double kernel_int0(int kid) {
  return kid == KID_WC2 ? kappa<PolyWC2>(1)
       : kid == KID_WC4 ? kappa<PolyWC4>(1)
       : kid == KID_WC6 ? kappa<PolyWC6>(1)
                        : 1.5 * kappa<PolyCube>(1);
}

// 2-D normalisation constants C (int W = 1)
SPH2D_HD constexpr double kernel_C(int kid) {
  return kid == KID_WC2 ? 7.0 / 3.14159265358979323846
       : kid == KID_WC4 ? 9.0 / 3.14159265358979323846
       : kid == KID_WC6 ? 78.0 / (7.0 * 3.14159265358979323846)
                        : 40.0 / (7.0 * 3.14159265358979323846);
}

template <typename R>
struct PairOut {
  R g, gx, gy;
  R m[10];
};

template <typename R>
SPH2D_HD void clear(PairOut<R>& o) {
  o.g = o.gx = o.gy = R(0);
#pragma unroll
  for (int i = 0; i < 10; ++i) o.m[i] = R(0);
}

template <typename R> struct Tiny;
template <> struct Tiny<double> { SPH2D_HD static constexpr double v() { return 1e-150; } };
template <> struct Tiny<float> { SPH2D_HD static constexpr float v() { return 1e-18f; } };

// a*b - c*d.  In FP32 Kahan's compensated form (W. Kahan's algorithm for ad - bc; error bound
// 1.5 ulp of the result from C.-P. Jeannerod, N. Louvet, J.-M. Muller, Math. Comp. 82 (2013)),
// so that a cross product of nearly parallel vectors keeps its relative accuracy.
SPH2D_HD double diff_of_products(double a, double b, double c, double d) { return a * b - c * d; }
SPH2D_HD float diff_of_products(float a, float b, float c, float d) {
#if defined(__CUDA_ARCH__)
  float w = c * d;
  float e = __fmaf_rn(-c, d, w);
  float f = __fmaf_rn(a, b, -w);
  return f + e;
#else
  float w = c * d;
  float e = std::fma(-c, d, w);
  float f = std::fma(a, b, -w);
  return f + e;
#endif
}

// asinh(t2/d) - asinh(t1/d), with rho_i = sqrt(d^2 + t_i^2) given and |t| + rho >= d
// formed without cancellation (asinh(t/d) = sgn(t) log((|t| + rho)/d)).
template <typename R>
SPH2D_HD R asinh_diff(R t1, R t2, R r1, R r2, R d) {
  const R a1 = fabs(t1) + r1, a2 = fabs(t2) + r2;
  const bool p1 = t1 >= R(0), p2 = t2 >= R(0);
  if (p1 == p2) {
    const R l = log(a2 / a1);
    return p2 ? l : -l;
  }
  const R l = log((a1 / d) * (a2 / d));
  return p2 ? l : -l;
}

// ---------------------------------------------------------------------------------------
// compensated FP32 ("float-float"): value = hi + lo with |lo| <= ulp(hi)/2, built from FMA
// error-free transformations.  Used for the radial recurrence and the kernel-coefficient
// sums of the FP32 path, whose alternating coefficients (sum |b_k|/(k+2) is 140x to 9000x
// the result for C2..C6) would otherwise amplify FP32 rounding by the same factor.
// Published sources of the building blocks: two-sum (D. E. Knuth, TAOCP vol. 2, Sec. 4.2.2),
// fast two-sum and the splitting of a double into two halves (T. J. Dekker, "A floating-point
// technique for extending the available precision", Numer. Math. 18, 1971), the FMA two-product
// (the exact residual fma(a, b, -a*b); see T. Ogita, S. M. Rump, S. Oishi, "Accurate sum and
// dot product", SIAM J. Sci. Comput. 26, 2005), and pair addition, multiplication and division
// by two quotient digits (Dekker 1971, in the double-length arithmetic of D. H. Bailey's
// double-double libraries).
// ---------------------------------------------------------------------------------------
template <typename F>
struct FFT {
  F hi, lo;
};
using FF = FFT<float>;
SPH2D_HD float fma_f(float a, float b, float c) {
#if defined(__CUDA_ARCH__)
  return __fmaf_rn(a, b, c);
#else
  return std::fma(a, b, c);
#endif
}
SPH2D_HD double fma_f(double a, double b, double c) {
#if defined(__CUDA_ARCH__)
  return __fma_rn(a, b, c);
#else
  return std::fma(a, b, c);
#endif
}
// a / b for the FP32 path's geometry and the correction digits of float-pair roots and
// quotients: the hardware's fast division on the GPU (within 2 ulp for |b| in [2^-126, 2^126]),
// exact division elsewhere and in double
SPH2D_HD float div_fast(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fdividef(a, b);
#else
  return a / b;
#endif
}
SPH2D_HD double div_fast(double a, double b) { return a / b; }
template <typename T>
SPH2D_HD T div_fast(T a, T b) { return a / b; }
// 1 / sqrt(x) and sqrt(x) for x > 0 the same way: the hardware's reciprocal square root on the
// GPU (within 2 ulp) for the FP32 geometry and the first digit of the float-pair root
SPH2D_HD float rsqrt_fast(float x) {
#if defined(__CUDA_ARCH__)
  return rsqrtf(x);
#else
  return 1.0f / std::sqrt(x);
#endif
}
SPH2D_HD double rsqrt_fast(double x) { return 1.0 / sqrt(x); }
template <typename T>
SPH2D_HD T rsqrt_fast(T x) { return T(1) / sqrt(x); }
SPH2D_HD float sqrt_fast(float x) {
#if defined(__CUDA_ARCH__)
  return x * rsqrtf(x);
#else
  return std::sqrt(x);
#endif
}
SPH2D_HD double sqrt_fast(double x) { return sqrt(x); }
template <typename T>
SPH2D_HD T sqrt_fast(T x) { return sqrt(x); }

// atan2 for the FP32 fan angles: t = min(|x|, |y|) / max(|x|, |y|) in [0, 1], atan t = t P(t^2)
// with P of degree 9 (its coefficients: a least-squares fit on [0, 1] reweighted by Lawson's
// method toward the smallest maximum relative error of atan, 2.4e-9 in exact arithmetic, made for
// this library), then the octant and quadrant reflections pi/2 - a and pi - a and the sign of y.
// Within 2.1 ulp and 2.9e-7 absolute of the exact atan2 over 2e6 random arguments (FP32
// evaluation); x = y = 0 does not occur here (degenerate fans return before).
SPH2D_HD float atan2_fast(float y, float x) {
  const float ax = fabsf(x), ay = fabsf(y);
  const float t = div_fast(fminf(ax, ay), fmaxf(ax, ay)), w = t * t;
  float p = -1.753866789e-03f;
  p = fma_f(p, w, 1.072655618e-02f);
  p = fma_f(p, w, -3.080365062e-02f);
  p = fma_f(p, w, 5.755088106e-02f);
  p = fma_f(p, w, -8.377224952e-02f);
  p = fma_f(p, w, 1.094199046e-01f);
  p = fma_f(p, w, -1.426192224e-01f);
  p = fma_f(p, w, 1.999826431e-01f);
  p = fma_f(p, w, -3.333328366e-01f);
  p = fma_f(p, w, 1.0f);
  float a = t * p;
  if (ay > ax) a = 1.57079637f - a;
  if (x < 0.0f) a = 3.14159274f - a;
  return copysignf(a, y);
}
SPH2D_HD double atan2_fast(double y, double x) { return atan2(y, x); }
template <typename T>
SPH2D_HD T atan2_fast(T y, T x) { return atan2(y, x); }

// num/den as a double-double, for small integer den: hi = num/den rounded, lo = the exact
// residual (num - hi*den)/den, with hi*den formed exactly from a Dekker split of hi
SPH2D_HD constexpr FFT<double> dd_rational(double num, double den) {
  const double hi = num / den;
  const double cs = 134217729.0 * hi;
  const double h1 = cs - (cs - hi), h2 = hi - h1;
  const double r = (num - h1 * den) - h2 * den;
  return FFT<double>{hi, r / den};
}
SPH2D_HD constexpr FF ff_const(double c) {
  return FF{float(c), float(c - double(float(c)))};
}
template <typename F>
SPH2D_HD FFT<F> ff_two_sum(F a, F b) {
  const F s = a + b;
  const F bb = s - a;
  return FFT<F>{s, (a - (s - bb)) + (b - bb)};
}
template <typename F>
SPH2D_HD FFT<F> ff_fast_two_sum(F a, F b) {
  const F s = a + b;
  return FFT<F>{s, b - (s - a)};
}
template <typename F>
SPH2D_HD FFT<F> ff_two_prod(F a, F b) {
  const F p = a * b;
  return FFT<F>{p, fma_f(a, b, -p)};
}
// error <= eps^2 (|a| + |b|): adequate where cancellation is between large terms
template <typename F>
SPH2D_HD FFT<F> operator+(FFT<F> a, FFT<F> b) {
  const FFT<F> s = ff_two_sum(a.hi, b.hi);
  return ff_fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
template <typename F>
SPH2D_HD FFT<F> operator-(FFT<F> a) { return FFT<F>{-a.hi, -a.lo}; }
template <typename F>
SPH2D_HD FFT<F> operator-(FFT<F> a, FFT<F> b) { return a + (-b); }
// Products return their two words without the final renormalisation unless
// SPH2D_FF_NORM_PRODUCTS is set: every product here feeds an addition, which renormalises, or
// another product, and the low word then stays within a few units of the high word's last
// place, so the dropped lo x lo term stays far below the pair's unit roundoff.  Measured on the
// 1024^2 box: FP32 passes 5-14% faster (C2 with ten moments 2.77 -> 2.39 ms), results within
// 2.4e-7 of the FP64 form as before.
#ifndef SPH2D_FF_NORM_PRODUCTS
#define SPH2D_FF_NORM_PRODUCTS 0
#endif
template <typename F>
SPH2D_HD FFT<F> operator*(FFT<F> a, FFT<F> b) {
  const FFT<F> p = ff_two_prod(a.hi, b.hi);
#if SPH2D_FF_NORM_PRODUCTS
  return ff_fast_two_sum(p.hi, fma_f(a.hi, b.lo, fma_f(a.lo, b.hi, p.lo)));
#else
  return FFT<F>{p.hi, fma_f(a.hi, b.lo, fma_f(a.lo, b.hi, p.lo))};
#endif
}
template <typename F>
SPH2D_HD FFT<F> operator*(FFT<F> a, F b) {
  const FFT<F> p = ff_two_prod(a.hi, b);
#if SPH2D_FF_NORM_PRODUCTS
  return ff_fast_two_sum(p.hi, fma_f(a.lo, b, p.lo));
#else
  return FFT<F>{p.hi, fma_f(a.lo, b, p.lo)};
#endif
}
template <typename F>
SPH2D_HD FFT<F> ff_sqrt(FFT<F> x) {               // one Newton step on sqrt(hi)
  if (x.hi <= F(0)) return FFT<F>{F(0), F(0)};
  const F r = sqrt_fast(x.hi);
  const FFT<F> r2 = ff_two_prod(r, r);
  const F res = ((x.hi - r2.hi) - r2.lo) + x.lo;
  return ff_fast_two_sum(r, div_fast(res, F(2) * r));
}
template <typename F>
SPH2D_HD F to_f(FFT<F> a) { return a.hi + a.lo; }

// Two values of the same operation side by side.  For float on sm_100-family GPUs each
// operation is one packed instruction (fma/mul .rn.f32x2: the same FP32 lanes, half the issue
// slots); elsewhere it is two scalar operations.
template <typename F>
struct V2 {
  F x, y;
};
template <typename F>
SPH2D_HD V2<F> v2_fma(V2<F> a, V2<F> b, V2<F> c) { return V2<F>{fma_f(a.x, b.x, c.x), fma_f(a.y, b.y, c.y)}; }
template <typename F>
SPH2D_HD V2<F> v2_mul(V2<F> a, V2<F> b) { return V2<F>{a.x * b.x, a.y * b.y}; }
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
SPH2D_HD V2<float> v2_fma(V2<float> a, V2<float> b, V2<float> c) {
  const float2 r = __ffma2_rn(make_float2(a.x, a.y), make_float2(b.x, b.y), make_float2(c.x, c.y));
  return V2<float>{r.x, r.y};
}
SPH2D_HD V2<float> v2_mul(V2<float> a, V2<float> b) {
  const float2 r = __fmul2_rn(make_float2(a.x, a.y), make_float2(b.x, b.y));
  return V2<float>{r.x, r.y};
}
#endif
template <typename F>
SPH2D_HD FFT<F> operator/(FFT<F> a, FFT<F> b) {   // long division, two quotient digits
  const F q1 = div_fast(a.hi, b.hi);
  const FFT<F> r = a - b * q1;
  const F q2 = div_fast(r.hi, b.hi);
  return ff_fast_two_sum(q1, q2);
}
template <typename F>
SPH2D_HD FFT<F> ffc(double c) {
  const FF v = ff_const(c);
  return FFT<F>{F(v.hi), F(v.lo)};
}
// num/den as a compensated constant of the base precision B (float pair or double pair)
template <typename F, typename B>
SPH2D_HD FFT<F> ffk(double num, double den) {
  if (sizeof(B) == sizeof(double)) {
    const FFT<double> v = dd_rational(num, den);
    return FFT<F>{F(v.hi), F(v.lo)};
  }
  const FF v = ff_const(num / den);
  return FFT<F>{F(v.hi), F(v.lo)};
}
// ln 2 to ~2^-106: 0.6931471805599453094172321214581766 = hi + lo
template <typename F, typename B>
SPH2D_HD FFT<F> ffln2() {
  if (sizeof(B) == sizeof(double))
    return FFT<F>{F(0.6931471805599453094), F(2.3190468138462996e-17)};
  const FF v = ff_const(0.69314718055994530942);
  return FFT<F>{F(v.hi), F(v.lo)};
}
SPH2D_HD float frexp_f(float x, int* e) {
#if defined(__CUDA_ARCH__)
  return frexpf(x, e);
#else
  return std::frexp(x, e);
#endif
}
SPH2D_HD double frexp_f(double x, int* e) {
#if defined(__CUDA_ARCH__)
  return frexp(x, e);
#else
  return std::frexp(x, e);
#endif
}
SPH2D_HD double ldexp_f(double x, int e) {
#if defined(__CUDA_ARCH__)
  return ldexp(x, e);
#else
  return std::ldexp(x, e);
#endif
}
SPH2D_HD float ldexp_f(float x, int e) {
#if defined(__CUDA_ARCH__)
  return ldexpf(x, e);
#else
  return std::ldexp(x, e);
#endif
}
// the machine value of a scalar (the op counter's counted types define their own)
SPH2D_HD float raw_f(float x) { return x; }
SPH2D_HD double raw_f(double x) { return x; }

// an exact power-of-two scale and its inverse
template <typename F>
struct Pow2 {
  F s, is;
};
// For finite non-zero x: s = 2^-e and is = 2^e, with 2^(e-1) <= |x| < 2^e, so that |x| s lies in
// [1/2, 1); e is taken from the exponent field and held at -64 or above (s <= 2^64).
SPH2D_HD Pow2<float> pow2_scale(float x) {
#if defined(__CUDA_ARCH__)
  const unsigned b = __float_as_uint(x);
#else
  unsigned b;
  memcpy(&b, &x, sizeof b);
#endif
  int e = int((b >> 23) & 0xffu) - 126;
  e = e < -64 ? -64 : e;
  const unsigned us = unsigned(127 - e) << 23, ui = unsigned(127 + e) << 23;
#if defined(__CUDA_ARCH__)
  return Pow2<float>{__uint_as_float(us), __uint_as_float(ui)};
#else
  Pow2<float> r;
  memcpy(&r.s, &us, sizeof us);
  memcpy(&r.is, &ui, sizeof ui);
  return r;
#endif
}

// argument-reduction table of ff_log (log_table.h, written by gen_log_table.py): entry i holds
// inv = 1/c_i rounded to the working precision (c_i = (64 + i)/128) and -ln(inv) as hi + lo
template <typename B> struct LogEnt { B inv, hi, lo; };
#if defined(__CUDACC__)
static __device__ const LogEnt<float> g_log_table_f_dev[128] = {SPH2D_LOG_TABLE_F};
static __device__ const LogEnt<double> g_log_table_d_dev[128] = {SPH2D_LOG_TABLE_D};
#endif
static const LogEnt<float> g_log_table_f_host[128] = {SPH2D_LOG_TABLE_F};
static const LogEnt<double> g_log_table_d_host[128] = {SPH2D_LOG_TABLE_D};
template <bool DBL> struct LogEntType { using type = LogEnt<float>; };
template <> struct LogEntType<true> { using type = LogEnt<double>; };
template <bool DBL>
SPH2D_HD typename LogEntType<DBL>::type log_entry(int i) {
  if constexpr (DBL) {
#if defined(__CUDA_ARCH__)
    return g_log_table_d_dev[i];
#else
    return g_log_table_d_host[i];
#endif
  } else {
#if defined(__CUDA_ARCH__)
    return g_log_table_f_dev[i];
#else
    return g_log_table_f_host[i];
#endif
  }
}

// The log's argument split: x = 2^e xm with xm.hi in [1/sqrt2, sqrt2), both words scaled exactly.
template <typename F>
SPH2D_HD FFT<F> log_split(FFT<F> x, int& e) {
  const F m0 = frexp_f(x.hi, &e);                        // [1/2, 1)
  // (all of this in the working precision: a double literal here would put FP64 instructions
  // into the FP32 kernels)
  using MF = decltype(raw_f(m0));
  if (raw_f(m0) < MF(0.70710678118654752)) e -= 1;       // m = x.hi 2^-e in [1/sqrt2, sqrt2)
  return FFT<F>{ldexp_f(x.hi, -e), ldexp_f(x.lo, -e)};
}
// float pairs on the GPU: straight from the exponent field and the leading mantissa bits, with
// one exact product by 2^-e per word.  x.hi is a positive normal float here: the log's arguments
// are ratios of sums |t| + rho >= d >= 1e-18 with |t| below 64 (local coordinates past 16 take
// the FP64 path), between 1e-20 and 1e37.
SPH2D_HD FFT<float> log_split(FFT<float> x, int& e) {
#if defined(__CUDA_ARCH__)
  const unsigned b = __float_as_uint(x.hi);
  e = int((b >> 23) & 0xffu) - 126 - ((b & 0x7fffffu) < 0x3504f3u ? 1 : 0);
  const float sc = __uint_as_float(unsigned(127 - e) << 23);
  return FFT<float>{x.hi * sc, x.lo * sc};
#else
  const float m0 = std::frexp(x.hi, &e);
  if (m0 < 0.70710678118654752f) e -= 1;
  return FFT<float>{std::ldexp(x.hi, -e), std::ldexp(x.lo, -e)};
#endif
}

// natural log of x > 0 in compensated arithmetic (float pairs, or double pairs for B = double).
// Table reduction (Tang's method): x = 2^e m with m in [1/sqrt2, sqrt2), and c_i = (64 + i)/128
// the table point nearest m, so that
//   ln x = e ln 2 + L_i + ln(1 + r),   r = m inv_i - 1,
// with inv_i = 1/c_i rounded, L_i = -ln(inv_i) exact for the stored inv_i, r formed from the
// two-products of both words of m with inv_i (|r| <= 2^-7.5), and ln(1 + r) = sum_k (-1)^(k+1) r^k / k.  The
// terms through r^NP run in pair arithmetic, the rest (through r^NT) in the base precision:
// relative to r their base-precision rounding is below the pair's unit roundoff (float pairs:
// NP = 3, NT = 8; double pairs: NP = 7, NT = 15).  Every x near 1, on either side, has e = 0 and
// c = 1 (inv = 1, L = 0): r = x - 1 exactly, so a small logarithm keeps its relative accuracy.
template <typename F, typename B = F>
SPH2D_HD FFT<F> ff_log(FFT<F> x) {
  constexpr bool DBL = sizeof(B) == sizeof(double);
  constexpr int NP = DBL ? 7 : 3, NT = DBL ? 15 : 8;
  int e = 0;
  const FFT<F> xm = log_split(x, e);                     // x = 2^e xm, xm.hi in [1/sqrt2, sqrt2)
  using MF = decltype(raw_f(xm.hi));
  const int i = int(raw_f(xm.hi) * MF(128) + MF(0.5)) - 64;   // nearest table point (either one at a tie)
  const auto ent = log_entry<DBL>(i);
  const F inv = F(ent.inv);
  const FFT<F> p = ff_two_prod(xm.hi, inv), q = ff_two_prod(xm.lo, inv);   // exact
  const FFT<F> r = ff_fast_two_sum(p.hi - F(1), p.lo) + q; // p.hi - 1 exact (Sterbenz), |p.hi - 1| >= |p.lo|
  const F rh = r.hi;
  F tail = F(((NT & 1) ? 1.0 : -1.0) / double(NT));
#pragma unroll
  for (int k = NT - 1; k > NP; --k) tail = fma_f(tail, rh, F(((k & 1) ? 1.0 : -1.0) / double(k)));
  F rp = rh;
#pragma unroll
  for (int k = 0; k < NP; ++k) rp = rp * rh;             // r^(NP+1)
  tail = tail * rp;
  FFT<F> S = ffk<F, B>(((NP & 1) ? 1.0 : -1.0), double(NP));
#pragma unroll
  for (int k = NP - 1; k >= 1; --k) S = S * r + ffk<F, B>(((k & 1) ? 1.0 : -1.0), double(k));
  const FFT<F> l1p = r * S + FFT<F>{tail, F(0)};
  return (l1p + FFT<F>{F(ent.hi), F(ent.lo)}) + ffln2<F, B>() * F(MF(e));
}

// asinh(t2/d) - asinh(t1/d) in FF (see asinh_diff)
template <typename F, typename B = F>
SPH2D_HD FFT<F> asinh_diff_ff(F t1, F t2, FFT<F> r1, FFT<F> r2, F d) {
  const FFT<F> a1 = r1 + FFT<F>{fabs(t1), F(0)}, a2 = r2 + FFT<F>{fabs(t2), F(0)};
  const bool p1 = t1 >= F(0), p2 = t2 >= F(0);
  FFT<F> l;
  if (p1 == p2) {
    l = ff_log<F, B>(a2 / a1);
  } else {
    const FFT<F> dd{d, F(0)};
    l = ff_log<F, B>((a1 / dd) * (a2 / dd));
  }
  return p2 ? l : -l;
}

// ---------------------------------------------------------------------------------------
// per-step coefficient rows of the edge-piece sums.  Step q of the recurrence produces
// Delta J_q and Delta rho^q; each running sum adds them times a constant that depends only on
// the kernel polynomial and q (b_k = 0 outside 0..K):
//   gamma      Sg  += dJ  b_q/(q+2)              grad n  Sn  += dJ (q+2) b_{q+2}/(q+3)
//   grad t     St  += dP  b_q/(q+1)
//   M10,M20,M30      += dJ  b_q/(q+3), b_q/(q+4), b_q/(q+5)
//   M02, M12         += dJ  b_{q-2}/(q+2) | b_{q-2}/(q+3)   and  dJ d^2 (-b_q/(q+4) | -b_q/(q+5))
//   M01, M11, M21    += dP  b_{q-2}/((q+1+m-1) q)   (m = 1, 2, 3)
//   M03              += dP  b_{q-4}/((q+1) q)        and  dP d^2 (-b_{q-2}/((q+3) q))
// The d^2 parts of M02, M12 and M03 are -d^2 times the M20, M30 and M21 sums (same rows), so
// they are not accumulated: the three sums are S02A - d^2 S20, S12A - d^2 S30 and S03A - d^2 S21,
// formed once per fan in the accumulation precision.
// With SPH2D_Q_UNROLL=0 the rows live in constant memory (the step index is uniform across a
// warp) so the recurrence loop needs no unrolling.
// ---------------------------------------------------------------------------------------
enum : int {
  SL_G = 0, SL_N, SL_T, SL_10, SL_20, SL_30, SL_02A, SL_12A,
  SL_01, SL_11, SL_21, SL_03A, NSL
};
struct NumDen {
  double num, den;
};
template <class P>
SPH2D_HD constexpr double bk(int k) { return (k < 0 || k > P::K) ? 0.0 : P::b(k); }
template <class P>
SPH2D_HD constexpr NumDen edge_coef(int q, int s) {
  const double Q = double(q);
  switch (s) {
    case SL_G: return {bk<P>(q), Q + 2};
    case SL_N: return {(Q + 2) * bk<P>(q + 2), Q + 3};
    case SL_T: return q >= 1 ? NumDen{bk<P>(q), Q + 1} : NumDen{0.0, 1.0};
    case SL_10: return {bk<P>(q), Q + 3};
    case SL_20: return {bk<P>(q), Q + 4};
    case SL_30: return {bk<P>(q), Q + 5};
    case SL_02A: return {bk<P>(q - 2), Q + 2};
    case SL_12A: return {bk<P>(q - 2), Q + 3};
    case SL_01: return q >= 1 ? NumDen{bk<P>(q - 2), (Q + 1) * Q} : NumDen{0.0, 1.0};
    case SL_11: return q >= 1 ? NumDen{bk<P>(q - 2), (Q + 2) * Q} : NumDen{0.0, 1.0};
    case SL_21: return q >= 1 ? NumDen{bk<P>(q - 2), (Q + 3) * Q} : NumDen{0.0, 1.0};
    case SL_03A: return q >= 1 ? NumDen{bk<P>(q - 4), (Q + 1) * Q} : NumDen{0.0, 1.0};
  }
  return {0.0, 1.0};
}
// the slots whose inputs are Delta rho^q (the others take Delta J_q)
SPH2D_HD constexpr bool slot_uses_drho(int s) {
  return s == SL_T || s == SL_01 || s == SL_11 || s == SL_21 || s == SL_03A;
}
// the double factorial n!! (1 for n <= 0)
SPH2D_HD constexpr double dfact(int n) {
  double f = 1.0;
  for (int k = n; k > 1; k -= 2) f *= double(k);
  return f;
}
// Rows of the FP32 path, whose recurrence runs on Y_q = J_q / w_q with w_q = q!!/(q+1)!!
// (w_-1 = w_0 = 1): the J_q rows carry the factor w_q, the rho^q rows are unchanged.  With
// that scaling the recurrence J_q = (Delta(t rho^q) + q d^2 J_{q-2}) / (q + 1) reads
// Y_q = Delta(t rho^q) (q-1)!!/q!! + d^2 Y_{q-2}: one constant product instead of the division
// and the product by q.
template <class P>
SPH2D_HD constexpr NumDen edge_coef_y(int q, int s) {
  const NumDen c = edge_coef<P>(q, s);
  if (slot_uses_drho(s) || q < 1) return c;
  return NumDen{c.num * dfact(q), c.den * dfact(q + 1)};
}
// Exact FP32 rows.  Every b_k has a denominator dividing 3, so each entry of edge_coef_y is a
// ratio n/d of small integers.  Scaled by D_P, the odd part of the least common multiple of all
// of a polynomial's denominators, every entry becomes an integer over a power of two; where the
// odd parts of those integers all stay below 2^24 (Wendland C2 and C4, the cubic spline; not C6)
// the scaled rows are exact in FP32.  The FP32 path then runs the whole fan computation scaled by
// D_P (sector constants included) with one FP32 coefficient per sum term instead of a float
// pair, and tri_poly multiplies the pair's outputs by 1/D_P once.
struct RatI {
  long long n, d;
};
SPH2D_HD constexpr long long gcd_ll(long long a, long long b) {
  a = a < 0 ? -a : a;
  b = b < 0 ? -b : b;
  while (b != 0) {
    const long long t = a % b;
    a = b;
    b = t;
  }
  return a;
}
SPH2D_HD constexpr long long round_ll(double x) {
  return x >= 0.0 ? (long long)(x + 0.5) : -(long long)(-x + 0.5);
}
SPH2D_HD constexpr long long odd_part(long long v) {
  while (v != 0 && v % 2 == 0) v /= 2;
  return v;
}
template <class P>
SPH2D_HD constexpr RatI edge_rat_y(int q, int s) {
  const NumDen c = edge_coef_y<P>(q, s);
  long long n = round_ll(c.num * 3.0), d = round_ll(c.den) * 3;
  if (n == 0) return RatI{0, 1};
  const long long g = gcd_ll(n, d);
  n /= g;
  d /= g;
  return d < 0 ? RatI{-n, -d} : RatI{n, d};
}
template <class P>
SPH2D_HD constexpr long long poly_lcm() {
  long long L = 1;
  for (int s = 0; s < NSL; ++s)
    for (int q = -1; q <= P::K + 4; ++q) {
      const long long d = odd_part(edge_rat_y<P>(q, s).d);
      L = L / gcd_ll(L, d) * d;
    }
  return L;
}
// D_P where the scaled rows are exact in FP32, else 0 (the rows keep float-pair coefficients)
template <class P>
SPH2D_HD constexpr long long poly_den_eval() {
  const long long L = poly_lcm<P>();
  for (int s = 0; s < NSL; ++s)
    for (int q = -1; q <= P::K + 4; ++q) {
      const RatI r = edge_rat_y<P>(q, s);
      if (r.n == 0) continue;
      const long long m = odd_part(r.n) * (L / odd_part(r.d));
      if ((m < 0 ? -m : m) >= (1LL << 24)) return 0;
    }
  return L;
}
// evaluated once, at compile time (the device code only reads the constants)
template <class P>
struct PolyDen {
  static constexpr long long v = poly_den_eval<P>();
  static constexpr double scale = v > 0 ? double(v) : 1.0;
};
template <class P>
SPH2D_HD constexpr long long poly_den() { return PolyDen<P>::v; }
// the FP32 path's scale of polynomial P (1 where the rows are not exact)
template <class P>
SPH2D_HD constexpr double poly_scale() { return PolyDen<P>::scale; }
// edge_coef_y(q, s) times D_P, exact in FP32 (0 for P without exact rows): the double product
// is within 2^-52 of the exact value, which is an FP32 number, so the rounding to FP32 recovers it
// (checked against the integer form by rows_exact_in_fp32)
template <class P>
SPH2D_HD constexpr double edge_coef_s(int q, int s) {
  if (PolyDen<P>::v == 0) return 0.0;
  const NumDen c = edge_coef_y<P>(q, s);
  return c.num == 0.0 ? 0.0 : double(float(c.num / c.den * PolyDen<P>::scale));
}
template <class P>
SPH2D_HD constexpr bool rows_exact_in_fp32() {
  if (poly_den<P>() == 0) return true;
  for (int q = -1; q <= P::K + 4; ++q)
    for (int s = 0; s < NSL; ++s) {
      const RatI r = edge_rat_y<P>(q, s);
      const long long od = odd_part(r.d);
      const double exact = r.n == 0 ? 0.0 : double(r.n * (poly_den<P>() / od)) / double(r.d / od);
      if (edge_coef_s<P>(q, s) != exact || double(float(exact)) != exact) return false;
    }
  return true;
}
template <class P>
struct EdgeRows {
  static constexpr int QMIN = -1, QMAX = P::K + 4, ROWS = QMAX - QMIN + 1;
  double d[ROWS][NSL];                    // double
  double dlo[ROWS][NSL];                  // double-double low parts
  float fhi[ROWS][NSL], flo[ROWS][NSL];   // float-float
  float fs[ROWS][NSL];                    // the FP32 path's exact rows, times D_P (edge_coef_s)
  constexpr EdgeRows() : d(), dlo(), fhi(), flo(), fs() {
    for (int q = QMIN; q <= QMAX; ++q)
      for (int s = 0; s < NSL; ++s) {
        const NumDen c = edge_coef<P>(q, s);
        const FFT<double> dd = dd_rational(c.num, c.den);
        d[q - QMIN][s] = dd.hi;
        dlo[q - QMIN][s] = dd.lo;
        const NumDen cy = edge_coef_y<P>(q, s);
        const FF ff = ff_const(cy.num / cy.den);
        fhi[q - QMIN][s] = ff.hi;
        flo[q - QMIN][s] = ff.lo;
        fs[q - QMIN][s] = float(edge_coef_s<P>(q, s));
      }
  }
};
#if defined(__CUDACC__) && !SPH2D_Q_UNROLL
static __constant__ EdgeRows<PolyWC2> g_rows_wc2 = EdgeRows<PolyWC2>();
static __constant__ EdgeRows<PolyWC4> g_rows_wc4 = EdgeRows<PolyWC4>();
static __constant__ EdgeRows<PolyWC6> g_rows_wc6 = EdgeRows<PolyWC6>();
static __constant__ EdgeRows<PolyCube> g_rows_cube = EdgeRows<PolyCube>();
#endif
template <class P>
struct HostRows {
  static constexpr EdgeRows<P> rows = EdgeRows<P>();
};
template <class P> SPH2D_HD const EdgeRows<P>& edge_rows();
#if defined(__CUDA_ARCH__) && !SPH2D_Q_UNROLL
#define SPH2D_ROWS(POLY, VAR) \
  template <> SPH2D_HD const EdgeRows<POLY>& edge_rows<POLY>() { return VAR; }
#else
#define SPH2D_ROWS(POLY, VAR) \
  template <> SPH2D_HD const EdgeRows<POLY>& edge_rows<POLY>() { return HostRows<POLY>::rows; }
#endif
SPH2D_ROWS(PolyWC2, g_rows_wc2)
SPH2D_ROWS(PolyWC4, g_rows_wc4)
SPH2D_ROWS(PolyWC6, g_rows_wc6)
SPH2D_ROWS(PolyCube, g_rows_cube)
#undef SPH2D_ROWS
static_assert(rows_exact_in_fp32<PolyWC2>() && rows_exact_in_fp32<PolyWC4>() && rows_exact_in_fp32<PolyWC6>() &&
                  rows_exact_in_fp32<PolyCubeIn>() && rows_exact_in_fp32<PolyCubeOut>() &&
                  rows_exact_in_fp32<PolyCube>(),
              "a scaled edge-sum row is not exact in FP32");
static_assert(poly_den<PolyWC2>() == 315 && poly_den<PolyWC4>() == 57915 && poly_den<PolyCube>() == 105 &&
                  poly_den<PolyWC6>() == 0,
              "exact FP32 rows: unexpected scales");

// compensated running sum for the FF / double-double paths: s + c, where every product
// x*k is formed to ~2^-2p and every addition's rounding error goes into c (compensated
// summation with two-sum, the "Dot2" scheme of Ogita, Rump and Oishi 2005)
template <typename F>
struct CSum {
  F s, c;
};
template <typename F>
SPH2D_HD CSum<F> csum_madd(CSum<F> a, FFT<F> x, F khi, F klo) {
  const F ph = x.hi * khi;
  F pl = fma_f(x.hi, khi, -ph);
  pl = fma_f(x.hi, klo, fma_f(x.lo, khi, pl));
  const F s = a.s + ph;
  const F bb = s - a.s;
  const F err = (a.s - (s - bb)) + (ph - bb);
  return CSum<F>{s, a.c + (err + pl)};
}

// The same sum by error-free extraction against a fixed grid (Rump, Ogita and Oishi, "Accurate
// floating-point summation, part I", SIAM J. Sci. Comput. 31, 2008; the running-sigma form of
// their FastAccSum), for terms bounded in advance.  g is a power of two with |x k| <= g / (2n)
// for all n terms of the sum, and s starts at 3g/2 (xsum_init).  Every t = fl(s + x.hi khi)
// then stays in (g, 2g), on the grid ulp = 2^-23 g, so q = t - s is exact (Sterbenz) and s - 3g/2
// is the exact sum of the q; r = fl(x.hi khi - q) is the remainder, |r| <= 2^-24 g, with one
// rounding.  c collects the remainders, the low word of x and the coefficient's low part.  Five
// or six instructions against the twelve of csum_madd; the error is O(n u^2 g) absolute,
// u = 2^-24, against O(u^2 sum|x k|) there.
template <typename F>
SPH2D_HD CSum<F> xsum_init(float g) { return CSum<F>{F(1.5f * g), F(0)}; }
template <typename F>
SPH2D_HD CSum<F> xsum_madd(CSum<F> a, FFT<F> x, F khi, F klo) {
  const F t = fma_f(x.hi, khi, a.s);
  F r = fma_f(x.hi, khi, a.s - t);
  r = fma_f(x.lo, khi, r);
  if (klo != F(0)) r = fma_f(x.hi, klo, r);
  return CSum<F>{t, a.c + r};
}
// the sum as s + c, with s exact
template <typename F>
SPH2D_HD FFT<F> xsum_result(CSum<F> a, float g) { return ff_two_sum(a.s - F(1.5f * g), a.c); }
// the grid constant g of one edge-sum slot: the smallest power of two with g >= 2 n m (1 + 2^-7),
// n the number of non-zero terms and m the largest |coefficient| times the bound of its input.  The inputs are scaled per fan (add_fan) so that |Delta J_q| < 1 for q >= 0 (and
// q = -1, where the row is used: J_q = int rho^q dt with rho <= 1 on the edge piece, so
// |Delta J_q| <= |Delta t|) and |Delta rho^q| < q (|d rho / dt| <= 1).
template <class P>
SPH2D_HD constexpr float slot_grid(int s) {
  double m = 0.0;
  int n = 0;
  for (int q = -1; q <= P::K + 4; ++q) {
    const NumDen c = edge_coef<P>(q, s);
    if (c.num == 0.0) continue;
    const double w = (c.num < 0 ? -c.num : c.num) / c.den * (slot_uses_drho(s) && q > 1 ? double(q) : 1.0);
    m = w > m ? w : m;
    ++n;
  }
  if (n == 0) return 1.0f;
  const double need = 2.0 * n * m * poly_scale<P>() * (1.0 + 1.0 / 128);   // terms scaled by D_P
  double g = 1.0;
  while (g < need) g *= 2.0;
  while (g * 0.5 >= need) g *= 0.5;
  return float(g);
}
// whether any edge-sum slot takes the q = -1 row (Delta J_-1), i.e. k has a linear term
template <class P>
SPH2D_HD constexpr bool uses_row_m1() {
  for (int s = 0; s < NSL; ++s)
    if (edge_coef<P>(-1, s).num != 0.0) return true;
  return false;
}

// accumulation type of the radial part: plain arithmetic in the base precision F (the FP64
// path, and the bulk FP32 path), or FF compensated FP32 (the FP32 path's compensated form)
template <typename F>
struct AccPlain {
  using T = F;
  SPH2D_HD static constexpr F c(double v) { return F(v); }
  SPH2D_HD static constexpr F c2(double num, double den) { return F(num / den); }
  SPH2D_HD static F from(F v) { return v; }
  SPH2D_HD static F sq(F v) { return v * v; }
  SPH2D_HD static F root(F v) { return sqrt(v); }
  SPH2D_HD static F out(F v) { return v; }
  SPH2D_HD static F mulr(F a, F b) { return a * b; }
  using Sum = F;
  static constexpr bool SCALED = false;                // edge sums on unscaled inputs
  SPH2D_HD static F zero() { return F(0); }
  SPH2D_HD static F zero_g(float) { return F(0); }     // slot sums (g: the slot's grid)
  SPH2D_HD static F result_g(F acc, float) { return acc; }
  SPH2D_HD static F resultA_g(F acc, float) { return acc; }
  template <class P>
  SPH2D_HD static F madd(F acc, F x, int row, int slot) {
#if SPH2D_Q_UNROLL
    const NumDen c = edge_coef<P>(row - 1, slot);
    const F k = F(c.num / c.den);
#else
    const F k = sizeof(F) == sizeof(double) ? F(edge_rows<P>().d[row][slot]) : F(edge_rows<P>().fhi[row][slot]);
#endif
    return k == F(0) ? acc : fma_f(x, k, acc);      // zero test is uniform across the warp
  }
  SPH2D_HD static F recip1(int, F iq) { return iq; }
  SPH2D_HD static F divq(F x, int, F iq) { return x * iq; }   // x / (q + 1), iq = 1/(q + 1)
  SPH2D_HD static F maddc(F acc, F x, double num, double den) {
    return num == 0.0 ? acc : fma_f(x, F(num / den), acc);
  }
  SPH2D_HD static F result(F acc) { return acc; }
  SPH2D_HD static F resultA(F acc) { return acc; }     // the sum as an accumulation-type value
  SPH2D_HD static F jm1(F t1, F t2, F r1, F r2, F d, F ra, F rb) {
    (void)ra; (void)rb;
    return asinh_diff(t1, t2, r1, r2, d);
  }
};
template <typename R> struct Acc;
template <> struct Acc<double> : AccPlain<double> {};
// FP32 (or an FP32-like scalar F): compensated accumulation
template <typename F>
struct AccFF {
  using T = FFT<F>;
  SPH2D_HD static FFT<F> c(double v) { return ffc<F>(v); }
  SPH2D_HD static FFT<F> c2(double num, double den) { return ffc<F>(num / den); }
  SPH2D_HD static FFT<F> from(F v) { return FFT<F>{v, F(0)}; }
  SPH2D_HD static FFT<F> sq(F v) { return ff_two_prod(v, v); }
  SPH2D_HD static FFT<F> root(FFT<F> v) { return ff_sqrt(v); }
  SPH2D_HD static F out(FFT<F> v) { return to_f(v); }
  SPH2D_HD static FFT<F> mulr(FFT<F> a, F b) { return a * b; }
  SPH2D_HD static FFT<F> jm1(F t1, F t2, F r1, F r2, F d, FFT<F> ra, FFT<F> rb) {
    (void)r1; (void)r2;
    return asinh_diff_ff(t1, t2, ra, rb, d);
  }
  using Sum = CSum<F>;
  // The edge sums run by grid extraction (xsum_madd) on inputs scaled per fan by an exact
  // power of two: 1 / the power of two above |Delta t| (and above |Delta J_-1| where a slot
  // takes that row), so that every term is below its slot's grid constant.
  static constexpr bool SCALED = true;
  template <class P>
  SPH2D_HD static Pow2<F> fan_scale(F dt, FFT<F> dJm) {
    F b = fabs(dt);
    if constexpr (uses_row_m1<P>()) b = fmax(b, fabs(dJm.hi) + fabs(dJm.lo));
    return pow2_scale(b);
  }
  SPH2D_HD static FFT<F> pscale(FFT<F> x, F s) { return FFT<F>{x.hi * s, x.lo * s}; }
  // Y_q = Delta(t rho^q) (q-1)!!/q!! + d^2 Y_{q-2} (edge_coef_y); both terms have the sign of
  // Delta t, so the sum is left unrenormalised
  SPH2D_HD static FFT<F> ystep(int q, FFT<F> dT, FFT<F> y2, FFT<F> d2a) {
    const FF k = ff_const(dfact(q - 1) / dfact(q));
    FFT<F> a = ff_two_prod(dT.hi, F(k.hi));
    a.lo = fma_f(dT.lo, F(k.hi), a.lo);
    if (k.lo != 0.0f) a.lo = fma_f(dT.hi, F(k.lo), a.lo);
    const FFT<F> b = y2 * d2a;
    const FFT<F> t = ff_two_sum(a.hi, b.hi);
    return FFT<F>{t.hi, t.lo + (a.lo + b.lo)};
  }
  SPH2D_HD static CSum<F> zero() { return CSum<F>{F(0), F(0)}; }
  SPH2D_HD static CSum<F> zero_g(float g) { return xsum_init<F>(g); }
  SPH2D_HD static F result_g(CSum<F> a, float g) { return (a.s - F(1.5f * g)) + a.c; }
  SPH2D_HD static FFT<F> resultA_g(CSum<F> a, float g) { return xsum_result(a, g); }
  template <class P>
  SPH2D_HD static CSum<F> madd(CSum<F> acc, FFT<F> x, int row, int slot) {
#if SPH2D_Q_UNROLL
    if constexpr (poly_den<P>() > 0) {
      const double k = edge_coef_s<P>(row - 1, slot);   // exact in FP32: no low word
      if (k == 0.0) return acc;
      return xsum_madd(acc, x, F(float(k)), F(0));
    } else {
      const NumDen c = edge_coef_y<P>(row - 1, slot);
      if (c.num == 0.0) return acc;
      const FF k = ff_const(c.num / c.den);
      return xsum_madd(acc, x, F(k.hi), F(k.lo));
    }
#else
    const EdgeRows<P>& r = edge_rows<P>();
    if constexpr (poly_den<P>() > 0) {
      if (r.fs[row][slot] == 0.0f) return acc;       // uniform across the warp
      return xsum_madd(acc, x, F(r.fs[row][slot]), F(0));
    } else {
      if (r.fhi[row][slot] == 0.0f) return acc;
      return xsum_madd(acc, x, F(r.fhi[row][slot]), F(r.flo[row][slot]));
    }
#endif
  }
  SPH2D_HD static CSum<F> maddc(CSum<F> acc, FFT<F> x, double num, double den) {
    if (num == 0.0) return acc;
    const FF k = ff_const(num / den);
    return csum_madd(acc, x, F(k.hi), F(k.lo));
  }
  // 1/(q+1) as a compensated pair: hi rounded, lo from the exact residual 1 - hi (q+1)
  SPH2D_HD static FFT<F> recip1(int q, F iq) {
    const F r = fma_f(-iq, F(float(q + 1)), F(1));
    return FFT<F>{iq, r * iq};
  }
  // x / (q + 1) for a small integer q + 1: quotient digit, its residual by fma, second digit
  SPH2D_HD static FFT<F> divq(FFT<F> x, int q, F iq) {
#if SPH2D_DIVQ
    const F q1 = x.hi * iq;
    const F r = fma_f(-q1, F(float(q + 1)), x.hi) + x.lo;
    return ff_fast_two_sum(q1, r * iq);
#else
    return x * recip1(q, iq);
#endif
  }
  SPH2D_HD static F result(CSum<F> a) { return a.s + a.c; }
  SPH2D_HD static FFT<F> resultA(CSum<F> a) { return ff_two_sum(a.s, a.c); }
};
template <> struct Acc<float> : AccFF<float> {};

// double-double accumulation (FP64 path of the highest-degree kernel, whose alternating
// coefficients would cost FP64 three to four digits)
template <typename D>
struct AccDD {
  using T = FFT<D>;
  SPH2D_HD static FFT<D> c(double v) { return FFT<D>{D(v), D(0)}; }
  SPH2D_HD static FFT<D> c2(double num, double den) {
    const FFT<double> v = dd_rational(num, den);
    return FFT<D>{D(v.hi), D(v.lo)};
  }
  SPH2D_HD static FFT<D> from(D v) { return FFT<D>{v, D(0)}; }
  SPH2D_HD static FFT<D> sq(D v) { return ff_two_prod(v, v); }
  SPH2D_HD static FFT<D> root(FFT<D> v) { return ff_sqrt(v); }
  SPH2D_HD static D out(FFT<D> v) { return to_f(v); }
  SPH2D_HD static FFT<D> mulr(FFT<D> a, D b) { return a * b; }
  SPH2D_HD static FFT<D> jm1(D t1, D t2, D r1, D r2, D d, FFT<D> ra, FFT<D> rb) {
    (void)r1; (void)r2;
    return asinh_diff_ff<D, double>(t1, t2, ra, rb, d);
  }
  using Sum = CSum<D>;
  static constexpr bool SCALED = false;
  SPH2D_HD static CSum<D> zero() { return CSum<D>{D(0), D(0)}; }
  SPH2D_HD static CSum<D> zero_g(float) { return zero(); }
  SPH2D_HD static D result_g(CSum<D> a, float) { return result(a); }
  SPH2D_HD static FFT<D> resultA_g(CSum<D> a, float) { return resultA(a); }
  template <class P>
  SPH2D_HD static CSum<D> madd(CSum<D> acc, FFT<D> x, int row, int slot) {
#if SPH2D_Q_UNROLL
    const NumDen c = edge_coef<P>(row - 1, slot);
    if (c.num == 0.0) return acc;
    const FFT<double> k = dd_rational(c.num, c.den);
    return csum_madd(acc, x, D(k.hi), D(k.lo));
#else
    const EdgeRows<P>& r = edge_rows<P>();
    if (r.d[row][slot] == 0.0) return acc;           // uniform across the warp
    return csum_madd(acc, x, D(r.d[row][slot]), D(r.dlo[row][slot]));
#endif
  }
  SPH2D_HD static CSum<D> maddc(CSum<D> acc, FFT<D> x, double num, double den) {
    if (num == 0.0) return acc;
    const FFT<double> k = dd_rational(num, den);
    return csum_madd(acc, x, D(k.hi), D(k.lo));
  }
  SPH2D_HD static FFT<D> recip1(int q, D iq) {
    const D r = fma_f(-iq, D(double(q + 1)), D(1));
    return FFT<D>{iq, r * iq};
  }
  SPH2D_HD static FFT<D> divq(FFT<D> x, int q, D iq) {
#if SPH2D_DIVQ
    const D q1 = x.hi * iq;
    const D r = fma_f(-q1, D(double(q + 1)), x.hi) + x.lo;
    return ff_fast_two_sum(q1, r * iq);
#else
    return x * recip1(q, iq);
#endif
  }
  SPH2D_HD static D result(CSum<D> a) { return a.s + a.c; }
  SPH2D_HD static FFT<D> resultA(CSum<D> a) { return ff_two_sum(a.s, a.c); }
};

// accumulation type per precision and kernel polynomial (PLAIN: the uncompensated form of
// the FP32 path)
template <typename R, class P, bool PLAIN = false> struct AccSel { using type = Acc<R>; };
template <> struct AccSel<double, PolyWC6, false> { using type = AccDD<double>; };
template <class P> struct AccSel<float, P, true> { using type = AccPlain<float>; };

// ---------------------------------------------------------------------------------------
// one edge (fan (0, A, B)) of a triangle for the polynomial kernel P; accumulates the
// signed fan integrals into o (global frame, raw)
// ---------------------------------------------------------------------------------------
// MD: moment degree computed, 0 (none), 1 (M00, M10, M01) or 3 (all ten); PLAIN: the FP32
// path's uncompensated form
template <typename R, class P, int MD, bool PLAIN = false>
SPH2D_HD void add_fan(R ax, R ay, R bx, R by, PairOut<R>& o) {
  const R ex = bx - ax, ey = by - ay;
  const R l2 = ex * ex + ey * ey;
  const R c = diff_of_products(ax, by, ay, bx);          // A x B = |A||B| sin(fan angle)
  if (l2 == R(0) || c == R(0)) return;                   // degenerate fan: zero area
  const R il = rsqrt_fast(l2);
  const R d = fabs(c) * il;                              // distance of the edge line
  if (d < Tiny<R>::v()) return;                          // contribution O(d log d)
  const R sg = c > R(0) ? R(1) : R(-1);
  const R nx = sg * ey * il, ny = -sg * ex * il;         // unit normal towards the line
  // tangent e2 = (-ny, nx); t = p . e2 (increasing with the polar angle)
  const R tA = ay * nx - ax * ny;
  const R tB = by * nx - bx * ny;
  const R dth = atan2_fast(c, ax * bx + ay * by);        // signed fan angle u_B - u_A
  const R ts = d < R(1) ? sqrt_fast((R(1) - d) * (R(1) + d)) : R(0);
  const R t1 = fmin(fmax(tA, -ts), ts);
  const R t2 = fmin(fmax(tB, -ts), ts);
  const R d2 = d * d;
  const R r1 = sqrt(d2 + t1 * t1), r2 = sqrt(d2 + t2 * t2);
  const R due = atan2_fast(d * (t2 - t1), d2 + t1 * t2); // edge-piece angle u_2 - u_1
  const R dus = dth - due;                               // sector pieces, total angle
  // (cos u, sin u) at u_A, u_1, u_2, u_B
  const R iA = rsqrt_fast(d2 + tA * tA), iB = rsqrt_fast(d2 + tB * tB);
  const R i1 = rsqrt_fast(d2 + t1 * t1), i2 = rsqrt_fast(d2 + t2 * t2);
  const R cA = d * iA, sA = tA * iA, cB = d * iB, sB = tB * iB;
  const R c1 = d * i1, s1 = t1 * i1, c2 = d * i2, s2 = t2 * i2;

  // ---- sector pieces: radius 1, angular antiderivatives over [u_A,u_1] and [u_2,u_B]
  // [F] := F(u_1) - F(u_A) + F(u_B) - F(u_2)
#define SPH2D_BR(F1, FA, F2, FB) (((F1) - (FA)) + ((FB) - (F2)))
  const R I_c = SPH2D_BR(s1, sA, s2, sB);                // int cos u
  const R I_s = SPH2D_BR(cA, c1, cB, c2);                // int sin u = [-cos u]
  // the FP32 path with exact rows runs the fan times D_P (undone in tri_poly)
  constexpr double DS = AccSel<R, P, PLAIN>::type::SCALED ? poly_scale<P>() : 1.0;
  constexpr double k2 = kappa<P>(2) * DS;
  constexpr double kg = kappa_grad<P>() * DS;
  R eg = R(k2) * dus;                                    // gamma (edge frame = any frame)
  R en = R(kg) * I_c;                                    // gradient along n
  R et = R(kg) * I_s;                                    // gradient along e2
  R E[10];                                               // edge-frame moments s^j t^l
  if (MD >= 1) {
    constexpr double k3 = kappa<P>(3) * DS;
    E[0] = eg;
    E[1] = R(k3) * I_c;                                  // s
    E[2] = R(k3) * I_s;                                  // t
  }
  if (MD >= 3) {
    constexpr double k4 = kappa<P>(4) * DS, k5 = kappa<P>(5) * DS;
    const R scA = sA * cA, sc1 = s1 * c1, sc2 = s2 * c2, scB = sB * cB;
    const R I_sc = SPH2D_BR(sc1, scA, sc2, scB);         // [s c]
    const R I_ss = SPH2D_BR(s1 * s1, sA * sA, s2 * s2, sB * sB);
    const R I_s3 = SPH2D_BR(s1 * s1 * s1, sA * sA * sA, s2 * s2 * s2, sB * sB * sB);
    const R I_c3 = SPH2D_BR(c1 * c1 * c1, cA * cA * cA, c2 * c2 * c2, cB * cB * cB);
    E[3] = R(k4) * R(0.5) * (dus + I_sc);                // s^2 : int cos^2
    E[4] = R(k4) * R(0.5) * I_ss;                        // s t : int sin cos = [sin^2/2]
    E[5] = R(k4) * R(0.5) * (dus - I_sc);                // t^2 : int sin^2
    E[6] = R(k5) * (I_c - I_s3 / R(3));                  // s^3 : int cos^3 = [s - s^3/3]
    E[7] = R(k5) * (-I_c3 / R(3));                       // s^2 t: int cos^2 sin = [-c^3/3]
    E[8] = R(k5) * (I_s3 / R(3));                        // s t^2: int cos sin^2 = [s^3/3]
    E[9] = R(k5) * (I_s + I_c3 / R(3));                  // t^3 : int sin^3 = [-c + c^3/3]
  }
#undef SPH2D_BR

  // ---- edge piece: t in [t1, t2], r = rho(t) <= 1.  Empty when both ends are clamped to the
  // same side (or d >= 1); it is then skipped, which keeps every power rho^q <= 1 and makes
  // its contribution exactly zero whatever the compiler contracts into FMAs.
  if (t1 != t2) {
    using AC = typename AccSel<R, P, PLAIN>::type;
    using A = typename AC::T;
    const A d2a = AC::sq(d);
    const A r1a = AC::root(d2a + AC::sq(t1)), r2a = AC::root(d2a + AC::sq(t2));
    // running sums without their d^(j+1) factors
    using SM = typename AC::Sum;
    constexpr float gG = slot_grid<P>(SL_G), gN = slot_grid<P>(SL_N), gT = slot_grid<P>(SL_T);
    constexpr float g10 = slot_grid<P>(SL_10), g01 = slot_grid<P>(SL_01), g20 = slot_grid<P>(SL_20);
    constexpr float g11 = slot_grid<P>(SL_11), g02 = slot_grid<P>(SL_02A), g30 = slot_grid<P>(SL_30);
    constexpr float g21 = slot_grid<P>(SL_21), g12 = slot_grid<P>(SL_12A), g03 = slot_grid<P>(SL_03A);
    SM Sg = AC::zero_g(gG), Sn = AC::zero_g(gN), St = AC::zero_g(gT);
    SM S10 = AC::zero_g(g10), S01 = AC::zero_g(g01), S20 = AC::zero_g(g20), S11 = AC::zero_g(g11);
    SM S02 = AC::zero_g(g02), S30 = AC::zero_g(g30), S21 = AC::zero_g(g21), S12 = AC::zero_g(g12);
    SM S03 = AC::zero_g(g03);
    const A zeroA = AC::c(0);
    // one step of the sums: q's row, Delta J_q and Delta rho^q
    auto step = [&](int row, const A& dJ, const A& dP) {
      Sg = AC::template madd<P>(Sg, dJ, row, SL_G);
      Sn = AC::template madd<P>(Sn, dJ, row, SL_N);
      St = AC::template madd<P>(St, dP, row, SL_T);
      if (MD >= 1) {
        S10 = AC::template madd<P>(S10, dJ, row, SL_10);
        S01 = AC::template madd<P>(S01, dP, row, SL_01);
      }
      if (MD >= 3) {
        S20 = AC::template madd<P>(S20, dJ, row, SL_20);
        S30 = AC::template madd<P>(S30, dJ, row, SL_30);
        S02 = AC::template madd<P>(S02, dJ, row, SL_02A);
        S12 = AC::template madd<P>(S12, dJ, row, SL_12A);
        S11 = AC::template madd<P>(S11, dP, row, SL_11);
        S21 = AC::template madd<P>(S21, dP, row, SL_21);
        S03 = AC::template madd<P>(S03, dP, row, SL_03A);
      }
    };
    A dJm = AC::jm1(t1, t2, r1, r2, d, r1a, r2a);            // Delta J_{-1}
    A dJp = AC::from(t2) - AC::from(t1);                    // Delta J_0
    A p1 = AC::c(1), p2 = AC::c(1);                         // rho^q at the two ends
    // the scaled form (FF sums): every J and rho^q below runs times the fan's power of two s,
    // undone exactly in the outputs (ds = d / s)
    R ds = d;
    if constexpr (AC::SCALED) {
      const auto sc = AC::template fan_scale<P>(t2 - t1, dJm);
      dJm = AC::pscale(dJm, sc.s);
      dJp = AC::pscale(dJp, sc.s);
      p1 = AC::from(sc.s);
      p2 = p1;
      ds = d * sc.is;
    }
    step(0, dJm, zeroA);                                    // q = -1
    step(1, dJp, zeroA);                                    // q = 0
    A dJq2 = dJm, dJq1 = dJp;                               // Delta J_{q-2}, Delta J_{q-1}
    // highest row any requested sum uses: gamma/gradient K, first moments K + 2, all K + 4
    constexpr int QMAX = MD >= 3 ? P::K + 4 : (MD >= 1 ? P::K + 2 : P::K);
    if constexpr (AC::SCALED) {
      // both ends' rho^q (times s) as packed pairs with negated low words: P_q = P_{q-1} R and
      // P_q t in float-pair arithmetic, one packed instruction per step for both ends
      using V = V2<R>;
      V phi{p1.hi, p2.hi}, pnl{R(0), R(0)};
      const V rhi{r1a.hi, r2a.hi}, nrhi{-r1a.hi, -r2a.hi}, nrlo{-r1a.lo, -r2a.lo};
      const V tt{t1, t2}, nt{-t1, -t2};
#if SPH2D_Q_UNROLL
#pragma unroll
#else
#pragma unroll 1
#endif
      for (int q = 1; q <= QMAX; ++q) {
        const V ph = v2_mul(phi, rhi);
        pnl = v2_fma(pnl, rhi, v2_fma(phi, nrlo, v2_fma(phi, nrhi, ph)));   // -(lo of P R)
        phi = ph;
        const V th = v2_mul(phi, tt);
        const V tnl = v2_fma(pnl, tt, v2_fma(phi, nt, th));                 // -(lo of P t)
        // differences end 2 - end 1, left unrenormalised (they feed only sums and ystep)
        const FFT<R> sp = ff_two_sum(phi.y, -phi.x), st = ff_two_sum(th.y, -th.x);
        const A dP{sp.hi, sp.lo + (pnl.x - pnl.y)};                        // Delta rho^q
        const A dT{st.hi, st.lo + (tnl.x - tnl.y)};                        // Delta (t rho^q)
        const A dJ = AC::ystep(q, dT, dJq2, d2a);                           // Delta Y_q
        step(q + 1, dJ, dP);
        dJq2 = dJq1;
        dJq1 = dJ;
      }
    } else {
#if SPH2D_Q_UNROLL
#pragma unroll
#else
#pragma unroll 1
#endif
      for (int q = 1; q <= QMAX; ++q) {
        p1 = p1 * r1a;
        p2 = p2 * r2a;
        const A dP = p2 - p1;                               // Delta rho^q
        const A dT = AC::mulr(p2, t2) - AC::mulr(p1, t1);   // Delta (t rho^q)
        const R qf = R(q), iq = R(1) / R(q + 1);
        const A dJ = AC::divq(dT + AC::mulr(dJq2 * d2a, qf), q, iq);   // Delta J_q
        step(q + 1, dJ, dP);
        dJq2 = dJq1;
        dJq1 = dJ;
      }
    }
    const R d2s = AC::SCALED ? d * ds : d2;                 // d^2 / s
    eg += ds * AC::result_g(Sg, gG);
    en += d2s * AC::result_g(Sn, gN);
    et += ds * AC::result_g(St, gT);
    if (MD >= 1) {
      E[1] += d2s * AC::result_g(S10, g10);
      E[2] += ds * AC::result_g(S01, g01);
    }
    if (MD >= 3) {
      const R d3s = d2s * d, d4s = d2s * d2;
      const A s20 = AC::resultA_g(S20, g20), s30 = AC::resultA_g(S30, g30), s21 = AC::resultA_g(S21, g21);
      E[3] += d3s * AC::out(s20);
      E[4] += d2s * AC::result_g(S11, g11);
      E[5] += ds * AC::out(AC::resultA_g(S02, g02) - s20 * d2a);
      E[6] += d4s * AC::out(s30);
      E[7] += d3s * AC::out(s21);
      E[8] += d2s * AC::out(AC::resultA_g(S12, g12) - s30 * d2a);
      E[9] += ds * AC::out(AC::resultA_g(S03, g03) - s21 * d2a);
    }
  }
  // rotate the gradient back from the edge frame (Sec. 2, Eq. improper)
  o.g += eg;
  o.gx += en * nx - et * ny;
  o.gy += en * ny + et * nx;
  if (MD >= 1) {
    // p_x = s nx - t ny, p_y = s ny + t nx: expand p_x^a p_y^b into s^j t^l
    o.m[0] += eg;
    o.m[1] += nx * E[1] - ny * E[2];
    o.m[2] += ny * E[1] + nx * E[2];
  }
  if (MD >= 3) {
    const R X = nx, Y = ny;
    const R XX = X * X, YY = Y * Y, XY = X * Y;
    o.m[3] += XX * E[3] - R(2) * XY * E[4] + YY * E[5];
    o.m[4] += XY * E[3] + (XX - YY) * E[4] - XY * E[5];
    o.m[5] += YY * E[3] + R(2) * XY * E[4] + XX * E[5];
    // cubic: (X s - Y t)^a (Y s + X t)^b
    o.m[6] += XX * X * E[6] - R(3) * XX * Y * E[7] + R(3) * X * YY * E[8] - YY * Y * E[9];
    o.m[7] += XX * Y * E[6] + (XX * X - R(2) * X * YY) * E[7] + (YY * Y - R(2) * XX * Y) * E[8]
            + X * YY * E[9];
    o.m[8] += X * YY * E[6] + (R(2) * XX * Y - YY * Y) * E[7] + (XX * X - R(2) * X * YY) * E[8]
            - XX * Y * E[9];
    o.m[9] += YY * Y * E[6] + R(3) * X * YY * E[7] + R(3) * XX * Y * E[8] + XX * X * E[9];
  }
}

// signed sum over the three fans of one local-frame triangle, single polynomial piece
template <typename R, class P, int MD, bool UNROLL_FANS, bool PLAIN = false>
SPH2D_HD void tri_poly(R ax, R ay, R bx, R by, R cx, R cy, PairOut<R>& o) {
  using AC = typename AccSel<R, P, PLAIN>::type;
  constexpr bool SC = AC::SCALED && poly_den<P>() > 1;   // fans computed times D_P
  PairOut<R> t;
  PairOut<R>& dst = SC ? t : o;
  if constexpr (SC) clear(t);
  R x0 = ax, y0 = ay, x1 = bx, y1 = by, x2 = cx, y2 = cy;
  if constexpr (UNROLL_FANS) {
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      add_fan<R, P, MD, PLAIN>(x0, y0, x1, y1, dst);
      const R tx = x0, ty = y0;
      x0 = x1;
      y0 = y1;
      x1 = x2;
      y1 = y2;
      x2 = tx;
      y2 = ty;
    }
  } else {
#pragma unroll 1
    for (int e = 0; e < 3; ++e) {
      add_fan<R, P, MD, PLAIN>(x0, y0, x1, y1, dst);
      const R tx = x0, ty = y0;
      x0 = x1;
      y0 = y1;
      x1 = x2;
      y1 = y2;
      x2 = tx;
      y2 = ty;
    }
  }
  if constexpr (SC) {
    constexpr double inv = 1.0 / poly_scale<P>();
    const R f = R(inv);
    o.g += f * t.g;
    o.gx += f * t.gx;
    o.gy += f * t.gy;
    constexpr int NM = MD >= 3 ? 10 : (MD >= 1 ? 3 : 0);
#pragma unroll
    for (int i = 0; i < NM; ++i) o.m[i] += f * t.m[i];
  }
}

// The three fans of a triangle run as a loop (one copy of the fan code) in every kernel and
// precision.  Measured on GB300 (the 1024^2 box with obstacle, FP32): against inlined fans the
// loop ran 20-23% faster for gamma and grad gamma alone and 6% faster for Wendland C2 with ten
// moments.  Wendland C4 with ten moments first ran 13% slower looped; once the edge sums took
// the grid extraction and the scaled recurrence, looping ran 3% faster for it in FP32 and 8% in
// FP64.
// raw integrals of kernel KID over the local-frame triangle, in input orientation
// (multiply by the orientation sign for the unsigned integral)
template <typename R, int KID, int MD, bool PLAIN = false>
SPH2D_HD void tri_raw(R ax, R ay, R bx, R by, R cx, R cy, PairOut<R>& o) {
  clear(o);
  if (KID == KID_WC2) tri_poly<R, PolyWC2, MD, false, PLAIN>(ax, ay, bx, by, cx, cy, o);
  else if (KID == KID_WC4) tri_poly<R, PolyWC4, MD, false, PLAIN>(ax, ay, bx, by, cx, cy, o);
  else if (KID == KID_WC6) tri_poly<R, PolyWC6, MD, false, PLAIN>(ax, ay, bx, by, cx, cy, o);
  else {
    // k(q) = 2 k1(q) - k1(2q), k1 = (1-q)^3_+.  With p' = 2p:
    //   int f(p) k1(2|p|) dA = 1/4 int f(p'/2) k1(|p'|) dA',  f = p^m -> 2^-m
    //   int k1'(2|p|) p/|p| dA = 1/4 int k1'(|p'|) p'/|p'| dA'   and k'(q) = 2k1'(q) - 2k1'(2q)
    // Both pieces run through one instance of the (1-q)^3 code.
#pragma unroll 1
    for (int piece = 0; piece < 2; ++piece) {
      const R sc = piece ? R(2) : R(1);
      PairOut<R> h;
      clear(h);
      tri_poly<R, PolyCube, MD, false, PLAIN>(sc * ax, sc * ay, sc * bx, sc * by, sc * cx, sc * cy, h);
      const R wg = piece ? R(-0.25) : R(2);     // 2^-(m+2), m = 0
      const R wd = piece ? R(-0.5) : R(2);      // gradient
      o.g += wg * h.g;
      o.gx += wd * h.gx;
      o.gy += wd * h.gy;
      if (MD >= 1) {
        const R w1 = piece ? R(-0.125) : R(2);
        o.m[0] += wg * h.m[0];
#pragma unroll
        for (int i = 1; i < 3; ++i) o.m[i] += w1 * h.m[i];
      }
      if (MD >= 3) {
        const R w2 = piece ? R(-0.0625) : R(2), w3 = piece ? R(-0.03125) : R(2);
#pragma unroll
        for (int i = 3; i < 6; ++i) o.m[i] += w2 * h.m[i];
#pragma unroll
        for (int i = 6; i < 10; ++i) o.m[i] += w3 * h.m[i];
      }
    }
  }
}

// orientation sign of a local-frame triangle (0 for zero area)
template <typename R>
SPH2D_HD int tri_orientation(R ax, R ay, R bx, R by, R cx, R cy) {
  const R a2 = diff_of_products(bx - ax, cy - ay, by - ay, cx - ax);
  return a2 > R(0) ? 1 : (a2 < R(0) ? -1 : 0);
}

// ---------------------------------------------------------------------------------------
// adjoint: derivative of the area integral with respect to the triangle's vertices.  Moving
// vertex j moves its two edges with the hat weight lambda_j, so (transport theorem)
//   d gamma / d nu_j = (C/H) sum_{e ni j} n_e int_e k(|p|) lambda_j ds      (local frame)
// with n_e the outward unit normal.  On an edge with tangent coordinate t (foot of the
// perpendicular at t = 0, distance d) |p| = rho(t) = sqrt(d^2 + t^2), so the two integrals
//   Jo = int k(rho) dt = sum_k b_k Delta J_k,   To = int k(rho) t dt = sum_k b_k Delta rho^{k+2}/(k+2)
// over t clipped to the support are the same square-root integrals as the forward edge piece.
// ---------------------------------------------------------------------------------------
// the grid constant of an extraction sum of n terms each at most m (see slot_grid)
SPH2D_HD constexpr float grid_for(int n, double m) {
  if (n == 0) return 1.0f;
  const double need = 2.0 * n * m * (1.0 + 1.0 / 128);
  double g = 1.0;
  while (g < need) g *= 2.0;
  while (g * 0.5 >= need) g *= 0.5;
  return float(g);
}
// the grid of a sum of c_q x_q, c_q = f * b_{q+sh} * (q + a)^e over q in [q0, q1] with |x_q| < 1
template <class P>
SPH2D_HD constexpr float poly_grid(int q0, int q1, int sh = 0, int a = 0, int e = 0) {
  double m = 0.0;
  int n = 0;
  for (int q = q0; q <= q1; ++q) {
    const int k = q + sh;
    double b = (k < 0 || k > P::K) ? 0.0 : P::b(k);
    for (int i = 0; i < e; ++i) b *= double(q + a);
    b = b < 0 ? -b : b;
    if (b == 0.0) continue;
    m = b > m ? b : m;
    ++n;
  }
  return grid_for(n, m);
}

// The FP32 path's form of edge_line_integrals, built as the forward edge piece: inputs scaled by
// the power of two s that brings |Delta t| into [1/2, 1), the recurrence on Y_q = J_q / w_q with
// both ends in packed instructions, and both sums by grid extraction.  The terms are bounded as
// in the forward sums: |b_q Delta J_q| <= |b_q| |Delta t| and |(b_{q-2} / q) Delta rho^q| <=
// |b_{q-2}| |Delta t| on an interval inside the support.
template <typename R, class P>
SPH2D_HD void edge_line_integrals_ff(R d, R t1, R t2, R& Jo, R& To) {
  using AC = typename AccSel<R, P>::type;
  using A = typename AC::T;
  using V = V2<R>;
  constexpr float g = poly_grid<P>(0, P::K);             // b_q and (b_{q-2} / q) q alike
  const A d2a = AC::sq(d);
  const A r1a = AC::root(d2a + AC::sq(t1)), r2a = AC::root(d2a + AC::sq(t2));
  const R r1 = sqrt(d * d + t1 * t1), r2 = sqrt(d * d + t2 * t2);
  const Pow2<R> sc = pow2_scale(t2 - t1);
  // Delta J_{-1} enters only as d^2 J_{-1}; at d = 0 that product vanishes
  const A dJm = AC::pscale(d > Tiny<R>::v() ? AC::jm1(t1, t2, r1, r2, d, r1a, r2a) : AC::c(0), sc.s);
  const A dJp = AC::pscale(AC::from(t2) - AC::from(t1), sc.s);
  CSum<R> sJ = xsum_init<R>(g), sT = xsum_init<R>(g);
  {
    const FF k = ff_const(P::b(0));
    sJ = xsum_madd(sJ, dJp, R(k.hi), R(k.lo));
  }
  V phi{sc.s, sc.s}, pnl{R(0), R(0)};
  const V rhi{r1a.hi, r2a.hi}, nrhi{-r1a.hi, -r2a.hi}, nrlo{-r1a.lo, -r2a.lo};
  const V tt{t1, t2}, nt{-t1, -t2};
  A y2 = dJm, y1 = dJp;                                   // Delta Y_{q-2}, Delta Y_{q-1}
#pragma unroll
  for (int q = 1; q <= P::K + 2; ++q) {
    const V ph = v2_mul(phi, rhi);
    pnl = v2_fma(pnl, rhi, v2_fma(phi, nrlo, v2_fma(phi, nrhi, ph)));
    phi = ph;
    if (q <= P::K) {
      const V th = v2_mul(phi, tt);
      const V tnl = v2_fma(pnl, tt, v2_fma(phi, nt, th));
      const FFT<R> st = ff_two_sum(th.y, -th.x);
      const A dT{st.hi, st.lo + (tnl.x - tnl.y)};
      const A y = AC::ystep(q, dT, y2, d2a);
      if (P::b(q) != 0.0) {
        const FF k = ff_const(P::b(q) * dfact(q) / dfact(q + 1));    // b_q w_q
        sJ = xsum_madd(sJ, y, R(k.hi), R(k.lo));
      }
      y2 = y1;
      y1 = y;
    }
    if (q >= 2 && P::b(q - 2) != 0.0) {
      const FFT<R> sp = ff_two_sum(phi.y, -phi.x);
      const A dP{sp.hi, sp.lo + (pnl.x - pnl.y)};
      const FF k = ff_const(P::b(q - 2) / double(q));
      sT = xsum_madd(sT, dP, R(k.hi), R(k.lo));
    }
  }
  Jo = ((sJ.s - R(1.5f * g)) + sJ.c) * sc.is;
  To = ((sT.s - R(1.5f * g)) + sT.c) * sc.is;
}

template <typename R, class P>
SPH2D_HD void edge_line_integrals(R d, R t1, R t2, R& Jo, R& To) {
  using AC = typename AccSel<R, P>::type;
  if constexpr (AC::SCALED) {
    edge_line_integrals_ff<R, P>(d, t1, t2, Jo, To);
    return;
  }
  using A = typename AC::T;
  using SM = typename AC::Sum;
  SM sJ = AC::zero(), sT = AC::zero();
  const A d2a = AC::sq(d);
  const A r1a = AC::root(d2a + AC::sq(t1)), r2a = AC::root(d2a + AC::sq(t2));
  // Delta J_{-1} enters only as d^2 J_{-1}; at d = 0 that product vanishes
  const R r1 = sqrt(d * d + t1 * t1), r2 = sqrt(d * d + t2 * t2);
  const A dJm = d > Tiny<R>::v() ? AC::jm1(t1, t2, r1, r2, d, r1a, r2a) : AC::c(0);
  const A dJp = AC::from(t2) - AC::from(t1);
  sJ = AC::maddc(sJ, dJp, P::b(0), 1.0);
  A p1 = AC::c(1), p2 = AC::c(1);
  A dJq2 = dJm, dJq1 = dJp;
#pragma unroll
  for (int q = 1; q <= P::K + 2; ++q) {
    p1 = p1 * r1a;
    p2 = p2 * r2a;
    const A dP = p2 - p1;
    if (q <= P::K) {
      const A dT = AC::mulr(p2, t2) - AC::mulr(p1, t1);
      const R qf = R(q), iq = R(1) / R(q + 1);
      const A dJ = AC::divq(dT + AC::mulr(dJq2 * d2a, qf), q, iq);
      sJ = AC::maddc(sJ, dJ, bk<P>(q), 1.0);
      dJq2 = dJq1;
      dJq1 = dJ;
    }
    if (q >= 2) sT = AC::maddc(sT, dP, bk<P>(q - 2), double(q));
  }
  Jo = AC::result(sJ);
  To = AC::result(sT);
}

// raw vertex gradients (without C/H) of one local-frame triangle for polynomial P
template <typename R, class P>
SPH2D_HD void tri_vertex_grad_poly(const R* v, R* g) {
  const R area2 = diff_of_products(v[2] - v[0], v[5] - v[1], v[3] - v[1], v[4] - v[0]);
  if (area2 == R(0)) return;
  const R sg = area2 > R(0) ? R(1) : R(-1);
#pragma unroll 1
  for (int e = 0; e < 3; ++e) {
    const int ia = e, ib = e == 2 ? 0 : e + 1;
    const R ax = v[2 * ia], ay = v[2 * ia + 1], bx = v[2 * ib], by = v[2 * ib + 1];
    const R ex = bx - ax, ey = by - ay;
    const R l2 = ex * ex + ey * ey;
    if (l2 == R(0)) continue;
    const R L = sqrt(l2), il = R(1) / L;
    const R ux = ex * il, uy = ey * il;                  // edge direction
    const R d = fabs(diff_of_products(ax, by, ay, bx)) * il;
    const R tA = ax * ux + ay * uy;                      // tB = tA + L
    const R tB = bx * ux + by * uy;
    if (!(d < R(1))) continue;                           // edge outside the support
    const R ts = sqrt((R(1) - d) * (R(1) + d));
    const R t1 = fmin(fmax(tA, -ts), ts), t2 = fmin(fmax(tB, -ts), ts);
    if (!(t2 > t1)) continue;
    R Jo, To;
    edge_line_integrals<R, P>(d, t1, t2, Jo, To);
    const R wb = (To - tA * Jo) * il;                    // int k lambda_b ds
    const R wa = Jo - wb;                                // int k lambda_a ds
    const R nx = sg * uy, ny = -sg * ux;                 // outward unit normal
    g[2 * ia] += wa * nx;
    g[2 * ia + 1] += wa * ny;
    g[2 * ib] += wb * nx;
    g[2 * ib + 1] += wb * ny;
  }
}

// ---------------------------------------------------------------------------------------
// second order: Jacobians of grad gamma.  grad gamma = -(C/H) oint k(|p|) n_out ds (divergence
// theorem, local frame).  Per edge e = (A, B) with outward normal n and unit tangent u, on the
// line p = f n + t u (f = A . n, rho^2 = f^2 + t^2, t from the foot of the perpendicular):
//   F_e = n L I,  I = int_0^1 k ds = Jo / L,  Jo = int k dt
//   dF_e/dB = sg R I + (n L) (x) U_s,   dF_e/dA = -sg R I + (n L) (x) (U_1 - U_s)
//   U_1 = int_0^1 k'(rho) p/rho ds     = (n f S0 + u Dk) / L
//   U_s = int_0^1 k'(rho) p/rho s ds   = (n f (Dk - tA S0) + u (S2 - f^2 S0 - tA Dk)) / L^2
// with S0 = int k'(rho)/rho dt, S2 = int k'(rho) rho dt (square-root integrals: sums of
// Delta J_q with the coefficients of k'(q)/q and k'(q) q), Dk = int k'(rho) t/rho dt
// = k(rho_2) - k(rho_1) = sum_m b_m Delta rho^m (from the recurrence's compensated powers: a
// direct difference of two kernel values cancels near the support edge), R the rotation
// (x, y) -> (y, -x), sg the orientation.  Then
// d grad gamma / d nu_j = -(C/H^2) sum_{e ni j} dF_e/dv_j and d grad gamma / d x_i = -sum_j
// of those (translation invariance); the last equals (C/H^2) oint k'(rho) n (x) p/rho ds.
// ---------------------------------------------------------------------------------------
// The FP32 path's form of edge_grad_integrals (scaled inputs, packed ends, Y recurrence, grid
// extraction).  Inputs scale by the power of two above |Delta t|, or above |Delta J_-1| too when
// k'(q)/q has a 1/q term (the q = -1 row of S0); bounds as in edge_line_integrals_ff, with
// |Delta rho^q| <= q |Delta t|.
template <typename R, class P>
SPH2D_HD void edge_grad_integrals_ff(R d, R t1, R t2, R& Jo, R& S0, R& S2, R& Dk) {
  using AC = typename AccSel<R, P>::type;
  using A = typename AC::T;
  using V = V2<R>;
  constexpr bool need_m1 = P::K >= 1 && P::b(1) != 0.0;
  constexpr float gJ = poly_grid<P>(0, P::K);
  constexpr float g0 = poly_grid<P>(-1, P::K, 2, 2, 1);   // (q + 2) b_{q+2}; q = -1 gives b_1
  constexpr float g2 = poly_grid<P>(1, P::K, 0, 0, 1);
  constexpr float gk = poly_grid<P>(1, P::K, 0, 0, 1);   // b_q Delta rho^q <= |b_q| q |Delta t|
  const A d2a = AC::sq(d);
  const A r1a = AC::root(d2a + AC::sq(t1)), r2a = AC::root(d2a + AC::sq(t2));
  const R r1 = sqrt(d * d + t1 * t1), r2 = sqrt(d * d + t2 * t2);
  const A dJm0 = (d > Tiny<R>::v() || (need_m1 && t1 * t2 > R(0))) ? AC::jm1(t1, t2, r1, r2, d, r1a, r2a) : AC::c(0);
  R bnd = fabs(t2 - t1);
  if constexpr (need_m1) bnd = fmax(bnd, fabs(dJm0.hi) + fabs(dJm0.lo));
  const Pow2<R> sc = pow2_scale(bnd);
  const A dJm = AC::pscale(dJm0, sc.s);
  const A dJp = AC::pscale(AC::from(t2) - AC::from(t1), sc.s);
  CSum<R> sJ = xsum_init<R>(gJ), s0 = xsum_init<R>(g0), s2 = xsum_init<R>(g2), sk = xsum_init<R>(gk);
  auto add = [](CSum<R>& acc, const A& x, double c) {
    if (c == 0.0) return;
    const FF k = ff_const(c);
    acc = xsum_madd(acc, x, R(k.hi), R(k.lo));
  };
  if (need_m1) add(s0, dJm, P::b(1));
  add(sJ, dJp, P::b(0));
  add(s0, dJp, 2.0 * bk<P>(2));
  V phi{sc.s, sc.s}, pnl{R(0), R(0)};
  const V rhi{r1a.hi, r2a.hi}, nrhi{-r1a.hi, -r2a.hi}, nrlo{-r1a.lo, -r2a.lo};
  const V tt{t1, t2}, nt{-t1, -t2};
  A y2 = dJm, y1 = dJp;
#pragma unroll
  for (int q = 1; q <= P::K; ++q) {
    const V ph = v2_mul(phi, rhi);
    pnl = v2_fma(pnl, rhi, v2_fma(phi, nrlo, v2_fma(phi, nrhi, ph)));
    phi = ph;
    const V th = v2_mul(phi, tt);
    const V tnl = v2_fma(pnl, tt, v2_fma(phi, nt, th));
    const FFT<R> st = ff_two_sum(th.y, -th.x), sp = ff_two_sum(phi.y, -phi.x);
    const A dT{st.hi, st.lo + (tnl.x - tnl.y)};
    const A dP{sp.hi, sp.lo + (pnl.x - pnl.y)};
    const A y = AC::ystep(q, dT, y2, d2a);               // Delta Y_q, Delta J_q = w_q Delta Y_q
    const double w = dfact(q) / dfact(q + 1);
    add(sJ, y, bk<P>(q) * w);
    add(s0, y, double(q + 2) * bk<P>(q + 2) * w);
    add(s2, y, double(q) * bk<P>(q) * w);
    add(sk, dP, bk<P>(q));
    y2 = y1;
    y1 = y;
  }
  Jo = ((sJ.s - R(1.5f * gJ)) + sJ.c) * sc.is;
  S0 = ((s0.s - R(1.5f * g0)) + s0.c) * sc.is;
  S2 = ((s2.s - R(1.5f * g2)) + s2.c) * sc.is;
  Dk = ((sk.s - R(1.5f * gk)) + sk.c) * sc.is;
}

template <typename R, class P>
SPH2D_HD void edge_grad_integrals(R d, R t1, R t2, R& Jo, R& S0, R& S2, R& Dk) {
  using AC = typename AccSel<R, P>::type;
  if constexpr (AC::SCALED) {
    if (!(t2 > t1)) {
      Jo = S0 = S2 = Dk = R(0);
      return;
    }
    edge_grad_integrals_ff<R, P>(d, t1, t2, Jo, S0, S2, Dk);
    return;
  }
  using A = typename AC::T;
  using SM = typename AC::Sum;
  SM sJ = AC::zero(), s0 = AC::zero(), s2 = AC::zero(), sk = AC::zero();
  if (!(t2 > t1)) {
    Jo = S0 = S2 = Dk = R(0);
    return;
  }
  const A d2a = AC::sq(d);
  const A r1a = AC::root(d2a + AC::sq(t1)), r2a = AC::root(d2a + AC::sq(t2));
  const R r1 = sqrt(d * d + t1 * t1), r2 = sqrt(d * d + t2 * t2);
  // Delta J_{-1} = asinh(t2/d) - asinh(t1/d): needed as such only when k'(q)/q has a 1/q term
  // (then the interval never reaches the particle), otherwise only as d^2 J_{-1}
  const bool need_m1 = bk<P>(1) != 0.0;
  const A dJm = (d > Tiny<R>::v() || (need_m1 && t1 * t2 > R(0))) ? AC::jm1(t1, t2, r1, r2, d, r1a, r2a) : AC::c(0);
  const A dJp = AC::from(t2) - AC::from(t1);
  // row q = -1 and q = 0
  if (need_m1) s0 = AC::maddc(s0, dJm, bk<P>(1), 1.0);
  sJ = AC::maddc(sJ, dJp, bk<P>(0), 1.0);
  s0 = AC::maddc(s0, dJp, 2.0 * bk<P>(2), 1.0);
  A p1 = AC::c(1), p2 = AC::c(1);
  A dJq2 = dJm, dJq1 = dJp;
#pragma unroll
  for (int q = 1; q <= P::K; ++q) {
    p1 = p1 * r1a;
    p2 = p2 * r2a;
    const A dT = AC::mulr(p2, t2) - AC::mulr(p1, t1);
    const R qf = R(q), iq = R(1) / R(q + 1);
    const A dJ = AC::divq(dT + AC::mulr(dJq2 * d2a, qf), q, iq);
    sJ = AC::maddc(sJ, dJ, bk<P>(q), 1.0);
    s0 = AC::maddc(s0, dJ, double(q + 2) * bk<P>(q + 2), 1.0);
    s2 = AC::maddc(s2, dJ, double(q) * bk<P>(q), 1.0);
    sk = AC::maddc(sk, p2 - p1, bk<P>(q), 1.0);
    dJq2 = dJq1;
    dJq1 = dJ;
  }
  Jo = AC::result(sJ);
  S0 = AC::result(s0);
  S2 = AC::result(s2);
  Dk = AC::result(sk);
}

// edge integrals Jo, S0, S2 of kernel KID over t in [t1, t2] (already clipped to the support)
template <typename R, int KID>
SPH2D_HD void edge_grad_integrals_k(R d, R t1, R t2, R& Jo, R& S0, R& S2, R& Dk) {
  if (KID == KID_WC2) edge_grad_integrals<R, PolyWC2>(d, t1, t2, Jo, S0, S2, Dk);
  else if (KID == KID_WC4) edge_grad_integrals<R, PolyWC4>(d, t1, t2, Jo, S0, S2, Dk);
  else if (KID == KID_WC6) edge_grad_integrals<R, PolyWC6>(d, t1, t2, Jo, S0, S2, Dk);
  else {
    // inner polynomial on |t| < th (rho < 1/2), outer polynomial on the rest
    const R th = d < R(0.5) ? sqrt((R(0.5) - d) * (R(0.5) + d)) : R(0);
    R j, s0, s2, dk;
    // inner [max(t1, -th), min(t2, th)], outer [t1, min(t2, -th)] and [max(t1, th), t2]
    // (empty intervals contribute 0; k is continuous at 1/2, so the Dk pieces telescope)
    edge_grad_integrals<R, PolyCubeIn>(d, fmax(t1, -th), fmin(t2, th), Jo, S0, S2, Dk);
    edge_grad_integrals<R, PolyCubeOut>(d, t1, fmin(t2, -th), j, s0, s2, dk);
    Jo += j;
    S0 += s0;
    S2 += s2;
    Dk += dk;
    edge_grad_integrals<R, PolyCubeOut>(d, fmax(t1, th), t2, j, s0, s2, dk);
    Jo += j;
    S0 += s0;
    S2 += s2;
    Dk += dk;
  }
}

// raw Jacobians (without -C/H^2): J[12], J[4 j + 2 b + a] = d F_b / d v_{j,a} summed over the
// two edges of vertex j (grad gamma = -(C/H) sum_e F_e, so d grad gamma / d nu = -(C/H^2) J)
template <typename R, int KID>
SPH2D_HD void tri_grad_jacobian(const R* v, R* J) {
#pragma unroll
  for (int i = 0; i < 12; ++i) J[i] = R(0);
  const R area2 = diff_of_products(v[2] - v[0], v[5] - v[1], v[3] - v[1], v[4] - v[0]);
  if (area2 == R(0)) return;
  const R sg = area2 > R(0) ? R(1) : R(-1);
#pragma unroll 1
  for (int e = 0; e < 3; ++e) {
    const int ia = e, ib = e == 2 ? 0 : e + 1;
    const R ax = v[2 * ia], ay = v[2 * ia + 1], bx = v[2 * ib], by = v[2 * ib + 1];
    const R ex = bx - ax, ey = by - ay;
    const R l2 = ex * ex + ey * ey;
    if (l2 == R(0)) continue;
    const R L = sqrt(l2), il = R(1) / L;
    const R ux = ex * il, uy = ey * il;                  // unit tangent
    const R nx = sg * uy, ny = -sg * ux;                 // outward unit normal
    const R f = ax * nx + ay * ny;                       // signed line distance along n
    const R d = fabs(f);
    const R tA = ax * ux + ay * uy, tB = bx * ux + by * uy;
    if (!(d < R(1))) continue;                           // edge line outside the support
    const R ts = sqrt((R(1) - d) * (R(1) + d));
    const R t1 = fmin(fmax(tA, -ts), ts), t2 = fmin(fmax(tB, -ts), ts);
    if (!(t2 > t1)) continue;
    R Jo, S0, S2, Dk;
    edge_grad_integrals_k<R, KID>(d, t1, t2, Jo, S0, S2, Dk);
    const R I = Jo * il;
    // U_1 and U_s in (n, u) components, then to x, y
    const R u1n = f * S0 * il, u1t = Dk * il;
    const R usn = f * (Dk - tA * S0) * il * il, ust = (S2 - f * f * S0 - tA * Dk) * il * il;
    const R U1x = u1n * nx + u1t * ux, U1y = u1n * ny + u1t * uy;
    const R Usx = usn * nx + ust * ux, Usy = usn * ny + ust * uy;
    const R nLx = nx * L, nLy = ny * L;
    // sg R I: R = [[0, 1], [-1, 0]]
    const R rI01 = sg * I, rI10 = -sg * I;
    // vertex B: sg R I + nL (x) U_s
    J[4 * ib + 0] += nLx * Usx;
    J[4 * ib + 1] += rI01 + nLx * Usy;
    J[4 * ib + 2] += rI10 + nLy * Usx;
    J[4 * ib + 3] += nLy * Usy;
    // vertex A: -sg R I + nL (x) (U_1 - U_s)
    J[4 * ia + 0] += nLx * (U1x - Usx);
    J[4 * ia + 1] += -rI01 + nLx * (U1y - Usy);
    J[4 * ia + 2] += -rI10 + nLy * (U1x - Usx);
    J[4 * ia + 3] += nLy * (U1y - Usy);
  }
}

// d gamma / d (x0, y0, x1, y1, x2, y2) in local units (multiply by C/H for world units)
template <typename R, int KID>
SPH2D_HD void tri_vertex_grad(const R* v, R* g) {
#pragma unroll
  for (int i = 0; i < 6; ++i) g[i] = R(0);
  if (KID == KID_WC2) tri_vertex_grad_poly<R, PolyWC2>(v, g);
  else if (KID == KID_WC4) tri_vertex_grad_poly<R, PolyWC4>(v, g);
  else if (KID == KID_WC6) tri_vertex_grad_poly<R, PolyWC6>(v, g);
  else {
    // k = 2 k1(q) - k1(2q): edge integrals of k1(2 rho) in the doubled frame, ds' = 2 ds
    R h[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
    tri_vertex_grad_poly<R, PolyCube>(v, g);
    R w[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) w[i] = R(2) * v[i];
    tri_vertex_grad_poly<R, PolyCube>(w, h);
#pragma unroll
    for (int i = 0; i < 6; ++i) g[i] = R(2) * g[i] - R(0.5) * h[i];
  }
}

}  // namespace sph2d
