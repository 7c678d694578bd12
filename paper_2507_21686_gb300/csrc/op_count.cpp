// Algorithmic operation count of the pair formula.  The closed-form pair integrals of
// pair_math.cuh are instantiated with a scalar type that counts every floating-point
// operation it performs, so the count is of exactly the formula the CUDA kernels execute.
// Three instantiations:
//   fp64    the FP64 path as it runs (double; double-double sums for Wendland C6)
//   fp32    the compensated FP32 form (float with compensated FF radial sums)
//   method  the closed form in plain arithmetic for every kernel: no compensation terms, the
//           method's own work (the roofline's algorithmic FLOPs per pair)
// Host code only.
//
// Counting convention: add/sub, mul, div, sqrt and each transcendental call (atan2, log)
// count 1 flop, fma counts 2; comparisons, min/max, abs and selects count 0 flops (reported
// separately as "other").
#include <cmath>
#include <cstdint>

namespace sph2d {
struct OpTally {
  int64_t add = 0, mul = 0, fma = 0, div = 0, sqrt = 0, transc = 0, other = 0;
};
static OpTally g_tally;

template <typename T>
struct Counted {
  T v;
  Counted() : v(0) {}
  Counted(double x) : v(T(x)) {}
  Counted(float x) : v(T(x)) {}
  Counted(int x) : v(T(x)) {}
  Counted(long double x) : v(T(x)) {}
  explicit operator bool() const { return v != 0; }
};
template <typename T> inline Counted<T> mk(T x) { Counted<T> r; r.v = x; return r; }
#define SPH2D_CBIN(op, field)                                                             \
  template <typename T> inline Counted<T> operator op(Counted<T> a, Counted<T> b) {         \
    ++g_tally.field;                                                                      \
    return mk<T>(a.v op b.v);                                                             \
  }
SPH2D_CBIN(+, add)
SPH2D_CBIN(-, add)
SPH2D_CBIN(*, mul)
SPH2D_CBIN(/, div)
#undef SPH2D_CBIN
template <typename T> inline Counted<T> operator-(Counted<T> a) { return mk<T>(-a.v); }
template <typename T> inline Counted<T>& operator+=(Counted<T>& a, Counted<T> b) { a = a + b; return a; }
#define SPH2D_CCMP(op)                                                                    \
  template <typename T> inline bool operator op(Counted<T> a, Counted<T> b) {               \
    ++g_tally.other;                                                                      \
    return a.v op b.v;                                                                    \
  }
SPH2D_CCMP(<)
SPH2D_CCMP(>)
SPH2D_CCMP(<=)
SPH2D_CCMP(>=)
SPH2D_CCMP(==)
SPH2D_CCMP(!=)
#undef SPH2D_CCMP
template <typename T> inline Counted<T> sqrt(Counted<T> a) { ++g_tally.sqrt; return mk<T>(std::sqrt(a.v)); }
template <typename T> inline Counted<T> log(Counted<T> a) { ++g_tally.transc; return mk<T>(std::log(a.v)); }
template <typename T> inline Counted<T> atan2(Counted<T> a, Counted<T> b) {
  ++g_tally.transc;
  return mk<T>(std::atan2(a.v, b.v));
}
template <typename T> inline Counted<T> fabs(Counted<T> a) { ++g_tally.other; return mk<T>(std::fabs(a.v)); }
template <typename T> inline Counted<T> fmin(Counted<T> a, Counted<T> b) { ++g_tally.other; return mk<T>(std::fmin(a.v, b.v)); }
template <typename T> inline Counted<T> fmax(Counted<T> a, Counted<T> b) { ++g_tally.other; return mk<T>(std::fmax(a.v, b.v)); }
inline Counted<float> fma_f(Counted<float> a, Counted<float> b, Counted<float> c) {
  ++g_tally.fma;
  return mk<float>(std::fma(a.v, b.v, c.v));
}
inline Counted<double> fma_f(Counted<double> a, Counted<double> b, Counted<double> c) {
  ++g_tally.fma;
  return mk<double>(std::fma(a.v, b.v, c.v));
}
inline Counted<long double> fma_f(Counted<long double> a, Counted<long double> b, Counted<long double> c) {
  ++g_tally.fma;
  return mk<long double>(std::fma(a.v, b.v, c.v));
}
template <typename T> inline T raw_f(Counted<T> x) { return x.v; }
inline Counted<double> frexp_f(Counted<double> x, int* e) { return mk<double>(std::frexp(x.v, e)); }
inline Counted<double> ldexp_f(Counted<double> x, int e) { return mk<double>(std::ldexp(x.v, e)); }
inline Counted<float> frexp_f(Counted<float> x, int* e) { return mk<float>(std::frexp(x.v, e)); }
inline Counted<float> ldexp_f(Counted<float> x, int e) { return mk<float>(std::ldexp(x.v, e)); }
template <typename F> struct Pow2;
// the exact power-of-two scale of the FF edge sums (exponent-field work: not counted)
inline Pow2<Counted<float>> pow2_scale(Counted<float> x);
// the FP32 path's polynomial atan2, counted operation by operation as the kernels run it
inline Counted<float> atan2_fast(Counted<float> y, Counted<float> x) {
  const Counted<float> ax = fabs(x), ay = fabs(y);
  const Counted<float> t = fmin(ax, ay) / fmax(ax, ay), w = t * t;
  static const float c[10] = {-1.753866789e-03f, 1.072655618e-02f, -3.080365062e-02f, 5.755088106e-02f,
                              -8.377224952e-02f, 1.094199046e-01f, -1.426192224e-01f, 1.999826431e-01f,
                              -3.333328366e-01f, 1.0f};
  Counted<float> p = Counted<float>(c[0]);
  for (int k = 1; k < 10; ++k) p = fma_f(p, w, Counted<float>(c[k]));
  Counted<float> a = t * p;
  if (ay > ax) a = Counted<float>(1.57079637f) - a;
  if (x < Counted<float>(0.0f)) a = Counted<float>(3.14159274f) - a;
  return y < Counted<float>(0.0f) ? -a : a;
}
}  // namespace sph2d

#include "pair_math.cuh"

namespace sph2d {
// FP32 semantics of diff_of_products and the tiny-distance cut for the counted types
inline Counted<float> diff_of_products(Counted<float> a, Counted<float> b, Counted<float> c, Counted<float> d) {
  const Counted<float> w = c * d;
  const Counted<float> e = fma_f(-c, d, w);
  const Counted<float> f = fma_f(a, b, -w);
  return f + e;
}
inline Counted<double> diff_of_products(Counted<double> a, Counted<double> b, Counted<double> c, Counted<double> d) {
  return a * b - c * d;
}
inline Counted<long double> diff_of_products(Counted<long double> a, Counted<long double> b, Counted<long double> c,
                                             Counted<long double> d) {
  return a * b - c * d;
}
template <> struct Tiny<Counted<long double>> { static Counted<long double> v() { return Counted<long double>(1e-150); } };
template <> struct Tiny<Counted<double>> { static Counted<double> v() { return Counted<double>(1e-150); } };
template <> struct Tiny<Counted<float>> { static Counted<float> v() { return Counted<float>(1e-18f); } };
template <> struct Acc<Counted<double>> {
  using R = Counted<double>;
  using T = R;
  static R c(double v) { return R(v); }
  static R c2(double num, double den) { return R(num / den); }
  static R from(R v) { return v; }
  static R sq(R v) { return v * v; }
  static R root(R v) { return sqrt(v); }
  static R out(R v) { return v; }
  static R mulr(R a, R b) { return a * b; }
  static R jm1(R t1, R t2, R r1, R r2, R d, R, R) { return asinh_diff(t1, t2, r1, r2, d); }
  using Sum = R;
  static constexpr bool SCALED = false;
  static R zero() { return R(0.0); }
  static R zero_g(float) { return R(0.0); }
  static R result_g(R a, float) { return a; }
  static R resultA_g(R a, float) { return a; }
  template <class P>
  static R madd(R acc, R x, int row, int slot) {
    const NumDen c = edge_coef<P>(row - 1, slot);
    const double k = c.num / c.den;
    if (k == 0.0) return acc;
    return fma_f(x, R(k), acc);
  }
  static R result(R a) { return a; }
  static R resultA(R a) { return a; }
  static R recip1(int, R iq) { return iq; }
  static R divq(R x, int, R iq) { return x * iq; }
};
// the method count: the plain closed form (uncompensated sums) for every kernel
template <> struct Acc<Counted<long double>> {
  using R = Counted<long double>;
  using T = R;
  static R c(double v) { return R(v); }
  static R c2(double num, double den) { return R(num / den); }
  static R from(R v) { return v; }
  static R sq(R v) { return v * v; }
  static R root(R v) { return sqrt(v); }
  static R out(R v) { return v; }
  static R mulr(R a, R b) { return a * b; }
  static R jm1(R t1, R t2, R r1, R r2, R d, R, R) { return asinh_diff(t1, t2, r1, r2, d); }
  using Sum = R;
  static constexpr bool SCALED = false;
  static R zero() { return R(0.0); }
  static R zero_g(float) { return R(0.0); }
  static R result_g(R a, float) { return a; }
  static R resultA_g(R a, float) { return a; }
  template <class P>
  static R madd(R acc, R x, int row, int slot) {
    const NumDen c = edge_coef<P>(row - 1, slot);
    const double k = c.num / c.den;
    if (k == 0.0) return acc;
    return fma_f(x, R(k), acc);
  }
  static R result(R a) { return a; }
  static R resultA(R a) { return a; }
  static R recip1(int, R iq) { return iq; }
  static R divq(R x, int, R iq) { return x * iq; }
};
inline Pow2<Counted<float>> pow2_scale(Counted<float> x) {
  const Pow2<float> p = pow2_scale(x.v);
  return Pow2<Counted<float>>{mk<float>(p.s), mk<float>(p.is)};
}
template <> struct Acc<Counted<float>> : AccFF<Counted<float>> {};
template <> struct AccSel<Counted<double>, PolyWC6> { using type = AccDD<Counted<double>>; };

// distance from the particle to the local triangle below 1/2: the cubic spline's second piece
// (support H/2) is non-zero only then (plain double; the decision is not counted as work)
static bool within_half(const double* l) {
  bool pos = false, neg = false, near = false;
  for (int e = 0; e < 3; ++e) {
    const int b = e == 2 ? 0 : e + 1;
    const double ax = l[2 * e], ay = l[2 * e + 1], bx = l[2 * b], by = l[2 * b + 1];
    const double ex = bx - ax, ey = by - ay, cr = ax * ey - ay * ex;
    pos = pos || cr > 0;
    neg = neg || cr < 0;
    const double l2 = ex * ex + ey * ey, tn = -(ax * ex + ay * ey);
    const double d2 = tn <= 0 ? ax * ax + ay * ay : (tn >= l2 ? bx * bx + by * by : cr * cr / l2);
    near = near || d2 < 0.25;
  }
  return near || (pos != neg);
}

template <typename R, int KID, int MD>
static void count_one(const double* l) {
  R v[6];
  for (int j = 0; j < 6; ++j) v[j] = R(l[j]);
  PairOut<R> o;
  (void)tri_orientation<R>(v[0], v[1], v[2], v[3], v[4], v[5]);
  if (KID == KID_CUBIC) {
    // first piece always, second piece only where it is non-zero, as the kernels evaluate it
    clear(o);
    tri_poly<R, PolyCube, MD, true>(v[0], v[1], v[2], v[3], v[4], v[5], o);
    if (within_half(l)) {
      PairOut<R> h;
      clear(h);
      const R sc(2.0);
      tri_poly<R, PolyCube, MD, true>(sc * v[0], sc * v[1], sc * v[2], sc * v[3], sc * v[4], sc * v[5], h);
      o.g = o.g + h.g;
      o.gx = o.gx + h.gx;
      o.gy = o.gy + h.gy;
      for (int m = 0; m < (MD >= 3 ? 10 : (MD >= 1 ? 3 : 0)); ++m) o.m[m] = o.m[m] + h.m[m];
    }
  } else {
    tri_raw<R, KID, MD>(v[0], v[1], v[2], v[3], v[4], v[5], o);
  }
  // constants and orientation applied per output, as in the kernels
  const R k(1.0);
  R s = k * o.g;
  s = k * o.gx;
  s = k * o.gy;
  for (int m = 0; m < (MD >= 3 ? 10 : (MD >= 1 ? 3 : 0)); ++m) s = k * o.m[m];
  (void)s;
}

template <typename R, int KID>
static void count_md(int md, const double* l) {
  if (md == 3) count_one<R, KID, 3>(l);
  else if (md == 1) count_one<R, KID, 1>(l);
  else count_one<R, KID, 0>(l);
}

template <typename R>
static void count_kernel(int kid, int md, const double* l) {
  switch (kid) {
    case 0: count_md<R, 0>(md, l); break;
    case 1: count_md<R, 1>(md, l); break;
    case 2: count_md<R, 2>(md, l); break;
    default: count_md<R, 3>(md, l); break;
  }
}
}  // namespace sph2d

extern "C" {
// Count the operations of one pair (local-frame triangle l[6], H = 1) with moments up to
// `moment_degree` (-1..3; 2 and 3 compute all ten, 1 the first three, as the kernels do).
// kind: 0 the FP64 path, 1 the compensated FP32 form, 2 the method (plain closed form).
// out[7] = add, mul, fma, div, sqrt, transcendental, other.  Returns flops (fma = 2).
int64_t sph2d_count_pair_ops(int kernel, int moment_degree, int kind, const double* l, int64_t* out) {
  sph2d::g_tally = sph2d::OpTally{};
  const int md = moment_degree >= 2 ? 3 : (moment_degree == 1 ? 1 : 0);
  if (kind == 1) sph2d::count_kernel<sph2d::Counted<float>>(kernel, md, l);
  else if (kind == 2) sph2d::count_kernel<sph2d::Counted<long double>>(kernel, md, l);
  else sph2d::count_kernel<sph2d::Counted<double>>(kernel, md, l);
  const sph2d::OpTally& t = sph2d::g_tally;
  if (out) {
    out[0] = t.add; out[1] = t.mul; out[2] = t.fma; out[3] = t.div;
    out[4] = t.sqrt; out[5] = t.transc; out[6] = t.other;
  }
  return t.add + t.mul + 2 * t.fma + t.div + t.sqrt + t.transc;
}
}
