// Lagrange boundary fields of order 1-3 (Sec. 3 interpolates a field linearly over each
// triangle; the paper's introduction names higher-order element fields as the extension).
//
// Node values of a triangle follow the principal lattice {(i, j, l)/k : i + j + l = k} in
// barycentric coordinates: vertices 0, 1, 2; then each edge (0,1), (1,2), (2,0) from its first
// vertex to its second; then the interior node (order 3: the centroid).  The interpolant is
// rewritten as a homogeneous polynomial of degree k in (lambda_0, lambda_1, lambda_2)
// (lambda_0 + lambda_1 + lambda_2 = 1) and expanded in the monomials xi^a eta^b of the local
// frame p = (x' - x_i)/H, so that per pair, with c_ab those coefficients,
//
//   <A>      = sum_ab c_ab M_ab                              (the moments, a + b <= 3)
//   <grad A> = (1/H) sum_ab (grad c)_ab M_ab - (C/H) sum_e n_e int_e A(p(t)) k(rho(t)) dt
//
// (integration by parts: int A grad_x W = int W grad A - oint A W n ds, n the outward normal).
// On an edge with unit tangent u, signed line distance f = a . n and t measured from the foot
// of the perpendicular, p(t) = f n + t u and rho^2 = f^2 + t^2; A(p(t)) is a cubic in t, and
// I_m = int k(rho) t^m dt (m = 0..3) are square-root integrals of the same recurrence as the
// forward edge piece:
//   I_0 = sum_q b_q dJ_q,  I_1 = sum_q b_q d rho^{q+2}/(q+2),
//   I_2 = sum_q b_q dJ_{q+2} - f^2 I_0,  I_3 = sum_q b_q d rho^{q+4}/(q+4) - f^2 I_1.
#pragma once

#include "pair_math.cuh"

namespace sph2d {

constexpr int nodes_of(int order) { return (order + 1) * (order + 2) / 2; }

// ---------------------------------------------------------------------------------------
// edge integrals I_m = int_{t1}^{t2} k(sqrt(d^2 + t^2)) t^m dt, m = 0..3 (t1, t2 already
// clipped to the support)
// ---------------------------------------------------------------------------------------
template <typename R, class P>
SPH2D_HD void edge_poly_integrals(R d, R t1, R t2, R* I) {
  using AC = typename AccSel<R, P>::type;
  using A = typename AC::T;
  using SM = typename AC::Sum;
  I[0] = I[1] = I[2] = I[3] = R(0);
  if (!(t2 > t1)) return;
  SM s0 = AC::zero(), s1 = AC::zero(), s2 = AC::zero(), s3 = AC::zero();
  const A d2a = AC::sq(d);
  const A r1a = AC::root(d2a + AC::sq(t1)), r2a = AC::root(d2a + AC::sq(t2));
  const R r1 = sqrt(d * d + t1 * t1), r2 = sqrt(d * d + t2 * t2);
  // Delta J_{-1} = asinh(t2/d) - asinh(t1/d) enters as d^2 J_{-1} (and through J_1 where the
  // polynomial has a linear term); at d = 0 the product vanishes
  const A dJm = d > Tiny<R>::v() ? AC::jm1(t1, t2, r1, r2, d, r1a, r2a) : AC::c(0);
  const A dJp = AC::from(t2) - AC::from(t1);
  s0 = AC::maddc(s0, dJp, bk<P>(0), 1.0);
  A p1 = AC::c(1), p2 = AC::c(1);
  A dJq2 = dJm, dJq1 = dJp;
#pragma unroll
  for (int q = 1; q <= P::K + 4; ++q) {
    p1 = p1 * r1a;                                       // rho^q at both ends
    p2 = p2 * r2a;
    if (q <= P::K + 2) {
      // (q + 1) J_q = t rho^q + q d^2 J_{q-2}
      const A dT = AC::mulr(p2, t2) - AC::mulr(p1, t1);
      const R qf = R(q), iq = R(1) / R(q + 1);
      const A dJ = AC::divq(dT + AC::mulr(dJq2 * d2a, qf), q, iq);
      if (q <= P::K) s0 = AC::maddc(s0, dJ, bk<P>(q), 1.0);
      if (q >= 2) s2 = AC::maddc(s2, dJ, bk<P>(q - 2), 1.0);
      dJq2 = dJq1;
      dJq1 = dJ;
    }
    const A dP = p2 - p1;
    if (q >= 2 && q - 2 <= P::K) s1 = AC::maddc(s1, dP, bk<P>(q - 2), double(q));
    if (q >= 4) s3 = AC::maddc(s3, dP, bk<P>(q - 4), double(q));
  }
  const R dd = d * d;
  I[0] = AC::result(s0);
  I[1] = AC::result(s1);
  I[2] = AC::result(s2) - dd * I[0];
  I[3] = AC::result(s3) - dd * I[1];
}

// the same for kernel KID (the cubic spline as its inner polynomial on rho < 1/2 and its outer
// one beyond, on split t-intervals)
template <typename R, int KID>
SPH2D_HD void edge_poly_integrals_k(R d, R t1, R t2, R* I) {
  if (KID == KID_WC2) edge_poly_integrals<R, PolyWC2>(d, t1, t2, I);
  else if (KID == KID_WC4) edge_poly_integrals<R, PolyWC4>(d, t1, t2, I);
  else if (KID == KID_WC6) edge_poly_integrals<R, PolyWC6>(d, t1, t2, I);
  else {
    const R th = d < R(0.5) ? sqrt((R(0.5) - d) * (R(0.5) + d)) : R(0);
    R J[4];
    edge_poly_integrals<R, PolyCubeIn>(d, fmax(t1, -th), fmin(t2, th), I);
    edge_poly_integrals<R, PolyCubeOut>(d, t1, fmin(t2, -th), J);
#pragma unroll
    for (int m = 0; m < 4; ++m) I[m] += J[m];
    edge_poly_integrals<R, PolyCubeOut>(d, fmax(t1, th), t2, J);
#pragma unroll
    for (int m = 0; m < 4; ++m) I[m] += J[m];
  }
}

// ---------------------------------------------------------------------------------------
// node values -> coefficients of the homogeneous barycentric form.  Monomials:
//   order 1: l0, l1, l2
//   order 2: l0^2, l1^2, l2^2, l0 l1, l1 l2, l2 l0
//   order 3: l0^3, l1^3, l2^3, l0^2 l1, l0 l1^2, l1^2 l2, l1 l2^2, l2^2 l0, l2 l0^2, l0 l1 l2
// Order 2: the vertex values, and 4 A_jk - A_j - A_k for the edge midpoint A_jk.  Order 3: on
// edge (j, k) with node values A_1 at (2/3, 1/3) and A_2 at (1/3, 2/3),
//   4 B_jjk + 2 B_jkk = 27 A_1 - 8 A_j - A_k =: R_1,  2 B_jjk + 4 B_jkk = 27 A_2 - A_j - 8 A_k =: R_2,
// so B_jjk = (2 R_1 - R_2)/6, B_jkk = (2 R_2 - R_1)/6; the centroid value fixes B_012 =
// 27 A_c - (sum of the other nine).  A: node values with stride `stride`.
// ---------------------------------------------------------------------------------------
template <typename R, int ORDER>
SPH2D_HD void lagrange_to_bary(const float* A, int stride, R* B) {
  const R a0 = R(A[0]), a1 = R(A[stride]), a2 = R(A[2 * stride]);
  B[0] = a0;
  B[1] = a1;
  B[2] = a2;
  if (ORDER == 2) {
    B[3] = R(4) * R(A[3 * stride]) - a0 - a1;
    B[4] = R(4) * R(A[4 * stride]) - a1 - a2;
    B[5] = R(4) * R(A[5 * stride]) - a2 - a0;
  } else if (ORDER == 3) {
    const R sixth = R(1) / R(6);
    const int ej[3] = {0, 1, 2};
    const R av[3] = {a0, a1, a2};
    R other = a0 + a1 + a2;
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      const int j = ej[e], k = e == 2 ? 0 : e + 1;
      const R n1 = R(A[(3 + 2 * e) * stride]), n2 = R(A[(4 + 2 * e) * stride]);
      const R r1 = R(27) * n1 - R(8) * av[j] - av[k];
      const R r2 = R(27) * n2 - av[j] - R(8) * av[k];
      B[3 + 2 * e] = (R(2) * r1 - r2) * sixth;       // l_j^2 l_k
      B[4 + 2 * e] = (R(2) * r2 - r1) * sixth;       // l_j l_k^2
      other += B[3 + 2 * e] + B[4 + 2 * e];
    }
    B[9] = R(27) * R(A[9 * stride]) - other;
  }
}

// ---------------------------------------------------------------------------------------
// the barycentric monomials above as polynomials in the local frame, coefficients in the
// moment order 1, xi, eta, xi^2, xi eta, eta^2, xi^3, xi^2 eta, xi eta^2, eta^3.
// lambda_j = (a x b + xi (a_y - b_y) + eta (b_x - a_x)) / D with (a, b) = (v_{j+1}, v_{j+2})
// and D = (v1 - v0) x (v2 - v0) (twice the signed area).  Returns false for zero area.
// ---------------------------------------------------------------------------------------
template <typename R>
SPH2D_HD void mul_aff(const R* a, const R* b, R* q) {
  q[0] = a[0] * b[0];
  q[1] = a[0] * b[1] + a[1] * b[0];
  q[2] = a[0] * b[2] + a[2] * b[0];
  q[3] = a[1] * b[1];
  q[4] = a[1] * b[2] + a[2] * b[1];
  q[5] = a[2] * b[2];
}
template <typename R>
SPH2D_HD void mul_quad_aff(const R* q, const R* a, R* c) {
  c[0] = q[0] * a[0];
  c[1] = q[0] * a[1] + q[1] * a[0];
  c[2] = q[0] * a[2] + q[2] * a[0];
  c[3] = q[1] * a[1] + q[3] * a[0];
  c[4] = q[1] * a[2] + q[2] * a[1] + q[4] * a[0];
  c[5] = q[2] * a[2] + q[5] * a[0];
  c[6] = q[3] * a[1];
  c[7] = q[3] * a[2] + q[4] * a[1];
  c[8] = q[4] * a[2] + q[5] * a[1];
  c[9] = q[5] * a[2];
}

template <typename R, int ORDER>
SPH2D_HD bool bary_monomials(const R* v, R (*prod)[10]) {
  const R D = diff_of_products(v[2] - v[0], v[5] - v[1], v[3] - v[1], v[4] - v[0]);
  if (D == R(0)) return false;
  const R iD = R(1) / D;
  R L[3][3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const int ia = j == 2 ? 0 : j + 1, ib = ia == 2 ? 0 : ia + 1;
    const R ax = v[2 * ia], ay = v[2 * ia + 1], bx = v[2 * ib], by = v[2 * ib + 1];
    L[j][0] = diff_of_products(ax, by, ay, bx) * iD;
    L[j][1] = (ay - by) * iD;
    L[j][2] = (bx - ax) * iD;
  }
  constexpr int NB = nodes_of(ORDER);
#pragma unroll
  for (int b = 0; b < NB; ++b)
#pragma unroll
    for (int i = 0; i < 10; ++i) prod[b][i] = R(0);
  if (ORDER == 1) {
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int i = 0; i < 3; ++i) prod[j][i] = L[j][i];
  } else if (ORDER == 2) {
    mul_aff(L[0], L[0], prod[0]);
    mul_aff(L[1], L[1], prod[1]);
    mul_aff(L[2], L[2], prod[2]);
    mul_aff(L[0], L[1], prod[3]);
    mul_aff(L[1], L[2], prod[4]);
    mul_aff(L[2], L[0], prod[5]);
  } else {
    R q[6];
    mul_aff(L[0], L[0], q);
    mul_quad_aff(q, L[0], prod[0]);                      // l0^3
    mul_quad_aff(q, L[1], prod[3]);                      // l0^2 l1
    mul_quad_aff(q, L[2], prod[8]);                      // l2 l0^2
    mul_aff(L[1], L[1], q);
    mul_quad_aff(q, L[1], prod[1]);                      // l1^3
    mul_quad_aff(q, L[0], prod[4]);                      // l0 l1^2
    mul_quad_aff(q, L[2], prod[5]);                      // l1^2 l2
    mul_aff(L[2], L[2], q);
    mul_quad_aff(q, L[2], prod[2]);                      // l2^3
    mul_quad_aff(q, L[1], prod[6]);                      // l1 l2^2
    mul_quad_aff(q, L[0], prod[7]);                      // l2^2 l0
    mul_aff(L[0], L[1], q);
    mul_quad_aff(q, L[2], prod[9]);                      // l0 l1 l2
  }
  return true;
}

// ---------------------------------------------------------------------------------------
// one pair in the local frame: nf (<= NFMAX) fields with homogeneous coefficients B[f][NB]
// -> out[3 f + {0, 1, 2}] = <A>, <grad A> (world units, as eval_local)
// ---------------------------------------------------------------------------------------
template <typename R, int KID, int ORDER, bool GRAD, int NFMAX>
SPH2D_HD void field_p_local(const R* v, const R (*B)[nodes_of(3)], int nf, double C, double invH, R* out) {
  constexpr int NB = nodes_of(ORDER);
#pragma unroll
  for (int i = 0; i < 3 * NFMAX; ++i) out[i] = R(0);
  const int s = tri_orientation<R>(v[0], v[1], v[2], v[3], v[4], v[5]);
  if (s == 0) return;
  // the moments first (the closed form's working set), then the field's expansion
  R M[10];
  {
    PairOut<R> o;
    tri_raw<R, KID, 3>(v[0], v[1], v[2], v[3], v[4], v[5], o);
    const R k = R(C) * R(s);
#pragma unroll
    for (int i = 0; i < 10; ++i) M[i] = k * o.m[i];
  }
  R c[NFMAX][10];
  {
    R prod[NB][10];
    if (!bary_monomials<R, ORDER>(v, prod)) return;
#pragma unroll
    for (int f = 0; f < NFMAX; ++f) {
#pragma unroll
      for (int i = 0; i < 10; ++i) c[f][i] = R(0);
      if (f < nf) {
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
          for (int i = 0; i < 10; ++i) c[f][i] += B[f][b] * prod[b][i];
      }
    }
  }
#pragma unroll
  for (int f = 0; f < NFMAX; ++f) {
    if (f < nf) {
      R val = R(0);
#pragma unroll
      for (int i = 0; i < 10; ++i) val += c[f][i] * M[i];
      out[3 * f] = val;
      if (GRAD) {
        // area term (1/H) int W grad A: d/dxi and d/deta of the monomials up to degree 3
        const R ih = R(invH);
        const R gx = c[f][1] * M[0] + R(2) * c[f][3] * M[1] + c[f][4] * M[2] + R(3) * c[f][6] * M[3] +
                     R(2) * c[f][7] * M[4] + c[f][8] * M[5];
        const R gy = c[f][2] * M[0] + c[f][4] * M[1] + R(2) * c[f][5] * M[2] + c[f][7] * M[3] +
                     R(2) * c[f][8] * M[4] + R(3) * c[f][9] * M[5];
        out[3 * f + 1] = ih * gx;
        out[3 * f + 2] = ih * gy;
      }
    }
  }
  if (!GRAD) return;
  // boundary term -(C/H) sum_e n_e int A(p(t)) k(rho) dt
  const R sg = R(s);
  const R kb = -R(C) * R(invH);
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
    const R fl = ax * nx + ay * ny;                      // signed line distance
    const R d = fabs(fl);
    if (!(d < R(1))) continue;                           // edge line outside the support
    const R tA = ax * ux + ay * uy, tB = bx * ux + by * uy;
    const R ts = sqrt((R(1) - d) * (R(1) + d));
    const R t1 = fmin(fmax(tA, -ts), ts), t2 = fmin(fmax(tB, -ts), ts);
    if (!(t2 > t1)) continue;
    R I[4];
    edge_poly_integrals_k<R, KID>(d, t1, t2, I);
    // xi = X0 + X1 t, eta = Y0 + Y1 t along the edge; powers as polynomials in t
    const R X0 = fl * nx, X1 = ux, Y0 = fl * ny, Y1 = uy;
    const R xx[3] = {X0 * X0, R(2) * X0 * X1, X1 * X1};
    const R yy[3] = {Y0 * Y0, R(2) * Y0 * Y1, Y1 * Y1};
    const R xy[3] = {X0 * Y0, X0 * Y1 + X1 * Y0, X1 * Y1};
    // int (monomial) k dt for the ten monomials
    R mi[10];
    mi[0] = I[0];
    mi[1] = X0 * I[0] + X1 * I[1];
    mi[2] = Y0 * I[0] + Y1 * I[1];
    mi[3] = xx[0] * I[0] + xx[1] * I[1] + xx[2] * I[2];
    mi[4] = xy[0] * I[0] + xy[1] * I[1] + xy[2] * I[2];
    mi[5] = yy[0] * I[0] + yy[1] * I[1] + yy[2] * I[2];
    if (ORDER >= 3) {
      // (a0 + a1 t + a2 t^2)(b0 + b1 t) integrated against k: cubic in t
      auto cub = [&](const R* q, R b0, R b1) {
        return q[0] * b0 * I[0] + (q[0] * b1 + q[1] * b0) * I[1] + (q[1] * b1 + q[2] * b0) * I[2] + q[2] * b1 * I[3];
      };
      mi[6] = cub(xx, X0, X1);
      mi[7] = cub(xx, Y0, Y1);
      mi[8] = cub(yy, X0, X1);
      mi[9] = cub(yy, Y0, Y1);
    } else {
      mi[6] = mi[7] = mi[8] = mi[9] = R(0);
    }
#pragma unroll
    for (int f = 0; f < NFMAX; ++f) {
      if (f < nf) {
        R a = R(0);
#pragma unroll
        for (int i = 0; i < 10; ++i) a += c[f][i] * mi[i];
        out[3 * f + 1] += kb * a * nx;
        out[3 * f + 2] += kb * a * ny;
      }
    }
  }
}

}  // namespace sph2d
