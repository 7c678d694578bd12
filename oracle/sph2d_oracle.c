/*
 * sph2d oracle -- plain, slow, FP64 CPU reference for the 2-D analytic SPH boundary
 * integrals of Winchenbach & Kolb, "Solving Boundary Handling Analytically in Two
 * Dimensions for SPH" (arXiv 2507.21686).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call this file;
 * only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg use it.  It shares no
 * code with the CUDA path: the method there is a closed-form edge/sector decomposition,
 * here every result is the plain definition evaluated by quadrature.
 *
 * What it computes (local frame of Sec. 2: p = (x' - x_i)/H, W = C/H^2 k(|p|)):
 *   gamma   = int_T W dx'               = C int_{T*} k(|p|) dA                   (Eq. sphintegral)
 *   grad    = d gamma / d x_i           = -(C/H) sum_e n_e int_e k(|p|) ds      (divergence theorem)
 *             cross-checked by the polar form -(C/H) int_{T*} k'(|p|) p/|p| dA  (Eq. basicdiff)
 *   M_ab    = int_T xi^a eta^b W dx'    = C int_{T*} p_x^a p_y^b k(|p|) dA,  a+b <= 3
 *   dgamma/dnu_j = (C/H) sum_{e ni j} n_e int_e k(|p|) lambda_j ds          (transport theorem)
 * Area integrals use polar coordinates about the particle (Eq. singleSpherical): for each
 * ray angle theta the triangle is clipped to an interval [r0, r1] (Cyrus-Beck), clipped again
 * to the unit support, and the radial integral is done by Gauss-Legendre on the factored
 * kernel (exact: the integrand is a polynomial in r on each kernel piece).  The angular
 * integral is adaptive Gauss-Legendre, split at vertex angles, foot angles and the angles
 * where edge lines cross the kernel's piece radii.  Line integrals are adaptive
 * Gauss-Legendre split at the foot point and the circle crossings.
 *
 * Kernels (Sec. 2, "W = C_d k(q)/h^d"; normalisation int W = 1 in 2-D):
 *   0 Wendland C2: k = (1-q)^4 (1+4q),                    C = 7/pi
 *   1 Wendland C4: k = (1-q)^6 (1+6q+35/3 q^2),           C = 9/pi
 *     (the paper prints 27/(16 pi) for this kernel; that value does not give int W = 1)
 *   2 Wendland C6: k = (1-q)^8 (1+8q+25q^2+32q^3),        C = 78/(7 pi)
 *   3 cubic B-spline: k = 1-6q^2+6q^3 (q<1/2), 2(1-q)^3 (1/2<=q<1), C = 40/(7 pi)
 *
 * Pair culling (Sec. 2: triangles overlapping the support): pair (i, T) is kept iff the
 * closed triangle's Euclidean distance to x_i is < H, evaluated in FP64 from the FP32
 * inputs with the operation order fixed in include/sph2d.h (built with -ffp-contract=off).
 *
 * Parity pins for every function here live in tests/test_oracle_pins.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* mutation hooks: tests compile deliberately wrong variants of this file (-DORC_MUTANT=n) to
 * show that the pins catch each plausible mistake.  The default build has none. */
#ifndef ORC_MUTANT
#define ORC_MUTANT 0
#endif

enum { K_WC2 = 0, K_WC4 = 1, K_WC6 = 2, K_CUBIC = 3 };

int orc_version(void) { return 1; }

/* ------------------------------------------------------------------------------------ */
/* kernels                                                                               */
/* ------------------------------------------------------------------------------------ */
static int kernel_ok(int kid) { return kid >= 0 && kid <= 3; }

double orc_kernel_C(int kid) {
  switch (kid) {
    case K_WC2: return (ORC_MUTANT == 1 ? 27.0 / 16.0 : 7.0) / M_PI;
    case K_WC4: return 9.0 / M_PI;
    case K_WC6: return 78.0 / (7.0 * M_PI);
    case K_CUBIC: return 40.0 / (7.0 * M_PI);
  }
  return 0.0;
}

/* k(q) in the factored form printed for the Wendland family */
double orc_kernel_k(int kid, double q) {
  if (q >= 1.0) return 0.0;
  double s = 1.0 - q;
  switch (kid) {
    case K_WC2: { double s2 = s * s; return s2 * s2 * (1.0 + 4.0 * q); }
    case K_WC4: { double s3 = s * s * s; return s3 * s3 * (1.0 + 6.0 * q + 35.0 / 3.0 * q * q); }
    case K_WC6: { double s4 = s * s * s * s;
                  return s4 * s4 * (1.0 + 8.0 * q + 25.0 * q * q + 32.0 * q * q * q); }
    case K_CUBIC: return q < 0.5 ? 1.0 - 6.0 * q * q + 6.0 * q * q * q : 2.0 * s * s * s;
  }
  return 0.0;
}

/* dk/dq (used only by the polar cross-check route of the gradient) */
double orc_kernel_dk(int kid, double q) {
  if (q >= 1.0) return 0.0;
  double s = 1.0 - q;
  switch (kid) {
    case K_WC2: return -20.0 * q * s * s * s;
    case K_WC4: { double s5 = s * s * s * s * s; return -(56.0 / 3.0) * q * s5 * (1.0 + 5.0 * q); }
    case K_WC6: { double s7 = s * s * s * s * s * s * s;
                  return -22.0 * q * s7 * (1.0 + 7.0 * q + 16.0 * q * q); }
    case K_CUBIC: return q < 0.5 ? -12.0 * q + 18.0 * q * q : -6.0 * s * s;
  }
  return 0.0;
}

/* radii where k changes its polynomial piece (besides 0): {1} or {1/2, 1} */
static int kernel_piece_radii(int kid, double* r) {
  if (kid == K_CUBIC) { r[0] = 0.5; r[1] = 1.0; return 2; }
  r[0] = 1.0;
  return 1;
}

/* ------------------------------------------------------------------------------------ */
/* Gauss-Legendre nodes by Newton iteration on P_n (no tables)                           */
/* ------------------------------------------------------------------------------------ */
#define GL_RAD 12   /* radial rule: exact for polynomials up to degree 23 */
#define GL_ANG 20   /* angular / line rule */
static double glr_x[GL_RAD], glr_w[GL_RAD];
static double gla_x[GL_ANG], gla_w[GL_ANG];
static int gl_ready = 0;

static void gauss_legendre(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1; p1 = p2;
      }
      /* P_n = p1, P_{n-1} = p0 */
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-17) break;
    }
    {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1; p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

static void gl_init(void) {
  if (gl_ready) return;
#pragma omp critical(orc_gl_init)
  {
    if (!gl_ready) {
      gauss_legendre(GL_RAD, glr_x, glr_w);
      gauss_legendre(GL_ANG, gla_x, gla_w);
      gl_ready = 1;
    }
  }
}

void orc_gauss_legendre(int n, double* x, double* w) { gauss_legendre(n, x, w); }

/* ------------------------------------------------------------------------------------ */
/* radial integrals on [r0, r1] within one kernel piece, exact by Gauss-Legendre         */
/*   out[0]          = int k(r) r dr                    (gamma density)                  */
/*   out[1]          = int k'(r) r dr                   (polar gradient density)         */
/*   out[2 + m]      = int k(r) r^(1+m) dr, m = 0..3   (moment densities)               */
/*   out[6]          = int k'(r) r^2 dr                  (gradient density, linear field) */
/* ------------------------------------------------------------------------------------ */
#define NRAD 7
static void radial_piece(int kid, double r0, double r1, double* out) {
  double h = 0.5 * (r1 - r0), c = 0.5 * (r1 + r0);
  for (int i = 0; i < GL_RAD; ++i) {
    double r = c + h * glr_x[i], w = h * glr_w[i];
    double k = orc_kernel_k(kid, r), dk = orc_kernel_dk(kid, r);
#if ORC_MUTANT == 4
    out[0] += w * k;              /* dropped the polar Jacobian r */
#else
    out[0] += w * k * r;
#endif
    out[1] += w * dk * r;
#if ORC_MUTANT == 5
    out[6] += w * dk * r;         /* lost a power of r in the linear-field gradient density */
#else
    out[6] += w * dk * r * r;
#endif
    double rm = r;                                   /* r^(1+m) */
    for (int m = 0; m < 4; ++m) { out[2 + m] += w * k * rm; rm *= r; }
  }
}

static void radial(int kid, double r0, double r1, double* out) {
  for (int i = 0; i < NRAD; ++i) out[i] = 0.0;
  if (r1 > 1.0) r1 = 1.0;
  if (r0 < 0.0) r0 = 0.0;
  if (!(r1 > r0)) return;
  if (kid == K_CUBIC && r0 < 0.5 && r1 > 0.5) {
    radial_piece(kid, r0, 0.5, out);
    radial_piece(kid, 0.5, r1, out);
  } else {
    radial_piece(kid, r0, r1, out);
  }
}

/* ------------------------------------------------------------------------------------ */
/* triangle geometry                                                                     */
/* ------------------------------------------------------------------------------------ */
typedef struct {
  double v[3][2];     /* local-frame vertices, counter-clockwise */
  double n[3][2];     /* outward edge normals (unnormalised), edge e = (v[e], v[e+1]) */
  double c[3];        /* half-planes n_e . p <= c_e */
} tri_t;

/* returns orientation sign of the input (+1 CCW, -1 CW, 0 degenerate) */
static int tri_setup(const double* p /* [6] local */, tri_t* t) {
  double ax = p[0], ay = p[1], bx = p[2], by = p[3], cx = p[4], cy = p[5];
  double area2 = (bx - ax) * (cy - ay) - (by - ay) * (cx - ax);
  if (area2 == 0.0) return 0;
  int s = area2 > 0 ? 1 : -1;
  if (s > 0) {
    t->v[0][0] = ax; t->v[0][1] = ay; t->v[1][0] = bx; t->v[1][1] = by; t->v[2][0] = cx; t->v[2][1] = cy;
  } else {
    t->v[0][0] = ax; t->v[0][1] = ay; t->v[1][0] = cx; t->v[1][1] = cy; t->v[2][0] = bx; t->v[2][1] = by;
  }
  for (int e = 0; e < 3; ++e) {
    const double* A = t->v[e];
    const double* B = t->v[(e + 1) % 3];
    double ex = B[0] - A[0], ey = B[1] - A[1];
    t->n[e][0] = ey; t->n[e][1] = -ex;       /* outward for CCW */
    t->c[e] = t->n[e][0] * A[0] + t->n[e][1] * A[1];
  }
  return s;
}

/* ray {r u : r >= 0} clipped by the triangle -> [r0, r1]; returns 0 if empty */
static int ray_clip(const tri_t* t, double ux, double uy, double* r0, double* r1) {
  double lo = 0.0, hi = INFINITY;
  for (int e = 0; e < 3; ++e) {
    double nu = t->n[e][0] * ux + t->n[e][1] * uy;
    double c = t->c[e];
    if (nu > 0.0) { double r = c / nu; if (r < hi) hi = r; }
    else if (nu < 0.0) { double r = c / nu; if (r > lo) lo = r; }
    else if (c < 0.0) return 0;
  }
  if (!(hi > lo)) return 0;
  *r0 = lo; *r1 = hi;
  return 1;
}

/* ------------------------------------------------------------------------------------ */
/* polar angular integrand: vector of area-integral densities at angle theta             */
/*   f[0] gamma, f[1..2] polar gradient (without -C/H), f[3..12] moments M_ab (no C)     */
/* ------------------------------------------------------------------------------------ */
#define NOUT 13
static const int MOM_A[10] = {0, 1, 0, 2, 1, 0, 3, 2, 1, 0};
static const int MOM_B[10] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3};

static void polar_density(int kid, const tri_t* t, double th, double* f) {
  for (int i = 0; i < NOUT; ++i) f[i] = 0.0;
  double ux = cos(th), uy = sin(th), r0, r1;
  if (!ray_clip(t, ux, uy, &r0, &r1)) return;
  if (r0 >= 1.0) return;
  double rad[NRAD];
  radial(kid, r0, r1, rad);
  f[0] = rad[0];
  f[1] = rad[1] * ux;
  f[2] = rad[1] * uy;
  for (int m = 0; m < 10; ++m) {
    int a = MOM_A[m], b = MOM_B[m];
#if ORC_MUTANT == 3
    { int tmp = a; a = b; b = tmp; }      /* transposed moment exponents */
#endif
    double ang = 1.0;
    for (int i = 0; i < a; ++i) ang *= ux;
    for (int i = 0; i < b; ++i) ang *= uy;
    f[3 + m] = rad[2 + a + b] * ang;
  }
}

/* ------------------------------------------------------------------------------------ */
/* adaptive Gauss-Legendre for vector integrands                                         */
/* ------------------------------------------------------------------------------------ */
typedef void (*vec_fn)(const void* ctx, double x, double* f);

typedef struct { int max_depth_hit; long evals; } quad_stats;

static void gl_fixed(vec_fn fn, const void* ctx, int nout, double a, double b, double* q, double* qabs) {
  double h = 0.5 * (b - a), c = 0.5 * (b + a), f[NOUT];
  for (int j = 0; j < nout; ++j) { q[j] = 0.0; qabs[j] = 0.0; }
  for (int i = 0; i < GL_ANG; ++i) {
    fn(ctx, c + h * gla_x[i], f);
    for (int j = 0; j < nout; ++j) { q[j] += h * gla_w[i] * f[j]; qabs[j] += fabs(h * gla_w[i] * f[j]); }
  }
}

static void adapt(vec_fn fn, const void* ctx, int nout, double a, double b, const double* whole,
                  int depth, double tol, double* acc, quad_stats* st) {
  double m = 0.5 * (a + b), ql[NOUT], qr[NOUT], al[NOUT], ar[NOUT];
  gl_fixed(fn, ctx, nout, a, m, ql, al);
  gl_fixed(fn, ctx, nout, m, b, qr, ar);
  st->evals += 2 * GL_ANG;
  int ok = 1;
  for (int j = 0; j < nout; ++j) {
    double err = fabs(whole[j] - (ql[j] + qr[j]));
    double floor_ = 32.0 * 2.220446049250313e-16 * (al[j] + ar[j]);
    if (err > tol && err > floor_) { ok = 0; break; }
  }
  if (ok || depth >= 70) {
    if (!ok) st->max_depth_hit = 1;
    for (int j = 0; j < nout; ++j) acc[j] += ql[j] + qr[j];
    return;
  }
  adapt(fn, ctx, nout, a, m, ql, depth + 1, tol, acc, st);
  adapt(fn, ctx, nout, m, b, qr, depth + 1, tol, acc, st);
}

static void integrate(vec_fn fn, const void* ctx, int nout, double a, double b, double tol,
                      double* acc, quad_stats* st) {
  if (!(b > a)) return;
  double q[NOUT], qa[NOUT];
  gl_fixed(fn, ctx, nout, a, b, q, qa);
  st->evals += GL_ANG;
  adapt(fn, ctx, nout, a, b, q, 0, tol, acc, st);
}

static int cmp_dbl(const void* x, const void* y) {
  double a = *(const double*)x, b = *(const double*)y;
  return (a > b) - (a < b);
}

/* ------------------------------------------------------------------------------------ */
/* area integrals over one local-frame triangle: gamma, polar gradient, moments          */
/* ------------------------------------------------------------------------------------ */
typedef struct { int kid; const tri_t* t; } polar_ctx;

static void polar_fn(const void* ctx, double th, double* f) {
  const polar_ctx* pc = (const polar_ctx*)ctx;
  polar_density(pc->kid, pc->t, th, f);
}

static double wrap2pi(double a) {
  a = fmod(a, 2.0 * M_PI);
  if (a < 0) a += 2.0 * M_PI;
  return a;
}

/* integrate the angular density fn over the triangle's angles, split at the breakpoints below */
static void polar_integrate(int kid, const tri_t* t, vec_fn fn, const void* ctx, int nout, double* out,
                            quad_stats* st);

/* raw area integrals (without the constant C): out[NOUT] */
static void area_integrals(int kid, const tri_t* t, double* out, quad_stats* st) {
  polar_ctx pc = {kid, t};
  polar_integrate(kid, t, polar_fn, &pc, NOUT, out, st);
}

static void polar_integrate(int kid, const tri_t* t, vec_fn fn, const void* ctx, int nout, double* out,
                            quad_stats* st) {
  double bp[512];
  int nb = 0;
  double radii[2];
  int nr = kernel_piece_radii(kid, radii);
  for (int e = 0; e < 3; ++e) {
    bp[nb++] = wrap2pi(atan2(t->v[e][1], t->v[e][0]));
    double nx = t->n[e][0], ny = t->n[e][1], L = hypot(nx, ny);
    double d = fabs(t->c[e]) / L;
    double phi = atan2(ny, nx);
    if (t->c[e] < 0) phi += M_PI;            /* foot direction */
    bp[nb++] = wrap2pi(phi);
    for (int k = 0; k < nr; ++k) {
      if (d < radii[k]) {
        double a = acos(d / radii[k]);
        bp[nb++] = wrap2pi(phi + a);
        bp[nb++] = wrap2pi(phi - a);
      }
    }
    /* an edge line passing within d << 1 of the particle: along the ray the hit distance is
     * r ~ d / w with w = pi/2 - |theta - phi|, so the radial limits change on the angular
     * scale d next to the two grazing directions.  Grade the angle geometrically there so
     * that the rule resolves it instead of stepping over it. */
    if (d > 0.0 && d < 0.1) {
      for (double w = d; w < 0.5 && nb < 500; w *= 2.0) {
        bp[nb++] = wrap2pi(phi + 0.5 * M_PI - w);
        bp[nb++] = wrap2pi(phi - 0.5 * M_PI + w);
      }
    }
  }
  qsort(bp, nb, sizeof(double), cmp_dbl);
  for (int j = 0; j < nout; ++j) out[j] = 0.0;
  const double tol = 1e-17;
  for (int i = 0; i < nb; ++i) {
    double a = bp[i], b = (i + 1 < nb) ? bp[i + 1] : bp[0] + 2.0 * M_PI;
    integrate(fn, ctx, nout, a, b, tol, out, st);
  }
}

/* ------------------------------------------------------------------------------------ */
/* linear boundary field A(p) = a0 + ax p_x + ay p_y over the triangle (local frame):     */
/*   f[0] = int A(r u) k(r) r dr,  f[1..2] = u int A(r u) k'(r) r dr                      */
/* along the ray of direction u, clipped to the triangle and the support                 */
/* ------------------------------------------------------------------------------------ */
typedef struct { int kid; const tri_t* t; double a0, ax, ay; } field_ctx;

static void field_fn(const void* ctx, double th, double* f) {
  const field_ctx* fc = (const field_ctx*)ctx;
  f[0] = f[1] = f[2] = 0.0;
  double ux = cos(th), uy = sin(th), r0, r1;
  if (!ray_clip(fc->t, ux, uy, &r0, &r1)) return;
  if (r0 >= 1.0) return;
  double rad[NRAD];
  radial(fc->kid, r0, r1, rad);
  double au = fc->ax * ux + fc->ay * uy;          /* A(r u) = a0 + r (a . u) */
  f[0] = fc->a0 * rad[0] + au * rad[3];            /* rad[3] = int k r^2 dr */
  double g = fc->a0 * rad[1] + au * rad[6];        /* int A k'(r) r dr */
  f[1] = g * ux;
  f[2] = g * uy;
}

/* ------------------------------------------------------------------------------------ */
/* Lagrange (P1, P2, P3) boundary fields over the triangle (Sec. 3 interpolates a field     */
/* linearly; the paper's introduction names higher-order element fields as the extension).  */
/* Nodes: the principal lattice {(i, j, l)/k : i + j + l = k} in barycentric coordinates,   */
/* ordered vertices 0, 1, 2; then each edge (0,1), (1,2), (2,0) from its first vertex to    */
/* its second; then the interior node (P3: the centroid).  The basis function of the node   */
/* with indices (i, j, l) is Silvester's product R_i(k lambda_0) R_j(k lambda_1)            */
/* R_l(k lambda_2), R_n(z) = prod_{s<n} (z - s)/(s + 1): 1 at its node, 0 at the others.    */
/* ------------------------------------------------------------------------------------ */
static const int NODES_P1[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
static const int NODES_P2[6][3] = {{2, 0, 0}, {0, 2, 0}, {0, 0, 2}, {1, 1, 0}, {0, 1, 1}, {1, 0, 1}};
#if ORC_MUTANT == 6
/* the two nodes of edge (0,1) swapped */
static const int NODES_P3[10][3] = {{3, 0, 0}, {0, 3, 0}, {0, 0, 3}, {1, 2, 0}, {2, 1, 0},
                                    {0, 2, 1}, {0, 1, 2}, {1, 0, 2}, {2, 0, 1}, {1, 1, 1}};
#else
static const int NODES_P3[10][3] = {{3, 0, 0}, {0, 3, 0}, {0, 0, 3}, {2, 1, 0}, {1, 2, 0},
                                    {0, 2, 1}, {0, 1, 2}, {1, 0, 2}, {2, 0, 1}, {1, 1, 1}};
#endif

static double silvester_r(int n, double z) {
  double v = 1.0;
  for (int s = 0; s < n; ++s) v *= (z - s) / (s + 1);
  return v;
}

typedef struct {
  int kid, order, nn;
  const tri_t* t;
  const int (*nodes)[3];
  double A[10];
  double l0x, l0y, l0c, l1x, l1y, l1c;   /* lambda_0, lambda_1 as affine functions of p */
} nfield_ctx;

/* the field at local point (x, y) */
static double nfield_eval(const nfield_ctx* fc, double x, double y) {
  double lam[3];
  lam[0] = fc->l0c + fc->l0x * x + fc->l0y * y;
  lam[1] = fc->l1c + fc->l1x * x + fc->l1y * y;
  lam[2] = 1.0 - lam[0] - lam[1];
  double v = 0.0;
  for (int n = 0; n < fc->nn; ++n) {
    double phi = 1.0;
    for (int m = 0; m < 3; ++m) phi *= silvester_r(fc->nodes[n][m], fc->order * lam[m]);
    v += fc->A[n] * phi;
  }
  return v;
}

/* along the ray of direction u, clipped to the triangle and the support:
 *   f[0] = int A(r u) k(r) r dr,  f[1..2] = u int A(r u) k'(r) r dr
 * by Gauss-Legendre on each kernel piece (exact: a polynomial in r there) */
static void nfield_radial_piece(const nfield_ctx* fc, double ux, double uy, double r0, double r1, double* f) {
  double h = 0.5 * (r1 - r0), c = 0.5 * (r1 + r0);
  for (int i = 0; i < GL_RAD; ++i) {
    double r = c + h * glr_x[i], w = h * glr_w[i];
    double a = nfield_eval(fc, r * ux, r * uy);
    f[0] += w * a * orc_kernel_k(fc->kid, r) * r;
    f[1] += w * a * orc_kernel_dk(fc->kid, r) * r;
  }
}

static void nfield_fn(const void* ctx, double th, double* f) {
  const nfield_ctx* fc = (const nfield_ctx*)ctx;
  f[0] = f[1] = f[2] = 0.0;
  double ux = cos(th), uy = sin(th), r0, r1;
  if (!ray_clip(fc->t, ux, uy, &r0, &r1)) return;
  if (r1 > 1.0) r1 = 1.0;
  if (!(r1 > r0)) return;
  double g[2] = {0.0, 0.0};
  if (fc->kid == K_CUBIC && r0 < 0.5 && r1 > 0.5) {
    nfield_radial_piece(fc, ux, uy, r0, 0.5, g);
    nfield_radial_piece(fc, ux, uy, 0.5, r1, g);
  } else {
    nfield_radial_piece(fc, ux, uy, r0, r1, g);
  }
  f[0] = g[0];
  f[1] = g[1] * ux;
  f[2] = g[1] * uy;
}

/* ------------------------------------------------------------------------------------ */
/* edge line integrals: int_0^1 k(|A + s(B-A)|) {1, s} L ds                              */
/* ------------------------------------------------------------------------------------ */
typedef struct { int kid; double ax, ay, ex, ey, L; } edge_ctx;

static void edge_fn(const void* ctx, double s, double* f) {
  const edge_ctx* ec = (const edge_ctx*)ctx;
  double px = ec->ax + s * ec->ex, py = ec->ay + s * ec->ey;
  double k = orc_kernel_k(ec->kid, hypot(px, py)) * ec->L;
  f[0] = k;
  f[1] = k * s;
}

static void edge_integrals(int kid, const double* A, const double* B, double* out2, quad_stats* st) {
  edge_ctx ec = {kid, A[0], A[1], B[0] - A[0], B[1] - A[1], 0.0};
  ec.L = hypot(ec.ex, ec.ey);
  out2[0] = out2[1] = 0.0;
  if (ec.L == 0.0) return;
  double bp[16];
  int nb = 0;
  bp[nb++] = 0.0;
  bp[nb++] = 1.0;
  double L2 = ec.L * ec.L;
  double sf = -(A[0] * ec.ex + A[1] * ec.ey) / L2;
  if (sf > 0.0 && sf < 1.0) bp[nb++] = sf;
  double radii[2];
  int nr = kernel_piece_radii(kid, radii);
  double a2 = A[0] * A[0] + A[1] * A[1];
  double dd = a2 - (A[0] * ec.ex + A[1] * ec.ey) * (A[0] * ec.ex + A[1] * ec.ey) / L2;  /* foot distance^2 */
  if (dd < 0) dd = 0;
  for (int k = 0; k < nr; ++k) {
    double R2 = radii[k] * radii[k];
    if (dd < R2) {
      double hw = sqrt((R2 - dd) / L2);
      double s1 = sf - hw, s2 = sf + hw;
      if (s1 > 0.0 && s1 < 1.0) bp[nb++] = s1;
      if (s2 > 0.0 && s2 < 1.0) bp[nb++] = s2;
    }
  }
  qsort(bp, nb, sizeof(double), cmp_dbl);
  for (int i = 0; i + 1 < nb; ++i) integrate(edge_fn, &ec, 2, bp[i], bp[i + 1], 1e-17, out2, st);
}

/* ------------------------------------------------------------------------------------ */
/* public: one pair                                                                      */
/* ------------------------------------------------------------------------------------ */
/* out layout (16 doubles):
 *   [0] gamma  [1..2] grad gamma (divergence theorem)  [3..4] grad gamma (polar, k')
 *   [5..14] moments M00 M10 M01 M20 M11 M02 M30 M21 M12 M03
 *   [15] flags: 1 = adaptive depth cap hit somewhere
 * xp: particle position, tri: 6 vertex coordinates, both in world units, H > 0.
 * returns 0 on success, -1 on bad arguments. */
int orc_pair(int kid, double H, const double* xp, const double* tri, double* out) {
  if (!kernel_ok(kid) || !(H > 0.0)) return -1;
  gl_init();
  for (int i = 0; i < 16; ++i) out[i] = 0.0;
  double p[6];
  for (int j = 0; j < 3; ++j) {
    p[2 * j] = (tri[2 * j] - xp[0]) / H;
    p[2 * j + 1] = (tri[2 * j + 1] - xp[1]) / H;
  }
  tri_t t;
  if (tri_setup(p, &t) == 0) return 0;          /* zero-area triangle: all integrals vanish */
  quad_stats st = {0, 0};
  double C = orc_kernel_C(kid);
  double a[NOUT];
  area_integrals(kid, &t, a, &st);
  out[0] = C * a[0];
  out[3] = -(C / H) * a[1];
  out[4] = -(C / H) * a[2];
  for (int m = 0; m < 10; ++m) out[5 + m] = C * a[3 + m];
  /* divergence theorem: grad = -(C/H) sum_e nhat_e int_e k ds (outward unit normals) */
  double gx = 0.0, gy = 0.0;
  for (int e = 0; e < 3; ++e) {
    double li[2];
    edge_integrals(kid, t.v[e], t.v[(e + 1) % 3], li, &st);
    double L = hypot(t.n[e][0], t.n[e][1]);
    if (L == 0.0) continue;
    gx += t.n[e][0] / L * li[0];
    gy += t.n[e][1] / L * li[0];
  }
#if ORC_MUTANT == 2
  out[1] = (C / H) * gx;       /* sign flip of the gradient */
  out[2] = (C / H) * gy;
#else
  out[1] = -(C / H) * gx;
  out[2] = -(C / H) * gy;
#endif
  out[15] = st.max_depth_hit ? 1.0 : 0.0;
  return 0;
}

/* d gamma / d nu_j for j = 0,1,2 (in the caller's vertex order): out[6] = (dx0,dy0,dx1,dy1,dx2,dy2)
 * transport theorem: moving vertex j moves the two adjacent edges with the hat weight
 * lambda_j; d gamma = sum_e int_e W (V . n_out) ds. */
int orc_vertex_grad(int kid, double H, const double* xp, const double* tri, double* out) {
  if (!kernel_ok(kid) || !(H > 0.0)) return -1;
  gl_init();
  for (int i = 0; i < 6; ++i) out[i] = 0.0;
  double p[6];
  for (int j = 0; j < 3; ++j) {
    p[2 * j] = (tri[2 * j] - xp[0]) / H;
    p[2 * j + 1] = (tri[2 * j + 1] - xp[1]) / H;
  }
  double area2 = (p[2] - p[0]) * (p[5] - p[1]) - (p[3] - p[1]) * (p[4] - p[0]);
  if (area2 == 0.0) return 0;
  double sgn = area2 > 0 ? 1.0 : -1.0;
  quad_stats st = {0, 0};
  double C = orc_kernel_C(kid);
  for (int e = 0; e < 3; ++e) {
    int ia = e, ib = (e + 1) % 3;
    const double* A = p + 2 * ia;
    const double* B = p + 2 * ib;
    double ex = B[0] - A[0], ey = B[1] - A[1], L = hypot(ex, ey);
    if (L == 0.0) continue;
    double nx = sgn * ey / L, ny = -sgn * ex / L;     /* outward unit normal */
    double li[2];
    edge_integrals(kid, A, B, li, &st);
    double wa = li[0] - li[1], wb = li[1];           /* hat weights: lambda_a = 1-s, lambda_b = s */
    out[2 * ia] += (C / H) * wa * nx;
    out[2 * ia + 1] += (C / H) * wa * ny;
    out[2 * ib] += (C / H) * wb * nx;
    out[2 * ib + 1] += (C / H) * wb * ny;
  }
  return 0;
}

/* Piecewise-linear field on one triangle (Sec. 3, Eq. singleSpherical and basicdiff): vertex
 * values A[3] in the caller's vertex order, interpolated barycentrically.
 *   out[0] = int_T A(x') W(x - x') dx'                   <A>
 *   out[1..2] = int_T A(x') grad_x W(x - x') dx'         <grad A> = -(C/H) int A k'(|p|) p/|p|
 * by polar quadrature of the field times the kernel (no moments, no integration by parts). */
int orc_pair_field(int kid, double H, const double* xp, const double* tri, const double* A, double* out) {
  if (!kernel_ok(kid) || !(H > 0.0)) return -1;
  gl_init();
  out[0] = out[1] = out[2] = 0.0;
  double p[6];
  for (int j = 0; j < 3; ++j) {
    p[2 * j] = (tri[2 * j] - xp[0]) / H;
    p[2 * j + 1] = (tri[2 * j + 1] - xp[1]) / H;
  }
  tri_t t;
  if (tri_setup(p, &t) == 0) return 0;
  /* barycentric weights (Sec. 3): D = (y1-y2)(x0-x2) + (x2-x1)(y0-y2),
   * lambda0 = ((y1-y2)(x-x2) + (x2-x1)(y-y2)) / D, lambda1 = ((y2-y0)(x-x2) + (x0-x2)(y-y2)) / D,
   * lambda2 = 1 - lambda0 - lambda1; A = A2 + lambda0 (A0 - A2) + lambda1 (A1 - A2).
   * Written as A(p) = a0 + ax p_x + ay p_y. */
  double x0 = p[0], y0 = p[1], x1 = p[2], y1 = p[3], x2 = p[4], y2 = p[5];
  double D = (y1 - y2) * (x0 - x2) + (x2 - x1) * (y0 - y2);
  double l0x = (y1 - y2) / D, l0y = (x2 - x1) / D, l0c = -(l0x * x2 + l0y * y2);
  double l1x = (y2 - y0) / D, l1y = (x0 - x2) / D, l1c = -(l1x * x2 + l1y * y2);
  double d0 = A[0] - A[2], d1 = A[1] - A[2];
  field_ctx fc = {kid, &t, A[2] + l0c * d0 + l1c * d1, l0x * d0 + l1x * d1, l0y * d0 + l1y * d1};
  quad_stats st = {0, 0};
  double q[3];
  polar_integrate(kid, &t, field_fn, &fc, 3, q, &st);
  double C = orc_kernel_C(kid);
  out[0] = C * q[0];
  out[1] = -(C / H) * q[1];
  out[2] = -(C / H) * q[2];
  return st.max_depth_hit ? 1 : 0;
}

/* ------------------------------------------------------------------------------------ */
/* second order: d grad gamma / d nu_j.  grad gamma = -(C/H) oint k(|p|) n_out ds in the    */
/* local frame (divergence theorem).  Edge e = (A, B): F_e = n_out L int_0^1 k(|A + s(B-A)|) */
/* ds; its derivative by B is sg R I + n_out L (x) U_s and by A is -sg R I + n_out L (x)     */
/* (U_1 - U_s), R (x, y) = (y, -x), I = int k ds, U_1 = int k'(rho) p/rho ds, U_s = int       */
/* k'(rho) p/rho s ds (s from A to B).  Here I, U_1, U_s are plain 1-D quadratures.         */
/* ------------------------------------------------------------------------------------ */
typedef struct { int kid; double ax, ay, ex, ey; } edge2_ctx;

static void edge2_fn(const void* ctx, double s, double* f) {
  const edge2_ctx* ec = (const edge2_ctx*)ctx;
  double px = ec->ax + s * ec->ex, py = ec->ay + s * ec->ey;
  double r = hypot(px, py);
  double k = orc_kernel_k(ec->kid, r);
  double dk = r > 0.0 ? orc_kernel_dk(ec->kid, r) / r : 0.0;     /* k'(r)/r, p/r direction */
  f[0] = k;
  f[1] = dk * px;
  f[2] = dk * py;
  f[3] = dk * px * s;
  f[4] = dk * py * s;
}

static void edge2_integrals(int kid, const double* A, const double* B, double* out5, quad_stats* st) {
  edge2_ctx ec = {kid, A[0], A[1], B[0] - A[0], B[1] - A[1]};
  for (int i = 0; i < 5; ++i) out5[i] = 0.0;
  double L2 = ec.ex * ec.ex + ec.ey * ec.ey;
  if (L2 == 0.0) return;
  double bp[16];
  int nb = 0;
  bp[nb++] = 0.0;
  bp[nb++] = 1.0;
  double sf = -(A[0] * ec.ex + A[1] * ec.ey) / L2;
  if (sf > 0.0 && sf < 1.0) bp[nb++] = sf;
  double radii[2];
  int nr = kernel_piece_radii(kid, radii);
  double dd = A[0] * A[0] + A[1] * A[1] - (A[0] * ec.ex + A[1] * ec.ey) * (A[0] * ec.ex + A[1] * ec.ey) / L2;
  if (dd < 0) dd = 0;
  for (int k = 0; k < nr; ++k) {
    double R2 = radii[k] * radii[k];
    if (dd < R2) {
      double hw = sqrt((R2 - dd) / L2);
      if (sf - hw > 0.0 && sf - hw < 1.0) bp[nb++] = sf - hw;
      if (sf + hw > 0.0 && sf + hw < 1.0) bp[nb++] = sf + hw;
    }
  }
  qsort(bp, nb, sizeof(double), cmp_dbl);
  for (int i = 0; i + 1 < nb; ++i) integrate(edge2_fn, &ec, 5, bp[i], bp[i + 1], 1e-17, out5, st);
}

/* out[12]: out[4 j + 2 b + a] = d (grad gamma)_b / d (nu_j)_a, caller's vertex order */
int orc_grad_jacobian(int kid, double H, const double* xp, const double* tri, double* out) {
  if (!kernel_ok(kid) || !(H > 0.0)) return -1;
  gl_init();
  for (int i = 0; i < 12; ++i) out[i] = 0.0;
  double p[6];
  for (int j = 0; j < 3; ++j) {
    p[2 * j] = (tri[2 * j] - xp[0]) / H;
    p[2 * j + 1] = (tri[2 * j + 1] - xp[1]) / H;
  }
  double area2 = (p[2] - p[0]) * (p[5] - p[1]) - (p[3] - p[1]) * (p[4] - p[0]);
  if (area2 == 0.0) return 0;
  double sg = area2 > 0 ? 1.0 : -1.0;
  quad_stats st = {0, 0};
  double scale = -orc_kernel_C(kid) / (H * H);
  for (int e = 0; e < 3; ++e) {
    int ia = e, ib = (e + 1) % 3;
    const double* A = p + 2 * ia;
    const double* B = p + 2 * ib;
    double ex = B[0] - A[0], ey = B[1] - A[1], L = hypot(ex, ey);
    if (L == 0.0) continue;
    double nLx = sg * ey, nLy = -sg * ex;        /* n_out L = sg R (B - A) */
    double q[5];
    edge2_integrals(kid, A, B, q, &st);
    double I = q[0], U1[2] = {q[1], q[2]}, Us[2] = {q[3], q[4]};
    double RI[2][2] = {{0.0, sg * I}, {-sg * I, 0.0}};
    double nL[2] = {nLx, nLy};
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 2; ++a) {
        out[4 * ib + 2 * b + a] += scale * (RI[b][a] + nL[b] * Us[a]);
        out[4 * ia + 2 * b + a] += scale * (-RI[b][a] + nL[b] * (U1[a] - Us[a]));
      }
  }
  return st.max_depth_hit ? 1 : 0;
}

int orc_pairs_grad_jacobian(int kid, double H, const double* pairs, int64_t P, double* out /*[P][12]*/) {
  if (!kernel_ok(kid) || !(H > 0.0)) return -1;
  gl_init();
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t q = 0; q < P; ++q) orc_grad_jacobian(kid, H, pairs + 8 * q, pairs + 8 * q + 2, out + 12 * q);
  return 0;
}

/* ------------------------------------------------------------------------------------ */
/* culling predicate: the operation order is part of the interface (include/sph2d.h)    */
/* ------------------------------------------------------------------------------------ */
static int cull_keep(double px, double py, const float* tf, double H2) {
  double x[3], y[3];
  for (int j = 0; j < 3; ++j) { x[j] = (double)tf[2 * j]; y[j] = (double)tf[2 * j + 1]; }
  double best = INFINITY;
  int npos = 0, nneg = 0;
  for (int e = 0; e < 3; ++e) {
    int b = (e + 1) % 3;
    double ex = x[b] - x[e], ey = y[b] - y[e];
    double wx = px - x[e], wy = py - y[e];
    double cr = wx * ey - wy * ex;
    if (cr > 0.0) ++npos;
    if (cr < 0.0) ++nneg;
    double l2 = ex * ex + ey * ey;
    double tn = wx * ex + wy * ey;
    double d2;
    if (tn <= 0.0) {
      d2 = wx * wx + wy * wy;
    } else if (tn >= l2) {
      double vx = px - x[b], vy = py - y[b];
      d2 = vx * vx + vy * vy;
    } else {
      d2 = cr * cr / l2;
    }
    if (d2 < best) best = d2;
  }
  /* inside or on the boundary: distance 0.  With every cross product 0 the particle lies on
   * the line of a zero-area triangle (a segment), whose distance decides. */
  if ((npos + nneg > 0) && (npos == 0 || nneg == 0)) return 1;
  return best < H2;
}

/* Brute force O(N M).  particles: float [N][stride] with x, y first.  Two-phase: call with
 * out_tri == NULL to get counts[N]; then with out_tri sized sum(counts) and offsets
 * computed by the caller (off[N+1]) to fill, triangles ascending within each particle. */
int orc_cull(const float* particles, int64_t N, int stride, const float* tris, int64_t M,
             double H, int64_t* counts, const int64_t* off, int32_t* out_tri) {
  if (N < 0 || M < 0 || !(H > 0.0) || stride < 2) return -1;
  double H2 = H * H;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < N; ++i) {
    double px = (double)particles[i * stride], py = (double)particles[i * stride + 1];
    int64_t c = 0;
    for (int64_t t = 0; t < M; ++t) {
      if (cull_keep(px, py, tris + 6 * t, H2)) {
        if (out_tri) out_tri[off[i] + c] = (int32_t)t;
        ++c;
      }
    }
    if (counts) counts[i] = c;
  }
  return 0;
}

/* ------------------------------------------------------------------------------------ */
/* per-particle sums over a given pair list (Eq. boundaryint), ascending triangle order  */
/* ------------------------------------------------------------------------------------ */
/* out_g[N], out_grad[N][2], out_mom[N][nm] (nm = 0 when moment_degree < 0), flags[N] */
int orc_particle_sums(int kid, double H, const float* particles, int64_t N, int stride,
                      const float* tris, const int64_t* off, const int32_t* pair_tri,
                      int moment_degree, double* out_g, double* out_grad, double* out_mom,
                      int32_t* flags) {
  if (!kernel_ok(kid) || !(H > 0.0) || moment_degree > 3) return -1;
  int nm = moment_degree < 0 ? 0 : (moment_degree + 1) * (moment_degree + 2) / 2;
  gl_init();
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < N; ++i) {
    double xp[2] = {(double)particles[i * stride], (double)particles[i * stride + 1]};
    double g = 0.0, gx = 0.0, gy = 0.0, mom[10] = {0};
    int fl = 0;
    for (int64_t q = off[i]; q < off[i + 1]; ++q) {
      const float* tf = tris + 6 * (int64_t)pair_tri[q];
      double tri[6];
      for (int j = 0; j < 6; ++j) tri[j] = (double)tf[j];
      double o[16];
      orc_pair(kid, H, xp, tri, o);
      g += o[0];
      gx += o[1];
      gy += o[2];
      for (int m = 0; m < nm; ++m) mom[m] += o[5 + m];
      if (o[15] != 0.0) fl = 1;
    }
    out_g[i] = g;
    out_grad[2 * i] = gx;
    out_grad[2 * i + 1] = gy;
    for (int m = 0; m < nm; ++m) out_mom[i * nm + m] = mom[m];
    if (flags) flags[i] = fl;
  }
  return 0;
}

/* many independent pairs (local frame or world frame), [P][8] = px py x0 y0 x1 y1 x2 y2 */
int orc_pairs(int kid, double H, const double* pairs, int64_t P, double* out /*[P][16]*/) {
  if (!kernel_ok(kid) || !(H > 0.0)) return -1;
  gl_init();
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t q = 0; q < P; ++q) orc_pair(kid, H, pairs + 8 * q, pairs + 8 * q + 2, out + 16 * q);
  return 0;
}

int orc_pairs_vertex_grad(int kid, double H, const double* pairs, int64_t P, double* out /*[P][6]*/) {
  if (!kernel_ok(kid) || !(H > 0.0)) return -1;
  gl_init();
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t q = 0; q < P; ++q) orc_vertex_grad(kid, H, pairs + 8 * q, pairs + 8 * q + 2, out + 6 * q);
  return 0;
}

/* Lagrange field of order k (1..3) on one triangle: node values A[(k+1)(k+2)/2] in the
 * node order above, the caller's vertex order.
 *   out[0] = int_T A(x') W(x - x') dx',  out[1..2] = int_T A(x') grad_x W(x - x') dx'
 * by polar quadrature of the field (evaluated from its nodal basis) times the kernel. */
int orc_pair_field_p(int kid, double H, const double* xp, const double* tri, int order, const double* A,
                     double* out) {
  if (!kernel_ok(kid) || !(H > 0.0) || order < 1 || order > 3) return -1;
  gl_init();
  out[0] = out[1] = out[2] = 0.0;
  double p[6];
  for (int j = 0; j < 3; ++j) {
    p[2 * j] = (tri[2 * j] - xp[0]) / H;
    p[2 * j + 1] = (tri[2 * j + 1] - xp[1]) / H;
  }
  tri_t t;
  if (tri_setup(p, &t) == 0) return 0;
  /* barycentric coordinates of the caller's vertices (Sec. 3), as in orc_pair_field */
  double x0 = p[0], y0 = p[1], x1 = p[2], y1 = p[3], x2 = p[4], y2 = p[5];
  double D = (y1 - y2) * (x0 - x2) + (x2 - x1) * (y0 - y2);
  nfield_ctx fc;
  fc.kid = kid;
  fc.order = order;
  fc.nn = (order + 1) * (order + 2) / 2;
  fc.t = &t;
  fc.nodes = order == 1 ? NODES_P1 : (order == 2 ? NODES_P2 : NODES_P3);
  for (int n = 0; n < fc.nn; ++n) fc.A[n] = A[n];
  fc.l0x = (y1 - y2) / D;
  fc.l0y = (x2 - x1) / D;
  fc.l0c = -(fc.l0x * x2 + fc.l0y * y2);
  fc.l1x = (y2 - y0) / D;
  fc.l1y = (x0 - x2) / D;
  fc.l1c = -(fc.l1x * x2 + fc.l1y * y2);
  quad_stats st = {0, 0};
  double q[3];
  polar_integrate(kid, &t, nfield_fn, &fc, 3, q, &st);
  double C = orc_kernel_C(kid);
  out[0] = C * q[0];
  out[1] = -(C / H) * q[1];
  out[2] = -(C / H) * q[2];
  return st.max_depth_hit ? 1 : 0;
}

/* world positions of the order-k nodes of one triangle -> xy[2 nn] */
int orc_field_nodes(const double* tri, int order, double* xy) {
  if (order < 1 || order > 3) return -1;
  const int (*nodes)[3] = order == 1 ? NODES_P1 : (order == 2 ? NODES_P2 : NODES_P3);
  int nn = (order + 1) * (order + 2) / 2;
  for (int n = 0; n < nn; ++n) {
    xy[2 * n] = xy[2 * n + 1] = 0.0;
    for (int m = 0; m < 3; ++m) {
      xy[2 * n] += tri[2 * m] * nodes[n][m] / (double)order;
      xy[2 * n + 1] += tri[2 * m + 1] * nodes[n][m] / (double)order;
    }
  }
  return 0;
}

int orc_pairs_field_p(int kid, double H, const double* pairs, int order, const double* A, int64_t P,
                      double* out) {
  if (!kernel_ok(kid) || !(H > 0.0) || order < 1 || order > 3) return -1;
  gl_init();
  const int nn = (order + 1) * (order + 2) / 2;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t q = 0; q < P; ++q) orc_pair_field_p(kid, H, pairs + 8 * q, pairs + 8 * q + 2, order, A + nn * q, out + 3 * q);
  return 0;
}

int orc_pairs_field(int kid, double H, const double* pairs, const double* A, int64_t P,
                    double* out /*[P][3]*/) {
  if (!kernel_ok(kid) || !(H > 0.0)) return -1;
  gl_init();
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t q = 0; q < P; ++q) orc_pair_field(kid, H, pairs + 8 * q, pairs + 8 * q + 2, A + 3 * q, out + 3 * q);
  return 0;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
