/*
 * sph2d -- analytic 2-D SPH boundary integrals on one GPU (sm_103a).
 *
 * For every (particle, triangle) pair within the kernel support H this library evaluates
 * the area integrals of a compact polynomial SPH kernel, of its gradient, and of its
 * monomial moments over the triangle, and sums them per particle:
 *
 *   gamma_i      = sum_T int_T W(x_i - x', H) dx'                       (Sec. 2, Eq. boundaryint
 *                                                                         with A = 1)
 *   grad_gamma_i = d gamma_i / d x_i = sum_T int_T grad_x W(x_i - x') dx'  (Sec. 2, Eq.
 *                                                                         nablaIntegral; Sec. 3,
 *                                                                         Eq. basicdiff)
 *   M_ab,i       = sum_T int_T xi^a eta^b W dx',  (xi, eta) = (x' - x_i)/H, a+b <= 3
 *                  (the monomial integrals of Sec. 3, Eq. taus, in the normalised frame of
 *                  Sec. 2)
 *
 * with W(r, H) = C/H^2 k(r/H) (Sec. 2, Dehnen-Aly form) and one of these kernels k(q), q < 1:
 *   SPH2D_WENDLAND_C2   (1-q)^4 (1+4q)                       C = 7/pi
 *   SPH2D_WENDLAND_C4   (1-q)^6 (1+6q+35/3 q^2)              C = 9/pi   (Sec. 2 uses this kernel;
 *                                                            its printed 27/(16 pi) does not
 *                                                            satisfy int W = 1 in 2-D)
 *   SPH2D_WENDLAND_C6   (1-q)^8 (1+8q+25q^2+32q^3)           C = 78/(7 pi)
 *   SPH2D_CUBIC_SPLINE  1-6q^2+6q^3 (q<1/2), 2(1-q)^3 (q<1)  C = 40/(7 pi)
 *
 * Triangles are disjoint (Sec. 2) and may be given in either orientation; a zero-area
 * triangle contributes exactly 0.  Moments are ordered
 *   M00 M10 M01 M20 M11 M02 M30 M21 M12 M03   (nm = (deg+1)(deg+2)/2 of them).
 *
 * Conventions for every entry point
 *   - All array arguments are DEVICE pointers on the context's device unless stated; the
 *     caller owns them.  The library owns only scratch memory held in the context, which it
 *     grows on demand and frees in sph2d_destroy.
 *   - Work is enqueued on the context's stream.  Calls that size a pair list synchronise
 *     that stream once or twice to read counts back (documented per call).
 *   - Real-valued outputs are double in SPH2D_FP64 mode and float in SPH2D_FP32_FIXUP mode.
 *   - Every call returns a status; no C++ exception crosses this boundary and no device code
 *     traps.  On error, sph2d_last_error() describes it and outputs are unspecified.
 *   - Inputs: particles are float4 per particle (x, y, unused, unused), 16-byte aligned;
 *     triangles are 6 floats (x0, y0, x1, y1, x2, y2), 4-byte aligned.
 *
 * Pair culling (Sec. 2: "triangles that overlap the support radius"): pair (i, T) is kept
 * iff the closed triangle T lies at Euclidean distance < H from x_i.  The test is evaluated
 * in IEEE double from the float inputs, without fused multiply-add, in this order:
 *   for each edge e = (v_e, v_{e+1}):  ex = x_{e+1}-x_e, ey = y_{e+1}-y_e,
 *       wx = px-x_e, wy = py-y_e, cr = wx*ey - wy*ex, l2 = ex*ex + ey*ey, tn = wx*ex + wy*ey,
 *       d2 = (tn <= 0) ? wx*wx + wy*wy
 *          : (tn >= l2) ? (px-x_{e+1})^2 + (py-y_{e+1})^2 : cr*cr / l2
 *   keep = (some cr != 0 and (no cr > 0 or no cr < 0))  ||  min_e d2 < H*H
 * (the first clause is "inside"; a zero-area triangle is a segment, and a particle on its
 * line, where every cr is 0, is decided by the distance alone).
 * Pair lists are particle-major in input particle order, ascending triangle id within a
 * particle.
 */
#ifndef SPH2D_H
#define SPH2D_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SPH2D_OK = 0,
  SPH2D_ERR_INVALID_ARG = 1,      /* null pointer, bad size, H <= 0 or not finite, bad enum */
  SPH2D_ERR_NONFINITE_INPUT = 2,  /* a particle or vertex coordinate is NaN or infinite */
  SPH2D_ERR_CAPACITY = 3,         /* caller buffer too small; *required holds the size */
  SPH2D_ERR_NOT_BUILT = 4,        /* no pair list in the context yet */
  SPH2D_ERR_CUDA = 5,             /* a CUDA runtime call failed (message in last_error) */
  SPH2D_ERR_UNSUPPORTED = 6,      /* valid request that this build does not provide */
  SPH2D_ERR_OUT_OF_MEMORY = 7     /* scratch allocation failed */
} sph2d_status;

typedef enum {
  SPH2D_WENDLAND_C2 = 0,
  SPH2D_WENDLAND_C4 = 1,
  SPH2D_WENDLAND_C6 = 2,
  SPH2D_CUBIC_SPLINE = 3
} sph2d_kernel;

typedef enum {
  SPH2D_FP64 = 0,        /* every step in IEEE double */
  SPH2D_FP32_FIXUP = 1,  /* FP32 arithmetic; pairs whose error bound exceeds the budget are
                            recomputed in FP64 (count reported by sph2d_last_stats) */
  SPH2D_SURROGATE = 2,   /* learned surrogate with guarded analytic fallback (gamma, grad only) */
  SPH2D_FP32_HYBRID = 3  /* FP32 with quadrature for triangles away from the particle (below) */
} sph2d_mode;

typedef struct sph2d_ctx sph2d_ctx;

/* SPH2D_FP32_HYBRID (the extension Sec. 6.1 suggests): a pair whose triangle lies at least
 * half its longest edge away from the particle, and either inside the support (every vertex
 * within H) or across its edge with one vertex inside and a longest edge below a per-kernel
 * size (Wendland C2 0.6 H, C4 0.75 H, C6 0.7 H, cubic spline 0.45 H), is integrated in FP32
 * by a 36-point conical-product Gauss-Legendre rule whose rays stop at the support circle
 * (measured error <= 1.5e-6 of the output scales per pair for every output, moments
 * included, against 1e-5 for SPH2D_FP32_FIXUP).  The cubic spline's second piece (support
 * H/2) joins the quadrature for a triangle inside H/2 and is zero for one at least H/2 away;
 * for a triangle in between with a vertex inside H/2 and a longest edge below 0.45 H, a
 * 60-point rule of the same form integrates it in the doubled frame, where its support is the
 * unit circle (measured <= 7.8e-7).  Every other pair takes the SPH2D_FP32_FIXUP closed form.
 * Float outputs; n_fallback counts the pairs left to the closed form.  Per-particle paths only
 * (sph2d_pair_integrals, the adjoint and the piecewise-linear sph2d_field_integrals return
 * UNSUPPORTED; sph2d_field_integrals_p has its own hybrid form, below). */

/* Statistics of the most recent integral call on a context. */
typedef struct {
  int64_t n_particles;
  int64_t n_triangles;
  int64_t n_pairs;          /* culled pairs evaluated */
  int64_t n_fixup;          /* pairs recomputed in FP64 (SPH2D_FP32_FIXUP) */
  int64_t n_fallback;       /* pairs routed to the closed form (SPH2D_SURROGATE, SPH2D_FP32_HYBRID) */
  int64_t n_cells;          /* cells of the culling grid */
  int64_t n_candidates;     /* (triangle, cell) incidences of the culling grid */
  int64_t n_launches;       /* kernels this context has launched since sph2d_init (cumulative) */
  /* SPH2D_SURROGATE serving audit (see sph2d_surrogate_set_audit) of the last surrogate call: */
  int64_t n_audit;          /* accepted pairs also evaluated by the analytic path */
  int64_t n_audit_over;     /* audited pairs whose network error exceeded the bound */
  double audit_max_err;     /* largest audited network error, in units of the output scales */
  int64_t n_redo;           /* pairs re-evaluated analytically because the audit failed (0 or all) */
  int64_t n_mma_timeouts;   /* tcgen05 serving: MMA completion waits that ran out (their pairs fell back) */
} sph2d_stats;

/* Create a context on CUDA device `device`; `stream` is a cudaStream_t (NULL = legacy
 * default stream).  *ctx receives the handle.  Errors: INVALID_ARG, CUDA. */
sph2d_status sph2d_init(sph2d_ctx** ctx, int device, void* stream);

/* Free the context and its scratch (synchronises its stream first).  NULL is a no-op. */
sph2d_status sph2d_destroy(sph2d_ctx* ctx);

/* Change the stream later calls enqueue on (a cudaStream_t). */
sph2d_status sph2d_set_stream(sph2d_ctx* ctx, void* stream);

/* Message for the last failed call on ctx (static storage inside ctx; "" if none). */
const char* sph2d_last_error(const sph2d_ctx* ctx);

/* Copy the statistics of the last integral call into *out (host pointer).  Synchronises the
 * context's stream when the last call's fix-up count is still in flight. */
sph2d_status sph2d_last_stats(const sph2d_ctx* ctx, sph2d_stats* out);

/* Library version, e.g. 100 for 1.0.0. */
int sph2d_version(void);

/*
 * Build the culling grid and the pair list for (particles, triangles, H) and keep them in
 * the context (Sec. 2: the neighbouring triangles N_T of each particle).
 *   particles  device float4 [N]     (x, y, _, _)
 *   tris       device float  [M][6]
 *   H          support radius (> 0, finite), in the same units as the coordinates
 * The grid covers the particles' bounding box with square cells of side >= H; each
 * triangle is binned into every cell its H-expanded bounding box touches, and each
 * particle tests the triangles of its own cell with the exact predicate above.
 * Synchronises the stream three times (bounds, grid size, pair count).
 * Errors: INVALID_ARG, NONFINITE_INPUT, OUT_OF_MEMORY, CUDA.
 */
sph2d_status sph2d_build_cells(sph2d_ctx* ctx, const float* particles, int64_t N,
                               const float* tris, int64_t M, double H);

/* Number of pairs in the context's current pair list (host pointer out).  NOT_BUILT if none. */
sph2d_status sph2d_pair_count(const sph2d_ctx* ctx, int64_t* n_pairs);

/*
 * Copy the current pair list into caller device buffers: off int64 [N+1] (CSR offsets in
 * input particle order), tri int32 [cap] (triangle ids, ascending within a particle).
 * If cap < number of pairs, returns CAPACITY and writes the number to *required (host).
 */
sph2d_status sph2d_pair_list(sph2d_ctx* ctx, int64_t* off, int32_t* tri, int64_t cap,
                             int64_t* required);

/*
 * Full hot path: build cells and pair list (as sph2d_build_cells), then evaluate every
 * pair's integrals in closed form and sum them per particle (Sec. 4-5 decomposition,
 * realised as the exact edge/sector fan form described in the implementation).
 *   kernel         sph2d_kernel
 *   moment_degree  -1 (no moments) or 0..3
 *   mode           SPH2D_FP64, SPH2D_FP32_FIXUP, SPH2D_FP32_HYBRID, or SPH2D_SURROGATE (needs
 *                  moment_degree = -1 and the kernel the surrogate was initialised for;
 *                  float outputs; see the surrogate section below)
 *   gamma          device real [N]
 *   grad_gamma     device real [N][2]          (may be NULL)
 *   moments        device real [N][nm]         (NULL iff moment_degree < 0)
 * "real" is double for SPH2D_FP64 and float otherwise.  Particles with no pair
 * get zeros.  Synchronises as sph2d_build_cells does.
 * Errors: INVALID_ARG, NONFINITE_INPUT, OUT_OF_MEMORY, UNSUPPORTED, NOT_BUILT (surrogate
 * mode before sph2d_surrogate_init), CUDA.
 */
sph2d_status sph2d_boundary_integrals(sph2d_ctx* ctx, const float* particles, int64_t N,
                                      const float* tris, int64_t M, int kernel, double H,
                                      int moment_degree, int mode, void* gamma,
                                      void* grad_gamma, void* moments);

/*
 * Integrals over the pair list already in the context (built by sph2d_build_cells or by a
 * previous sph2d_boundary_integrals on the same inputs), so that several kernels or modes
 * can reuse one culling pass.  The particle and triangle arrays of that build must still
 * hold the same data.  Does not synchronise.  Arguments as sph2d_boundary_integrals.
 * Errors: NOT_BUILT, INVALID_ARG, UNSUPPORTED, CUDA.
 */
sph2d_status sph2d_integrals_from_pairs(sph2d_ctx* ctx, int kernel, int moment_degree,
                                        int mode, void* gamma, void* grad_gamma,
                                        void* moments);

/*
 * Independent pairs, no culling and no per-particle sum (precision studies, surrogate
 * training labels).
 *   pairs   device double [P][8] = (px, py, x0, y0, x1, y1, x2, y2); world units, H > 0
 *   out     device real [P][3+nm] = (gamma, dgamma/dpx, dgamma/dpy, M00..)
 * In SPH2D_FP32_FIXUP mode the local-frame geometry (v - p)/H is formed in double and
 * rounded once to float; outputs are float.  Does not synchronise.
 * Errors: INVALID_ARG, UNSUPPORTED, CUDA.
 */
sph2d_status sph2d_pair_integrals(sph2d_ctx* ctx, const double* pairs, int64_t P, int kernel,
                                  double H, int moment_degree, int mode, void* out);

/*
 * Adjoint of sph2d_boundary_integrals for a loss L(gamma, grad gamma): given dL/dgamma and
 * optionally dL/dgrad gamma, returns
 *   d_particles [N][2] = dL/dx_i  = dL/dgamma_i grad gamma_i           (Sec. 3, Eq. basicdiff)
 *                                  + (d grad gamma_i / d x_i)^T dL/dgrad gamma_i
 *   d_tris      [M][6] = dL/dnu_j = sum_i dL/dgamma_i d gamma_i / d nu_j
 *                                  + (d grad gamma_i / d nu_j)^T dL/dgrad gamma_i
 * where d gamma_i/d nu_j is the transport-theorem edge integral of W weighted by the vertex's
 * hat function, and d grad gamma / d nu_j the derivative of the divergence-theorem boundary
 * form grad gamma = -oint W n ds edge by edge (closed-form square-root integrals of k'(r)/r and
 * k'(r) r, and k at the clipped edge ends); d grad gamma_i / d x_i = -sum_j d grad gamma_i /
 * d nu_j.  None of these is printed in the paper: they are derivatives of its integrals.
 * The pair list is rebuilt from the inputs; per-pair geometry is recomputed, nothing is stored
 * from the forward call.  Vertex gradients are reduced triangle-major and the second-order
 * particle terms particle-major, both in fixed orders (deterministic).
 *   d_gamma       device real [N]
 *   d_grad_gamma  device real [N][2], or NULL for a loss of gamma alone
 * Errors: INVALID_ARG, NONFINITE_INPUT, OUT_OF_MEMORY, UNSUPPORTED (surrogate mode; more than
 * 2^31 - 1 pairs), CUDA.
 */
sph2d_status sph2d_boundary_integrals_backward(sph2d_ctx* ctx, const float* particles,
                                               int64_t N, const float* tris, int64_t M,
                                               int kernel, double H, int mode,
                                               const void* d_gamma, const void* d_grad_gamma,
                                               void* d_particles, void* d_tris);

/*
 * sph2d_boundary_integrals_backward over the pair list of the context's last build
 * (sph2d_build_cells, sph2d_boundary_integrals or a backward call), without rebuilding it: a
 * training loop's backward after its forward call skips the cull.  The particle and triangle
 * arrays of that build must still hold the same data (as for sph2d_integrals_from_pairs).
 * d_gamma [N], d_grad_gamma [N][2] or NULL, d_particles [N][2], d_tris [M][6] as in
 * sph2d_boundary_integrals_backward, with N and M of the last build; results are identical to
 * that call's on the same inputs.  Does not synchronise.
 * Errors: NOT_BUILT, INVALID_ARG, UNSUPPORTED (surrogate and hybrid modes; more than
 * 2^31 - 1 pairs), OUT_OF_MEMORY, CUDA.
 */
sph2d_status sph2d_backward_from_pairs(sph2d_ctx* ctx, int kernel, int mode, const void* d_gamma,
                                       const void* d_grad_gamma, void* d_particles, void* d_tris);

/*
 * Allocation-free integrals over a caller-supplied pair list (gamma and grad gamma).
 * The paper has no counterpart: this serves callers that cannot allocate device memory while
 * they run -- memory pools that forbid cudaMalloc inside a solver step, frameworks that own
 * all device memory, code that must not risk an allocation's implicit synchronisation or
 * failure.  It takes no context (creating one allocates) and calls no cudaMalloc, cudaFree or
 * allocating library routine.  Its only scratch is a file-scope device array of
 * SPH2D_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until process exit.
 *   particles   device float4 [N]; tris device float [M][6]
 *   pair_off    device int64 [N+1], pair_tri device int32 [P]: the pair list of
 *               sph2d_pair_list (particle-major CSR, P = pair_off[N])
 *   kernel, H, mode as sph2d_boundary_integrals (SPH2D_FP64 or SPH2D_FP32_FIXUP)
 *   gamma       device real [N];  grad_gamma device real [N][2] or NULL
 *   stream      cudaStream_t (NULL = legacy default stream); runs on the current device
 * Limit: P <= 32 * floor((SPH2D_NOALLOC_SCRATCH_BYTES - 256) / (6 * sizeof(real))), i.e.
 * 5,592,224 pairs in SPH2D_FP64 and 11,184,448 in SPH2D_FP32_FIXUP; larger lists return
 * SPH2D_ERR_CAPACITY before any work is enqueued.
 * All calls share the array: calls that overlap on the GPU (other streams or host threads at
 * the same time) race.  The first call on a device resolves the array's address with that
 * device current; make it before any stream capture.
 * Errors (status only, there is no context for a message): INVALID_ARG, CAPACITY, CUDA.
 */
#define SPH2D_NOALLOC_SCRATCH_BYTES (8u << 20)
sph2d_status sph2d_pair_list_integrals_noalloc(const float* particles, int64_t N,
                                               const float* tris, int64_t M,
                                               const int64_t* pair_off, const int32_t* pair_tri,
                                               int64_t P, int kernel, double H, int mode,
                                               void* gamma, void* grad_gamma, void* stream);

/*
 * Piecewise-linear boundary fields (Sec. 3, Eq. taus and basicdiff) over the pair list in the
 * context (sph2d_build_cells first; the particle and triangle arrays of that build must still
 * hold the same data).  Each triangle carries per-vertex values A_j of nf fields, interpolated
 * barycentrically (linear on the triangle); for every particle and field
 *   value[i][f]   = sum_T int_T A_T(x') W(x_i - x', H) dx'
 *   grad[i][f][:] = sum_T int_T A_T(x') grad_x W(x_i - x', H) dx'     (d value / d x_i)
 * Per pair the value is A_T's constant part times gamma plus its gradient dotted with the first
 * moments; the gradient is the constant-gradient area term minus the boundary term
 * sum_j A_j d gamma / d nu_j (integration by parts; the edge integrals are those of
 * sph2d_boundary_integrals_backward).  Difference and symmetric gradient forms and divergence
 * or curl are linear in the per-vertex values: evaluate fields such as rho A and rho and
 * combine per particle.
 *   vertex_values  device float [M][3][nf] (triangle, vertex in input order, field)
 *   nf             1..SPH2D_MAX_FIELDS
 *   value          device real [N][nf]; grad device real [N][nf][2] or NULL (then the
 *                  vertex-gradient work is skipped)
 *   mode           SPH2D_FP64 (double outputs) or SPH2D_FP32_FIXUP (float outputs)
 * Does not synchronise.  Errors: NOT_BUILT, INVALID_ARG, UNSUPPORTED, OUT_OF_MEMORY, CUDA.
 */
#define SPH2D_MAX_FIELDS 4
sph2d_status sph2d_field_integrals(sph2d_ctx* ctx, int kernel, int mode, const float* vertex_values,
                                   int nf, void* value, void* grad);

/*
 * Lagrange boundary fields of order 2 or 3 (the higher-order element fields the paper's
 * introduction names as the extension of Sec. 3's linear interpolation).  Each triangle carries
 * nodes_of(order) = (order+1)(order+2)/2 node values per field on the principal lattice
 * {(i, j, l)/order : i + j + l = order} in barycentric coordinates, in this order: the three
 * vertices (input order); then the nodes inside edge (0,1), edge (1,2), edge (2,0), each edge
 * from its first vertex to its second (order 2: the midpoints; order 3: the points at 1/3 and
 * 2/3); then, for order 3, the centroid.  The field is the unique polynomial of that degree
 * through the nodes; value and grad as for sph2d_field_integrals.
 *   node_values  device float [M][nodes_of(order)][nf]
 *   order        2 or 3 (order 1 is sph2d_field_integrals)
 *   mode         SPH2D_FP64: closed form (moments to degree 3 and the boundary term's edge
 *                integrals of k(rho) t^m, m <= 3) for every pair, double outputs.  Its rounding
 *                error grows like (distance / element size)^order: ~1e-11 of the field scale
 *                for elements of H/3.
 *                SPH2D_FP32_HYBRID: the hybrid mode's quadrature in FP32 (the field evaluated
 *                from its nodes at every quadrature point) for pairs that qualify, the FP64
 *                closed form for the rest; float outputs; n_fallback in sph2d_last_stats
 *                counts the closed-form pairs.
 *                SPH2D_FP32_FIXUP: UNSUPPORTED (the closed form in FP32 loses up to
 *                (distance / size)^order digits of the field scale).
 * Does not synchronise.  Errors: NOT_BUILT, INVALID_ARG, UNSUPPORTED, OUT_OF_MEMORY, CUDA.
 */
sph2d_status sph2d_field_integrals_p(sph2d_ctx* ctx, int kernel, int mode, int order, const float* node_values,
                                     int nf, void* value, void* grad);

/*
 * ---- Boundary pressure coupling (Appendix A) ---------------------------------------------
 * Uses the particles and triangles of the context's build (sph2d_build_cells); the particles
 * double as the fluid whose pressures are extrapolated.  Per-particle inputs are device float
 * [N]: density rho_i, pressure p_i, volume V_i = m_i / rho_i.
 *
 * sph2d_mls_pressure: moving-least-squares pressure at Q points (device float [Q][2]) -> out
 * (device real [Q]: double for SPH2D_FP64, float for SPH2D_FP32_FIXUP).  At a point b the
 * linear fit a + g . (x_j - b)/H to the pressures of the particles within H, weighted by
 * V_j k(|x_j - b|/H), gives p(b) = a; where the fit's 3 x 3 normal matrix has determinant
 * <= 1e-6 (sum w)^3 (fewer than three neighbours, or collinear) the weighted average
 * sum w p / sum w; 0 where no particle lies within H.  (The appendix cites Band et al.'s MLS
 * pressure extrapolation without a formula; this is the reading used.)
 *
 * sph2d_boundary_pressure: the boundary's pressure acceleration (device real [N][2])
 *   a_i = - int_Omega rho_0b (p(x')/rho_0b^2 + p_i/rho_i^2) grad_x W(x_i - x') dx'
 * with the boundary density at rho_0b > 0 and p(x') by
 *   model 1: MLS at each triangle vertex (stored as float), interpolated barycentrically:
 *            a_i = -(1/rho_0b) <grad p>_i - rho_0b p_i/rho_i^2 grad gamma_i
 *   model 2: MLS at the point of each culled triangle's boundary closest to x_i, constant on
 *            that triangle for that particle:
 *            a_i = - sum_T rho_0b (p(x_iT)/rho_0b^2 + p_i/rho_i^2) grad gamma_iT
 * Modes SPH2D_FP64 and SPH2D_FP32_FIXUP (the integrals as in sph2d_boundary_integrals; MLS in
 * the mode's precision).  Does not synchronise.  Errors: NOT_BUILT, INVALID_ARG, UNSUPPORTED,
 * OUT_OF_MEMORY, CUDA.
 */
sph2d_status sph2d_mls_pressure(sph2d_ctx* ctx, int kernel, int mode, const float* volume, const float* pressure,
                                const float* points, int64_t Q, void* out);
sph2d_status sph2d_boundary_pressure(sph2d_ctx* ctx, int kernel, int mode, int model, const float* density,
                                     const float* pressure, const float* volume, double rho0_b, void* accel);

/*
 * ---- Learned surrogate -------------------------------------------------------------------
 * The paper has no counterpart: a small network that replaces the closed form for pairs
 * inside a trained domain, evaluated on tensor cores (FP16 operands, FP32 accumulation; the
 * training backward pass uses BF16 operands); every other pair takes the analytic path
 * (SPH2D_FP32_FIXUP arithmetic).  Outputs are gamma and grad
 * gamma only, always float.
 *
 * Canonical frame (H = 1): the pair's triangle, relative to the particle, is rotated so that
 * its centroid lies on +x, reflected y -> -y if it is then clockwise, and its vertices are
 * listed from the one closest to the particle.  Network: 6 canonical coordinates -> 64 -> 64
 * -> 64 -> 3 (tanh-form GELU between layers), predicting gamma / area and the canonical
 * local-frame gradient / area; outputs are multiplied by the exact area and mapped back by
 * the inverse reflection and rotation (gamma is invariant under both).
 * Guard (the network is used only if all hold, else the pair falls back): largest edge in
 * [SPH2D_SURROGATE_MIN_SIZE, SPH2D_SURROGATE_MAX_SIZE] H, smallest angle >= 15 degrees,
 * centroid >= SPH2D_SURROGATE_MIN_CENTROID H from the particle, every vertex within
 * SPH2D_SURROGATE_MAX_RADIUS H, non-zero finite area.  The guard is evaluated in FP32 on the
 * FP32 local frame.
 * Parameters: SPH2D_SURROGATE_PARAMS FP32 values in the order W1[64][6] b1[64] W2[64][64]
 * b2[64] W3[64][64] b3[64] W4[3][64] b4[3] (W[out][in], row-major); forward tensor-core
 * operands are their FP16 roundings, and the GELU is evaluated in packed FP16 arithmetic.
 */
#define SPH2D_SURROGATE_PARAMS 8963
#define SPH2D_SURROGATE_MIN_SIZE 0.1
#define SPH2D_SURROGATE_MAX_SIZE 0.45
#define SPH2D_SURROGATE_MIN_CENTROID 0.3
#define SPH2D_SURROGATE_MAX_RADIUS 1.5

/* (Re)initialise the surrogate for `kernel`: Glorot-uniform weights from `seed` (64-bit
 * Mersenne twister, mt19937_64), zero biases and optimiser state.  Synchronises.
 * Errors: INVALID_ARG, OUT_OF_MEMORY, CUDA. */
sph2d_status sph2d_surrogate_init(sph2d_ctx* ctx, int kernel, uint64_t seed);

/*
 * Train on independent pairs (device double [P][8], as sph2d_pair_integrals, support H):
 * labels are the FP64 analytic integrals; pairs outside the guard are dropped.  Loss: mean
 * over a batch of sum_c w_c (y_c - t_c)^2 with w = (1/C^2, 1/(4C^2), 1/(4C^2)); AdamW
 * (beta 0.9, 0.999, eps 1e-8, decoupled weight decay `weight_decay`) with a learning rate
 * rising from lr/10 to lr over the first 5% of the steps, then a cosine decay to lr/100.
 * Each epoch visits floor(used / batch) batches in an order shuffled from `seed`.  The run
 * is deterministic.  *final_loss (host, may be NULL) = loss of the last batch; *n_used (host,
 * may be NULL) = pairs inside the guard.  Synchronises once per epoch.
 * Errors: NOT_BUILT (no sph2d_surrogate_init), INVALID_ARG (bad sizes, fewer usable pairs
 * than one batch), OUT_OF_MEMORY, CUDA.
 */
sph2d_status sph2d_surrogate_train(sph2d_ctx* ctx, const double* pairs, int64_t P, double H,
                                   int epochs, int batch, double lr, double weight_decay,
                                   uint64_t seed, double* final_loss, int64_t* n_used);

/*
 * Independent pairs through the surrogate: out device float [P][3] = (gamma, dgamma/dpx,
 * dgamma/dpy) in world units; accepted device int32 [P] (may be NULL) = 1 where the network
 * was used.  sph2d_last_stats reports n_fallback.  Does not synchronise.
 * Errors: NOT_BUILT, INVALID_ARG, OUT_OF_MEMORY, CUDA.
 */
sph2d_status sph2d_surrogate_pairs(sph2d_ctx* ctx, const double* pairs, int64_t P, double H,
                                   float* out, int32_t* accepted);

/*
 * The network alone: canonical inputs x device float [B][6] -> raw outputs y device float
 * [B][3] (gamma/area, canonical gradient/area), no guard.  Does not synchronise.
 * Errors: NOT_BUILT, INVALID_ARG, CUDA.
 */
sph2d_status sph2d_surrogate_forward(sph2d_ctx* ctx, const float* x, int64_t B, float* y);

/*
 * Loss and parameter gradient of one batch (the training step without the update):
 * x device float [B][6], t device float [B][3] -> grad device float [SPH2D_SURROGATE_PARAMS],
 * loss device float [1].  Does not synchronise.  Errors: NOT_BUILT, INVALID_ARG, CUDA.
 */
sph2d_status sph2d_surrogate_grad(sph2d_ctx* ctx, const float* x, const float* t, int64_t B,
                                  float* grad, float* loss);

/*
 * Serving-time audit of the network by the analytic path (sph2d_surrogate_pairs and the
 * SPH2D_SURROGATE mode).  Of the pairs the guard accepts, those whose index hashes into one of
 * `period` buckets (about 1 in `period`) are also evaluated by the analytic FP32 path, which
 * judges the network: the pair's error is the largest over gamma and grad gamma of
 * |network - analytic| / max(|analytic|, S), S = 1 for gamma and 2 C int_0^1 k(q) dq / H for
 * the gradient, and the pair returns its analytic value.  If any audited pair's error exceeds
 * `tol`, the network is not trusted for the call: every pair of the call is re-evaluated by the
 * analytic path (accepted[] reports 0 for all, n_redo = the pair count).  sph2d_last_stats
 * reports n_audit, n_audit_over, audit_max_err and n_redo.  period: 0 (off) or a power of two
 * in [1, 65536]; tol > 0 and finite.  Default for a new context: period 64, tol 1e-3.
 * Errors: INVALID_ARG.
 */
sph2d_status sph2d_surrogate_set_audit(sph2d_ctx* ctx, int period, double tol);

/*
 * Tensor-core engine of the serving network (sph2d_surrogate_pairs, SPH2D_SURROGATE mode):
 * 0 (default) mma.sync m16n8k16, one warp per 32 pairs with the activations chained in
 * registers; 1 tcgen05 (fifth-generation tensor cores), one CTA per 128 pairs with the
 * accumulators in tensor memory and the activations staged in shared memory between layers.
 * Both evaluate the same FP16-operand network with FP32 accumulation; results agree to FP32
 * accumulation order.  A tcgen05 MMA whose completion wait runs out of its poll budget sends the
 * CTA's remaining pairs to the analytic fallback (n_mma_timeouts in sph2d_last_stats).
 * Errors: INVALID_ARG.
 */
sph2d_status sph2d_surrogate_set_engine(sph2d_ctx* ctx, int engine);

/*
 * Tensor-core engine of the training GEMMs (sph2d_surrogate_train, sph2d_surrogate_grad):
 * 0 (default) mma.sync m16n8k16 in 64 x 64 block tiles; 1 tcgen05 in 128 x 64 tiles with the
 * FP32 accumulators in tensor memory.  Both round the same FP32 operands to FP16 (forward) or
 * BF16 (backward) and accumulate in FP32, with the same split of long K sums; results agree to
 * FP32 accumulation order.  With engine 1, sph2d_surrogate_train returns CUDA if an MMA
 * completion wait ran out of its poll budget.  Errors: INVALID_ARG.
 */
sph2d_status sph2d_surrogate_set_train_engine(sph2d_ctx* ctx, int engine);

/* Copy the FP32 parameters to / from host memory (n = SPH2D_SURROGATE_PARAMS).  get returns
 * CAPACITY if cap is smaller.  Synchronise.  Errors: NOT_BUILT, INVALID_ARG, CAPACITY, CUDA. */
sph2d_status sph2d_surrogate_get_params(sph2d_ctx* ctx, float* host, int64_t cap);
sph2d_status sph2d_surrogate_set_params(sph2d_ctx* ctx, const float* host, int64_t n);

/*
 * Checkpoint: a versioned binary file (magic "SPH2DSUR", version 1, kernel, layer sizes,
 * parameter count, optimiser step, FNV-1a 64 checksum) followed by the FP32 parameters and
 * both Adam moment vectors, so that training resumes exactly.  load checks every header
 * field, the length and the checksum before it touches the context.  Synchronise.
 * Errors: NOT_BUILT (save), INVALID_ARG (unreadable or incompatible file), CUDA.
 */
sph2d_status sph2d_surrogate_save(sph2d_ctx* ctx, const char* path);
sph2d_status sph2d_surrogate_load(sph2d_ctx* ctx, const char* path);

/*
 * Measurement aid (the paper has no counterpart): FMA throughput of device `device` in
 * TFLOP/s (2 flops per fma), FP64 (precision 0) or FP32 (precision 1), from eight independent
 * fma chains per thread over an occupancy-sized grid, timed with CUDA events on a launch of
 * about `seconds` (0 < seconds <= 10) after a calibration launch; best of three.  Allocates and
 * frees its own small output buffer and synchronises the device.  The benchmark reports the
 * pair kernels' FP32 and FP64 arithmetic against these measured peaks.
 * Errors: INVALID_ARG, OUT_OF_MEMORY, CUDA.
 */
sph2d_status sph2d_measure_fma_peak(int device, int precision, double seconds, double* tflops);

#ifdef __cplusplus
}
#endif

#endif /* SPH2D_H */
