// Boundary pressure coupling (Appendix A): the boundary's pressure acceleration of each
// particle,
//   a_i = - int_Omega f(x') grad_x W(x_i - x') dx',   f = rho_0b (p(x')/rho_0b^2 + p_i/rho_i^2),
// with the boundary density at its rest value rho_0b and the boundary pressure p(x') from a
// moving-least-squares fit to the particles' pressures, in the appendix's two models:
//   1 (vertex pressure):  p by MLS at each triangle vertex, interpolated barycentrically;
//     a_i = -(1/rho_0b) <grad p>_i - rho_0b p_i/rho_i^2 grad gamma_i  (one fused pair pass:
//     the linear-field gradient of the vertex pressures and grad gamma from one evaluation)
//   2 (contact pressure): per pair one value p(x_iT) at the point of the triangle's boundary
//     closest to x_i;  a_i = - sum_T rho_0b (p(x_iT)/rho_0b^2 + p_i/rho_i^2) grad gamma_iT
//     (two pair passes: contact point, MLS and the pair's weight into a per-pair buffer; then
//     grad gamma_iT and the weighted segmented sum.  Fused, the MLS loops and the closed form
//     together overran the instruction cache: ncu showed 9.3 warps per issue stalled on
//     instruction fetch and the FMA pipe 25% active).
//
// MLS at a point b: the linear fit a + g . d_j, d_j = (x_j - b)/H, to the pressures p_j of the
// particles within H, weighted by w_j = V_j k(|d_j|) (the kernel's constant cancels); p(b) = a
// (solved in centred form, mls_eval).  Where the 3 x 3 normal matrix has determinant at most
// 1e-6 (sum w)^3 (fewer than three neighbours, or all on a line) the weighted average
// sum w p / sum w is used, and 0 where no particle lies within H.  Neighbours come from a particle grid
// on the culling grid's cells (side >= H), each cell's particles in ascending index, visited
// in cell order: every sum has a fixed order.
#include <cuda_runtime.h>

#include "fields_common.cuh"

namespace sph2d {

struct PGrid {
  double x0, y0, inv_cs, H;
  int nx, ny;
  const int64_t* start;      // [nx ny + 1]
  const int32_t* ids;        // [N], ascending within each cell
};

static PGrid pgrid_of(const Ctx* c) {
  PGrid g;
  g.x0 = c->cells.x0;
  g.y0 = c->cells.y0;
  g.inv_cs = 1.0 / c->cells.cs;
  g.H = c->cells.H;
  g.nx = c->cells.nx;
  g.ny = c->cells.ny;
  g.start = static_cast<const int64_t*>(c->part_start.ptr);
  g.ids = static_cast<const int32_t*>(c->part_ids.ptr);
  return g;
}

__device__ __forceinline__ int pcell_clamped(double v, int n) {
  const int i = int(floor(v));
  return i < 0 ? 0 : (i > n - 1 ? n - 1 : i);
}

__global__ void part_count_kernel(PGrid g, const float4* __restrict__ parts, int64_t N,
                                  unsigned long long* __restrict__ count) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const float4 p = parts[i];
  const int ix = pcell_clamped((double(p.x) - g.x0) * g.inv_cs, g.nx);
  const int iy = pcell_clamped((double(p.y) - g.y0) * g.inv_cs, g.ny);
  atomicAdd(count + int64_t(iy) * g.nx + ix, 1ull);
}

__global__ void part_fill_kernel(PGrid g, const float4* __restrict__ parts, int64_t N,
                                 unsigned long long* __restrict__ cursor, int32_t* __restrict__ ids) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const float4 p = parts[i];
  const int ix = pcell_clamped((double(p.x) - g.x0) * g.inv_cs, g.nx);
  const int iy = pcell_clamped((double(p.y) - g.y0) * g.inv_cs, g.ny);
  const int64_t cidx = int64_t(iy) * g.nx + ix;
  const unsigned long long k = atomicAdd(cursor + cidx, 1ull);
  ids[g.start[cidx] + int64_t(k)] = int32_t(i);
}

// the particle grid of the current build (once per build)
static sph2d_status ensure_particle_grid(Ctx* c) {
  Cells& cl = c->cells;
  if (cl.part_grid) return SPH2D_OK;
  const int64_t C = int64_t(cl.nx) * cl.ny, N = cl.N;
  sph2d_status s = ensure(c, c->part_start, size_t(C + 1) * sizeof(int64_t));
  if (s == SPH2D_OK) s = ensure(c, c->part_cursor, size_t(C > 0 ? C : 1) * sizeof(unsigned long long));
  if (s == SPH2D_OK) s = ensure(c, c->part_ids, size_t(N > 0 ? N : 1) * sizeof(int32_t));
  if (s != SPH2D_OK) return s;
  if (C > 0 && N > 0) {
    auto* cnt = static_cast<unsigned long long*>(c->part_cursor.ptr);
    cudaError_t e = cudaMemsetAsync(cnt, 0, size_t(C) * sizeof(unsigned long long), c->stream);
    if (e != cudaSuccess) return cuda_err(c, e, "memset");
    PGrid g = pgrid_of(c);
    const auto* parts = reinterpret_cast<const float4*>(cl.particles);
    SPH2D_LAUNCH(c, part_count_kernel, unsigned((N + 255) / 256), 256, g, parts, N, cnt);
    s = exclusive_scan_i64(c, reinterpret_cast<const int64_t*>(cnt), static_cast<int64_t*>(c->part_start.ptr), C);
    if (s != SPH2D_OK) return s;
    e = cudaMemsetAsync(cnt, 0, size_t(C) * sizeof(unsigned long long), c->stream);
    if (e != cudaSuccess) return cuda_err(c, e, "memset");
    SPH2D_LAUNCH(c, part_fill_kernel, unsigned((N + 255) / 256), 256, g, parts, N, cnt,
                 static_cast<int32_t*>(c->part_ids.ptr));
    s = launch_sort_segments(c, static_cast<const int64_t*>(c->part_start.ptr), static_cast<int32_t*>(c->part_ids.ptr), C);
    if (s != SPH2D_OK) return s;
  } else if (C >= 0) {
    cudaError_t e = cudaMemsetAsync(c->part_start.ptr, 0, size_t(C + 1) * sizeof(int64_t), c->stream);
    if (e != cudaSuccess) return cuda_err(c, e, "memset");
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(c, e, "particle grid");
  cl.part_grid = true;
  return SPH2D_OK;
}

// k(r) for r < 1 in factored form, precision R
template <typename R, int KID>
__device__ __forceinline__ R kernel_k(R r) {
  const R m = R(1) - r, m2 = m * m, m4 = m2 * m2;
  if (KID == KID_WC2) return m4 * (R(1) + R(4) * r);
  if (KID == KID_WC4) return m4 * m2 * (R(1) + r * (R(6) + r * (R(35) / R(3))));
  if (KID == KID_WC6) return m4 * m4 * (R(1) + r * (R(8) + r * (R(25) + R(32) * r)));
  return r < R(0.5) ? R(1) + r * r * (R(-6) + R(6) * r) : R(2) * m2 * m;
}

// MLS pressure at (bx, by) in precision R, in two passes over the neighbours: the weighted
// centroid c and mean pressure pb, then the centred second moments S = sum w (d - c)(d - c)^T and
// q = sum w (p - pb)(d - c); the fit's gradient g = S^-1 q and p(b) = pb - g . c.  The same
// least-squares solution as the 3 x 3 normal equations (det of those = s0 det S), without
// their cancellation: FP32 stays within ~3e-7 of the pressure scale where the uncentred
// solve lost 4e-4 at the fringe of the fluid.
template <typename R, int KID, bool SECOND>
__device__ __forceinline__ void mls_pass(const PGrid& g, const float4* __restrict__ parts, const float* __restrict__ vol,
                                         const float* __restrict__ pres, R bx, R by, R* acc, R cx, R cy, R pb) {
  const R ih = R(1.0 / g.H);
  const int ix = int(floor((double(bx) - g.x0) * g.inv_cs)), iy = int(floor((double(by) - g.y0) * g.inv_cs));
  // the (up to) three cells of a row are consecutive in the grid, so their particles form one
  // range of ids: cells in row order, each cell's particles ascending
  const int x_lo = ix - 1 < 0 ? 0 : ix - 1, x_hi = ix + 1 >= g.nx ? g.nx - 1 : ix + 1;
  for (int cyi = iy - 1; cyi <= iy + 1; ++cyi) {
    if (cyi < 0 || cyi >= g.ny || x_lo > x_hi) continue;
    const int64_t row = int64_t(cyi) * g.nx;
    const int64_t j0 = __ldg(g.start + row + x_lo), j1 = __ldg(g.start + row + x_hi + 1);
    for (int64_t jj = j0; jj < j1; ++jj) {
      const int j = __ldg(g.ids + jj);
      const float4 q = parts[j];
      const R dx = (R(q.x) - bx) * ih, dy = (R(q.y) - by) * ih;
      const R r2 = dx * dx + dy * dy;
      if (!(r2 < R(1))) continue;
      const R w = R(__ldg(vol + j)) * kernel_k<R, KID>(sqrt(r2));
      const R pj = R(__ldg(pres + j));
      if (!SECOND) {
        acc[0] += w;
        acc[1] += w * dx;
        acc[2] += w * dy;
        acc[3] += w * pj;
      } else {
        const R ex = dx - cx, ey = dy - cy, wq = w * (pj - pb);
        acc[0] += w * ex * ex;
        acc[1] += w * ex * ey;
        acc[2] += w * ey * ey;
        acc[3] += wq * ex;
        acc[4] += wq * ey;
      }
    }
  }
}

template <typename R, int KID>
__device__ __forceinline__ R mls_eval(const PGrid& g, const float4* __restrict__ parts, const float* __restrict__ vol,
                                      const float* __restrict__ pres, R bx, R by) {
  R m[4] = {R(0), R(0), R(0), R(0)};
  mls_pass<R, KID, false>(g, parts, vol, pres, bx, by, m, R(0), R(0), R(0));
  const R s0 = m[0];
  if (!(s0 > R(0))) return R(0);
  const R cx = m[1] / s0, cy = m[2] / s0, pb = m[3] / s0;
  R c[5] = {R(0), R(0), R(0), R(0), R(0)};
  mls_pass<R, KID, true>(g, parts, vol, pres, bx, by, c, cx, cy, pb);
  const R det = c[0] * c[2] - c[1] * c[1];
  if (det <= R(1e-6) * s0 * s0) return pb;             // singular fit: the weighted average
  const R gx = (c[3] * c[2] - c[4] * c[1]) / det, gy = (c[4] * c[0] - c[3] * c[1]) / det;
  return pb - gx * cx - gy * cy;
}

template <typename R, int KID>
__global__ void mls_points_kernel(PGrid g, const float4* __restrict__ parts, const float* __restrict__ vol,
                                  const float* __restrict__ pres, const float* __restrict__ pts, int64_t Q,
                                  R* __restrict__ out) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= Q) return;
  out[i] = mls_eval<R, KID>(g, parts, vol, pres, R(pts[2 * i]), R(pts[2 * i + 1]));
}

// model 1: pressures at the triangle vertices, in the mode's precision (double for FP64)
template <typename R, int KID>
__global__ void mls_vertices_kernel(PGrid g, const float4* __restrict__ parts, const float* __restrict__ vol,
                                    const float* __restrict__ pres, const float* __restrict__ tris, int64_t M3,
                                    R* __restrict__ out) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= M3) return;
  out[i] = mls_eval<R, KID>(g, parts, vol, pres, R(tris[2 * i]), R(tris[2 * i + 1]));
}

// point of the triangle's boundary closest to (x, y)
template <typename R>
__device__ __forceinline__ void closest_on_boundary(R x, R y, const float* t, R& cx, R& cy) {
  R bd = R(3.0e38);
  cx = R(t[0]);
  cy = R(t[1]);
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const int b = e == 2 ? 0 : e + 1;
    const R ax = R(t[2 * e]), ay = R(t[2 * e + 1]);
    const R ex = R(t[2 * b]) - ax, ey = R(t[2 * b + 1]) - ay;
    const R l2 = ex * ex + ey * ey;
    R s = l2 > R(0) ? ((x - ax) * ex + (y - ay) * ey) / l2 : R(0);
    s = s < R(0) ? R(0) : (s > R(1) ? R(1) : s);
    const R qx = ax + s * ex, qy = ay + s * ey;
    const R d2 = (x - qx) * (x - qx) + (y - qy) * (y - qy);
    if (d2 < bd) {
      bd = d2;
      cx = qx;
      cy = qy;
    }
  }
}

struct PressArgs {
  PGrid g;
  const float* vol;
  const float* pres;
  const float* rho;
  double rho0b;
  const void* wts;           // model 2: per-pair weights of contact_weight_kernel (OT [P])
};

// model 2, first pass, one thread per pair: the contact point, the MLS pressure there and the
// pair's weight rho_0b (p(x_iT)/rho_0b^2 + p_i/rho_i^2)
template <typename OT, int KID>
__global__ void __launch_bounds__(128) contact_weight_kernel(IntArgs a, PressArgs pa, OT* __restrict__ wts) {
  for (int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < a.P; q += int64_t(gridDim.x) * blockDim.x) {
    const int pid = __ldg(a.pair_pid + q);
    const int tid = __ldg(a.pair_tri + q);
    const float4 p = a.parts[pid];
    OT cx, cy;
    closest_on_boundary<OT>(OT(p.x), OT(p.y), a.tris + 6 * int64_t(tid), cx, cy);
    const OT pc = mls_eval<OT, KID>(pa.g, a.parts, pa.vol, pa.pres, cx, cy);
    const OT r = OT(__ldg(pa.rho + pid));
    const OT rb = OT(pa.rho0b);
    wts[q] = rb * (pc / (rb * rb) + OT(__ldg(pa.pres + pid)) / (r * r));
  }
}

// model 2, second pass: one warp per 32 consecutive pairs; v[0] = sum_T w_iT gamma_iT,
// v[1..2] = a_i
template <typename OT, int KID>
__global__ void __launch_bounds__(128) contact_pressure_kernel(FieldArgs f, PressArgs pa) {
  constexpr int NV = 3 * kMaxFields;
  const IntArgs& a = f.a;
  const int64_t nchunks = (a.P + 31) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  unsigned long long fixes = 0;
  for (int64_t ch = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; ch < nchunks;) {
    const unsigned long long nx = chunk_prefetch(a.work);
    const int64_t q = ch * 32 + (threadIdx.x & 31);
    int pid = -1, fix = 0;
    OT v[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = OT(0);
    if (q < a.P) {
      pid = __ldg(a.pair_pid + q);
      const int tid = __ldg(a.pair_tri + q);
      OT w[nv_of(0)];
      fix = eval_pair<OT, KID, 0>(a, pid, tid, w);
      const OT wt = static_cast<const OT*>(pa.wts)[q];
      v[0] = wt * w[0];
      v[1] = -wt * w[1];
      v[2] = -wt * w[2];
    }
    fixes += __popc(__ballot_sync(0xffffffffu, fix));
    field_warp_sum<OT>(f, ch, pid, v);
    ch = chunk_next(a.work, ch, nw, nx);
  }
  if ((threadIdx.x & 31) == 0 && fixes) atomicAdd(a.nfix, fixes);
}

// model 1, one pair: the linear vertex-pressure field's gradient term and the pair's grad gamma
// from one closed-form evaluation; v[1..2] = -(1/rho_0b) <grad p>_T - rho_0b p_i/rho_i^2 grad
// gamma_T (the field gradient as in the linear-field pass: (a/H) gamma - sum_j p_j d gamma /
// d nu_j); v[0] = <p>_T.  The vertex sum is taken relative to the first vertex's pressure:
// sum_j p_j d gamma/d nu_j = -p_0 grad gamma_T + sum_j (p_j - p_0) d gamma/d nu_j, because the
// vertex gradients of a triangle sum to -grad gamma_T (translation invariance).  The same value,
// without the cancelling sum p_0 sum_j d gamma/d nu_j (terms of size 1/H summing to grad gamma).
template <typename OT, int KID>
__device__ __forceinline__ int vertex_pressure_pair(const IntArgs& a, const PressArgs& pa, const OT* pv, int pid,
                                                    int tid, OT* v) {
  OT w[nv_of(1)];                           // gamma, grad gamma, M00, M10, M01
  int fix = eval_pair<OT, KID, 1>(a, pid, tid, w);
  OT g[6];
  const float* t = a.tris + 6 * int64_t(tid);
  const float4 p = a.parts[pid];
  fix |= vertex_grad_pair<OT, KID>(p, t, a.invH, a.C, g);
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
  const OT D = diff_of_products(e1x, e2y, e1y, e2x);
  if (D == OT(0)) {
    v[0] = v[1] = v[2] = OT(0);
    return fix;
  }
  const OT r = OT(__ldg(pa.rho + pid));
  const OT kg = OT(pa.rho0b) * OT(__ldg(pa.pres + pid)) / (r * r);
  const OT ib = OT(1.0 / pa.rho0b);
  const OT iD = OT(1) / D;
  const OT* P = pv + 3 * int64_t(tid);
  const OT a0 = __ldg(P), a1 = __ldg(P + 1), a2 = __ldg(P + 2);
  const OT d1 = a1 - a0, d2 = a2 - a0;
  const OT gx = (d1 * e2y - d2 * e1y) * iD, gy = (d2 * e1x - d1 * e2x) * iD;
  const OT ih = OT(a.invH);
  const OT fx = gx * ih * w[0] + a0 * w[1] - (d1 * g[2] + d2 * g[4]);
  const OT fy = gy * ih * w[0] + a0 * w[2] - (d1 * g[3] + d2 * g[5]);
  v[0] = a0 * w[0] + gx * (w[4] - l[0] * w[0]) + gy * (w[5] - l[1] * w[0]);
  v[1] = -ib * fx - kg * w[1];
  v[2] = -ib * fy - kg * w[2];
  return fix;
}

// model 1: one fused pair pass, segmented sums as contact_pressure_kernel
template <typename OT, int KID>
__global__ void __launch_bounds__(128) vertex_pressure_kernel(FieldArgs f, PressArgs pa, const OT* __restrict__ pv) {
  constexpr int NV = 3 * kMaxFields;
  const IntArgs& a = f.a;
  const int64_t nchunks = (a.P + 31) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  unsigned long long fixes = 0;
  for (int64_t ch = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; ch < nchunks;) {
    const unsigned long long nx = chunk_prefetch(a.work);
    const int64_t q = ch * 32 + (threadIdx.x & 31);
    int pid = -1, fix = 0;
    OT v[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = OT(0);
    if (q < a.P) {
      pid = __ldg(a.pair_pid + q);
      fix = vertex_pressure_pair<OT, KID>(a, pa, pv, pid, __ldg(a.pair_tri + q), v);
    }
    fixes += __popc(__ballot_sync(0xffffffffu, fix));
    field_warp_sum<OT>(f, ch, pid, v);
    ch = chunk_next(a.work, ch, nw, nx);
  }
  if ((threadIdx.x & 31) == 0 && fixes) atomicAdd(a.nfix, fixes);
}

template <typename R>
static sph2d_status mls_points_t(Ctx* c, int kernel, const float* vol, const float* pres, const float* pts,
                                 int64_t Q, void* out) {
  const PGrid g = pgrid_of(c);
  const auto* parts = reinterpret_cast<const float4*>(c->cells.particles);
  const unsigned b = unsigned((Q + 127) / 128);
  R* o = static_cast<R*>(out);
  switch (kernel) {
    case KID_WC2: SPH2D_LAUNCH(c, (mls_points_kernel<R, KID_WC2>), b, 128, g, parts, vol, pres, pts, Q, o); break;
    case KID_WC4: SPH2D_LAUNCH(c, (mls_points_kernel<R, KID_WC4>), b, 128, g, parts, vol, pres, pts, Q, o); break;
    case KID_WC6: SPH2D_LAUNCH(c, (mls_points_kernel<R, KID_WC6>), b, 128, g, parts, vol, pres, pts, Q, o); break;
    default: SPH2D_LAUNCH(c, (mls_points_kernel<R, KID_CUBIC>), b, 128, g, parts, vol, pres, pts, Q, o); break;
  }
  return SPH2D_OK;
}

sph2d_status launch_mls_points(Ctx* c, int kernel, int mode, const float* vol, const float* pres, const float* pts,
                               int64_t Q, void* out) {
  sph2d_status s = ensure_particle_grid(c);
  if (s != SPH2D_OK) return s;
  if (Q > 0) {
    s = mode == SPH2D_FP64 ? mls_points_t<double>(c, kernel, vol, pres, pts, Q, out)
                           : mls_points_t<float>(c, kernel, vol, pres, pts, Q, out);
    if (s != SPH2D_OK) return s;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(c, e, "mls launch");
  return SPH2D_OK;
}

template <typename R>
static sph2d_status mls_vertices_t(Ctx* c, int kernel, const float* vol, const float* pres, R* out) {
  const PGrid g = pgrid_of(c);
  const auto* parts = reinterpret_cast<const float4*>(c->cells.particles);
  const int64_t M3 = 3 * c->cells.M;
  const unsigned b = unsigned((M3 + 127) / 128);
  const float* t = c->cells.tris;
  switch (kernel) {
    case KID_WC2: SPH2D_LAUNCH(c, (mls_vertices_kernel<R, KID_WC2>), b, 128, g, parts, vol, pres, t, M3, out); break;
    case KID_WC4: SPH2D_LAUNCH(c, (mls_vertices_kernel<R, KID_WC4>), b, 128, g, parts, vol, pres, t, M3, out); break;
    case KID_WC6: SPH2D_LAUNCH(c, (mls_vertices_kernel<R, KID_WC6>), b, 128, g, parts, vol, pres, t, M3, out); break;
    default: SPH2D_LAUNCH(c, (mls_vertices_kernel<R, KID_CUBIC>), b, 128, g, parts, vol, pres, t, M3, out); break;
  }
  return SPH2D_OK;
}

template <typename OT, int KID>
static sph2d_status launch_pass(Ctx* c, int model, const FieldArgs& f, const PressArgs& pa, const OT* pv,
                                int64_t want) {
  if (model == 1) {
    SPH2D_LAUNCH(c, (vertex_pressure_kernel<OT, KID>), resident_blocks(c, vertex_pressure_kernel<OT, KID>, want), 128,
                 f, pa, pv);
  } else {
    OT* wts = static_cast<OT*>(const_cast<void*>(pa.wts));
    SPH2D_LAUNCH(c, (contact_weight_kernel<OT, KID>),
                 resident_blocks(c, contact_weight_kernel<OT, KID>, (f.a.P + 127) / 128), 128, f.a, pa, wts);
    SPH2D_LAUNCH(c, (contact_pressure_kernel<OT, KID>), resident_blocks(c, contact_pressure_kernel<OT, KID>, want), 128,
                 f, pa);
  }
  return SPH2D_OK;
}

// one fused pair pass of model 1 (pv: vertex pressures) or model 2
template <typename OT>
static sph2d_status run_pressure_pass(Ctx* c, int kernel, int model, FieldArgs f, PressArgs pa, const OT* pv) {
  constexpr int NV = 3 * kMaxFields;
  const int64_t nchunks = (f.a.P + 31) >> 5;
  sph2d_status s = ensure(c, c->slots, size_t(nchunks * 2 * NV + 1) * sizeof(OT));
  if (s != SPH2D_OK) return s;
  f.a.slots = c->slots.ptr;
  if (f.a.P > 0) {
    const int64_t want = (nchunks + 3) / 4;
    switch (kernel) {
      case KID_WC2: s = launch_pass<OT, KID_WC2>(c, model, f, pa, pv, want); break;
      case KID_WC4: s = launch_pass<OT, KID_WC4>(c, model, f, pa, pv, want); break;
      case KID_WC6: s = launch_pass<OT, KID_WC6>(c, model, f, pa, pv, want); break;
      default: s = launch_pass<OT, KID_CUBIC>(c, model, f, pa, pv, want); break;
    }
    if (s != SPH2D_OK) return s;
  }
  if (f.a.N > 0) SPH2D_LAUNCH(c, (field_finalize_kernel<OT>), unsigned((f.a.N + 255) / 256), 256, f);
  return SPH2D_OK;
}

sph2d_status launch_boundary_pressure(Ctx* c, int kernel, int mode, int model, const float* rho, const float* pres,
                                      const float* vol, double rho0b, void* accel) {
  Cells& cl = c->cells;
  sph2d_status s = ensure_particle_grid(c);
  if (s != SPH2D_OK) return s;
  const size_t osz = mode == SPH2D_FP64 ? sizeof(double) : sizeof(float);
  const int64_t N = cl.N;
  s = ensure(c, c->pres_tmp, size_t(N > 0 ? N : 1) * osz);
  if (s == SPH2D_OK) s = ensure(c, c->host_flags_dev, 64);
  if (s != SPH2D_OK) return s;
  const void* pv = nullptr;
  if (model == 1) {
    // vertex pressures in the mode's precision, three per triangle
    s = ensure(c, c->pres_vertex, size_t(3 * cl.M > 0 ? 3 * cl.M : 1) * osz);
    if (s != SPH2D_OK) return s;
    if (cl.M > 0) {
      s = mode == SPH2D_FP64 ? mls_vertices_t<double>(c, kernel, vol, pres, static_cast<double*>(c->pres_vertex.ptr))
                             : mls_vertices_t<float>(c, kernel, vol, pres, static_cast<float*>(c->pres_vertex.ptr));
      if (s != SPH2D_OK) return s;
    }
    pv = c->pres_vertex.ptr;
  }
  FieldArgs f{};
  IntArgs& a = f.a;
  a.parts = reinterpret_cast<const float4*>(cl.particles);
  a.tris = cl.tris;
  a.pair_tri = static_cast<const int32_t*>(c->pair_tri.ptr);
  a.pair_pid = static_cast<const int32_t*>(c->pair_pid.ptr);
  a.pair_off = static_cast<const int64_t*>(c->pair_off.ptr);
  a.P = cl.P;
  a.N = N;
  a.H = cl.H;
  a.invH = 1.0 / cl.H;
  a.C = kernel_C(kernel);
  a.nfix = static_cast<unsigned long long*>(c->host_flags_dev.ptr);
  a.work = a.nfix + 1;                               // chunk counter
  cudaError_t e = cudaMemsetAsync(a.nfix, 0, 2 * sizeof(unsigned long long), c->stream);
  if (e != cudaSuccess) return cuda_err(c, e, "memset");
  f.values = nullptr;
  f.nf = 1;
  f.value = c->pres_tmp.ptr;                         // per particle: model 1 <p>, model 2 sum_T w_iT gamma_iT
  f.grad = accel;
  if (model == 2) {
    s = ensure(c, c->pair_vals, size_t(cl.P > 0 ? cl.P : 1) * osz);   // per-pair weights
    if (s != SPH2D_OK) return s;
  }
  PressArgs pa{pgrid_of(c), vol, pres, rho, rho0b, model == 2 ? c->pair_vals.ptr : nullptr};
  s = mode == SPH2D_FP64 ? run_pressure_pass<double>(c, kernel, model, f, pa, static_cast<const double*>(pv))
                         : run_pressure_pass<float>(c, kernel, model, f, pa, static_cast<const float*>(pv));
  if (s != SPH2D_OK) return s;
  e = cudaMemcpyAsync(c->pinned + 8, a.nfix, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return cuda_err(c, e, "fixup count copy");
  c->stats.n_pairs = cl.P;
  c->stats.n_fallback = 0;
  c->fixup_pending = true;
  c->fallback_pending = false;
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(c, e, "boundary pressure launch");
  return SPH2D_OK;
}

}  // namespace sph2d
