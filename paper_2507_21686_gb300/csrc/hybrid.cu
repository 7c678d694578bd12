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
// on a triangle inside r < 1/2 (taken with the first) and zero on one at least 1/2 away; on a
// triangle in between whose innermost vertex lies inside r < 1/2 and whose longest edge is
// below 0.45 H, a finer rule (10 rays of 6 nodes) takes it in the doubled frame, where its
// support is the unit disk (add_second_piece); other such pairs take the closed form.  On the
// box benchmark this covers 92% of the pairs at a fifth of the closed form's arithmetic.
//
// Launch structure: the pair list is partitioned (stable, in pair order within each region)
// into region 0, the pairs left to the closed form (FP32 + FP64 fix-up); region 1, the cubic
// spline's near pairs whose second piece the finer rule takes in the doubled frame; region 2,
// the other quadrature pairs.  A class pass stores each pair's region, apex and inner flag; a
// scan and the partition pass order the pairs; two chunk kernels evaluate the positions, the
// closed form over the leading chunks and the quadrature over the rest, summing per (particle,
// region); the finalize adds the region sums in region order (deterministic).
#include <cuda_runtime.h>

#include <cmath>

#include "integrals_impl.cuh"
#include "quad.cuh"

namespace sph2d {

// quadrature of one pair -> v (gamma, grad, moments), world-scaled like eval_local.
// Conical product with the apex at vertex `apex`: p = v0 + s d(t), d(t) = (v1 - v0) + t (v2 - v1),
// Jacobian s |(v1 - v0) x (v2 - v0)|; rays t from the rule rt, s from the 6-node rule qs; along
// each ray s runs to min(1, s+), s+ the exit from the unit disk (|v0| < 1), taken as
// -c / (b + sqrt(b^2 - a c)) with a = |d|^2, b = v0 . d, c = |v0|^2 - 1 (no cancellation:
// b + sqrt(.) > 0 whenever c < 0).
template <int KID, int MD, class RT>
__device__ __forceinline__ void quad_pair(const RT& rt, const QuadRule& qs, const float* vin, int apex, bool inner,
                                          double C, double invH, float* out) {
  const int i0 = apex, i1 = i0 == 2 ? 0 : i0 + 1, i2 = i1 == 2 ? 0 : i1 + 1;
  const float v0x = vin[2 * i0], v0y = vin[2 * i0 + 1];
  const float e1x = vin[2 * i1] - v0x, e1y = vin[2 * i1 + 1] - v0y;
  const float e2x = vin[2 * i2] - vin[2 * i1], e2y = vin[2 * i2 + 1] - vin[2 * i1 + 1];
  const float a2 = fabsf(diff_of_products(e1x, vin[2 * i2 + 1] - v0y, e1y, vin[2 * i2] - v0x));
  const float c0 = v0x * v0x + v0y * v0y - 1.0f;
  float g = 0.0f, gx = 0.0f, gy = 0.0f;
  float m[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll 2
  for (int j = 0; j < RT::N; ++j) {
    const float dx = e1x + rt.u[j] * e2x, dy = e1y + rt.u[j] * e2y;
    const float aa = dx * dx + dy * dy, bb = v0x * dx + v0y * dy;
    const float sp = div_fast(-c0, bb + sqrtf(fmaxf(bb * bb - aa * c0, 0.0f)));
    const float ss = fminf(1.0f, sp);
    const float wj = rt.w[j] * ss * ss;
#pragma unroll
    for (int i = 0; i < kQuadN; ++i) {
      const float s = ss * qs.u[i];
      const float px = v0x + s * dx, py = v0y + s * dy;
      const float r = sqrt_fast(px * px + py * py);      // > 0: the particle is off the triangle
      float k, kd;
      kernel_and_slope<KID>(r, inner, k, kd);
      const float w = wj * qs.wu[i];
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

// region of each pair (0 closed form, 1 cubic near pair with its second piece by the finer
// rule, 2 quadrature) into the partition masks; class byte: apex | inner << 2
template <int KID>
__global__ void __launch_bounds__(128) hybrid_class_kernel(IntArgs a, PairSplit sp, uint32_t* __restrict__ mask,
                                                           int64_t* __restrict__ cnt, uint8_t* __restrict__ cls) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  const float ih = float(a.invH);
  for (int64_t ch = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; ch < sp.nchunks; ch += nw) {
    const int64_t q = ch * 32 + lane;
    int region = -1;
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
      region = !qc.quad ? 0 : (qc.near ? (qc.half ? 1 : 0) : 2);
      cls[q] = uint8_t(qc.apex | (qc.inner ? 4 : 0));
    }
    store_region_masks(mask, cnt, sp.nchunks, 3, ch, region);
  }
}

// the cubic spline's second piece of a near pair by the finer rule in the doubled frame, added
// to v: there the piece is (1 - r')^3_+, half the first piece's form 2 (1 - r)^3 that the rule
// evaluates; mapped back with the weights of Sec. 2's piecewise split (2^-(m+2) for a moment
// of degree m, -1/2 for the gradient), each halved
template <int MD>
__device__ __forceinline__ void add_second_piece(const QuadRaysFine& qf, const QuadRule& qs, const float* v6, int apex,
                                                 double C, double invH, float* v) {
  float d[6], w[13];
#pragma unroll
  for (int j = 0; j < 6; ++j) d[j] = 2.0f * v6[j];
  quad_pair<KID_CUBIC, MD>(qf, qs, d, apex, false, C, invH, w);
  v[0] += -0.125f * w[0];
  v[1] += -0.25f * w[1];
  v[2] += -0.25f * w[2];
  if (MD >= 1) {
    v[3] += -0.125f * w[3];
    v[4] += -0.0625f * w[4];
    v[5] += -0.0625f * w[5];
  }
  if (MD >= 3) {
#pragma unroll
    for (int i = 6; i < 9; ++i) v[i] += -0.03125f * w[i];
#pragma unroll
    for (int i = 9; i < 13; ++i) v[i] += -0.015625f * w[i];
  }
}

// Chunks of 32 positions of the partition.  CLOSED: the chunks up to the one holding the last
// closed-form position, every lane by the closed form (a boundary chunk's quadrature lanes
// too: each position is still evaluated once and keyed by its region); else the chunks after
// them, by quadrature.  Two kernels, so that the quadrature code keeps its own register
// allocation (~60 registers) and occupancy rather than the closed form's 128-168.
template <int KID, int MD, bool CLOSED>
__device__ __forceinline__ void hybrid_chunks(const IntArgs& a, const QuadRule& qr, const QuadRaysFine& qf,
                                              const PairSplit& sp, const uint8_t* __restrict__ cls) {
  constexpr int NV = nv_of(MD);
  const int lane = threadIdx.x & 31;
  const int64_t nchunks = (a.P + 31) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  const int64_t b1 = sp.off[sp.nchunks], b2 = sp.off[2 * sp.nchunks];   // first positions of regions 1, 2
  const int64_t cb = (b1 + 31) >> 5;                                   // chunks holding closed-form positions
  const int64_t c0 = CLOSED ? 0 : cb, n = CLOSED ? cb : nchunks - cb;
  const float ih = float(a.invH);
  unsigned long long fixes = 0;
  for (int64_t j = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; j < n;) {
    const unsigned long long nx = chunk_prefetch(a.work);
    const int64_t ch = c0 + j;
    const int64_t i = ch * 32 + lane;
    bool valid = false;
    unsigned long long key = 0;
    float v[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = 0.0f;
    int fix = 0;
    if (i < a.P) {
      const int64_t q = sp.order[i];
      const int pid = __ldg(a.pair_pid + q), tid = __ldg(a.pair_tri + q);
      const int r = i < b1 ? 0 : (i < b2 ? 1 : 2);
      valid = true;
      key = 3ull * unsigned(pid) + unsigned(r);
      const float4 p = a.parts[pid];
      const float* t = a.tris + 6 * int64_t(tid);
      float v6[6];
#pragma unroll
      for (int jj = 0; jj < 3; ++jj) {
        v6[2 * jj] = (__ldg(t + 2 * jj) - p.x) * ih;
        v6[2 * jj + 1] = (__ldg(t + 2 * jj + 1) - p.y) * ih;
      }
      if constexpr (CLOSED) {
        if constexpr (KID == KID_CUBIC) fix = cubic_split_pair<float, MD>(a, pid, tid, near_half<float>(v6), v);
        else fix = eval_pair<float, KID, MD>(a, pid, tid, v);
      } else {
        const unsigned c = cls[q];
        quad_pair<KID, MD>(qr, qr, v6, int(c & 3u), (c & 4u) != 0, a.C, a.invH, v);
        if constexpr (KID == KID_CUBIC) {
          if (r == 1) add_second_piece<MD>(qf, qr, v6, int(c & 3u), a.C, a.invH, v);
        }
      }
    }
    if constexpr (CLOSED) fixes += __popc(__ballot_sync(0xffffffffu, fix));
    keyed_chunk_sums<float, NV, 3, unsigned long long>(a, sp, ch, valid, key, v);
    j = chunk_next(a.work, j, nw, nx);
  }
  if (CLOSED && lane == 0 && fixes) atomicAdd(a.nfix, fixes);
}

// the cubic spline's closed form takes 3 resident blocks per SM with ten moments (as its
// chunk kernel over the near/far partition); the Wendland kernels 4
template <int KID, int MD> constexpr int hybrid_minb() {
  return KID == KID_CUBIC ? cubic_split_minb<float, MD>() : int_minb<float>();
}

template <int KID, int MD>
__global__ void __launch_bounds__(128, hybrid_minb<KID, MD>()) hybrid_closed_kernel(IntArgs a, QuadRule qr,
                                                                                   QuadRaysFine qf, PairSplit sp,
                                                                                   const uint8_t* __restrict__ cls) {
  hybrid_chunks<KID, MD, true>(a, qr, qf, sp, cls);
}

template <int KID, int MD>
__global__ void __launch_bounds__(128) hybrid_quad_kernel(IntArgs a, QuadRule qr, QuadRaysFine qf, PairSplit sp,
                                                          const uint8_t* __restrict__ cls) {
  hybrid_chunks<KID, MD, false>(a, qr, qf, sp, cls);
}

template <int KID, int MD>
static sph2d_status run_hybrid(Ctx* c, IntArgs a) {
  constexpr int NV = nv_of(MD);
  PairSplit sp;
  int64_t* cnt;
  unsigned long long* hdr;
  unsigned char* cls;
  sph2d_status s = split_scratch<float>(c, a, 3, NV, size_t(a.P > 0 ? a.P : 1), sp, cnt, hdr, cls);
  if (s != SPH2D_OK) return s;
  a.slots = c->slots.ptr;
  cudaError_t e = cudaMemsetAsync(hdr, 0, 64, c->stream);
  if (e != cudaSuccess) return cuda_err(c, e, "memset");
  if (a.P > 0) {
    a.work = hdr + 4;                                // chunk counters in the zeroed header
    SPH2D_LAUNCH(c, (hybrid_class_kernel<KID>), resident_blocks(c, hybrid_class_kernel<KID>, (sp.nchunks + 3) / 4),
                 128, a, sp, const_cast<uint32_t*>(sp.mask), cnt, cls);
    s = split_order(c, a, sp, cnt);
    if (s != SPH2D_OK) return s;
    IntArgs aq = a;
    aq.work = hdr + 5;                               // the quadrature kernel's own chunk counter
    SPH2D_LAUNCH(c, (hybrid_closed_kernel<KID, MD>),
                 resident_blocks(c, hybrid_closed_kernel<KID, MD>, (sp.nchunks + 3) / 4), 128, a, quad_rule(),
                 quad_rays_fine(), sp, cls);
    SPH2D_LAUNCH(c, (hybrid_quad_kernel<KID, MD>),
                 resident_blocks(c, hybrid_quad_kernel<KID, MD>, (sp.nchunks + 3) / 4), 128, aq, quad_rule(),
                 quad_rays_fine(), sp, cls);
  }
  if (a.N > 0) SPH2D_LAUNCH(c, (split_finalize_kernel<float, MD>), unsigned((a.N + 255) / 256), 256, a, sp);
  // the number of pairs left to the closed form (region 0), as the fallback count
  const void* n0 = a.P > 0 ? static_cast<const void*>(sp.off + sp.nchunks) : static_cast<const void*>(hdr);
  e = cudaMemcpyAsync(c->pinned + 10, n0, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream);
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
