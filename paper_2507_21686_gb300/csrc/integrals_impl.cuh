// Pair-integral kernels: evaluate every culled (particle, triangle) pair in closed form and
// sum per particle (Sec. 2, Eq. boundaryint), and the independent-pair entry point.
//
// Work layout.  The pair list is particle-major.  Each warp takes chunks of 32 consecutive
// pairs (one pair per lane), so the work per warp is uniform whatever the number of pairs
// per particle.  Per-particle sums use a segmented suffix sum over the lanes with warp
// shuffles; a particle whose pairs lie inside one chunk is written by the head lane of its
// segment.  A particle whose pairs cross chunk boundaries leaves its in-chunk partial sums
// in two slots per chunk (first and last segment), which a second kernel adds in chunk
// order.  Both orders are fixed, so results are deterministic run to run.
//
// Precision modes.
//   FP64:       local frame, geometry, transcendentals and recurrences in IEEE double.
//   FP32+fixup: local frame, geometry, angles and sector parts in FP32; the radial
//               recurrence and the kernel-coefficient sums in compensated FP32 (FF, see
//               pair_math.cuh); a pair whose local vertices lie beyond 16 H of the particle,
//               or whose FP32 result is not finite, is recomputed in FP64 by its lane.
#pragma once

#include <cuda_runtime.h>

#include "pair_math.cuh"
#include "sph2d_internal.h"

namespace sph2d {

constexpr float kFixupCoordLimit = 16.0f;

// moments carried per pair for moment degree MD (0: none, 1: M00 M10 M01, 3: all ten), and
// values per pair including gamma and grad gamma
constexpr int nmom_of(int MD) { return MD >= 3 ? 10 : (MD >= 1 ? 3 : 0); }
constexpr int nv_of(int MD) { return 3 + nmom_of(MD); }   // |p| in units of H beyond which FP32 is not used

struct IntArgs {
  const float4* parts;
  const float* tris;
  const int32_t* pair_tri;
  const int32_t* pair_pid;
  const int64_t* pair_off;
  int64_t P, N;
  double H, invH, C;
  // 1/H and the kernel constant rounded to FP32 once on the host (0: not set, then the FP32
  // path rounds a.invH and a.C per pair)
  float invHf = 0.0f, Cf = 0.0f;
  void* gamma;
  void* grad;
  void* mom;
  int nm;
  void* slots;
  unsigned long long* nfix;
  // zeroed counter for dynamic chunk scheduling of the pair kernels (null: static grid stride)
  unsigned long long* work = nullptr;
};

// Chunk scheduling of the pair kernels.  Each warp starts at its own chunk; with a counter it
// then takes the next free chunk (index nw + counter), fetched one chunk ahead so that the
// atomic's latency hides behind the chunk's arithmetic.  Pair costs vary by a factor of several
// across the mesh, and a static grid stride left the average SM idle for the last ~15% of the
// kernel (ncu: sm__cycles_active.avg / sm__cycles_elapsed.avg = 0.85 for C2).  Results do not
// depend on which warp takes a chunk.
__device__ __forceinline__ unsigned long long chunk_prefetch(unsigned long long* work) {
  unsigned long long nx = 0;
  if (work && (threadIdx.x & 31) == 0) nx = atomicAdd(work, 1ull);
  return nx;
}
__device__ __forceinline__ int64_t chunk_next(unsigned long long* work, int64_t ch, int64_t nw,
                                              unsigned long long nx) {
  return work ? nw + int64_t(__shfl_sync(0xffffffffu, nx, 0)) : ch + nw;
}

// raw integrals of one local-frame triangle -> v = (gamma, grad x, grad y, M00..M03)
template <typename R, int KID, int MD, typename S>
__device__ __forceinline__ void eval_local(const R* l, S C, S invH, R* v) {
  const int s = tri_orientation<R>(l[0], l[1], l[2], l[3], l[4], l[5]);
  if (s == 0) {
#pragma unroll
    for (int i = 0; i < nv_of(MD); ++i) v[i] = R(0);
    return;
  }
  PairOut<R> o;
  tri_raw<R, KID, MD>(l[0], l[1], l[2], l[3], l[4], l[5], o);
  const R k = R(C) * R(s);
  const R kg = -k * R(invH);
  v[0] = k * o.g;
  v[1] = kg * o.gx;
  v[2] = kg * o.gy;
#pragma unroll
  for (int m = 0; m < nmom_of(MD); ++m) v[3 + m] = k * o.m[m];
}

// evaluate from double-precision local coordinates in the mode's precision; returns 1 if the
// FP64 fix-up path was taken
template <typename OT, int KID, int MD>
__device__ __forceinline__ int eval_mode(const double* ld, double C, double invH, OT* v) {
  if (sizeof(OT) == sizeof(double)) {
    double w[13];
    eval_local<double, KID, MD>(ld, C, invH, w);
#pragma unroll
    for (int i = 0; i < nv_of(MD); ++i) v[i] = OT(w[i]);
    return 0;
  } else {
    float lf[6];
    bool ok = true;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      lf[j] = float(ld[j]);
      ok = ok && fabsf(lf[j]) <= kFixupCoordLimit;
    }
    if (ok) {
      float w[13];
      eval_local<float, KID, MD>(lf, C, invH, w);
#pragma unroll
      for (int i = 0; i < nv_of(MD); ++i) ok = ok && isfinite(w[i]);
      if (ok) {
#pragma unroll
        for (int i = 0; i < nv_of(MD); ++i) v[i] = OT(w[i]);
        return 0;
      }
    }
    double w[13];
    eval_local<double, KID, MD>(ld, C, invH, w);
#pragma unroll
    for (int i = 0; i < nv_of(MD); ++i) v[i] = OT(w[i]);
    return 1;
  }
}

// FP64 fix-up of one FP32 pair, kept out of line: it runs for few pairs, and inlined its FP64
// working set and code would sit in the FP32 kernel's register budget and instruction stream
template <int KID, int MD>
__device__ __noinline__ void eval_fixup64(const float4 p, const float* t, double invH, double C, float* v) {
  double ld[6];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    ld[2 * j] = (double(__ldg(t + 2 * j)) - double(p.x)) * invH;
    ld[2 * j + 1] = (double(__ldg(t + 2 * j + 1)) - double(p.y)) * invH;
  }
  double w[13];
  eval_local<double, KID, MD>(ld, C, invH, w);
#pragma unroll
  for (int i = 0; i < nv_of(MD); ++i) v[i] = float(w[i]);
}

template <typename OT, int KID, int MD>
__device__ __forceinline__ int eval_pair(const IntArgs& a, int pid, int tid, OT* v) {
  const float4 p = a.parts[pid];
  const float* t = a.tris + 6 * int64_t(tid);
  if (sizeof(OT) == sizeof(double)) {
    const double px = p.x, py = p.y;
    double ld[6];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      ld[2 * j] = (double(__ldg(t + 2 * j)) - px) * a.invH;
      ld[2 * j + 1] = (double(__ldg(t + 2 * j + 1)) - py) * a.invH;
    }
    return eval_mode<OT, KID, MD>(ld, a.C, a.invH, v);
  } else {
    // FP32 local frame straight from the FP32 inputs
    const float ih = a.invHf != 0.0f ? a.invHf : float(a.invH), cf = a.Cf != 0.0f ? a.Cf : float(a.C);
    float lf[6];
    bool ok = true;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      lf[2 * j] = (__ldg(t + 2 * j) - p.x) * ih;
      lf[2 * j + 1] = (__ldg(t + 2 * j + 1) - p.y) * ih;
      ok = ok && fabsf(lf[2 * j]) <= kFixupCoordLimit && fabsf(lf[2 * j + 1]) <= kFixupCoordLimit;
    }
    if (ok) {
      float w[13];
      eval_local<float, KID, MD>(lf, cf, ih, w);
#pragma unroll
      for (int i = 0; i < nv_of(MD); ++i) ok = ok && isfinite(w[i]);
      if (ok) {
#pragma unroll
        for (int i = 0; i < nv_of(MD); ++i) v[i] = OT(w[i]);
        return 0;
      }
    }
    float w[13];
    eval_fixup64<KID, MD>(p, t, a.invH, a.C, w);
#pragma unroll
    for (int i = 0; i < nv_of(MD); ++i) v[i] = OT(w[i]);
    return 1;
  }
}

// d gamma / d (x0, y0, x1, y1, x2, y2) of one culled pair in world units (transport-theorem
// edge integrals of pair_math.cuh, times C/H) in the mode's precision; returns 1 if the FP64
// path was used
template <typename OT, int KID>
__device__ __forceinline__ int vertex_grad_pair(const float4 p, const float* t, double invH, double C, OT* g) {
  if (sizeof(OT) == sizeof(float)) {
    const float ih = float(invH);
    float v[6];
    float pmax = 0.0f;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      v[2 * j] = (__ldg(t + 2 * j) - p.x) * ih;
      v[2 * j + 1] = (__ldg(t + 2 * j + 1) - p.y) * ih;
      pmax = fmaxf(pmax, fmaxf(fabsf(v[2 * j]), fabsf(v[2 * j + 1])));
    }
    // FP32 geometry is trusted when the vertices are near the particle and the triangle's
    // smallest height is at least |p|max/64 (thinner slivers can flip orientation under
    // FP32 rounding, which flips their vertex gradients)
    const float a2 = fabsf(diff_of_products(v[2] - v[0], v[5] - v[1], v[3] - v[1], v[4] - v[0]));
    float lmax = 0.0f;
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      const int b = e == 2 ? 0 : e + 1;
      const float ex = v[2 * b] - v[2 * e], ey = v[2 * b + 1] - v[2 * e + 1];
      lmax = fmaxf(lmax, sqrtf(ex * ex + ey * ey));
    }
    if (pmax <= kFixupCoordLimit && (a2 == 0.0f || 64.0f * a2 >= lmax * pmax)) {
      float w[6];
      tri_vertex_grad<float, KID>(v, w);
      bool ok = true;
#pragma unroll
      for (int i = 0; i < 6; ++i) ok = ok && isfinite(w[i]);
      if (ok) {
        const float k = float(C * invH);
#pragma unroll
        for (int i = 0; i < 6; ++i) g[i] = OT(k * w[i]);
        return 0;
      }
    }
  }
  double v[6], w[6];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    v[2 * j] = (double(__ldg(t + 2 * j)) - double(p.x)) * invH;
    v[2 * j + 1] = (double(__ldg(t + 2 * j + 1)) - double(p.y)) * invH;
  }
  tri_vertex_grad<double, KID>(v, w);
  const double k = C * invH;
#pragma unroll
  for (int i = 0; i < 6; ++i) g[i] = OT(k * w[i]);
  return sizeof(OT) == sizeof(float) ? 1 : 0;
}

// d grad gamma / d nu_j of one culled pair in world units, J[12] with J[4 j + 2 b + a] =
// d (grad gamma)_b / d (nu_j)_a, in the mode's precision; FP32 geometry is trusted under the
// same rule as vertex_grad_pair; returns 1 if the FP64 path was used
template <typename OT, int KID>
__device__ __forceinline__ int grad_jacobian_pair(const float4 p, const float* t, double invH, double C, OT* J) {
  if (sizeof(OT) == sizeof(float)) {
    const float ih = float(invH);
    float v[6];
    float pmax = 0.0f;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      v[2 * j] = (__ldg(t + 2 * j) - p.x) * ih;
      v[2 * j + 1] = (__ldg(t + 2 * j + 1) - p.y) * ih;
      pmax = fmaxf(pmax, fmaxf(fabsf(v[2 * j]), fabsf(v[2 * j + 1])));
    }
    const float a2 = fabsf(diff_of_products(v[2] - v[0], v[5] - v[1], v[3] - v[1], v[4] - v[0]));
    float lmax = 0.0f;
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      const int b = e == 2 ? 0 : e + 1;
      const float ex = v[2 * b] - v[2 * e], ey = v[2 * b + 1] - v[2 * e + 1];
      lmax = fmaxf(lmax, sqrtf(ex * ex + ey * ey));
    }
    if (pmax <= kFixupCoordLimit && (a2 == 0.0f || 64.0f * a2 >= lmax * pmax)) {
      float w[12];
      tri_grad_jacobian<float, KID>(v, w);
      bool ok = true;
#pragma unroll
      for (int i = 0; i < 12; ++i) ok = ok && isfinite(w[i]);
      if (ok) {
        const float k = float(-C * invH * invH);
#pragma unroll
        for (int i = 0; i < 12; ++i) J[i] = OT(k * w[i]);
        return 0;
      }
    }
  }
  double v[6], w[12];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    v[2 * j] = (double(__ldg(t + 2 * j)) - double(p.x)) * invH;
    v[2 * j + 1] = (double(__ldg(t + 2 * j + 1)) - double(p.y)) * invH;
  }
  tri_grad_jacobian<double, KID>(v, w);
  const double k = -C * invH * invH;
#pragma unroll
  for (int i = 0; i < 12; ++i) J[i] = OT(k * w[i]);
  return sizeof(OT) == sizeof(float) ? 1 : 0;
}

template <typename OT, int MD>
__device__ __forceinline__ void write_particle(const IntArgs& a, int64_t pid, const OT* v) {
  static_cast<OT*>(a.gamma)[pid] = v[0];
  if (a.grad) {
    static_cast<OT*>(a.grad)[2 * pid] = v[1];
    static_cast<OT*>(a.grad)[2 * pid + 1] = v[2];
  }
  if (a.nm == 1) {
    static_cast<OT*>(a.mom)[pid] = v[0];
  } else if (MD >= 1) {
    OT* m = static_cast<OT*>(a.mom) + pid * a.nm;
#pragma unroll
    for (int i = 0; i < nmom_of(MD); ++i)
      if (i < a.nm) m[i] = v[3 + i];
  }
}

// Minimum resident 128-thread blocks per SM for the FP32 pair kernels: 5 caps them at 96
// registers (20 warps per SM).  Measured on the 1024^2 box: 4 blocks (128 registers) ran 25%
// faster for Wendland C2 with moments than the compiler's own 148-register allocation, and
// once the fan code had shrunk (grid-extraction sums, fast division and square roots) 5 blocks
// ran 3-7% faster than 4 although the ten-moment instances spill 80-150 bytes per thread.  The
// FP64 instantiations keep the compiler's choice.  Without the ten moments (MD <= 1) 6 blocks
// (80 registers) measured another 1-3% faster; with them, 3% slower than 5.
#ifndef SPH2D_INT_MINB
#define SPH2D_INT_MINB 5
#endif
#ifndef SPH2D_INT_MINB_LOW
#define SPH2D_INT_MINB_LOW 6
#endif
#ifndef SPH2D_INT_MINB64
#define SPH2D_INT_MINB64 1
#endif
template <typename OT, int MD = 3> constexpr int int_minb() {
  return sizeof(OT) == sizeof(float) ? (MD <= 1 ? SPH2D_INT_MINB_LOW : SPH2D_INT_MINB) : SPH2D_INT_MINB64;
}

template <typename OT, int KID, int MD>
__global__ void __launch_bounds__(128, int_minb<OT, MD>()) integrals_kernel(IntArgs a) {
  constexpr int NV = nv_of(MD);
  const int lane = threadIdx.x & 31;
  const int64_t nchunks = (a.P + 31) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  unsigned long long fixes = 0;
  for (int64_t ch = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; ch < nchunks;) {
    const unsigned long long nx = chunk_prefetch(a.work);
    const int64_t q = ch * 32 + lane;
    int pid = -1;
    OT v[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = OT(0);
    int fix = 0;
    if (q < a.P) {
      pid = __ldg(a.pair_pid + q);
      fix = eval_pair<OT, KID, MD>(a, pid, __ldg(a.pair_tri + q), v);
    }
    fixes += __popc(__ballot_sync(0xffffffffu, fix));
    // segmented suffix sum: lane l accumulates the lanes l.. of its own particle
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int pn = __shfl_down_sync(0xffffffffu, pid, o);
      const bool same = (lane + o < 32) && (pn == pid);
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        const OT t = __shfl_down_sync(0xffffffffu, v[i], o);
        if (same) v[i] += t;
      }
    }
    const int pprev = __shfl_up_sync(0xffffffffu, pid, 1);
    const bool head = pid >= 0 && (lane == 0 || pprev != pid);
    const unsigned heads = __ballot_sync(0xffffffffu, head);
    const int last_head = 31 - __clz(heads);
    if (head) {
      const int64_t cs = ch * 32;
      const int64_t s0 = __ldg(a.pair_off + pid), s1 = __ldg(a.pair_off + pid + 1);
      if (s0 >= cs && s1 <= cs + 32) write_particle<OT, MD>(a, pid, v);
      OT* slots = static_cast<OT*>(a.slots);
      if (lane == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) slots[(ch * 2) * NV + i] = v[i];
      }
      if (lane == last_head) {
#pragma unroll
        for (int i = 0; i < NV; ++i) slots[(ch * 2 + 1) * NV + i] = v[i];
      }
    }
    ch = chunk_next(a.work, ch, nw, nx);
  }
  if (lane == 0 && fixes) atomicAdd(a.nfix, fixes);
}

// ---------------------------------------------------------------------------------------
// cubic spline.  k = 2 (1-q)^3_+ - (1-2q)^3_+ (scaled as in tri_raw): the second piece has
// support H/2 and is exactly zero for a triangle at distance >= H/2, which holds for most pairs;
// evaluated in place it would still run on every lane of a warp that holds one near pair.
//
// Per-particle path (run_cubic): cubic_batch_kernel below gathers the near pairs of several
// chunks into full warp-wide rounds of second pieces.  The hybrid mode's closed-form pairs
// (few, mostly near) take cubic_split_pair, both pieces in one lane, with a per-lane flag.
// ---------------------------------------------------------------------------------------
// origin within 1/2 (+ a small margin) of the local triangle: inside, or an edge segment
// closer than that (no division)
template <typename R>
__device__ __forceinline__ bool near_half(const R* l) {
  const R lim2 = R(0.501) * R(0.501);
  bool pos = false, neg = false, near = false;
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const int b = e == 2 ? 0 : e + 1;
    const R ax = l[2 * e], ay = l[2 * e + 1], bx = l[2 * b], by = l[2 * b + 1];
    const R ex = bx - ax, ey = by - ay;
    const R cr = ax * ey - ay * ex;
    pos = pos || cr > R(0);
    neg = neg || cr < R(0);
    const R l2 = ex * ex + ey * ey, tn = -(ax * ex + ay * ey);
    const bool n = tn <= R(0) ? (ax * ax + ay * ay < lim2)
                              : (tn >= l2 ? (bx * bx + by * by < lim2) : (cr * cr < lim2 * l2));
    near = near || n;
  }
  return near || (pos != neg);
}

// one piece of the cubic spline for a local triangle of orientation s != 0 -> v (scaled)
template <typename R, int MD, typename S>
__device__ __forceinline__ void cubic_piece(const R* l, int piece, int s, S C, S invH, R* v) {
  const R sc = piece ? R(2) : R(1);
  PairOut<R> h;
  clear(h);
  tri_poly<R, PolyCube, MD, false>(sc * l[0], sc * l[1], sc * l[2], sc * l[3], sc * l[4], sc * l[5], h);
  const R k = R(C) * R(s);
  const R wg = piece ? R(-0.25) : R(2), wd = piece ? R(-0.5) : R(2);
  v[0] = (k * wg) * h.g;
  v[1] = (-k * R(invH) * wd) * h.gx;
  v[2] = (-k * R(invH) * wd) * h.gy;
  if (MD >= 1) {
    const R w1 = piece ? R(-0.125) : R(2);
    v[3] = (k * wg) * h.m[0];
#pragma unroll
    for (int i = 1; i < 3; ++i) v[3 + i] = (k * w1) * h.m[i];
  }
  if (MD >= 3) {
    const R w2 = piece ? R(-0.0625) : R(2), w3 = piece ? R(-0.03125) : R(2);
#pragma unroll
    for (int i = 3; i < 6; ++i) v[3 + i] = (k * w2) * h.m[i];
#pragma unroll
    for (int i = 6; i < 10; ++i) v[3 + i] = (k * w3) * h.m[i];
  }
}

// warp-aggregated append of the lanes with flag set to list (count: its length)
__device__ __forceinline__ void warp_append(bool flag, int64_t q, int64_t* __restrict__ list,
                                            unsigned long long* __restrict__ count) {
  const int lane = threadIdx.x & 31;
  const unsigned m = __ballot_sync(0xffffffffu, flag);
  if (m) {
    unsigned long long b = 0;
    const int leader = __ffs(m) - 1;
    if (lane == leader) b = atomicAdd(count, (unsigned long long)__popc(m));
    b = __shfl_sync(0xffffffffu, b, leader);
    if (flag) list[b + __popc(m & ((1u << lane) - 1u))] = q;
  }
}

// per-particle sums of per-pair values [P][NV] in pair order
template <typename OT, int MD>
__global__ void __launch_bounds__(128) reduce_pairs_kernel(IntArgs a, const OT* __restrict__ vals) {
  constexpr int NV = nv_of(MD);
  const int lane = threadIdx.x & 31;
  const int64_t nchunks = (a.P + 31) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t ch = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; ch < nchunks; ch += nw) {
    const int64_t q = ch * 32 + lane;
    int pid = -1;
    OT v[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = OT(0);
    if (q < a.P) {
      pid = __ldg(a.pair_pid + q);
#pragma unroll
      for (int i = 0; i < NV; ++i) v[i] = vals[q * NV + i];
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int pn = __shfl_down_sync(0xffffffffu, pid, o);
      const bool same = (lane + o < 32) && (pn == pid);
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        const OT t = __shfl_down_sync(0xffffffffu, v[i], o);
        if (same) v[i] += t;
      }
    }
    const int pprev = __shfl_up_sync(0xffffffffu, pid, 1);
    const bool head = pid >= 0 && (lane == 0 || pprev != pid);
    const unsigned heads = __ballot_sync(0xffffffffu, head);
    const int last_head = 31 - __clz(heads);
    if (head) {
      const int64_t cs = ch * 32;
      const int64_t s0 = __ldg(a.pair_off + pid), s1 = __ldg(a.pair_off + pid + 1);
      if (s0 >= cs && s1 <= cs + 32) write_particle<OT, MD>(a, pid, v);
      OT* slots = static_cast<OT*>(a.slots);
      if (lane == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) slots[(ch * 2) * NV + i] = v[i];
      }
      if (lane == last_head) {
#pragma unroll
        for (int i = 0; i < NV; ++i) slots[(ch * 2 + 1) * NV + i] = v[i];
      }
    }
  }
}

// one warp's rows of a per-particle output of `width` values (out: the row of the warp's first
// particle), transposed through shared memory so that the stores are coalesced; a particle is
// written when its bit is set in `mine`
template <typename OT, int W>
__device__ __forceinline__ void warp_rows(OT* __restrict__ out, int width, unsigned mine, const OT* vals,
                                          OT* __restrict__ buf) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < W; ++k)
    if (k < width) buf[lane * width + k] = vals[k];
  __syncwarp();
  for (int j = 0; j < width; ++j) {
    const int w = 32 * j + lane;
    if ((mine >> (w / width)) & 1u) out[w] = buf[w];
  }
  __syncwarp();
}

// the outputs of a warp's 32 consecutive particles (i: this lane's particle, mine: whether it
// writes), rows transposed through shared memory; blocks of 256 threads
template <typename OT, int MD>
__device__ __forceinline__ void write_particles_warp(const IntArgs& a, int64_t i, bool mine, const OT* v) {
  constexpr int NM = nmom_of(MD), WB = NM > 2 ? NM : 2;
  __shared__ OT s_buf[8][32 * WB];
  const unsigned m = __ballot_sync(0xffffffffu, mine);
  if (m == 0u) return;                                   // warp-uniform
  const int64_t i0 = i - (threadIdx.x & 31);
  OT* buf = s_buf[threadIdx.x >> 5];
  if (mine) static_cast<OT*>(a.gamma)[i] = v[0];
  if (a.grad) warp_rows<OT, 2>(static_cast<OT*>(a.grad) + 2 * i0, 2, m, v + 1, buf);
  if (a.nm == 1) {
    if (mine) static_cast<OT*>(a.mom)[i] = v[0];
  } else if (MD >= 1 && a.nm > 0) {
    warp_rows<OT, NM>(static_cast<OT*>(a.mom) + int64_t(a.nm) * i0, a.nm, m, v + 3, buf);
  }
}

// particles without pairs get zeros; particles whose pairs span chunks add their partials.  A
// warp writes its 32 consecutive particles' rows together (blocks of 256 threads).
template <typename OT, int MD>
__global__ void __launch_bounds__(256) finalize_kernel(IntArgs a) {
  constexpr int NV = nv_of(MD);
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  OT v[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = OT(0);
  bool mine = false;
  if (i < a.N) {
    const int64_t s0 = a.pair_off[i], s1 = a.pair_off[i + 1];
    mine = true;
    if (s1 > s0) {
      const int64_t c0 = s0 >> 5, c1 = (s1 - 1) >> 5;
      if (c0 == c1) {
        mine = false;        // written by the chunk kernel
      } else {
        const OT* slots = static_cast<const OT*>(a.slots);
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] = slots[(c0 * 2 + 1) * NV + k];
        for (int64_t c = c0 + 1; c < c1; ++c) {
#pragma unroll
          for (int k = 0; k < NV; ++k) v[k] += slots[(c * 2) * NV + k];
        }
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] += slots[(c1 * 2) * NV + k];
      }
    }
  }
  write_particles_warp<OT, MD>(a, i, mine, v);
}

// grid of at most the blocks of 128 threads that stay resident at once (grid-stride kernels)
template <typename K>
static unsigned resident_blocks(Ctx* c, K kern, int64_t wanted) {
  int per_sm = 0, sms = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, 0);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  const int64_t cap = int64_t(per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
  return unsigned(wanted < cap ? (wanted > 0 ? wanted : 1) : cap);
}

// ---------------------------------------------------------------------------------------
// Stable partition of the pair list into K regions (pair kinds that take different code),
// each region in pair order, regions one after another.  A pass flags each pair's region per
// 32-pair chunk (one 32-bit mask per region and chunk) and counts the flags; one exclusive scan
// over the counts, region-major, gives every (region, chunk) its first position; the partition
// pass writes the pair at each position.  A chunk kernel over the positions then sums per
// (particle, region) with the segmented sums and crossing slots of integrals_kernel, and the
// finalize adds a particle's region sums in region order.  Every order is fixed, so results
// are deterministic run to run.
// A particle's sum over the last region, when held in one chunk, goes straight to the outputs
// (the last region holds most pairs: the cubic spline's far pairs, the hybrid mode's quadrature
// pairs); the finalize reads it back only for a particle that also has pairs in another region
// or whose last-region pairs cross chunks.  The other regions' in-chunk sums go to a
// [K-1][N][NV] buffer.
// ---------------------------------------------------------------------------------------
struct PairSplit {
  const uint32_t* mask;    // [K][nchunks] bit l of word (r, ch): pair 32 ch + l is of region r
  const int64_t* off;      // [K nchunks + 1] region-major exclusive scan of the mask counts
  const int32_t* order;    // [P] pair at each position of the partition (P < 2^31)
  void* part;              // [K-1][N][NV] sums of a particle's region r < K-1 held in one chunk
  int64_t nchunks;
  int nreg;
};

// position of the first pair of region r at or after pair q (0 <= q <= P)
__device__ __forceinline__ int64_t region_before(const PairSplit& s, int r, int64_t q) {
  const int64_t ch = q >> 5;
  if (ch >= s.nchunks) return s.off[(r + 1) * s.nchunks];
  const int64_t w = r * s.nchunks + ch;
  return s.off[w] + __popc(s.mask[w] & ((1u << (q & 31)) - 1u));
}

// positions [s0, s1) of particle pid's pairs of region r
__device__ __forceinline__ void part_range(const IntArgs& a, const PairSplit& s, int64_t pid, int r,
                                           int64_t& s0, int64_t& s1) {
  s0 = region_before(s, r, __ldg(a.pair_off + pid));
  s1 = region_before(s, r, __ldg(a.pair_off + pid + 1));
}

// flags of one chunk: every valid lane sets exactly one region; lane 0 stores the masks and
// their counts
__device__ __forceinline__ void store_region_masks(uint32_t* __restrict__ mask, int64_t* __restrict__ cnt,
                                                   int64_t nchunks, int nreg, int64_t ch, int region) {
  for (int r = 0; r < nreg; ++r) {
    const unsigned m = __ballot_sync(0xffffffffu, region == r);
    if ((threadIdx.x & 31) == 0) {
      mask[r * nchunks + ch] = m;
      cnt[r * nchunks + ch] = __popc(m);
    }
  }
}

// the partition: each pair at its rank within its region
static __global__ void __launch_bounds__(128) partition_kernel(PairSplit s, int64_t P, int32_t* __restrict__ order) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t ch = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; ch < s.nchunks; ch += nw) {
    const int64_t q = ch * 32 + lane;
    if (q >= P) continue;
    for (int r = 0; r < s.nreg; ++r) {
      const unsigned m = s.mask[r * s.nchunks + ch];
      if ((m >> lane) & 1u) {
        order[s.off[r * s.nchunks + ch] + __popc(m & ((1u << lane) - 1u))] = int32_t(q);
        break;
      }
    }
  }
}

// segmented sums of one chunk of positions keyed by K pid + region (K regions), written
// like integrals_kernel's: a key held within the chunk to part[region][pid] (the last region:
// to the particle's outputs), the chunk's first and last keys to its two slots
// (KT: the key type, 32-bit where K N stays below 2^32)
template <typename OT, int NV, int K, typename KT>
__device__ __forceinline__ void keyed_chunk_sums(const IntArgs& a, const PairSplit& sp, int64_t ch, bool valid,
                                                 KT key, OT* v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const KT kn = __shfl_down_sync(0xffffffffu, key, o);
    const bool same = (lane + o < 32) && (kn == key);
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const OT t = __shfl_down_sync(0xffffffffu, v[k], o);
      if (same) v[k] += t;
    }
  }
  const KT kprev = __shfl_up_sync(0xffffffffu, key, 1);
  const bool head = valid && (lane == 0 || kprev != key);
  const unsigned heads = __ballot_sync(0xffffffffu, head);
  const int last_head = 31 - __clz(heads);
  if (head) {
    const int64_t cs = ch * 32;
    const int64_t pid = int64_t(key / KT(K));
    const int r = int(key - KT(K) * KT(pid));
    int64_t s0, s1;
    part_range(a, sp, pid, r, s0, s1);
    if (s0 >= cs && s1 <= cs + 32) {
      if (r == K - 1) {
        write_particle<OT, NV == 3 ? 0 : (NV == 6 ? 1 : 3)>(a, pid, v);
      } else {
        OT* w = static_cast<OT*>(sp.part) + (int64_t(r) * a.N + pid) * NV;
#pragma unroll
        for (int k = 0; k < NV; ++k) w[k] = v[k];
      }
    }
    OT* slots = static_cast<OT*>(a.slots);
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < NV; ++k) slots[(ch * 2) * NV + k] = v[k];
    }
    if (lane == last_head) {
#pragma unroll
      for (int k = 0; k < NV; ++k) slots[(ch * 2 + 1) * NV + k] = v[k];
    }
  }
}

// a particle's outputs as write_particle stored them (the components it does not store are 0)
template <typename OT, int MD>
__device__ __forceinline__ void read_particle(const IntArgs& a, int64_t pid, OT* v) {
  constexpr int NV = nv_of(MD);
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = OT(0);
  v[0] = static_cast<const OT*>(a.gamma)[pid];
  if (a.grad) {
    v[1] = static_cast<const OT*>(a.grad)[2 * pid];
    v[2] = static_cast<const OT*>(a.grad)[2 * pid + 1];
  }
  if (MD >= 1) {
    if (a.nm == 1) {
      v[3] = v[0];                                 // M00 = gamma
    } else {
      const OT* m = static_cast<const OT*>(a.mom) + pid * a.nm;
#pragma unroll
      for (int k = 0; k < nmom_of(MD); ++k)
        if (k < a.nm) v[3 + k] = m[k];
    }
  }
}

// per particle: the region sums in region order, each from its chunk (the last region's from
// the outputs) or its crossing slots.  A particle whose pairs are all in the last region and
// within one chunk already has its sum in the outputs.
template <typename OT, int MD>
__global__ void __launch_bounds__(256) split_finalize_kernel(IntArgs a, PairSplit sp) {
  constexpr int NV = nv_of(MD);
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  OT v[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = OT(0);
  bool mine = i < a.N;
  if (mine && a.pair_off[i + 1] > a.pair_off[i]) {
    const int last = sp.nreg - 1;
    int64_t l0, l1;
    part_range(a, sp, i, last, l0, l1);
    if (l1 - l0 == a.pair_off[i + 1] - a.pair_off[i] && (l0 >> 5) == ((l1 - 1) >> 5)) {
      mine = false;          // written by the chunk kernel
    } else {
      const OT* slots = static_cast<const OT*>(a.slots);
      bool first = true;
#pragma unroll 1
      for (int r = 0; r < sp.nreg; ++r) {
        int64_t s0, s1;
        part_range(a, sp, i, r, s0, s1);
        if (s1 <= s0) continue;
        OT w[NV];
        const int64_t c0 = s0 >> 5, c1 = (s1 - 1) >> 5;
        if (c0 == c1) {
          if (r == last) {
            read_particle<OT, MD>(a, i, w);
          } else {
            const OT* src = static_cast<const OT*>(sp.part) + (int64_t(r) * a.N + i) * NV;
#pragma unroll
            for (int k = 0; k < NV; ++k) w[k] = src[k];
          }
        } else {
#pragma unroll
          for (int k = 0; k < NV; ++k) w[k] = slots[(c0 * 2 + 1) * NV + k];
          for (int64_t c = c0 + 1; c < c1; ++c) {
#pragma unroll
            for (int k = 0; k < NV; ++k) w[k] += slots[(c * 2) * NV + k];
          }
#pragma unroll
          for (int k = 0; k < NV; ++k) w[k] += slots[(c1 * 2) * NV + k];
        }
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] = first ? w[k] : v[k] + w[k];
        first = false;
      }
    }
  }
  write_particles_warp<OT, MD>(a, i, mine, v);
}

// scratch of a K-region partition in pair_list2: header (chunk counter at [4]) | counts
// [K nchunks + 1] | offsets [K nchunks + 1] | order int32 [P] (padded to 8 bytes) | masks
// [K nchunks] | extra bytes; region sums [K-1][N][NV] in pair_vals
inline size_t split_list_bytes(int64_t P, int64_t nchunks, int K, size_t extra) {
  return 64 + size_t(2 * (K * nchunks + 1)) * sizeof(int64_t) + size_t((P + 1) / 2) * 8 +
         size_t(K * nchunks + 1) * 4 + extra;
}
template <typename OT>
static sph2d_status split_scratch(Ctx* c, const IntArgs& a, int K, int NV, size_t extra, PairSplit& sp,
                                  int64_t*& cnt, unsigned long long*& hdr, unsigned char*& extra_ptr) {
  if (a.P >= (int64_t(1) << 31))
    return set_err(c, SPH2D_ERR_CAPACITY, "a partitioned pair list (cubic spline, hybrid mode) holds < 2^31 pairs");
  const int64_t nchunks = (a.P + 31) >> 5;
  sph2d_status s = ensure(c, c->slots, size_t(nchunks * 2 * NV + 1) * sizeof(OT));
  if (s == SPH2D_OK)
    s = ensure(c, c->pair_vals, size_t(K - 1 > 0 ? K - 1 : 1) * size_t(a.N > 0 ? a.N : 1) * NV * sizeof(OT));
  if (s == SPH2D_OK) s = ensure(c, c->pair_list2, split_list_bytes(a.P, nchunks, K, extra));
  if (s != SPH2D_OK) return s;
  hdr = static_cast<unsigned long long*>(c->pair_list2.ptr);
  cnt = reinterpret_cast<int64_t*>(static_cast<char*>(c->pair_list2.ptr) + 64);
  int64_t* off = cnt + (K * nchunks + 1);
  int32_t* order = reinterpret_cast<int32_t*>(off + (K * nchunks + 1));
  uint32_t* mask = reinterpret_cast<uint32_t*>(order + 2 * ((a.P + 1) / 2));
  extra_ptr = reinterpret_cast<unsigned char*>(mask + (K * nchunks + 1));
  sp = PairSplit{mask, off, order, c->pair_vals.ptr, nchunks, K};
  return SPH2D_OK;
}

// after the masks: scan, partition
static sph2d_status split_order(Ctx* c, const IntArgs& a, PairSplit& sp, const int64_t* cnt) {
  sph2d_status s = exclusive_scan_i64(c, cnt, const_cast<int64_t*>(sp.off), int64_t(sp.nreg) * sp.nchunks);
  if (s != SPH2D_OK) return s;
  SPH2D_LAUNCH(c, (partition_kernel), resident_blocks(c, partition_kernel, (sp.nchunks + 3) / 4), 128, sp, a.P,
               const_cast<int32_t*>(sp.order));
  return SPH2D_OK;
}

// ---------------------------------------------------------------------------------------
// cubic spline over the near/far partition: region 0 the pairs within H/2 of their triangle
// (both pieces), region 1 the others (the first piece only)
// ---------------------------------------------------------------------------------------
// one pair: the first piece, plus the second for a near pair; FP32 pairs whose
// coordinates leave the FP32 range or whose result is not finite take the whole kernel in FP64
// (eval_fixup64, out of line).  Returns 1 for a fix-up.
template <typename OT, int MD>
__device__ __forceinline__ int cubic_split_pair(const IntArgs& a, int pid, int tid, bool near, OT* v) {
  constexpr int NV = nv_of(MD);
  const float4 p = a.parts[pid];
  const float* t = a.tris + 6 * int64_t(tid);
  if constexpr (sizeof(OT) == sizeof(float)) {
    const float ih = a.invHf != 0.0f ? a.invHf : float(a.invH), cf = a.Cf != 0.0f ? a.Cf : float(a.C);
    float lf[6];
    bool ok = true;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      lf[2 * j] = (__ldg(t + 2 * j) - p.x) * ih;
      lf[2 * j + 1] = (__ldg(t + 2 * j + 1) - p.y) * ih;
      ok = ok && fabsf(lf[2 * j]) <= kFixupCoordLimit && fabsf(lf[2 * j + 1]) <= kFixupCoordLimit;
    }
    if (ok) {
      const int s = tri_orientation<float>(lf[0], lf[1], lf[2], lf[3], lf[4], lf[5]);
#pragma unroll
      for (int i = 0; i < NV; ++i) v[i] = 0.0f;
      if (s == 0) return 0;
      const int npieces = near ? 2 : 1;
#pragma unroll 1
      for (int piece = 0; piece < npieces; ++piece) {
        float w[13];
        cubic_piece<float, MD>(lf, piece, s, cf, ih, w);
#pragma unroll
        for (int i = 0; i < NV; ++i) v[i] = piece ? v[i] + w[i] : w[i];
      }
#pragma unroll
      for (int i = 0; i < NV; ++i) ok = ok && isfinite(v[i]);
      if (ok) return 0;
    }
    eval_fixup64<KID_CUBIC, MD>(p, t, a.invH, a.C, v);
    return 1;
  } else {
    double ld[6];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      ld[2 * j] = (double(__ldg(t + 2 * j)) - double(p.x)) * a.invH;
      ld[2 * j + 1] = (double(__ldg(t + 2 * j + 1)) - double(p.y)) * a.invH;
    }
    const int s = tri_orientation<double>(ld[0], ld[1], ld[2], ld[3], ld[4], ld[5]);
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = 0.0;
    if (s == 0) return 0;
    const int npieces = near ? 2 : 1;
#pragma unroll 1
    for (int piece = 0; piece < npieces; ++piece) {
      double w[13];
      cubic_piece<double, MD>(ld, piece, s, a.C, a.invH, w);
#pragma unroll
      for (int i = 0; i < NV; ++i) v[i] = piece ? v[i] + w[i] : w[i];
    }
    return 0;
  }
}

// The cubic spline's pair kernels run at the Wendland kernels' cap.  The earlier partition
// kernel, with its pieces' fans inlined, ran best at 3 blocks (168 registers); with the fans
// looped, 4 blocks measured 6.5% faster than 3 with ten moments, and later 5 blocks as fast as 4
// with ten moments and 7% faster without.
template <typename OT, int MD> constexpr int cubic_split_minb() { return int_minb<OT, MD>(); }


// ---------------------------------------------------------------------------------------
// Single-pass cubic spline (run_cubic).  Each warp fills a batch with the chunks it takes
// (32 consecutive pairs each, in the pair list's own order, at most kCubicBatch chunks) for as
// long as their near pairs (within H/2 of their triangle: both pieces) number at most
// kCubicNearCap.  Rounds over the batch's near pairs, one per lane, evaluate the second piece
// into shared memory; then each chunk of the batch runs the first piece on every lane, adds a
// near pair's second piece (piece1 + piece2, in that order) and sums per particle with the
// segmented sums and crossing slots of integrals_kernel.  The near pairs of several chunks so share their
// warp-wide rounds, the pair list is read in place and the per-particle sums are those of the
// single-polynomial kernels (finalize_kernel).  Every order is fixed, so results are
// deterministic run to run.
// ---------------------------------------------------------------------------------------
constexpr int kCubicBatch = 8, kCubicNearCap = 64;

// bit position of the n-th (from 0) set bit of m; m has more than n set bits
__device__ __forceinline__ int nth_set_bit(unsigned m, int n) {
  int pos = 0;
#pragma unroll
  for (int w = 16; w >= 1; w >>= 1) {
    const unsigned low = m & ((1u << w) - 1u);
    const int c = __popc(low);
    if (n >= c) {
      n -= c;
      m >>= w;
      pos += w;
    } else {
      m = low;
    }
  }
  return pos;
}

// local frame of pair (pid, tid) in the output precision; false if an FP32 coordinate leaves
// the FP32 range (the pair then takes the FP64 fix-up)
template <typename OT>
__device__ __forceinline__ bool cubic_local(const IntArgs& a, int pid, int tid, OT* l) {
  const float4 p = a.parts[pid];
  const float* t = a.tris + 6 * int64_t(tid);
  bool ok = true;
  if constexpr (sizeof(OT) == sizeof(float)) {
    const float ih = a.invHf != 0.0f ? a.invHf : float(a.invH);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      l[2 * j] = (__ldg(t + 2 * j) - p.x) * ih;
      l[2 * j + 1] = (__ldg(t + 2 * j + 1) - p.y) * ih;
      ok = ok && fabsf(l[2 * j]) <= kFixupCoordLimit && fabsf(l[2 * j + 1]) <= kFixupCoordLimit;
    }
  } else {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      l[2 * j] = (double(__ldg(t + 2 * j)) - double(p.x)) * a.invH;
      l[2 * j + 1] = (double(__ldg(t + 2 * j + 1)) - double(p.y)) * a.invH;
    }
  }
  return ok;
}

// one piece of a pair from its local frame (zeros for a degenerate triangle)
template <typename OT, int MD>
__device__ __forceinline__ void cubic_piece_pair(const IntArgs& a, const OT* l, int piece, OT* v) {
  constexpr int NV = nv_of(MD);
  const int s = tri_orientation<OT>(l[0], l[1], l[2], l[3], l[4], l[5]);
  if (s == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = OT(0);
    return;
  }
  if constexpr (sizeof(OT) == sizeof(float)) {
    const float ih = a.invHf != 0.0f ? a.invHf : float(a.invH), cf = a.Cf != 0.0f ? a.Cf : float(a.C);
    float w[13];
    cubic_piece<float, MD>(l, piece, s, cf, ih, w);
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = w[i];
  } else {
    double w[13];
    cubic_piece<double, MD>(l, piece, s, a.C, a.invH, w);
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = w[i];
  }
}

// near flags of chunk ch (bit l: pair 32 ch + l is within H/2 of its triangle)
template <typename OT>
__device__ __forceinline__ unsigned cubic_near_flags(const IntArgs& a, int64_t ch) {
  const int64_t q = ch * 32 + (threadIdx.x & 31);
  bool near = false;
  if (q < a.P) {
    OT l[6];
    cubic_local<OT>(a, __ldg(a.pair_pid + q), __ldg(a.pair_tri + q), l);
    near = near_half<OT>(l);
  }
  return __ballot_sync(0xffffffffu, near);
}

// the segmented per-particle sums of one chunk (pid -1 for a lane past the list), as in
// integrals_kernel: a particle held in the chunk is written by the head lane of its segment,
// the chunk's first and last segments go to its two crossing slots
template <typename OT, int MD>
__device__ __forceinline__ void chunk_particle_sums(const IntArgs& a, int64_t ch, int pid, OT* v) {
  constexpr int NV = nv_of(MD);
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int pn = __shfl_down_sync(0xffffffffu, pid, o);
    const bool same = (lane + o < 32) && (pn == pid);
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      const OT t = __shfl_down_sync(0xffffffffu, v[i], o);
      if (same) v[i] += t;
    }
  }
  const int pprev = __shfl_up_sync(0xffffffffu, pid, 1);
  const bool head = pid >= 0 && (lane == 0 || pprev != pid);
  const unsigned heads = __ballot_sync(0xffffffffu, head);
  const int last_head = 31 - __clz(heads);
  if (head) {
    const int64_t cs = ch * 32;
    const int64_t s0 = __ldg(a.pair_off + pid), s1 = __ldg(a.pair_off + pid + 1);
    if (s0 >= cs && s1 <= cs + 32) write_particle<OT, MD>(a, pid, v);
    OT* slots = static_cast<OT*>(a.slots);
    if (lane == 0) {
#pragma unroll
      for (int i = 0; i < NV; ++i) slots[(ch * 2) * NV + i] = v[i];
    }
    if (lane == last_head) {
#pragma unroll
      for (int i = 0; i < NV; ++i) slots[(ch * 2 + 1) * NV + i] = v[i];
    }
  }
}

template <typename OT, int MD>
__global__ void __launch_bounds__(128, cubic_split_minb<OT, MD>()) cubic_batch_kernel(IntArgs a) {
  constexpr int NV = nv_of(MD);
  __shared__ OT s_w2[4][kCubicNearCap][NV];          // second pieces of the batch's near pairs
  __shared__ int64_t s_ch[4][kCubicBatch];
  __shared__ unsigned s_mask[4][kCubicBatch];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t nchunks = (a.P + 31) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  unsigned long long fixes = 0;
  int64_t carry = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;   // taken, not yet batched
  unsigned long long nx = 0;
  unsigned cmask = 0;
  if (carry < nchunks) {
    nx = chunk_prefetch(a.work);
    cmask = cubic_near_flags<OT>(a, carry);
  }
  while (carry < nchunks) {
    // fill the batch (warp-uniform): a single chunk never holds more than 32 near pairs.  Once
    // fewer than two chunks per warp remain, a batch takes one chunk, so that the last batches
    // end together
    int k = 0, tot = 0;
    while (carry < nchunks && k < kCubicBatch && tot + __popc(cmask) <= kCubicNearCap &&
           (k == 0 || nchunks - carry > 2 * nw)) {
      if (lane == 0) {
        s_ch[wib][k] = carry;
        s_mask[wib][k] = cmask;
      }
      tot += __popc(cmask);
      ++k;
      carry = chunk_next(a.work, carry, nw, nx);
      if (carry < nchunks) {
        nx = chunk_prefetch(a.work);
        cmask = cubic_near_flags<OT>(a, carry);
      }
    }
    __syncwarp();
    // rounds r < n2: lane l takes the second piece of the batch's near pair j = 32 r + l; round
    // n2 + i: the first piece of every pair of the batch's chunk i, plus its second piece, and
    // the sums.  One call site for both pieces keeps one copy of the piece code.
    const int n2 = (tot + 31) >> 5;
    int base = 0;
#pragma unroll 1
    for (int r = 0; r < n2 + k; ++r) {
      int64_t q = -1;
      unsigned m = 0;
      const int j2 = 32 * r + lane;
      if (r < n2) {
        if (j2 < tot) {
          int i = 0, b = 0;
          while (b + __popc(s_mask[wib][i]) <= j2) {
            b += __popc(s_mask[wib][i]);
            ++i;
          }
          q = s_ch[wib][i] * 32 + nth_set_bit(s_mask[wib][i], j2 - b);
        }
      } else {
        m = s_mask[wib][r - n2];
        q = s_ch[wib][r - n2] * 32 + lane;
        if (q >= a.P) q = -1;
      }
      int pid = -1, tid = 0;
      bool ok = true;
      OT v[NV];
#pragma unroll
      for (int x = 0; x < NV; ++x) v[x] = OT(0);
      if (q >= 0) {
        pid = __ldg(a.pair_pid + q);
        tid = __ldg(a.pair_tri + q);
        OT l[6];
        ok = cubic_local<OT>(a, pid, tid, l);
        if (ok) cubic_piece_pair<OT, MD>(a, l, r < n2 ? 1 : 0, v);
      }
      if (r < n2) {
        if (q >= 0) {
#pragma unroll
          for (int x = 0; x < NV; ++x) s_w2[wib][j2][x] = ok ? v[x] : OT(NAN);   // NaN: the owner's fix-up
        }
        __syncwarp();
        continue;
      }
      int fix = 0;
      if (q >= 0) {
        if (ok && ((m >> lane) & 1u)) {
          const int j = base + __popc(m & ((1u << lane) - 1u));
#pragma unroll
          for (int x = 0; x < NV; ++x) v[x] += s_w2[wib][j][x];
        }
        if constexpr (sizeof(OT) == sizeof(float)) {
#pragma unroll
          for (int x = 0; x < NV; ++x) ok = ok && isfinite(v[x]);
          if (!ok) {
            float w[13];
            eval_fixup64<KID_CUBIC, MD>(a.parts[pid], a.tris + 6 * int64_t(tid), a.invH, a.C, w);
#pragma unroll
            for (int x = 0; x < NV; ++x) v[x] = OT(w[x]);
            fix = 1;
          }
        }
      }
      base += __popc(m);
      fixes += __popc(__ballot_sync(0xffffffffu, fix));
      chunk_particle_sums<OT, MD>(a, s_ch[wib][r - n2], pid, v);
    }
    __syncwarp();
  }
  if (lane == 0 && fixes) atomicAdd(a.nfix, fixes);
}

// independent pairs: [P][8] doubles -> [P][3+nm]
template <typename OT, int KID, int MD>
__global__ void __launch_bounds__(256) pair_entry_kernel(const double* __restrict__ pairs, int64_t P,
                                                         double invH, double C, int nm,
                                                         OT* __restrict__ out,
                                                         unsigned long long* nfix) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  int fix = 0;
  if (i < P) {
    const double* q = pairs + 8 * i;
    const double px = q[0], py = q[1];
    double ld[6];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      ld[2 * j] = (q[2 + 2 * j] - px) * invH;
      ld[2 * j + 1] = (q[3 + 2 * j] - py) * invH;
    }
    OT v[nv_of(MD)];
    fix = eval_mode<OT, KID, MD>(ld, C, invH, v);
    OT* o = out + i * (3 + nm);
    o[0] = v[0];
    o[1] = v[1];
    o[2] = v[2];
    if (nm == 1) o[3] = v[0];
    else if (MD >= 1) {
#pragma unroll
      for (int m = 0; m < nmom_of(MD); ++m)
        if (m < nm) o[3 + m] = v[3 + m];
    }
  }
  const unsigned b = __ballot_sync(0xffffffffu, fix);
  if ((threadIdx.x & 31) == 0 && b) atomicAdd(nfix, (unsigned long long)__popc(b));
}

// ---------------------------------------------------------------------------------------
// host launchers for one output precision
// ---------------------------------------------------------------------------------------
template <typename OT, int MD>
static sph2d_status run_cubic(Ctx* c, IntArgs a) {
  constexpr int NV = nv_of(MD);
  const int64_t nchunks = (a.P + 31) >> 5;
  sph2d_status s = ensure(c, c->slots, size_t(nchunks * 2 * NV + 1) * sizeof(OT));
  if (s != SPH2D_OK) return s;
  a.slots = c->slots.ptr;
  if (a.P > 0)
    SPH2D_LAUNCH(c, (cubic_batch_kernel<OT, MD>),
                 resident_blocks(c, cubic_batch_kernel<OT, MD>, (nchunks + 3) / 4), 128, a);
  if (a.N > 0) SPH2D_LAUNCH(c, (finalize_kernel<OT, MD>), unsigned((a.N + 255) / 256), 256, a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(c, e, "integrals launch");
  return SPH2D_OK;
}

template <typename OT, int KID, int MD>
static sph2d_status run_integrals(Ctx* c, IntArgs a) {
  if constexpr (KID == KID_CUBIC) {
    return run_cubic<OT, MD>(c, a);
  } else {
  constexpr int NV = nv_of(MD);
  const int64_t nchunks = (a.P + 31) >> 5;
  sph2d_status s = ensure(c, c->slots, size_t(nchunks * 2 * NV + 1) * sizeof(OT));
  if (s != SPH2D_OK) return s;
  a.slots = c->slots.ptr;
  if (a.P > 0) {
    const int64_t want = (nchunks + 3) / 4;              // 4 warps per block
    SPH2D_LAUNCH(c, (integrals_kernel<OT, KID, MD>), resident_blocks(c, integrals_kernel<OT, KID, MD>, want), 128, a);
  }
  if (a.N > 0) SPH2D_LAUNCH(c, (finalize_kernel<OT, MD>), unsigned((a.N + 255) / 256), 256, a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(c, e, "integrals launch");
  return SPH2D_OK;
  }
}

// moment degree computed for a requested moment_degree: -1/0 -> 0, 1 -> 1, 2/3 -> 3
inline int md_for(int moment_degree) { return moment_degree >= 2 ? 3 : (moment_degree == 1 ? 1 : 0); }

template <typename OT, int KID>
static sph2d_status run_md(Ctx* c, int md, IntArgs a) {
  return md == 3 ? run_integrals<OT, KID, 3>(c, a)
                 : (md == 1 ? run_integrals<OT, KID, 1>(c, a) : run_integrals<OT, KID, 0>(c, a));
}

template <typename OT>
static sph2d_status dispatch_integrals(Ctx* c, int kernel, int md, IntArgs a) {
  a.invHf = float(a.invH);
  a.Cf = float(a.C);
  switch (kernel) {
    case KID_WC2: return run_md<OT, KID_WC2>(c, md, a);
    case KID_WC4: return run_md<OT, KID_WC4>(c, md, a);
    case KID_WC6: return run_md<OT, KID_WC6>(c, md, a);
    default: return run_md<OT, KID_CUBIC>(c, md, a);
  }
}

template <typename OT>
static sph2d_status dispatch_pairs(Ctx* c, const double* pairs, int64_t P, int kernel, double H,
                                   int deg, unsigned long long* nfix, void* out) {
  const int nm = num_moments(deg);
  const int md = md_for(deg);
  const double invH = 1.0 / H, C = kernel_C(kernel);
  const unsigned blocks = unsigned((P + 255) / 256);
  if (P == 0) return SPH2D_OK;
  OT* o = static_cast<OT*>(out);
#define SPH2D_PE(K, MM) SPH2D_LAUNCH(c, (pair_entry_kernel<OT, K, MM>), blocks, 256, pairs, P, invH, C, nm, o, nfix)
#define SPH2D_PEK(K) \
  do { if (md == 3) SPH2D_PE(K, 3); else if (md == 1) SPH2D_PE(K, 1); else SPH2D_PE(K, 0); } while (0)
  switch (kernel) {
    case KID_WC2: SPH2D_PEK(KID_WC2); break;
    case KID_WC4: SPH2D_PEK(KID_WC4); break;
    case KID_WC6: SPH2D_PEK(KID_WC6); break;
    default: SPH2D_PEK(KID_CUBIC); break;
  }
#undef SPH2D_PEK
#undef SPH2D_PE
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(c, e, "pair integrals launch");
  return SPH2D_OK;
}

}  // namespace sph2d
