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

constexpr float kFixupCoordLimit = 16.0f;   // |p| in units of H beyond which FP32 is not used

struct IntArgs {
  const float4* parts;
  const float* tris;
  const int32_t* pair_tri;
  const int32_t* pair_pid;
  const int64_t* pair_off;
  int64_t P, N;
  double H, invH, C;
  void* gamma;
  void* grad;
  void* mom;
  int nm;
  void* slots;
  unsigned long long* nfix;
};

// raw integrals of one local-frame triangle -> v = (gamma, grad x, grad y, M00..M03)
template <typename R, int KID, bool MOM>
__device__ __forceinline__ void eval_local(const R* l, double C, double invH, R* v) {
  const int s = tri_orientation<R>(l[0], l[1], l[2], l[3], l[4], l[5]);
  if (s == 0) {
#pragma unroll
    for (int i = 0; i < (MOM ? 13 : 3); ++i) v[i] = R(0);
    return;
  }
  PairOut<R> o;
  tri_raw<R, KID, MOM>(l[0], l[1], l[2], l[3], l[4], l[5], o);
  const R k = R(C) * R(s);
  const R kg = -k * R(invH);
  v[0] = k * o.g;
  v[1] = kg * o.gx;
  v[2] = kg * o.gy;
  if (MOM) {
#pragma unroll
    for (int m = 0; m < 10; ++m) v[3 + m] = k * o.m[m];
  }
}

// evaluate from double-precision local coordinates in the mode's precision; returns 1 if the
// FP64 fix-up path was taken
template <typename OT, int KID, bool MOM>
__device__ __forceinline__ int eval_mode(const double* ld, double C, double invH, OT* v) {
  if (sizeof(OT) == sizeof(double)) {
    double w[13];
    eval_local<double, KID, MOM>(ld, C, invH, w);
#pragma unroll
    for (int i = 0; i < (MOM ? 13 : 3); ++i) v[i] = OT(w[i]);
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
      eval_local<float, KID, MOM>(lf, C, invH, w);
#pragma unroll
      for (int i = 0; i < (MOM ? 13 : 3); ++i) ok = ok && isfinite(w[i]);
      if (ok) {
#pragma unroll
        for (int i = 0; i < (MOM ? 13 : 3); ++i) v[i] = OT(w[i]);
        return 0;
      }
    }
    double w[13];
    eval_local<double, KID, MOM>(ld, C, invH, w);
#pragma unroll
    for (int i = 0; i < (MOM ? 13 : 3); ++i) v[i] = OT(w[i]);
    return 1;
  }
}

template <typename OT, int KID, bool MOM>
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
    return eval_mode<OT, KID, MOM>(ld, a.C, a.invH, v);
  } else {
    // FP32 local frame straight from the FP32 inputs
    const float ih = float(a.invH);
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
      eval_local<float, KID, MOM>(lf, a.C, a.invH, w);
#pragma unroll
      for (int i = 0; i < (MOM ? 13 : 3); ++i) ok = ok && isfinite(w[i]);
      if (ok) {
#pragma unroll
        for (int i = 0; i < (MOM ? 13 : 3); ++i) v[i] = OT(w[i]);
        return 0;
      }
    }
    double ld[6];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      ld[2 * j] = (double(__ldg(t + 2 * j)) - double(p.x)) * a.invH;
      ld[2 * j + 1] = (double(__ldg(t + 2 * j + 1)) - double(p.y)) * a.invH;
    }
    double w[13];
    eval_local<double, KID, MOM>(ld, a.C, a.invH, w);
#pragma unroll
    for (int i = 0; i < (MOM ? 13 : 3); ++i) v[i] = OT(w[i]);
    return 1;
  }
}

template <typename OT, bool MOM>
__device__ __forceinline__ void write_particle(const IntArgs& a, int64_t pid, const OT* v) {
  static_cast<OT*>(a.gamma)[pid] = v[0];
  if (a.grad) {
    static_cast<OT*>(a.grad)[2 * pid] = v[1];
    static_cast<OT*>(a.grad)[2 * pid + 1] = v[2];
  }
  if (a.nm == 1) {
    static_cast<OT*>(a.mom)[pid] = v[0];
  } else if (MOM) {
    OT* m = static_cast<OT*>(a.mom) + pid * a.nm;
#pragma unroll
    for (int i = 0; i < 10; ++i)
      if (i < a.nm) m[i] = v[3 + i];
  }
}

template <typename OT, int KID, bool MOM>
__global__ void __launch_bounds__(128) integrals_kernel(IntArgs a) {
  constexpr int NV = MOM ? 13 : 3;
  const int lane = threadIdx.x & 31;
  const int64_t nchunks = (a.P + 31) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  unsigned long long fixes = 0;
  for (int64_t ch = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; ch < nchunks; ch += nw) {
    const int64_t q = ch * 32 + lane;
    int pid = -1;
    OT v[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = OT(0);
    int fix = 0;
    if (q < a.P) {
      pid = __ldg(a.pair_pid + q);
      fix = eval_pair<OT, KID, MOM>(a, pid, __ldg(a.pair_tri + q), v);
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
      if (s0 >= cs && s1 <= cs + 32) write_particle<OT, MOM>(a, pid, v);
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
  if (lane == 0 && fixes) atomicAdd(a.nfix, fixes);
}

// particles without pairs get zeros; particles whose pairs span chunks add their partials
template <typename OT, bool MOM>
__global__ void finalize_kernel(IntArgs a) {
  constexpr int NV = MOM ? 13 : 3;
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= a.N) return;
  const int64_t s0 = a.pair_off[i], s1 = a.pair_off[i + 1];
  OT v[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = OT(0);
  if (s1 > s0) {
    const int64_t c0 = s0 >> 5, c1 = (s1 - 1) >> 5;
    if (c0 == c1) return;   // written by the chunk kernel
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
  write_particle<OT, MOM>(a, i, v);
}

// independent pairs: [P][8] doubles -> [P][3+nm]
template <typename OT, int KID, bool MOM>
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
    OT v[MOM ? 13 : 3];
    fix = eval_mode<OT, KID, MOM>(ld, C, invH, v);
    OT* o = out + i * (3 + nm);
    o[0] = v[0];
    o[1] = v[1];
    o[2] = v[2];
    if (nm == 1) o[3] = v[0];
    else if (MOM) {
#pragma unroll
      for (int m = 0; m < 10; ++m)
        if (m < nm) o[3 + m] = v[3 + m];
    }
  }
  const unsigned b = __ballot_sync(0xffffffffu, fix);
  if ((threadIdx.x & 31) == 0 && b) atomicAdd(nfix, (unsigned long long)__popc(b));
}

// ---------------------------------------------------------------------------------------
// host launchers for one output precision
// ---------------------------------------------------------------------------------------
template <typename OT, int KID, bool MOM>
static sph2d_status run_integrals(Ctx* c, IntArgs a) {
  static int grid_blocks = 0;
  if (grid_blocks == 0) {
    int per_sm = 0, sms = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, integrals_kernel<OT, KID, MOM>, 128, 0);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    grid_blocks = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
  }
  constexpr int NV = MOM ? 13 : 3;
  const int64_t nchunks = (a.P + 31) >> 5;
  sph2d_status s = ensure(c, c->slots, size_t(nchunks * 2 * NV + 1) * sizeof(OT));
  if (s != SPH2D_OK) return s;
  a.slots = c->slots.ptr;
  if (a.P > 0) {
    int64_t want = (nchunks + 3) / 4;                    // 4 warps per block
    const unsigned blocks = unsigned(want < grid_blocks ? (want > 0 ? want : 1) : grid_blocks);
    SPH2D_LAUNCH(c, (integrals_kernel<OT, KID, MOM>), blocks, 128, a);
  }
  if (a.N > 0) SPH2D_LAUNCH(c, (finalize_kernel<OT, MOM>), unsigned((a.N + 255) / 256), 256, a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(c, e, "integrals launch");
  return SPH2D_OK;
}

template <typename OT>
static sph2d_status dispatch_integrals(Ctx* c, int kernel, bool mom, IntArgs a) {
  switch (kernel) {
    case KID_WC2: return mom ? run_integrals<OT, KID_WC2, true>(c, a) : run_integrals<OT, KID_WC2, false>(c, a);
    case KID_WC4: return mom ? run_integrals<OT, KID_WC4, true>(c, a) : run_integrals<OT, KID_WC4, false>(c, a);
    case KID_WC6: return mom ? run_integrals<OT, KID_WC6, true>(c, a) : run_integrals<OT, KID_WC6, false>(c, a);
    default: return mom ? run_integrals<OT, KID_CUBIC, true>(c, a) : run_integrals<OT, KID_CUBIC, false>(c, a);
  }
}

template <typename OT>
static sph2d_status dispatch_pairs(Ctx* c, const double* pairs, int64_t P, int kernel, double H,
                                   int deg, unsigned long long* nfix, void* out) {
  const int nm = num_moments(deg);
  const bool mom = deg >= 1;
  const double invH = 1.0 / H, C = kernel_C(kernel);
  const unsigned blocks = unsigned((P + 255) / 256);
  if (P == 0) return SPH2D_OK;
  OT* o = static_cast<OT*>(out);
#define SPH2D_PE(K, MM) SPH2D_LAUNCH(c, (pair_entry_kernel<OT, K, MM>), blocks, 256, pairs, P, invH, C, nm, o, nfix)
  switch (kernel) {
    case KID_WC2: if (mom) SPH2D_PE(KID_WC2, true); else SPH2D_PE(KID_WC2, false); break;
    case KID_WC4: if (mom) SPH2D_PE(KID_WC4, true); else SPH2D_PE(KID_WC4, false); break;
    case KID_WC6: if (mom) SPH2D_PE(KID_WC6, true); else SPH2D_PE(KID_WC6, false); break;
    default: if (mom) SPH2D_PE(KID_CUBIC, true); else SPH2D_PE(KID_CUBIC, false); break;
  }
#undef SPH2D_PE
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(c, e, "pair integrals launch");
  return SPH2D_OK;
}

}  // namespace sph2d
