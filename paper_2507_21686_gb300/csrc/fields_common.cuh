// Shared parts of the boundary-field passes: arguments, the per-particle writer and the
// finalize pass that adds partial sums of particles whose pairs cross warp chunks.
#pragma once

#include "integrals_impl.cuh"

namespace sph2d {

constexpr int kMaxFields = 4;

struct FieldArgs {
  IntArgs a;              // pair list, geometry, kernel constants (a.gamma etc. unused)
  const float* values;    // [M][nodes][nf] (3 nodes: linear; 6 or 10: order 2 or 3)
  int nf;
  void* value;            // [N][nf]
  void* grad;             // [N][nf][2] or null
};

template <typename OT>
__device__ __forceinline__ void write_fields(const FieldArgs& f, int64_t pid, const OT* v) {
  OT* val = static_cast<OT*>(f.value) + pid * f.nf;
  OT* gr = f.grad ? static_cast<OT*>(f.grad) + pid * f.nf * 2 : nullptr;
#pragma unroll
  for (int k = 0; k < kMaxFields; ++k) {
    if (k < f.nf) {
      val[k] = v[3 * k];
      if (gr) {
        gr[2 * k] = v[3 * k + 1];
        gr[2 * k + 1] = v[3 * k + 2];
      }
    }
  }
}

// segmented per-particle sum of one warp chunk (32 consecutive pairs, lane values v[3 kMaxFields],
// pid = -1 past the end): particles whose pairs all lie in the chunk are written, and the
// chunk's first and last partial sums go to the crossing slots for field_finalize_kernel
template <typename OT>
__device__ __forceinline__ void field_warp_sum(const FieldArgs& f, int64_t ch, int pid, OT* v) {
  constexpr int NV = 3 * kMaxFields;
  const IntArgs& a = f.a;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int pn = __shfl_down_sync(0xffffffffu, pid, o);
    const bool same = (lane + o < 32) && (pn == pid);
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      const OT tv = __shfl_down_sync(0xffffffffu, v[i], o);
      if (same) v[i] += tv;
    }
  }
  const int pprev = __shfl_up_sync(0xffffffffu, pid, 1);
  const bool head = pid >= 0 && (lane == 0 || pprev != pid);
  const unsigned heads = __ballot_sync(0xffffffffu, head);
  const int last_head = 31 - __clz(heads);
  if (head) {
    const int64_t cs = ch * 32;
    const int64_t s0 = __ldg(a.pair_off + pid), s1 = __ldg(a.pair_off + pid + 1);
    if (s0 >= cs && s1 <= cs + 32) write_fields<OT>(f, pid, v);
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

// particles without pairs get zeros; particles whose pairs cross chunks add their partials
template <typename OT>
static __global__ void field_finalize_kernel(FieldArgs f) {
  constexpr int NV = 3 * kMaxFields;
  const IntArgs& a = f.a;
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= a.N) return;
  const int64_t s0 = a.pair_off[i], s1 = a.pair_off[i + 1];
  OT v[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = OT(0);
  if (s1 > s0) {
    const int64_t c0 = s0 >> 5, c1 = (s1 - 1) >> 5;
    if (c0 == c1) return;
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
  write_fields<OT>(f, i, v);
}

}  // namespace sph2d
