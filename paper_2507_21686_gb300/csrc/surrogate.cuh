// Learned surrogate for the per-pair integrals (gamma, grad gamma) with a guarded analytic
// fallback.  This part has no counterpart in the paper: it is a small MLP evaluated on BF16
// tensor cores (FP32 accumulation) that replaces the closed form for pairs inside the domain
// it was trained on; every other pair goes to the analytic path.
//
// Canonical frame.  The pair's triangle in the particle frame (H = 1) is rotated so that its
// centroid lies on the +x axis and reflected (y -> -y) if its vertex closest to the particle
// then lies below the axis; its vertices are listed counter-clockwise starting from that
// closest one.  The result depends on the triangle as a point set only.  gamma is invariant
// under the rotation and the reflection; the gradient is mapped back by their inverses.
//
// Network.  6 inputs (canonical vertices) -> 64 -> 64 -> 64 -> 3, tanh-GELU, predicting the
// triangle-averaged kernel and kernel gradient (gamma/area, grad/area); multiplying by the
// exactly computed area removes most of the dynamic range the network would otherwise have to
// learn.  Parameters are FP32 masters.  Forward tensor-core operands (inference and the
// training forward) are FP16 and the GELU between layers is evaluated in packed FP16
// arithmetic on the FP32 accumulators rounded to FP16, so training sees exactly the function
// inference evaluates; the backward GEMMs use BF16 operands (gradients span many decades).
// All accumulation is FP32.
//
// Guard.  A pair is evaluated by the network only if its canonical triangle lies in the
// training domain: largest edge in [kSurMinSize, kSurMaxSize] H, smallest angle >= 15 deg,
// centroid at least kSurMinCentroid H from the particle (the canonical rotation is unstable
// near the centroid), all vertices within kSurMaxRadius H.  Everything else is analytic.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "pair_math.cuh"

namespace sph2d {

constexpr int kSurIn = 6, kSurHid = 64, kSurOut = 3;
constexpr int kSurK1 = 16;     // layer-1 reduction padded to one k16 step
constexpr int kSurN4 = 8;      // output layer padded to one n8 tile
// FP32 master parameter layout (flat): W1[64][6] b1[64] W2[64][64] b2[64] W3[64][64] b3[64]
// W4[3][64] b4[3]
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kSurHid * kSurIn;
constexpr int kOffW2 = kOffB1 + kSurHid, kOffB2 = kOffW2 + kSurHid * kSurHid;
constexpr int kOffW3 = kOffB2 + kSurHid, kOffB3 = kOffW3 + kSurHid * kSurHid;
constexpr int kOffW4 = kOffB3 + kSurHid, kOffB4 = kOffW4 + kSurOut * kSurHid;
constexpr int kSurParams = kOffB4 + kSurOut;   // 8963

constexpr float kSurMinSize = 0.1f, kSurMaxSize = 0.45f;
constexpr float kSurMinCentroid = 0.3f, kSurMaxRadius = 1.5f;
constexpr float kSurSinMinAngle = 0.25881904510252074f;   // sin 15 deg

struct Canon {
  float x[6];          // canonical vertices
  float cs, sn;        // rotation taking the centroid direction to +x
  float refl;          // +1 or -1 (reflection y -> -y applied after the rotation)
  float area;
  bool accept;         // inside the surrogate's domain
};

SPH2D_HD float rsqrt_canon(float x) {
#if defined(__CUDA_ARCH__)
  return rsqrtf(x);
#else
  return 1.0f / sqrtf(x);
#endif
}

SPH2D_HD Canon canonicalize(const float* v) {
  Canon c;
  const float cx = (v[0] + v[2] + v[4]) * (1.0f / 3.0f), cy = (v[1] + v[3] + v[5]) * (1.0f / 3.0f);
  const float r2 = cx * cx + cy * cy;
  const float rinv = r2 > 0.0f ? rsqrt_canon(r2) : 0.0f;
  c.cs = r2 > 0.0f ? cx * rinv : 1.0f;
  c.sn = r2 > 0.0f ? cy * rinv : 0.0f;
  float q[6];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    q[2 * j] = c.cs * v[2 * j] + c.sn * v[2 * j + 1];
    q[2 * j + 1] = -c.sn * v[2 * j] + c.cs * v[2 * j + 1];
  }
  const float cr = diff_of_products(q[2] - q[0], q[5] - q[1], q[3] - q[1], q[4] - q[0]);
  // closest vertex to the particle (lowest index on ties); the mirror image y -> -y is taken
  // when that vertex lies below the axis, so the canonical triangle depends on the geometry
  // only, not on how its vertices are labelled
  const float d0 = q[0] * q[0] + q[1] * q[1], d1 = q[2] * q[2] + q[3] * q[3], d2 = q[4] * q[4] + q[5] * q[5];
  const int k = (d1 < d0 && d1 <= d2) ? 1 : ((d2 < d0 && d2 < d1) ? 2 : 0);
  c.refl = q[2 * k + 1] < 0.0f ? -1.0f : 1.0f;
  // counter-clockwise order from the closest vertex: forward if the (reflected) labelled
  // order is counter-clockwise, backward otherwise
  const int step = (c.refl * cr < 0.0f) ? 2 : 1;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const int s = (k + step * j) % 3;
    c.x[2 * j] = q[2 * s];
    c.x[2 * j + 1] = c.refl * q[2 * s + 1];
  }
  c.area = 0.5f * fabsf(cr);
  // domain guard on squared quantities (no division or square root): edge lengths L_e^2,
  // and sin(angle at a vertex) = 2 area / (product of its edges), compared squared
  float L[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const int b = e == 2 ? 0 : e + 1;
    const float ex = c.x[2 * b] - c.x[2 * e], ey = c.x[2 * b + 1] - c.x[2 * e + 1];
    L[e] = ex * ex + ey * ey;
  }
  const float lmax2 = fmaxf(L[0], fmaxf(L[1], L[2]));
  const float cr2 = cr * cr, sm2 = kSurSinMinAngle * kSurSinMinAngle;
  const bool angles = cr2 >= sm2 * (L[0] * L[2]) && cr2 >= sm2 * (L[0] * L[1]) && cr2 >= sm2 * (L[1] * L[2]);
  const float rmax2 = fmaxf(d0, fmaxf(d1, d2));
  c.accept = c.area > 0.0f && lmax2 >= kSurMinSize * kSurMinSize && lmax2 <= kSurMaxSize * kSurMaxSize &&
             angles && r2 >= kSurMinCentroid * kSurMinCentroid && rmax2 <= kSurMaxRadius * kSurMaxRadius &&
             isfinite(c.area) && isfinite(r2);
  return c;
}

// canonical gradient -> particle frame
SPH2D_HD void uncanonicalize_grad(const Canon& c, float gx_c, float gy_c, float& gx, float& gy) {
  const float gy_r = c.refl * gy_c;
  gx = c.cs * gx_c - c.sn * gy_r;
  gy = c.sn * gx_c + c.cs * gy_r;
}

// derivative of the tanh-form GELU (backward pass, FP32).  On the device tanh is the hardware
// approximation tanh.approx.f32 (relative error about 2^-11).
SPH2D_HD float tanh_act(float u) {
#if defined(__CUDA_ARCH__)
  float t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(u));
  return t;
#else
  return tanhf(u);
#endif
}
SPH2D_HD float gelu_grad_f(float z) {
  const float k = 0.7978845608028654f;
  const float u = k * z * (1.0f + 0.044715f * z * z);
  const float t = tanh_act(u);
  return 0.5f * (1.0f + t) + 0.5f * z * (1.0f - t * t) * k * (1.0f + 3.0f * 0.044715f * z * z);
}

#if defined(__CUDACC__)
// m16n8k16 tensor-core MMA, FP32 accumulation (row.col), BF16 or FP16 operands
__device__ __forceinline__ void mma_16816(float* d, const uint32_t* a, const uint32_t* b, __nv_bfloat16) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
__device__ __forceinline__ void mma_16816(float* d, const uint32_t* a, const uint32_t* b, __half) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
__device__ __forceinline__ __nv_bfloat16 to_op(float v, __nv_bfloat16) { return __float2bfloat16_rn(v); }
__device__ __forceinline__ __half to_op(float v, __half) { return __float2half_rn(v); }

__device__ __forceinline__ uint32_t h2_bits(__half2 v) { return *reinterpret_cast<const uint32_t*>(&v); }
__device__ __forceinline__ uint32_t pack_f16(float lo, float hi) { return h2_bits(__floats2half2_rn(lo, hi)); }

// four 8x8 b16 matrices from shared memory; lane l gives the address of row (l & 7) of
// matrix (l >> 3); register i of every lane receives its fragment of matrix i
__device__ __forceinline__ void ldsm_x4(uint32_t* r, const void* smem_row) {
  const unsigned addr = static_cast<unsigned>(__cvta_generic_to_shared(smem_row));
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}

// tanh-form GELU on a packed FP16 pair: g = h + h tanh(u), h = z/2, u = k z (1 + a z^2).
// For |z| > 255, z^2 overflows to inf, tanh(u) = +-1 and g is z or 0 as the limit requires.
__device__ __forceinline__ __half2 tanh_u_h2(__half2 z) {
  const __half2 k = __float2half2_rn(0.7978845608028654f);
  const __half2 ka = __float2half2_rn(0.7978845608028654f * 0.044715f);
  const __half2 u = __hmul2(__hfma2(__hmul2(z, z), ka, k), z);
  uint32_t t;
  asm("tanh.approx.f16x2 %0, %1;" : "=r"(t) : "r"(h2_bits(u)));
  return *reinterpret_cast<const __half2*>(&t);
}
__device__ __forceinline__ __half2 gelu_h2(__half2 z) {
  const __half2 h = __hmul2(z, __float2half2_rn(0.5f));
  return __hfma2(h, tanh_u_h2(z), h);
}
// 2 GELU(z) = z + z tanh(u): the same value times two, exactly (scaling by 2 commutes with
// every FP16 rounding above, outside the subnormal range); inference folds the 1/2 into the
// next layer's weights
__device__ __forceinline__ __half2 gelu2x_h2(__half2 z) { return __hfma2(z, tanh_u_h2(z), z); }

// m16n8k16 FP16 MMA whose accumulator input is a per-column bias (bx, by) of the lane's two
// columns, for both of its rows
__device__ __forceinline__ void mma_16816_bias(float* d, const uint32_t* a, const uint32_t* b, float bx, float by) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%10,%11,%10,%11};\n"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]), "f"(bx), "f"(by));
}
#endif

}  // namespace sph2d
