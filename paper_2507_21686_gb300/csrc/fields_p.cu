// Lagrange boundary fields of order 2 and 3 (P2: 6 nodes, P3: 10 nodes per triangle; the
// node order and the closed form are described in field_p_math.cuh).
//
// Precision.  The closed form writes the field as monomials about the particle, so its
// rounding error grows like (|p|max |grad lambda|)^k against the field scale: a triangle
// small against its distance loses (distance / size)^k digits (the fan decomposition's own
// cancellation, raised to the field's degree).  FP64 keeps ~1e-11 (P3) on meshes of H/3
// elements; FP32 does not reach 1e-5 for P3 even near the particle.  So:
//   SPH2D_FP64         the closed form in FP64 for every pair (double outputs);
//   SPH2D_FP32_HYBRID  the 6 x 6 quadrature of the hybrid mode, in FP32, for pairs at least
//                      half their longest edge from the particle (inside the support or across
//                      its edge below the kernel's size limit; the cubic spline only beyond
//                      H/2 or inside it), where the field is evaluated from its barycentric
//                      form at each node; the closed form in FP64 for the rest (float outputs).
// The hybrid pass writes per-pair values, the FP64 closed form fills the listed pairs, and a
// pair-order segmented sum gives per-particle results (deterministic).
#include <cuda_runtime.h>

#include "field_p_math.cuh"
#include "fields_common.cuh"
#include "quad.cuh"

namespace sph2d {

// node index of rotated position n when the rule's apex is vertex `rot` (a cyclic relabelling
// maps vertices to vertices and edges to edges, keeping each edge's direction)
template <int ORDER>
__device__ __forceinline__ int rotated_node(int n, int rot) {
  if (n < 3) return n + rot >= 3 ? n + rot - 3 : n + rot;
  if (ORDER == 2) return 3 + (n - 3 + rot >= 3 ? n - 3 + rot - 3 : n - 3 + rot);
  if (n == 9) return 9;
  const int e = (n - 3) >> 1, w = (n - 3) & 1;
  const int er = e + rot >= 3 ? e + rot - 3 : e + rot;
  return 3 + 2 * er + w;
}

// the homogeneous barycentric coefficients of field k in the rotated labelling
template <int ORDER>
__device__ __forceinline__ void bary_rotated(const float* A, int nf, int rot, float* B) {
  constexpr int NB = nodes_of(ORDER);
  float An[NB];
#pragma unroll
  for (int n = 0; n < NB; ++n) An[n] = __ldg(A + rotated_node<ORDER>(n, rot) * nf);
  lagrange_to_bary<float, ORDER>(An, 1, B);
}

// barycentric monomials (order of lagrange_to_bary) at (m0, m1, m2)
template <int ORDER>
__device__ __forceinline__ void bary_values(float m0, float m1, float m2, float* mono) {
  if (ORDER == 2) {
    mono[0] = m0 * m0;
    mono[1] = m1 * m1;
    mono[2] = m2 * m2;
    mono[3] = m0 * m1;
    mono[4] = m1 * m2;
    mono[5] = m2 * m0;
  } else {
    const float a = m0 * m0, b = m1 * m1, c = m2 * m2;
    mono[0] = a * m0;
    mono[1] = b * m1;
    mono[2] = c * m2;
    mono[3] = a * m1;
    mono[4] = m0 * b;
    mono[5] = b * m2;
    mono[6] = m1 * c;
    mono[7] = c * m0;
    mono[8] = m2 * a;
    mono[9] = m0 * m1 * m2;
  }
}

// quadrature of nf fields over one pair (rule and apex of quad_classify) -> out[3 f + {0,1,2}]
template <int KID, int ORDER>
__device__ __forceinline__ void field_p_quad(const QuadRule& qr, const float* vin, const QuadClass& qc,
                                             const float* A, int nf, double C, double invH, bool grad,
                                             float* out) {
  constexpr int NB = nodes_of(ORDER);
  const int i0 = qc.apex, i1 = i0 == 2 ? 0 : i0 + 1, i2 = i1 == 2 ? 0 : i1 + 1;
  float B[kMaxFields][NB];
#pragma unroll
  for (int k = 0; k < kMaxFields; ++k)
    if (k < nf) bary_rotated<ORDER>(A + k, nf, i0, B[k]);
  const float v0x = vin[2 * i0], v0y = vin[2 * i0 + 1];
  const float e1x = vin[2 * i1] - v0x, e1y = vin[2 * i1 + 1] - v0y;
  const float e2x = vin[2 * i2] - vin[2 * i1], e2y = vin[2 * i2 + 1] - vin[2 * i1 + 1];
  const float a2 = fabsf(diff_of_products(e1x, vin[2 * i2 + 1] - v0y, e1y, vin[2 * i2] - v0x));
  const float c0 = v0x * v0x + v0y * v0y - 1.0f;
  float acc[3 * kMaxFields];
#pragma unroll
  for (int i = 0; i < 3 * kMaxFields; ++i) acc[i] = 0.0f;
#pragma unroll 1
  for (int j = 0; j < kQuadN; ++j) {
    const float tj = qr.u[j];
    const float dx = e1x + tj * e2x, dy = e1y + tj * e2y;
    const float aa = dx * dx + dy * dy, bb = v0x * dx + v0y * dy;
    const float sp = -c0 / (bb + sqrtf(fmaxf(bb * bb - aa * c0, 0.0f)));
    const float ss = fminf(1.0f, sp);
    const float wj = qr.w[j] * ss * ss;
#pragma unroll 2
    for (int i = 0; i < kQuadN; ++i) {
      const float s = ss * qr.u[i];
      const float px = v0x + s * dx, py = v0y + s * dy;
      const float r = sqrtf(px * px + py * py);
      float k, kd;
      kernel_and_slope<KID>(r, qc.inner, k, kd);
      const float w = wj * qr.wu[i];
      // barycentric coordinates in the rotated labelling: (1 - s, s (1 - t), s t)
      const float st = s * tj;
      float mono[NB];
      bary_values<ORDER>(1.0f - s, s - st, st, mono);
      const float wk = w * k, wdx = w * kd * px, wdy = w * kd * py;
#pragma unroll
      for (int f = 0; f < kMaxFields; ++f) {
        if (f < nf) {
          float av = 0.0f;
#pragma unroll
          for (int b = 0; b < NB; ++b) av = fmaf(B[f][b], mono[b], av);
          acc[3 * f] = fmaf(wk, av, acc[3 * f]);
          acc[3 * f + 1] = fmaf(wdx, av, acc[3 * f + 1]);
          acc[3 * f + 2] = fmaf(wdy, av, acc[3 * f + 2]);
        }
      }
    }
  }
  const float c = float(C) * a2, cg = -c * float(invH);
#pragma unroll
  for (int f = 0; f < kMaxFields; ++f) {
    out[3 * f] = c * acc[3 * f];
    out[3 * f + 1] = grad ? cg * acc[3 * f + 1] : 0.0f;
    out[3 * f + 2] = grad ? cg * acc[3 * f + 2] : 0.0f;
  }
}

// FP64 closed form of one pair -> v[3 kMaxFields]
template <int KID, int ORDER, bool GRAD>
__device__ __forceinline__ void field_p_pair64(const FieldArgs& f, int pid, int tid, double* v) {
  const IntArgs& a = f.a;
  const float4 p = a.parts[pid];
  const float* t = a.tris + 6 * int64_t(tid);
  double l[6];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    l[2 * j] = (double(__ldg(t + 2 * j)) - double(p.x)) * a.invH;
    l[2 * j + 1] = (double(__ldg(t + 2 * j + 1)) - double(p.y)) * a.invH;
  }
  const float* A = f.values + int64_t(tid) * nodes_of(ORDER) * f.nf;
  double B[kMaxFields][nodes_of(3)];
#pragma unroll
  for (int k = 0; k < kMaxFields; ++k) {
    if (k < f.nf) {
      float An[nodes_of(ORDER)];
#pragma unroll
      for (int n = 0; n < nodes_of(ORDER); ++n) An[n] = __ldg(A + n * f.nf + k);
      lagrange_to_bary<double, ORDER>(An, 1, B[k]);
    }
  }
  field_p_local<double, KID, ORDER, GRAD, kMaxFields>(l, B, f.nf, a.C, a.invH, v);
}

// FP64 mode: one warp per 32 consecutive pairs, segmented per-particle sums
template <int KID, int ORDER, bool GRAD>
__global__ void __launch_bounds__(128) field_p_kernel(FieldArgs f) {
  constexpr int NV = 3 * kMaxFields;
  const IntArgs& a = f.a;
  const int64_t nchunks = (a.P + 31) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t ch = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
       ch < nchunks;) {
    const unsigned long long nx = chunk_prefetch(a.work);
    const int64_t q = ch * 32 + (threadIdx.x & 31);
    int pid = -1;
    double v[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = 0.0;
    if (q < a.P) {
      pid = __ldg(a.pair_pid + q);
      field_p_pair64<KID, ORDER, GRAD>(f, pid, __ldg(a.pair_tri + q), v);
    }
    field_warp_sum<double>(f, ch, pid, v);
    ch = chunk_next(a.work, ch, nw, nx);
  }
}

// hybrid mode, pass 1: quadrature for the pairs that qualify into vals[q][3 nf], the others
// appended to list
template <int KID, int ORDER, bool GRAD>
__global__ void __launch_bounds__(128) field_p_quad_kernel(FieldArgs f, QuadRule qr, float* __restrict__ vals,
                                                           int64_t* __restrict__ list,
                                                           unsigned long long* __restrict__ count) {
  const IntArgs& a = f.a;
  const int lane = threadIdx.x & 31;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  const float ih = float(a.invH);
  const int nv = 3 * f.nf;
  const int64_t nchunks = (a.P + 31) >> 5, nw = stride >> 5;
  for (int64_t ch = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; ch < nchunks;) {
    const unsigned long long nx = chunk_prefetch(a.work);
    const int64_t q = ch * 32 + lane;
    bool analytic = false;
    if (q < a.P) {
      const int tid = __ldg(a.pair_tri + q);
      const float4 p = a.parts[__ldg(a.pair_pid + q)];
      const float* t = a.tris + 6 * int64_t(tid);
      float v[6];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        v[2 * j] = (__ldg(t + 2 * j) - p.x) * ih;
        v[2 * j + 1] = (__ldg(t + 2 * j + 1) - p.y) * ih;
      }
      const QuadClass qc = quad_classify<KID>(v);
      // the cubic spline's second piece is not split off here: pairs that straddle r = 1/2
      // take the closed form
      if (qc.quad && !qc.near) {
        float w[3 * kMaxFields];
        field_p_quad<KID, ORDER>(qr, v, qc, f.values + int64_t(tid) * nodes_of(ORDER) * f.nf, f.nf, a.C, a.invH,
                                 GRAD, w);
        float* o = vals + q * nv;
#pragma unroll
        for (int i = 0; i < 3 * kMaxFields; ++i)
          if (i < nv) o[i] = w[i];
      } else {
        analytic = true;
      }
    }
    warp_append(analytic, q, list, count);
    ch = chunk_next(a.work, ch, nw, nx);
  }
}

// hybrid mode, pass 2: the FP64 closed form over the list
template <int KID, int ORDER, bool GRAD>
__global__ void __launch_bounds__(128) field_p_list_kernel(FieldArgs f, float* __restrict__ vals,
                                                           const int64_t* __restrict__ list,
                                                           const unsigned long long* __restrict__ count) {
  const IntArgs& a = f.a;
  const int64_t n = int64_t(*count);
  const int nv = 3 * f.nf;
  const int64_t nchunks = (n + 31) >> 5, nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t ch = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; ch < nchunks;) {
    const unsigned long long nx = chunk_prefetch(a.work);
    const int64_t i = ch * 32 + (threadIdx.x & 31);
    if (i < n) {
      const int64_t q = list[i];
      double v[3 * kMaxFields];
      field_p_pair64<KID, ORDER, GRAD>(f, __ldg(a.pair_pid + q), __ldg(a.pair_tri + q), v);
      float* o = vals + q * nv;
#pragma unroll
      for (int k = 0; k < 3 * kMaxFields; ++k)
        if (k < nv) o[k] = float(v[k]);
    }
    ch = chunk_next(a.work, ch, nw, nx);
  }
}

// hybrid mode, pass 3: per-particle sums of the per-pair values in pair order
__global__ void __launch_bounds__(128) field_p_sum_kernel(FieldArgs f, const float* __restrict__ vals) {
  constexpr int NV = 3 * kMaxFields;
  const IntArgs& a = f.a;
  const int nv = 3 * f.nf;
  const int64_t nchunks = (a.P + 31) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t ch = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; ch < nchunks; ch += nw) {
    const int64_t q = ch * 32 + (threadIdx.x & 31);
    int pid = -1;
    float v[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = 0.0f;
    if (q < a.P) {
      pid = __ldg(a.pair_pid + q);
#pragma unroll
      for (int i = 0; i < NV; ++i)
        if (i < nv) v[i] = vals[q * nv + i];
    }
    field_warp_sum<float>(f, ch, pid, v);
  }
}

template <int KID, int ORDER, bool GRAD>
static sph2d_status run_fields_p(Ctx* c, int mode, FieldArgs f) {
  constexpr int NV = 3 * kMaxFields;
  const int64_t nchunks = (f.a.P + 31) >> 5;
  if (mode == SPH2D_FP64) {
    sph2d_status s = ensure(c, c->slots, size_t(nchunks * 2 * NV + 1) * sizeof(double));
    if (s == SPH2D_OK) s = ensure(c, c->host_flags_dev, 64);
    if (s != SPH2D_OK) return s;
    f.a.slots = c->slots.ptr;
    f.a.work = static_cast<unsigned long long*>(c->host_flags_dev.ptr) + 1;   // chunk counter
    cudaError_t e0 = cudaMemsetAsync(f.a.work, 0, sizeof(unsigned long long), c->stream);
    if (e0 != cudaSuccess) return cuda_err(c, e0, "memset");
    if (f.a.P > 0)
      SPH2D_LAUNCH(c, (field_p_kernel<KID, ORDER, GRAD>),
                   resident_blocks(c, field_p_kernel<KID, ORDER, GRAD>, (nchunks + 3) / 4), 128, f);
    if (f.a.N > 0) SPH2D_LAUNCH(c, (field_finalize_kernel<double>), unsigned((f.a.N + 255) / 256), 256, f);
  } else {
    const int64_t cap = f.a.P > 0 ? f.a.P : 1;
    sph2d_status s = ensure(c, c->slots, size_t(nchunks * 2 * NV + 1) * sizeof(float));
    if (s == SPH2D_OK) s = ensure(c, c->pair_vals, size_t(cap) * 3 * f.nf * sizeof(float));
    if (s == SPH2D_OK) s = ensure(c, c->pair_list2, size_t(cap) * sizeof(int64_t) + 64);
    if (s != SPH2D_OK) return s;
    f.a.slots = c->slots.ptr;
    float* vals = static_cast<float*>(c->pair_vals.ptr);
    int64_t* list = reinterpret_cast<int64_t*>(static_cast<char*>(c->pair_list2.ptr) + 64);
    auto* count = static_cast<unsigned long long*>(c->pair_list2.ptr);
    cudaError_t e = cudaMemsetAsync(count, 0, 64, c->stream);   // list length, chunk counters
    if (e != cudaSuccess) return cuda_err(c, e, "memset");
    if (f.a.P > 0) {
      const int64_t blocks = (f.a.P + 127) / 128;
      FieldArgs fq = f, fl = f;
      fq.a.work = count + 4;
      fl.a.work = count + 5;
      SPH2D_LAUNCH(c, (field_p_quad_kernel<KID, ORDER, GRAD>),
                   resident_blocks(c, field_p_quad_kernel<KID, ORDER, GRAD>, blocks), 128, fq, quad_rule(), vals, list,
                   count);
      SPH2D_LAUNCH(c, (field_p_list_kernel<KID, ORDER, GRAD>),
                   resident_blocks(c, field_p_list_kernel<KID, ORDER, GRAD>, blocks), 128, fl, vals, list, count);
      SPH2D_LAUNCH(c, field_p_sum_kernel, resident_blocks(c, field_p_sum_kernel, (nchunks + 3) / 4), 128, f, vals);
    }
    if (f.a.N > 0) SPH2D_LAUNCH(c, (field_finalize_kernel<float>), unsigned((f.a.N + 255) / 256), 256, f);
    e = cudaMemcpyAsync(c->pinned + 10, count, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_err(c, e, "fallback count copy");
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(c, e, "field integrals launch");
  return SPH2D_OK;
}

template <int ORDER, bool GRAD>
static sph2d_status dispatch_fields_p(Ctx* c, int kernel, int mode, const FieldArgs& f) {
  switch (kernel) {
    case KID_WC2: return run_fields_p<KID_WC2, ORDER, GRAD>(c, mode, f);
    case KID_WC4: return run_fields_p<KID_WC4, ORDER, GRAD>(c, mode, f);
    case KID_WC6: return run_fields_p<KID_WC6, ORDER, GRAD>(c, mode, f);
    default: return run_fields_p<KID_CUBIC, ORDER, GRAD>(c, mode, f);
  }
}

sph2d_status launch_fields_p(Ctx* c, int kernel, int mode, int order, const float* values, int nf, void* value,
                             void* grad) {
  const Cells& cl = c->cells;
  FieldArgs f{};
  IntArgs& a = f.a;
  a.parts = reinterpret_cast<const float4*>(cl.particles);
  a.tris = cl.tris;
  a.pair_tri = static_cast<const int32_t*>(c->pair_tri.ptr);
  a.pair_pid = static_cast<const int32_t*>(c->pair_pid.ptr);
  a.pair_off = static_cast<const int64_t*>(c->pair_off.ptr);
  a.P = cl.P;
  a.N = cl.N;
  a.H = cl.H;
  a.invH = 1.0 / cl.H;
  a.C = kernel_C(kernel);
  f.values = values;
  f.nf = nf;
  f.value = value;
  f.grad = grad;
  const bool g = grad != nullptr;
  sph2d_status s;
  if (order == 2) s = g ? dispatch_fields_p<2, true>(c, kernel, mode, f) : dispatch_fields_p<2, false>(c, kernel, mode, f);
  else s = g ? dispatch_fields_p<3, true>(c, kernel, mode, f) : dispatch_fields_p<3, false>(c, kernel, mode, f);
  if (s != SPH2D_OK) return s;
  c->stats.n_pairs = cl.P;
  c->stats.n_fixup = 0;
  c->stats.n_fallback = 0;
  c->fixup_pending = false;
  c->fallback_pending = mode == SPH2D_FP32_HYBRID;
  return SPH2D_OK;
}

}  // namespace sph2d
