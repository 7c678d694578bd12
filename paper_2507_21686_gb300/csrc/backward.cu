// Adjoint of the boundary integrals for a loss L(gamma, grad gamma).
//
//   dL/dx_i  = dL/dgamma_i grad gamma_i + (d grad gamma_i / d x_i)^T dL/dgrad gamma_i
//   dL/dnu_j = sum_i dL/dgamma_i d gamma_i / d nu_j + (d grad gamma_i / d nu_j)^T dL/dgrad gamma_i
// with d gamma_i / d nu_j the transport-theorem edge integral and d grad gamma / d nu_j its
// second-order counterpart (pair_math.cuh); d grad gamma_i / d x_i = -sum_j d grad gamma_i /
// d nu_j.  The vertex gradients are summed triangle-major: the particle-major pair list is
// transposed into per-triangle lists of pair indices, each sorted ascending (= particle
// order); warps take 32 consecutive entries of that list and reduce them with segmented sums
// by triangle (vertex_grad_kernel); the second-order particle terms are written per pair and
// summed particle-major in pair order.  Results do not depend on scheduling.  Nothing from the forward call is
// stored: pair geometry is recomputed.
#include <cuda_runtime.h>

#include "integrals_impl.cuh"

namespace sph2d {

struct BwdArgs {
  const float4* parts;
  const float* tris;
  const int64_t* tri_off;
  const int32_t* tri_q;       // per-triangle pair indices, ascending
  const int32_t* pair_pid;
  const int32_t* pair_tri;
  int64_t M, P;
  void* slots;                // per-chunk partial sums of triangles that cross chunks
  unsigned long long* work;   // zeroed chunk counter
  double invH, C;
  const void* d_gamma;
  const void* d_grad;         // [N][2] or null
  void* d_tris;
  void* pair_terms;           // [P][3] second-order particle terms (0, x, y) or null
  unsigned long long* nfix;
};

// d gamma / d vertices of one pair in the mode's precision; returns 1 if FP64 was used
template <typename OT, int KID>
__device__ __forceinline__ int pair_vertex_grad(const BwdArgs& a, int pid, const float* t, OT* g) {
  return vertex_grad_pair<OT, KID>(a.parts[pid], t, a.invH, a.C, g);
}

// vertex gradients pair-parallel over the triangle-sorted pair list: 32 consecutive positions
// per warp chunk (taken dynamically), each lane one pair's weighted vertex gradients, segmented
// suffix sums by triangle; a triangle whose pairs lie in one chunk is written here, the partial
// sums of triangles that cross chunks go to per-chunk slots (the chunk's first and last
// segment) for tri_finalize_kernel.  The order of every sum is fixed by the list.
template <typename OT, int KID, bool SECOND>
__global__ void __launch_bounds__(128) vertex_grad_kernel(BwdArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t nchunks = (a.P + 31) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  const OT* dg = static_cast<const OT*>(a.d_gamma);
  const OT* dgr = static_cast<const OT*>(a.d_grad);
  unsigned long long fixes = 0;
  for (int64_t ch = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; ch < nchunks;) {
    const unsigned long long nx = chunk_prefetch(a.work);
    const int64_t k = ch * 32 + lane;
    int t = -1;
    OT v[6] = {OT(0), OT(0), OT(0), OT(0), OT(0), OT(0)};
    if (k < a.P) {
      const int32_t q = __ldg(a.tri_q + k);
      const int pid = __ldg(a.pair_pid + q);
      t = __ldg(a.pair_tri + q);
      const float* tp = a.tris + 6 * int64_t(t);
      OT g[6];
      fixes += pair_vertex_grad<OT, KID>(a, pid, tp, g);
      const OT w = dg[pid];
#pragma unroll
      for (int i = 0; i < 6; ++i) v[i] = w * g[i];
      if (SECOND) {
        OT J[12];
        fixes += grad_jacobian_pair<OT, KID>(a.parts[pid], tp, a.invH, a.C, J);
        const OT Gx = dgr[2 * pid], Gy = dgr[2 * pid + 1];
        OT hx = OT(0), hy = OT(0);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          // (J_j^T G)_a = sum_b J[j][b][a] G_b
          const OT vx = J[4 * j + 0] * Gx + J[4 * j + 2] * Gy;
          const OT vy = J[4 * j + 1] * Gx + J[4 * j + 3] * Gy;
          v[2 * j] += vx;
          v[2 * j + 1] += vy;
          hx -= vx;
          hy -= vy;
        }
        OT* pt = static_cast<OT*>(a.pair_terms) + 3 * int64_t(q);
        pt[0] = OT(0);
        pt[1] = hx;
        pt[2] = hy;
      }
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int tn = __shfl_down_sync(0xffffffffu, t, o);
      const bool same = (lane + o < 32) && (tn == t);
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        const OT x = __shfl_down_sync(0xffffffffu, v[i], o);
        if (same) v[i] += x;
      }
    }
    const int tprev = __shfl_up_sync(0xffffffffu, t, 1);
    const bool head = t >= 0 && (lane == 0 || tprev != t);
    const unsigned heads = __ballot_sync(0xffffffffu, head);
    const int last_head = 31 - __clz(heads);
    if (head) {
      const int64_t cs = ch * 32;
      const int64_t s0 = __ldg(a.tri_off + t), s1 = __ldg(a.tri_off + t + 1);
      if (s0 >= cs && s1 <= cs + 32) {
        OT* out = static_cast<OT*>(a.d_tris) + 6 * int64_t(t);
#pragma unroll
        for (int i = 0; i < 6; ++i) out[i] = v[i];
      }
      OT* slots = static_cast<OT*>(a.slots);
      if (lane == 0) {
#pragma unroll
        for (int i = 0; i < 6; ++i) slots[(ch * 2) * 6 + i] = v[i];
      }
      if (lane == last_head) {
#pragma unroll
        for (int i = 0; i < 6; ++i) slots[(ch * 2 + 1) * 6 + i] = v[i];
      }
    }
    ch = chunk_next(a.work, ch, nw, nx);
  }
  if ((threadIdx.x & 31) == 0 && fixes) atomicAdd(a.nfix, fixes);
}

// triangles without pairs get zeros; triangles whose pairs cross chunks add their partials in
// chunk order
template <typename OT>
__global__ void tri_finalize_kernel(const int64_t* __restrict__ tri_off, int64_t M, const OT* __restrict__ slots,
                                    OT* __restrict__ d_tris) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= M) return;
  const int64_t s0 = tri_off[t], s1 = tri_off[t + 1];
  OT v[6] = {OT(0), OT(0), OT(0), OT(0), OT(0), OT(0)};
  if (s1 > s0) {
    const int64_t c0 = s0 >> 5, c1 = (s1 - 1) >> 5;
    if (c0 == c1) return;
#pragma unroll
    for (int i = 0; i < 6; ++i) v[i] = slots[(c0 * 2 + 1) * 6 + i];
    for (int64_t cc = c0 + 1; cc < c1; ++cc) {
#pragma unroll
      for (int i = 0; i < 6; ++i) v[i] += slots[(cc * 2) * 6 + i];
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) v[i] += slots[(c1 * 2) * 6 + i];
  }
  OT* out = d_tris + 6 * t;
#pragma unroll
  for (int i = 0; i < 6; ++i) out[i] = v[i];
}

__global__ void tri_pair_count_kernel(const int32_t* __restrict__ pair_tri, int64_t P,
                                      unsigned long long* __restrict__ cnt) {
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q < P) atomicAdd(cnt + pair_tri[q], 1ull);
}

// per-triangle lists of pair indices (particle-major pair order = ascending particle)
__global__ void tri_pair_fill_kernel(const int32_t* __restrict__ pair_tri, int64_t P,
                                     const int64_t* __restrict__ tri_off,
                                     unsigned long long* __restrict__ cursor, int32_t* __restrict__ tri_q) {
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= P) return;
  const int32_t t = pair_tri[q];
  const unsigned long long k = atomicAdd(cursor + t, 1ull);
  tri_q[tri_off[t] + int64_t(k)] = int32_t(q);
}

// dL/dx_i = dL/dgamma_i grad gamma_i (+ the summed second-order terms when given)
template <typename OT>
__global__ void particle_grad_kernel(const OT* __restrict__ dg, const OT* __restrict__ grad, int64_t N,
                                     const OT* __restrict__ second, OT* __restrict__ dp) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= N) return;
  OT x = dg[i] * grad[2 * i], y = dg[i] * grad[2 * i + 1];
  if (second) {
    x += second[2 * i];
    y += second[2 * i + 1];
  }
  dp[2 * i] = x;
  dp[2 * i + 1] = y;
}

template <typename OT, int KID, bool SECOND>
static void launch_vertex_grads(Ctx* c, const BwdArgs& a) {
  int per_sm = 0, sms = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, vertex_grad_kernel<OT, KID, SECOND>, 128, 0);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  const int64_t cap = int64_t(per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
  const int64_t want = (((a.P + 31) >> 5) + 3) / 4;
  if (a.P > 0) SPH2D_LAUNCH(c, (vertex_grad_kernel<OT, KID, SECOND>), unsigned(want < cap ? want : cap), 128, a);
  SPH2D_LAUNCH(c, (tri_finalize_kernel<OT>), unsigned((a.M + 255) / 256), 256, a.tri_off, a.M,
               static_cast<const OT*>(a.slots), static_cast<OT*>(a.d_tris));
}

template <typename OT>
static sph2d_status run_vertex_grads(Ctx* c, int kernel, BwdArgs a) {
  if (a.M == 0) return SPH2D_OK;
  const int64_t nchunks = (a.P + 31) >> 5;
  sph2d_status s = ensure(c, c->slots, size_t(nchunks * 2 * 6 + 1) * sizeof(OT));
  if (s != SPH2D_OK) return s;
  a.slots = c->slots.ptr;
  const bool second = a.d_grad != nullptr;
  switch (kernel) {
    case KID_WC2: second ? launch_vertex_grads<OT, KID_WC2, true>(c, a) : launch_vertex_grads<OT, KID_WC2, false>(c, a); break;
    case KID_WC4: second ? launch_vertex_grads<OT, KID_WC4, true>(c, a) : launch_vertex_grads<OT, KID_WC4, false>(c, a); break;
    case KID_WC6: second ? launch_vertex_grads<OT, KID_WC6, true>(c, a) : launch_vertex_grads<OT, KID_WC6, false>(c, a); break;
    default: second ? launch_vertex_grads<OT, KID_CUBIC, true>(c, a) : launch_vertex_grads<OT, KID_CUBIC, false>(c, a); break;
  }
  return SPH2D_OK;
}

// per-particle sums of the per-pair second-order terms [P][3] in pair order -> out [N][2]
template <typename OT>
static sph2d_status sum_pair_terms(Ctx* c, const OT* terms, OT* scratch_n, OT* out) {
  const Cells& cl = c->cells;
  IntArgs r{};
  r.pair_pid = static_cast<const int32_t*>(c->pair_pid.ptr);
  r.pair_off = static_cast<const int64_t*>(c->pair_off.ptr);
  r.P = cl.P;
  r.N = cl.N;
  r.gamma = scratch_n;
  r.grad = out;
  r.mom = nullptr;
  r.nm = 0;
  const int64_t nchunks = (r.P + 31) >> 5;
  sph2d_status s = ensure(c, c->slots, size_t(nchunks * 2 * 3 + 1) * sizeof(OT));
  if (s != SPH2D_OK) return s;
  r.slots = c->slots.ptr;
  if (r.P > 0) {
    int per_sm = 0, sms = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, reduce_pairs_kernel<OT, 0>, 128, 0);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    const int64_t cap = int64_t(per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
    const int64_t want = (nchunks + 3) / 4;
    SPH2D_LAUNCH(c, (reduce_pairs_kernel<OT, 0>), unsigned(want < cap ? want : cap), 128, r, terms);
  }
  if (r.N > 0) SPH2D_LAUNCH(c, (finalize_kernel<OT, 0>), unsigned((r.N + 255) / 256), 256, r);
  return SPH2D_OK;
}

sph2d_status launch_backward(Ctx* c, int kernel, int mode, const void* d_gamma, const void* d_grad,
                             void* d_particles, void* d_tris) {
  const Cells& cl = c->cells;
  const int64_t N = cl.N, M = cl.M, P = cl.P;
  const size_t elem = mode == SPH2D_FP64 ? sizeof(double) : sizeof(float);
  const bool second = d_grad != nullptr;
  cudaStream_t st = c->stream;
  cudaError_t e;
  if (P > (int64_t(1) << 31) - 1)
    return set_err(c, SPH2D_ERR_UNSUPPORTED, "the adjoint indexes pairs with int32: P must be < 2^31");
  // grad gamma recomputed with the forward kernel (gamma itself is not needed)
  sph2d_status s = ensure(c, c->bwd_g, size_t(N > 0 ? N : 1) * elem);
  if (s == SPH2D_OK) s = ensure(c, c->bwd_grad, size_t(2 * (N > 0 ? N : 1)) * elem * (second ? 2 : 1));
  if (s != SPH2D_OK) return s;
  s = launch_integrals(c, kernel, -1, mode, c->bwd_g.ptr, c->bwd_grad.ptr, nullptr);
  if (s != SPH2D_OK) return s;
  void* second_sum = second ? static_cast<char*>(c->bwd_grad.ptr) + size_t(2 * N) * elem : nullptr;
  if (M > 0 && P > 0) {
    // transpose the pair list into per-triangle lists of pair indices, sorted ascending
    s = ensure(c, c->tri_cursor, size_t(M) * sizeof(unsigned long long));
    if (s == SPH2D_OK) s = ensure(c, c->tri_off, size_t(M + 1) * sizeof(int64_t));
    if (s == SPH2D_OK) s = ensure(c, c->tri_pid, size_t(P) * sizeof(int32_t));
    if (s == SPH2D_OK && second) s = ensure(c, c->pair_vals, size_t(P) * 3 * elem);
    if (s != SPH2D_OK) return s;
    auto* cnt = static_cast<unsigned long long*>(c->tri_cursor.ptr);
    auto* toff = static_cast<int64_t*>(c->tri_off.ptr);
    auto* tq = static_cast<int32_t*>(c->tri_pid.ptr);
    e = cudaMemsetAsync(cnt, 0, size_t(M) * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return cuda_err(c, e, "memset");
    const unsigned pb = unsigned((P + 255) / 256);
    const int32_t* ptri = static_cast<const int32_t*>(c->pair_tri.ptr);
    SPH2D_LAUNCH(c, (tri_pair_count_kernel), pb, 256, ptri, P, cnt);
    s = exclusive_scan_i64(c, reinterpret_cast<const int64_t*>(cnt), toff, M);
    if (s != SPH2D_OK) return s;
    e = cudaMemsetAsync(cnt, 0, size_t(M) * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return cuda_err(c, e, "memset");
    SPH2D_LAUNCH(c, (tri_pair_fill_kernel), pb, 256, ptri, P, toff, cnt, tq);
    s = launch_sort_segments(c, toff, tq, M);
    if (s != SPH2D_OK) return s;
    // vertex gradients: segmented per-triangle sums over the transposed list
    s = ensure(c, c->host_flags_dev, 64);
    if (s != SPH2D_OK) return s;
    BwdArgs a;
    a.parts = reinterpret_cast<const float4*>(cl.particles);
    a.tris = cl.tris;
    a.tri_off = toff;
    a.tri_q = tq;
    a.pair_pid = static_cast<const int32_t*>(c->pair_pid.ptr);
    a.pair_tri = ptri;
    a.M = M;
    a.P = P;
    a.invH = 1.0 / cl.H;
    a.C = kernel_C(kernel);
    a.d_gamma = d_gamma;
    a.d_grad = d_grad;
    a.d_tris = d_tris;
    a.pair_terms = second ? c->pair_vals.ptr : nullptr;
    a.nfix = static_cast<unsigned long long*>(c->host_flags_dev.ptr) + 2;
    a.work = a.nfix + 1;                               // chunk counter
    e = cudaMemsetAsync(a.nfix, 0, 2 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return cuda_err(c, e, "memset");
    s = mode == SPH2D_FP64 ? run_vertex_grads<double>(c, kernel, a) : run_vertex_grads<float>(c, kernel, a);
    if (s != SPH2D_OK) return s;
    if (second) {
      s = mode == SPH2D_FP64
              ? sum_pair_terms<double>(c, static_cast<const double*>(c->pair_vals.ptr),
                                       static_cast<double*>(c->bwd_g.ptr), static_cast<double*>(second_sum))
              : sum_pair_terms<float>(c, static_cast<const float*>(c->pair_vals.ptr),
                                      static_cast<float*>(c->bwd_g.ptr), static_cast<float*>(second_sum));
      if (s != SPH2D_OK) return s;
    }
  } else {
    if (M > 0) {
      e = cudaMemsetAsync(d_tris, 0, size_t(M) * 6 * elem, st);
      if (e != cudaSuccess) return cuda_err(c, e, "memset");
    }
    if (second && N > 0) {
      e = cudaMemsetAsync(second_sum, 0, size_t(2 * N) * elem, st);
      if (e != cudaSuccess) return cuda_err(c, e, "memset");
    }
  }
  if (N > 0) {
    const unsigned b = unsigned((N + 255) / 256);
    if (mode == SPH2D_FP64)
      SPH2D_LAUNCH(c, (particle_grad_kernel<double>), b, 256, static_cast<const double*>(d_gamma),
                   static_cast<const double*>(c->bwd_grad.ptr), N, static_cast<const double*>(second_sum),
                   static_cast<double*>(d_particles));
    else
      SPH2D_LAUNCH(c, (particle_grad_kernel<float>), b, 256, static_cast<const float*>(d_gamma),
                   static_cast<const float*>(c->bwd_grad.ptr), N, static_cast<const float*>(second_sum),
                   static_cast<float*>(d_particles));
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(c, e, "backward launch");
  return SPH2D_OK;
}

}  // namespace sph2d
