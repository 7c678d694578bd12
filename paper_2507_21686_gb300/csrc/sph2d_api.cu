// C-ABI entry points of libsph2d (declared in include/sph2d.h): context handling, argument
// validation, status codes, and the device-wide exclusive scan used by the culling pass.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "sph2d_internal.h"

namespace sph2d {

sph2d_status set_err(Ctx* c, sph2d_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

sph2d_status cuda_err(Ctx* c, cudaError_t e, const char* where) {
  return set_err(c, SPH2D_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

sph2d_status ensure(Ctx* c, DevBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return SPH2D_OK;
  if (b.ptr) {
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_err(c, e, "sync before realloc");
    cudaFree(b.ptr);
    b.ptr = nullptr;
    b.bytes = 0;
  }
  size_t want = bytes + bytes / 4;   // headroom for repeated calls with growing sizes
  cudaError_t e = cudaMalloc(&b.ptr, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b.ptr = nullptr;
    return set_err(c, SPH2D_ERR_OUT_OF_MEMORY,
                   "scratch allocation of " + std::to_string(want) + " bytes failed");
  }
  b.bytes = want;
  return SPH2D_OK;
}

// ---------------------------------------------------------------------------------------
// exclusive scan: tiles of 2048 int64 per 256-thread block, recursive over block totals
// ---------------------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__global__ void scan_tiles(const int64_t* __restrict__ in, int64_t* __restrict__ out, int64_t n,
                           int64_t* __restrict__ block_sums) {
  __shared__ int64_t warp_tot[kScanThreads / 32];
  const int64_t base = int64_t(blockIdx.x) * kScanTile + int64_t(threadIdx.x) * kScanItems;
  int64_t v[kScanItems];
  int64_t run = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t idx = base + i;
    v[i] = idx < n ? in[idx] : 0;
    run += v[i];
  }
  // inclusive scan of thread totals within the warp
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t incl = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int64_t w = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = w;   // inclusive over warps
  }
  __syncthreads();
  int64_t excl = incl - run + (warp > 0 ? warp_tot[warp - 1] : 0);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t idx = base + i;
    if (idx < n) out[idx] = excl;
    excl += v[i];
  }
  if (threadIdx.x == kScanThreads - 1) block_sums[blockIdx.x] = warp_tot[kScanThreads / 32 - 1];
}

__global__ void scan_add(int64_t* __restrict__ out, int64_t n, const int64_t* __restrict__ offs) {
  const int64_t idx = int64_t(blockIdx.x) * kScanTile + threadIdx.x;
  const int64_t add = offs[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t j = idx + int64_t(i) * kScanThreads;
    if (j < n) out[j] += add;
  }
}

__global__ void scan_single(const int64_t* __restrict__ in, int64_t* __restrict__ out, int64_t n) {
  // n <= kScanTile, one block; writes out[0..n] (out[n] = total)
  __shared__ int64_t buf[kScanTile + 1];
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) buf[i] = in[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t s = 0;
    for (int64_t i = 0; i < n; ++i) {
      const int64_t v = buf[i];
      buf[i] = s;
      s += v;
    }
    buf[n] = s;
  }
  __syncthreads();
  for (int64_t i = threadIdx.x; i <= n; i += blockDim.x) out[i] = buf[i];
}

// scan of n values using scratch from offset `level` of c->scan_tmp
static sph2d_status scan_rec(Ctx* c, const int64_t* in, int64_t* out, int64_t n, size_t tmp_off) {
  if (n <= kScanTile) {
    SPH2D_LAUNCH(c, (scan_single), 1, kScanThreads, in, out, n);
    return SPH2D_OK;
  }
  const int64_t nb = (n + kScanTile - 1) / kScanTile;
  int64_t* sums = reinterpret_cast<int64_t*>(static_cast<char*>(c->scan_tmp.ptr) + tmp_off);
  int64_t* sums_scan = sums + nb;
  SPH2D_LAUNCH(c, (scan_tiles), (unsigned)nb, kScanThreads, in, out, n, sums);
  sph2d_status s = scan_rec(c, sums, sums_scan, nb, tmp_off + size_t(2 * nb + 2) * sizeof(int64_t));
  if (s != SPH2D_OK) return s;
  SPH2D_LAUNCH(c, (scan_add), (unsigned)nb, kScanThreads, out, n, sums_scan);
  // total
  cudaMemcpyAsync(out + n, sums_scan + nb, sizeof(int64_t), cudaMemcpyDeviceToDevice, c->stream);
  return SPH2D_OK;
}

sph2d_status exclusive_scan_i64(Ctx* c, const int64_t* in, int64_t* out, int64_t n) {
  // scratch: sum over levels of 2*(nb+1) <= 2*(n/2048 + n/2048^2 + ...) + small
  size_t need = size_t(2 * (n / kScanTile + 8) + 64) * sizeof(int64_t) * 2;
  sph2d_status s = ensure(c, c->scan_tmp, need);
  if (s != SPH2D_OK) return s;
  s = scan_rec(c, in, out, n, 0);
  if (s != SPH2D_OK) return s;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(c, e, "scan launch");
  return SPH2D_OK;
}

static bool valid_kernel(int k) { return k >= SPH2D_WENDLAND_C2 && k <= SPH2D_CUBIC_SPLINE; }

}  // namespace sph2d

using namespace sph2d;

struct sph2d_ctx {
  Ctx c;
};

extern "C" {

int sph2d_version(void) { return 100; }

sph2d_status sph2d_init(sph2d_ctx** out, int device, void* stream) {
  if (!out) return SPH2D_ERR_INVALID_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess) {
    cudaGetLastError();
    return SPH2D_ERR_CUDA;
  }
  if (device < 0 || device >= n) return SPH2D_ERR_INVALID_ARG;
  sph2d_ctx* h = new (std::nothrow) sph2d_ctx();
  if (!h) return SPH2D_ERR_OUT_OF_MEMORY;
  h->c.device = device;
  h->c.stream = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaMallocHost(&h->c.pinned, 64 * sizeof(int64_t));
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return SPH2D_ERR_CUDA;
  }
  *out = h;
  return SPH2D_OK;
}

sph2d_status sph2d_destroy(sph2d_ctx* h) {
  if (!h) return SPH2D_OK;
  Ctx& c = h->c;
  cudaSetDevice(c.device);
  cudaStreamSynchronize(c.stream);
  DevBuf* bufs[] = {&c.cell_start, &c.cell_cursor, &c.cell_tris, &c.block_tmp, &c.scan_tmp,
                    &c.pair_off,  &c.pair_tri,    &c.pair_pid,  &c.counts,    &c.slots,
                    &c.host_flags_dev, &c.misc, &c.tri_off, &c.tri_pid, &c.tri_cursor,
                    &c.bwd_g, &c.bwd_grad, &c.pair_vals, &c.pair_list2, &c.sur_prm, &c.sur_split, &c.sur_act,
                    &c.sur_data, &c.sur_idx, &c.sur_vals, &c.sur_fb, &c.part_start, &c.part_cursor,
                    &c.part_ids, &c.pres_vertex, &c.pres_tmp, &c.cand_off, &c.cand_kept, &c.sort_flag};
  for (DevBuf* b : bufs)
    if (b->ptr) cudaFree(b->ptr);
  if (c.pinned) cudaFreeHost(c.pinned);
  delete h;
  return SPH2D_OK;
}

sph2d_status sph2d_set_stream(sph2d_ctx* h, void* stream) {
  if (!h) return SPH2D_ERR_INVALID_ARG;
  h->c.stream = static_cast<cudaStream_t>(stream);
  return SPH2D_OK;
}

const char* sph2d_last_error(const sph2d_ctx* h) { return h ? h->c.err.c_str() : "null context"; }

sph2d_status sph2d_last_stats(const sph2d_ctx* h, sph2d_stats* out) {
  if (!h || !out) return SPH2D_ERR_INVALID_ARG;
  const Ctx& c = h->c;
  *out = c.stats;
  out->n_launches = c.launches;
  if (c.fixup_pending) {
    cudaSetDevice(c.device);
    cudaError_t e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) return SPH2D_ERR_CUDA;
    out->n_fixup = c.pinned[8];
  }
  if (c.fallback_pending) {
    cudaSetDevice(c.device);
    cudaError_t e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) return SPH2D_ERR_CUDA;
    out->n_fallback = c.pinned[10];
    out->n_audit = c.pinned[11];
    out->n_audit_over = c.pinned[12];
    uint32_t bits = uint32_t(uint64_t(c.pinned[13]) & 0xffffffffu);
    float emax;
    std::memcpy(&emax, &bits, sizeof(emax));
    out->audit_max_err = emax;
    out->n_redo = out->n_audit_over > 0 ? out->n_pairs : 0;
    out->n_mma_timeouts = c.pinned[14];
  }
  return SPH2D_OK;
}

static sph2d_status check_geom(Ctx* c, const float* particles, int64_t N, const float* tris,
                               int64_t M, double H) {
  if (N < 0 || M < 0 || N > (int64_t(1) << 31) - 2 || M > (int64_t(1) << 31) - 2)
    return set_err(c, SPH2D_ERR_INVALID_ARG, "N and M must be in [0, 2^31-2]");
  if ((N > 0 && !particles) || (M > 0 && !tris))
    return set_err(c, SPH2D_ERR_INVALID_ARG, "null particle or triangle pointer");
  if (particles && (reinterpret_cast<uintptr_t>(particles) & 15u))
    return set_err(c, SPH2D_ERR_INVALID_ARG, "particles must be 16-byte aligned (float4)");
  if (tris && (reinterpret_cast<uintptr_t>(tris) & 3u))
    return set_err(c, SPH2D_ERR_INVALID_ARG, "triangles must be 4-byte aligned");
  if (!(H > 0.0) || !std::isfinite(H)) return set_err(c, SPH2D_ERR_INVALID_ARG, "H must be finite and > 0");
  return SPH2D_OK;
}

static sph2d_status check_outputs(Ctx* c, int kernel, int moment_degree, int mode, void* gamma,
                                  void* moments, int64_t N) {
  if (!valid_kernel(kernel)) return set_err(c, SPH2D_ERR_INVALID_ARG, "unknown kernel id");
  if (moment_degree < -1 || moment_degree > 3)
    return set_err(c, SPH2D_ERR_INVALID_ARG, "moment_degree must be -1..3");
  if (mode == SPH2D_SURROGATE) {
    if (moment_degree >= 0)
      return set_err(c, SPH2D_ERR_UNSUPPORTED, "the surrogate provides gamma and grad gamma only");
    if (!c->sur_ready) return set_err(c, SPH2D_ERR_NOT_BUILT, "surrogate not initialised");
    if (kernel != c->sur_kernel)
      return set_err(c, SPH2D_ERR_INVALID_ARG, "the surrogate was initialised for another kernel");
  } else if (mode != SPH2D_FP64 && mode != SPH2D_FP32_FIXUP && mode != SPH2D_FP32_HYBRID) {
    return set_err(c, SPH2D_ERR_INVALID_ARG, "unknown mode");
  }
  if (N > 0 && !gamma) return set_err(c, SPH2D_ERR_INVALID_ARG, "gamma must not be NULL");
  if (moment_degree >= 0 && N > 0 && !moments)
    return set_err(c, SPH2D_ERR_INVALID_ARG, "moments must not be NULL when moment_degree >= 0");
  if (moment_degree < 0 && moments)
    return set_err(c, SPH2D_ERR_INVALID_ARG, "moments must be NULL when moment_degree < 0");
  return SPH2D_OK;
}

sph2d_status sph2d_build_cells(sph2d_ctx* h, const float* particles, int64_t N, const float* tris,
                               int64_t M, double H) {
  if (!h) return SPH2D_ERR_INVALID_ARG;
  Ctx* c = &h->c;
  c->err.clear();
  sph2d_status s = check_geom(c, particles, N, tris, M, H);
  if (s != SPH2D_OK) return s;
  cudaSetDevice(c->device);
  return build_cells(c, particles, N, tris, M, H);
}

sph2d_status sph2d_pair_count(const sph2d_ctx* h, int64_t* n_pairs) {
  if (!h || !n_pairs) return SPH2D_ERR_INVALID_ARG;
  if (!h->c.cells.built) return SPH2D_ERR_NOT_BUILT;
  *n_pairs = h->c.cells.P;
  return SPH2D_OK;
}

sph2d_status sph2d_pair_list(sph2d_ctx* h, int64_t* off, int32_t* tri, int64_t cap,
                             int64_t* required) {
  if (!h) return SPH2D_ERR_INVALID_ARG;
  Ctx* c = &h->c;
  c->err.clear();
  if (!c->cells.built) return set_err(c, SPH2D_ERR_NOT_BUILT, "no pair list built");
  const int64_t P = c->cells.P, N = c->cells.N;
  if (required) *required = P;
  if (!off || (P > 0 && !tri)) return set_err(c, SPH2D_ERR_INVALID_ARG, "null output pointer");
  if (cap < P) return set_err(c, SPH2D_ERR_CAPACITY, "pair buffer too small");
  cudaSetDevice(c->device);
  cudaError_t e = cudaMemcpyAsync(off, c->pair_off.ptr, size_t(N + 1) * sizeof(int64_t),
                                  cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess && P > 0)
    e = cudaMemcpyAsync(tri, c->pair_tri.ptr, size_t(P) * sizeof(int32_t), cudaMemcpyDeviceToDevice,
                        c->stream);
  if (e != cudaSuccess) return cuda_err(c, e, "pair list copy");
  return SPH2D_OK;
}

sph2d_status sph2d_boundary_integrals(sph2d_ctx* h, const float* particles, int64_t N,
                                      const float* tris, int64_t M, int kernel, double H,
                                      int moment_degree, int mode, void* gamma, void* grad_gamma,
                                      void* moments) {
  if (!h) return SPH2D_ERR_INVALID_ARG;
  Ctx* c = &h->c;
  c->err.clear();
  sph2d_status s = check_geom(c, particles, N, tris, M, H);
  if (s != SPH2D_OK) return s;
  s = check_outputs(c, kernel, moment_degree, mode, gamma, moments, N);
  if (s != SPH2D_OK) return s;
  cudaSetDevice(c->device);
  s = build_cells(c, particles, N, tris, M, H);
  if (s != SPH2D_OK) return s;
  if (mode == SPH2D_SURROGATE) return surrogate_integrals(c, gamma, grad_gamma);
  return launch_integrals(c, kernel, moment_degree, mode, gamma, grad_gamma, moments);
}

sph2d_status sph2d_integrals_from_pairs(sph2d_ctx* h, int kernel, int moment_degree, int mode,
                                        void* gamma, void* grad_gamma, void* moments) {
  if (!h) return SPH2D_ERR_INVALID_ARG;
  Ctx* c = &h->c;
  c->err.clear();
  if (!c->cells.built) return set_err(c, SPH2D_ERR_NOT_BUILT, "no pair list built");
  sph2d_status s = check_outputs(c, kernel, moment_degree, mode, gamma, moments, c->cells.N);
  if (s != SPH2D_OK) return s;
  cudaSetDevice(c->device);
  if (mode == SPH2D_SURROGATE) return surrogate_integrals(c, gamma, grad_gamma);
  return launch_integrals(c, kernel, moment_degree, mode, gamma, grad_gamma, moments);
}

sph2d_status sph2d_pair_integrals(sph2d_ctx* h, const double* pairs, int64_t P, int kernel,
                                  double H, int moment_degree, int mode, void* out) {
  if (!h) return SPH2D_ERR_INVALID_ARG;
  Ctx* c = &h->c;
  c->err.clear();
  if (P < 0) return set_err(c, SPH2D_ERR_INVALID_ARG, "P must be >= 0");
  if (P > 0 && (!pairs || !out)) return set_err(c, SPH2D_ERR_INVALID_ARG, "null pointer");
  if (!(H > 0.0) || !std::isfinite(H)) return set_err(c, SPH2D_ERR_INVALID_ARG, "H must be finite and > 0");
  if (!valid_kernel(kernel)) return set_err(c, SPH2D_ERR_INVALID_ARG, "unknown kernel id");
  if (moment_degree < -1 || moment_degree > 3)
    return set_err(c, SPH2D_ERR_INVALID_ARG, "moment_degree must be -1..3");
  if (mode == SPH2D_SURROGATE)
    return set_err(c, SPH2D_ERR_UNSUPPORTED, "independent pairs go through sph2d_surrogate_pairs");
  if (mode == SPH2D_FP32_HYBRID)
    return set_err(c, SPH2D_ERR_UNSUPPORTED, "the hybrid mode runs over a culled pair list only");
  if (mode != SPH2D_FP64 && mode != SPH2D_FP32_FIXUP)
    return set_err(c, SPH2D_ERR_INVALID_ARG, "unknown mode");
  if (reinterpret_cast<uintptr_t>(pairs) & 7u)
    return set_err(c, SPH2D_ERR_INVALID_ARG, "pairs must be 8-byte aligned");
  cudaSetDevice(c->device);
  return launch_pair_integrals(c, pairs, P, kernel, H, moment_degree, mode, out);
}

sph2d_status sph2d_boundary_integrals_backward(sph2d_ctx* h, const float* particles, int64_t N,
                                               const float* tris, int64_t M, int kernel, double H,
                                               int mode, const void* d_gamma,
                                               const void* d_grad_gamma, void* d_particles,
                                               void* d_tris) {
  if (!h) return SPH2D_ERR_INVALID_ARG;
  Ctx* c = &h->c;
  c->err.clear();
  sph2d_status s = check_geom(c, particles, N, tris, M, H);
  if (s != SPH2D_OK) return s;
  if (!valid_kernel(kernel)) return set_err(c, SPH2D_ERR_INVALID_ARG, "unknown kernel id");
  if (mode != SPH2D_FP64 && mode != SPH2D_FP32_FIXUP)
    return set_err(c, (mode == SPH2D_SURROGATE || mode == SPH2D_FP32_HYBRID) ? SPH2D_ERR_UNSUPPORTED
                                                                            : SPH2D_ERR_INVALID_ARG,
                   "backward supports SPH2D_FP64 and SPH2D_FP32_FIXUP");
  if ((N > 0 && (!d_gamma || !d_particles)) || (M > 0 && !d_tris))
    return set_err(c, SPH2D_ERR_INVALID_ARG, "null gradient pointer");
  cudaSetDevice(c->device);
  s = build_cells(c, particles, N, tris, M, H);
  if (s != SPH2D_OK) return s;
  return launch_backward(c, kernel, mode, d_gamma, d_grad_gamma, d_particles, d_tris);
}

sph2d_status sph2d_backward_from_pairs(sph2d_ctx* h, int kernel, int mode, const void* d_gamma,
                                       const void* d_grad_gamma, void* d_particles, void* d_tris) {
  if (!h) return SPH2D_ERR_INVALID_ARG;
  Ctx* c = &h->c;
  c->err.clear();
  if (!c->cells.built) return set_err(c, SPH2D_ERR_NOT_BUILT, "no pair list built");
  if (!valid_kernel(kernel)) return set_err(c, SPH2D_ERR_INVALID_ARG, "unknown kernel id");
  if (mode != SPH2D_FP64 && mode != SPH2D_FP32_FIXUP)
    return set_err(c, (mode == SPH2D_SURROGATE || mode == SPH2D_FP32_HYBRID) ? SPH2D_ERR_UNSUPPORTED
                                                                            : SPH2D_ERR_INVALID_ARG,
                   "backward supports SPH2D_FP64 and SPH2D_FP32_FIXUP");
  if ((c->cells.N > 0 && (!d_gamma || !d_particles)) || (c->cells.M > 0 && !d_tris))
    return set_err(c, SPH2D_ERR_INVALID_ARG, "null gradient pointer");
  cudaSetDevice(c->device);
  return launch_backward(c, kernel, mode, d_gamma, d_grad_gamma, d_particles, d_tris);
}

sph2d_status sph2d_field_integrals(sph2d_ctx* h, int kernel, int mode, const float* vertex_values, int nf,
                                   void* value, void* grad) {
  if (!h) return SPH2D_ERR_INVALID_ARG;
  Ctx* c = &h->c;
  c->err.clear();
  if (!c->cells.built) return set_err(c, SPH2D_ERR_NOT_BUILT, "no pair list built");
  if (!valid_kernel(kernel)) return set_err(c, SPH2D_ERR_INVALID_ARG, "unknown kernel id");
  if (mode != SPH2D_FP64 && mode != SPH2D_FP32_FIXUP)
    return set_err(c, (mode == SPH2D_SURROGATE || mode == SPH2D_FP32_HYBRID) ? SPH2D_ERR_UNSUPPORTED
                                                                            : SPH2D_ERR_INVALID_ARG,
                   "field integrals support SPH2D_FP64 and SPH2D_FP32_FIXUP");
  if (nf < 1 || nf > SPH2D_MAX_FIELDS) return set_err(c, SPH2D_ERR_INVALID_ARG, "nf must be 1..SPH2D_MAX_FIELDS");
  if ((c->cells.M > 0 && !vertex_values) || (c->cells.N > 0 && !value))
    return set_err(c, SPH2D_ERR_INVALID_ARG, "null pointer");
  if (reinterpret_cast<uintptr_t>(vertex_values) & 3u)
    return set_err(c, SPH2D_ERR_INVALID_ARG, "vertex values must be 4-byte aligned");
  cudaSetDevice(c->device);
  return launch_fields(c, kernel, mode, vertex_values, nf, value, grad);
}

sph2d_status sph2d_field_integrals_p(sph2d_ctx* h, int kernel, int mode, int order, const float* node_values,
                                     int nf, void* value, void* grad) {
  if (!h) return SPH2D_ERR_INVALID_ARG;
  Ctx* c = &h->c;
  c->err.clear();
  if (!c->cells.built) return set_err(c, SPH2D_ERR_NOT_BUILT, "no pair list built");
  if (!valid_kernel(kernel)) return set_err(c, SPH2D_ERR_INVALID_ARG, "unknown kernel id");
  if (order != 2 && order != 3) return set_err(c, SPH2D_ERR_INVALID_ARG, "order must be 2 or 3");
  if (mode != SPH2D_FP64 && mode != SPH2D_FP32_HYBRID)
    return set_err(c, (mode == SPH2D_SURROGATE || mode == SPH2D_FP32_FIXUP) ? SPH2D_ERR_UNSUPPORTED
                                                                           : SPH2D_ERR_INVALID_ARG,
                   "order 2 and 3 fields support SPH2D_FP64 and SPH2D_FP32_HYBRID");
  if (nf < 1 || nf > SPH2D_MAX_FIELDS) return set_err(c, SPH2D_ERR_INVALID_ARG, "nf must be 1..SPH2D_MAX_FIELDS");
  if ((c->cells.M > 0 && !node_values) || (c->cells.N > 0 && !value))
    return set_err(c, SPH2D_ERR_INVALID_ARG, "null pointer");
  if (reinterpret_cast<uintptr_t>(node_values) & 3u)
    return set_err(c, SPH2D_ERR_INVALID_ARG, "node values must be 4-byte aligned");
  cudaSetDevice(c->device);
  return launch_fields_p(c, kernel, mode, order, node_values, nf, value, grad);
}

// ---- boundary pressure coupling (Appendix A) ----------------------------------------------
static sph2d_status press_check(Ctx* c, int kernel, int mode) {
  if (!c->cells.built) return set_err(c, SPH2D_ERR_NOT_BUILT, "no pair list built");
  if (!valid_kernel(kernel)) return set_err(c, SPH2D_ERR_INVALID_ARG, "unknown kernel id");
  if (mode != SPH2D_FP64 && mode != SPH2D_FP32_FIXUP)
    return set_err(c, (mode == SPH2D_SURROGATE || mode == SPH2D_FP32_HYBRID) ? SPH2D_ERR_UNSUPPORTED
                                                                            : SPH2D_ERR_INVALID_ARG,
                   "boundary pressure supports SPH2D_FP64 and SPH2D_FP32_FIXUP");
  return SPH2D_OK;
}

sph2d_status sph2d_mls_pressure(sph2d_ctx* h, int kernel, int mode, const float* volume, const float* pressure,
                                const float* points, int64_t Q, void* out) {
  if (!h) return SPH2D_ERR_INVALID_ARG;
  Ctx* c = &h->c;
  c->err.clear();
  sph2d_status s = press_check(c, kernel, mode);
  if (s != SPH2D_OK) return s;
  if (Q < 0) return set_err(c, SPH2D_ERR_INVALID_ARG, "Q < 0");
  if (Q > 0 && (!points || !out || (c->cells.N > 0 && (!volume || !pressure))))
    return set_err(c, SPH2D_ERR_INVALID_ARG, "null pointer");
  cudaSetDevice(c->device);
  return launch_mls_points(c, kernel, mode, volume, pressure, points, Q, out);
}

sph2d_status sph2d_boundary_pressure(sph2d_ctx* h, int kernel, int mode, int model, const float* density,
                                     const float* pressure, const float* volume, double rho0_b, void* accel) {
  if (!h) return SPH2D_ERR_INVALID_ARG;
  Ctx* c = &h->c;
  c->err.clear();
  sph2d_status s = press_check(c, kernel, mode);
  if (s != SPH2D_OK) return s;
  if (model != 1 && model != 2) return set_err(c, SPH2D_ERR_INVALID_ARG, "model must be 1 or 2");
  if (!(rho0_b > 0.0) || !std::isfinite(rho0_b)) return set_err(c, SPH2D_ERR_INVALID_ARG, "rho0_b must be > 0");
  if (c->cells.N > 0 && (!density || !pressure || !volume || !accel))
    return set_err(c, SPH2D_ERR_INVALID_ARG, "null pointer");
  cudaSetDevice(c->device);
  return launch_boundary_pressure(c, kernel, mode, model, density, pressure, volume, rho0_b, accel);
}

// ---- learned surrogate -----------------------------------------------------------------
static sph2d_status sur_ctx(sph2d_ctx* h, Ctx** out, bool need_ready) {
  if (!h) return SPH2D_ERR_INVALID_ARG;
  Ctx* c = &h->c;
  c->err.clear();
  *out = c;
  if (need_ready && !c->sur_ready) return set_err(c, SPH2D_ERR_NOT_BUILT, "surrogate not initialised");
  cudaSetDevice(c->device);
  return SPH2D_OK;
}

sph2d_status sph2d_surrogate_init(sph2d_ctx* h, int kernel, uint64_t seed) {
  Ctx* c;
  sph2d_status s = sur_ctx(h, &c, false);
  if (s != SPH2D_OK) return s;
  if (!valid_kernel(kernel)) return set_err(c, SPH2D_ERR_INVALID_ARG, "unknown kernel id");
  return surrogate_init(c, kernel, seed);
}

sph2d_status sph2d_surrogate_train(sph2d_ctx* h, const double* pairs, int64_t P, double H, int epochs,
                                   int batch, double lr, double weight_decay, uint64_t seed,
                                   double* final_loss, int64_t* n_used) {
  Ctx* c;
  sph2d_status s = sur_ctx(h, &c, true);
  if (s != SPH2D_OK) return s;
  if (P <= 0 || P > (int64_t(1) << 31) - 1 || !pairs || (reinterpret_cast<uintptr_t>(pairs) & 7u))
    return set_err(c, SPH2D_ERR_INVALID_ARG, "pairs must be a non-empty 8-byte aligned [P][8] array, P < 2^31");
  if (!(H > 0.0) || !std::isfinite(H)) return set_err(c, SPH2D_ERR_INVALID_ARG, "H must be finite and > 0");
  if (epochs < 0 || batch < 1 || batch > (1 << 20))
    return set_err(c, SPH2D_ERR_INVALID_ARG, "epochs >= 0 and 1 <= batch <= 2^20 required");
  if (!(lr > 0.0) || !std::isfinite(lr) || !(weight_decay >= 0.0) || !std::isfinite(weight_decay))
    return set_err(c, SPH2D_ERR_INVALID_ARG, "lr > 0 and weight_decay >= 0 required");
  return surrogate_train(c, pairs, P, H, epochs, batch, lr, weight_decay, seed, final_loss, n_used);
}

sph2d_status sph2d_surrogate_pairs(sph2d_ctx* h, const double* pairs, int64_t P, double H, float* out,
                                   int32_t* accepted) {
  Ctx* c;
  sph2d_status s = sur_ctx(h, &c, true);
  if (s != SPH2D_OK) return s;
  if (P < 0) return set_err(c, SPH2D_ERR_INVALID_ARG, "P must be >= 0");
  if (P > 0 && (!pairs || !out)) return set_err(c, SPH2D_ERR_INVALID_ARG, "null pointer");
  if (reinterpret_cast<uintptr_t>(pairs) & 7u) return set_err(c, SPH2D_ERR_INVALID_ARG, "pairs must be 8-byte aligned");
  if (reinterpret_cast<uintptr_t>(out) & 3u) return set_err(c, SPH2D_ERR_INVALID_ARG, "out must be 4-byte aligned");
  if (!(H > 0.0) || !std::isfinite(H)) return set_err(c, SPH2D_ERR_INVALID_ARG, "H must be finite and > 0");
  return surrogate_pairs(c, pairs, P, H, out, accepted);
}

sph2d_status sph2d_surrogate_forward(sph2d_ctx* h, const float* x, int64_t B, float* y) {
  Ctx* c;
  sph2d_status s = sur_ctx(h, &c, true);
  if (s != SPH2D_OK) return s;
  if (B < 0 || (B > 0 && (!x || !y))) return set_err(c, SPH2D_ERR_INVALID_ARG, "bad batch or null pointer");
  return surrogate_forward(c, x, B, y);
}

sph2d_status sph2d_surrogate_grad(sph2d_ctx* h, const float* x, const float* t, int64_t B, float* grad,
                                  float* loss) {
  Ctx* c;
  sph2d_status s = sur_ctx(h, &c, true);
  if (s != SPH2D_OK) return s;
  if (B < 1 || B > (1 << 20) || !x || !t || !grad || !loss)
    return set_err(c, SPH2D_ERR_INVALID_ARG, "1 <= B <= 2^20 and non-null pointers required");
  return surrogate_grad(c, x, t, B, grad, loss);
}

sph2d_status sph2d_surrogate_get_params(sph2d_ctx* h, float* host, int64_t cap) {
  Ctx* c;
  sph2d_status s = sur_ctx(h, &c, true);
  if (s != SPH2D_OK) return s;
  if (!host) return set_err(c, SPH2D_ERR_INVALID_ARG, "null pointer");
  if (cap < SPH2D_SURROGATE_PARAMS) return set_err(c, SPH2D_ERR_CAPACITY, "buffer smaller than SPH2D_SURROGATE_PARAMS");
  return surrogate_get_params(c, host);
}

sph2d_status sph2d_surrogate_set_audit(sph2d_ctx* h, int period, double tol) {
  if (!h) return SPH2D_ERR_INVALID_ARG;
  Ctx* c = &h->c;
  if (period < 0 || period > 65536 || (period & (period - 1)) != 0)
    return set_err(c, SPH2D_ERR_INVALID_ARG, "audit period must be 0 or a power of two up to 65536");
  if (!(tol > 0.0) || !std::isfinite(tol)) return set_err(c, SPH2D_ERR_INVALID_ARG, "audit bound must be > 0");
  c->sur_audit_period = period;
  c->sur_audit_tol = tol;
  return SPH2D_OK;
}

sph2d_status sph2d_surrogate_set_engine(sph2d_ctx* h, int engine) {
  if (!h) return SPH2D_ERR_INVALID_ARG;
  if (engine != 0 && engine != 1) return set_err(&h->c, SPH2D_ERR_INVALID_ARG, "engine must be 0 (mma.sync) or 1 (tcgen05)");
  h->c.sur_engine = engine;
  return SPH2D_OK;
}

sph2d_status sph2d_surrogate_set_train_engine(sph2d_ctx* h, int engine) {
  if (!h) return SPH2D_ERR_INVALID_ARG;
  if (engine != 0 && engine != 1) return set_err(&h->c, SPH2D_ERR_INVALID_ARG, "engine must be 0 (mma.sync) or 1 (tcgen05)");
  h->c.sur_train_engine = engine;
  return SPH2D_OK;
}

sph2d_status sph2d_surrogate_set_params(sph2d_ctx* h, const float* host, int64_t n) {
  Ctx* c;
  sph2d_status s = sur_ctx(h, &c, true);
  if (s != SPH2D_OK) return s;
  if (!host || n != SPH2D_SURROGATE_PARAMS)
    return set_err(c, SPH2D_ERR_INVALID_ARG, "expected SPH2D_SURROGATE_PARAMS host floats");
  return surrogate_set_params(c, host);
}

sph2d_status sph2d_surrogate_save(sph2d_ctx* h, const char* path) {
  Ctx* c;
  sph2d_status s = sur_ctx(h, &c, true);
  if (s != SPH2D_OK) return s;
  if (!path) return set_err(c, SPH2D_ERR_INVALID_ARG, "null path");
  return surrogate_save(c, path);
}

sph2d_status sph2d_surrogate_load(sph2d_ctx* h, const char* path) {
  Ctx* c;
  sph2d_status s = sur_ctx(h, &c, false);
  if (s != SPH2D_OK) return s;
  if (!path) return set_err(c, SPH2D_ERR_INVALID_ARG, "null path");
  return surrogate_load(c, path);
}

}  // extern "C"
