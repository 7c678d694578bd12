// Allocation-free variant of the per-particle integral kernel.
//
// Who needs it: callers that must not allocate device memory while they run -- code inside a
// memory pool that forbids cudaMalloc during a solver step, frameworks that own all device
// memory and reject foreign allocations, and code running where an allocation could
// synchronise the device or fail under memory pressure.  They call
// sph2d_pair_list_integrals_noalloc with their own inputs and outputs; the only scratch it
// needs, the per-chunk partial sums of particles whose pairs cross a 32-pair chunk, lives in
// the file-scope array below, sized at build time (SPH2D_NOALLOC_SCRATCH_BYTES) and held by
// every GPU that loads the library until the process exits.
//
// Contract: nothing here calls cudaMalloc, cudaFree, cudaMallocHost or any allocating library
// routine.  The array is shared by every call on a device and keeps the last call's
// contents; the fix-up counter at its start is cleared by each call, the partial-sum slots are
// always written before they are read.  Calls that overlap on the GPU (different streams,
// or host threads, at the same time) race on the array.  The first call on a device resolves
// the array's device address (cudaGetSymbolAddress) with that device current; make that
// first call before any stream capture.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "integrals_impl.cuh"

namespace sph2d {

static __device__ __align__(256) unsigned char g_noalloc_scratch[SPH2D_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// device address of the scratch array on the current device (resolved once per device)
cudaError_t scratch_address(int dev, void** out) {
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

// occupancy-sized grid of kernel `kern` on device dev (resolved once per device and kernel;
// slot: the kernel's index among the noalloc instantiations)
constexpr int kNoallocKernels = 8;
int g_grid_blocks[kMaxDevices][kNoallocKernels] = {};

template <typename K>
int grid_blocks_for(int dev, int slot, K kern) {
  std::lock_guard<std::mutex> lock(g_setup_mu);
  int& gb = g_grid_blocks[dev][slot];
  if (gb == 0) {
    int per_sm = 0, sms = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, 0);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    gb = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
  }
  return gb;
}
}  // namespace

// Same chunked warp reduction as integrals_kernel (gamma and grad gamma, no moments), except
// that each lane finds its particle by binary search in the caller's CSR offsets instead of
// reading a pair-to-particle array (which would be more scratch).
template <typename OT, int KID>
__global__ void __launch_bounds__(128) integrals_noalloc_kernel(IntArgs a) {
  constexpr int NV = 3;
  const int lane = threadIdx.x & 31;
  const int64_t nchunks = (a.P + 31) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  unsigned long long fixes = 0;
  for (int64_t ch = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; ch < nchunks; ch += nw) {
    const int64_t q = ch * 32 + lane;
    int pid = -1;
    OT v[NV] = {OT(0), OT(0), OT(0)};
    int fix = 0;
    if (q < a.P) {
      int64_t lo = 0, hi = a.N - 1;                  // largest i with off[i] <= q
      while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (__ldg(a.pair_off + mid) <= q) lo = mid;
        else hi = mid - 1;
      }
      pid = int(lo);
      fix = eval_pair<OT, KID, 0>(a, pid, __ldg(a.pair_tri + q), v);
    }
    fixes += __popc(__ballot_sync(0xffffffffu, fix));
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
      if (s0 >= cs && s1 <= cs + 32) write_particle<OT, 0>(a, pid, v);
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

template <typename OT, int KID>
static cudaError_t launch_noalloc(int dev, const IntArgs& a, cudaStream_t st) {
  const int grid_blocks =
      grid_blocks_for(dev, KID + (sizeof(OT) == sizeof(double) ? 4 : 0), integrals_noalloc_kernel<OT, KID>);
  const int64_t nchunks = (a.P + 31) >> 5;
  if (a.P > 0) {
    const int64_t want = (nchunks + 3) / 4;
    const unsigned blocks = unsigned(want < grid_blocks ? (want > 0 ? want : 1) : grid_blocks);
    integrals_noalloc_kernel<OT, KID><<<blocks, 128, 0, st>>>(a);
  }
  if (a.N > 0) finalize_kernel<OT, 0><<<unsigned((a.N + 255) / 256), 256, 0, st>>>(a);
  return cudaGetLastError();
}

template <typename OT>
static cudaError_t dispatch_noalloc(int dev, int kernel, const IntArgs& a, cudaStream_t st) {
  switch (kernel) {
    case KID_WC2: return launch_noalloc<OT, KID_WC2>(dev, a, st);
    case KID_WC4: return launch_noalloc<OT, KID_WC4>(dev, a, st);
    case KID_WC6: return launch_noalloc<OT, KID_WC6>(dev, a, st);
    default: return launch_noalloc<OT, KID_CUBIC>(dev, a, st);
  }
}

}  // namespace sph2d

extern "C" sph2d_status sph2d_pair_list_integrals_noalloc(
    const float* particles, int64_t N, const float* tris, int64_t M, const int64_t* pair_off,
    const int32_t* pair_tri, int64_t P, int kernel, double H, int mode, void* gamma,
    void* grad_gamma, void* stream) {
  using namespace sph2d;
  if (N < 0 || M < 0 || P < 0 || N > (int64_t(1) << 31) - 2 || M > (int64_t(1) << 31) - 2)
    return SPH2D_ERR_INVALID_ARG;
  if (N > 0 && (!particles || !pair_off || !gamma)) return SPH2D_ERR_INVALID_ARG;
  if (N == 0 && P > 0) return SPH2D_ERR_INVALID_ARG;
  if (P > 0 && (!tris || !pair_tri || M == 0)) return SPH2D_ERR_INVALID_ARG;
  if (particles && (reinterpret_cast<uintptr_t>(particles) & 15u)) return SPH2D_ERR_INVALID_ARG;
  if (!(H > 0.0) || !std::isfinite(H)) return SPH2D_ERR_INVALID_ARG;
  if (kernel < SPH2D_WENDLAND_C2 || kernel > SPH2D_CUBIC_SPLINE) return SPH2D_ERR_INVALID_ARG;
  if (mode != SPH2D_FP64 && mode != SPH2D_FP32_FIXUP) return SPH2D_ERR_INVALID_ARG;
  // scratch layout: [0, 256) fix-up counter, then 2 slots x 3 values per 32-pair chunk
  const size_t elem = mode == SPH2D_FP64 ? sizeof(double) : sizeof(float);
  const size_t nchunks = size_t((P + 31) / 32);
  if (256 + nchunks * 2 * 3 * elem > size_t(SPH2D_NOALLOC_SCRATCH_BYTES)) return SPH2D_ERR_CAPACITY;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return SPH2D_ERR_CUDA;
  }
  void* base = nullptr;
  if (scratch_address(dev, &base) != cudaSuccess) {
    cudaGetLastError();
    return SPH2D_ERR_CUDA;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  IntArgs a;
  a.parts = reinterpret_cast<const float4*>(particles);
  a.tris = tris;
  a.pair_tri = pair_tri;
  a.pair_pid = nullptr;
  a.pair_off = pair_off;
  a.P = P;
  a.N = N;
  a.H = H;
  a.invH = 1.0 / H;
  a.C = kernel_C(kernel);
  a.gamma = gamma;
  a.grad = grad_gamma;
  a.mom = nullptr;
  a.nm = 0;
  a.nfix = static_cast<unsigned long long*>(base);
  a.slots = static_cast<char*>(base) + 256;
  if (cudaMemsetAsync(base, 0, sizeof(unsigned long long), st) != cudaSuccess) {
    cudaGetLastError();
    return SPH2D_ERR_CUDA;
  }
  const cudaError_t e = mode == SPH2D_FP64 ? dispatch_noalloc<double>(dev, kernel, a, st)
                                           : dispatch_noalloc<float>(dev, kernel, a, st);
  return e == cudaSuccess ? SPH2D_OK : SPH2D_ERR_CUDA;
}
