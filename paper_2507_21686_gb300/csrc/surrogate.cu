// Learned surrogate: tensor-core (mma.sync m16n8k16, FP32 accumulation) training and
// inference of the 6-64-64-64-3 MLP of surrogate.cuh (FP16 forward operands, BF16 backward
// operands), with the guarded analytic fallback.
// This part has no counterpart in the paper.
//
// Training runs entirely in this file's kernels: canonicalisation of analytic training pairs,
// per-step forward (GEMM + bias + GELU), loss gradient, backward (GEMMs for activation and
// weight gradients, GELU derivative, bias column sums), AdamW on FP32 master weights.  Weight
// gradients reduce over the batch with split-K partials summed in a fixed order, so a
// training run is reproducible bit for bit.
//
// Serving, three kernels:
//   values   one warp per 32 pairs: every lane canonicalises its pair and applies the guard;
//            the 32 rows go through the network as two m16 tiles with the layer outputs kept
//            in registers and fed back as the next layer's A operand (the accumulator fragment
//            of two adjacent n8 tiles is exactly the A fragment of one k16 step); weight
//            fragments come from shared memory by ldmatrix.  Accepted
//            pairs write their value; rejected pairs are appended to a fallback list (one
//            atomic per warp).
//   fallback the analytic FP32 path (with its FP64 fix-up) over the compacted list, so a
//            warp's lanes all do analytic work instead of idling beside network lanes.
//   reduce   per-particle sums over the per-pair values in pair order (the same 32-pair
//            chunk reduction and crossing slots as the analytic kernel), so the result does
//            not depend on the order in which the list was filled.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include <string>
#include <type_traits>
#include <vector>

#include "integrals_impl.cuh"
#include "surrogate.cuh"
#include "umma.cuh"

namespace sph2d {

static_assert(kSurParams == SPH2D_SURROGATE_PARAMS, "parameter count differs from the header");
static_assert(kSurMinSize == float(SPH2D_SURROGATE_MIN_SIZE) && kSurMaxSize == float(SPH2D_SURROGATE_MAX_SIZE) &&
                  kSurMinCentroid == float(SPH2D_SURROGATE_MIN_CENTROID) &&
                  kSurMaxRadius == float(SPH2D_SURROGATE_MAX_RADIUS),
              "guard constants differ from the header");

// ---------------------------------------------------------------------------------------
// generic GEMM: C[M][N] = alpha * op(A) op(B)   (FP32 in/out, T = FP16 or BF16 operands rounded
// to nearest even on the way into shared memory, FP32 accumulation)
//   op(A) is M x K: ta=0 -> A[m*lda + k], ta=1 -> A[k*lda + m]
//   op(B) is K x N: tb=0 -> B[n*ldb + k],  tb=1 -> B[k*ldb + n]
// Block tile 64 x 64 x 32, 4 warps of 32 x 32.  blockIdx.z splits K; with ksplit > 1 each
// split writes its own partial (M x N, row stride N) at C + z * M * N.
// ---------------------------------------------------------------------------------------
constexpr int GBM = 64, GBN = 64, GBK = 32, GPAD = 8;

template <typename T>
__global__ void __launch_bounds__(128) gemm_tc_kernel(int M, int N, int K, const float* __restrict__ A,
                                                      int lda, int ta, const float* __restrict__ B, int ldb,
                                                      int tb, float* __restrict__ C, int ldc, float alpha,
                                                      int ksplit) {
  __shared__ __align__(16) T As[GBM][GBK + GPAD];
  __shared__ __align__(16) T Bs[GBN][GBK + GPAD];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int m0 = blockIdx.x * GBM, n0 = blockIdx.y * GBN;
  const int kper = (K + ksplit - 1) / ksplit;
  const int kbeg = blockIdx.z * kper, kend = min(K, kbeg + kper);
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.0f;
  for (int k0 = kbeg; k0 < kend; k0 += GBK) {
#pragma unroll
    for (int i = 0; i < (GBM * GBK) / 128; ++i) {
      const int e = tid + 128 * i;
      int m, k;
      if (!ta) { m = e / GBK; k = e % GBK; } else { k = e / GBM; m = e % GBM; }
      const int gm = m0 + m, gk = k0 + k;
      float v = 0.0f;
      if (gm < M && gk < kend) v = ta ? A[size_t(gk) * lda + gm] : A[size_t(gm) * lda + gk];
      As[m][k] = to_op(v, T());
    }
#pragma unroll
    for (int i = 0; i < (GBN * GBK) / 128; ++i) {
      const int e = tid + 128 * i;
      int n, k;
      if (!tb) { n = e / GBK; k = e % GBK; } else { k = e / GBN; n = e % GBN; }
      const int gn = n0 + n, gk = k0 + k;
      float v = 0.0f;
      if (gn < N && gk < kend) v = tb ? B[size_t(gk) * ldb + gn] : B[size_t(gn) * ldb + gk];
      Bs[n][k] = to_op(v, T());
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < GBK; ks += 16) {
      uint32_t af[2][4], bf[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r = wm + i * 16 + g;
        af[i][0] = *reinterpret_cast<const uint32_t*>(&As[r][ks + 2 * t]);
        af[i][1] = *reinterpret_cast<const uint32_t*>(&As[r + 8][ks + 2 * t]);
        af[i][2] = *reinterpret_cast<const uint32_t*>(&As[r][ks + 2 * t + 8]);
        af[i][3] = *reinterpret_cast<const uint32_t*>(&As[r + 8][ks + 2 * t + 8]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int cn = wn + j * 8 + g;
        bf[j][0] = *reinterpret_cast<const uint32_t*>(&Bs[cn][ks + 2 * t]);
        bf[j][1] = *reinterpret_cast<const uint32_t*>(&Bs[cn][ks + 2 * t + 8]);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma_16816(acc[i][j], af[i], bf[j], T());
    }
    __syncthreads();
  }
  float* Cz = ksplit > 1 ? C + size_t(blockIdx.z) * M * N : C;
  const int ld = ksplit > 1 ? N : ldc;
  const float sc = ksplit > 1 ? 1.0f : alpha;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int gm = m0 + wm + i * 16 + g + (r >= 2 ? 8 : 0);
        const int gn = n0 + wn + j * 8 + 2 * t + (r & 1);
        if (gm < M && gn < N) Cz[size_t(gm) * ld + gn] = sc * acc[i][j][r];
      }
}

// sum of split-K partials in split order (deterministic); C[m*ldc + n] = alpha * sum
__global__ void splitk_reduce_kernel(const float* __restrict__ part, int splits, int M, int N,
                                     float* __restrict__ C, int ldc, float alpha) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M * N) return;
  float s = 0.0f;
  for (int z = 0; z < splits; ++z) s += part[size_t(z) * M * N + i];
  C[size_t(i / N) * ldc + (i % N)] = alpha * s;
}

// ---------------------------------------------------------------------------------------
// the same GEMM on the fifth-generation tensor cores (training engine 1): CTA tile 128 x 64,
// K blocks of 32 staged (FP32 -> FP16/BF16, round to nearest even, zero padded) into shared
// memory in the K-major no-swizzle core-matrix layout of umma.cuh; one thread issues two
// tcgen05.mma kind::f16 (M = 128, N = 64, K = 16) per block into FP32 accumulators in tensor
// memory (64 columns) and commits them to an mbarrier that every thread waits on (bounded);
// the epilogue reads each row's 64 accumulators with one tcgen05.ld.  Same split-K contract as
// gemm_tc_kernel.  A wait that runs out of its poll budget adds 1 to *timeouts, lets the MMA
// drain (bounded) and leaves the tile's outputs unwritten.
// ---------------------------------------------------------------------------------------
constexpr int UBM = 128, UBN = 64, UBK = 32;
constexpr uint32_t kGemmSpin = 1u << 22;

template <typename T>
struct GemmTcSmem {
  T a[UBM * UBK];               // 8 KB: row r, column c at kmajor_offset(r, c, 32) bytes
  T b[UBN * UBK];               // 4 KB
  uint64_t mbar;
  uint32_t tmem;
};

template <typename T>
__global__ void __launch_bounds__(128) gemm_umma_kernel(int M, int N, int K, const float* __restrict__ A,
                                                        int lda, int ta, const float* __restrict__ B, int ldb,
                                                        int tb, float* __restrict__ C, int ldc, float alpha,
                                                        int ksplit, unsigned long long* timeouts) {
  using umma::kmajor_offset;
  __shared__ __align__(128) GemmTcSmem<T> s;
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) {
    umma::tmem_alloc(&s.tmem, 64);
    umma::tmem_relinquish();
  }
  if (tid == 0) {
    umma::mbar_init(&s.mbar, 1);
    umma::mbar_init_fence();
  }
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tm = s.tmem, sa = umma::smem_u32(s.a), sb = umma::smem_u32(s.b);
  constexpr uint32_t ID = umma::idesc_f16(UBM, UBN, std::is_same<T, __nv_bfloat16>::value);
  const int m0 = blockIdx.x * UBM, n0 = blockIdx.y * UBN;
  const int kper = (K + ksplit - 1) / ksplit;
  const int kbeg = blockIdx.z * kper, kend = min(K, kbeg + kper);
  uint32_t phase = 0;
  bool ok = true, any = false;
  for (int k0 = kbeg; k0 < kend; k0 += UBK) {
#pragma unroll 4
    for (int i = 0; i < (UBM * UBK) / 128; ++i) {
      const int e = tid + 128 * i;
      int m, k;
      if (!ta) { m = e / UBK; k = e % UBK; } else { k = e / UBM; m = e % UBM; }
      const int gm = m0 + m, gk = k0 + k;
      float v = 0.0f;
      if (gm < M && gk < kend) v = ta ? A[size_t(gk) * lda + gm] : A[size_t(gm) * lda + gk];
      s.a[kmajor_offset(m, k, UBK) / 2] = to_op(v, T());
    }
#pragma unroll 4
    for (int i = 0; i < (UBN * UBK) / 128; ++i) {
      const int e = tid + 128 * i;
      int n, k;
      if (!tb) { n = e / UBK; k = e % UBK; } else { k = e / UBN; n = e % UBN; }
      const int gn = n0 + n, gk = k0 + k;
      float v = 0.0f;
      if (gn < N && gk < kend) v = tb ? B[size_t(gk) * ldb + gn] : B[size_t(gn) * ldb + gk];
      s.b[kmajor_offset(n, k, UBK) / 2] = to_op(v, T());
    }
    umma::fence_proxy_async();
    umma::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      umma::fence_after_sync();
#pragma unroll
      for (int kk = 0; kk < UBK / 16; ++kk)
        umma::mma_f16(tm, umma::smem_desc(sa + 256 * kk, 128, 128 * UBK / 8),
                      umma::smem_desc(sb + 256 * kk, 128, 128 * UBK / 8), ID, any || kk > 0);
      umma::mma_commit(&s.mbar);
    }
    any = true;
    ok = __syncthreads_and(umma::mbar_wait(&s.mbar, phase, kGemmSpin) ? 1 : 0) != 0;
    umma::fence_after_sync();
    if (!ok) break;
    phase ^= 1u;
  }
  float* Cz = ksplit > 1 ? C + size_t(blockIdx.z) * M * N : C;
  const int ld = ksplit > 1 ? N : ldc;
  const float sc = ksplit > 1 ? 1.0f : alpha;
  const int gm = m0 + 32 * warp + (tid & 31);
  if (ok && any) {
    float acc[UBN];
    umma::tmem_ld64(tm + (uint32_t(32 * warp) << 16), acc);
    if (gm < M)
#pragma unroll
      for (int j = 0; j < UBN; ++j)
        if (n0 + j < N) Cz[size_t(gm) * ld + n0 + j] = sc * acc[j];
  } else if (ok) {                                   // an empty K split: its partial is zero
    if (gm < M)
      for (int j = 0; j < UBN; ++j)
        if (n0 + j < N) Cz[size_t(gm) * ld + n0 + j] = 0.0f;
  } else {
    if (tid == 0) atomicAdd(timeouts, 1ull);
    umma::mbar_wait(&s.mbar, phase, kGemmSpin);      // let the overdue MMA drain
  }
  umma::fence_before_sync();
  __syncthreads();
  if (warp == 0) umma::tmem_dealloc(tm, 64);
}

// ---------------------------------------------------------------------------------------
// elementwise kernels of the training step
// ---------------------------------------------------------------------------------------
// Z += b (row broadcast, n even); H = GELU(Z) in packed FP16 arithmetic (exactly the
// inference activation), stored as FP32
__global__ void bias_gelu_kernel(float* __restrict__ Z, const float* __restrict__ b, float* __restrict__ Hh,
                                 int64_t rows, int n) {
  const int64_t i = 2 * (int64_t(blockIdx.x) * blockDim.x + threadIdx.x);
  if (i >= rows * n) return;
  const int col = int(i % n);
  const float z0 = Z[i] + b[col], z1 = Z[i + 1] + b[col + 1];
  Z[i] = z0;
  Z[i + 1] = z1;
  const float2 g = __half22float2(gelu_h2(__floats2half2_rn(z0, z1)));
  Hh[i] = g.x;
  Hh[i + 1] = g.y;
}

__global__ void bias_kernel(float* __restrict__ Z, const float* __restrict__ b, int64_t rows, int n) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < rows * n) Z[i] += b[i % n];
}

__global__ void gelu_back_kernel(float* __restrict__ dH, const float* __restrict__ Z, int64_t count) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < count) dH[i] *= gelu_grad_f(Z[i]);
}

// loss = (1/B) sum_rows sum_c w_c (Y - T)^2; dY = 2 w_c (Y - T) / B; per-block partial sums
__global__ void loss_grad_kernel(const float* __restrict__ Y, const float* __restrict__ T, int64_t rows,
                                 float w0, float w1, float w2, float* __restrict__ dY,
                                 float* __restrict__ partial) {
  __shared__ float red[256];
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  float l = 0.0f;
  if (i < rows * 3) {
    const int c = int(i % 3);
    const float w = c == 0 ? w0 : (c == 1 ? w1 : w2);
    const float d = Y[i] - T[i];
    dY[i] = 2.0f * w * d / float(rows);
    l = w * d * d / float(rows);
  }
  red[threadIdx.x] = l;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void sum_kernel(const float* __restrict__ x, int n, float* __restrict__ out) {
  __shared__ float red[256];
  float s = 0.0f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += x[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// column sums of dZ [rows][n] -> db [n], one block per column, fixed tree order
__global__ void colsum_kernel(const float* __restrict__ dZ, int64_t rows, int n, float* __restrict__ db) {
  __shared__ float red[256];
  const int c = blockIdx.x;
  float s = 0.0f;
  for (int64_t r = threadIdx.x; r < rows; r += blockDim.x) s += dZ[r * n + c];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) db[c] = red[0];
}

// AdamW (decoupled weight decay) on the FP32 masters
__global__ void adamw_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                             float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float wd,
                             float bc1, float bc2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] = p[i] * (1.0f - lr * wd) - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

__global__ void gather_rows_kernel(const float* __restrict__ X, const float* __restrict__ T,
                                   const int32_t* __restrict__ idx, int64_t rows, float* __restrict__ Xb,
                                   float* __restrict__ Tb) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  const int64_t s = idx[r];
#pragma unroll
  for (int j = 0; j < 6; ++j) Xb[r * 6 + j] = X[s * 6 + j];
#pragma unroll
  for (int j = 0; j < 3; ++j) Tb[r * 3 + j] = T[s * 3 + j];
}

// local frame of an independent pair [x, y, v0x, v0y, v1x, v1y, v2x, v2y] (double and float)
__device__ __forceinline__ void pair_local(const double* q, double invH, double* ld, float* lf) {
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    ld[2 * j] = (q[2 + 2 * j] - q[0]) * invH;
    ld[2 * j + 1] = (q[3 + 2 * j] - q[1]) * invH;
    lf[2 * j] = float(ld[2 * j]);
    lf[2 * j + 1] = float(ld[2 * j + 1]);
  }
}

// training data: analytic (gamma, grad) [P][3] in world units for pairs [P][8] -> canonical
// inputs X [P][6], targets T [P][3] = (gamma, canonical local-frame grad) / area, guard flags
__global__ void canon_training_kernel(const double* __restrict__ pairs, const double* __restrict__ ana,
                                      int64_t P, double invH, double H, float* __restrict__ X,
                                      float* __restrict__ T, int32_t* __restrict__ ok) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= P) return;
  double ld[6];
  float v[6];
  pair_local(pairs + 8 * i, invH, ld, v);
  const Canon c = canonicalize(v);
  const double* a = ana + 3 * i;
  // local-frame gradient = H * world gradient; rotate (then reflect) into the canonical frame
  const float gx = float(a[1] * H), gy = float(a[2] * H);
  const float gxc = c.cs * gx + c.sn * gy;
  const float gyc = c.refl * (-c.sn * gx + c.cs * gy);
  const float ia = c.area > 0.0f ? 1.0f / c.area : 0.0f;
#pragma unroll
  for (int j = 0; j < 6; ++j) X[6 * i + j] = c.x[j];
  T[3 * i] = float(a[0]) * ia;
  T[3 * i + 1] = gxc * ia;
  T[3 * i + 2] = gyc * ia;
  ok[i] = c.accept ? 1 : 0;
}

// ---------------------------------------------------------------------------------------
// inference: the network on register-resident fragments
// ---------------------------------------------------------------------------------------
constexpr int kW1Stride = kSurK1 + 8;     // padded FP16 row strides: 16-byte aligned rows whose
constexpr int kWStride = kSurHid + 8;     // 8-row ldmatrix groups hit distinct bank quads
constexpr int kXStride = kSurK1 + 8;
struct SurSmem {
  __half w1[kSurHid][kW1Stride];           // W[out][in], FP16
  __half w2[kSurHid][kWStride];
  __half w3[kSurHid][kWStride];
  __half w4[kSurN4][kWStride];
  float b1[kSurHid], b2[kSurHid], b3[kSurHid], b4[kSurN4];
  alignas(16) __half xin[4][32][kXStride];   // per-warp staged inputs
  float yout[4][32][kSurN4];                 // per-warp outputs
};

// The hidden activations are carried as 2 GELU(z) (one FP16 operation less per pair of
// values), so the weights that consume them, W2, W3 and W4, are stored halved: exact in FP16.
__device__ void load_sur_weights(SurSmem& s, const float* __restrict__ prm) {
  for (int i = threadIdx.x; i < kSurHid * kW1Stride; i += blockDim.x) {
    const int n = i / kW1Stride, k = i % kW1Stride;
    s.w1[n][k] = __float2half_rn(k < kSurIn ? prm[kOffW1 + n * kSurIn + k] : 0.0f);
  }
  for (int i = threadIdx.x; i < kSurHid * kWStride; i += blockDim.x) {
    const int n = i / kWStride, k = i % kWStride;
    s.w2[n][k] = __hmul(__float2half_rn(k < kSurHid ? prm[kOffW2 + n * kSurHid + k] : 0.0f), __float2half(0.5f));
    s.w3[n][k] = __hmul(__float2half_rn(k < kSurHid ? prm[kOffW3 + n * kSurHid + k] : 0.0f), __float2half(0.5f));
  }
  for (int i = threadIdx.x; i < kSurN4 * kWStride; i += blockDim.x) {
    const int n = i / kWStride, k = i % kWStride;
    s.w4[n][k] = __hmul(__float2half_rn(n < kSurOut && k < kSurHid ? prm[kOffW4 + n * kSurHid + k] : 0.0f),
                        __float2half(0.5f));
  }
  for (int i = threadIdx.x; i < kSurHid; i += blockDim.x) {
    s.b1[i] = prm[kOffB1 + i];
    s.b2[i] = prm[kOffB2 + i];
    s.b3[i] = prm[kOffB3 + i];
  }
  for (int i = threadIdx.x; i < kSurN4; i += blockDim.x) s.b4[i] = i < kSurOut ? prm[kOffB4 + i] : 0.0f;
}

// hidden layer on a 16-row tile: acc[8 n8 tiles][4] = bias + a W^T.  One ldmatrix.x4 gives the
// B fragments of two n8 tiles for one k16 block (matrices: tile j k0-7, tile j k8-15,
// tile j+1 k0-7, tile j+1 k8-15); the first k16 block takes the bias as its accumulator input.
template <int KBLOCKS, int WSTRIDE>
__device__ __forceinline__ void layer_hidden(const __half (*w)[WSTRIDE], const float* b, const uint32_t (*a)[4],
                                             float (*acc)[4]) {
  const int lane = threadIdx.x & 31, t = lane & 3, mat = lane >> 3, r = lane & 7;
#pragma unroll
  for (int j = 0; j < 8; j += 2) {
    const float2 b0 = *reinterpret_cast<const float2*>(&b[j * 8 + 2 * t]);
    const float2 b1 = *reinterpret_cast<const float2*>(&b[(j + 1) * 8 + 2 * t]);
#pragma unroll
    for (int kb = 0; kb < KBLOCKS; ++kb) {
      uint32_t f[4];
      ldsm_x4(f, &w[(j + (mat >> 1)) * 8 + r][kb * 16 + (mat & 1) * 8]);
      if (kb == 0) {
        mma_16816_bias(acc[j], a[0], f, b0.x, b0.y);
        mma_16816_bias(acc[j + 1], a[0], f + 2, b1.x, b1.y);
      } else {
        mma_16816(acc[j], a[kb], f, __half());
        mma_16816(acc[j + 1], a[kb], f + 2, __half());
      }
    }
  }
}

// output layer (one n8 tile, four k16 blocks): one ldmatrix.x4 covers two k16 blocks
__device__ __forceinline__ void layer_out(const __half (*w)[kWStride], const float* b, const uint32_t (*a)[4],
                                          float* acc) {
  const int lane = threadIdx.x & 31, t = lane & 3, mat = lane >> 3, r = lane & 7;
  const float2 bb = *reinterpret_cast<const float2*>(&b[2 * t]);
#pragma unroll
  for (int kb = 0; kb < 4; kb += 2) {
    uint32_t f[4];
    ldsm_x4(f, &w[r][kb * 16 + mat * 8]);
    if (kb == 0) mma_16816_bias(acc, a[0], f, bb.x, bb.y);
    else mma_16816(acc, a[kb], f, __half());
    mma_16816(acc, a[kb + 1], f + 2, __half());
  }
}

// 2 GELU on the accumulators (rounded to FP16, packed arithmetic), repacked as the next
// layer's A fragments: k16 block kb takes the n8 tiles 2kb and 2kb+1
__device__ __forceinline__ void act_to_a(const float (*acc)[4], uint32_t (*a)[4]) {
#pragma unroll
  for (int kb = 0; kb < 4; ++kb) {
    a[kb][0] = h2_bits(gelu2x_h2(__floats2half2_rn(acc[2 * kb][0], acc[2 * kb][1])));
    a[kb][1] = h2_bits(gelu2x_h2(__floats2half2_rn(acc[2 * kb][2], acc[2 * kb][3])));
    a[kb][2] = h2_bits(gelu2x_h2(__floats2half2_rn(acc[2 * kb + 1][0], acc[2 * kb + 1][1])));
    a[kb][3] = h2_bits(gelu2x_h2(__floats2half2_rn(acc[2 * kb + 1][2], acc[2 * kb + 1][3])));
  }
}

// the network on the warp's 32 staged rows (xin -> yout).  All 32 lanes must call it.
__device__ void mlp_warp32(SurSmem& s, int warp) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3, mat = lane >> 3, r = lane & 7;
  float (*yout)[kSurN4] = s.yout[warp];
#pragma unroll 1
  for (int tile = 0; tile < 2; ++tile) {
    const int r0 = tile * 16;
    uint32_t a[4][4];
    // A fragment of the input tile (matrices: rows 0-7 k0-7, rows 8-15 k0-7, rows 0-7 k8-15,
    // rows 8-15 k8-15)
    ldsm_x4(a[0], &s.xin[warp][r0 + (mat & 1) * 8 + r][(mat >> 1) * 8]);
    float acc[8][4];
    layer_hidden<1, kW1Stride>(s.w1, s.b1, a, acc);
    act_to_a(acc, a);
    layer_hidden<4, kWStride>(s.w2, s.b2, a, acc);
    act_to_a(acc, a);
    layer_hidden<4, kWStride>(s.w3, s.b3, a, acc);
    act_to_a(acc, a);
    layer_out(s.w4, s.b4, a, acc[0]);
    yout[r0 + g][2 * t] = acc[0][0];
    yout[r0 + g][2 * t + 1] = acc[0][1];
    yout[r0 + g + 8][2 * t] = acc[0][2];
    yout[r0 + g + 8][2 * t + 1] = acc[0][3];
  }
  __syncwarp();
}

// stage one lane's canonical input row (zeros when the lane has no accepted pair)
__device__ __forceinline__ void stage_row(SurSmem& s, int warp, int lane, const float* x, bool use) {
  __half* row = s.xin[warp][lane];
#pragma unroll
  for (int j = 0; j < kSurK1; j += 2) {
    const float lo = (j < kSurIn && use) ? x[j] : 0.0f;
    const float hi = (j + 1 < kSurIn && use) ? x[j + 1] : 0.0f;
    *reinterpret_cast<uint32_t*>(row + j) = pack_f16(lo, hi);
  }
}

// raw network on canonical inputs X [B][6] -> Y [B][3] (tests and diagnostics)
__global__ void __launch_bounds__(128) surrogate_forward_kernel(const float* __restrict__ prm,
                                                                const float* __restrict__ X, int64_t B,
                                                                float* __restrict__ Y) {
  __shared__ __align__(16) SurSmem s;
  load_sur_weights(s, prm);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t nch = (B + 31) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t ch = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; ch < nch; ch += nw) {
    const int64_t i = ch * 32 + lane;
    float x[6] = {0, 0, 0, 0, 0, 0};
    if (i < B) {
#pragma unroll
      for (int j = 0; j < 6; ++j) x[j] = X[6 * i + j];
    }
    stage_row(s, warp, lane, x, i < B);
    __syncwarp();
    mlp_warp32(s, warp);
    if (i < B) {
#pragma unroll
      for (int j = 0; j < 3; ++j) Y[3 * i + j] = s.yout[warp][lane][j];
    }
    __syncwarp();
  }
}

struct SurArgs {
  const float* prm;               // FP32 master parameters
  double C, H, invH;
  float* vals;                    // per-pair (gamma, dgamma/dx, dgamma/dy), world units [P][3]
  int32_t* accepted;              // optional per-pair guard result [P]
  int64_t* fb_list;               // fallback pair indices from the front, audited ones from the back (capacity P)
  unsigned long long* fb_count;   // number of fallback entries in fb_list
  // serving-time audit: one accepted pair in audit_period (0: none) is also evaluated
  // analytically; au_* are zeroed device counters
  int audit_period;
  unsigned audit_shift;           // 64 - log2(audit_period)
  float audit_tol;                // error bound in units of the output scales
  float grad_scale;               // scale of the gradient outputs, 2 C int_0^1 k(q) dq / H
  unsigned long long* au_count;   // audited pairs (entries at the back of fb_list)
  unsigned long long* au_over;    // audited pairs with an error above audit_tol
  unsigned* au_max;               // largest audited error (float bits; errors are >= 0)
  unsigned long long* tc_timeouts; // tensor-core serving: MMA waits that ran out (pairs then fall back)
};

// whether accepted pair q is audited: a multiplicative hash of its index falls in the first
// of audit_period buckets (audit_period a power of two)
__device__ __forceinline__ bool audited(const SurArgs& sa, int64_t q) {
  if (sa.audit_period <= 0) return false;
  if (sa.audit_period == 1) return true;
  return ((unsigned long long)q * 0x9E3779B97F4A7C15ull) >> sa.audit_shift == 0ull;
}

// per-pair FP32 local frame for the two pair sources: independent pairs (double [P][8]) or
// the culled pair list (FP32 particles and triangles, same arithmetic as the analytic kernel)
template <bool LIST>
__device__ __forceinline__ void load_local(const IntArgs& a, const double* pairs, int64_t q, float ih, float* lf) {
  if (LIST) {
    const float4 p = a.parts[__ldg(a.pair_pid + q)];
    const float* t = a.tris + 6 * int64_t(__ldg(a.pair_tri + q));
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      lf[2 * j] = (__ldg(t + 2 * j) - p.x) * ih;
      lf[2 * j + 1] = (__ldg(t + 2 * j + 1) - p.y) * ih;
    }
  } else {
    double ld[6];
    pair_local(pairs + 8 * q, a.invH, ld, lf);
  }
}

template <int KID, bool LIST>
__global__ void __launch_bounds__(128, 6) surrogate_values_kernel(IntArgs a, const double* __restrict__ pairs,
                                                               SurArgs sa) {
  __shared__ __align__(16) SurSmem s;
  load_sur_weights(s, sa.prm);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t nch = (a.P + 31) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  const float ih = float(a.invH);
  for (int64_t ch = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; ch < nch; ch += nw) {
    const int64_t q = ch * 32 + lane;
    float lf[6] = {0, 0, 0, 0, 0, 0};
    if (q < a.P) load_local<LIST>(a, pairs, q, ih, lf);
    const Canon c = canonicalize(lf);
    const bool use = (q < a.P) && c.accept;
    stage_row(s, warp, lane, c.x, use);
    __syncwarp();
    mlp_warp32(s, warp);
    if (use) {
      const float* y = s.yout[warp][lane];
      float lx, ly;
      uncanonicalize_grad(c, c.area * y[1], c.area * y[2], lx, ly);
      sa.vals[3 * q] = c.area * y[0];
      sa.vals[3 * q + 1] = lx * ih;
      sa.vals[3 * q + 2] = ly * ih;
    }
    if (sa.accepted && q < a.P) sa.accepted[q] = use ? 1 : 0;
    // append the rejected pairs to the fallback list, one atomic per warp
    const unsigned rej = __ballot_sync(0xffffffffu, (q < a.P) && !use);
    if (rej) {
      unsigned long long base = 0;
      const int leader = __ffs(rej) - 1;
      if (lane == leader) base = atomicAdd(sa.fb_count, (unsigned long long)__popc(rej));
      base = __shfl_sync(0xffffffffu, base, leader);
      if ((q < a.P) && !use) sa.fb_list[base + __popc(rej & ((1u << lane) - 1u))] = q;
    }
    // and the audited ones to the back of the same list (a pair is in at most one part, so
    // the two parts never meet)
    const bool aud = use && audited(sa, q);
    const unsigned am = __ballot_sync(0xffffffffu, aud);
    if (am) {
      unsigned long long base = 0;
      const int leader = __ffs(am) - 1;
      if (lane == leader) base = atomicAdd(sa.au_count, (unsigned long long)__popc(am));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (aud) sa.fb_list[a.P - 1 - int64_t(base + __popc(am & ((1u << lane) - 1u)))] = q;
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------------------
// Serving on the fifth-generation tensor cores (tcgen05), the alternative to the mma.sync
// values kernel above.  A CTA of four warps takes 128 pairs at a time.  Each layer is a
// 128 x N x 16 sequence of kind::f16 MMAs (FP16 operands from shared memory, FP32 accumulators
// in tensor memory) issued by one thread; every thread then reads its row's accumulators with
// tcgen05.ld, adds the bias, applies the same packed-FP16 2 GELU as the mma.sync kernel and
// writes the row back to shared memory as the next layer's A operand (K-major core matrices,
// umma.cuh).  An MMA whose completion wait runs out of its poll budget sends the CTA's pairs to
// the analytic fallback from then on (results stay correct) and is counted.
// ---------------------------------------------------------------------------------------
struct SurTcSmem {
  __half w1[kSurHid * 16];      // layer-1 B operand: N = 64 rows, K = 16 (6 inputs, zero padded)
  __half w2[kSurHid * kSurHid];
  __half w3[kSurHid * kSurHid];
  __half w4[16 * kSurHid];      // output layer: N = 16 (3 outputs, zero padded)
  __half a0[128 * 16];          // the tile's canonical inputs
  __half act[128 * kSurHid];    // the tile's activations (2 GELU) between layers
  float b1[kSurHid], b2[kSurHid], b3[kSurHid], b4[16];
  uint64_t mbar;
  uint32_t tmem;
};

// the same FP16 values as load_sur_weights (W2, W3, W4 halved for the 2 GELU activations), in
// the tensor core's K-major layout
__device__ void load_tc_weights(SurTcSmem& s, const float* __restrict__ prm) {
  using umma::kmajor_offset;
  for (int i = threadIdx.x; i < kSurHid * 16; i += blockDim.x) {
    const int n = i / 16, k = i % 16;
    s.w1[kmajor_offset(n, k, 16) / 2] = __float2half_rn(k < kSurIn ? prm[kOffW1 + n * kSurIn + k] : 0.0f);
  }
  for (int i = threadIdx.x; i < kSurHid * kSurHid; i += blockDim.x) {
    const int n = i / kSurHid, k = i % kSurHid;
    s.w2[kmajor_offset(n, k, kSurHid) / 2] = __hmul(__float2half_rn(prm[kOffW2 + n * kSurHid + k]), __float2half(0.5f));
    s.w3[kmajor_offset(n, k, kSurHid) / 2] = __hmul(__float2half_rn(prm[kOffW3 + n * kSurHid + k]), __float2half(0.5f));
  }
  for (int i = threadIdx.x; i < 16 * kSurHid; i += blockDim.x) {
    const int n = i / kSurHid, k = i % kSurHid;
    s.w4[kmajor_offset(n, k, kSurHid) / 2] =
        __hmul(__float2half_rn(n < kSurOut ? prm[kOffW4 + n * kSurHid + k] : 0.0f), __float2half(0.5f));
  }
  for (int i = threadIdx.x; i < kSurHid; i += blockDim.x) {
    s.b1[i] = prm[kOffB1 + i];
    s.b2[i] = prm[kOffB2 + i];
    s.b3[i] = prm[kOffB3 + i];
  }
  for (int i = threadIdx.x; i < 16; i += blockDim.x) s.b4[i] = i < kSurOut ? prm[kOffB4 + i] : 0.0f;
}

constexpr uint32_t kTcSpin = 1u << 22;          // polls of an MMA completion wait before giving up

// wait for the next MMA completion on the CTA's mbarrier; the CTA agrees on the outcome
__device__ __forceinline__ bool tc_wait(SurTcSmem& s, uint32_t& phase) {
  const bool ok = __syncthreads_and(umma::mbar_wait(&s.mbar, phase, kTcSpin) ? 1 : 0) != 0;
  if (ok) phase ^= 1u;
  umma::fence_after_sync();
  return ok;
}

// this thread's row of a hidden layer: accumulators + bias -> FP16 -> 2 GELU -> the next A operand
__device__ __forceinline__ void tc_hidden_row(const SurTcSmem& s, uint32_t trow, const float* bias, __half* act, int row) {
  float acc[kSurHid];
  umma::tmem_ld64(trow, acc);
#pragma unroll
  for (int c16 = 0; c16 < kSurHid / 16; ++c16) {
    const float* v = acc + 16 * c16;
    uint32_t w[8];
#pragma unroll
    for (int j = 0; j < 8; ++j)
      w[j] = h2_bits(gelu2x_h2(__floats2half2_rn(v[2 * j] + bias[16 * c16 + 2 * j], v[2 * j + 1] + bias[16 * c16 + 2 * j + 1])));
    *reinterpret_cast<uint4*>(act + umma::kmajor_offset(row, 16 * c16, kSurHid) / 2) = make_uint4(w[0], w[1], w[2], w[3]);
    *reinterpret_cast<uint4*>(act + umma::kmajor_offset(row, 16 * c16 + 8, kSurHid) / 2) = make_uint4(w[4], w[5], w[6], w[7]);
  }
}

// one thread issues a layer: D[tm] = A (K = 16 kblocks) x B^T, then commits to the mbarrier
__device__ __forceinline__ void tc_issue(SurTcSmem& s, uint32_t tm, uint32_t a_addr, uint32_t b_addr, int kblocks,
                                         uint32_t a_sbo, uint32_t b_sbo, uint32_t idesc) {
  umma::fence_after_sync();
  for (int kb = 0; kb < kblocks; ++kb)
    umma::mma_f16(tm, umma::smem_desc(a_addr + 256 * kb, 128, a_sbo), umma::smem_desc(b_addr + 256 * kb, 128, b_sbo),
                  idesc, kb > 0);
  umma::mma_commit(&s.mbar);
}

template <int KID, bool LIST>
__global__ void __launch_bounds__(128) surrogate_values_tc_kernel(IntArgs a, const double* __restrict__ pairs,
                                                                  SurArgs sa) {
  __shared__ __align__(128) SurTcSmem s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  load_tc_weights(s, sa.prm);
  if (warp == 0) {
    umma::tmem_alloc(&s.tmem, 64);
    umma::tmem_relinquish();
  }
  if (tid == 0) {
    umma::mbar_init(&s.mbar, 1);
    umma::mbar_init_fence();
  }
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tm = s.tmem, trow = tm + (uint32_t(32 * warp) << 16);
  const uint32_t sa0 = umma::smem_u32(s.a0), sact = umma::smem_u32(s.act);
  const uint32_t sw1 = umma::smem_u32(s.w1), sw2 = umma::smem_u32(s.w2), sw3 = umma::smem_u32(s.w3),
                 sw4 = umma::smem_u32(s.w4);
  constexpr uint32_t ID64 = umma::idesc_f16(128, 64, false), ID16 = umma::idesc_f16(128, 16, false);
  uint32_t phase = 0;
  bool healthy = true;
  unsigned long long timeouts = 0;
  const float ih = float(a.invH);
  const int64_t ntiles = (a.P + 127) / 128;
  // Software pipeline over the CTA's tiles (t, t + grid, ...), so that work that does not depend
  // on the tensor core overlaps its MMAs: tile t+2's local frame is loaded while tile t runs;
  // tile t+1's canonical frame is computed and its input row staged while tile t's output
  // layer runs (the input operand is free once tile t's first layer has completed); tile t's
  // epilogue (values, guard flags, fallback and audit lists) runs while tile t+1's first
  // layer runs.
  auto stage_input = [&](const Canon& c, bool use) {
    uint32_t w[8];
#pragma unroll
    for (int j = 0; j < 8; ++j)
      w[j] = pack_f16(2 * j < kSurIn && use ? c.x[2 * j] : 0.0f, 2 * j + 1 < kSurIn && use ? c.x[2 * j + 1] : 0.0f);
    *reinterpret_cast<uint4*>(s.a0 + umma::kmajor_offset(tid, 0, 16) / 2) = make_uint4(w[0], w[1], w[2], w[3]);
    *reinterpret_cast<uint4*>(s.a0 + umma::kmajor_offset(tid, 8, 16) / 2) = make_uint4(w[4], w[5], w[6], w[7]);
  };
  // one tile's results: values of the accepted pairs, guard flags, fallback and audit entries
  // (every thread of the CTA calls it: the list appends are warp-wide)
  auto epilogue = [&](int64_t q, const Canon& c, bool use, const float* y) {
    if (use) {
      float lx, ly;
      uncanonicalize_grad(c, c.area * y[1], c.area * y[2], lx, ly);
      sa.vals[3 * q] = c.area * y[0];
      sa.vals[3 * q + 1] = lx * ih;
      sa.vals[3 * q + 2] = ly * ih;
    }
    if (sa.accepted && q < a.P) sa.accepted[q] = use ? 1 : 0;
    const unsigned rej = __ballot_sync(0xffffffffu, (q < a.P) && !use);
    if (rej) {
      unsigned long long base = 0;
      const int leader = __ffs(rej) - 1;
      if (lane == leader) base = atomicAdd(sa.fb_count, (unsigned long long)__popc(rej));
      base = __shfl_sync(0xffffffffu, base, leader);
      if ((q < a.P) && !use) sa.fb_list[base + __popc(rej & ((1u << lane) - 1u))] = q;
    }
    const bool aud = use && audited(sa, q);
    const unsigned am = __ballot_sync(0xffffffffu, aud);
    if (am) {
      unsigned long long base = 0;
      const int leader = __ffs(am) - 1;
      if (lane == leader) base = atomicAdd(sa.au_count, (unsigned long long)__popc(am));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (aud) sa.fb_list[a.P - 1 - int64_t(base + __popc(am & ((1u << lane) - 1u)))] = q;
    }
  };
  int64_t tile = blockIdx.x;
  float lf[6] = {0, 0, 0, 0, 0, 0}, lnext[6] = {0, 0, 0, 0, 0, 0};
  if (tile * 128 + tid < a.P) load_local<LIST>(a, pairs, tile * 128 + tid, ih, lf);
  if ((tile + gridDim.x) * 128 + tid < a.P) load_local<LIST>(a, pairs, (tile + gridDim.x) * 128 + tid, ih, lnext);
  Canon c_cur = canonicalize(lf);
  bool use_cur = tile * 128 + tid < a.P && c_cur.accept;
  stage_input(c_cur, use_cur);
  Canon c_prev = c_cur;
  bool use_prev = false, have_prev = false;
  int64_t q_prev = 0;
  float y_prev[3] = {0, 0, 0};
  const float* bias[3] = {s.b1, s.b2, s.b3};
  const uint32_t wl[3] = {sw2, sw3, sw4};
  for (; tile < ntiles; tile += gridDim.x) {
    const int64_t q = tile * 128 + tid;
    bool tile_ok = healthy;
    umma::fence_proxy_async();
    umma::fence_before_sync();
    __syncthreads();
    if (healthy && tid == 0) tc_issue(s, tm, sa0, sw1, 1, 256, 256, ID64);
    if (have_prev) epilogue(q_prev, c_prev, use_prev, y_prev);
    if (healthy) tile_ok = tc_wait(s, phase);
#pragma unroll 1
    for (int l = 0; l < 3 && tile_ok; ++l) {
      tc_hidden_row(s, trow, bias[l], s.act, tid);
      umma::fence_proxy_async();
      umma::fence_before_sync();
      __syncthreads();
      if (tid == 0) tc_issue(s, tm, sact, wl[l], 4, 1024, 1024, l < 2 ? ID64 : ID16);
      if (l < 2) tile_ok = tc_wait(s, phase);
    }
    // the output layer's MMA is in flight (if the tile is healthy): the next tile's inputs
    const int64_t qn = q + int64_t(gridDim.x) * 128;
    const Canon c_next = canonicalize(lnext);
    const bool use_next = qn < a.P && c_next.accept;
    stage_input(c_next, use_next);
    if (qn + int64_t(gridDim.x) * 128 < a.P) load_local<LIST>(a, pairs, qn + int64_t(gridDim.x) * 128, ih, lnext);
    if (tile_ok) tile_ok = tc_wait(s, phase);
    float y[16];
    if (tile_ok) {
      umma::tmem_ld16(trow, y);
#pragma unroll
      for (int j = 0; j < kSurOut; ++j) y_prev[j] = y[j] + s.b4[j];
    } else if (healthy) {
      healthy = false;
      ++timeouts;
    }
    c_prev = c_cur;
    use_prev = use_cur && tile_ok;
    q_prev = q;
    have_prev = true;
    c_cur = c_next;
    use_cur = use_next;
  }
  if (have_prev) epilogue(q_prev, c_prev, use_prev, y_prev);
  if (!healthy) umma::mbar_wait(&s.mbar, phase, kTcSpin);   // let an overdue MMA drain
  umma::fence_before_sync();
  __syncthreads();
  if (warp == 0) umma::tmem_dealloc(tm, 64);
  if (tid == 0 && timeouts) atomicAdd(sa.tc_timeouts, timeouts);
}

// the analytic FP32 path (with the FP64 fix-up for far or non-finite geometry) for pair q
template <int KID, bool LIST>
__device__ __forceinline__ void analytic_pair(const IntArgs& a, const double* pairs, int64_t q, float* v) {
  if (LIST) {
    eval_pair<float, KID, 0>(a, __ldg(a.pair_pid + q), __ldg(a.pair_tri + q), v);
  } else {
    double ld[6];
    float lf[6];
    pair_local(pairs + 8 * q, a.invH, ld, lf);
    eval_mode<float, KID, 0>(ld, a.C, a.invH, v);
  }
}

// the analytic path over the fallback list, then over the audited pairs: each audited pair's
// network value is judged against its analytic value, which replaces it
template <int KID, bool LIST>
__global__ void __launch_bounds__(128) surrogate_fallback_kernel(IntArgs a, const double* __restrict__ pairs,
                                                                 SurArgs sa) {
  const int64_t n = int64_t(*sa.fb_count);
  const int64_t na = sa.audit_period > 0 ? int64_t(*sa.au_count) : 0;
  float emax = 0.0f;
  unsigned over = 0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n + na; i += int64_t(gridDim.x) * blockDim.x) {
    const bool aud = i >= n;
    const int64_t q = aud ? sa.fb_list[a.P - 1 - (i - n)] : sa.fb_list[i];
    float v[3];
    analytic_pair<KID, LIST>(a, pairs, q, v);
    if (aud) {
      const float s[3] = {1.0f, sa.grad_scale, sa.grad_scale};
      float e = 0.0f;
#pragma unroll
      for (int k = 0; k < 3; ++k) e = fmaxf(e, fabsf(sa.vals[3 * q + k] - v[k]) / fmaxf(fabsf(v[k]), s[k]));
      if (!(e <= sa.audit_tol)) ++over;           // NaN counts as over
      emax = fmaxf(emax, isfinite(e) ? e : 3.0e38f);
    }
    sa.vals[3 * q] = v[0];
    sa.vals[3 * q + 1] = v[1];
    sa.vals[3 * q + 2] = v[2];
  }
  if (sa.audit_period > 0) {
    const unsigned wmax = __reduce_max_sync(0xffffffffu, __float_as_uint(emax));
    const unsigned wover = __reduce_add_sync(0xffffffffu, over);
    if ((threadIdx.x & 31) == 0) {
      if (wmax) atomicMax(sa.au_max, wmax);
      if (wover) atomicAdd(sa.au_over, (unsigned long long)wover);
    }
  }
}

// the audit's verdict: if an audited pair was off by more than the bound, the network is not
// trusted for this call and every pair is evaluated analytically (and reported as not
// accepted); otherwise the kernel returns at once
template <int KID, bool LIST>
__global__ void __launch_bounds__(128) surrogate_redo_kernel(IntArgs a, const double* __restrict__ pairs,
                                                             SurArgs sa) {
  if (*sa.au_over == 0ull) return;
  for (int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < a.P; q += int64_t(gridDim.x) * blockDim.x) {
    float v[3];
    analytic_pair<KID, LIST>(a, pairs, q, v);
    sa.vals[3 * q] = v[0];
    sa.vals[3 * q + 1] = v[1];
    sa.vals[3 * q + 2] = v[2];
    if (sa.accepted) sa.accepted[q] = 0;
  }
}

// per-particle sums of the per-pair values in pair order (chunk reduction + crossing slots,
// completed by finalize_kernel)
__global__ void __launch_bounds__(128) reduce_vals_kernel(IntArgs a, const float* __restrict__ vals) {
  constexpr int NV = 3;
  const int lane = threadIdx.x & 31;
  const int64_t nchunks = (a.P + 31) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t ch = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; ch < nchunks; ch += nw) {
    const int64_t q = ch * 32 + lane;
    int pid = -1;
    float v[NV] = {0.0f, 0.0f, 0.0f};
    if (q < a.P) {
      pid = __ldg(a.pair_pid + q);
#pragma unroll
      for (int i = 0; i < NV; ++i) v[i] = vals[3 * q + i];
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int pn = __shfl_down_sync(0xffffffffu, pid, o);
      const bool same = (lane + o < 32) && (pn == pid);
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        const float tv = __shfl_down_sync(0xffffffffu, v[i], o);
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
      if (s0 >= cs && s1 <= cs + 32) write_particle<float, 0>(a, pid, v);
      float* slots = static_cast<float*>(a.slots);
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

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------
static unsigned nblk(int64_t n, int b = 256) { return unsigned((n + b - 1) / b); }

// occupancy-limited persistent grid of 128-thread blocks, no larger than the work needs
template <typename K>
static unsigned persistent_grid(Ctx* c, K kern, int64_t blocks_wanted) {
  int per_sm = 0, sms = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, 0);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  const int64_t cap = int64_t(per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
  const int64_t want = blocks_wanted > 0 ? blocks_wanted : 1;
  return unsigned(want < cap ? want : cap);
}

template <typename T>
static sph2d_status gemm(Ctx* c, int M, int N, int K, const float* A, int lda, int ta, const float* B,
                         int ldb, int tb, float* C, int ldc) {
  const bool tc = c->sur_train_engine == 1;
  const int bm = tc ? UBM : GBM, bn = tc ? UBN : GBN;
  // split K when the output tile grid is small and K is long (weight gradients over the batch)
  const int tiles = ((M + bm - 1) / bm) * ((N + bn - 1) / bn);
  // (the tcgen05 engine waits on each K block's MMA, so it takes shorter splits: K / 256)
  int splits = 1;
  if (K >= 4096 && tiles < 64) splits = tc ? std::min(128, K / 256) : std::min(64, K / 1024);
  dim3 grid((M + bm - 1) / bm, (N + bn - 1) / bn, splits);
  float* out = C;
  int ldo = ldc;
  if (splits > 1) {
    sph2d_status s = ensure(c, c->sur_split, size_t(splits) * M * N * sizeof(float));
    if (s != SPH2D_OK) return s;
    out = static_cast<float*>(c->sur_split.ptr);
    ldo = N;
  }
  if (tc) {
    sph2d_status s = ensure(c, c->host_flags_dev, 64);
    if (s != SPH2D_OK) return s;
    auto* tmo = static_cast<unsigned long long*>(c->host_flags_dev.ptr) + 7;
    SPH2D_LAUNCH(c, (gemm_umma_kernel<T>), grid, 128, M, N, K, A, lda, ta, B, ldb, tb, out, ldo, 1.0f, splits, tmo);
  } else {
    SPH2D_LAUNCH(c, (gemm_tc_kernel<T>), grid, 128, M, N, K, A, lda, ta, B, ldb, tb, out, ldo, 1.0f, splits);
  }
  if (splits == 1) return SPH2D_OK;
  float* part = out;
  SPH2D_LAUNCH(c, (splitk_reduce_kernel), nblk(int64_t(M) * N), 256, part, splits, M, N, C, ldc, 1.0f);
  return SPH2D_OK;
}

// one forward + backward over a batch (Xb [B][6], Tb [B][3]) -> grad (flat parameter layout)
// and the batch loss (device scalar)
static sph2d_status sur_grad_batch(Ctx* c, const float* prm, const float* Xb, const float* Tb, int64_t B,
                                   float* grad, float* loss_dev) {
  const int Hd = kSurHid;
  const int64_t lb = (B * 3 + 255) / 256;
  sph2d_status s = ensure(c, c->sur_act, size_t(B * (6 * Hd + 6) + lb) * sizeof(float));
  if (s != SPH2D_OK) return s;
  float* base = static_cast<float*>(c->sur_act.ptr);
  float *Z1 = base, *H1 = Z1 + B * Hd, *Z2 = H1 + B * Hd, *H2 = Z2 + B * Hd, *Z3 = H2 + B * Hd;
  float *H3 = Z3 + B * Hd, *Y = H3 + B * Hd, *dY = Y + B * 3, *part = dY + B * 3;
  const int iB = int(B);
#define SUR_FWD(...)                                                   \
  do {                                                                 \
    if ((s = gemm<__half>(c, __VA_ARGS__)) != SPH2D_OK) return s;      \
  } while (0)
#define SUR_BWD(...)                                                   \
  do {                                                                 \
    if ((s = gemm<__nv_bfloat16>(c, __VA_ARGS__)) != SPH2D_OK) return s; \
  } while (0)
  // forward (FP16 operands): Z = H_prev W^T + b, H = GELU(Z)
  SUR_FWD(iB, Hd, kSurIn, Xb, kSurIn, 0, prm + kOffW1, kSurIn, 0, Z1, Hd);
  SPH2D_LAUNCH(c, (bias_gelu_kernel), nblk(B * Hd / 2), 256, Z1, prm + kOffB1, H1, B, Hd);
  SUR_FWD(iB, Hd, Hd, H1, Hd, 0, prm + kOffW2, Hd, 0, Z2, Hd);
  SPH2D_LAUNCH(c, (bias_gelu_kernel), nblk(B * Hd / 2), 256, Z2, prm + kOffB2, H2, B, Hd);
  SUR_FWD(iB, Hd, Hd, H2, Hd, 0, prm + kOffW3, Hd, 0, Z3, Hd);
  SPH2D_LAUNCH(c, (bias_gelu_kernel), nblk(B * Hd / 2), 256, Z3, prm + kOffB3, H3, B, Hd);
  SUR_FWD(iB, kSurOut, Hd, H3, Hd, 0, prm + kOffW4, Hd, 0, Y, kSurOut);
  SPH2D_LAUNCH(c, (bias_kernel), nblk(B * 3), 256, Y, prm + kOffB4, B, kSurOut);
  SPH2D_LAUNCH(c, (loss_grad_kernel), unsigned(lb), 256, Y, Tb, B, c->sur_w[0], c->sur_w[1], c->sur_w[2], dY,
               part);
  SPH2D_LAUNCH(c, (sum_kernel), 1, 256, part, int(lb), loss_dev);
  // backward (BF16 operands).  dW = dZ^T H_prev, db = column sums of dZ, dH_prev = dZ W; each
  // dZ overwrites a buffer whose last reader has run: dZ3 -> H3, dZ2 -> Z3, dZ1 -> Z2.
  SUR_BWD(kSurOut, Hd, iB, dY, kSurOut, 1, H3, Hd, 1, grad + kOffW4, Hd);
  SPH2D_LAUNCH(c, (colsum_kernel), kSurOut, 256, dY, B, kSurOut, grad + kOffB4);
  float* dZ3 = H3;
  SUR_BWD(iB, Hd, kSurOut, dY, kSurOut, 0, prm + kOffW4, Hd, 1, dZ3, Hd);
  SPH2D_LAUNCH(c, (gelu_back_kernel), nblk(B * Hd), 256, dZ3, Z3, B * Hd);
  SUR_BWD(Hd, Hd, iB, dZ3, Hd, 1, H2, Hd, 1, grad + kOffW3, Hd);
  SPH2D_LAUNCH(c, (colsum_kernel), Hd, 256, dZ3, B, Hd, grad + kOffB3);
  float* dZ2 = Z3;
  SUR_BWD(iB, Hd, Hd, dZ3, Hd, 0, prm + kOffW3, Hd, 1, dZ2, Hd);
  SPH2D_LAUNCH(c, (gelu_back_kernel), nblk(B * Hd), 256, dZ2, Z2, B * Hd);
  SUR_BWD(Hd, Hd, iB, dZ2, Hd, 1, H1, Hd, 1, grad + kOffW2, Hd);
  SPH2D_LAUNCH(c, (colsum_kernel), Hd, 256, dZ2, B, Hd, grad + kOffB2);
  float* dZ1 = Z2;
  SUR_BWD(iB, Hd, Hd, dZ2, Hd, 0, prm + kOffW2, Hd, 1, dZ1, Hd);
  SPH2D_LAUNCH(c, (gelu_back_kernel), nblk(B * Hd), 256, dZ1, Z1, B * Hd);
  SUR_BWD(Hd, kSurIn, iB, dZ1, Hd, 1, Xb, kSurIn, 1, grad + kOffW1, kSurIn);
  SPH2D_LAUNCH(c, (colsum_kernel), Hd, 256, dZ1, B, Hd, grad + kOffB1);
#undef SUR_FWD
#undef SUR_BWD
  return SPH2D_OK;
}

// deterministic Glorot-uniform initialisation (host generator), biases zero
static void init_params(std::vector<float>& p, uint64_t seed) {
  std::mt19937_64 rng(seed);
  p.assign(kSurParams, 0.0f);
  auto fill = [&](int off, int fan_out, int fan_in) {
    const double lim = std::sqrt(6.0 / double(fan_in + fan_out));
    for (int i = 0; i < fan_out * fan_in; ++i) {
      const double u = double(rng() >> 11) * (1.0 / 9007199254740992.0);   // [0, 1)
      p[off + i] = float((2.0 * u - 1.0) * lim);
    }
  };
  fill(kOffW1, kSurHid, kSurIn);
  fill(kOffW2, kSurHid, kSurHid);
  fill(kOffW3, kSurHid, kSurHid);
  fill(kOffW4, kSurOut, kSurHid);
}

sph2d_status surrogate_init(Ctx* c, int kernel, uint64_t seed) {
  // masters, Adam first and second moments, one spare block
  sph2d_status s = ensure(c, c->sur_prm, 4 * size_t(kSurParams) * sizeof(float));
  if (s != SPH2D_OK) return s;
  std::vector<float> p;
  init_params(p, seed);
  float* prm = static_cast<float*>(c->sur_prm.ptr);
  cudaError_t e = cudaMemcpyAsync(prm, p.data(), kSurParams * sizeof(float), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(prm + kSurParams, 0, 3 * size_t(kSurParams) * sizeof(float), c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_err(c, e, "surrogate init");
  c->sur_kernel = kernel;
  c->sur_ready = true;
  c->sur_step = 0;
  // loss weights 1/scale^2: the averaged kernel is at most C, the averaged gradient about 2C
  const double C = kernel_C(kernel);
  c->sur_w[0] = float(1.0 / (C * C));
  c->sur_w[1] = c->sur_w[2] = float(1.0 / (4.0 * C * C));
  return SPH2D_OK;
}

sph2d_status surrogate_set_params(Ctx* c, const float* host) {
  cudaError_t e = cudaMemcpyAsync(c->sur_prm.ptr, host, kSurParams * sizeof(float), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_err(c, e, "surrogate params");
  return SPH2D_OK;
}

sph2d_status surrogate_get_params(Ctx* c, float* host) {
  cudaError_t e = cudaMemcpyAsync(host, c->sur_prm.ptr, kSurParams * sizeof(float), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_err(c, e, "surrogate params");
  return SPH2D_OK;
}

sph2d_status surrogate_grad(Ctx* c, const float* X, const float* T, int64_t B, float* grad, float* loss) {
  return sur_grad_batch(c, static_cast<const float*>(c->sur_prm.ptr), X, T, B, grad, loss);
}

sph2d_status surrogate_forward(Ctx* c, const float* X, int64_t B, float* Y) {
  if (B == 0) return SPH2D_OK;
  const unsigned g = persistent_grid(c, surrogate_forward_kernel, ((B + 31) / 32 + 3) / 4);
  SPH2D_LAUNCH(c, (surrogate_forward_kernel), g, 128, static_cast<const float*>(c->sur_prm.ptr), X, B, Y);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(c, e, "surrogate forward");
  return SPH2D_OK;
}

sph2d_status surrogate_train(Ctx* c, const double* pairs, int64_t P, double H, int epochs, int batch,
                             double lr, double wd, uint64_t seed, double* final_loss, int64_t* used) {
  cudaStream_t st = c->stream;
  // analytic labels in FP64: the closed form is the ground truth the network learns
  sph2d_status s = ensure(c, c->sur_data, size_t(P) * (3 * sizeof(double) + 9 * sizeof(float) + sizeof(int32_t)));
  if (s != SPH2D_OK) return s;
  double* ana = static_cast<double*>(c->sur_data.ptr);
  float* X = reinterpret_cast<float*>(ana + 3 * P);
  float* T = X + 6 * P;
  int32_t* ok = reinterpret_cast<int32_t*>(T + 3 * P);
  s = launch_pair_integrals(c, pairs, P, c->sur_kernel, H, -1, SPH2D_FP64, ana);
  if (s != SPH2D_OK) return s;
  SPH2D_LAUNCH(c, (canon_training_kernel), nblk(P), 256, pairs, ana, P, 1.0 / H, H, X, T, ok);
  // keep the rows inside the guard's domain
  std::vector<int32_t> okh(P);
  cudaError_t e = cudaMemcpyAsync(okh.data(), ok, P * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_err(c, e, "training labels");
  std::vector<int32_t> rows;
  rows.reserve(P);
  for (int64_t i = 0; i < P; ++i)
    if (okh[i]) rows.push_back(int32_t(i));
  const int64_t R = int64_t(rows.size());
  if (used) *used = R;
  if (R < batch) return set_err(c, SPH2D_ERR_INVALID_ARG, "fewer in-domain training pairs than one batch");
  s = ensure(c, c->sur_idx, size_t(R) * sizeof(int32_t) + size_t(batch) * 9 * sizeof(float) +
                                size_t(kSurParams + 64) * sizeof(float));
  if (s != SPH2D_OK) return s;
  int32_t* idx = static_cast<int32_t*>(c->sur_idx.ptr);
  float* Xb = reinterpret_cast<float*>(idx + R);
  float* Tb = Xb + size_t(batch) * 6;
  float* grad = Tb + size_t(batch) * 3;
  float* loss = grad + kSurParams;
  float* prm = static_cast<float*>(c->sur_prm.ptr);
  float *m = prm + kSurParams, *v = m + kSurParams;
  unsigned long long* tmo = nullptr;               // tensor-core GEMM waits that ran out
  if (c->sur_train_engine == 1) {
    s = ensure(c, c->host_flags_dev, 64);
    if (s != SPH2D_OK) return s;
    tmo = static_cast<unsigned long long*>(c->host_flags_dev.ptr) + 7;
    e = cudaMemsetAsync(tmo, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return cuda_err(c, e, "training");
  }
  std::mt19937_64 rng(seed);
  const int64_t steps_per = R / batch;
  const int64_t total = steps_per * epochs;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  int64_t step = 0;
  for (int ep = 0; ep < epochs; ++ep) {
    // Fisher-Yates with the context's own generator (identical on every platform)
    for (int64_t i = R - 1; i > 0; --i) std::swap(rows[i], rows[int64_t(rng() % uint64_t(i + 1))]);
    e = cudaMemcpyAsync(idx, rows.data(), R * sizeof(int32_t), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // rows is reshuffled next epoch
    if (e != cudaSuccess) return cuda_err(c, e, "training indices");
    for (int64_t b = 0; b < steps_per; ++b, ++step) {
      SPH2D_LAUNCH(c, (gather_rows_kernel), nblk(batch), 256, X, T, idx + b * batch, int64_t(batch), Xb, Tb);
      s = sur_grad_batch(c, prm, Xb, Tb, batch, grad, loss);
      if (s != SPH2D_OK) return s;
      // warm-up from lr/10 over the first 5% of the steps, then cosine decay to lr/100
      const double f = double(step) / double(total);
      const double lr_t = f < 0.05 ? lr * (0.1 + 0.9 * f / 0.05)
                                   : lr * (0.01 + 0.99 * 0.5 * (1.0 + std::cos(3.141592653589793 * (f - 0.05) / 0.95)));
      const int64_t tt = ++c->sur_step;
      SPH2D_LAUNCH(c, (adamw_kernel), nblk(kSurParams), 256, prm, grad, m, v, kSurParams, float(lr_t), b1, b2,
                   eps, float(wd), float(1.0 - std::pow(double(b1), double(tt))),
                   float(1.0 - std::pow(double(b2), double(tt))));
    }
  }
  float lh = 0.0f;
  unsigned long long nt = 0;
  e = cudaMemcpyAsync(&lh, loss, sizeof(float), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && tmo) e = cudaMemcpyAsync(&nt, tmo, sizeof(nt), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_err(c, e, "training");
  if (nt) return set_err(c, SPH2D_ERR_CUDA, "tensor-core GEMM: an MMA completion wait ran out of its poll budget");
  if (final_loss) *final_loss = lh;
  return SPH2D_OK;
}

// the values and fallback kernels for one pair source (fb_count already cleared)
// Resident CTAs of the tcgen05 serving kernel per SM, from its three limits: shared memory
// (static size plus the per-block reservation), registers, and tensor memory (64 of the SM's
// 512 columns per CTA).  The runtime's occupancy query reports one block per SM for this kernel,
// yet five run: measured 17.7 ms with one CTA per SM and 8.6 ms with five on the same pair list.
template <typename K>
static unsigned tc_grid(Ctx* c, K kern, int64_t wanted) {
  cudaFuncAttributes fa{};
  cudaFuncGetAttributes(&fa, kern);
  int smem_sm = 0, res = 0, regs_sm = 0, sms = 0;
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, c->device);
  cudaDeviceGetAttribute(&res, cudaDevAttrReservedSharedMemoryPerBlock, c->device);
  cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, c->device);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  const int64_t by_smem = int64_t(smem_sm) / std::max<int64_t>(1, int64_t(fa.sharedSizeBytes) + res);
  const int64_t by_regs = int64_t(regs_sm) / std::max<int64_t>(1, int64_t(fa.numRegs) * 128);
  const int64_t per_sm = std::max<int64_t>(1, std::min<int64_t>(std::min(by_smem, by_regs), std::min<int64_t>(512 / 64, 16)));
  const int64_t cap = per_sm * std::max(1, sms);
  const int64_t want = wanted > 0 ? wanted : 1;
  return unsigned(want < cap ? want : cap);
}

template <int KID, bool LIST>
static void launch_serving(Ctx* c, const IntArgs& a, const double* pairs, const SurArgs& sa) {
  if (c->sur_engine == 1) {
    const unsigned g1 = tc_grid(c, surrogate_values_tc_kernel<KID, LIST>, (a.P + 127) / 128);
    SPH2D_LAUNCH(c, (surrogate_values_tc_kernel<KID, LIST>), g1, 128, a, pairs, sa);
  } else {
    const int64_t nch = (a.P + 31) / 32;
    const unsigned g1 = persistent_grid(c, surrogate_values_kernel<KID, LIST>, (nch + 3) / 4);
    SPH2D_LAUNCH(c, (surrogate_values_kernel<KID, LIST>), g1, 128, a, pairs, sa);
  }
  // the list length is only known on the device: a persistent grid strides over it
  const unsigned g2 = persistent_grid(c, surrogate_fallback_kernel<KID, LIST>, (a.P + 127) / 128);
  SPH2D_LAUNCH(c, (surrogate_fallback_kernel<KID, LIST>), g2, 128, a, pairs, sa);
  if (sa.audit_period > 0) {
    const unsigned g3 = persistent_grid(c, surrogate_redo_kernel<KID, LIST>, (a.P + 127) / 128);
    SPH2D_LAUNCH(c, (surrogate_redo_kernel<KID, LIST>), g3, 128, a, pairs, sa);
  }
}

template <bool LIST>
static void dispatch_serving(Ctx* c, const IntArgs& a, const double* pairs, const SurArgs& sa) {
  switch (c->sur_kernel) {
    case KID_WC2: launch_serving<KID_WC2, LIST>(c, a, pairs, sa); break;
    case KID_WC4: launch_serving<KID_WC4, LIST>(c, a, pairs, sa); break;
    case KID_WC6: launch_serving<KID_WC6, LIST>(c, a, pairs, sa); break;
    default: launch_serving<KID_CUBIC, LIST>(c, a, pairs, sa); break;
  }
}

// counters in host_flags_dev: [2] fallback count, [3] audited pairs, [4] audited pairs over the
// bound, [5] largest audited error (float bits), [6] tensor-core MMA waits that ran out; copied
// to pinned[10..14] after the call
static sph2d_status serving_setup(Ctx* c, int64_t P, double H, SurArgs& sa) {
  sph2d_status s = ensure(c, c->sur_fb, size_t(P > 0 ? P : 1) * sizeof(int64_t));
  if (s == SPH2D_OK) s = ensure(c, c->host_flags_dev, 64);
  if (s != SPH2D_OK) return s;
  auto* flags = static_cast<unsigned long long*>(c->host_flags_dev.ptr);
  sa.prm = static_cast<const float*>(c->sur_prm.ptr);
  sa.fb_list = static_cast<int64_t*>(c->sur_fb.ptr);
  sa.fb_count = flags + 2;
  sa.au_count = flags + 3;
  sa.au_over = flags + 4;
  sa.au_max = reinterpret_cast<unsigned*>(flags + 5);
  sa.tc_timeouts = flags + 6;
  sa.audit_period = c->sur_audit_period;
  int lg = 0;
  while ((1 << lg) < sa.audit_period) ++lg;
  sa.audit_shift = unsigned(64 - lg);
  sa.audit_tol = float(c->sur_audit_tol);
  sa.grad_scale = float(2.0 * kernel_C(c->sur_kernel) * kernel_int0(c->sur_kernel) / H);
  cudaError_t e = cudaMemsetAsync(sa.fb_count, 0, 5 * sizeof(unsigned long long), c->stream);
  if (e != cudaSuccess) return cuda_err(c, e, "memset");
  return SPH2D_OK;
}

static sph2d_status serving_finish(Ctx* c, const SurArgs& sa, int64_t P) {
  cudaError_t e = cudaMemcpyAsync(c->pinned + 10, sa.fb_count, 5 * sizeof(unsigned long long),
                                  cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return cuda_err(c, e, "fallback count copy");
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(c, e, "surrogate launch");
  c->stats.n_pairs = P;
  c->stats.n_fixup = 0;
  c->fixup_pending = false;
  c->fallback_pending = true;
  return SPH2D_OK;
}

sph2d_status surrogate_pairs(Ctx* c, const double* pairs, int64_t P, double H, float* out, int32_t* accepted) {
  SurArgs sa{};
  sph2d_status s = serving_setup(c, P, H, sa);
  if (s != SPH2D_OK) return s;
  sa.C = kernel_C(c->sur_kernel);
  sa.H = H;
  sa.invH = 1.0 / H;
  sa.vals = out;
  sa.accepted = accepted;
  IntArgs a{};
  a.P = P;
  a.H = H;
  a.invH = 1.0 / H;
  a.C = sa.C;
  c->stats = sph2d_stats{};
  if (P > 0) dispatch_serving<false>(c, a, pairs, sa);
  return serving_finish(c, sa, P);
}

// serving over the context's pair list: per-particle gamma and grad gamma (float)
sph2d_status surrogate_integrals(Ctx* c, void* gamma, void* grad) {
  const Cells& cl = c->cells;
  IntArgs a{};
  a.parts = reinterpret_cast<const float4*>(cl.particles);
  a.tris = cl.tris;
  a.pair_tri = static_cast<const int32_t*>(c->pair_tri.ptr);
  a.pair_pid = static_cast<const int32_t*>(c->pair_pid.ptr);
  a.pair_off = static_cast<const int64_t*>(c->pair_off.ptr);
  a.P = cl.P;
  a.N = cl.N;
  a.H = cl.H;
  a.invH = 1.0 / cl.H;
  a.C = kernel_C(c->sur_kernel);
  a.gamma = gamma;
  a.grad = grad;
  a.mom = nullptr;
  a.nm = 0;
  SurArgs sa{};
  sph2d_status s = serving_setup(c, a.P, cl.H, sa);
  if (s == SPH2D_OK) s = ensure(c, c->sur_vals, size_t(a.P > 0 ? a.P : 1) * 3 * sizeof(float));
  if (s == SPH2D_OK) s = ensure(c, c->slots, size_t(((a.P + 31) >> 5) * 2 * 3 + 1) * sizeof(float));
  if (s != SPH2D_OK) return s;
  a.slots = c->slots.ptr;
  a.nfix = sa.fb_count;
  sa.C = a.C;
  sa.H = a.H;
  sa.invH = a.invH;
  sa.vals = static_cast<float*>(c->sur_vals.ptr);
  sa.accepted = nullptr;
  if (a.P > 0) {
    dispatch_serving<true>(c, a, nullptr, sa);
    const unsigned g = persistent_grid(c, reduce_vals_kernel, ((a.P + 31) / 32 + 3) / 4);
    SPH2D_LAUNCH(c, (reduce_vals_kernel), g, 128, a, sa.vals);
  }
  if (a.N > 0) SPH2D_LAUNCH(c, (finalize_kernel<float, 0>), nblk(a.N), 256, a);
  return serving_finish(c, sa, cl.P);
}

// versioned binary checkpoint: header, FP32 masters + Adam moments, FNV-1a checksum
struct SurHeader {
  char magic[8];
  uint32_t version, kernel, in, hidden, out, reserved;
  uint64_t nparams, step, checksum;
};

static uint64_t fnv1a(const void* p, size_t n) {
  const unsigned char* b = static_cast<const unsigned char*>(p);
  uint64_t h = 1469598103934665603ull;
  for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
  return h;
}

sph2d_status surrogate_save(Ctx* c, const char* path) {
  std::vector<float> buf(3 * size_t(kSurParams));
  cudaError_t e = cudaMemcpyAsync(buf.data(), c->sur_prm.ptr, buf.size() * sizeof(float), cudaMemcpyDeviceToHost,
                                  c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_err(c, e, "surrogate save");
  SurHeader h{};
  memcpy(h.magic, "SPH2DSUR", 8);
  h.version = 1;
  h.kernel = uint32_t(c->sur_kernel);
  h.in = kSurIn;
  h.hidden = kSurHid;
  h.out = kSurOut;
  h.nparams = kSurParams;
  h.step = uint64_t(c->sur_step);
  h.checksum = fnv1a(buf.data(), buf.size() * sizeof(float));
  FILE* f = fopen(path, "wb");
  if (!f) return set_err(c, SPH2D_ERR_INVALID_ARG, std::string("cannot open ") + path);
  const bool ok = fwrite(&h, sizeof(h), 1, f) == 1 && fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
  const bool closed = fclose(f) == 0;
  return ok && closed ? SPH2D_OK : set_err(c, SPH2D_ERR_INVALID_ARG, "short write");
}

sph2d_status surrogate_load(Ctx* c, const char* path) {
  FILE* f = fopen(path, "rb");
  if (!f) return set_err(c, SPH2D_ERR_INVALID_ARG, std::string("cannot open ") + path);
  SurHeader h{};
  std::vector<float> buf(3 * size_t(kSurParams));
  bool ok = fread(&h, sizeof(h), 1, f) == 1 && fread(buf.data(), sizeof(float), buf.size(), f) == buf.size();
  ok = ok && fgetc(f) == EOF;
  fclose(f);
  if (!ok || memcmp(h.magic, "SPH2DSUR", 8) != 0 || h.version != 1 || h.nparams != uint64_t(kSurParams) ||
      h.in != uint32_t(kSurIn) || h.hidden != uint32_t(kSurHid) || h.out != uint32_t(kSurOut) || h.kernel > 3)
    return set_err(c, SPH2D_ERR_INVALID_ARG, "not a compatible surrogate checkpoint");
  if (fnv1a(buf.data(), buf.size() * sizeof(float)) != h.checksum)
    return set_err(c, SPH2D_ERR_INVALID_ARG, "checkpoint checksum mismatch");
  sph2d_status s = surrogate_init(c, int(h.kernel), 0);
  if (s != SPH2D_OK) return s;
  cudaError_t e = cudaMemcpyAsync(c->sur_prm.ptr, buf.data(), buf.size() * sizeof(float), cudaMemcpyHostToDevice,
                                  c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_err(c, e, "surrogate load");
  c->sur_step = int64_t(h.step);
  return SPH2D_OK;
}

}  // namespace sph2d
