// Culling grid and pair list (Sec. 2: the triangles N_T overlapping the support of each
// particle).
//
//   1. particle bounds + non-finite scan           (one pass, block reduce, 4 atomics/block)
//   2. triangle binning: each triangle goes into every cell its H-expanded bounding box
//      touches (count -> exclusive scan -> fill), then each cell list is sorted by id
//   3. cull: every particle tests the triangles of its own cell.  A conservative FP32 test
//      decides clear cases; pairs near the threshold (or with far-away geometry) use the
//      exact FP64 predicate whose operation order is fixed in include/sph2d.h, so the pair
//      list is bit-identical to an independent FP64 evaluation.  One pass writes each
//      particle's kept triangles, compacted, into a scratch segment sized by its candidate
//      count (the total is known from particles per cell x list lengths at the binning
//      readback); a scan of the kept counts and a copy give the particle-major CSR list,
//      ascending triangle id within each particle.
#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>
#include <cstring>

#include "sph2d_internal.h"

namespace sph2d {

// ---------------------------------------------------------------------------------------
// 1. bounds
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned int f2ord(float f) {
  const unsigned int u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__host__ __device__ inline float ord2f(unsigned int o) {
  const unsigned int u = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
  float f;
  memcpy(&f, &u, 4);
  return f;
}

// out[0..3] = ord(minx), ord(miny), ord(maxx), ord(maxy); out[4] = non-finite flag
__global__ void bounds_kernel(const float4* __restrict__ parts, int64_t N,
                              const float* __restrict__ tris, int64_t M,
                              unsigned int* __restrict__ out) {
  float mnx = FLT_MAX, mny = FLT_MAX, mxx = -FLT_MAX, mxy = -FLT_MAX;
  unsigned int bad = 0;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += stride) {
    const float4 p = parts[i];
    if (!isfinite(p.x) || !isfinite(p.y)) {
      bad = 1;
      continue;
    }
    mnx = fminf(mnx, p.x);
    mny = fminf(mny, p.y);
    mxx = fmaxf(mxx, p.x);
    mxy = fmaxf(mxy, p.y);
  }
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < 6 * M; i += stride)
    if (!isfinite(tris[i])) bad = 1;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mnx = fminf(mnx, __shfl_xor_sync(0xffffffffu, mnx, o));
    mny = fminf(mny, __shfl_xor_sync(0xffffffffu, mny, o));
    mxx = fmaxf(mxx, __shfl_xor_sync(0xffffffffu, mxx, o));
    mxy = fmaxf(mxy, __shfl_xor_sync(0xffffffffu, mxy, o));
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(out + 0, f2ord(mnx));
    atomicMin(out + 1, f2ord(mny));
    atomicMax(out + 2, f2ord(mxx));
    atomicMax(out + 3, f2ord(mxy));
    if (bad) atomicOr(out + 4, 1u);
  }
}

__global__ void bounds_init(unsigned int* out) {
  out[0] = 0xffffffffu;
  out[1] = 0xffffffffu;
  out[2] = 0u;
  out[3] = 0u;
  out[4] = 0u;
}

// ---------------------------------------------------------------------------------------
// grid geometry (device side mirrors of the host values)
// ---------------------------------------------------------------------------------------
struct Grid {
  double x0, y0, inv_cs, margin, H;
  int nx, ny;
};

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

__device__ __forceinline__ void tri_cell_range(const Grid& g, const float* __restrict__ t, int& ix0,
                                               int& ix1, int& iy0, int& iy1) {
  const double xa = t[0], ya = t[1], xb = t[2], yb = t[3], xc = t[4], yc = t[5];
  const double lox = fmin(xa, fmin(xb, xc)) - g.H - g.margin;
  const double hix = fmax(xa, fmax(xb, xc)) + g.H + g.margin;
  const double loy = fmin(ya, fmin(yb, yc)) - g.H - g.margin;
  const double hiy = fmax(ya, fmax(yb, yc)) + g.H + g.margin;
  const double fx0 = floor((lox - g.x0) * g.inv_cs), fx1 = floor((hix - g.x0) * g.inv_cs);
  const double fy0 = floor((loy - g.y0) * g.inv_cs), fy1 = floor((hiy - g.y0) * g.inv_cs);
  if (fx1 < 0.0 || fy1 < 0.0 || fx0 > double(g.nx - 1) || fy0 > double(g.ny - 1)) {
    ix0 = 1;
    ix1 = 0;
    iy0 = 1;
    iy1 = 0;
    return;
  }
  ix0 = int(fmax(fx0, 0.0));
  ix1 = int(fmin(fx1, double(g.nx - 1)));
  iy0 = int(fmax(fy0, 0.0));
  iy1 = int(fmin(fy1, double(g.ny - 1)));
}

__device__ __forceinline__ int64_t particle_cell(const Grid& g, float px, float py) {
  const int ix = clampi(int(floor((double(px) - g.x0) * g.inv_cs)), 0, g.nx - 1);
  const int iy = clampi(int(floor((double(py) - g.y0) * g.inv_cs)), 0, g.ny - 1);
  return int64_t(iy) * g.nx + ix;
}

// ---------------------------------------------------------------------------------------
// 2. triangle binning
// ---------------------------------------------------------------------------------------
__global__ void tri_count_kernel(Grid g, const float* __restrict__ tris, int64_t M,
                                 unsigned long long* __restrict__ cell_count) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= M) return;
  int ix0, ix1, iy0, iy1;
  tri_cell_range(g, tris + 6 * t, ix0, ix1, iy0, iy1);
  for (int iy = iy0; iy <= iy1; ++iy)
    for (int ix = ix0; ix <= ix1; ++ix) atomicAdd(cell_count + int64_t(iy) * g.nx + ix, 1ull);
}

__global__ void tri_fill_kernel(Grid g, const float* __restrict__ tris, int64_t M,
                                const int64_t* __restrict__ cell_start,
                                unsigned long long* __restrict__ cursor, int32_t* __restrict__ cell_tris) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= M) return;
  int ix0, ix1, iy0, iy1;
  tri_cell_range(g, tris + 6 * t, ix0, ix1, iy0, iy1);
  for (int iy = iy0; iy <= iy1; ++iy)
    for (int ix = ix0; ix <= ix1; ++ix) {
      const int64_t c = int64_t(iy) * g.nx + ix;
      const unsigned long long k = atomicAdd(cursor + c, 1ull);
      cell_tris[cell_start[c] + int64_t(k)] = int32_t(t);
    }
}

// sort each list of up to 512 ids ascending: one warp per list, a bitonic network over E ids per
// lane (index lane + 32 r, r < E, E the smallest power of two with 32 E >= n), padded with
// INT32_MAX.  Compare-exchanges across lanes (distance < 32) go through shuffles, the others
// between a lane's own registers.  Longer lists are left to sort_cells_kernel.
constexpr int kWarpSortMax = 512;
template <int E>
__device__ __forceinline__ void warp_bitonic(int32_t* __restrict__ d, int64_t n, int lane) {
  int32_t a[E];
#pragma unroll
  for (int r = 0; r < E; ++r) a[r] = lane + 32 * r < n ? d[lane + 32 * r] : 0x7fffffff;
#pragma unroll
  for (int k = 2; k <= 32 * E; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j >= 32) {
        const int rj = j >> 5;
#pragma unroll
        for (int r = 0; r < E; ++r) {
          if ((r & rj) != 0) continue;
          const bool up = ((lane + 32 * r) & k) == 0;
          const int32_t lo = min(a[r], a[r | rj]), hi = max(a[r], a[r | rj]);
          a[r] = up ? lo : hi;
          a[r | rj] = up ? hi : lo;
        }
      } else {
        const bool lower = (lane & j) == 0;
#pragma unroll
        for (int r = 0; r < E; ++r) {
          const int32_t p = __shfl_xor_sync(0xffffffffu, a[r], j);
          const bool up = ((lane + 32 * r) & k) == 0;
          a[r] = (lower == up) ? min(a[r], p) : max(a[r], p);
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < E; ++r)
    if (lane + 32 * r < n) d[lane + 32 * r] = a[r];
}
// (long: set to 1 when some list is longer than kWarpSortMax, for sort_cells_kernel)
__global__ void sort_small_kernel(const int64_t* __restrict__ start, int32_t* __restrict__ data, int64_t nseg,
                                  unsigned int* __restrict__ long_flag) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t c = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; c < nseg; c += nw) {
    const int64_t s = start[c], n = start[c + 1] - s;   // warp-uniform
    if (n > kWarpSortMax && lane == 0) *long_flag = 1u;
    if (n <= 1 || n > kWarpSortMax) continue;
    if (n <= 64) warp_bitonic<2>(data + s, n, lane);
    else if (n <= 128) warp_bitonic<4>(data + s, n, lane);
    else if (n <= 256) warp_bitonic<8>(data + s, n, lane);
    else warp_bitonic<16>(data + s, n, lane);
  }
}

// sort each cell list of more than kWarpSortMax ids ascending: bitonic in shared memory (<= 4096
// ids), else insertion sort
constexpr int kSortCap = 4096;
__global__ void sort_cells_kernel(const int64_t* __restrict__ cell_start, int32_t* __restrict__ cell_tris,
                                  int64_t n_cells, const unsigned int* __restrict__ long_flag) {
  __shared__ int32_t buf[kSortCap];
  if (*long_flag == 0u) return;                 // no list longer than kWarpSortMax (block-uniform)
  for (int64_t c = blockIdx.x; c < n_cells; c += gridDim.x) {
    const int64_t s = cell_start[c], n = cell_start[c + 1] - s;
    if (n <= kWarpSortMax) continue;
    if (n <= kSortCap) {
      int p2 = 1;
      while (p2 < n) p2 <<= 1;
      for (int i = threadIdx.x; i < p2; i += blockDim.x) buf[i] = i < n ? cell_tris[s + i] : 0x7fffffff;
      __syncthreads();
      for (int k = 2; k <= p2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
          for (int i = threadIdx.x; i < p2; i += blockDim.x) {
            const int l = i ^ j;
            if (l > i) {
              const int32_t a = buf[i], b = buf[l];
              const bool up = (i & k) == 0;
              if ((a > b) == up) {
                buf[i] = b;
                buf[l] = a;
              }
            }
          }
          __syncthreads();
        }
      }
      for (int i = threadIdx.x; i < n; i += blockDim.x) cell_tris[s + i] = buf[i];
      __syncthreads();
    } else if (threadIdx.x == 0) {
      int32_t* a = cell_tris + s;
      for (int64_t i = 1; i < n; ++i) {
        const int32_t v = a[i];
        int64_t j = i - 1;
        while (j >= 0 && a[j] > v) {
          a[j + 1] = a[j];
          --j;
        }
        a[j + 1] = v;
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------
// 3. the pair predicate
// ---------------------------------------------------------------------------------------
// exact FP64 predicate in the operation order of include/sph2d.h (no FMA contraction)
__device__ __noinline__ bool keep_exact(double px, double py, const float* __restrict__ t, double H2) {
  double x[3], y[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    x[j] = double(t[2 * j]);
    y[j] = double(t[2 * j + 1]);
  }
  double best = __longlong_as_double(0x7ff0000000000000LL);   // +inf
  int npos = 0, nneg = 0;
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const int b = e == 2 ? 0 : e + 1;
    const double ex = __dsub_rn(x[b], x[e]), ey = __dsub_rn(y[b], y[e]);
    const double wx = __dsub_rn(px, x[e]), wy = __dsub_rn(py, y[e]);
    const double cr = __dsub_rn(__dmul_rn(wx, ey), __dmul_rn(wy, ex));
    if (cr > 0.0) ++npos;
    if (cr < 0.0) ++nneg;
    const double l2 = __dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey));
    const double tn = __dadd_rn(__dmul_rn(wx, ex), __dmul_rn(wy, ey));
    double d2;
    if (tn <= 0.0) {
      d2 = __dadd_rn(__dmul_rn(wx, wx), __dmul_rn(wy, wy));
    } else if (tn >= l2) {
      const double vx = __dsub_rn(px, x[b]), vy = __dsub_rn(py, y[b]);
      d2 = __dadd_rn(__dmul_rn(vx, vx), __dmul_rn(vy, vy));
    } else {
      d2 = __ddiv_rn(__dmul_rn(cr, cr), l2);
    }
    if (d2 < best) best = d2;
  }
  if ((npos + nneg > 0) && (npos == 0 || nneg == 0)) return true;   // inside (not collinear)
  return best < H2;
}

// FP32 screen: returns 1 keep, 0 reject, -1 undecided (caller runs keep_exact); v the vertices
__device__ __forceinline__ int keep_screen(float px, float py, const float* v, float Hf,
                                           float H2lo, float H2hi) {
  float x[3], y[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    x[j] = v[2 * j];
    y[j] = v[2 * j + 1];
  }
  float best = FLT_MAX, wmax = 0.0f;
  bool pos_sure = false, neg_sure = false, all_pos = true, all_neg = true;
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const int b = e == 2 ? 0 : e + 1;
    const float ex = x[b] - x[e], ey = y[b] - y[e];
    const float wx = px - x[e], wy = py - y[e];
    wmax = fmaxf(wmax, fmaxf(fabsf(wx), fabsf(wy)));
    const float cr = wx * ey - wy * ex;
    const float tol = 7.62939453125e-06f * (fabsf(wx) + fabsf(wy)) * (fabsf(ex) + fabsf(ey));  // 2^-17
    if (cr > tol) pos_sure = true;
    if (cr < -tol) neg_sure = true;
    if (!(cr > tol)) all_pos = false;
    if (!(cr < -tol)) all_neg = false;
    const float l2 = ex * ex + ey * ey;
    const float tn = wx * ex + wy * ey;
    float d2;
    if (tn <= 0.0f) {
      d2 = wx * wx + wy * wy;
    } else if (tn >= l2) {
      const float vx = px - x[b], vy = py - y[b];
      d2 = vx * vx + vy * vy;
    } else {
      d2 = cr * cr / l2;
    }
    best = fminf(best, d2);
  }
  if (!(wmax <= 64.0f * Hf)) {
    // far geometry: a clear miss if every vertex is far and the bound is generous
    if (best > 4.0f * H2hi && pos_sure && neg_sure) return 0;
    return -1;
  }
  if (all_pos || all_neg) return 1;           // clearly inside
  if (best < H2lo) return 1;                  // clearly within H
  if (best > H2hi && pos_sure && neg_sure) return 0;
  return -1;
}

struct CullArgs {
  Grid g;
  double H2;
  float Hf, H2lo, H2hi;
};

// particles per cell (for the candidate total of the single-pass cull)
__global__ void part_cell_count_kernel(Grid g, const float4* __restrict__ parts, int64_t N,
                                       unsigned long long* __restrict__ npart) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const float4 p = parts[i];
  atomicAdd(npart + particle_cell(g, p.x, p.y), 1ull);
}

// sum over cells of (particles in the cell) x (triangles in its list): the scratch size of the
// cull's candidate lists
__global__ void cand_total_kernel(const unsigned long long* __restrict__ npart,
                                  const int64_t* __restrict__ cell_start, int64_t C,
                                  unsigned long long* __restrict__ total) {
  unsigned long long acc = 0;
  for (int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; c < C; c += int64_t(gridDim.x) * blockDim.x)
    acc += npart[c] * (unsigned long long)(cell_start[c + 1] - cell_start[c]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc) atomicAdd(total, acc);
}

// candidates of each particle: the length of its cell's triangle list
__global__ void cand_count_kernel(Grid g, const float4* __restrict__ parts, int64_t N,
                                  const int64_t* __restrict__ cell_start, int64_t* __restrict__ cand) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const float4 p = parts[i];
  const int64_t c = particle_cell(g, p.x, p.y);
  cand[i] = cell_start[c + 1] - cell_start[c];
}

// the pair predicate over each particle's candidates, once: the kept triangles (ascending id,
// the cell list's order) go compacted to the particle's scratch segment, their number to counts
__global__ void cull_kernel(CullArgs a, const float4* __restrict__ parts, int64_t N,
                            const float* __restrict__ tris, const int64_t* __restrict__ cell_start,
                            const int32_t* __restrict__ cell_tris, const int64_t* __restrict__ cand_off,
                            int32_t* __restrict__ kept, int64_t* __restrict__ counts) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const float4 p = parts[i];
  const int64_t c = particle_cell(a.g, p.x, p.y);
  const int64_t s = cell_start[c], e = cell_start[c + 1];
  int32_t* out = kept + cand_off[i];
  int64_t n = 0;
  // software pipeline: the next candidate's id and vertices load while this one is screened
  int32_t t = s < e ? __ldg(cell_tris + s) : 0;
  int32_t t1 = s + 1 < e ? __ldg(cell_tris + s + 1) : 0;
  float v[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) v[j] = s < e ? __ldg(tris + 6 * int64_t(t) + j) : 0.0f;
  for (int64_t k = s; k < e; ++k) {
    const int32_t t2 = k + 2 < e ? __ldg(cell_tris + k + 2) : 0;
    float vn[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) vn[j] = k + 1 < e ? __ldg(tris + 6 * int64_t(t1) + j) : 0.0f;
    int r = keep_screen(p.x, p.y, v, a.Hf, a.H2lo, a.H2hi);
    if (r < 0) r = keep_exact(double(p.x), double(p.y), tris + 6 * int64_t(t), a.H2) ? 1 : 0;
    if (r) out[n++] = t;
    t = t1;
    t1 = t2;
#pragma unroll
    for (int j = 0; j < 6; ++j) v[j] = vn[j];
  }
  counts[i] = n;
}

// the compacted lists into the particle-major pair list: one warp per 32 consecutive particles,
// its lanes striding over the warp's whole output range [pair_off[i0], pair_off[i0 + 32]) so
// that every store is coalesced; a lane finds the particle of its output position by a binary
// search over the 33 offsets, which the lanes hold in registers
__global__ void pair_copy_kernel(int64_t N, const int64_t* __restrict__ cand_off, const int32_t* __restrict__ kept,
                                 const int64_t* __restrict__ pair_off, int32_t* __restrict__ pair_tri,
                                 int32_t* __restrict__ pair_pid) {
  const int64_t i0 = ((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5) << 5;
  const int lane = threadIdx.x & 31;
  if (i0 >= N) return;                                    // warp-uniform
  const int64_t il = i0 + lane < N ? i0 + lane : N;
  const int64_t off = pair_off[il];                       // lane j: start of particle i0 + j
  const int64_t coff = i0 + lane < N ? cand_off[i0 + lane] : 0;
  const int64_t beg = __shfl_sync(0xffffffffu, off, 0);
  const int64_t end = pair_off[i0 + 32 < N ? i0 + 32 : N];
  // four output positions per lane per step, so that four searches and four gathers are in
  // flight together; uniform trip count: every lane shuffles
  constexpr int U = 4;
  for (int64_t base = beg; base < end; base += 32 * U) {
    int64_t pos[U];
    int j[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      pos[u] = base + 32 * u + lane;
      j[u] = 0;
    }
    // largest j with off_j <= pos (particles with no pairs share their offset with the next)
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t o = __shfl_sync(0xffffffffu, off, j[u] + step);
        if (o <= pos[u] && i0 + j[u] + step < N) j[u] += step;
      }
    }
    int32_t t[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t oj = __shfl_sync(0xffffffffu, off, j[u]), cj = __shfl_sync(0xffffffffu, coff, j[u]);
      t[u] = pos[u] < end ? kept[cj + (pos[u] - oj)] : 0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (pos[u] < end) {
        pair_tri[pos[u]] = t[u];
        pair_pid[pos[u]] = int32_t(i0 + j[u]);
      }
    }
  }
}

// sort the int32 segments data[start[i] .. start[i+1]) ascending (used for cell lists and,
// by the adjoint, for per-triangle particle lists)
sph2d_status launch_sort_segments(Ctx* c, const int64_t* start, int32_t* data, int64_t nseg) {
  if (nseg <= 0) return SPH2D_OK;
  sph2d_status s = ensure(c, c->sort_flag, 256);
  if (s != SPH2D_OK) return s;
  auto* flag = static_cast<unsigned int*>(c->sort_flag.ptr);
  const cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(unsigned int), c->stream);
  if (e != cudaSuccess) return cuda_err(c, e, "memset");
  const int64_t wblocks = (nseg + 7) / 8;                 // 8 warps of 256 threads per block
  SPH2D_LAUNCH(c, (sort_small_kernel), unsigned(wblocks < 65535 ? wblocks : 65535), 256, start, data, nseg, flag);
  const int blocks = nseg < 1216 ? int(nseg) : 1216;     // the few long lists
  SPH2D_LAUNCH(c, (sort_cells_kernel), blocks, 256, start, data, nseg, flag);
  return SPH2D_OK;
}

// ---------------------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------------------
sph2d_status build_cells(Ctx* c, const float* particles, int64_t N, const float* tris, int64_t M,
                         double H) {
  Cells& cl = c->cells;
  cl.built = false;
  cl.part_grid = false;
  cl.particles = particles;
  cl.tris = tris;
  cl.N = N;
  cl.M = M;
  cl.H = H;
  cl.P = 0;
  c->stats = sph2d_stats{};
  c->stats.n_particles = N;
  c->stats.n_triangles = M;
  cudaError_t e;
  sph2d_status s;
  cudaStream_t st = c->stream;

  // pair offsets always exist (N+1 zeros when nothing pairs up)
  s = ensure(c, c->pair_off, size_t(N + 1) * sizeof(int64_t));
  if (s != SPH2D_OK) return s;

  // ---- 1. bounds and finiteness
  s = ensure(c, c->misc, 64);
  if (s != SPH2D_OK) return s;
  unsigned int* bnd = static_cast<unsigned int*>(c->misc.ptr);
  SPH2D_LAUNCH(c, (bounds_init), 1, 1, bnd);
  {
    int64_t work = N > 6 * M ? N : 6 * M;
    int blocks = int((work + kBlock - 1) / kBlock);
    if (blocks > 1024) blocks = 1024;
    if (blocks < 1) blocks = 1;
    SPH2D_LAUNCH(c, (bounds_kernel), blocks, kBlock, reinterpret_cast<const float4*>(particles), N, tris, M, bnd);
  }
  e = cudaMemcpyAsync(c->pinned, bnd, 5 * sizeof(unsigned int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_err(c, e, "bounds");
  unsigned int hb[5];
  memcpy(hb, c->pinned, sizeof(hb));
  if (hb[4]) return set_err(c, SPH2D_ERR_NONFINITE_INPUT, "non-finite particle or vertex coordinate");
  if (N == 0) {
    // no particles: an empty grid (the particle grid of the MLS pressure is empty too)
    cl.nx = cl.ny = 0;
    cl.n_cells = 0;
    e = cudaMemsetAsync(c->pair_off.ptr, 0, size_t(N + 1) * sizeof(int64_t), st);
    if (e != cudaSuccess) return cuda_err(c, e, "memset");
    cl.built = true;
    return SPH2D_OK;
  }
  const double mnx = ord2f(hb[0]), mny = ord2f(hb[1]), mxx = ord2f(hb[2]), mxy = ord2f(hb[3]);

  // ---- grid: square cells of side >= H over the particle box, at most ~4N+4096 cells
  double cs = H;
  const double ext_x = mxx - mnx, ext_y = mxy - mny;
  const double max_cells = 4.0 * double(N) + 4096.0;
  for (;;) {
    const double nxd = floor(ext_x / cs) + 1.0, nyd = floor(ext_y / cs) + 1.0;
    if (nxd * nyd <= max_cells && nxd < 1048576.0 && nyd < 1048576.0) break;
    cs *= 1.5;
  }
  Grid g;
  g.x0 = mnx - 1e-3 * cs;
  g.y0 = mny - 1e-3 * cs;
  g.nx = int(floor((mxx - g.x0) / cs)) + 1;
  g.ny = int(floor((mxy - g.y0) / cs)) + 1;
  g.inv_cs = 1.0 / cs;
  g.H = H;
  g.margin = 1e-9 * (fabs(mnx) + fabs(mny) + fabs(mxx) + fabs(mxy) + H + cs);
  cl.x0 = g.x0;
  cl.y0 = g.y0;
  cl.cs = cs;
  cl.nx = g.nx;
  cl.ny = g.ny;
  const int64_t C = int64_t(g.nx) * g.ny;
  cl.n_cells = C;

  if (M == 0) {
    // no triangles: no pairs; the grid above still serves the particle grid of the MLS pressure
    e = cudaMemsetAsync(c->pair_off.ptr, 0, size_t(N + 1) * sizeof(int64_t), st);
    if (e != cudaSuccess) return cuda_err(c, e, "memset");
    cl.built = true;
    return SPH2D_OK;
  }

  // ---- 2. bin triangles
  s = ensure(c, c->cell_cursor, size_t(C) * sizeof(unsigned long long));
  if (s == SPH2D_OK) s = ensure(c, c->cell_start, size_t(C + 1) * sizeof(int64_t));
  if (s != SPH2D_OK) return s;
  auto* ccount = static_cast<unsigned long long*>(c->cell_cursor.ptr);
  auto* cstart = static_cast<int64_t*>(c->cell_start.ptr);
  // particles per cell and the candidate total, read back with the incidence count
  s = ensure(c, c->part_cursor, size_t(C) * sizeof(unsigned long long) + 64);
  if (s != SPH2D_OK) return s;
  auto* npart = static_cast<unsigned long long*>(c->part_cursor.ptr);
  auto* cand_total = npart + C;
  e = cudaMemsetAsync(ccount, 0, size_t(C) * sizeof(unsigned long long), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(npart, 0, size_t(C) * sizeof(unsigned long long) + 64, st);
  if (e != cudaSuccess) return cuda_err(c, e, "memset");
  const unsigned tblocks = unsigned((M + kBlock - 1) / kBlock);
  const unsigned pblocks = unsigned((N + kBlock - 1) / kBlock);
  const float4* parts4 = reinterpret_cast<const float4*>(particles);
  SPH2D_LAUNCH(c, (tri_count_kernel), tblocks, kBlock, g, tris, M, ccount);
  SPH2D_LAUNCH(c, (part_cell_count_kernel), pblocks, kBlock, g, parts4, N, npart);
  s = exclusive_scan_i64(c, reinterpret_cast<const int64_t*>(ccount), cstart, C);
  if (s != SPH2D_OK) return s;
  {
    const int64_t want = (C + kBlock - 1) / kBlock;
    SPH2D_LAUNCH(c, (cand_total_kernel), unsigned(want < 1024 ? (want > 0 ? want : 1) : 1024), kBlock, npart, cstart,
                 C, cand_total);
  }
  e = cudaMemcpyAsync(c->pinned, cstart + C, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->pinned + 1, cand_total, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_err(c, e, "triangle binning");
  const int64_t n_incid = c->pinned[0], n_cand = c->pinned[1];
  cl.n_incid = n_incid;
  c->stats.n_cells = C;
  c->stats.n_candidates = n_incid;
  s = ensure(c, c->cell_tris, size_t(n_incid > 0 ? n_incid : 1) * sizeof(int32_t));
  if (s != SPH2D_OK) return s;
  e = cudaMemsetAsync(ccount, 0, size_t(C) * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return cuda_err(c, e, "memset");
  auto* ctris = static_cast<int32_t*>(c->cell_tris.ptr);
  SPH2D_LAUNCH(c, (tri_fill_kernel), tblocks, kBlock, g, tris, M, cstart, ccount, ctris);
  s = launch_sort_segments(c, cstart, ctris, C);
  if (s != SPH2D_OK) return s;

  // ---- 3. cull: each particle's candidates once into a scratch segment, then scan and copy
  CullArgs a;
  a.g = g;
  a.H2 = H * H;
  a.Hf = float(H);
  const float H2f = float(H) * float(H);
  a.H2lo = H2f * (1.0f - 1.0f / 1024.0f);
  a.H2hi = H2f * (1.0f + 1.0f / 1024.0f);
  s = ensure(c, c->counts, size_t(N) * sizeof(int64_t));
  if (s == SPH2D_OK) s = ensure(c, c->cand_off, size_t(N + 1) * sizeof(int64_t));
  if (s == SPH2D_OK) s = ensure(c, c->cand_kept, size_t(n_cand > 0 ? n_cand : 1) * sizeof(int32_t));
  if (s != SPH2D_OK) return s;
  auto* cnt = static_cast<int64_t*>(c->counts.ptr);
  auto* coff = static_cast<int64_t*>(c->cand_off.ptr);
  auto* kept = static_cast<int32_t*>(c->cand_kept.ptr);
  auto* poff = static_cast<int64_t*>(c->pair_off.ptr);
  SPH2D_LAUNCH(c, (cand_count_kernel), pblocks, kBlock, g, parts4, N, cstart, cnt);
  s = exclusive_scan_i64(c, cnt, coff, N);
  if (s != SPH2D_OK) return s;
  SPH2D_LAUNCH(c, (cull_kernel), pblocks, kBlock, a, parts4, N, tris, cstart, ctris, coff, kept, cnt);
  s = exclusive_scan_i64(c, cnt, poff, N);
  if (s != SPH2D_OK) return s;
  e = cudaMemcpyAsync(c->pinned, poff + N, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_err(c, e, "cull count");
  const int64_t P = c->pinned[0];
  if (P > (int64_t(1) << 31) - 64)
    return set_err(c, SPH2D_ERR_UNSUPPORTED, "more than 2^31 pairs in one call");
  s = ensure(c, c->pair_tri, size_t(P > 0 ? P : 1) * sizeof(int32_t));
  if (s == SPH2D_OK) s = ensure(c, c->pair_pid, size_t(P > 0 ? P : 1) * sizeof(int32_t));
  if (s != SPH2D_OK) return s;
  {
    const int64_t threads = ((N + 31) / 32) * 32;             // one warp per 32 particles
    SPH2D_LAUNCH(c, (pair_copy_kernel), unsigned((threads + kBlock - 1) / kBlock), kBlock, N, coff, kept, poff,
                 static_cast<int32_t*>(c->pair_tri.ptr), static_cast<int32_t*>(c->pair_pid.ptr));
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(c, e, "cull launch");
  cl.P = P;
  c->stats.n_pairs = P;
  cl.built = true;
  return SPH2D_OK;
}

}  // namespace sph2d
