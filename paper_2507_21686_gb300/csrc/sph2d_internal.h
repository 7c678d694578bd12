// Internal declarations shared by the translation units of libsph2d.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/sph2d.h"

namespace sph2d {

// grows on demand; never shrinks until the context is destroyed
struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
};

// culling grid + pair list of the last build
struct Cells {
  bool built = false;
  bool part_grid = false;     // particle grid of this build made (boundary pressure / MLS)
  const float* particles = nullptr;
  const float* tris = nullptr;
  int64_t N = 0, M = 0;
  double H = 0.0;
  // grid
  double x0 = 0.0, y0 = 0.0, cs = 1.0;
  int nx = 0, ny = 0;
  int64_t n_cells = 0, n_incid = 0;
  // pair list
  int64_t P = 0;
};

struct Ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  sph2d_stats stats{};
  Cells cells;
  // scratch buffers (named slots)
  DevBuf cell_start, cell_cursor, cell_tris, block_tmp, scan_tmp, pair_off, pair_tri, pair_pid,
      counts, slots, host_flags_dev, misc, tri_off, tri_pid, tri_cursor, bwd_g, bwd_grad,
      pair_vals, pair_list2;   // per-pair values or per-(particle, region) sums; partition scratch
  // learned surrogate: parameters (+ Adam state), training data and scratch, serving scratch
  DevBuf sur_prm, sur_split, sur_act, sur_data, sur_idx, sur_vals, sur_fb;
  // boundary pressure coupling: particle grid (cell starts, cursors, ids) and scratch
  DevBuf part_start, part_cursor, part_ids, pres_vertex, pres_tmp;
  // single-pass cull: per-particle candidate offsets and the compacted kept triangles
  DevBuf cand_off, cand_kept;
  DevBuf sort_flag;            // set when a sorted segment is too long for the warp sort
  int64_t* pinned = nullptr;   // small pinned host staging area (64 int64)
  bool fixup_pending = false;  // pinned[8] holds the fix-up count of the last integral call
  bool fallback_pending = false;  // pinned[10..14]: fallback count, audit and MMA timeouts of the last surrogate call
  int64_t launches = 0;        // kernels launched by this context (cumulative)
  bool sur_ready = false;      // surrogate parameters initialised
  int sur_kernel = -1;         // kernel the surrogate is trained for
  int64_t sur_step = 0;        // optimiser steps taken
  float sur_w[3] = {1.0f, 1.0f, 1.0f};   // per-output loss weights
  int sur_audit_period = 64;   // serving audit: one accepted pair in this many (0: off)
  double sur_audit_tol = 1e-3; // audit bound in units of the output scales
  int sur_engine = 0;          // serving MMAs: 0 mma.sync (register-chained), 1 tcgen05 (TMEM)
  int sur_train_engine = 0;    // training GEMMs: 0 mma.sync, 1 tcgen05 (TMEM accumulators)
};

// error helpers ------------------------------------------------------------------------
sph2d_status set_err(Ctx* c, sph2d_status s, const std::string& msg);
sph2d_status cuda_err(Ctx* c, cudaError_t e, const char* where);
sph2d_status ensure(Ctx* c, DevBuf& b, size_t bytes);

// device-wide exclusive scan of int64 [n] -> out [n+1] (out[n] = total), on c->stream
sph2d_status exclusive_scan_i64(Ctx* c, const int64_t* in, int64_t* out, int64_t n);

// culling (cells.cu): builds c->cells and the pair list buffers pair_off/pair_tri/pair_pid
sph2d_status build_cells(Ctx* c, const float* particles, int64_t N, const float* tris,
                         int64_t M, double H);

// ascending sort of int32 segments (cells.cu)
sph2d_status launch_sort_segments(Ctx* c, const int64_t* start, int32_t* data, int64_t nseg);

// forward integrals over the context's pair list (integrals.cu)
sph2d_status launch_integrals(Ctx* c, int kernel, int moment_degree, int mode, void* gamma,
                              void* grad, void* moments);

// independent pairs (integrals.cu)
sph2d_status launch_pair_integrals(Ctx* c, const double* pairs, int64_t P, int kernel, double H,
                                   int moment_degree, int mode, void* out);

// piecewise-linear boundary fields over the context's pair list (fields.cu)
sph2d_status launch_fields(Ctx* c, int kernel, int mode, const float* values, int nf, void* value,
                           void* grad);
sph2d_status launch_fields_p(Ctx* c, int kernel, int mode, int order, const float* values, int nf, void* value,
                             void* grad);

// boundary pressure coupling (pressure.cu)
sph2d_status launch_mls_points(Ctx* c, int kernel, int mode, const float* vol, const float* pres, const float* pts,
                               int64_t Q, void* out);
sph2d_status launch_boundary_pressure(Ctx* c, int kernel, int mode, int model, const float* rho, const float* pres,
                                      const float* vol, double rho0b, void* accel);

// adjoint (backward.cu)
sph2d_status launch_backward(Ctx* c, int kernel, int mode, const void* d_gamma,
                             const void* d_grad, void* d_particles, void* d_tris);

// learned surrogate (surrogate.cu); callers validate arguments and sur_ready
sph2d_status surrogate_init(Ctx* c, int kernel, uint64_t seed);
sph2d_status surrogate_train(Ctx* c, const double* pairs, int64_t P, double H, int epochs, int batch,
                             double lr, double wd, uint64_t seed, double* final_loss, int64_t* used);
sph2d_status surrogate_pairs(Ctx* c, const double* pairs, int64_t P, double H, float* out, int32_t* accepted);
sph2d_status surrogate_integrals(Ctx* c, void* gamma, void* grad);
sph2d_status surrogate_forward(Ctx* c, const float* X, int64_t B, float* Y);
sph2d_status surrogate_grad(Ctx* c, const float* X, const float* T, int64_t B, float* grad, float* loss);
sph2d_status surrogate_set_params(Ctx* c, const float* host);
sph2d_status surrogate_get_params(Ctx* c, float* host);
sph2d_status surrogate_save(Ctx* c, const char* path);
sph2d_status surrogate_load(Ctx* c, const char* path);

inline int num_moments(int deg) { return deg < 0 ? 0 : (deg + 1) * (deg + 2) / 2; }

constexpr int kBlock = 256;

// every kernel launch of the library goes through this, so the context can report a count
#define SPH2D_LAUNCH(ctx, kern, grid, block, ...)                          \
  do {                                                                     \
    (kern)<<<(grid), (block), 0, (ctx)->stream>>>(__VA_ARGS__);          \
    ++(ctx)->launches;                                                     \
  } while (0)

}  // namespace sph2d
