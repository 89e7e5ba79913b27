// Context internals shared by api.cu (single problem) and batch.cu (batched
// form): one multigrid hierarchy with its device buffers and tables.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "biharm.h"
#include "ops.h"
#include "setup.h"

namespace bh {

struct Level {
  LevelGeom g{};
  double ascale = 0;  // A_l = ascale * A_ref      (h^(d-4))
  double pscale = 0;  // A_v^-1 = pscale * A_ref^-1 (h^(4-d))
  double *x64 = nullptr, *b64 = nullptr, *r64 = nullptr;
  float *x32 = nullptr, *b32 = nullptr, *r32 = nullptr;
  // BH_MIXED_FP32_R64: FP64 right-hand side of the FP32 V-cycle and FP64 copy
  // of its iterate (kept apart from x64 / b64, which bh_solve_host stages in)
  double *db64 = nullptr, *dx64 = nullptr;
  int* verts = nullptr;  // vertex ids sorted by color
  int coff[17] = {0};    // color offsets into verts
};

}  // namespace bh

struct bh_ctx {
  bh_params p{};
  cudaStream_t st = nullptr;
  bh::Setup1D s;
  void* tab64 = nullptr;
  void* tab32 = nullptr;
  std::vector<bh::Level> lv;  // index = level, lv[0] unused
  double* scr64 = nullptr;
  float* scr32 = nullptr;
  double* xs64[2] = {nullptr, nullptr};
  float* xs32[2] = {nullptr, nullptr};
  double* coarse_inv = nullptr;
  int coarse_n = 0;
  double* ainv64 = nullptr;
  float* ainv32 = nullptr;
  // GMRES workspace (allocated on first solve)
  int m = 0;
  double* V = nullptr;
  double* Z = nullptr;
  double* w = nullptr;
  double* t = nullptr;
  double* dots = nullptr;
  double* partials = nullptr;
  double* hdots = nullptr;  // pinned host
  // CG workspace (allocated on first CG solve): r, z, p, q, z_prev
  double* cgv = nullptr;
  int tile = 0;  // patches per block of the fused MVS kernels (0: automatic)
  std::vector<void*> dev_allocs;
  // stats
  long long n_apply = 0, n_smooth = 0, n_vcycle = 0, n_solve = 0;
  int last_iters = 0;
  double last_relres = 0;
  double last_solve_ms = 0;           // CUDA-event device time of the last bh_solve(_host)
  cudaEvent_t ev[2] = {nullptr, nullptr};
  int ncolors() const { return p.dim == 2 ? 8 : 16; }
};
