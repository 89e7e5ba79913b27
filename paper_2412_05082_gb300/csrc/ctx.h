// Context internals shared by api.cu (single problem) and batch.cu (batched
// form): one multigrid hierarchy with its device buffers and tables.
#pragma once
#include <cuda_runtime.h>

#include <array>
#include <vector>

#include "biharm.h"
#include "ops.h"
#include "setup.h"

namespace bh {

// Patch size m^d from which the exact local solver multiplies the patches of a
// run with its dense inverse as one matrix product (gemm.cu): the per-patch
// product streams the whole inverse from L2 for every few patches.  Measured
// on one 3D MVS step: at m^d = 343 (k = 4) the per-patch kernel is still 15 %
// faster; at 729 and above the product is the only usable form.
constexpr int kExactGemmMin = 512;

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
  // exact local solver by dense products: per color, runs of verts sharing a
  // boundary-type combination {first, count, combination slot}
  std::vector<std::array<int, 3>> runs[16];
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
  // exact local solver on large patches (m^d >= kExactGemmMin): the patch
  // tensors of one run as matrix columns, multiplied by the inverse (gemm.cu)
  bool exact_gemm = false;
  int gemm_cols = 0;  // largest run
  double *gR64 = nullptr, *gY64 = nullptr;
  float *gR32 = nullptr, *gY32 = nullptr;
  // FP64 product by FP16 slices (gemm.cu): the slices of every inverse slot
  // ([slot][kSlices][m^d][ld]) with their row exponents ([slot][m^d]), and the
  // slices of one run's gathered patch tensors with their column exponents
  uint16_t* ainv_sl = nullptr;
  int* ainv_ex = nullptr;
  uint16_t* gRs = nullptr;
  int* gRe = nullptr;
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
  // warm-start workspace (allocated on first bh_solve_guess): r0, correction
  double* guess = nullptr;
  int tile = 0;  // patches per block of the fused MVS kernels (0: automatic)
  std::vector<void*> dev_allocs;
  // stats
  long long n_apply = 0, n_smooth = 0, n_vcycle = 0, n_solve = 0;
  int last_iters = 0;
  double last_relres = 0;
  double last_estimate = 0;           // the stopping test's residual ratio at the last stop
  double last_solve_ms = 0;           // CUDA-event device time of the last bh_solve(_host)
  cudaEvent_t ev[2] = {nullptr, nullptr};
  int ncolors() const { return p.dim == 2 ? 8 : 16; }
};
