// Host-visible interface of the CUDA kernels (no device code here).
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "setup.h"

namespace bh {

// Kernels launched by this process (all contexts).
extern std::atomic<long long> g_kernel_launches;

struct LevelGeom {
  int d;       // dimension
  int k;       // degree
  int N;       // cells per direction
  int n;       // interior nodes per direction, k N - 1
  int64_t nd;  // n^d
};

// Number of scratch arrays (each nd values) that apply() needs.
inline int apply_scratch_arrays(int d) { return d == 2 ? 3 : 6; }

enum ApplyMode { kStore = 0, kResidual = 1 };

// device copies of a context's tables: `tables` points to Tables<T, K> in
// device memory, `dinv` to the reciprocal eigenvalue sums
struct DevTables {
  const void* tables;
  const void* dinv;
};

template <typename T>
struct Ops {
  // Kernel-parameter tables (1D class tables, FDM eigendata, prolongation)
  // converted to T; opaque, freed with free_tables.
  static void* make_tables(const Setup1D& s, int d);
  static void free_tables(void* tab, int k);
  static DevTables device_tables(const void* tab, int k);
  // host copy of the interior tiles' tables of the fused MVS kernel
  // (CanonTab<T, k>) and its size
  static const void* host_mvs_tables(const void* tab, int k, size_t* bytes);

  // mode kStore: y = scale * A_ref x; mode kResidual: y = b - scale * A_ref x.
  static cudaError_t apply(const void* tab, const LevelGeom& g, const T* x, const T* b, T* y,
                           double scale, int mode, T* scratch, cudaStream_t st);

  // x += scale * sum_{v in verts} R_v^T A~_v,ref^-1 R_v r  (fast diagonalization).
  static cudaError_t patch_fdm(const void* tab, const LevelGeom& g, const T* r, T* x,
                               const int* verts, int count, double scale, bool atomic,
                               cudaStream_t st);

  // One color of the colored MVS, fused (2D and 3D, fast diagonalization): for every
  // patch v in verts, x_v += pscale * A~_v,ref^-1 R_v (b - ascale * A_ref x).
  // pb: patches per block (0: automatic)
  static cudaError_t mvs_color(const void* tab, const LevelGeom& g, T* x, const T* b,
                               const int* verts, int count, double ascale, double pscale,
                               int pb, cudaStream_t st);

  // x += scale * sum_{v in verts} R_v^T Ainv[combo(v)] R_v r  (dense exact inverse;
  // Ainv holds 4^d slots of m^d x m^d matrices, slot = sum_a type_a 4^a).
  static cudaError_t patch_exact(const LevelGeom& g, const T* Ainv, const T* r, T* x,
                                 const int* verts, int count, double scale, bool atomic,
                                 cudaStream_t st);

  // R[:, j] = R_v r for the patches v = verts[j] (m^d rows, column-major), and
  // x += R_v^T Y[:, j] (atomic for overlapping patches): the gather and scatter
  // around a dense-matrix product of the exact local solver.
  static cudaError_t patch_gather(const LevelGeom& g, const T* r, const int* verts, int count,
                                  T* R, cudaStream_t st);
  static cudaError_t patch_scatter(const LevelGeom& g, const T* Y, const int* verts, int count,
                                   T* x, bool atomic, cudaStream_t st);

  // xf += P xc (embedding), fine geometry given; s0, s1 scratch of fine nd each.
  static cudaError_t prolongate_add(const void* tab, const LevelGeom& fine, const T* xc, T* xf,
                                    T* s0, T* s1, cudaStream_t st);

  // bc = P^T rf (and, when bc32 is given, bc rounded to FP32 into bc32).
  static cudaError_t restrict_(const void* tab, const LevelGeom& fine, const T* rf, T* bc, T* s0,
                               T* s1, cudaStream_t st, float* bc32 = nullptr);

  // y += x
  static cudaError_t add(T* y, const T* x, int64_t n, cudaStream_t st);

  // out = scale * A (n x n dense symmetric, FP64) * in.
  static cudaError_t dense_symv(int n, const double* A, const T* in, T* out, double scale,
                                cudaStream_t st);
};

// ---- dense products of the exact local solver (gemm.cu) ----------------------
// FP64 by FP16 slices: kSlices slices of kSliceBits bits per value.
constexpr int kSlices = 9, kSliceBits = 6;  // 54 bits: the FP64 significand
// leading dimension (FP16 values, a multiple of 8) of the slices of `rows`-long columns
int slice_ld(int rows);
// the slices of the columns of X (rows x cols, column-major): Xs holds kSlices
// planes of cols x slice_ld(rows) FP16 values (as 16-bit words), F one
// power-of-two exponent per column
cudaError_t slice_cols(const double* X, int rows, int cols, uint16_t* Xs, int* F,
                       cudaStream_t st);
// Y = alpha A R (md x cnt, column-major) from the slices of the rows of A (As, Ea:
// slice_cols of A^T, i.e. of A's columns when A is symmetric) and of the columns
// of R (Rs, Fr)
cudaError_t gemm_f64_sliced(int md, int cnt, double alpha, const uint16_t* As, const int* Ea,
                            const uint16_t* Rs, const int* Fr, double* Y, cudaStream_t st);
// FP32: Y = alpha A R, A md x md, R and Y md x cnt, all column-major.
cudaError_t gemm_f32(int md, int cnt, float alpha, const float* A, const float* R, float* Y,
                     cudaStream_t st);

// ---- compensated defect of the FP32 V-cycle (defect_ff.cu) -------------------
// r = b - scale * A_ref x for an FP32 x, in double-float arithmetic on the FP32
// pipes (ffsweep.cuh), from the FP32 tables `tab32` (Ops<float>::make_tables);
// scratch: apply_scratch_arrays(d) * nd float2 values (8 bytes each).
cudaError_t defect_ff(const void* tab32, const LevelGeom& g, const float* x, const double* b,
                      double* r, double scale, void* scratch, cudaStream_t st);
// device copy of the hi + lo class tables (FfTab<k>) of FP32 tables
const void* ff_device_tables(const void* tab32, int k);
// the batched form's list kernel of degree k (ff_sweep_list_kernel; kind 0: the
// split of the FP32 x, 2: the residual), as the address the runtime API takes
const void* ff_list_kernel(int k, int kind);

// ---- vector kernels (FP64 unless noted) -------------------------------------
// Deterministic dot product: partial sums per block, then one block in fixed order.
constexpr int kDotBlocks = 608;  // 4 x 152 SMs
cudaError_t vec_dot(const double* x, const double* y, int64_t n, double* partials, double* out,
                    cudaStream_t st);
// y += a x (host scalar)
cudaError_t vec_axpy(double* y, double a, const double* x, int64_t n, cudaStream_t st);
// y += sign * (*a) x (device scalar)
cudaError_t vec_axpy_dev(double* y, const double* a, double sign, const double* x, int64_t n,
                         cudaStream_t st);
// y = a x
cudaError_t vec_scale(double* y, double a, const double* x, int64_t n, cudaStream_t st);
// y = x + a y (x must not alias y)
cudaError_t vec_xpay(double* y, double a, const double* x, int64_t n, cudaStream_t st);
// r = b - y
cudaError_t vec_sub(double* r, const double* b, const double* y, int64_t n, cudaStream_t st);
// conversions
cudaError_t vec_d2f(float* y, const double* x, int64_t n, cudaStream_t st);
cudaError_t vec_f2d(double* y, const float* x, int64_t n, cudaStream_t st);
// b = sum_terms c_t (F_t0 (x) F_t1 [(x) F_t2]) on the interior nodes of a level:
// separable right-hand sides; F holds nterms * d rows of n values.
cudaError_t rhs_separable(int d, int n, int nterms, const double* coef, const double* F,
                          double* b, cudaStream_t st);

}  // namespace bh
