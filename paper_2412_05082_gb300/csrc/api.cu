// C ABI (include/biharm.h): contexts, the V-cycle of Algorithm 1, the vertex-
// patch smoothers of Sec. 3 and the FP64 GMRES driver of Sec. 5.1.  Host code
// that enqueues the kernels of kernels.cuh / vec.cu on the context's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "biharm.h"
#include "ctx.h"
#include "ops.h"
#include "setup.h"

using namespace bh;

namespace {

thread_local std::string g_err;

bh_status fail(bh_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

#define CK(call)                                                                     \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess)                                                           \
      return fail(BH_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));     \
  } while (0)

#define CKS(call)                   \
  do {                              \
    bh_status s_ = (call);          \
    if (s_ != BH_OK) return s_;     \
  } while (0)

}  // namespace

namespace bh {
// message returned by bh_last_error() on this thread (used by noalloc.cu, batch.cu)
void set_last_error(const std::string& msg) { g_err = msg; }

// Host-side fault injection (bh_fault_inject_alloc): after g_alloc_skip more
// device allocations, the next g_alloc_fail ones fail as if cudaMalloc had
// returned cudaErrorMemoryAllocation, without calling it.
std::atomic<long long> g_alloc_skip{0}, g_alloc_fail{0};

bool alloc_fault() {
  if (g_alloc_fail.load() <= 0) return false;
  if (g_alloc_skip.fetch_sub(1) > 0) return false;
  g_alloc_skip.store(0);
  return g_alloc_fail.fetch_sub(1) > 0;
}
}  // namespace bh

namespace {

template <typename T>
bh_status dmalloc(bh_ctx* c, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) return BH_OK;
  cudaError_t e = alloc_fault() ? cudaErrorMemoryAllocation : cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(BH_ENOMEM, "cudaMalloc of " + std::to_string(count * sizeof(T)) +
                               " bytes failed: " + cudaGetErrorString(e));
  }
  c->dev_allocs.push_back(*p);
  return BH_OK;
}

int64_t ipow64(int64_t b, int e) {
  int64_t r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

int color_of(const int* v, int d) {
  int par = 0, rb = 0;
  for (int a = 0; a < d; ++a) {
    par |= (v[a] & 1) << a;
    rb += v[a] / 2;
  }
  return 2 * par + (rb & 1);
}

bool mixed(const bh_ctx* c) { return c->p.precision != BH_FP64; }
// FP32 V-cycle whose defects before each restriction are evaluated in FP64
// the FP32 V-cycle's defect before each restriction outside FP32 arithmetic:
// in FP64 (BH_MIXED_FP32_R64) or compensated FP32 (BH_MIXED_FP32_RC)
bool defect64(const bh_ctx* c) {
  return c->p.precision == BH_MIXED_FP32_R64 || c->p.precision == BH_MIXED_FP32_RC;
}

// typed accessors for the V-cycle template
template <typename T> struct TypeOf;
template <> struct TypeOf<double> {
  static double* x(Level& l) { return l.x64; }
  static double* b(Level& l) { return l.b64; }
  static double* r(Level& l) { return l.r64; }
  static void* tab(bh_ctx* c) { return c->tab64; }
  static double* scr(bh_ctx* c) { return c->scr64; }
  static double* xs(bh_ctx* c, int i) { return c->xs64[i]; }
  static double* ainv(bh_ctx* c) { return c->ainv64; }
  static double* gR(bh_ctx* c) { return c->gR64; }
  static double* gY(bh_ctx* c) { return c->gY64; }
};
template <> struct TypeOf<float> {
  static float* x(Level& l) { return l.x32; }
  static float* b(Level& l) { return l.b32; }
  static float* r(Level& l) { return l.r32; }
  static void* tab(bh_ctx* c) { return c->tab32; }
  static float* scr(bh_ctx* c) { return c->scr32; }
  static float* xs(bh_ctx* c, int i) { return c->xs32[i]; }
  static float* ainv(bh_ctx* c) { return c->ainv32; }
  static float* gR(bh_ctx* c) { return c->gR32; }
  static float* gY(bh_ctx* c) { return c->gY32; }
};

template <typename T>
bh_status residual_t(bh_ctx* c, int l, const T* x, const T* b, T* r) {
  Level& L = c->lv[l];
  CK(Ops<T>::apply(TypeOf<T>::tab(c), L.g, x, b, r, L.ascale, kResidual, TypeOf<T>::scr(c), c->st));
  return BH_OK;
}

// x += omega * sum_{v in verts[lo, hi)} R_v^T A_v^-1 R_v r
template <typename T>
bh_status patches_t(bh_ctx* c, int l, const T* r, T* x, int lo, int hi, bool atomic) {
  Level& L = c->lv[l];
  const double sc = c->p.omega * L.pscale;
  if (c->p.local_solver == BH_EXACT && c->exact_gemm) {
    // per color in [lo, hi) and run of one type combination: gather the patch
    // tensors as columns, Y = sc Ainv R (dense product, gemm.cu), scatter-add Y
    const int md = (int)std::lround(std::pow(2 * c->p.degree - 1, c->p.dim));
    const size_t msz = (size_t)md * md;
    T* R = TypeOf<T>::gR(c);
    T* Y = TypeOf<T>::gY(c);
    for (int col = 0; col < c->ncolors(); ++col) {
      if (L.coff[col] < lo || L.coff[col + 1] > hi) continue;
      for (const auto& run : L.runs[col]) {
        const int* vs = L.verts + run[0];
        const int cnt = run[1];
        const T* Ainv = TypeOf<T>::ainv(c) + (size_t)run[2] * msz;
        CK(Ops<T>::patch_gather(L.g, r, vs, cnt, R, c->st));
        if constexpr (std::is_same<T, double>::value) {
          // FP64 by FP16 slices: slice the run's columns, then the sliced product
          const size_t sl = (size_t)kSlices * md * slice_ld(md);
          CK(slice_cols(R, md, cnt, c->gRs, c->gRe, c->st));
          CK(gemm_f64_sliced(md, cnt, sc, c->ainv_sl + (size_t)run[2] * sl,
                             c->ainv_ex + (size_t)run[2] * md, c->gRs, c->gRe, Y, c->st));
        } else {
          CK(gemm_f32(md, cnt, (float)sc, Ainv, R, Y, c->st));
        }
        CK(Ops<T>::patch_scatter(L.g, Y, vs, cnt, x, atomic, c->st));
      }
    }
  } else if (c->p.local_solver == BH_EXACT)
    CK(Ops<T>::patch_exact(L.g, TypeOf<T>::ainv(c), r, x, L.verts + lo, hi - lo, sc, atomic,
                           c->st));
  else
    CK(Ops<T>::patch_fdm(TypeOf<T>::tab(c), L.g, r, x, L.verts + lo, hi - lo, sc, atomic,
                         c->st));
  return BH_OK;
}

// colors c0 .. c1-1 of one colored MVS step on level l; zero: x holds zeros on
// entry (the first color skips its residual)
template <typename T>
bh_status mvs_colors_t(bh_ctx* c, int l, T* x, const T* b, int c0, int c1, bool zero) {
  Level& L = c->lv[l];
  T* R = TypeOf<T>::r(L);
  for (int col = c0; col < c1; ++col) {
    if (c->p.local_solver == BH_FDM) {
      // fused kernel: local residual, fast diagonalization and update per patch
      CK(Ops<T>::mvs_color(TypeOf<T>::tab(c), L.g, x, b, L.verts + L.coff[col],
                           L.coff[col + 1] - L.coff[col], L.ascale, c->p.omega * L.pscale,
                           c->tile, c->st));
    } else {
      const T* r = b;
      if (!(zero && col == c0)) {
        CKS(residual_t<T>(c, l, x, b, R));
        r = R;
      }
      CKS(patches_t<T>(c, l, r, x, L.coff[col], L.coff[col + 1], false));
    }
  }
  return BH_OK;
}

// steps smoothing steps on level l; x_zero: x holds zeros on entry (skips a residual)
template <typename T>
bh_status smooth_t(bh_ctx* c, int l, T* x, const T* b, int steps, bool x_zero) {
  Level& L = c->lv[l];
  T* R = TypeOf<T>::r(L);
  const int d = c->p.dim, nc = c->ncolors();
  for (int s = 0; s < steps; ++s) {
    const bool zero = x_zero && s == 0;
    if (c->p.smoother == BH_MVS_COLORED) {
      CKS(mvs_colors_t<T>(c, l, x, b, 0, nc, zero));
    } else {
      const T* r = b;
      if (!zero) {
        CKS(residual_t<T>(c, l, x, b, R));
        r = R;
      }
      if (c->p.smoother == BH_AVS_ATOMIC) {
        CKS(patches_t<T>(c, l, r, x, 0, L.coff[nc], true));
      } else {  // colored AVS: 2^d write colors = MVS color pairs (2 par, 2 par + 1)
        for (int par = 0; par < (1 << d); ++par)
          CKS(patches_t<T>(c, l, r, x, L.coff[2 * par], L.coff[2 * par + 2], false));
      }
    }
  }
  return BH_OK;
}

// BH_MIXED_FP32_R64: the defect b_l - A_l x of the FP32 V-cycle, evaluated in
// FP64 arithmetic from the FP32 iterate (exactly representable in FP64) and the
// FP64 right-hand side L.db64, restricted in FP64 into Lc.db64 and rounded into
// Lc.b32.  In FP32 arithmetic the cancellation in A x leaves a rounding error
// of about eps_32 ||A|| ||x||, whose smooth part the coarse-grid correction
// amplifies like the condition number of A_l.
//
// BH_MIXED_FP32_RC: the same defect in compensated FP32 arithmetic (double-float
// values, exact products by FMA, error-free sums: defect_ff.cu), about 2^-44 of
// sum |terms| accurate, on the FP32 pipes; the restriction stays FP64.
bh_status restrict_defect64(bh_ctx* c, int l, const float* x, bool x_zero) {
  Level& L = c->lv[l];
  Level& Lc = c->lv[l - 1];
  const double* r = L.db64;
  if (!(x_zero && c->p.pre_steps == 0)) {
    if (c->p.precision == BH_MIXED_FP32_RC) {
      CK(defect_ff(c->tab32, L.g, x, L.db64, L.r64, L.ascale, c->scr64, c->st));
    } else {
      CK(vec_f2d(L.dx64, x, L.g.nd, c->st));
      CKS(residual_t<double>(c, l, L.dx64, L.db64, L.r64));
    }
    r = L.r64;
  }
  // the FP32 right-hand side of level l-1 written by the restriction's last pass
  CK(Ops<double>::restrict_(c->tab64, L.g, r, Lc.db64, c->xs64[0], c->xs64[1], c->st, Lc.b32));
  return BH_OK;
}

template <typename T>
bh_status coarse_t(bh_ctx* c, T* x, const T* b, bool x_zero) {
  Level& L = c->lv[1];
  if (c->p.coarse == BH_COARSE_SMOOTH) return smooth_t<T>(c, 1, x, b, 1, x_zero);
  if (x_zero) {
    CK(Ops<T>::dense_symv(c->coarse_n, c->coarse_inv, b, x, L.pscale, c->st));
  } else {
    T* R = TypeOf<T>::r(L);
    T* tmp = TypeOf<T>::scr(c);
    CKS(residual_t<T>(c, 1, x, b, R));
    CK(Ops<T>::dense_symv(c->coarse_n, c->coarse_inv, R, tmp, L.pscale, c->st));
    CK(Ops<T>::add(x, tmp, L.g.nd, c->st));
  }
  return BH_OK;
}

// Algorithm 1: x <- MG_l(x, b)
template <typename T>
bh_status vcycle_t(bh_ctx* c, int l, T* x, const T* b, bool x_zero) {
  if (l == 1) return coarse_t<T>(c, x, b, x_zero);
  Level& L = c->lv[l];
  Level& Lc = c->lv[l - 1];
  T* R = TypeOf<T>::r(L);
  CKS(smooth_t<T>(c, l, x, b, c->p.pre_steps, x_zero));
  if constexpr (std::is_same<T, float>::value) {
    if (defect64(c)) {
      CKS(restrict_defect64(c, l, x, x_zero));
    } else {
      if (x_zero && c->p.pre_steps == 0)
        CK(cudaMemcpyAsync(R, b, L.g.nd * sizeof(T), cudaMemcpyDeviceToDevice, c->st));
      else
        CKS(residual_t<T>(c, l, x, b, R));
      CK(Ops<T>::restrict_(TypeOf<T>::tab(c), L.g, R, TypeOf<T>::b(Lc), TypeOf<T>::xs(c, 0),
                           TypeOf<T>::xs(c, 1), c->st));
    }
  } else {
    if (x_zero && c->p.pre_steps == 0)
      CK(cudaMemcpyAsync(R, b, L.g.nd * sizeof(T), cudaMemcpyDeviceToDevice, c->st));
    else
      CKS(residual_t<T>(c, l, x, b, R));
    CK(Ops<T>::restrict_(TypeOf<T>::tab(c), L.g, R, TypeOf<T>::b(Lc), TypeOf<T>::xs(c, 0),
                         TypeOf<T>::xs(c, 1), c->st));
  }
  CK(cudaMemsetAsync(TypeOf<T>::x(Lc), 0, Lc.g.nd * sizeof(T), c->st));
  CKS(vcycle_t<T>(c, l - 1, TypeOf<T>::x(Lc), TypeOf<T>::b(Lc), true));
  CK(Ops<T>::prolongate_add(TypeOf<T>::tab(c), L.g, TypeOf<T>::x(Lc), x, TypeOf<T>::xs(c, 0),
                            TypeOf<T>::xs(c, 1), c->st));
  CKS(smooth_t<T>(c, l, x, b, c->p.post_steps, false));
  return BH_OK;
}

// z = MG_L(0, v) in the context's precision (FP64 in and out)
bh_status precondition(bh_ctx* c, const double* v, double* z) {
  const int L = c->p.level;
  Level& F = c->lv[L];
  if (!mixed(c)) {
    CK(cudaMemsetAsync(z, 0, F.g.nd * sizeof(double), c->st));
    return vcycle_t<double>(c, L, z, v, true);
  }
  CK(vec_d2f(F.b32, v, F.g.nd, c->st));
  if (defect64(c))
    CK(cudaMemcpyAsync(F.db64, v, F.g.nd * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  CK(cudaMemsetAsync(F.x32, 0, F.g.nd * sizeof(float), c->st));
  CKS(vcycle_t<float>(c, L, F.x32, F.b32, true));
  CK(vec_f2d(z, F.x32, F.g.nd, c->st));
  return BH_OK;
}

bh_status check_level(const bh_ctx* c, int level) {
  if (!c) return fail(BH_EINVAL, "null context");
  if (level < 1 || level > c->p.level)
    return fail(BH_EINVAL, "level " + std::to_string(level) + " outside 1.." +
                               std::to_string(c->p.level));
  return BH_OK;
}

void destroy_ctx(bh_ctx* c) {
  if (!c) return;
  if (c->st) cudaStreamSynchronize(c->st);
  for (void* p : c->dev_allocs) cudaFree(p);
  if (c->hdots) cudaFreeHost(c->hdots);
  for (cudaEvent_t e : c->ev)
    if (e) cudaEventDestroy(e);
  if (c->tab64) Ops<double>::free_tables(c->tab64, c->p.degree);
  if (c->tab32) Ops<float>::free_tables(c->tab32, c->p.degree);
  delete c;
}

// device dot results, reduction partials and their pinned host copy
bh_status ensure_scalars(bh_ctx* c) {
  if (c->dots) return BH_OK;
  const int cnt = std::max(1, c->p.gmres_restart) + 2;
  CKS(dmalloc(c, &c->dots, (size_t)cnt));
  CKS(dmalloc(c, &c->partials, (size_t)kDotBlocks));
  if (cudaMallocHost((void**)&c->hdots, cnt * sizeof(double)) != cudaSuccess) {
    c->hdots = nullptr;
    return fail(BH_ENOMEM, "cudaMallocHost failed");
  }
  return BH_OK;
}

bh_status ensure_gmres(bh_ctx* c) {
  CKS(ensure_scalars(c));
  if (c->V) return BH_OK;
  const int m = std::max(1, c->p.gmres_restart);
  const int64_t n = c->lv[c->p.level].g.nd;
  c->m = m;
  CKS(dmalloc(c, &c->V, (size_t)(m + 1) * n));
  CKS(dmalloc(c, &c->Z, (size_t)m * n));
  CKS(dmalloc(c, &c->w, (size_t)n));
  CKS(dmalloc(c, &c->t, (size_t)n));
  return BH_OK;
}

bh_status ensure_cg(bh_ctx* c) {
  CKS(ensure_scalars(c));
  if (c->cgv) return BH_OK;
  return dmalloc(c, &c->cgv, (size_t)5 * c->lv[c->p.level].g.nd);
}

// copy the first cnt device dot results to the host (one synchronization)
bh_status fetch_dots(bh_ctx* c, int cnt) {
  CK(cudaMemcpyAsync(c->hdots, c->dots, cnt * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  return BH_OK;
}

bh_status norm2(bh_ctx* c, const double* x, double* out) {
  const int64_t n = c->lv[c->p.level].g.nd;
  CK(vec_dot(x, x, n, c->partials, c->dots, c->st));
  CK(cudaMemcpyAsync(c->hdots, c->dots, sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  *out = std::sqrt(c->hdots[0]);
  return BH_OK;
}

// one Arnoldi column: w = op(V_j); MGS against V_0..V_j on the device
bh_status arnoldi_column(bh_ctx* c, int j, double* hcol, double* hnorm) {
  const int L = c->p.level;
  const int64_t n = c->lv[L].g.nd;
  double* Vj = c->V + (int64_t)j * n;
  Level& F = c->lv[L];
  if (c->p.gmres_side == BH_LEFT) {
    CK(Ops<double>::apply(c->tab64, F.g, Vj, nullptr, c->t, F.ascale, kStore, c->scr64, c->st));
    CKS(precondition(c, c->t, c->w));
  } else {
    double* Zj = c->Z + (int64_t)j * n;
    CKS(precondition(c, Vj, Zj));
    CK(Ops<double>::apply(c->tab64, F.g, Zj, nullptr, c->w, F.ascale, kStore, c->scr64, c->st));
  }
  for (int i = 0; i <= j; ++i) {
    const double* Vi = c->V + (int64_t)i * n;
    CK(vec_dot(c->w, Vi, n, c->partials, c->dots + i, c->st));
    CK(vec_axpy_dev(c->w, c->dots + i, -1.0, Vi, n, c->st));
  }
  CK(vec_dot(c->w, c->w, n, c->partials, c->dots + j + 1, c->st));
  CK(cudaMemcpyAsync(c->hdots, c->dots, (j + 2) * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  for (int i = 0; i <= j; ++i) hcol[i] = c->hdots[i];
  *hnorm = std::sqrt(c->hdots[j + 1]);
  return BH_OK;
}

// Preconditioned conjugate gradients, x0 = 0 (Sec. 5.1 uses it with the
// additive smoother).  Stops on the recursively updated residual
// ||r_j|| <= rtol ||b||.  The FP32 V-cycle is not a fixed linear operator, so
// the mixed form takes the Polak-Ribiere coefficient
// beta = r_{j+1}.(z_{j+1} - z_j) / r_j.z_j (flexible CG); for a fixed
// preconditioner r_{j+1}.z_j = 0 and it equals r_{j+1}.z_{j+1} / r_j.z_j.
bh_status solve_cg(bh_ctx* c, const double* b, double* x, double rtol, int maxit, int* iters,
                   double* relres) {
  CKS(ensure_cg(c));
  const int L = c->p.level;
  Level& F = c->lv[L];
  const int64_t n = F.g.nd;
  const bool flexible = mixed(c);
  double* r = c->cgv;
  double* z = r + n;
  double* p = z + n;
  double* q = p + n;
  double* zp = q + n;
  CK(cudaMemsetAsync(x, 0, n * sizeof(double), c->st));
  double bnorm;
  CKS(norm2(c, b, &bnorm));
  *iters = 0;
  *relres = 0.0;
  if (bnorm == 0.0) return BH_OK;
  if (!std::isfinite(bnorm)) return fail(BH_EINVAL, "right-hand side is not finite");
  CK(cudaMemcpyAsync(r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  CKS(precondition(c, r, z));
  CK(cudaMemcpyAsync(p, z, n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  CK(vec_dot(r, z, n, c->partials, c->dots, c->st));
  CKS(fetch_dots(c, 1));
  double rz = c->hdots[0];
  int it = 0;
  double rn = bnorm;
  while (it < maxit) {
    CK(Ops<double>::apply(c->tab64, F.g, p, nullptr, q, F.ascale, kStore, c->scr64, c->st));
    CK(vec_dot(p, q, n, c->partials, c->dots, c->st));
    CKS(fetch_dots(c, 1));
    const double pq = c->hdots[0];
    if (!(pq > 0.0) || !std::isfinite(pq) || !std::isfinite(rz))
      return fail(BH_ENOCONV, "CG breakdown: p.Ap <= 0 or not finite after " +
                                  std::to_string(it) + " iterations");
    const double alpha = rz / pq;
    CK(vec_axpy(x, alpha, p, n, c->st));
    CK(vec_axpy(r, -alpha, q, n, c->st));
    ++it;
    CKS(norm2(c, r, &rn));
    if (!std::isfinite(rn)) return fail(BH_ENOCONV, "CG breakdown: non-finite residual");
    if (rn <= rtol * bnorm) break;
    if (flexible) std::swap(z, zp);  // zp = z_j, z is overwritten by z_{j+1}
    CKS(precondition(c, r, z));
    CK(vec_dot(r, z, n, c->partials, c->dots, c->st));
    if (flexible) CK(vec_dot(r, zp, n, c->partials, c->dots + 1, c->st));
    CKS(fetch_dots(c, flexible ? 2 : 1));
    const double rz_new = c->hdots[0];
    const double beta = flexible ? (rz_new - c->hdots[1]) / rz : rz_new / rz;
    CK(vec_xpay(p, beta, z, n, c->st));
    rz = rz_new;
  }
  CKS(residual_t<double>(c, L, x, b, q));
  double tn;
  CKS(norm2(c, q, &tn));
  *iters = it;
  *relres = tn / bnorm;
  c->n_solve++;
  c->last_iters = it;
  c->last_relres = *relres;
  c->last_estimate = rn / bnorm;
  if (!(rn <= rtol * bnorm))
    return fail(BH_ENOCONV, "CG stopped after " + std::to_string(it) +
                                " iterations above the tolerance");
  return BH_OK;
}

bh_status solve_dev(bh_ctx* c, const double* b, double* x, double rtol, int maxit, int* iters,
                    double* relres) {
  if (c->p.krylov == BH_CG) return solve_cg(c, b, x, rtol, maxit, iters, relres);
  CKS(ensure_gmres(c));
  const int L = c->p.level, m = c->m;
  Level& F = c->lv[L];
  const int64_t n = F.g.nd;
  const bool left = c->p.gmres_side == BH_LEFT;
  CK(cudaMemsetAsync(x, 0, n * sizeof(double), c->st));
  double bnorm;
  CKS(norm2(c, b, &bnorm));
  *iters = 0;
  *relres = 0.0;
  if (bnorm == 0.0) return BH_OK;
  if (!std::isfinite(bnorm)) return fail(BH_EINVAL, "right-hand side is not finite");
  // r0 = b (x0 = 0), or M^-1 b
  double* r = c->t;
  if (left) {
    CKS(precondition(c, b, c->t));
  } else {
    CK(cudaMemcpyAsync(c->t, b, n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  }
  double beta;
  CKS(norm2(c, r, &beta));
  const double ref = beta;
  std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), g(m + 1), y(m), hcol(m + 2);
  int it = 0;
  bool stop = false;
  double est = beta;
  while (true) {
    if (!(beta > 0.0) || !std::isfinite(beta)) break;
    CK(vec_scale(c->V, 1.0 / beta, r, n, c->st));
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int jdone = 0;
    for (int j = 0; j < m; ++j) {
      double hn;
      CKS(arnoldi_column(c, j, hcol.data(), &hn));
      auto Hij = [&](int i, int jj) -> double& { return H[(size_t)i * m + jj]; };
      for (int i = 0; i <= j; ++i) Hij(i, j) = hcol[i];
      Hij(j + 1, j) = hn;
      for (int i = 0; i < j; ++i) {
        const double tt = cs[i] * Hij(i, j) + sn[i] * Hij(i + 1, j);
        Hij(i + 1, j) = -sn[i] * Hij(i, j) + cs[i] * Hij(i + 1, j);
        Hij(i, j) = tt;
      }
      const double rho = std::hypot(Hij(j, j), Hij(j + 1, j));
      cs[j] = Hij(j, j) / rho;
      sn[j] = Hij(j + 1, j) / rho;
      Hij(j, j) = rho;
      Hij(j + 1, j) = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++it;
      jdone = j + 1;
      est = std::fabs(g[j + 1]);
      if (!std::isfinite(est)) return fail(BH_ENOCONV, "GMRES breakdown: non-finite residual");
      if (est <= rtol * ref || it >= maxit || hn == 0.0) {
        stop = true;
        break;
      }
      CK(vec_scale(c->V + (int64_t)(j + 1) * n, 1.0 / hn, c->w, n, c->st));
    }
    for (int i = jdone - 1; i >= 0; --i) {
      double sacc = g[i];
      for (int jj = i + 1; jj < jdone; ++jj) sacc -= H[(size_t)i * m + jj] * y[jj];
      y[i] = sacc / H[(size_t)i * m + i];
    }
    const double* basis = left ? c->V : c->Z;
    for (int i = 0; i < jdone; ++i) CK(vec_axpy(x, y[i], basis + (int64_t)i * n, n, c->st));
    CKS(residual_t<double>(c, L, x, b, c->t));
    if (stop) break;
    if (left) {
      CK(cudaMemcpyAsync(c->w, c->t, n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
      CKS(precondition(c, c->w, c->t));
    }
    r = c->t;
    CKS(norm2(c, r, &beta));
  }
  // the true residual b - A x is in c->t after the last update
  double rn;
  CKS(norm2(c, c->t, &rn));
  *iters = it;
  *relres = rn / bnorm;
  c->n_solve++;
  c->last_iters = it;
  c->last_relres = *relres;
  c->last_estimate = est / ref;
  if (!(est <= rtol * ref)) return fail(BH_ENOCONV, "GMRES stopped after " + std::to_string(it) +
                                                        " iterations above the tolerance");
  return BH_OK;
}

// solve_dev bracketed by CUDA events on the context's stream: the device time
// of the last solve, for bh_stats
bh_status timed_solve(bh_ctx* c, const double* b, double* x, double rtol, int maxit, int* iters,
                      double* relres) {
  if (!c->ev[0]) {
    if (cudaEventCreate(&c->ev[0]) != cudaSuccess || cudaEventCreate(&c->ev[1]) != cudaSuccess)
      return fail(BH_ECUDA, "event creation failed");
  }
  CK(cudaEventRecord(c->ev[0], c->st));
  const bh_status s = solve_dev(c, b, x, rtol, maxit, iters, relres);
  if (s != BH_OK && s != BH_ENOCONV) return s;
  CK(cudaEventRecord(c->ev[1], c->st));
  CK(cudaEventSynchronize(c->ev[1]));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
  c->last_solve_ms = ms;
  return s;
}

// 1D load vectors int s^(deriv)(x) phi_g(x) dx over the N cells of a level
void load_1d(const Setup1D& s, int N, int kind, std::vector<double>& out) {
  const int k = s.k, n = k * N - 1;
  std::vector<double> x, w;
  gauss_rule(k + 3, x, w);
  out.assign(n, 0.0);
  const double h = 1.0 / N, pi = M_PI;
  for (int c = 0; c < N; ++c)
    for (size_t q = 0; q < x.size(); ++q) {
      const double X = (c + x[q]) * h;
      double f;
      switch (kind) {
        case 0: f = std::sin(pi * X) * std::sin(pi * X); break;       // sin^2
        case 2: f = 2.0 * pi * pi * std::cos(2.0 * pi * X); break;    // (sin^2)''
        case 4: f = -8.0 * std::pow(pi, 4) * std::cos(2.0 * pi * X); break;  // (sin^2)''''
        default: f = std::sin(pi * X); break;                         // sin
      }
      for (int i = 0; i <= k; ++i) {
        const int g = k * c + i;
        if (g < 1 || g > n) continue;
        out[g - 1] += h * w[q] * f * lagrange(s.z, i, x[q], 0);
      }
    }
}

}  // namespace

extern "C" {

const char* bh_last_error(void) { return g_err.c_str(); }

bh_status bh_default_params(int dim, int degree, int level, bh_params* out) {
  if (!out) return fail(BH_EINVAL, "null params");
  if (dim != 2 && dim != 3) return fail(BH_EINVAL, "dim must be 2 or 3");
  if (degree < 2 || degree > kMaxK) return fail(BH_EINVAL, "degree must be in 2..7");
  if (level < 1 || level > 14) return fail(BH_EINVAL, "level must be in 1..14");
  bh_params p{};
  p.dim = dim;
  p.degree = degree;
  p.level = level;
  p.gamma = 0.0;
  p.smoother = BH_MVS_COLORED;
  p.local_solver = BH_FDM;
  p.pre_steps = 1;
  p.post_steps = 1;
  p.omega = 0.0;
  p.precision = BH_FP64;
  p.gmres_restart = 50;
  p.gmres_side = BH_RIGHT;
  p.coarse = BH_COARSE_EXACT;
  p.krylov = BH_GMRES;
  *out = p;
  return BH_OK;
}

bh_status bh_create(const bh_params* params, void* stream, bh_ctx** out) {
  if (!params || !out) return fail(BH_EINVAL, "null argument");
  *out = nullptr;
  bh_params p = *params;
  if (p.dim != 2 && p.dim != 3) return fail(BH_EINVAL, "dim must be 2 or 3");
  if (p.degree < 2 || p.degree > kMaxK) return fail(BH_EINVAL, "degree must be in 2..7");
  if (p.level < 1 || p.level > 14) return fail(BH_EINVAL, "level must be in 1..14");
  if (p.smoother < 0 || p.smoother > 2) return fail(BH_EINVAL, "unknown smoother");
  if (p.local_solver < 0 || p.local_solver > 1) return fail(BH_EINVAL, "unknown local solver");
  if (p.precision < 0 || p.precision > 3) return fail(BH_EINVAL, "unknown precision");
  if (p.pre_steps < 0 || p.post_steps < 0) return fail(BH_EINVAL, "negative smoothing steps");
  if (p.gmres_side < 0 || p.gmres_side > 1) return fail(BH_EINVAL, "unknown GMRES side");
  if (p.coarse < 0 || p.coarse > 1) return fail(BH_EINVAL, "unknown coarse solver");
  if (p.krylov < 0 || p.krylov > 1) return fail(BH_EINVAL, "unknown Krylov method");
  if (p.krylov == BH_CG && p.smoother == BH_MVS_COLORED)
    return fail(BH_EINVAL,
                "CG needs a symmetric preconditioner: the V-cycle with the additive smoother "
                "(the multiplicative one goes with GMRES)");
  if (p.krylov == BH_GMRES && p.precision != BH_FP64 && p.gmres_side == BH_LEFT)
    return fail(BH_EINVAL,
                "the FP32 V-cycle is not a fixed linear operator (its rounding varies): mixed "
                "precision needs the flexible right-preconditioned GMRES, gmres_side = BH_RIGHT");
  const int d = p.dim, k = p.degree;
  if (!(p.gamma > 0.0)) p.gamma = k * (k + 1.0);
  if (!(p.omega > 0.0)) {
    if (p.smoother == BH_MVS_COLORED)
      p.omega = d == 2 ? 1.0 : 0.7;
    else
      p.omega = d == 2 ? 0.25 : (p.local_solver == BH_EXACT ? 0.125 : 0.1);
  }
  if (p.gmres_restart <= 0) p.gmres_restart = 50;
  // patch vertex ids are int32 and every sweep line is indexed in int32
  if (ipow64((int64_t)k * (1 << p.level) - 1, d) > ((int64_t)1 << 40))
    return fail(BH_EINVAL, "problem too large");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(BH_ECUDA, "no CUDA device available");
  }
  bh_ctx* c = new (std::nothrow) bh_ctx();
  if (!c) return fail(BH_ENOMEM, "host allocation failed");
  c->p = p;
  c->st = (cudaStream_t)stream;
  bh_status status = BH_OK;
  auto bail = [&](bh_status s) {
    destroy_ctx(c);
    return s;
  };
  try {
    build_setup(k, p.gamma, c->s);
  } catch (const std::exception& e) {
    delete c;
    return fail(BH_EINVAL, std::string("setup failed: ") + e.what());
  }
  const bool mx = p.precision != BH_FP64;
  c->tab64 = Ops<double>::make_tables(c->s, d);
  if (!c->tab64) return bail(fail(BH_ENOMEM, "device tables"));
  if (mx) {
    c->tab32 = Ops<float>::make_tables(c->s, d);
    if (!c->tab32) return bail(fail(BH_ENOMEM, "device tables"));
  }
  c->lv.resize(p.level + 1);
  int md_local = 1;
  for (int a = 0; a < d; ++a) md_local *= 2 * k - 1;
  const bool gemm_exact = p.local_solver == BH_EXACT && md_local >= kExactGemmMin;
  c->exact_gemm = gemm_exact;
  for (int l = 1; l <= p.level; ++l) {
    Level& L = c->lv[l];
    L.g.d = d;
    L.g.k = k;
    L.g.N = 1 << l;
    L.g.n = k * L.g.N - 1;
    L.g.nd = ipow64(L.g.n, d);
    L.ascale = std::pow((double)L.g.N, 4 - d);
    L.pscale = 1.0 / L.ascale;
    const size_t nd = (size_t)L.g.nd;
    if ((status = dmalloc(c, &L.x64, nd)) || (status = dmalloc(c, &L.b64, nd)) ||
        (status = dmalloc(c, &L.r64, nd)))
      return bail(status);
    if (mx && ((status = dmalloc(c, &L.x32, nd)) || (status = dmalloc(c, &L.b32, nd)) ||
               (status = dmalloc(c, &L.r32, nd))))
      return bail(status);
    if ((p.precision == BH_MIXED_FP32_R64 || p.precision == BH_MIXED_FP32_RC) &&
        (status = dmalloc(c, &L.db64, nd)))
      return bail(status);
    if (p.precision == BH_MIXED_FP32_R64 && (status = dmalloc(c, &L.dx64, nd)))
      return bail(status);
    // vertex patches sorted by color (Sec. 3), lexicographic inside a color
    const int Nm = L.g.N - 1;
    const int64_t nv = ipow64(Nm, d);
    std::vector<int> ids[16];
    // inside a color: patches away from the boundary first, then the rest, so
    // that thread blocks of the patch kernels see one code path
    std::vector<int> edge[16];
    for (int64_t vid = 0; vid < nv; ++vid) {
      int v[3] = {(int)(vid % Nm) + 1, (int)((vid / Nm) % Nm) + 1,
                  d == 3 ? (int)(vid / ((int64_t)Nm * Nm)) + 1 : 0};
      bool inner = true;
      for (int a = 0; a < d; ++a) inner &= v[a] >= 2 && v[a] <= Nm - 1;
      (inner ? ids : edge)[color_of(v, d)].push_back((int)vid);
    }
    for (int col = 0; col < 16; ++col) ids[col].insert(ids[col].end(), edge[col].begin(), edge[col].end());
    // exact solver by dense products: inside a color, runs of one boundary-type
    // combination (the interior one first)
    auto combo_of = [&](int vid) {
      int combo = 0, mul = 1;
      for (int a = 0; a < d; ++a) {
        const int v = vid % Nm + 1;
        vid /= Nm;
        combo += (L.g.N == 2 ? kBoth : (v == 1 ? kLeft : (v == Nm ? kRight : kInterior))) * mul;
        mul *= 4;
      }
      return combo;
    };
    if (gemm_exact)
      for (int col = 0; col < 16; ++col)
        std::stable_sort(ids[col].begin(), ids[col].end(),
                         [&](int x, int y) { return combo_of(x) < combo_of(y); });
    std::vector<int> all;
    all.reserve(nv);
    for (int col = 0; col < c->ncolors(); ++col) {
      L.coff[col] = (int)all.size();
      if (gemm_exact) {
        for (size_t i = 0; i < ids[col].size();) {
          const int cb = combo_of(ids[col][i]);
          size_t j = i;
          while (j < ids[col].size() && combo_of(ids[col][j]) == cb) ++j;
          L.runs[col].push_back({L.coff[col] + (int)i, (int)(j - i), cb});
          c->gemm_cols = std::max(c->gemm_cols, (int)(j - i));
          i = j;
        }
      }
      all.insert(all.end(), ids[col].begin(), ids[col].end());
    }
    L.coff[c->ncolors()] = (int)all.size();
    if ((status = dmalloc(c, &L.verts, all.size()))) return bail(status);
    if (cudaMemcpy(L.verts, all.data(), all.size() * sizeof(int), cudaMemcpyHostToDevice) !=
        cudaSuccess)
      return bail(fail(BH_ECUDA, "upload of patch lists failed"));
  }
  const size_t ndL = (size_t)c->lv[p.level].g.nd;
  const int arrays = apply_scratch_arrays(d);
  if ((status = dmalloc(c, &c->scr64, ndL * arrays)) || (status = dmalloc(c, &c->xs64[0], ndL)) ||
      (status = dmalloc(c, &c->xs64[1], ndL)))
    return bail(status);
  if (mx && ((status = dmalloc(c, &c->scr32, ndL * arrays)) ||
             (status = dmalloc(c, &c->xs32[0], ndL)) || (status = dmalloc(c, &c->xs32[1], ndL))))
    return bail(status);
  // dense inverses: coarse level (one patch touching both faces in every
  // direction) and, for the exact local solver, every patch type combination
  const int m = 2 * k - 1;
  int md = 1;
  for (int a = 0; a < d; ++a) md *= m;
  {
    int types[3] = {kBoth, kBoth, kBoth};
    std::vector<double> A;
    patch_matrix(c->s, d, types, true, A);
    if (!spd_inverse(md, A.data())) return bail(fail(BH_EINVAL, "coarse matrix not SPD"));
    c->coarse_n = md;
    if ((status = dmalloc(c, &c->coarse_inv, A.size()))) return bail(status);
    if (cudaMemcpy(c->coarse_inv, A.data(), A.size() * sizeof(double), cudaMemcpyHostToDevice) !=
        cudaSuccess)
      return bail(fail(BH_ECUDA, "upload of the coarse inverse failed"));
  }
  if (gemm_exact) {
    const size_t cols = (size_t)md * c->gemm_cols;
    if ((status = dmalloc(c, &c->gR64, cols)) || (status = dmalloc(c, &c->gY64, cols)))
      return bail(status);
    const size_t slices = (size_t)kSlices * slice_ld(md);
    if ((status = dmalloc(c, &c->gRs, slices * c->gemm_cols)) ||
        (status = dmalloc(c, &c->gRe, (size_t)c->gemm_cols)) ||
        (status = dmalloc(c, &c->ainv_sl, slices * md * (d == 2 ? 16 : 64))) ||
        (status = dmalloc(c, &c->ainv_ex, (size_t)md * (d == 2 ? 16 : 64))))
      return bail(status);
    if (mx && ((status = dmalloc(c, &c->gR32, cols)) || (status = dmalloc(c, &c->gY32, cols))))
      return bail(status);
  }
  if (p.local_solver == BH_EXACT) {
    const int slots = d == 2 ? 16 : 64;
    const size_t msz = (size_t)md * md;
    if ((status = dmalloc(c, &c->ainv64, msz * slots))) return bail(status);
    if (mx && (status = dmalloc(c, &c->ainv32, msz * slots))) return bail(status);
    // The slots' patch matrices are related by symmetry: reflecting an axis
    // exchanges the types "left boundary" and "right boundary", and the terms
    // of the tensor form are invariant under axis permutations.  Each inverse
    // is therefore gathered from the inverse of one canonical slot (no right-
    // boundary type, types non-increasing over the axes): 4 dense inversions
    // instead of 27 in 3D.
    std::vector<std::pair<std::vector<int>, std::vector<double>>> canon;
    std::vector<double> A(msz);
    std::vector<float> Af;
    for (int slot = 0; slot < slots; ++slot) {
      int types[3] = {slot % 4, (slot / 4) % 4, slot / 16};
      bool any_both = false, all_both = true;
      for (int a = 0; a < d; ++a) {
        any_both |= types[a] == kBoth;
        all_both &= types[a] == kBoth;
      }
      if (any_both && !all_both) continue;  // "both" occurs only on the N = 2 level
      int u[3] = {0, 0, 0}, ord[3] = {0, 1, 2};
      bool refl[3] = {false, false, false};
      for (int a = 0; a < d; ++a) {
        refl[a] = types[a] == kRight;
        u[a] = refl[a] ? kLeft : types[a];
      }
      std::stable_sort(ord, ord + d, [&](int x, int y) { return u[x] > u[y]; });
      std::vector<int> key(d);
      for (int b = 0; b < d; ++b) key[b] = u[ord[b]];
      auto it = std::find_if(canon.begin(), canon.end(),
                             [&](const std::pair<std::vector<int>, std::vector<double>>& e) {
                               return e.first == key;
                             });
      if (it == canon.end()) {
        int kt[3] = {0, 0, 0};
        for (int b = 0; b < d; ++b) kt[b] = key[b];
        std::vector<double> Ac;
        patch_matrix(c->s, d, kt, true, Ac);
        if (!spd_inverse(md, Ac.data())) return bail(fail(BH_EINVAL, "patch matrix not SPD"));
        canon.emplace_back(key, std::move(Ac));
        it = canon.end() - 1;
      }
      // canonical index of a local index: axis b of the canonical slot is axis
      // ord[b] of this one, reversed where this one has the right-boundary type
      std::vector<int> cidx(md);
      for (int I = 0; I < md; ++I) {
        const int ii[3] = {I % m, (I / m) % m, I / (m * m)};
        int C = 0, mul = 1;
        for (int b = 0; b < d; ++b) {
          const int a = ord[b];
          C += (refl[a] ? m - 1 - ii[a] : ii[a]) * mul;
          mul *= m;
        }
        cidx[I] = C;
      }
      const std::vector<double>& Ac = it->second;
#pragma omp parallel for schedule(static)
      for (int I = 0; I < md; ++I)
        for (int J = 0; J < md; ++J) A[(size_t)I * md + J] = Ac[(size_t)cidx[I] * md + cidx[J]];
      if (cudaMemcpy(c->ainv64 + slot * msz, A.data(), msz * sizeof(double),
                     cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(fail(BH_ECUDA, "upload of local inverses failed"));
      if (gemm_exact) {  // slices of the rows (= columns: the inverse is symmetric)
        const size_t sl = (size_t)kSlices * md * slice_ld(md);
        if (slice_cols(c->ainv64 + slot * msz, md, md, c->ainv_sl + slot * sl,
                       c->ainv_ex + (size_t)slot * md, c->st) != cudaSuccess)
          return bail(fail(BH_ECUDA, "slicing of the local inverses failed"));
      }
      if (mx) {
        Af.assign(A.begin(), A.end());
        if (cudaMemcpy(c->ainv32 + slot * msz, Af.data(), msz * sizeof(float),
                       cudaMemcpyHostToDevice) != cudaSuccess)
          return bail(fail(BH_ECUDA, "upload of local inverses failed"));
      }
    }
  }
  // the uploads above are synchronous; wait only for this context's stream, not
  // for the device, so that a context created while others solve (the serving
  // form's slots) does not wait for their work
  if (cudaStreamSynchronize(c->st) != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return bail(fail(BH_ECUDA, std::string("setup: ") + cudaGetErrorString(cudaGetLastError())));
  *out = c;
  return BH_OK;
}

bh_status bh_destroy(bh_ctx* ctx) {
  if (!ctx) return fail(BH_EINVAL, "null context");
  destroy_ctx(ctx);
  return BH_OK;
}

bh_status bh_num_unknowns(const bh_ctx* ctx, int level, int64_t* n) {
  CKS(check_level(ctx, level));
  if (!n) return fail(BH_EINVAL, "null output");
  *n = ctx->lv[level].g.nd;
  return BH_OK;
}

bh_status bh_apply_A(bh_ctx* ctx, int level, const double* x, double* y) {
  CKS(check_level(ctx, level));
  if (!x || !y || x == y) return fail(BH_EINVAL, "bad vector arguments");
  Level& L = ctx->lv[level];
  CK(Ops<double>::apply(ctx->tab64, L.g, x, nullptr, y, L.ascale, kStore, ctx->scr64, ctx->st));
  ctx->n_apply++;
  return BH_OK;
}

bh_status bh_residual(bh_ctx* ctx, int level, const double* x, const double* b, double* r) {
  CKS(check_level(ctx, level));
  if (!x || !b || !r || r == x) return fail(BH_EINVAL, "bad vector arguments");
  CKS(residual_t<double>(ctx, level, x, b, r));
  ctx->n_apply++;
  return BH_OK;
}

bh_status bh_defect_compensated(bh_ctx* ctx, int level, const float* x, const double* b,
                                double* r) {
  CKS(check_level(ctx, level));
  if (!ctx->tab32)
    return fail(BH_EINVAL, "compensated defect: needs a mixed-precision context (FP32 tables)");
  if (!x || !b || !r || (const void*)r == (const void*)x)
    return fail(BH_EINVAL, "bad vector arguments");
  Level& L = ctx->lv[level];
  CK(defect_ff(ctx->tab32, L.g, x, b, r, L.ascale, ctx->scr64, ctx->st));
  ctx->n_apply++;
  return BH_OK;
}

bh_status bh_smooth(bh_ctx* ctx, int level, double* x, const double* b, int steps) {
  CKS(check_level(ctx, level));
  if (!x || !b || x == b || steps < 0) return fail(BH_EINVAL, "bad arguments");
  CKS(smooth_t<double>(ctx, level, x, b, steps, false));
  ctx->n_smooth += steps;
  return BH_OK;
}

bh_status bh_smooth_colors(bh_ctx* ctx, int level, double* x, const double* b, int first_color,
                           int end_color) {
  CKS(check_level(ctx, level));
  if (!x || !b || x == b) return fail(BH_EINVAL, "bad arguments");
  if (ctx->p.smoother != BH_MVS_COLORED)
    return fail(BH_EINVAL, "color ranges belong to the colored multiplicative smoother");
  if (first_color < 0 || end_color > ctx->ncolors() || first_color > end_color)
    return fail(BH_EINVAL, "color range outside 0.." + std::to_string(ctx->ncolors()));
  return mvs_colors_t<double>(ctx, level, x, b, first_color, end_color, false);
}

bh_status bh_prolongate_add(bh_ctx* ctx, int level, const double* xc, double* xf) {
  CKS(check_level(ctx, level));
  if (level < 2) return fail(BH_EINVAL, "prolongation needs a fine level >= 2");
  if (!xc || !xf) return fail(BH_EINVAL, "null vector");
  CK(Ops<double>::prolongate_add(ctx->tab64, ctx->lv[level].g, xc, xf, ctx->xs64[0],
                                 ctx->xs64[1], ctx->st));
  return BH_OK;
}

bh_status bh_restrict(bh_ctx* ctx, int level, const double* rf, double* bc) {
  CKS(check_level(ctx, level));
  if (level < 2) return fail(BH_EINVAL, "restriction needs a fine level >= 2");
  if (!rf || !bc) return fail(BH_EINVAL, "null vector");
  CK(Ops<double>::restrict_(ctx->tab64, ctx->lv[level].g, rf, bc, ctx->xs64[0], ctx->xs64[1],
                            ctx->st));
  return BH_OK;
}

bh_status bh_vcycle(bh_ctx* ctx, int level, double* x, const double* b) {
  CKS(check_level(ctx, level));
  if (!x || !b || x == b) return fail(BH_EINVAL, "bad vector arguments");
  ctx->n_vcycle++;
  if (!mixed(ctx)) return vcycle_t<double>(ctx, level, x, b, false);
  // FP32 V-cycle on the defect: x += MG_f32(0, b - A x)
  Level& L = ctx->lv[level];
  CKS(residual_t<double>(ctx, level, x, b, L.r64));
  CK(vec_d2f(L.b32, L.r64, L.g.nd, ctx->st));
  if (defect64(ctx))
    CK(cudaMemcpyAsync(L.db64, L.r64, L.g.nd * sizeof(double), cudaMemcpyDeviceToDevice,
                       ctx->st));
  CK(cudaMemsetAsync(L.x32, 0, L.g.nd * sizeof(float), ctx->st));
  CKS(vcycle_t<float>(ctx, level, L.x32, L.b32, true));
  CK(vec_f2d(L.r64, L.x32, L.g.nd, ctx->st));
  CK(Ops<double>::add(x, L.r64, L.g.nd, ctx->st));
  return BH_OK;
}

bh_status bh_set_tile(bh_ctx* ctx, int patches_per_block) {
  if (!ctx) return fail(BH_EINVAL, "null context");
  if (patches_per_block < 0) return fail(BH_EINVAL, "negative tile");
  ctx->tile = patches_per_block;
  return BH_OK;
}

bh_status bh_solve(bh_ctx* ctx, const double* b, double* x, double rtol, int maxit, int* iters,
                   double* relres) {
  if (!ctx || !b || !x || b == x || !iters || !relres || !(rtol > 0.0) || maxit < 1)
    return fail(BH_EINVAL, "bad arguments");
  return timed_solve(ctx, b, x, rtol, maxit, iters, relres);
}

bh_status bh_solve_guess(bh_ctx* ctx, const double* b, double* x, double rtol, int maxit,
                         int* iters, double* relres) {
  if (!ctx || !b || !x || b == x || !iters || !relres || !(rtol > 0.0) || maxit < 1)
    return fail(BH_EINVAL, "bad arguments");
  const int L = ctx->p.level;
  Level& F = ctx->lv[L];
  const int64_t n = F.g.nd;
  if (!ctx->guess) CKS(dmalloc(ctx, &ctx->guess, (size_t)(2 * n)));
  double* r0 = ctx->guess;
  double* d = ctx->guess + n;
  double bnorm, rnorm;
  CKS(norm2(ctx, b, &bnorm));
  *iters = 0;
  if (!std::isfinite(bnorm)) return fail(BH_EINVAL, "right-hand side is not finite");
  if (bnorm == 0.0) {  // the solution is zero whatever the guess
    CK(cudaMemsetAsync(x, 0, n * sizeof(double), ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    *relres = 0.0;
    return BH_OK;
  }
  // solve A d = r0 = b - A x from zero, to the tolerance that makes the
  // stopping test of a solve from zero on b: relative to ||b|| (true residual,
  // right GMRES and CG) or to ||M^-1 b|| (left GMRES)
  CKS(residual_t<double>(ctx, L, x, b, r0));
  CKS(norm2(ctx, r0, &rnorm));
  double ref_b = bnorm, ref_r = rnorm;
  const bool left = ctx->p.krylov == BH_GMRES && ctx->p.gmres_side == BH_LEFT;
  if (left) {
    CKS(precondition(ctx, b, d));
    CKS(norm2(ctx, d, &ref_b));
    CKS(precondition(ctx, r0, d));
    CKS(norm2(ctx, d, &ref_r));
  }
  if (!std::isfinite(rnorm)) return fail(BH_EINVAL, "initial guess gives a non-finite residual");
  if (ref_r <= rtol * ref_b) {  // the guess already meets the tolerance
    *relres = rnorm / bnorm;
    ctx->last_iters = 0;
    ctx->last_relres = *relres;
    ctx->last_estimate = ref_r / ref_b;
    return BH_OK;
  }
  int it = 0;
  double rr = 0.0;
  const bh_status s = timed_solve(ctx, r0, d, rtol * ref_b / ref_r, maxit, &it, &rr);
  if (s != BH_OK && s != BH_ENOCONV) return s;
  CK(vec_axpy(x, 1.0, d, n, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  *iters = it;
  *relres = rr * rnorm / bnorm;  // rr is relative to ||r0||
  ctx->last_relres = *relres;
  ctx->last_estimate *= ref_r / ref_b;  // the inner estimate is relative to ref_r
  if (s == BH_ENOCONV)
    return fail(BH_ENOCONV, "solve from the guess stopped after " + std::to_string(it) +
                                " iterations above the tolerance");
  return BH_OK;
}

bh_status bh_solve_host(bh_ctx* ctx, const double* b_host, double* x_host, double rtol,
                        int maxit, int* iters, double* relres) {
  if (!ctx || !b_host || !x_host || !iters || !relres) return fail(BH_EINVAL, "bad arguments");
  Level& F = ctx->lv[ctx->p.level];
  const size_t bytes = F.g.nd * sizeof(double);
  CK(cudaMemcpyAsync(F.b64, b_host, bytes, cudaMemcpyHostToDevice, ctx->st));
  bh_status s = timed_solve(ctx, F.b64, F.x64, rtol, maxit, iters, relres);
  if (s != BH_OK && s != BH_ENOCONV) return s;
  CK(cudaMemcpyAsync(x_host, F.x64, bytes, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return s;
}

bh_status bh_rhs(bh_ctx* ctx, int level, int kind, double* b) {
  CKS(check_level(ctx, level));
  if (!b) return fail(BH_EINVAL, "null vector");
  if (kind != BH_RHS_MANUFACTURED && kind != BH_RHS_PAPER_SINE)
    return fail(BH_EINVAL, "unknown right-hand side");
  const int d = ctx->p.dim, N = 1 << level, n = ctx->p.degree * N - 1;
  std::vector<double> F0, F2, F4, S;
  std::vector<double> coef, F;
  auto push = [&](double cf, std::initializer_list<const std::vector<double>*> fs) {
    coef.push_back(cf);
    for (auto* f : fs) F.insert(F.end(), f->begin(), f->end());
  };
  if (kind == BH_RHS_MANUFACTURED) {
    // f = Delta^2 prod sin^2: sum_a s''''_a prod s + 2 sum_{a<b} s''_a s''_b prod s
    load_1d(ctx->s, N, 0, F0);
    load_1d(ctx->s, N, 2, F2);
    load_1d(ctx->s, N, 4, F4);
    if (d == 2) {
      push(1.0, {&F4, &F0});
      push(1.0, {&F0, &F4});
      push(2.0, {&F2, &F2});
    } else {
      push(1.0, {&F4, &F0, &F0});
      push(1.0, {&F0, &F4, &F0});
      push(1.0, {&F0, &F0, &F4});
      push(2.0, {&F2, &F2, &F0});
      push(2.0, {&F2, &F0, &F2});
      push(2.0, {&F0, &F2, &F2});
    }
  } else {  // f = d^2 pi^4 prod sin(pi x_a)
    load_1d(ctx->s, N, 1, S);
    const double p4 = std::pow(M_PI, 4);
    if (d == 2)
      push(4.0 * p4, {&S, &S});
    else
      push(9.0 * p4, {&S, &S, &S});
  }
  double *dcoef = nullptr, *dF = nullptr;
  CK(cudaMalloc(&dcoef, coef.size() * sizeof(double)));
  if (cudaMalloc(&dF, F.size() * sizeof(double)) != cudaSuccess) {
    cudaFree(dcoef);
    return fail(BH_ENOMEM, "cudaMalloc failed");
  }
  cudaError_t e = cudaMemcpy(dcoef, coef.data(), coef.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(dF, F.data(), F.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = rhs_separable(d, n, (int)coef.size(), dcoef, dF, b, ctx->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
  cudaFree(dcoef);
  cudaFree(dF);
  if (e != cudaSuccess) return fail(BH_ECUDA, std::string("bh_rhs: ") + cudaGetErrorString(e));
  return BH_OK;
}

bh_status bh_stats(const bh_ctx* ctx, char* buf, size_t len) {
  if (!ctx || !buf || len == 0) return fail(BH_EINVAL, "bad arguments");
  std::snprintf(buf, len,
                "{\"dim\": %d, \"degree\": %d, \"level\": %d, \"gamma\": %.17g, \"omega\": %.17g, "
                "\"smoother\": %d, \"local_solver\": %d, \"precision\": %d, \"applies\": %lld, "
                "\"smooth_steps\": %lld, \"vcycles\": %lld, \"solves\": %lld, "
                "\"last_iters\": %d, \"last_relres\": %.17g, \"last_estimate\": %.17g, "
                "\"last_solve_ms\": %.6g, "
                "\"kernel_launches\": %lld}",
                ctx->p.dim, ctx->p.degree, ctx->p.level, ctx->p.gamma, ctx->p.omega,
                ctx->p.smoother, ctx->p.local_solver, ctx->p.precision, ctx->n_apply,
                ctx->n_smooth, ctx->n_vcycle, ctx->n_solve, ctx->last_iters, ctx->last_relres,
                ctx->last_estimate, ctx->last_solve_ms, (long long)g_kernel_launches.load());
  return BH_OK;
}

long long bh_kernel_launches(void) { return g_kernel_launches.load(); }

bh_status bh_fault_inject_alloc(long long skip, long long count) {
  if (skip < 0 || count < 0) return fail(BH_EINVAL, "bh_fault_inject_alloc: negative count");
  g_alloc_fail.store(0);
  g_alloc_skip.store(skip);
  g_alloc_fail.store(count);
  return BH_OK;
}

bh_status bh_setup_1d(int degree, double gamma, int cells, int which, double* out) {
  if (degree < 2 || degree > kMaxK || cells < 1 || which < 0 || which > 2 || !out)
    return fail(BH_EINVAL, "bad arguments");
  if (!(gamma > 0.0)) gamma = degree * (degree + 1.0);
  std::vector<double> M, L, B;
  global_1d(degree, gamma, cells, M, L, B);
  const std::vector<double>& src = which == 0 ? M : (which == 1 ? L : B);
  std::memcpy(out, src.data(), src.size() * sizeof(double));
  return BH_OK;
}

bh_status bh_setup_fdm(int degree, double gamma, int type, double* S, double* lambda) {
  if (degree < 2 || degree > kMaxK || type < 0 || type > 3 || !S || !lambda)
    return fail(BH_EINVAL, "bad arguments");
  if (!(gamma > 0.0)) gamma = degree * (degree + 1.0);
  Setup1D s;
  try {
    build_setup(degree, gamma, s);
  } catch (const std::exception& e) {
    return fail(BH_EINVAL, std::string("setup failed: ") + e.what());
  }
  const int m = 2 * degree - 1;
  std::memcpy(S, s.fdmS[type].data(), (size_t)m * m * sizeof(double));
  std::memcpy(lambda, s.fdmLam[type].data(), (size_t)m * sizeof(double));
  return BH_OK;
}

}  // extern "C"
