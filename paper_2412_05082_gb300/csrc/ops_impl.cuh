// Host launchers of the kernels in kernels.cuh: degree dispatch, grid sizing
// and the per-context tables.  Included once per value type (inst_f64.cu,
// inst_f32.cu).
#pragma once
#include <cstring>
#include <new>
#include <vector>

#include "ffsweep.cuh"
#include "kernels.cuh"
#include "mvs.cuh"
#include "mvs3.cuh"

namespace bh {

template <typename T, int K>
struct HostTables {
  Tables<T, K> t;
  MvsTab<T, K> mvs;  // operator + FDM tables for the fused MVS kernel
  CanonTab<T, K> canon;  // the interior tiles' part of mvs (batched FP32 kernel parameter)
  Tables<T, K>* dev = nullptr;  // device copy of t (batched kernels read it from memory)
  T* dinv = nullptr;  // device, 4^d slots x m^d reciprocals of the eigenvalue sums
  // FP32 tables only: the operator's class tables as hi + lo FP32 parts for the
  // compensated defect (ffsweep.cuh), host copy and device copy
  FfTab<K>* ff = nullptr;
  FfTab<K>* dev_ff = nullptr;
  int d = 0;
};

template <typename T, int K>
static void* make_tables_k(const Setup1D& s, int d) {
  auto* h = new (std::nothrow) HostTables<T, K>();
  if (!h) return nullptr;
  const int nc = 3 * K + 1, bw = 4 * K + 1, m = 2 * K - 1;
  for (int c = 0; c < nc; ++c)
    for (int t = 0; t < bw; ++t) {
      h->t.op.M[c][t] = (T)s.tabM[c * bw + t];
      h->t.op.L[c][t] = (T)s.tabL[c * bw + t];
      h->t.op.B[c][t] = (T)s.tabB[c * bw + t];
    }
  for (int ty = 0; ty < 4; ++ty) {
    for (int i = 0; i < m; ++i) {
      for (int j = 0; j < m; ++j) h->t.fdm.S[ty][i][j] = (T)s.fdmS[ty][i * m + j];
      h->t.fdm.lam[ty][i] = (T)s.fdmLam[ty][i];
    }
  }
  for (int r = 0; r < 2 * K; ++r)
    for (int q = 0; q <= K; ++q) h->t.xfer.P[r][q] = (T)s.prolong[r * (K + 1) + q];
  h->mvs.op = h->t.op;
  h->mvs.fdm = h->t.fdm;
  for (int q = 0; q < K; ++q)
    for (int t = 0; t < bw; ++t) {
      h->canon.M[q][t] = h->t.op.M[q][t];
      h->canon.L[q][t] = h->t.op.L[q][t];
      h->canon.B[q][t] = h->t.op.B[q][t];
    }
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) h->canon.S[0][i][j] = h->t.fdm.S[0][i][j];
  // reciprocal eigenvalue sums per type combination (FP64, then converted)
  int md = 1, slots = 1;
  for (int a = 0; a < d; ++a) {
    md *= m;
    slots *= 4;
  }
  std::vector<T> dinv((size_t)slots * md);
  for (int slot = 0; slot < slots; ++slot)
    for (int l = 0; l < md; ++l) {
      double sum = 0.0;
      int ll = l, ss = slot;
      for (int a = 0; a < d; ++a) {
        sum += s.fdmLam[ss % 4][ll % m];
        ll /= m;
        ss /= 4;
      }
      dinv[(size_t)slot * md + l] = (T)(1.0 / sum);
    }
  h->d = d;
  if constexpr (sizeof(T) == 4) {
    h->ff = new (std::nothrow) FfTab<K>();
    if (!h->ff) {
      delete h;
      return nullptr;
    }
    const double* src[3] = {s.tabM.data(), s.tabL.data(), s.tabB.data()};
    float(*hi[3])[4 * K + 1] = {h->ff->hi.M, h->ff->hi.L, h->ff->hi.B};
    float(*lo[3])[4 * K + 1] = {h->ff->lo.M, h->ff->lo.L, h->ff->lo.B};
    for (int o = 0; o < 3; ++o)
      for (int c = 0; c < nc; ++c)
        for (int t = 0; t < bw; ++t) {
          const double v = src[o][c * bw + t];
          const float vh = (float)v;
          hi[o][c][t] = vh;
          lo[o][c][t] = (float)(v - (double)vh);
        }
    if (cudaMalloc(&h->dev_ff, sizeof(FfTab<K>)) != cudaSuccess ||
        cudaMemcpy(h->dev_ff, h->ff, sizeof(FfTab<K>), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaFree(h->dev_ff);
      delete h->ff;
      delete h;
      return nullptr;
    }
  }
  if (cudaMalloc(&h->dev, sizeof(Tables<T, K>)) != cudaSuccess ||
      cudaMemcpy(h->dev, &h->t, sizeof(Tables<T, K>), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(h->dev);
    cudaFree(h->dev_ff);
    delete h->ff;
    delete h;
    return nullptr;
  }
  if (cudaMalloc(&h->dinv, dinv.size() * sizeof(T)) != cudaSuccess ||
      cudaMemcpy(h->dinv, dinv.data(), dinv.size() * sizeof(T), cudaMemcpyHostToDevice) !=
          cudaSuccess) {
    cudaFree(h->dinv);
    cudaFree(h->dev);
    cudaFree(h->dev_ff);
    delete h->ff;
    delete h;
    return nullptr;
  }
  return h;
}

#define BH_K_DISPATCH(k, CALL) \
  switch (k) {                 \
    case 2: CALL(2); break;    \
    case 3: CALL(3); break;    \
    case 4: CALL(4); break;    \
    case 5: CALL(5); break;    \
    case 6: CALL(6); break;    \
    case 7: CALL(7); break;    \
    default: return cudaErrorInvalidValue; \
  }

inline unsigned grid_for(int64_t threads, int block) {
  return (unsigned)((threads + block - 1) / block);
}

template <typename T>
void* Ops<T>::make_tables(const Setup1D& s, int d) {
  switch (s.k) {
    case 2: return make_tables_k<T, 2>(s, d);
    case 3: return make_tables_k<T, 3>(s, d);
    case 4: return make_tables_k<T, 4>(s, d);
    case 5: return make_tables_k<T, 5>(s, d);
    case 6: return make_tables_k<T, 6>(s, d);
    case 7: return make_tables_k<T, 7>(s, d);
  }
  return nullptr;
}

template <typename T, int K>
static void free_tables_k(void* p) {
  auto* h = static_cast<HostTables<T, K>*>(p);
  cudaFree(h->dinv);
  cudaFree(h->dev);
  cudaFree(h->dev_ff);
  delete h->ff;
  delete h;
}

template <typename T, int K>
static DevTables device_tables_k(const void* p) {
  const auto* h = static_cast<const HostTables<T, K>*>(p);
  return DevTables{h->dev, h->dinv};
}

template <typename T>
DevTables Ops<T>::device_tables(const void* p, int k) {
  switch (k) {
    case 2: return device_tables_k<T, 2>(p);
    case 3: return device_tables_k<T, 3>(p);
    case 4: return device_tables_k<T, 4>(p);
    case 5: return device_tables_k<T, 5>(p);
    case 6: return device_tables_k<T, 6>(p);
    case 7: return device_tables_k<T, 7>(p);
  }
  return DevTables{nullptr, nullptr};
}

template <typename T, int K>
static const void* host_mvs_tables_k(const void* p, size_t* bytes) {
  *bytes = sizeof(CanonTab<T, K>);
  return &static_cast<const HostTables<T, K>*>(p)->canon;
}

template <typename T>
const void* Ops<T>::host_mvs_tables(const void* p, int k, size_t* bytes) {
  switch (k) {
    case 2: return host_mvs_tables_k<T, 2>(p, bytes);
    case 3: return host_mvs_tables_k<T, 3>(p, bytes);
    case 4: return host_mvs_tables_k<T, 4>(p, bytes);
    case 5: return host_mvs_tables_k<T, 5>(p, bytes);
    case 6: return host_mvs_tables_k<T, 6>(p, bytes);
    case 7: return host_mvs_tables_k<T, 7>(p, bytes);
  }
  *bytes = 0;
  return nullptr;
}

template <typename T>
void Ops<T>::free_tables(void* p, int k) {
  if (!p) return;
  switch (k) {
    case 2: free_tables_k<T, 2>(p); break;
    case 3: free_tables_k<T, 3>(p); break;
    case 4: free_tables_k<T, 4>(p); break;
    case 5: free_tables_k<T, 5>(p); break;
    case 6: free_tables_k<T, 6>(p); break;
    case 7: free_tables_k<T, 7>(p); break;
  }
}

template <typename T, int K, int KIND>
static cudaError_t launch_sweep(const OpTab<T, K>& tab, const SweepArgs<T>& a, cudaStream_t st) {
  const int block = 128;
  sweep_kernel<T, K, KIND><<<grid_for(sweep_launch_threads(KIND, a.lines, a.N), block), block, 0,
                             st>>>(tab, a);
  g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

template <typename T, int K>
static cudaError_t apply_k(const void* tabp, const LevelGeom& g, const T* x, const T* b, T* y,
                           double scale, int mode, T* scratch, cudaStream_t st) {
  const auto& tab = static_cast<const HostTables<T, K>*>(tabp)->t.op;
  SweepArgs<T> a{};
  a.d = g.d;
  a.N = g.N;
  a.n = g.n;
  a.lines = g.nd / g.n;
  a.scale = scale;
  a.mode = mode;
  a.b = b;
  T* s[6];
  for (int i = 0; i < 6; ++i) s[i] = scratch + (int64_t)i * g.nd;
  // pass x: split into M x, L x, B x
  a.axis = 0;
  a.stride = 1;
  a.in[0] = x;
  a.out[0] = s[0];
  a.out[1] = s[1];
  a.out[2] = s[2];
  cudaError_t e = launch_sweep<T, K, 0>(tab, a, st);
  if (e != cudaSuccess) return e;
  if (g.d == 2) {
    a.axis = 1;
    a.stride = g.n;
    a.in[0] = s[0];
    a.in[1] = s[1];
    a.in[2] = s[2];
    a.out[0] = y;
    return launch_sweep<T, K, 2>(tab, a, st);
  }
  a.axis = 1;
  a.stride = g.n;
  a.in[0] = s[0];
  a.in[1] = s[1];
  a.in[2] = s[2];
  a.out[0] = s[3];
  a.out[1] = s[4];
  a.out[2] = s[5];
  e = launch_sweep<T, K, 1>(tab, a, st);
  if (e != cudaSuccess) return e;
  a.axis = 2;
  a.stride = (int64_t)g.n * g.n;
  a.in[0] = s[3];
  a.in[1] = s[4];
  a.in[2] = s[5];
  a.out[0] = y;
  return launch_sweep<T, K, 3>(tab, a, st);
}

template <typename T>
cudaError_t Ops<T>::apply(const void* tab, const LevelGeom& g, const T* x, const T* b, T* y,
                          double scale, int mode, T* scratch, cudaStream_t st) {
#define BH_CALL(KK) return apply_k<T, KK>(tab, g, x, b, y, scale, mode, scratch, st)
  BH_K_DISPATCH(g.k, BH_CALL)
#undef BH_CALL
  return cudaErrorInvalidValue;
}

template <typename T, int D, int K>
static cudaError_t patch_fdm_k(const void* tabp, const LevelGeom& g, const T* r, T* x,
                               const int* verts, int count, double scale, bool atomic,
                               cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const auto* h = static_cast<const HostTables<T, K>*>(tabp);
  PatchArgs<T> a{};
  a.r = r;
  a.x = x;
  a.verts = verts;
  a.count = count;
  a.N = g.N;
  a.n = g.n;
  a.scale = scale;
  a.dinv = h->dinv;
  constexpr int PB = PatchCfg<T, D, K>::PB;
  const unsigned grid = (unsigned)((count + PB - 1) / PB);
  if (atomic)
    patch_fdm_kernel<T, D, K, true><<<grid, 256, 0, st>>>(h->t.fdm, a);
  else
    patch_fdm_kernel<T, D, K, false><<<grid, 256, 0, st>>>(h->t.fdm, a);
  g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Ops<T>::patch_fdm(const void* tab, const LevelGeom& g, const T* r, T* x,
                              const int* verts, int count, double scale, bool atomic,
                              cudaStream_t st) {
  if (g.d == 2) {
#define BH_CALL(KK) return patch_fdm_k<T, 2, KK>(tab, g, r, x, verts, count, scale, atomic, st)
    BH_K_DISPATCH(g.k, BH_CALL)
#undef BH_CALL
  } else {
#define BH_CALL(KK) return patch_fdm_k<T, 3, KK>(tab, g, r, x, verts, count, scale, atomic, st)
    BH_K_DISPATCH(g.k, BH_CALL)
#undef BH_CALL
  }
  return cudaErrorInvalidValue;
}

// Patches per block of the fused MVS kernels at which one smoothing step (FP64)
// or one V-cycle (FP32) at the paper's sizes (2D: 512^2 cells for k <= 4, 256^2
// above; 3D: 128^3 for k <= 3, 64^3 above) ran fastest on GB300; the automatic
// choice is min(ceil(count / (2 * 152)), this, the shared-memory limit), so
// levels with few patches still spread over the SMs (0: no cap).  In FP32 the
// 3D kernel's shared memory, not its FMAs, sets the pace: smaller tiles leave
// room for more blocks per SM.
constexpr int kMvs2TileF64[8] = {0, 0, 32, 18, 12, 14, 6, 8};
constexpr int kMvs3TileF64[8] = {0, 0, 12, 16, 16, 16, 16, 16};
constexpr int kMvs2TileF32[8] = {0, 0, 0, 0, 0, 0, 0, 0};
constexpr int kMvs3TileF32[8] = {0, 0, 12, 8, 4, 3, 0, 0};

template <typename T>
inline int auto_tile(int count, int pref_f64, int pref_f32) {
  int pb = (count + 2 * 152 - 1) / (2 * 152);
  const int pref = sizeof(T) == 8 ? pref_f64 : pref_f32;
  if (pref > 0 && pb > pref) pb = pref;
  return pb;
}

template <typename T, int K>
static cudaError_t mvs_color_k(const void* tabp, const LevelGeom& g, T* x, const T* b,
                               const int* verts, int count, double ascale, double pscale,
                               int pb_req, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const auto* h = static_cast<const HostTables<T, K>*>(tabp);
  MvsArgs<T> a{};
  a.x = x;
  a.b = b;
  a.verts = verts;
  a.count = count;
  a.N = g.N;
  a.n = g.n;
  a.ascale = ascale;
  a.pscale = pscale;
  a.dinv = h->dinv;
  a.dtab = h->dev;
  using C = Mvs2Cfg<T, K>;
  // patches per block: enough blocks for two waves on 152 SMs, at most PB_MAX
  int pb = pb_req > 0 ? pb_req : auto_tile<T>(count, kMvs2TileF64[K], kMvs2TileF32[K]);
  pb = pb < 1 ? 1 : (pb > C::PB_MAX ? C::PB_MAX : pb);
  a.pb = pb;
  // opt in to the dynamic shared memory once per instantiation (thread-safe static init)
  static const cudaError_t attr = cudaFuncSetAttribute(
      mvs2_color_kernel<T, K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
      (int)C::smem_bytes(C::PB_MAX));
  if (attr != cudaSuccess) return attr;
  mvs2_color_kernel<T, K><<<(unsigned)((count + pb - 1) / pb), 256, C::smem_bytes(pb), st>>>(
      h->mvs, a);
  g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

template <typename T, int K>
static cudaError_t mvs3_color_k(const void* tabp, const LevelGeom& g, T* x, const T* b,
                                const int* verts, int count, double ascale, double pscale,
                                int pb_req, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const auto* h = static_cast<const HostTables<T, K>*>(tabp);
  MvsArgs<T> a{};
  a.x = x;
  a.b = b;
  a.verts = verts;
  a.count = count;
  a.N = g.N;
  a.n = g.n;
  a.ascale = ascale;
  a.pscale = pscale;
  a.dinv = h->dinv;
  a.dtab = h->dev;
  using C = Mvs3Cfg<T, K>;
  int pb = pb_req > 0 ? pb_req : auto_tile<T>(count, kMvs3TileF64[K], kMvs3TileF32[K]);
  pb = pb < 1 ? 1 : (pb > C::PB_MAX ? C::PB_MAX : pb);
  a.pb = pb;
  static const cudaError_t attr = cudaFuncSetAttribute(
      mvs3_color_kernel<T, K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
      (int)C::smem_bytes(C::PB_MAX));
  if (attr != cudaSuccess) return attr;
  mvs3_color_kernel<T, K><<<(unsigned)((count + pb - 1) / pb), C::THREADS, C::smem_bytes(pb), st>>>(
      h->mvs, a);
  g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Ops<T>::mvs_color(const void* tab, const LevelGeom& g, T* x, const T* b,
                              const int* verts, int count, double ascale, double pscale, int pb,
                              cudaStream_t st) {
  if (g.d == 2) {
#define BH_CALL(KK) return mvs_color_k<T, KK>(tab, g, x, b, verts, count, ascale, pscale, pb, st)
    BH_K_DISPATCH(g.k, BH_CALL)
#undef BH_CALL
  } else {
#define BH_CALL(KK) \
  return mvs3_color_k<T, KK>(tab, g, x, b, verts, count, ascale, pscale, pb, st)
    BH_K_DISPATCH(g.k, BH_CALL)
#undef BH_CALL
  }
  return cudaErrorInvalidValue;
}

template <typename T, int D, int K>
static cudaError_t patch_exact_k(const LevelGeom& g, const T* ainv, const T* r, T* x,
                                 const int* verts, int count, double scale, bool atomic,
                                 cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  PatchArgs<T> a{};
  a.r = r;
  a.x = x;
  a.verts = verts;
  a.count = count;
  a.N = g.N;
  a.n = g.n;
  a.scale = scale;
  a.ainv = ainv;
  constexpr int PB = PatchCfg<T, D, K>::PB;
  const unsigned grid = (unsigned)((count + PB - 1) / PB);
  if (atomic)
    patch_exact_kernel<T, D, K, true><<<grid, 256, 0, st>>>(a);
  else
    patch_exact_kernel<T, D, K, false><<<grid, 256, 0, st>>>(a);
  g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Ops<T>::patch_exact(const LevelGeom& g, const T* Ainv, const T* r, T* x,
                                const int* verts, int count, double scale, bool atomic,
                                cudaStream_t st) {
  if (g.d == 2) {
#define BH_CALL(KK) return patch_exact_k<T, 2, KK>(g, Ainv, r, x, verts, count, scale, atomic, st)
    BH_K_DISPATCH(g.k, BH_CALL)
#undef BH_CALL
  } else {
#define BH_CALL(KK) return patch_exact_k<T, 3, KK>(g, Ainv, r, x, verts, count, scale, atomic, st)
    BH_K_DISPATCH(g.k, BH_CALL)
#undef BH_CALL
  }
  return cudaErrorInvalidValue;
}

template <typename T, int D, int K>
static cudaError_t patch_gather_k(const LevelGeom& g, const T* r, const int* verts, int count,
                                  T* R, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const int64_t tot = (int64_t)count * PatchCfg<T, D, K>::MD;
  patch_gather_kernel<T, D, K><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(r, verts, count,
                                                                            g.N, g.n, R);
  g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

template <typename T, int D, int K>
static cudaError_t patch_scatter_k(const LevelGeom& g, const T* Y, const int* verts, int count,
                                   T* x, bool atomic, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const int64_t tot = (int64_t)count * PatchCfg<T, D, K>::MD;
  const unsigned grid = (unsigned)((tot + 255) / 256);
  if (atomic)
    patch_scatter_kernel<T, D, K, true><<<grid, 256, 0, st>>>(Y, verts, count, g.N, g.n, x);
  else
    patch_scatter_kernel<T, D, K, false><<<grid, 256, 0, st>>>(Y, verts, count, g.N, g.n, x);
  g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Ops<T>::patch_gather(const LevelGeom& g, const T* r, const int* verts, int count,
                                 T* R, cudaStream_t st) {
  if (g.d == 2) {
#define BH_CALL(KK) return patch_gather_k<T, 2, KK>(g, r, verts, count, R, st)
    BH_K_DISPATCH(g.k, BH_CALL)
#undef BH_CALL
  } else {
#define BH_CALL(KK) return patch_gather_k<T, 3, KK>(g, r, verts, count, R, st)
    BH_K_DISPATCH(g.k, BH_CALL)
#undef BH_CALL
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t Ops<T>::patch_scatter(const LevelGeom& g, const T* Y, const int* verts, int count,
                                  T* x, bool atomic, cudaStream_t st) {
  if (g.d == 2) {
#define BH_CALL(KK) return patch_scatter_k<T, 2, KK>(g, Y, verts, count, x, atomic, st)
    BH_K_DISPATCH(g.k, BH_CALL)
#undef BH_CALL
  } else {
#define BH_CALL(KK) return patch_scatter_k<T, 3, KK>(g, Y, verts, count, x, atomic, st)
    BH_K_DISPATCH(g.k, BH_CALL)
#undef BH_CALL
  }
  return cudaErrorInvalidValue;
}

// one transfer pass along `axis`; shapes per axis given for input and output
template <typename T, int K, bool PROLONG>
static cudaError_t xfer_pass(const XferTab<T, K>& tab, int d, int axis, const int* din,
                             const int* dout, int Nc, int nc, int nf, const T* in, T* out,
                             bool add, cudaStream_t st, float* out32 = nullptr) {
  XferArgs<T> a{};
  a.in = in;
  a.out = out;
  a.out32 = out32;
  a.d = d;
  a.axis = axis;
  a.Nc = Nc;
  a.nc = nc;
  a.nf = nf;
  a.add = add;
  int64_t si = 1, so = 1, lines = 1;
  for (int i = 0; i < 3; ++i) {
    a.dims_in[i] = i < d ? din[i] : 1;
    a.dims_out[i] = i < d ? dout[i] : 1;
    a.str_in[i] = si;
    a.str_out[i] = so;
    si *= a.dims_in[i];
    so *= a.dims_out[i];
    if (i < d && i != axis) lines *= din[i];
  }
  a.lines = lines;
  const int block = 128;
  if (PROLONG)
    prolong_kernel<T, K><<<grid_for(lines * Nc, block), block, 0, st>>>(tab, a);
  else
    restrict_kernel<T, K><<<grid_for(lines * Nc, block), block, 0, st>>>(tab, a);
  g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

template <typename T, int K, bool PROLONG>
static cudaError_t transfer_k(const void* tabp, const LevelGeom& fine, const T* in, T* out,
                              T* s0, T* s1, cudaStream_t st, float* out32 = nullptr) {
  const auto& tab = static_cast<const HostTables<T, K>*>(tabp)->t.xfer;
  const int d = fine.d, Nc = fine.N / 2, nc = K * Nc - 1, nf = fine.n;
  int dims[3];
  for (int i = 0; i < 3; ++i) dims[i] = PROLONG ? nc : nf;
  const T* src = in;
  T* bufs[2] = {s0, s1};
  for (int axis = 0; axis < d; ++axis) {
    int dn[3] = {dims[0], dims[1], dims[2]};
    dn[axis] = PROLONG ? nf : nc;
    const bool last = axis == d - 1;
    T* dst = last ? out : bufs[axis % 2];
    cudaError_t e =
        xfer_pass<T, K, PROLONG>(tab, d, axis, dims, dn, Nc, nc, nf, src, dst, PROLONG && last, st,
                                 last ? out32 : nullptr);
    if (e != cudaSuccess) return e;
    for (int i = 0; i < 3; ++i) dims[i] = dn[i];
    src = dst;
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t Ops<T>::prolongate_add(const void* tab, const LevelGeom& fine, const T* xc, T* xf,
                                   T* s0, T* s1, cudaStream_t st) {
#define BH_CALL(KK) return transfer_k<T, KK, true>(tab, fine, xc, xf, s0, s1, st)
  BH_K_DISPATCH(fine.k, BH_CALL)
#undef BH_CALL
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t Ops<T>::restrict_(const void* tab, const LevelGeom& fine, const T* rf, T* bc, T* s0,
                              T* s1, cudaStream_t st, float* bc32) {
#define BH_CALL(KK) return transfer_k<T, KK, false>(tab, fine, rf, bc, s0, s1, st, bc32)
  BH_K_DISPATCH(fine.k, BH_CALL)
#undef BH_CALL
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t Ops<T>::add(T* y, const T* x, int64_t n, cudaStream_t st) {
  int64_t g = (n + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  add_kernel<T><<<(unsigned)(g < 1 ? 1 : g), 256, 0, st>>>(y, x, n);
  g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

template <typename T>
cudaError_t Ops<T>::dense_symv(int n, const double* A, const T* in, T* out, double scale,
                               cudaStream_t st) {
  dense_symv_kernel<T><<<grid_for(n, 128), 128, 0, st>>>(n, A, in, out, scale);
  g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

}  // namespace bh
