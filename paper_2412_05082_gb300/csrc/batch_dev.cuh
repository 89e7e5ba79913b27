// Device side of the batched form (batch.cu): the per-problem metadata, the
// work-list kernels of the level operations, the per-degree colored-MVS
// kernels and the persistent V-cycle kernel.  Shared by batch.cu (host side
// and the light kernels) and the translation units that instantiate the
// heavy kernels (batch_mvs_*.cu, batch_pers_*.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "ops_impl.cuh"

namespace bh {
namespace bdev {

// ---------------------------------------------------------------------------
// device side
// ---------------------------------------------------------------------------
struct Meta {                 // per problem, indexed by problem id
  const int* k;               // degree
  const void* const* tabs;    // Tables<T, K>* (device) of the launch's value type
  const int* active;          // 0: problem finished, skip it
};

#define BH_KSWITCH(k, CALL) \
  switch (k) {              \
    case 2: CALL(2); break; \
    case 3: CALL(3); break; \
    case 4: CALL(4); break; \
    case 5: CALL(5); break; \
    case 6: CALL(6); break; \
    case 7: CALL(7); break; \
  }

// Every problem's range holds sweep_launch_threads(KIND, ...) threads, whole
// blocks, so that a block of the split (KIND 0, in tiles) works on one problem.
template <typename T, int KIND>
__global__ void __launch_bounds__(128) sweep_batch_kernel(Meta m, const SweepArgs<T>* args,
                                                          const int64_t* prefix, const int* pid,
                                                          int n) {
  if constexpr (KIND == 0) {
    __shared__ T sx[kSplitTileLines * SplitTile<kMaxK>::RS];
    const int64_t bstart = (int64_t)blockIdx.x * blockDim.x;
    if (bstart >= prefix[n]) return;
    const int s = find_seg(prefix, n, bstart);  // the same for the whole block
    const int p = pid[s];
    if (!m.active[p]) return;
    const int64_t blk = (bstart - prefix[s]) / kSplitBlock;
#define BH_CALL(KK) \
  sweep_split_tile<T, KK>(static_cast<const Tables<T, KK>*>(m.tabs[p])->op, args[s], blk, sx)
    BH_KSWITCH(m.k[p], BH_CALL)
#undef BH_CALL
  } else {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= prefix[n]) return;
    const int s = find_seg(prefix, n, tid);
    const int p = pid[s];
    if (!m.active[p]) return;
    const int64_t local = tid - prefix[s];
    if (local >= args[s].lines * args[s].N) return;  // padding of the range
#define BH_CALL(KK) \
  sweep_thread<T, KK, KIND>(static_cast<const Tables<T, KK>*>(m.tabs[p])->op, args[s], local)
    BH_KSWITCH(m.k[p], BH_CALL)
#undef BH_CALL
  }
}

template <typename T, bool PROLONG>
__global__ void __launch_bounds__(128) xfer_batch_kernel(Meta m, const XferArgs<T>* args,
                                                         const int64_t* prefix, const int* pid,
                                                         int n) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= prefix[n]) return;
  const int s = find_seg(prefix, n, tid);
  const int p = pid[s];
  if (!m.active[p]) return;
  const int64_t local = tid - prefix[s];
#define BH_CALL(KK)                                                                          \
  if (PROLONG)                                                                               \
    prolong_thread<T, KK>(static_cast<const Tables<T, KK>*>(m.tabs[p])->xfer, args[s], local); \
  else                                                                                       \
    restrict_thread<T, KK>(static_cast<const Tables<T, KK>*>(m.tabs[p])->xfer, args[s], local)
  BH_KSWITCH(m.k[p], BH_CALL)
#undef BH_CALL
}

struct Tile {
  int s;      // index into the op's problem list
  int first;  // first patch of the color list
  int count;
};

// Degrees whose interior tiles take the folded path inside the persistent
// kernel, which dispatches on the degree at run time and so has the register
// count of the largest tile code it holds (128, capped for two blocks per SM).
// The per-degree kernels of the graph form take it for every degree.
constexpr int kBatchInteriorMaxK = 4;

// The FP32 launches' kernel parameter: the interior tiles' tables, read as
// constant-bank operands (FP64 reads every table from device memory through
// shared memory, and takes no parameter table).
template <typename T, int K>
struct BatchCoef {
  CanonTab<T, K> c;
};
template <int K>
struct BatchCoef<double, K> {
  int unused;
};

// One color of the colored MVS for the tiles of one degree K: one block per
// tile (any grid size).  One instantiation per degree, so that each has the
// register count of its own tile code.  In FP32 every problem of a launch has
// the same interior tables (one degree and penalty), passed as the parameter.
template <typename T, int K>
__global__ void __launch_bounds__(256) mvs2_batch_kernel(Meta m, const MvsArgs<T>* args,
                                                         const int* pid, const Tile* tiles,
                                                         int ntiles,
                                                         const __grid_constant__ BatchCoef<T, K> bc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    __syncthreads();  // the previous tile's last stage still reads shared memory
    const Tile tl = tiles[t];
    const int p = pid[tl.s];
    if (!m.active[p]) continue;
    const auto* tb = static_cast<const Tables<T, K>*>(m.tabs[p]);
    if (mvs2_tile_is_interior(args[tl.s], tl.first, tl.count)) {
      if constexpr (sizeof(T) == 4)
        mvs2_tile_interior<T, K, true>(bc.c, bc.c, args[tl.s], tl.first, tl.count, smem_raw);
      else
        mvs2_tile_interior<T, K>(tb->op, tb->fdm, args[tl.s], tl.first, tl.count, smem_raw);
    } else {
      mvs2_tile<T, K>(tb->op, tb->fdm, args[tl.s], tl.first, tl.count, smem_raw);
    }
  }
}

// the kernels by degree, as the address the runtime API takes; defined in
// batch_mvs_f64.cu / batch_mvs_f32.cu and batch_pers_f64.cu / batch_pers_f32.cu
// (one translation unit each, compiled in parallel)
const void* mvs2_batch_kernel_f64(int k);
const void* mvs2_batch_kernel_f32(int k);
const void* vcycle_persistent_kernel_f64();
const void* vcycle_persistent_kernel_f32();
template <typename T>
inline const void* mvs2_batch_kernel_for(int k) {
  return sizeof(T) == 8 ? mvs2_batch_kernel_f64(k) : mvs2_batch_kernel_f32(k);
}
template <typename T>
inline const void* vcycle_persistent_kernel_for() {
  return sizeof(T) == 8 ? vcycle_persistent_kernel_f64() : vcycle_persistent_kernel_f32();
}

template <typename T>
inline const void* mvs2_batch_kernel_table(int k) {
  switch (k) {
    case 2: return (const void*)mvs2_batch_kernel<T, 2>;
    case 3: return (const void*)mvs2_batch_kernel<T, 3>;
    case 4: return (const void*)mvs2_batch_kernel<T, 4>;
    case 5: return (const void*)mvs2_batch_kernel<T, 5>;
    case 6: return (const void*)mvs2_batch_kernel<T, 6>;
    case 7: return (const void*)mvs2_batch_kernel<T, 7>;
  }
  return nullptr;
}

template <typename T>
struct Symv {  // coarse solve x = scale A b, A dense symmetric FP64 (n x n)
  const double* A;
  const T* b;
  T* x;
  int n;
  double scale;
};

template <typename T>
__global__ void coarse_batch_kernel(Meta m, const Symv<T>* ops, const int* pid, int count) {
  const int s = blockIdx.y;
  if (s >= count || !m.active[pid[s]]) return;
  const Symv<T> o = ops[s];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= o.n) return;
  double acc = 0.0;
  for (int j = 0; j < o.n; ++j) acc = fma(o.A[(int64_t)j * o.n + i], (double)o.b[j], acc);
  o.x[i] = (T)(o.scale * acc);
}

template <typename T>
struct Vec {  // one problem's vector operands: y + yslot * ys, x + xslot * xs, n values
  T* y;
  const T* x;
  int64_t n;
  int64_t ys, xs;
};

// zero, copy, y += c x, y = x / sqrt(c): one launch over the concatenation
enum VecOp { kZero = 0, kCopy = 1, kAxpyDev = 2, kScaleInvSqrt = 3 };

template <typename T>
__global__ void vec_batch_kernel(Meta m, const Vec<T>* v, const int64_t* prefix, const int* pid,
                                 int n, int op, const double* coef, int cstride, int cslot,
                                 double sign, int yslot, int xslot) {
  const int64_t total = prefix[n];
  for (int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; tid < total;
       tid += (int64_t)gridDim.x * blockDim.x) {
    const int s = find_seg(prefix, n, tid);
    const int p = pid[s];
    if (!m.active[p]) continue;
    const int64_t i = tid - prefix[s];
    const Vec<T> o = v[s];
    T* y = o.y + yslot * o.ys;
    const T* x = o.x + xslot * o.xs;
    switch (op) {
      case kZero: y[i] = T(0); break;
      case kCopy: y[i] = x[i]; break;
      case kAxpyDev: y[i] = T(fma(sign * coef[p * cstride + cslot], (double)x[i], (double)y[i])); break;
      default: y[i] = T((double)x[i] / sqrt(coef[p * cstride + cslot])); break;
    }
  }
}

// conversion between an FP64 vector (d + slot * ds) and an FP32 one
struct Conv {
  double* d;
  float* f;
  int64_t n;
  int64_t ds;
};
enum ConvDir { kD2F = 0, kF2D = 1 };

// ---------------------------------------------------------------------------
// persistent form: the whole V-cycle in one cooperative launch
// ---------------------------------------------------------------------------
// The V-cycle's level operations become phases of one kernel: every block
// walks the phase list; inside a phase the blocks share its work list (tiles
// of the patch kernel, threads of the sweeps, transfers, vector operations and
// the coarse solve); a grid barrier separates the phases.
enum PhaseKind : int {
  kPhMvs = 0,      // colored-MVS tiles (value type of the V-cycle)
  kPhSweep0 = 1,   // FP64 x-split sweep
  kPhSweep2 = 2,   // FP64 y-combination (residual)
  kPhRestr = 3,    // FP64 restriction pass
  kPhProl = 4,     // prolongation pass (value type of the V-cycle)
  kPhZero = 5,     // zero vectors (value type of the V-cycle)
  kPhCoarse = 6,   // coarse solve (value type of the V-cycle)
  kPhConv = 7      // FP64 <-> FP32 conversions
};

struct MvsGroup {  // the tiles of one degree in an MVS phase
  const void* args;  // MvsArgs<T>[]
  const int* pid;
  const Tile* tiles;
  int ntiles;
};

struct Phase {
  int kind;
  int n;              // entries of the work list
  int64_t total;      // items: threads, or tiles (MVS), or (problem, row) pairs (coarse)
  const void* args;   // SweepArgs / XferArgs / Vec / Conv / Symv entries
  const int64_t* prefix;
  const int* pid;
  int dir;            // conversion direction
  int maxn;           // coarse: largest coarse size
  int ngroups;        // MVS: degree groups
  MvsGroup groups[kMaxK + 1];
};

// Grid barrier with a bounded wait: thread 0 of every block arrives on a
// counter; the last one to arrive resets it and advances the generation, the
// others spin on the generation for at most `budget` clock cycles.  A wait
// that runs out sets *status (1) and every block leaves the kernel at its next
// barrier, so a barrier that can never complete (fewer co-resident blocks than
// `expected`) ends the kernel with an error status instead of a hang.
__device__ __forceinline__ bool grid_barrier(unsigned* count, unsigned* gen, unsigned expected,
                                             int* status, long long budget) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned* vgen = gen;
    volatile int* vstatus = status;
    const unsigned g = *vgen;
    __threadfence();  // this block's writes of the phase before its arrival
    if (atomicAdd(count, 1u) == expected - 1) {
      atomicExch(count, 0u);
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      const long long t0 = clock64();
      while (*vgen == g) {
        if (*vstatus != 0 || clock64() - t0 > budget) {
          atomicExch(status, 1);
          ok = 0;
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

template <typename T>
__global__ void __launch_bounds__(256, 2) vcycle_persistent_kernel(
    Meta m64, Meta mT, const Phase* __restrict__ phases, int nphases, unsigned* bar,
    unsigned expected, int* status, long long budget) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
  for (int f = 0; f < nphases; ++f) {
    const Phase& P = phases[f];
    const int kind = P.kind;
    if (kind == kPhSweep0 || kind == kPhSweep2) {
      const SweepArgs<double>* args = static_cast<const SweepArgs<double>*>(P.args);
      for (int64_t tid = gtid; tid < P.total; tid += gthreads) {
        const int s = find_seg(P.prefix, P.n, tid);
        const int p = P.pid[s];
        if (!m64.active[p]) continue;
        const int64_t local = tid - P.prefix[s];
        if (local >= args[s].lines * args[s].N) continue;  // padding of the range
#define BH_CALL(KK)                                                                              \
  if (kind == kPhSweep0)                                                                         \
    sweep_thread<double, KK, 0, true>(static_cast<const Tables<double, KK>*>(m64.tabs[p])->op,    \
                                      args[s], local);                                           \
  else                                                                                           \
    sweep_thread<double, KK, 2, true>(static_cast<const Tables<double, KK>*>(m64.tabs[p])->op,    \
                                      args[s], local)
        BH_KSWITCH(m64.k[p], BH_CALL)
#undef BH_CALL
      }
    } else if (kind == kPhRestr) {
      const XferArgs<double>* args = static_cast<const XferArgs<double>*>(P.args);
      for (int64_t tid = gtid; tid < P.total; tid += gthreads) {
        const int s = find_seg(P.prefix, P.n, tid);
        const int p = P.pid[s];
        if (!m64.active[p]) continue;
        const int64_t local = tid - P.prefix[s];
#define BH_CALL(KK) \
  restrict_thread<double, KK>(static_cast<const Tables<double, KK>*>(m64.tabs[p])->xfer, args[s], local)
        BH_KSWITCH(m64.k[p], BH_CALL)
#undef BH_CALL
      }
    } else if (kind == kPhProl) {
      const XferArgs<T>* args = static_cast<const XferArgs<T>*>(P.args);
      for (int64_t tid = gtid; tid < P.total; tid += gthreads) {
        const int s = find_seg(P.prefix, P.n, tid);
        const int p = P.pid[s];
        if (!mT.active[p]) continue;
        const int64_t local = tid - P.prefix[s];
#define BH_CALL(KK) \
  prolong_thread<T, KK>(static_cast<const Tables<T, KK>*>(mT.tabs[p])->xfer, args[s], local)
        BH_KSWITCH(mT.k[p], BH_CALL)
#undef BH_CALL
      }
    } else if (kind == kPhZero) {
      const Vec<T>* v = static_cast<const Vec<T>*>(P.args);
      for (int64_t tid = gtid; tid < P.total; tid += gthreads) {
        const int s = find_seg(P.prefix, P.n, tid);
        if (!mT.active[P.pid[s]]) continue;
        v[s].y[tid - P.prefix[s]] = T(0);
      }
    } else if (kind == kPhConv) {
      const Conv* v = static_cast<const Conv*>(P.args);
      for (int64_t tid = gtid; tid < P.total; tid += gthreads) {
        const int s = find_seg(P.prefix, P.n, tid);
        if (!m64.active[P.pid[s]]) continue;
        const int64_t i = tid - P.prefix[s];
        if (P.dir == kD2F)
          v[s].f[i] = (float)v[s].d[i];
        else
          v[s].d[i] = (double)v[s].f[i];
      }
    } else if (kind == kPhCoarse) {
      const Symv<T>* ops = static_cast<const Symv<T>*>(P.args);
      for (int64_t it = gtid; it < P.total; it += gthreads) {
        const int s = (int)(it / P.maxn), i = (int)(it - (int64_t)s * P.maxn);
        const Symv<T> o = ops[s];
        if (i >= o.n || !mT.active[P.pid[s]]) continue;
        double acc = 0.0;
        for (int j = 0; j < o.n; ++j) acc = fma(o.A[(int64_t)j * o.n + i], (double)o.b[j], acc);
        o.x[i] = (T)(o.scale * acc);
      }
    } else {  // kPhMvs: one tile per block at a time, the degree groups one after another
      for (int64_t t = blockIdx.x; t < P.total; t += gridDim.x) {
        int g = 0;
        int64_t tl = t;
        while (g + 1 < P.ngroups && tl >= P.groups[g].ntiles) tl -= P.groups[g++].ntiles;
        const MvsGroup G = P.groups[g];
        const Tile tile = G.tiles[tl];
        const MvsArgs<T>* args = static_cast<const MvsArgs<T>*>(G.args);
        const int p = G.pid[tile.s];
        __syncthreads();  // the previous tile's last stage still reads shared memory
        if (!mT.active[p]) continue;
#define BH_CALL(KK)                                                                           \
  {                                                                                           \
    const auto* tb = static_cast<const Tables<T, KK>*>(mT.tabs[p]);                           \
    if (KK <= kBatchInteriorMaxK && mvs2_tile_is_interior(args[tile.s], tile.first, tile.count)) \
      mvs2_tile_interior<T, KK>(tb->op, tb->fdm, args[tile.s], tile.first, tile.count, smem_raw); \
    else                                                                                      \
      mvs2_tile<T, KK>(tb->op, tb->fdm, args[tile.s], tile.first, tile.count, smem_raw);       \
  }
        BH_KSWITCH(mT.k[p], BH_CALL)
#undef BH_CALL
      }
    }
    if (f + 1 < nphases && !grid_barrier(bar, bar + 1, expected, status, budget)) return;
  }
}

// the persistent kernel's address for the runtime API
template <typename T>
inline const void* vcycle_persistent_kernel_table() {
  return (const void*)vcycle_persistent_kernel<T>;
}

}  // namespace bdev
}  // namespace bh
