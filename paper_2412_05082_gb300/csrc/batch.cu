// Batched form: many independent 2D problems (different degrees and levels)
// solved together.  Every level operation of the V-cycle processes all
// problems in ONE launch: the launch walks a precomputed work list of
// (problem, range) entries and dispatches on the problem's degree.  The
// smoother's patch work of one color is one launch per degree present (one
// block per tile, each launch with the shared memory of its own tile shape),
// the launches forked into parallel branches of the graph; the tile shape
// (patches per block) of each degree comes from the autotuner.  The V-cycle
// runs in lockstep by depth (depth t works on level L_p - t of every problem
// p) and is captured once as a CUDA graph that maps b_L to x_L = MG(0, b_L)
// for every problem.  It runs in FP64, or in FP32 with the defect before each
// restriction evaluated and restricted in FP64 (BH_MIXED_FP32_R64).  GMRES(m)
// runs in lockstep with a per-problem activity mask and one host
// synchronization per iteration for all problems: left preconditioning
// (preconditioned residual, the paper's tables), or right preconditioning in
// the flexible form (true residual b - A x, required by the FP32 V-cycle),
// with restarts.  Every problem follows exactly the arithmetic of its own
// context, so a result does not depend on the other problems of the batch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "biharm.h"
#include "ctx.h"
#include "ops_impl.cuh"

#include <cuda_runtime_api.h>

namespace bh {
void set_last_error(const std::string& msg);  // api.cu
bool alloc_fault();                           // api.cu: host-side fault injection
}

using namespace bh;

namespace {

bh_status berr(bh_status s, const std::string& msg) {
  set_last_error(msg);
  return s;
}

#define BCK(call)                                                                       \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return berr(BH_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));        \
  } while (0)

#define BCKS(call)              \
  do {                          \
    bh_status s_ = (call);      \
    if (s_ != BH_OK) return s_; \
  } while (0)

}  // namespace

#include "batch_dev.cuh"

using namespace bh::bdev;

namespace {

__global__ void conv_batch_kernel(Meta m, const Conv* v, const int64_t* prefix, const int* pid,
                                  int n, int dir, int slot) {
  const int64_t total = prefix[n];
  for (int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; tid < total;
       tid += (int64_t)gridDim.x * blockDim.x) {
    const int s = find_seg(prefix, n, tid);
    if (!m.active[pid[s]]) continue;
    const int64_t i = tid - prefix[s];
    const Conv o = v[s];
    double* d = o.d + slot * o.ds;
    if (dir == kD2F)
      o.f[i] = (float)d[i];
    else
      d[i] = (double)o.f[i];
  }
}

// deterministic per-problem dot products: fixed chunks, then a fixed-order sum
constexpr int kChunk = 8192;

__global__ void dot_batch_partial(Meta m, const Vec<double>* v, const int64_t* cprefix,
                                  const int* pid, int n, double* partials, int yslot, int xslot) {
  const int64_t c = blockIdx.x;
  if (c >= cprefix[n]) return;
  const int s = find_seg(cprefix, n, c);
  const int p = pid[s];
  double acc = 0.0;
  if (m.active[p]) {
    const Vec<double> o = v[s];
    const double* y = o.y + yslot * o.ys;
    const double* x = o.x + xslot * o.xs;
    const int64_t i0 = (c - cprefix[s]) * kChunk;
    const int64_t i1 = min(o.n, i0 + kChunk);
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) acc = fma(y[i], x[i], acc);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  __shared__ double ws[8];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
    partials[c] = t;
  }
}

__global__ void dot_batch_final(const int64_t* cprefix, const int* pid, int n,
                                const double* partials, double* out, int cstride, int cslot) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  double t = 0.0;
  for (int64_t c = cprefix[s]; c < cprefix[s + 1]; ++c) t += partials[c];
  out[pid[s] * cstride + cslot] = t;
}

}  // namespace

namespace {

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <typename A>
struct DevArray {  // a device copy of a host vector
  A* d = nullptr;
  int n = 0;
};

template <typename T>
struct SweepOp {  // one batched sweep launch
  DevArray<SweepArgs<T>> args;
  DevArray<int64_t> prefix;
  DevArray<int> pid;
  int64_t total = 0;
};

struct FfOp {  // one batched compensated-defect sweep launch (problems of one degree)
  DevArray<FfSweepArgs> args;
  DevArray<int64_t> prefix;
  DevArray<int> pid;
  int64_t total = 0;
  int k = 0;
};

template <typename T>
struct XferOp {
  DevArray<XferArgs<T>> args;
  DevArray<int64_t> prefix;
  DevArray<int> pid;
  int64_t total = 0;
};

template <typename T>
struct MvsOp {
  DevArray<MvsArgs<T>> args;
  DevArray<int> pid;
  DevArray<Tile> tiles;
  size_t smem = 0;
  int k = 0;                  // the degree of every problem of the op
  const void* htab = nullptr;  // FP32: their common CanonTab<float, k> (host copy; the kernel
                               // parameter); FP64: a placeholder for the unused parameter
};

template <typename T>
struct VecOpList {
  DevArray<Vec<T>> v;
  DevArray<int64_t> prefix;   // element prefix
  DevArray<int64_t> cprefix;  // chunk prefix (dots)
  DevArray<int> pid;
  int64_t total = 0, chunks = 0;
};

struct ConvOpList {
  DevArray<Conv> v;
  DevArray<int64_t> prefix;
  DevArray<int> pid;
  int64_t total = 0;
};

// the operations of the V-cycle's own value type T at one depth
template <typename T>
struct VDepth {
  // per color, one MVS launch per degree present at this depth (each with the
  // shared memory its own tile needs); they run as parallel graph branches
  std::vector<MvsOp<T>> mvs[8];
  XferOp<T> prol[2];
  VecOpList<T> zero_coarse;  // x at level - 1
  DevArray<Symv<T>> symv;
};

struct Depth {  // operations at depth t of the lockstep V-cycle
  bool smooth = false, coarse = false;
  VDepth<double> v64;  // FP64 V-cycle
  VDepth<float> v32;   // FP32 V-cycle (BH_MIXED_FP32_R64)
  // the defect b_l - A_l x before the restriction, always in FP64: of x64
  // against b64 (FP64), or of the FP64 copy dx64 of x32 against the FP64
  // right-hand side (b64 on the finest level, db64 below) (R64)
  SweepOp<double> res_x, res_y;
  XferOp<double> restr[2];  // FP64 restriction into b64 (FP64) / db64 (R64) of level l-1
  ConvOpList x_f2d;         // R64: dx64 = x32 on level l
  // RC: the defect of x32 in compensated FP32, a launch per degree (replaces
  // res_x, res_y and x_f2d)
  std::vector<FfOp> ff_x, ff_y;
  DevArray<int> symv_pid;
  int nsymv = 0, maxn_symv = 0;
};

struct SolvePlan {  // GMRES work lists built once per batch
  std::vector<SweepOp<double>> apply_x;  // per j: (V_j left | Z_j right) -> scratch
  SweepOp<double> apply_y;               // scratch -> w (b64_L left | r64_L right)
  SweepOp<double> resid_x, resid_y;      // x -> scratch, b - A x -> r64_L (caller vectors)
  VecOpList<double> ww, wV, Vw, Vr, rr, xcopyZ, Vcopy, rcopy, x64dot;
  VecOpList<double> zero_x, copy_b, bnorm, xV;  // caller vectors (refreshed per call)
  std::vector<Vec<double>> h_zero_x, h_copy_b, h_bnorm, h_xV;
  std::vector<SweepArgs<double>> h_rx, h_ry;
  std::vector<double> hd, hcoef;
};

}  // namespace

struct bh_batch {
  int P = 0;
  cudaStream_t st = nullptr;    // the batch's own non-blocking stream (graph capture needs one)
  cudaStream_t user = nullptr;  // the caller's stream: solves wait for its pending work
  cudaEvent_t ev = nullptr;
  std::vector<bh_ctx*> ctx;
  std::vector<int> k, L;
  int m = 0;           // GMRES restart length
  bool mixed = false;  // FP32 V-cycle with FP64 (R64) or compensated FP32 (RC) defects
  bool rc = false;     // BH_MIXED_FP32_RC
  bool right = false;  // right (flexible) preconditioning
  int pre = 1, post = 1;
  int tile[8] = {0};  // patches per block per degree (0 = default)
  // device meta
  int* d_k = nullptr;
  const void** d_tabs64 = nullptr;
  const void** d_tabs32 = nullptr;
  const void** d_tabsff = nullptr;  // RC: FfTab<k> per problem
  int* d_active = nullptr;
  double* d_dots = nullptr;      // [P][m + 2]
  double* d_coef = nullptr;      // [P][m + 2]
  double* d_partials = nullptr;
  std::vector<Depth> depth;
  std::vector<void*> allocs;
  SolvePlan* plan = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  std::vector<double*> stage_b, stage_x;  // device staging for bh_batch_solve_host
  // side streams and events that fork the per-degree MVS launches of one
  // color into parallel branches of the captured V-cycle graph
  std::vector<cudaStream_t> side;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  long long launches = 0;        // kernels run by the batch (graph replays count their nodes)
  long long graph_kernels = 0;   // kernel nodes of the captured V-cycle graph
  // persistent form: the V-cycle's phases for one cooperative launch
  bool persistent = false;
  Phase* d_phases = nullptr;
  int nphases = 0;
  size_t psmem = 0;              // dynamic shared memory of the persistent kernel
  int pgrid = 0;                 // its co-resident grid
  unsigned* d_bar = nullptr;     // [count, generation, status, -]
  int* h_status = nullptr;       // pinned copy of the status word
  long long budget_cycles = 0;   // bounded barrier wait (clock64 cycles)
  std::vector<int> last_iters;
};

namespace {

template <typename A>
bh_status upload(bh_batch* b, const std::vector<A>& h, DevArray<A>& d) {
  d.n = (int)h.size();
  d.d = nullptr;
  if (h.empty()) return BH_OK;
  if (alloc_fault() || cudaMalloc(&d.d, h.size() * sizeof(A)) != cudaSuccess) {
    d.d = nullptr;
    cudaGetLastError();
    return berr(BH_ENOMEM, "cudaMalloc failed in batch setup");
  }
  b->allocs.push_back(d.d);
  BCK(cudaMemcpy(d.d, h.data(), h.size() * sizeof(A), cudaMemcpyHostToDevice));
  return BH_OK;
}

template <typename T>
Meta meta(const bh_batch* b) {
  return Meta{b->d_k, sizeof(T) == 8 ? b->d_tabs64 : b->d_tabs32, b->d_active};
}

unsigned blocks_for(int64_t threads, int bs) { return (unsigned)((threads + bs - 1) / bs); }

// one compensated-defect sweep of level Lv along axis 0 (x: FP32 iterate ->
// out) or 1 (in -> r = b - A x)
FfSweepArgs ff_args(const Level& Lv, int axis, const float* x, float2* const* io,
                    const double* bvec, double* r) {
  FfSweepArgs a{};
  a.d = 2;
  a.N = Lv.g.N;
  a.n = Lv.g.n;
  a.lines = Lv.g.nd / Lv.g.n;
  a.stride = axis == 0 ? 1 : Lv.g.n;
  a.axis = axis;
  a.scale = Lv.ascale;
  a.x = x;
  for (int i = 0; i < 3; ++i) {
    a.in[i] = axis == 1 ? io[i] : nullptr;
    a.out[i] = axis == 0 ? io[i] : nullptr;
  }
  a.b = bvec;
  a.r = r;
  return a;
}

template <typename T>
SweepArgs<T> sweep_args(const Level& Lv, int axis, const T* in0, const T* in1, const T* in2,
                        T* o0, T* o1, T* o2, const T* bvec, int mode) {
  SweepArgs<T> a{};
  a.d = 2;
  a.N = Lv.g.N;
  a.n = Lv.g.n;
  a.lines = Lv.g.nd / Lv.g.n;
  a.stride = axis == 0 ? 1 : Lv.g.n;
  a.axis = axis;
  a.scale = Lv.ascale;
  a.mode = mode;
  a.b = bvec;
  a.in[0] = in0;
  a.in[1] = in1;
  a.in[2] = in2;
  a.out[0] = o0;
  a.out[1] = o1;
  a.out[2] = o2;
  return a;
}

// build a sweep op over (problem id, args) pairs
template <typename T>
bh_status make_sweep(bh_batch* b, const std::vector<std::pair<int, SweepArgs<T>>>& items,
                     SweepOp<T>& op) {
  std::vector<SweepArgs<T>> args;
  std::vector<int64_t> prefix{0};
  std::vector<int> pid;
  for (auto& it : items) {
    args.push_back(it.second);
    pid.push_back(it.first);
    // whole blocks per problem (sweep_batch_kernel): the split along axis 0 in tiles
    prefix.push_back(prefix.back() + sweep_launch_threads(it.second.axis == 0 ? 0 : 2,
                                                          it.second.lines, it.second.N));
  }
  op.total = prefix.back();
  BCKS(upload(b, args, op.args));
  BCKS(upload(b, prefix, op.prefix));
  BCKS(upload(b, pid, op.pid));
  return BH_OK;
}

bh_status make_ff(bh_batch* b, const std::vector<std::pair<int, FfSweepArgs>>& items, FfOp& op) {
  std::vector<FfSweepArgs> args;
  std::vector<int64_t> prefix{0};
  std::vector<int> pid;
  for (auto& it : items) {
    args.push_back(it.second);
    pid.push_back(it.first);
    // each problem's range in whole blocks (ff_sweep_list_kernel): KIND 0 (axis
    // 0) in tiles of lines and cells, the others one thread per cell
    prefix.push_back(prefix.back() +
                     ff_sweep_threads(it.second.axis == 0 ? 0 : 2, it.second.lines, it.second.N));
  }
  op.total = prefix.back();
  BCKS(upload(b, args, op.args));
  BCKS(upload(b, prefix, op.prefix));
  BCKS(upload(b, pid, op.pid));
  return BH_OK;
}

template <typename T, bool PROLONG>
XferArgs<T> xfer_args(int axis, const LevelGeom& fine, const T* in, T* out, bool add) {
  const int K = fine.k, Nc = fine.N / 2, nc = K * Nc - 1, nf = fine.n;
  XferArgs<T> a{};
  a.in = in;
  a.out = out;
  a.d = 2;
  a.axis = axis;
  a.Nc = Nc;
  a.nc = nc;
  a.nf = nf;
  a.add = add;
  int din[2], dout[2];
  for (int i = 0; i < 2; ++i) {
    // pass 0 maps coarse x (prolongation) / fine x (restriction) of axis 0
    const int before = PROLONG ? nc : nf, after = PROLONG ? nf : nc;
    din[i] = i < axis ? after : before;
    dout[i] = i <= axis ? after : before;
  }
  int64_t si = 1, so = 1;
  for (int i = 0; i < 3; ++i) {
    a.dims_in[i] = i < 2 ? din[i] : 1;
    a.dims_out[i] = i < 2 ? dout[i] : 1;
    a.str_in[i] = si;
    a.str_out[i] = so;
    si *= a.dims_in[i];
    so *= a.dims_out[i];
  }
  a.lines = din[1 - axis];
  return a;
}

template <typename T>
bh_status make_xfer(bh_batch* b, const std::vector<std::pair<int, XferArgs<T>>>& items,
                    XferOp<T>& op) {
  std::vector<XferArgs<T>> args;
  std::vector<int64_t> prefix{0};
  std::vector<int> pid;
  for (auto& it : items) {
    args.push_back(it.second);
    pid.push_back(it.first);
    prefix.push_back(prefix.back() + it.second.lines * it.second.Nc);
  }
  op.total = prefix.back();
  BCKS(upload(b, args, op.args));
  BCKS(upload(b, prefix, op.prefix));
  BCKS(upload(b, pid, op.pid));
  return BH_OK;
}

// per-call lists: same shape every call, pointers refreshed with an async copy
bh_status refresh_vec(bh_batch* b, const std::vector<std::pair<int, Vec<double>>>& items,
                      VecOpList<double>& op, std::vector<Vec<double>>& host) {
  host.clear();
  for (auto& it : items) host.push_back(it.second);
  BCK(cudaMemcpyAsync(op.v.d, host.data(), host.size() * sizeof(Vec<double>),
                      cudaMemcpyHostToDevice, b->st));
  return BH_OK;
}

template <typename T>
bh_status make_vec(bh_batch* b, const std::vector<std::pair<int, Vec<T>>>& items,
                   VecOpList<T>& op) {
  std::vector<Vec<T>> v;
  std::vector<int64_t> prefix{0}, cprefix{0};
  std::vector<int> pid;
  for (auto& it : items) {
    v.push_back(it.second);
    pid.push_back(it.first);
    prefix.push_back(prefix.back() + it.second.n);
    cprefix.push_back(cprefix.back() + (it.second.n + kChunk - 1) / kChunk);
  }
  op.total = prefix.back();
  op.chunks = cprefix.back();
  BCKS(upload(b, v, op.v));
  BCKS(upload(b, prefix, op.prefix));
  BCKS(upload(b, cprefix, op.cprefix));
  BCKS(upload(b, pid, op.pid));
  return BH_OK;
}

bh_status make_conv(bh_batch* b, const std::vector<std::pair<int, Conv>>& items, ConvOpList& op) {
  std::vector<Conv> v;
  std::vector<int64_t> prefix{0};
  std::vector<int> pid;
  for (auto& it : items) {
    v.push_back(it.second);
    pid.push_back(it.first);
    prefix.push_back(prefix.back() + it.second.n);
  }
  op.total = prefix.back();
  BCKS(upload(b, v, op.v));
  BCKS(upload(b, prefix, op.prefix));
  BCKS(upload(b, pid, op.pid));
  return BH_OK;
}

int mvs_pb(const bh_batch* b, int k) {
  if (b->tile[k] > 0) return b->tile[k];
  return 4;  // default before tuning
}

template <typename T>
size_t mvs_smem(int k, int pb) {
  switch (k) {
    case 2: return Mvs2Cfg<T, 2>::smem_bytes(pb);
    case 3: return Mvs2Cfg<T, 3>::smem_bytes(pb);
    case 4: return Mvs2Cfg<T, 4>::smem_bytes(pb);
    case 5: return Mvs2Cfg<T, 5>::smem_bytes(pb);
    case 6: return Mvs2Cfg<T, 6>::smem_bytes(pb);
    default: return Mvs2Cfg<T, 7>::smem_bytes(pb);
  }
}

template <typename T>
int mvs_pb_max_t(int k) {
  switch (k) {
    case 2: return Mvs2Cfg<T, 2>::PB_MAX;
    case 3: return Mvs2Cfg<T, 3>::PB_MAX;
    case 4: return Mvs2Cfg<T, 4>::PB_MAX;
    case 5: return Mvs2Cfg<T, 5>::PB_MAX;
    case 6: return Mvs2Cfg<T, 6>::PB_MAX;
    default: return Mvs2Cfg<T, 7>::PB_MAX;
  }
}

int mvs_pb_max(const bh_batch* b, int k) {
  return b->mixed ? mvs_pb_max_t<float>(k) : mvs_pb_max_t<double>(k);
}

size_t mvs_smem_for(const bh_batch* b, int k, int pb) {
  return b->mixed ? mvs_smem<float>(k, pb) : mvs_smem<double>(k, pb);
}

// typed level buffers of the V-cycle
template <typename T> struct LvBuf;
template <> struct LvBuf<double> {
  static double* x(Level& l) { return l.x64; }
  static double* b(Level& l) { return l.b64; }
  static double* xs(bh_ctx* c) { return c->xs64[0]; }
  static const void* tab(bh_ctx* c) { return c->tab64; }
};
template <> struct LvBuf<float> {
  static float* x(Level& l) { return l.x32; }
  static float* b(Level& l) { return l.b32; }
  static float* xs(bh_ctx* c) { return c->xs32[0]; }
  static const void* tab(bh_ctx* c) { return c->tab32; }
};

// the V-cycle ops of value type T at one depth (smoothing, prolongation,
// zeroing of the coarse iterate, coarse solve) for the problems in `ps`
template <typename T>
bh_status build_vdepth(bh_batch* b, int t, VDepth<T>& V, Depth& D) {
  std::vector<std::pair<int, XferArgs<T>>> p0, p1;
  std::vector<std::pair<int, Vec<T>>> zc;
  std::vector<Symv<T>> sv;
  std::vector<int> svp;
  // per color, degree and table class (problems of one degree whose tables
  // agree byte for byte, i.e. of one penalty): patch-list arguments, problems,
  // tiles
  struct Group {
    std::vector<MvsArgs<T>> args;
    std::vector<int> pid;
    std::vector<Tile> tiles;
    const void* htab = nullptr;
  };
  std::map<std::tuple<int, int, int>, Group> groups;  // (color, degree, table class)
  std::vector<const void*> reps[kMaxK + 1];           // one host table per class
  size_t smem_k[kMaxK + 1] = {0};
  for (int p = 0; p < b->P; ++p) {
    const int l = b->L[p] - t;
    if (l < 1) continue;
    bh_ctx* c = b->ctx[p];
    Level& Lv = c->lv[l];
    if (l == 1) {
      sv.push_back(Symv<T>{c->coarse_inv, LvBuf<T>::b(Lv), LvBuf<T>::x(Lv), c->coarse_n, Lv.pscale});
      svp.push_back(p);
      D.maxn_symv = std::max(D.maxn_symv, c->coarse_n);
      continue;
    }
    Level& Lc = c->lv[l - 1];
    p0.push_back({p, xfer_args<T, true>(0, Lv.g, LvBuf<T>::x(Lc), LvBuf<T>::xs(c), false)});
    p1.push_back({p, xfer_args<T, true>(1, Lv.g, LvBuf<T>::xs(c), LvBuf<T>::x(Lv), true)});
    zc.push_back({p, Vec<T>{LvBuf<T>::x(Lc), nullptr, Lc.g.nd, 0, 0}});
    const int k = b->k[p];
    const int pb = std::min(mvs_pb(b, k), mvs_pb_max_t<T>(k));
    smem_k[k] = mvs_smem<T>(k, pb);
    const DevTables dt = Ops<T>::device_tables(LvBuf<T>::tab(c), k);
    // FP32: one launch per class of problems whose interior tables agree byte
    // for byte (one penalty), the tables being the launch's parameter
    static const int kNoTable = 0;
    size_t tbytes = 0;
    const void* htab = &kNoTable;
    if (sizeof(T) == 4) htab = Ops<T>::host_mvs_tables(LvBuf<T>::tab(c), k, &tbytes);
    int cls = 0;
    while (cls < (int)reps[k].size() && tbytes && std::memcmp(reps[k][cls], htab, tbytes) != 0)
      ++cls;
    if (cls == (int)reps[k].size()) reps[k].push_back(htab);
    for (int col = 0; col < 8; ++col) {
      MvsArgs<T> a{};
      a.x = LvBuf<T>::x(Lv);
      a.b = LvBuf<T>::b(Lv);
      a.verts = Lv.verts + Lv.coff[col];
      a.count = Lv.coff[col + 1] - Lv.coff[col];
      a.N = Lv.g.N;
      a.n = Lv.g.n;
      a.pb = pb;
      a.ascale = Lv.ascale;
      a.pscale = c->p.omega * Lv.pscale;
      a.dinv = static_cast<const T*>(dt.dinv);
      Group& G = groups[std::make_tuple(col, k, cls)];
      G.htab = reps[k][cls];
      const int s = (int)G.args.size();
      G.args.push_back(a);
      G.pid.push_back(p);
      for (int f = 0; f < a.count; f += pb) G.tiles.push_back(Tile{s, f, std::min(pb, a.count - f)});
    }
  }
  if (!p0.empty()) {
    BCKS(make_xfer(b, p0, V.prol[0]));
    BCKS(make_xfer(b, p1, V.prol[1]));
    BCKS(make_vec(b, zc, V.zero_coarse));
    for (auto& [key, G] : groups) {  // in (color, degree, class) order
      if (G.tiles.empty()) continue;
      const int col = std::get<0>(key), k = std::get<1>(key);
      V.mvs[col].emplace_back();
      MvsOp<T>& op = V.mvs[col].back();
      BCKS(upload(b, G.args, op.args));
      BCKS(upload(b, G.pid, op.pid));
      BCKS(upload(b, G.tiles, op.tiles));
      op.smem = smem_k[k];
      op.k = k;
      op.htab = G.htab;
    }
  }
  if (!sv.empty()) {
    BCKS(upload(b, sv, V.symv));
    BCKS(upload(b, svp, D.symv_pid));
    D.nsymv = (int)sv.size();
  }
  return BH_OK;
}

// the lockstep V-cycle's work lists (depends on the tile shapes)
bh_status build_depths(bh_batch* b) {
  const int P = b->P;
  const int T_ = *std::max_element(b->L.begin(), b->L.end());
  b->depth.assign(T_, Depth());
  for (int t = 0; t < T_; ++t) {
    Depth& D = b->depth[t];
    std::vector<std::pair<int, SweepArgs<double>>> rx, ry;
    std::vector<std::pair<int, XferArgs<double>>> r0, r1;
    std::vector<std::pair<int, Conv>> xf;
    std::vector<std::pair<int, FfSweepArgs>> fx[kMaxK + 1], fy[kMaxK + 1];
    for (int p = 0; p < P; ++p) {
      const int l = b->L[p] - t;
      if (l < 1) continue;
      if (l == 1) {
        D.coarse = true;
        continue;
      }
      D.smooth = true;
      bh_ctx* c = b->ctx[p];
      Level& Lv = c->lv[l];
      Level& Lc = c->lv[l - 1];
      double* s0 = c->scr64;
      double* s1 = c->scr64 + Lv.g.nd;
      double* s2 = c->scr64 + 2 * Lv.g.nd;
      // defect in FP64: of x64 (FP64) or of dx64 = x32 (R64), against the FP64
      // right-hand side of the level (R64: b64 on the finest level, db64 below)
      const double* xin = b->mixed ? Lv.dx64 : Lv.x64;
      const double* bin = (b->mixed && l != b->L[p]) ? Lv.db64 : Lv.b64;
      double* bc = b->mixed ? Lc.db64 : Lc.b64;
      if (b->rc) {
        // double-float intermediates in the FP64 scratch (8 bytes per value)
        float2* io[3] = {reinterpret_cast<float2*>(s0), reinterpret_cast<float2*>(s1),
                         reinterpret_cast<float2*>(s2)};
        fx[b->k[p]].push_back({p, ff_args(Lv, 0, Lv.x32, io, nullptr, nullptr)});
        fy[b->k[p]].push_back({p, ff_args(Lv, 1, nullptr, io, bin, Lv.r64)});
      } else {
        rx.push_back({p, sweep_args<double>(Lv, 0, xin, nullptr, nullptr, s0, s1, s2, nullptr, kStore)});
        ry.push_back({p, sweep_args<double>(Lv, 1, s0, s1, s2, Lv.r64, nullptr, nullptr, bin, kResidual)});
      }
      r0.push_back({p, xfer_args<double, false>(0, Lv.g, Lv.r64, c->xs64[0], false)});
      XferArgs<double> a1 = xfer_args<double, false>(1, Lv.g, c->xs64[0], bc, false);
      if (b->mixed) {
        // the FP32 right-hand side of level l-1, written by the restriction's
        // last pass
        a1.out32 = Lc.b32;
        if (!b->rc) xf.push_back({p, Conv{Lv.dx64, Lv.x32, Lv.g.nd, 0}});
      }
      r1.push_back({p, a1});
    }
    if (D.smooth) {
      BCKS(make_sweep(b, rx, D.res_x));
      BCKS(make_sweep(b, ry, D.res_y));
      for (int k = 0; k <= kMaxK; ++k) {
        if (fx[k].empty()) continue;
        D.ff_x.emplace_back();
        D.ff_y.emplace_back();
        D.ff_x.back().k = D.ff_y.back().k = k;
        BCKS(make_ff(b, fx[k], D.ff_x.back()));
        BCKS(make_ff(b, fy[k], D.ff_y.back()));
      }
      BCKS(make_xfer(b, r0, D.restr[0]));
      BCKS(make_xfer(b, r1, D.restr[1]));
      if (b->mixed) {
        BCKS(make_conv(b, xf, D.x_f2d));
      }
    }
    if (b->mixed)
      BCKS(build_vdepth<float>(b, t, D.v32, D));
    else
      BCKS(build_vdepth<double>(b, t, D.v64, D));
  }
  return BH_OK;
}

// ---- launches (all on b->st, graph-capturable) ---------------------------------
void count_launch(bh_batch* b, int n = 1) {
  b->launches += n;
  g_kernel_launches.fetch_add(n);
}

template <typename T>
cudaError_t run_sweep(bh_batch* b, const SweepOp<T>& op, int kind) {
  if (op.total == 0) return cudaSuccess;
  const unsigned g = blocks_for(op.total, 128);
  if (kind == 0)
    sweep_batch_kernel<T, 0><<<g, 128, 0, b->st>>>(meta<T>(b), op.args.d, op.prefix.d, op.pid.d,
                                                   op.pid.n);
  else
    sweep_batch_kernel<T, 2><<<g, 128, 0, b->st>>>(meta<T>(b), op.args.d, op.prefix.d, op.pid.d,
                                                   op.pid.n);
  count_launch(b);
  return cudaGetLastError();
}

// one compensated-defect sweep: a launch per degree, forked onto the side
// streams and joined back like the patch launches
cudaError_t run_ff(bh_batch* b, const std::vector<FfOp>& ops, int kind) {
  if (ops.empty()) return cudaSuccess;
  cudaError_t e;
  const bool fork = ops.size() > 1;
  if (fork && (e = cudaEventRecord(b->fork, b->st)) != cudaSuccess) return e;
  for (size_t i = 0; i < ops.size(); ++i) {
    const FfOp& op = ops[i];
    cudaStream_t st = fork ? b->side[i] : b->st;
    if (fork && (e = cudaStreamWaitEvent(st, b->fork, 0)) != cudaSuccess) return e;
    const FfSweepArgs* args = op.args.d;
    const int64_t* prefix = op.prefix.d;
    const int* pid = op.pid.d;
    int n = op.pid.n;
    const int* active = b->d_active;
    const void* const* tabs = b->d_tabsff;
    void* params[] = {&args, &prefix, &pid, &n, &active, &tabs};
    if ((e = cudaLaunchKernel(ff_list_kernel(op.k, kind), dim3(blocks_for(op.total, kFfBlock)),
                              dim3(kFfBlock), params, 0, st)) != cudaSuccess)
      return e;
    count_launch(b);
    if (fork && (e = cudaEventRecord(b->join[i], st)) != cudaSuccess) return e;
  }
  if (fork)
    for (size_t i = 0; i < ops.size(); ++i)
      if ((e = cudaStreamWaitEvent(b->st, b->join[i], 0)) != cudaSuccess) return e;
  return cudaSuccess;
}

template <typename T>
cudaError_t run_xfer(bh_batch* b, const XferOp<T>& op, bool prolong) {
  if (op.total == 0) return cudaSuccess;
  const unsigned g = blocks_for(op.total, 128);
  if (prolong)
    xfer_batch_kernel<T, true><<<g, 128, 0, b->st>>>(meta<T>(b), op.args.d, op.prefix.d, op.pid.d,
                                                     op.pid.n);
  else
    xfer_batch_kernel<T, false><<<g, 128, 0, b->st>>>(meta<T>(b), op.args.d, op.prefix.d,
                                                      op.pid.d, op.pid.n);
  count_launch(b);
  return cudaGetLastError();
}

template <typename T>
cudaError_t run_vec(bh_batch* b, const VecOpList<T>& op, int kind, const double* coef,
                    int cstride, int cslot, double sign, int yslot = 0, int xslot = 0) {
  if (op.total == 0) return cudaSuccess;
  int64_t g = blocks_for(op.total, 256);
  if (g > 152 * 16) g = 152 * 16;
  vec_batch_kernel<T><<<(unsigned)g, 256, 0, b->st>>>(meta<T>(b), op.v.d, op.prefix.d, op.pid.d,
                                                      op.pid.n, kind, coef, cstride, cslot, sign,
                                                      yslot, xslot);
  count_launch(b);
  return cudaGetLastError();
}

cudaError_t run_conv(bh_batch* b, const ConvOpList& op, int dir, int slot = 0) {
  if (op.total == 0) return cudaSuccess;
  int64_t g = blocks_for(op.total, 256);
  if (g > 152 * 16) g = 152 * 16;
  conv_batch_kernel<<<(unsigned)g, 256, 0, b->st>>>(meta<double>(b), op.v.d, op.prefix.d,
                                                    op.pid.d, op.pid.n, dir, slot);
  count_launch(b);
  return cudaGetLastError();
}

cudaError_t run_dot(bh_batch* b, const VecOpList<double>& op, int cslot, int yslot = 0,
                    int xslot = 0) {
  if (op.chunks == 0) return cudaSuccess;
  dot_batch_partial<<<(unsigned)op.chunks, 256, 0, b->st>>>(meta<double>(b), op.v.d,
                                                            op.cprefix.d, op.pid.d, op.pid.n,
                                                            b->d_partials, yslot, xslot);
  dot_batch_final<<<blocks_for(op.pid.n, 64), 64, 0, b->st>>>(op.cprefix.d, op.pid.d, op.pid.n,
                                                             b->d_partials, b->d_dots, b->m + 2,
                                                             cslot);
  count_launch(b, 2);
  return cudaGetLastError();
}

// one color: a launch per degree group, one block per tile, each with the
// shared memory of its own tile shape; with several groups the launches fork
// from b->st onto side streams and join back (parallel graph branches)
template <typename T>
cudaError_t run_mvs(bh_batch* b, const std::vector<MvsOp<T>>& ops) {
  if (ops.empty()) return cudaSuccess;
  cudaError_t e;
  const bool fork = ops.size() > 1;
  if (fork && (e = cudaEventRecord(b->fork, b->st)) != cudaSuccess) return e;
  for (size_t i = 0; i < ops.size(); ++i) {
    const MvsOp<T>& op = ops[i];
    cudaStream_t st = fork ? b->side[i] : b->st;
    if (fork && (e = cudaStreamWaitEvent(st, b->fork, 0)) != cudaSuccess) return e;
    Meta m = meta<T>(b);
    const MvsArgs<T>* args = op.args.d;
    const int* pid = op.pid.d;
    const Tile* tiles = op.tiles.d;
    int ntiles = op.tiles.n;
    void* params[] = {&m, &args, &pid, &tiles, &ntiles, const_cast<void*>(op.htab)};
    if ((e = cudaLaunchKernel(mvs2_batch_kernel_for<T>(op.k), dim3((unsigned)ntiles), dim3(256),
                              params, op.smem, st)) != cudaSuccess)
      return e;
    count_launch(b);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (fork && (e = cudaEventRecord(b->join[i], st)) != cudaSuccess) return e;
  }
  if (fork)
    for (size_t i = 0; i < ops.size(); ++i)
      if ((e = cudaStreamWaitEvent(b->st, b->join[i], 0)) != cudaSuccess) return e;
  return cudaSuccess;
}

template <typename T>
cudaError_t run_colors(bh_batch* b, const VDepth<T>& V, int c0, int c1) {
  cudaError_t e;
  for (int col = c0; col < c1; ++col)
    if ((e = run_mvs<T>(b, V.mvs[col])) != cudaSuccess) return e;
  return cudaSuccess;
}

struct TopOps;
template <typename T> const VecOpList<T>& vdepth_top(const TopOps& top);
template <typename T> const VDepth<T>& vdepth(const Depth& D);
template <> const VDepth<double>& vdepth<double>(const Depth& D) { return D.v64; }
template <> const VDepth<float>& vdepth<float>(const Depth& D) { return D.v32; }

// lockstep V-cycle from depth t in value type T: x_l = MG_l(0, b_l) on level
// l = L_p - t of every problem (x_l zero on entry)
template <typename T>
cudaError_t vcycle_from(bh_batch* b, int t) {
  if (t >= (int)b->depth.size()) return cudaSuccess;
  Depth& D = b->depth[t];
  const VDepth<T>& V = vdepth<T>(D);
  cudaError_t e;
  if (D.coarse) {
    dim3 grid(blocks_for(D.maxn_symv, 128), D.nsymv);
    coarse_batch_kernel<T><<<grid, 128, 0, b->st>>>(meta<T>(b), V.symv.d, D.symv_pid.d, D.nsymv);
    count_launch(b);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (!D.smooth) return cudaSuccess;
  for (int s = 0; s < b->pre; ++s)
    if ((e = run_colors<T>(b, V, 0, 8)) != cudaSuccess) return e;
  if (b->rc) {
    if ((e = run_ff(b, D.ff_x, 0)) != cudaSuccess) return e;
    if ((e = run_ff(b, D.ff_y, 2)) != cudaSuccess) return e;
  } else {
    if (b->mixed && (e = run_conv(b, D.x_f2d, kF2D)) != cudaSuccess) return e;
    if ((e = run_sweep<double>(b, D.res_x, 0)) != cudaSuccess) return e;
    if ((e = run_sweep<double>(b, D.res_y, 2)) != cudaSuccess) return e;
  }
  if ((e = run_xfer<double>(b, D.restr[0], false)) != cudaSuccess) return e;
  if ((e = run_xfer<double>(b, D.restr[1], false)) != cudaSuccess) return e;
  if ((e = run_vec<T>(b, V.zero_coarse, kZero, nullptr, 0, 0, 0.0)) != cudaSuccess) return e;
  if ((e = vcycle_from<T>(b, t + 1)) != cudaSuccess) return e;
  if ((e = run_xfer<T>(b, V.prol[0], true)) != cudaSuccess) return e;
  if ((e = run_xfer<T>(b, V.prol[1], true)) != cudaSuccess) return e;
  for (int s = 0; s < b->post; ++s)
    if ((e = run_colors<T>(b, V, 0, 8)) != cudaSuccess) return e;
  return cudaSuccess;
}

// The captured graph: x64_L = MG(0, b64_L) for every problem.  FP64: zero
// x64_L, V-cycle.  R64: zero x32_L, b32_L = b64_L, FP32 V-cycle (FP64 defects
// against b64_L on the finest level), x64_L = x32_L.
// the first and last operations of the V-cycle (x_L zeroed, and for the FP32
// V-cycle the conversions of b_L and x_L), built once per prepare()
struct TopOps {
  VecOpList<double> zero64;
  VecOpList<float> zero32;
  ConvOpList cin, cout_;
};

template <> const VecOpList<double>& vdepth_top<double>(const TopOps& top) { return top.zero64; }
template <> const VecOpList<float>& vdepth_top<float>(const TopOps& top) { return top.zero32; }

bh_status build_top(bh_batch* b, TopOps& top) {
  std::vector<std::pair<int, Vec<double>>> zf64;
  std::vector<std::pair<int, Vec<float>>> zf32;
  std::vector<std::pair<int, Conv>> bin, xout;
  for (int p = 0; p < b->P; ++p) {
    Level& F = b->ctx[p]->lv[b->L[p]];
    zf64.push_back({p, Vec<double>{F.x64, nullptr, F.g.nd, 0, 0}});
    zf32.push_back({p, Vec<float>{F.x32, nullptr, F.g.nd, 0, 0}});
    bin.push_back({p, Conv{F.b64, F.b32, F.g.nd, 0}});
    xout.push_back({p, Conv{F.x64, F.x32, F.g.nd, 0}});
  }
  if (b->mixed) {
    BCKS(make_vec(b, zf32, top.zero32));
    BCKS(make_conv(b, bin, top.cin));
    BCKS(make_conv(b, xout, top.cout_));
  } else {
    BCKS(make_vec(b, zf64, top.zero64));
  }
  return BH_OK;
}

bh_status capture_vcycle(bh_batch* b, const TopOps& top) {
  if (b->gexec) {
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
  }
  if (b->graph) {
    cudaGraphDestroy(b->graph);
    b->graph = nullptr;
  }
  const VecOpList<double>& zero64 = top.zero64;
  const VecOpList<float>& zero32 = top.zero32;
  const ConvOpList &cin = top.cin, &cout_ = top.cout_;
  const long long before = b->launches, before_g = g_kernel_launches.load();
  BCK(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
  cudaError_t e;
  if (b->mixed) {
    e = run_vec<float>(b, zero32, kZero, nullptr, 0, 0, 0.0);
    if (e == cudaSuccess) e = run_conv(b, cin, kD2F);
    if (e == cudaSuccess) e = vcycle_from<float>(b, 0);
    if (e == cudaSuccess) e = run_conv(b, cout_, kF2D);
  } else {
    e = run_vec<double>(b, zero64, kZero, nullptr, 0, 0, 0.0);
    if (e == cudaSuccess) e = vcycle_from<double>(b, 0);
  }
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(b->st, &g);
  // captured kernels run when the graph is replayed and are counted then
  g_kernel_launches.fetch_sub(b->launches - before);
  b->launches = before;
  (void)before_g;
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return berr(BH_ECUDA, std::string("V-cycle capture failed: ") +
                              cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  b->graph = g;
  size_t nodes = 0;
  BCK(cudaGraphGetNodes(g, nullptr, &nodes));
  b->graph_kernels = (long long)nodes;
  BCK(cudaGraphInstantiate(&b->gexec, g, 0));
  return BH_OK;
}

bh_status set_active(bh_batch* b, const std::vector<int>& act) {
  BCK(cudaMemcpyAsync(b->d_active, act.data(), act.size() * sizeof(int), cudaMemcpyHostToDevice,
                      b->st));
  BCK(cudaStreamSynchronize(b->st));  // act is a host temporary
  return BH_OK;
}

bh_status launch_persistent(bh_batch* b, unsigned extra, long long budget);

// one V-cycle x64_L = MG(0, b64_L): the captured graph, or the persistent kernel
bh_status launch_graph(bh_batch* b) {
  if (b->persistent) return launch_persistent(b, 0, b->budget_cycles);
  BCK(cudaGraphLaunch(b->gexec, b->st));
  count_launch(b, (int)b->graph_kernels);
  return BH_OK;
}

// clear the persistent kernel's status word (before a call) / read it (after
// a synchronization): BH_ETIMEOUT if a bounded barrier wait ran out
bh_status clear_status(bh_batch* b) {
  if (!b->persistent) return BH_OK;
  BCK(cudaMemsetAsync(b->d_bar + 2, 0, sizeof(unsigned), b->st));
  *b->h_status = 0;
  return BH_OK;
}

bh_status check_status(const bh_batch* b) {
  if (b->persistent && *b->h_status != 0)
    return berr(BH_ETIMEOUT, "persistent V-cycle: a grid-barrier wait ran out (status word set)");
  return BH_OK;
}

// only ever raise a kernel's shared-memory limit: graphs of other live batches
// may launch it with more shared memory than this batch needs
template <typename T>
bh_status raise_smem_limit(int k, size_t smem) {
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  const void* kernel = mvs2_batch_kernel_for<T>(k);
  cudaFuncAttributes fa{};
  BCK(cudaFuncGetAttributes(&fa, kernel));
  if ((int)smem > fa.maxDynamicSharedSizeBytes)
    BCK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  return BH_OK;
}

// ---- persistent form: the phase list of one V-cycle ------------------------
template <typename T>
struct PhaseBuilder {
  std::vector<Phase>& ph;
  size_t smem = 0;
  void list(int kind, int n, int64_t total, const void* args, const int64_t* prefix,
            const int* pid, int dir = 0) {
    if (total <= 0) return;
    Phase P{};
    P.kind = kind;
    P.n = n;
    P.total = total;
    P.args = args;
    P.prefix = prefix;
    P.pid = pid;
    P.dir = dir;
    ph.push_back(P);
  }
  void sweep(const SweepOp<double>& op, int kind) {
    list(kind, op.pid.n, op.total, op.args.d, op.prefix.d, op.pid.d);
  }
  template <typename U>
  void xfer(const XferOp<U>& op, int kind) {
    list(kind, op.pid.n, op.total, op.args.d, op.prefix.d, op.pid.d);
  }
  void zero(const VecOpList<T>& op) { list(kPhZero, op.pid.n, op.total, op.v.d, op.prefix.d, op.pid.d); }
  void conv(const ConvOpList& op, int dir) {
    list(kPhConv, op.pid.n, op.total, op.v.d, op.prefix.d, op.pid.d, dir);
  }
  void mvs(const std::vector<MvsOp<T>>& ops) {
    if (ops.empty()) return;
    Phase P{};
    P.kind = kPhMvs;
    for (const MvsOp<T>& op : ops) {
      if (P.ngroups == kMaxK + 1) {  // more table classes than a phase holds: one
        ph.push_back(P);             // more phase (its problems are independent)
        P = Phase{};
        P.kind = kPhMvs;
      }
      MvsGroup& G = P.groups[P.ngroups++];
      G.args = op.args.d;
      G.pid = op.pid.d;
      G.tiles = op.tiles.d;
      G.ntiles = op.tiles.n;
      P.total += op.tiles.n;
      smem = std::max(smem, op.smem);
    }
    ph.push_back(P);
  }
};

// the phases in the order of vcycle_from: per depth (descending) the coarse
// solve, pre-smoothing, defect, restriction and zeroed coarse iterate; per
// depth (ascending) the prolongation and post-smoothing
template <typename T>
bh_status build_phases(bh_batch* b, const TopOps& top) {
  std::vector<Phase> ph;
  PhaseBuilder<T> B{ph};
  const int T_ = (int)b->depth.size();
  if (b->mixed) {
    B.zero(vdepth_top<T>(top));
    B.conv(top.cin, kD2F);
  } else {
    B.zero(vdepth_top<T>(top));
  }
  for (int t = 0; t < T_; ++t) {
    const Depth& D = b->depth[t];
    const VDepth<T>& V = vdepth<T>(D);
    if (D.coarse) {
      Phase P{};
      P.kind = kPhCoarse;
      P.n = D.nsymv;
      P.maxn = D.maxn_symv;
      P.total = (int64_t)D.nsymv * D.maxn_symv;
      P.args = V.symv.d;
      P.pid = D.symv_pid.d;
      ph.push_back(P);
    }
    if (!D.smooth) break;  // no deeper depth holds smoothing work
    for (int s = 0; s < b->pre; ++s)
      for (int col = 0; col < 8; ++col) B.mvs(V.mvs[col]);
    if (b->mixed) B.conv(D.x_f2d, kF2D);
    B.sweep(D.res_x, kPhSweep0);
    B.sweep(D.res_y, kPhSweep2);
    B.xfer(D.restr[0], kPhRestr);
    B.xfer(D.restr[1], kPhRestr);
    B.zero(V.zero_coarse);
  }
  for (int t = T_ - 1; t >= 0; --t) {
    const Depth& D = b->depth[t];
    if (!D.smooth) continue;
    const VDepth<T>& V = vdepth<T>(D);
    B.xfer(V.prol[0], kPhProl);
    B.xfer(V.prol[1], kPhProl);
    for (int s = 0; s < b->post; ++s)
      for (int col = 0; col < 8; ++col) B.mvs(V.mvs[col]);
  }
  if (b->mixed) B.conv(top.cout_, kF2D);
  DevArray<Phase> dph;
  BCKS(upload(b, ph, dph));
  b->d_phases = dph.d;
  b->nphases = (int)ph.size();
  b->psmem = std::max<size_t>(B.smem, 64);
  // co-resident grid of the cooperative launch; the kernel's shared-memory
  // limit is only ever raised (other live batches may launch it with more)
  const void* kernel = vcycle_persistent_kernel_for<T>();
  {
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    cudaFuncAttributes fa{};
    BCK(cudaFuncGetAttributes(&fa, kernel));
    if ((int)b->psmem > fa.maxDynamicSharedSizeBytes)
      BCK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->psmem));
  }
  int per_sm = 0, dev = 0, sms = 0, clock_khz = 0, coop = 0;
  BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, b->psmem));
  BCK(cudaGetDevice(&dev));
  BCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  BCK(cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, dev));
  BCK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (per_sm < 1 || !coop)
    return berr(BH_EINVAL, "persistent V-cycle: no co-resident block fits (tile too large)");
  b->pgrid = per_sm * sms;
  b->budget_cycles = (long long)clock_khz * 2000;  // a 2 s bound on one barrier wait
  return BH_OK;
}

// one persistent V-cycle: x64_L = MG(0, b64_L) for every problem; `extra`
// more arrivals than the grid provides make every barrier wait run out
// (the failure-path check), with a wait of `budget` cycles
bh_status launch_persistent(bh_batch* b, unsigned extra, long long budget) {
  BCK(cudaMemsetAsync(b->d_bar, 0, 2 * sizeof(unsigned), b->st));  // count, generation
  Meta m64 = meta<double>(b);
  Meta mT = b->mixed ? meta<float>(b) : meta<double>(b);
  const Phase* phases = b->d_phases;
  int nph = b->nphases;
  unsigned* bar = b->d_bar;
  unsigned expected = (unsigned)b->pgrid + extra;
  int* status = reinterpret_cast<int*>(b->d_bar + 2);
  void* args[] = {&m64, &mT, &phases, &nph, &bar, &expected, &status, &budget};
  const void* kernel = b->mixed ? vcycle_persistent_kernel_for<float>()
                                : vcycle_persistent_kernel_for<double>();
  BCK(cudaLaunchCooperativeKernel(kernel, dim3(b->pgrid), dim3(256), args, b->psmem, b->st));
  count_launch(b);
  BCK(cudaMemcpyAsync(b->h_status, status, sizeof(int), cudaMemcpyDeviceToHost, b->st));
  return BH_OK;
}

bh_status prepare(bh_batch* b) {
  // mvs kernels: allow the dynamic shared memory of each degree's tile shape
  for (int p = 0; p < b->P; ++p) {
    const int k = b->k[p];
    const size_t smem = mvs_smem_for(b, k, std::min(mvs_pb(b, k), mvs_pb_max(b, k)));
    if (b->mixed)
      BCKS(raise_smem_limit<float>(k, smem));
    else
      BCKS(raise_smem_limit<double>(k, smem));
  }
  BCKS(build_depths(b));
  // one side stream and join event per parallel launch of a color or a
  // compensated sweep (a degree and table class each; created once)
  size_t groups = 0;
  for (const Depth& D : b->depth) {
    for (int col = 0; col < 8; ++col)
      groups = std::max(groups, b->mixed ? D.v32.mvs[col].size() : D.v64.mvs[col].size());
    groups = std::max(groups, D.ff_x.size());
  }
  if (!b->fork) BCK(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
  while (b->side.size() < groups) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    BCK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    b->side.push_back(st);
    BCK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    b->join.push_back(ev);
  }
  TopOps top;
  BCKS(build_top(b, top));
  BCKS(capture_vcycle(b, top));
  if (!b->d_bar) {
    DevArray<unsigned> bar;
    BCKS(upload(b, std::vector<unsigned>(4, 0u), bar));
    b->d_bar = bar.d;
    if (cudaMallocHost((void**)&b->h_status, sizeof(int)) != cudaSuccess) {
      b->h_status = nullptr;
      cudaGetLastError();
      return berr(BH_ENOMEM, "cudaMallocHost failed");
    }
    *b->h_status = 0;
  }
  if (b->rc) return BH_OK;  // graph form only
  return b->mixed ? build_phases<float>(b, top) : build_phases<double>(b, top);
}

bh_status ensure_plan(bh_batch* b) {
  if (b->plan) return BH_OK;
  const int P = b->P, m = b->m;
  for (int p = 0; p < P; ++p) {  // Krylov basis V_0..V_m (and Z_0..Z_{m-1} for right) per problem
    bh_ctx* c = b->ctx[p];
    const int64_t n = c->lv[b->L[p]].g.nd;
    double** bufs[2] = {&c->V, &c->Z};
    const int64_t cnt[2] = {m + 1, b->right ? m : 0};
    for (int i = 0; i < 2; ++i) {
      if (*bufs[i] || cnt[i] == 0) continue;
      if (alloc_fault() || cudaMalloc(bufs[i], (size_t)cnt[i] * n * sizeof(double)) != cudaSuccess) {
        *bufs[i] = nullptr;
        cudaGetLastError();
        return berr(BH_ENOMEM, "Krylov basis allocation failed");
      }
      c->dev_allocs.push_back(*bufs[i]);
    }
  }
  SolvePlan* S = new (std::nothrow) SolvePlan();
  if (!S) return berr(BH_ENOMEM, "host allocation failed");
  b->plan = S;
  S->apply_x.resize(m);
  std::vector<std::pair<int, SweepArgs<double>>> ay, rx, ry;
  std::vector<std::vector<std::pair<int, SweepArgs<double>>>> ax(m);
  std::vector<std::pair<int, Vec<double>>> ww, wV, Vw, Vr, rr, xz, vc, rc, x64, z;
  for (int p = 0; p < P; ++p) {
    bh_ctx* c = b->ctx[p];
    Level& F = c->lv[b->L[p]];
    const int64_t n = F.g.nd;
    double* s0 = c->scr64;
    double* s1 = s0 + n;
    double* s2 = s1 + n;
    // w = A (Z_j | V_j): into r64_L (right; the graph's input b64_L carries V_j)
    // or into b64_L (left; the graph then gives w = M^-1 A V_j in x64_L)
    double* basis = b->right ? c->Z : c->V;
    double* aout = b->right ? F.r64 : F.b64;
    double* w = b->right ? F.r64 : F.x64;
    for (int j = 0; j < m; ++j)
      ax[j].push_back({p, sweep_args<double>(F, 0, basis + (int64_t)j * n, nullptr, nullptr, s0,
                                             s1, s2, nullptr, kStore)});
    ay.push_back({p, sweep_args<double>(F, 1, s0, s1, s2, aout, nullptr, nullptr, nullptr, kStore)});
    rx.push_back({p, sweep_args<double>(F, 0, F.x64, nullptr, nullptr, s0, s1, s2, nullptr, kStore)});
    ry.push_back({p, sweep_args<double>(F, 1, s0, s1, s2, F.r64, nullptr, nullptr, F.b64, kResidual)});
    ww.push_back({p, Vec<double>{w, w, n, 0, 0}});
    wV.push_back({p, Vec<double>{w, c->V, n, 0, n}});
    Vw.push_back({p, Vec<double>{c->V, w, n, n, 0}});
    Vr.push_back({p, Vec<double>{c->V, F.r64, n, n, 0}});    // V_0 = r / sqrt(r.r)
    rr.push_back({p, Vec<double>{F.r64, F.r64, n, 0, 0}});
    xz.push_back({p, Vec<double>{c->Z, F.x64, n, n, 0}});    // Z_j = x64_L
    vc.push_back({p, Vec<double>{F.b64, c->V, n, 0, n}});    // b64_L = V_j
    rc.push_back({p, Vec<double>{F.b64, F.r64, n, 0, 0}});   // b64_L = r
    x64.push_back({p, Vec<double>{F.x64, F.x64, n, 0, 0}});
    z.push_back({p, Vec<double>{F.x64, nullptr, n, 0, 0}});
  }
  for (int j = 0; j < m; ++j) BCKS(make_sweep(b, ax[j], S->apply_x[j]));
  BCKS(make_sweep(b, ay, S->apply_y));
  BCKS(make_sweep(b, rx, S->resid_x));
  BCKS(make_sweep(b, ry, S->resid_y));
  BCKS(make_vec(b, ww, S->ww));
  BCKS(make_vec(b, wV, S->wV));
  BCKS(make_vec(b, Vw, S->Vw));
  BCKS(make_vec(b, Vr, S->Vr));
  BCKS(make_vec(b, rr, S->rr));
  BCKS(make_vec(b, xz, S->xcopyZ));
  BCKS(make_vec(b, vc, S->Vcopy));
  BCKS(make_vec(b, rc, S->rcopy));
  BCKS(make_vec(b, x64, S->x64dot));
  BCKS(make_vec(b, z, S->zero_x));
  BCKS(make_vec(b, z, S->copy_b));
  BCKS(make_vec(b, z, S->bnorm));
  BCKS(make_vec(b, z, S->xV));
  S->hd.assign((size_t)P * (m + 2), 0.0);
  S->hcoef.assign((size_t)P * (m + 2), 0.0);
  return BH_OK;
}

// inputs written on the caller's stream must be complete before the batch reads them
bh_status wait_user(bh_batch* b) {
  BCK(cudaEventRecord(b->ev, b->user));
  BCK(cudaStreamWaitEvent(b->st, b->ev, 0));
  return BH_OK;
}

// after a batch call: later work on the caller's stream sees its results
bh_status signal_user(bh_batch* b) {
  BCK(cudaEventRecord(b->ev, b->st));
  BCK(cudaStreamWaitEvent(b->user, b->ev, 0));
  return BH_OK;
}

// copies between the caller's vectors and the finest-level buffers of every
// problem (one launch each; dst[p] = src[p])
bh_status copy_lists(bh_batch* b, double* const* dst, const double* const* src) {
  std::vector<std::pair<int, Vec<double>>> items;
  for (int p = 0; p < b->P; ++p)
    items.push_back({p, Vec<double>{dst[p], src[p], b->ctx[p]->lv[b->L[p]].g.nd, 0, 0}});
  VecOpList<double> op;
  BCKS(make_vec(b, items, op));
  BCK(run_vec<double>(b, op, kCopy, nullptr, 0, 0, 0.0));
  // make_vec's device lists are batch allocations; this one is used once
  BCK(cudaStreamSynchronize(b->st));
  for (void* ptr : {(void*)op.v.d, (void*)op.prefix.d, (void*)op.cprefix.d, (void*)op.pid.d}) {
    auto it = std::find(b->allocs.begin(), b->allocs.end(), ptr);
    if (it != b->allocs.end()) {
      cudaFree(*it);
      b->allocs.erase(it);
    }
  }
  return BH_OK;
}

}  // namespace

extern "C" {

bh_status bh_batch_create(const bh_params* params, int count, void* stream, bh_batch** out) {
  if (!params || !out || count < 1) return berr(BH_EINVAL, "bh_batch_create: bad arguments");
  *out = nullptr;
  for (int i = 0; i < count; ++i) {
    const bh_params& p = params[i];
    if (p.dim != 2) return berr(BH_EINVAL, "bh_batch_create: the batched form supports 2D problems");
    if (p.smoother != BH_MVS_COLORED || p.local_solver != BH_FDM || p.coarse != BH_COARSE_EXACT ||
        p.krylov != BH_GMRES)
      return berr(BH_EINVAL, "bh_batch_create: the batched form runs colored MVS with FDM local "
                             "solvers, the exact coarse solve and GMRES");
    if (p.precision != BH_FP64 && p.precision != BH_MIXED_FP32_R64 &&
        p.precision != BH_MIXED_FP32_RC)
      return berr(BH_EINVAL, "bh_batch_create: the batched form runs the FP64 V-cycle or the FP32 "
                             "V-cycle with FP64 or compensated defects (BH_MIXED_FP32_R64, "
                             "BH_MIXED_FP32_RC)");
    if (p.precision != params[0].precision || p.gmres_side != params[0].gmres_side ||
        p.pre_steps != params[0].pre_steps || p.post_steps != params[0].post_steps)
      return berr(BH_EINVAL, "bh_batch_create: precision, GMRES side and smoothing steps must be "
                             "the same for every problem of a batch");
    if (p.precision != BH_FP64 && p.gmres_side != BH_RIGHT)
      return berr(BH_EINVAL, "bh_batch_create: the FP32 V-cycle needs the flexible right-"
                             "preconditioned GMRES (gmres_side = BH_RIGHT)");
    if (p.pre_steps < 0 || p.post_steps < 0 || p.pre_steps + p.post_steps > 8)
      return berr(BH_EINVAL, "bh_batch_create: smoothing steps must be in 0..8 in total");
  }
  bh_batch* b = new (std::nothrow) bh_batch();
  if (!b) return berr(BH_ENOMEM, "host allocation failed");
  b->P = count;
  b->user = (cudaStream_t)stream;
  b->mixed = params[0].precision == BH_MIXED_FP32_R64 || params[0].precision == BH_MIXED_FP32_RC;
  b->rc = params[0].precision == BH_MIXED_FP32_RC;
  b->right = params[0].gmres_side == BH_RIGHT;
  b->pre = params[0].pre_steps;
  b->post = params[0].post_steps;
  if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return berr(BH_ECUDA, "bh_batch_create: stream creation failed");
  }
  auto bail = [&](bh_status s) {
    bh_batch_destroy(b);
    return s;
  };
  int m = 0;
  for (int i = 0; i < count; ++i) m = std::max(m, params[i].gmres_restart > 0 ? params[i].gmres_restart : 50);
  b->m = m;
  for (int i = 0; i < count; ++i) {
    bh_params p = params[i];
    p.gmres_restart = m;
    bh_ctx* c = nullptr;
    bh_status s = bh_create(&p, stream, &c);
    if (s != BH_OK) return bail(s);
    b->ctx.push_back(c);
    b->k.push_back(p.degree);
    b->L.push_back(p.level);
  }
  std::vector<const void*> tabs64, tabs32, tabsff;
  for (int p = 0; p < count; ++p) {
    tabs64.push_back(Ops<double>::device_tables(b->ctx[p]->tab64, b->k[p]).tables);
    tabs32.push_back(b->mixed ? Ops<float>::device_tables(b->ctx[p]->tab32, b->k[p]).tables
                              : nullptr);
    tabsff.push_back(b->rc ? ff_device_tables(b->ctx[p]->tab32, b->k[p]) : nullptr);
  }
  DevArray<int> dk;
  DevArray<const void*> dt64, dt32, dtff;
  bh_status s;
  if ((s = upload(b, b->k, dk)) || (s = upload(b, tabs64, dt64)) || (s = upload(b, tabs32, dt32)) ||
      (s = upload(b, tabsff, dtff)))
    return bail(s);
  b->d_k = dk.d;
  b->d_tabs64 = dt64.d;
  b->d_tabs32 = dt32.d;
  b->d_tabsff = dtff.d;
  std::vector<int> act(count, 1);
  DevArray<int> da;
  if ((s = upload(b, act, da))) return bail(s);
  b->d_active = da.d;
  std::vector<double> zeros((size_t)count * (m + 2), 0.0);
  DevArray<double> dd, dc;
  if ((s = upload(b, zeros, dd)) || (s = upload(b, zeros, dc))) return bail(s);
  b->d_dots = dd.d;
  b->d_coef = dc.d;
  int64_t chunks = 0;
  for (int p = 0; p < count; ++p)
    chunks += (b->ctx[p]->lv[b->L[p]].g.nd + kChunk - 1) / kChunk;
  std::vector<double> pz((size_t)chunks + 1, 0.0);
  DevArray<double> dp;
  if ((s = upload(b, pz, dp))) return bail(s);
  b->d_partials = dp.d;
  if ((s = prepare(b))) return bail(s);
  *out = b;
  return BH_OK;
}

bh_status bh_batch_destroy(bh_batch* b) {
  if (!b) return berr(BH_EINVAL, "null batch");
  if (b->st) cudaStreamSynchronize(b->st);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (void* p : b->allocs) cudaFree(p);
  for (bh_ctx* c : b->ctx) bh_destroy(c);
  if (b->ev) cudaEventDestroy(b->ev);
  if (b->fork) cudaEventDestroy(b->fork);
  for (cudaEvent_t e : b->join) cudaEventDestroy(e);
  for (cudaStream_t st : b->side) cudaStreamDestroy(st);
  if (b->st) cudaStreamDestroy(b->st);
  if (b->h_status) cudaFreeHost(b->h_status);
  delete b->plan;
  delete b;
  return BH_OK;
}

bh_status bh_batch_set_tile(bh_batch* b, int degree, int patches_per_block) {
  if (!b || degree < 2 || degree > 7 || patches_per_block < 1 || patches_per_block > 32)
    return berr(BH_EINVAL, "bh_batch_set_tile: bad arguments");
  if (patches_per_block > mvs_pb_max(b, degree))
    return berr(BH_EINVAL, "bh_batch_set_tile: tile exceeds the shared-memory budget (max " +
                               std::to_string(mvs_pb_max(b, degree)) + " patches for this degree)");
  b->tile[degree] = patches_per_block;
  return prepare(b);
}

bh_status bh_batch_set_persistent(bh_batch* b, int on) {
  if (!b || (on != 0 && on != 1)) return berr(BH_EINVAL, "bh_batch_set_persistent: bad arguments");
  if (on == 1 && b->rc)
    return berr(BH_EINVAL, "bh_batch_set_persistent: the compensated defect (BH_MIXED_FP32_RC) "
                           "runs in the graph form only");
  b->persistent = on == 1;
  return BH_OK;
}

bh_status bh_batch_check_barrier_timeout(bh_batch* b, double wait_ms) {
  if (!b || !(wait_ms > 0.0) || wait_ms > 10000.0)
    return berr(BH_EINVAL, "bh_batch_check_barrier_timeout: wait_ms must be in (0, 10000]");
  if (b->rc)
    return berr(BH_EINVAL, "bh_batch_check_barrier_timeout: no persistent form for "
                           "BH_MIXED_FP32_RC");
  int dev = 0, clock_khz = 0;
  BCK(cudaGetDevice(&dev));
  BCK(cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, dev));
  std::vector<int> act(b->P, 1);
  BCKS(set_active(b, act));
  BCKS(wait_user(b));
  const bool was = b->persistent;
  b->persistent = true;
  bh_status s = clear_status(b);
  if (s == BH_OK) s = launch_persistent(b, 1u, (long long)(clock_khz * wait_ms));
  b->persistent = was;
  if (s != BH_OK) return s;
  BCK(cudaStreamSynchronize(b->st));
  if (*b->h_status == 0) return berr(BH_EINVAL, "barrier check: the barrier completed");
  return berr(BH_ETIMEOUT, "barrier check: the bounded grid-barrier wait ran out as arranged");
}

bh_status bh_batch_vcycle_time(bh_batch* b, int reps, double* ms) {
  if (!b || reps < 1 || !ms) return berr(BH_EINVAL, "bad arguments");
  std::vector<int> act(b->P, 1);
  BCKS(set_active(b, act));
  BCKS(wait_user(b));
  cudaEvent_t e0, e1;
  BCK(cudaEventCreate(&e0));
  BCK(cudaEventCreate(&e1));
  BCKS(clear_status(b));
  BCKS(launch_graph(b));
  BCK(cudaEventRecord(e0, b->st));
  for (int r = 0; r < reps; ++r) BCKS(launch_graph(b));
  BCK(cudaEventRecord(e1, b->st));
  BCK(cudaEventSynchronize(e1));
  float t = 0.f;
  BCK(cudaEventElapsedTime(&t, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  BCKS(check_status(b));
  *ms = t / reps;
  return BH_OK;
}

bh_status bh_batch_vcycle(bh_batch* b, const double* const* b_dev, double* const* x_dev) {
  if (!b || !b_dev || !x_dev) return berr(BH_EINVAL, "bh_batch_vcycle: bad arguments");
  for (int p = 0; p < b->P; ++p)
    if (!b_dev[p] || !x_dev[p] || b_dev[p] == x_dev[p])
      return berr(BH_EINVAL, "bh_batch_vcycle: null or aliased vectors");
  std::vector<int> act(b->P, 1);
  BCKS(set_active(b, act));
  BCKS(wait_user(b));
  std::vector<double*> bl(b->P), xl(b->P);
  for (int p = 0; p < b->P; ++p) {
    Level& F = b->ctx[p]->lv[b->L[p]];
    bl[p] = F.b64;
    xl[p] = F.x64;
  }
  BCKS(copy_lists(b, bl.data(), b_dev));
  BCKS(clear_status(b));
  BCKS(launch_graph(b));
  BCKS(copy_lists(b, x_dev, xl.data()));  // synchronizes the batch's stream
  BCKS(check_status(b));
  return signal_user(b);
}

bh_status bh_batch_smooth_colors(bh_batch* b, double* const* x_dev, const double* const* b_dev,
                                 int first_color, int end_color) {
  if (!b || !b_dev || !x_dev) return berr(BH_EINVAL, "bh_batch_smooth_colors: bad arguments");
  if (first_color < 0 || end_color > 8 || first_color > end_color)
    return berr(BH_EINVAL, "bh_batch_smooth_colors: color range outside 0..8");
  for (int p = 0; p < b->P; ++p) {
    if (!b_dev[p] || !x_dev[p] || (const double*)x_dev[p] == b_dev[p])
      return berr(BH_EINVAL, "bh_batch_smooth_colors: null or aliased vectors");
    if (b->L[p] < 2)
      return berr(BH_EINVAL, "bh_batch_smooth_colors: a level-1 problem has no smoother");
  }
  std::vector<int> act(b->P, 1);
  BCKS(set_active(b, act));
  BCKS(wait_user(b));
  std::vector<double*> bl(b->P), xl(b->P);
  for (int p = 0; p < b->P; ++p) {
    Level& F = b->ctx[p]->lv[b->L[p]];
    bl[p] = F.b64;
    xl[p] = F.x64;
  }
  BCKS(copy_lists(b, bl.data(), b_dev));
  BCKS(copy_lists(b, xl.data(), x_dev));
  if (b->mixed) {
    std::vector<std::pair<int, Conv>> cb, cx;
    for (int p = 0; p < b->P; ++p) {
      Level& F = b->ctx[p]->lv[b->L[p]];
      cb.push_back({p, Conv{F.b64, F.b32, F.g.nd, 0}});
      cx.push_back({p, Conv{F.x64, F.x32, F.g.nd, 0}});
    }
    ConvOpList ob, ox;
    BCKS(make_conv(b, cb, ob));
    BCKS(make_conv(b, cx, ox));
    BCK(run_conv(b, ob, kD2F));
    BCK(run_conv(b, ox, kD2F));
    BCK(run_colors<float>(b, b->depth[0].v32, first_color, end_color));
    BCK(run_conv(b, ox, kF2D));
  } else {
    BCK(run_colors<double>(b, b->depth[0].v64, first_color, end_color));
  }
  BCKS(copy_lists(b, x_dev, xl.data()));
  return signal_user(b);
}

bh_status bh_batch_solve(bh_batch* b, const double* const* b_dev, double* const* x_dev,
                         double rtol, int maxit, int* iters, double* relres) {
  if (!b || !b_dev || !x_dev || !iters || !relres || !(rtol > 0.0) || maxit < 1)
    return berr(BH_EINVAL, "bh_batch_solve: bad arguments");
  for (int p = 0; p < b->P; ++p)
    if (!b_dev[p] || !x_dev[p] || (const double*)x_dev[p] == b_dev[p])
      return berr(BH_EINVAL, "bh_batch_solve: null or aliased vectors");
  const int P = b->P, m = b->m;
  const int cs = b->m + 2;  // stride of the dots and coefficient arrays
  const bool right = b->right;
  BCKS(ensure_plan(b));
  SolvePlan& S = *b->plan;
  BCKS(wait_user(b));
  // caller vectors: x (zeroed, updated), b (norm; copied to b64_L for the left
  // start and the residual)
  {
    std::vector<std::pair<int, Vec<double>>> lx, lb, lbb, lxv;
    for (int p = 0; p < P; ++p) {
      bh_ctx* c = b->ctx[p];
      Level& F = c->lv[b->L[p]];
      const int64_t n = F.g.nd;
      lx.push_back({p, Vec<double>{x_dev[p], nullptr, n, 0, 0}});
      lb.push_back({p, Vec<double>{right ? F.r64 : F.b64, b_dev[p], n, 0, 0}});
      lbb.push_back({p, Vec<double>{const_cast<double*>(b_dev[p]), b_dev[p], n, 0, 0}});
      lxv.push_back({p, Vec<double>{x_dev[p], right ? c->Z : c->V, n, 0, n}});
    }
    BCKS(refresh_vec(b, lx, S.zero_x, S.h_zero_x));
    BCKS(refresh_vec(b, lb, S.copy_b, S.h_copy_b));
    BCKS(refresh_vec(b, lbb, S.bnorm, S.h_bnorm));
    BCKS(refresh_vec(b, lxv, S.xV, S.h_xV));
    S.h_rx.clear();
    S.h_ry.clear();
    for (int p = 0; p < P; ++p) {
      bh_ctx* c = b->ctx[p];
      Level& F = c->lv[b->L[p]];
      double* s0 = c->scr64;
      double* s1 = s0 + F.g.nd;
      double* s2 = s1 + F.g.nd;
      S.h_rx.push_back(sweep_args<double>(F, 0, x_dev[p], nullptr, nullptr, s0, s1, s2, nullptr, kStore));
      S.h_ry.push_back(sweep_args<double>(F, 1, s0, s1, s2, F.r64, nullptr, nullptr, b_dev[p], kResidual));
    }
    BCK(cudaMemcpyAsync(S.resid_x.args.d, S.h_rx.data(), P * sizeof(SweepArgs<double>),
                        cudaMemcpyHostToDevice, b->st));
    BCK(cudaMemcpyAsync(S.resid_y.args.d, S.h_ry.data(), P * sizeof(SweepArgs<double>),
                        cudaMemcpyHostToDevice, b->st));
  }
  std::vector<int> act(P, 1);
  BCKS(set_active(b, act));
  BCKS(clear_status(b));
  BCK(run_vec<double>(b, S.zero_x, kZero, nullptr, 0, 0, 0.0));
  // r0 = b (right, in r64_L) or M^-1 b (left, in x64_L); beta = ||r0||, ||b||
  BCK(run_vec<double>(b, S.copy_b, kCopy, nullptr, 0, 0, 0.0));
  if (right) {
    BCK(run_dot(b, S.rr, 0));
  } else {
    BCKS(launch_graph(b));
    BCK(run_dot(b, S.x64dot, 0));
  }
  BCK(run_dot(b, S.bnorm, 1));
  std::vector<double>& hd = S.hd;
  BCK(cudaMemcpyAsync(hd.data(), b->d_dots, hd.size() * sizeof(double), cudaMemcpyDeviceToHost, b->st));
  BCK(cudaStreamSynchronize(b->st));
  BCKS(check_status(b));
  std::vector<double> beta(P), bnorm(P), ref(P);
  for (int p = 0; p < P; ++p) {
    beta[p] = std::sqrt(hd[(size_t)p * cs]);
    bnorm[p] = std::sqrt(hd[(size_t)p * cs + 1]);
    ref[p] = beta[p];
    if (!std::isfinite(bnorm[p]) || !std::isfinite(beta[p]))
      return berr(BH_EINVAL, "right-hand side is not finite");
    if (!(bnorm[p] > 0.0) || !(beta[p] > 0.0)) act[p] = 0;
  }
  std::vector<int> total(P, 0), conv(P, 0), ran(P, 0);
  std::vector<double> est_last(P, 0.0);
  for (int p = 0; p < P; ++p) conv[p] = act[p] ? 0 : 1;
  std::vector<std::vector<double>> H(P, std::vector<double>((size_t)(m + 1) * m, 0.0));
  std::vector<std::vector<double>> cn(P, std::vector<double>(m)), sn(P, std::vector<double>(m)),
      g(P, std::vector<double>(m + 1, 0.0));
  std::vector<int> done_j(P, 0);
  std::vector<double>& coef = S.hcoef;
  // restart cycles: V_0 = r / beta, Arnoldi until every active problem stops
  while (true) {
    bool any = false;
    for (int p = 0; p < P; ++p) any |= act[p] != 0;
    if (!any) break;
    BCKS(set_active(b, act));
    BCK(run_vec<double>(b, right ? S.Vr : S.Vw, kScaleInvSqrt, b->d_dots, cs, 0, 1.0, 0, 0));
    ran = act;
    for (int p = 0; p < P; ++p) {
      if (!act[p]) continue;
      std::fill(g[p].begin(), g[p].end(), 0.0);
      g[p][0] = beta[p];
      done_j[p] = 0;
    }
    for (int j = 0; j < m; ++j) {
      any = false;
      for (int p = 0; p < P; ++p) any |= act[p] != 0;
      if (!any) break;
      if (right) {  // z_j = M^-1 V_j (kept in Z_j), w = A z_j
        BCK(run_vec<double>(b, S.Vcopy, kCopy, nullptr, 0, 0, 0.0, 0, j));
        BCKS(launch_graph(b));
        BCK(run_vec<double>(b, S.xcopyZ, kCopy, nullptr, 0, 0, 0.0, j, 0));
        BCK(run_sweep<double>(b, S.apply_x[j], 0));
        BCK(run_sweep<double>(b, S.apply_y, 2));
      } else {  // w = M^-1 A V_j
        BCK(run_sweep<double>(b, S.apply_x[j], 0));
        BCK(run_sweep<double>(b, S.apply_y, 2));
        BCKS(launch_graph(b));
      }
      for (int i = 0; i <= j; ++i) {  // modified Gram-Schmidt
        BCK(run_dot(b, S.wV, i, 0, i));
        BCK(run_vec<double>(b, S.wV, kAxpyDev, b->d_dots, cs, i, -1.0, 0, i));
      }
      BCK(run_dot(b, S.ww, j + 1));
      BCK(cudaMemcpyAsync(hd.data(), b->d_dots, hd.size() * sizeof(double), cudaMemcpyDeviceToHost,
                          b->st));
      BCK(cudaStreamSynchronize(b->st));
      BCKS(check_status(b));
      bool changed = false;
      for (int p = 0; p < P; ++p) {
        if (!act[p]) continue;
        auto Hij = [&](int i, int jj) -> double& { return H[p][(size_t)i * m + jj]; };
        for (int i = 0; i <= j; ++i) Hij(i, j) = hd[(size_t)p * cs + i];
        const double hn = std::sqrt(hd[(size_t)p * cs + j + 1]);
        Hij(j + 1, j) = hn;
        for (int i = 0; i < j; ++i) {
          const double tt = cn[p][i] * Hij(i, j) + sn[p][i] * Hij(i + 1, j);
          Hij(i + 1, j) = -sn[p][i] * Hij(i, j) + cn[p][i] * Hij(i + 1, j);
          Hij(i, j) = tt;
        }
        const double rho = std::hypot(Hij(j, j), Hij(j + 1, j));
        cn[p][j] = Hij(j, j) / rho;
        sn[p][j] = Hij(j + 1, j) / rho;
        Hij(j, j) = rho;
        Hij(j + 1, j) = 0.0;
        g[p][j + 1] = -sn[p][j] * g[p][j];
        g[p][j] = cn[p][j] * g[p][j];
        done_j[p] = j + 1;
        total[p]++;
        const double est = std::fabs(g[p][j + 1]);
        est_last[p] = est;
        if (!std::isfinite(est)) return berr(BH_ENOCONV, "batched GMRES: non-finite residual");
        const bool ok = est <= rtol * ref[p] || hn == 0.0;
        if (ok || total[p] >= maxit || j + 1 >= m) {
          conv[p] = ok;
          act[p] = 0;
          changed = true;
        }
      }
      if (changed) BCKS(set_active(b, act));
      BCK(run_vec<double>(b, S.Vw, kScaleInvSqrt, b->d_dots, cs, j + 1, 1.0, j + 1, 0));  // V_{j+1}
    }
    // x += (Z | V) y for the problems of this cycle (back substitution on the
    // host), then their true residual r = b - A x in r64_L
    std::fill(coef.begin(), coef.end(), 0.0);
    int jmax = 0;
    for (int p = 0; p < P; ++p) {
      if (!ran[p]) continue;
      const int jd = done_j[p];
      jmax = std::max(jmax, jd);
      for (int i = jd - 1; i >= 0; --i) {
        double sacc = g[p][i];
        for (int jj = i + 1; jj < jd; ++jj) sacc -= H[p][(size_t)i * m + jj] * coef[(size_t)p * cs + jj];
        coef[(size_t)p * cs + i] = sacc / H[p][(size_t)i * m + i];
      }
    }
    BCKS(set_active(b, ran));
    BCK(cudaMemcpyAsync(b->d_coef, coef.data(), coef.size() * sizeof(double), cudaMemcpyHostToDevice,
                        b->st));
    for (int i = 0; i < jmax; ++i) BCK(run_vec<double>(b, S.xV, kAxpyDev, b->d_coef, cs, i, 1.0, 0, i));
    BCK(run_sweep<double>(b, S.resid_x, 0));
    BCK(run_sweep<double>(b, S.resid_y, 2));
    // restart the problems that stopped at the end of the cycle above the tolerance
    std::vector<int> again(P, 0);
    bool any_again = false;
    for (int p = 0; p < P; ++p) {
      again[p] = ran[p] && !conv[p] && total[p] < maxit;
      any_again |= again[p] != 0;
    }
    if (!any_again) break;
    BCKS(set_active(b, again));
    if (right) {
      BCK(run_dot(b, S.rr, 0));
    } else {
      BCK(run_vec<double>(b, S.rcopy, kCopy, nullptr, 0, 0, 0.0));
      BCKS(launch_graph(b));
      BCK(run_dot(b, S.x64dot, 0));
    }
    BCK(cudaMemcpyAsync(hd.data(), b->d_dots, hd.size() * sizeof(double), cudaMemcpyDeviceToHost,
                        b->st));
    BCK(cudaStreamSynchronize(b->st));
    for (int p = 0; p < P; ++p) {
      act[p] = again[p];
      if (!again[p]) continue;
      beta[p] = std::sqrt(hd[(size_t)p * cs]);
      if (!std::isfinite(beta[p])) return berr(BH_ENOCONV, "batched GMRES: non-finite residual");
      if (!(beta[p] > 0.0)) {
        conv[p] = 1;
        act[p] = 0;
      }
    }
  }
  // true relative residuals of every problem that ran (r64_L holds b - A x)
  for (int p = 0; p < P; ++p) act[p] = bnorm[p] > 0.0 ? 1 : 0;
  BCKS(set_active(b, act));
  BCK(run_dot(b, S.rr, 0));
  BCK(cudaMemcpyAsync(hd.data(), b->d_dots, hd.size() * sizeof(double), cudaMemcpyDeviceToHost, b->st));
  BCK(cudaStreamSynchronize(b->st));
  bool all_conv = true;
  b->last_iters = total;
  for (int p = 0; p < P; ++p) {
    iters[p] = total[p];
    relres[p] = bnorm[p] > 0.0 ? std::sqrt(hd[(size_t)p * cs]) / bnorm[p] : 0.0;
    if (bnorm[p] > 0.0 && !conv[p]) all_conv = false;
  }
  BCKS(signal_user(b));
  if (!all_conv) return berr(BH_ENOCONV, "batched GMRES: some problems did not reach the tolerance");
  return BH_OK;
}

bh_status bh_batch_solve_host(bh_batch* b, const double* const* b_host, double* const* x_host,
                              double rtol, int maxit, int* iters, double* relres) {
  if (!b || !b_host || !x_host || !iters || !relres)
    return berr(BH_EINVAL, "bh_batch_solve_host: bad arguments");
  if (b->stage_b.empty()) {
    for (int p = 0; p < b->P; ++p) {
      const size_t bytes = b->ctx[p]->lv[b->L[p]].g.nd * sizeof(double);
      double *db = nullptr, *dx = nullptr;
      if (cudaMalloc(&db, bytes) != cudaSuccess || cudaMalloc(&dx, bytes) != cudaSuccess) {
        cudaFree(db);
        cudaGetLastError();
        return berr(BH_ENOMEM, "staging allocation failed");
      }
      b->allocs.push_back(db);
      b->allocs.push_back(dx);
      b->stage_b.push_back(db);
      b->stage_x.push_back(dx);
    }
  }
  // the copies run on the caller's stream, which bh_batch_solve waits for
  for (int p = 0; p < b->P; ++p)
    BCK(cudaMemcpyAsync(b->stage_b[p], b_host[p], b->ctx[p]->lv[b->L[p]].g.nd * sizeof(double),
                        cudaMemcpyHostToDevice, b->user));
  bh_status s = bh_batch_solve(b, b->stage_b.data(), b->stage_x.data(), rtol, maxit, iters, relres);
  if (s != BH_OK && s != BH_ENOCONV) return s;
  for (int p = 0; p < b->P; ++p)
    BCK(cudaMemcpyAsync(x_host[p], b->stage_x[p], b->ctx[p]->lv[b->L[p]].g.nd * sizeof(double),
                        cudaMemcpyDeviceToHost, b->user));
  BCK(cudaStreamSynchronize(b->user));
  return s;
}

bh_status bh_batch_stats(const bh_batch* b, long long* launches) {
  if (!b || !launches) return berr(BH_EINVAL, "bad arguments");
  *launches = b->launches;
  return BH_OK;
}

}  // extern "C"
