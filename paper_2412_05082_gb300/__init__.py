"""Python binding of libbiharm.so, the GB300 multigrid library for the C0IP
biharmonic problem (arXiv 2412.05082).

Argument marshalling only: every computation runs in the CUDA library behind
the C ABI declared in ``include/biharm.h``; PyTorch supplies device memory and
streams.  There is no CPU fallback -- without the built library (or without a
CUDA device) the calls raise.
"""

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbiharm.so")

# enums of biharm.h
BH_OK, BH_EINVAL, BH_ENOMEM, BH_ECUDA, BH_ENOCONV, BH_ETIMEOUT, BH_EBUSY = 0, -1, -2, -3, -4, -5, -6
BH_ECANCELED = -7
AVS_ATOMIC, AVS_COLORED, MVS_COLORED = 0, 1, 2
FDM, EXACT = 0, 1
FP64, MIXED_FP32, MIXED_FP32_R64, MIXED_FP32_RC = 0, 1, 2, 3
RIGHT, LEFT = 0, 1
COARSE_EXACT, COARSE_SMOOTH = 0, 1
GMRES, CG = 0, 1
RHS_MANUFACTURED, RHS_PAPER_SINE = 0, 1

STATUS_NAMES = {0: "BH_OK", -1: "BH_EINVAL", -2: "BH_ENOMEM", -3: "BH_ECUDA",
                -4: "BH_ENOCONV", -5: "BH_ETIMEOUT", -6: "BH_EBUSY", -7: "BH_ECANCELED"}


class BiharmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("degree", ctypes.c_int), ("level", ctypes.c_int),
                ("gamma", ctypes.c_double), ("smoother", ctypes.c_int),
                ("local_solver", ctypes.c_int), ("pre_steps", ctypes.c_int),
                ("post_steps", ctypes.c_int), ("omega", ctypes.c_double),
                ("precision", ctypes.c_int), ("gmres_restart", ctypes.c_int),
                ("gmres_side", ctypes.c_int), ("coarse", ctypes.c_int),
                ("krylov", ctypes.c_int)]


# every entry point of biharm.h with its ctypes signature
_c = ctypes
_P, _D, _I, _I64 = _c.c_void_p, _c.c_double, _c.c_int, _c.c_int64
SIGNATURES = {
    "bh_default_params": (_I, [_I, _I, _I, _c.POINTER(Params)]),
    "bh_create": (_I, [_c.POINTER(Params), _P, _c.POINTER(_P)]),
    "bh_destroy": (_I, [_P]),
    "bh_num_unknowns": (_I, [_P, _I, _c.POINTER(_I64)]),
    "bh_apply_A": (_I, [_P, _I, _P, _P]),
    "bh_residual": (_I, [_P, _I, _P, _P, _P]),
    "bh_defect_compensated": (_I, [_P, _I, _P, _P, _P]),
    "bh_smooth": (_I, [_P, _I, _P, _P, _I]),
    "bh_smooth_colors": (_I, [_P, _I, _P, _P, _I, _I]),
    "bh_prolongate_add": (_I, [_P, _I, _P, _P]),
    "bh_restrict": (_I, [_P, _I, _P, _P]),
    "bh_vcycle": (_I, [_P, _I, _P, _P]),
    "bh_solve": (_I, [_P, _P, _P, _D, _I, _c.POINTER(_I), _c.POINTER(_D)]),
    "bh_solve_host": (_I, [_P, _P, _P, _D, _I, _c.POINTER(_I), _c.POINTER(_D)]),
    "bh_solve_guess": (_I, [_P, _P, _P, _D, _I, _c.POINTER(_I), _c.POINTER(_D)]),
    "bh_rhs": (_I, [_P, _I, _I, _P]),
    "bh_stats": (_I, [_P, _c.c_char_p, _c.c_size_t]),
    "bh_last_error": (_c.c_char_p, []),
    "bh_kernel_launches": (_c.c_longlong, []),
    "bh_fault_inject_alloc": (_I, [_c.c_longlong, _c.c_longlong]),
    "bh_fp64_fma_rate": (_I, [_P, _c.POINTER(_D)]),
    "bh_fp64_mma_rate": (_I, [_P, _c.POINTER(_D)]),
    "bh_setup_1d": (_I, [_I, _D, _I, _I, _P]),
    "bh_setup_fdm": (_I, [_I, _D, _I, _P, _P]),
    "bh_apply_A_noalloc": (_I, [_I, _I, _I, _D, _P, _P, _P]),
    "bh_batch_create": (_I, [_c.POINTER(Params), _I, _P, _c.POINTER(_P)]),
    "bh_batch_destroy": (_I, [_P]),
    "bh_batch_set_tile": (_I, [_P, _I, _I]),
    "bh_set_tile": (_I, [_P, _I]),
    "bh_batch_vcycle_time": (_I, [_P, _I, _c.POINTER(_D)]),
    "bh_batch_vcycle": (_I, [_P, _P, _P]),
    "bh_batch_set_persistent": (_I, [_P, _I]),
    "bh_batch_check_barrier_timeout": (_I, [_P, _D]),
    "bh_batch_smooth_colors": (_I, [_P, _P, _P, _I, _I]),
    "bh_batch_solve": (_I, [_P, _P, _P, _D, _I, _P, _P]),
    "bh_batch_stats": (_I, [_P, _c.POINTER(_c.c_longlong)]),
    "bh_batch_solve_host": (_I, [_P, _P, _P, _D, _I, _P, _P]),
}

class ServerConfig(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int), ("mem_budget_bytes", ctypes.c_double),
                ("mixed_max_degree", ctypes.c_int), ("rtol", ctypes.c_double),
                ("maxit", ctypes.c_int), ("gmres_restart", ctypes.c_int),
                ("queue_capacity", ctypes.c_int64)]


class ServerResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("relres", ctypes.c_double),
                ("latency_s", ctypes.c_double), ("service_s", ctypes.c_double)]


SIGNATURES.update({
    "bh_server_default_config": (_I, [_c.POINTER(ServerConfig)]),
    "bh_server_create": (_I, [_c.POINTER(ServerConfig), _c.POINTER(_P)]),
    "bh_server_submit": (_I, [_P, _I, _I, _I, _P, _P, _c.POINTER(_I64)]),
    "bh_server_submit_deadline": (_I, [_P, _I, _I, _I, _P, _P, _D, _c.POINTER(_I64)]),
    "bh_server_cancel": (_I, [_P, _I64]),
    "bh_server_wait": (_I, [_P, _I64, _D, _c.POINTER(ServerResult)]),
    "bh_server_stats": (_I, [_P, _c.c_char_p, _c.c_size_t]),
    "bh_server_destroy": (_I, [_P]),
})

_lib = None


def load():
    """Load libbiharm.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise BiharmError(BH_ECUDA, "libbiharm.so is not built (run build.build())")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _check(status):
    if status != BH_OK:
        raise BiharmError(status, load().bh_last_error().decode())
    return status


def default_params(dim, degree, level, **overrides):
    p = Params()
    _check(load().bh_default_params(dim, degree, level, ctypes.byref(p)))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def kernel_launches():
    return int(load().bh_kernel_launches())


def fault_inject_alloc(skip, fail):
    """bh_fault_inject_alloc: after `skip` more device allocations, make the
    next `fail` ones fail with BH_ENOMEM (host-side; (0, 0) switches it off)."""
    _check(load().bh_fault_inject_alloc(int(skip), int(fail)))


def fp64_fma_rate(stream=None):
    """Measured FP64 FMA throughput of the current device (TFLOP/s)."""
    out = ctypes.c_double()
    st = ctypes.c_void_p(stream.cuda_stream if stream is not None else 0)
    _check(load().bh_fp64_fma_rate(st, ctypes.byref(out)))
    return out.value


def fp64_mma_rate(stream=None):
    """Measured FP64 tensor-core (m8n8k4 MMA) throughput of the device (TFLOP/s)."""
    out = ctypes.c_double()
    st = ctypes.c_void_p(stream.cuda_stream if stream is not None else 0)
    _check(load().bh_fp64_mma_rate(st, ctypes.byref(out)))
    return out.value


def last_error():
    return load().bh_last_error().decode()


def setup_1d(degree, gamma, cells, which):
    """Host FP64 1D matrix (0 = M, 1 = L, 2 = B) on `cells` cells of size 1."""
    import numpy as np
    n = degree * cells + 1
    out = np.zeros((n, n))
    _check(load().bh_setup_1d(degree, gamma, cells, which, out.ctypes.data))
    return out


def setup_fdm(degree, gamma, ptype):
    """Host FP64 fast-diagonalization data (S, lambda) of a patch type."""
    import numpy as np
    m = 2 * degree - 1
    S = np.zeros((m, m))
    lam = np.zeros(m)
    _check(load().bh_setup_fdm(degree, gamma, ptype, S.ctypes.data, lam.ctypes.data))
    return S, lam


def apply_A_noalloc(dim, degree, level, gamma, x, y, stream=None):
    """y = A_level x without any device allocation (static scratch array
    shared by all calls: serialize calls that could overlap on the GPU)."""
    import torch
    n = (degree * 2 ** level - 1) ** dim
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(load().bh_apply_A_noalloc(dim, degree, level, gamma, _dev(x, n, "x"),
                                     _dev(y, n, "y"), ctypes.c_void_p(stream.cuda_stream)))


def _dev(t, n, name, dtype=None):
    import torch
    dtype = torch.float64 if dtype is None else dtype
    if not isinstance(t, torch.Tensor) or t.device.type != "cuda":
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype or not t.is_contiguous() or t.numel() != n:
        raise ValueError("%s must be a contiguous %s tensor with %d values" % (name, dtype, n))
    return ctypes.c_void_p(t.data_ptr())


class Context:
    """One multigrid hierarchy (levels 1..L) on the current CUDA device."""

    def __init__(self, params, stream=None):
        import torch
        self.params = params
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        _check(load().bh_create(ctypes.byref(params), ctypes.c_void_p(stream.cuda_stream),
                                ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        if self._h is None:
            raise BiharmError(BH_EINVAL, "context closed")
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None:
            _check(load().bh_destroy(self._h))
            self._h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def num_unknowns(self, level=None):
        """bh_num_unknowns: (k N - 1)^d on `level` (default: the finest)."""
        level = self.params.level if level is None else level
        n = ctypes.c_int64()
        _check(load().bh_num_unknowns(self.handle, level, ctypes.byref(n)))
        return n.value

    def apply_A(self, level, x, y):
        """bh_apply_A: y = A_l x (Eq. (bfc0ip) in the Kronecker form of Sec. 4)."""
        n = self.num_unknowns(level)
        _check(load().bh_apply_A(self.handle, level, _dev(x, n, "x"), _dev(y, n, "y")))

    def residual(self, level, x, b, r):
        """bh_residual: r = b - A_l x."""
        n = self.num_unknowns(level)
        _check(load().bh_residual(self.handle, level, _dev(x, n, "x"), _dev(b, n, "b"),
                                  _dev(r, n, "r")))

    def defect_compensated(self, level, x, b, r):
        """bh_defect_compensated: r = b - A_l x for a float32 x, in compensated
        FP32 arithmetic (mixed-precision contexts)."""
        import torch
        n = self.num_unknowns(level)
        _check(load().bh_defect_compensated(self.handle, level, _dev(x, n, "x", torch.float32),
                                            _dev(b, n, "b"), _dev(r, n, "r")))

    def smooth(self, level, x, b, steps=1):
        """bh_smooth: `steps` steps of the context's smoother (Sec. 3), x in place."""
        n = self.num_unknowns(level)
        _check(load().bh_smooth(self.handle, level, _dev(x, n, "x"), _dev(b, n, "b"), steps))

    def smooth_colors(self, level, x, b, first_color, end_color):
        """Colors first_color .. end_color-1 of one colored MVS step."""
        n = self.num_unknowns(level)
        _check(load().bh_smooth_colors(self.handle, level, _dev(x, n, "x"), _dev(b, n, "b"),
                                       first_color, end_color))

    def prolongate_add(self, level, xc, xf):
        """bh_prolongate_add: xf += P xc, the embedding from level - 1 (Sec. 3)."""
        _check(load().bh_prolongate_add(self.handle, level,
                                        _dev(xc, self.num_unknowns(level - 1), "xc"),
                                        _dev(xf, self.num_unknowns(level), "xf")))

    def restrict(self, level, rf, bc):
        """bh_restrict: bc = P^T rf onto level - 1."""
        _check(load().bh_restrict(self.handle, level, _dev(rf, self.num_unknowns(level), "rf"),
                                  _dev(bc, self.num_unknowns(level - 1), "bc")))

    def vcycle(self, level, x, b):
        """bh_vcycle: x = MG_level(x, b), Algorithm 1."""
        n = self.num_unknowns(level)
        _check(load().bh_vcycle(self.handle, level, _dev(x, n, "x"), _dev(b, n, "b")))

    def set_tile(self, patches_per_block):
        """Patches per block of the fused MVS kernels (0: automatic)."""
        _check(load().bh_set_tile(self._h, int(patches_per_block)))

    def solve(self, b, x, rtol=1e-8, maxit=200, raise_on_noconv=True):
        """bh_solve: x = A^-1 b by the context's Krylov method preconditioned by
        one V-cycle (Sec. 5.1), from x = 0; returns (iterations, true relres)."""
        n = self.num_unknowns()
        it, rr = ctypes.c_int(), ctypes.c_double()
        st = load().bh_solve(self.handle, _dev(b, n, "b"), _dev(x, n, "x"), rtol, maxit,
                             ctypes.byref(it), ctypes.byref(rr))
        if st != BH_ENOCONV or raise_on_noconv:
            _check(st)
        return it.value, rr.value

    def solve_guess(self, b, x, rtol=1e-8, maxit=200, raise_on_noconv=True):
        """bh_solve starting from the guess in x (x is updated in place)."""
        n = self.num_unknowns()
        it, rr = ctypes.c_int(), ctypes.c_double()
        st = load().bh_solve_guess(self.handle, _dev(b, n, "b"), _dev(x, n, "x"), rtol, maxit,
                                   ctypes.byref(it), ctypes.byref(rr))
        if st != BH_ENOCONV or raise_on_noconv:
            _check(st)
        return it.value, rr.value

    def solve_host(self, b, x, rtol=1e-8, maxit=200):
        """b, x: host float64 arrays (numpy or CPU tensors, contiguous)."""
        import numpy as np
        n = self.num_unknowns()
        for a in (b, x):
            arr = a.numpy() if hasattr(a, "numpy") else a
            if arr.dtype != np.float64 or arr.size != n or not arr.flags.c_contiguous:
                raise ValueError("host buffers must be contiguous float64 with %d values" % n)
        pb = (b.numpy() if hasattr(b, "numpy") else b).ctypes.data
        px = (x.numpy() if hasattr(x, "numpy") else x).ctypes.data
        it, rr = ctypes.c_int(), ctypes.c_double()
        _check(load().bh_solve_host(self.handle, pb, px, rtol, maxit, ctypes.byref(it),
                                    ctypes.byref(rr)))
        return it.value, rr.value

    def rhs(self, level, kind, b):
        """bh_rhs: the load vector of RHS_MANUFACTURED or RHS_PAPER_SINE on `level`."""
        _check(load().bh_rhs(self.handle, level, kind, _dev(b, self.num_unknowns(level), "b")))

    def stats(self):
        """bh_stats as a dict (counters, last_iters, last_relres, last_estimate,
        last_solve_ms)."""
        import json
        buf = ctypes.create_string_buffer(4096)
        _check(load().bh_stats(self.handle, buf, len(buf)))
        return json.loads(buf.value.decode())


class Batch:
    """Many independent 2D problems solved together (batched form): one launch
    per level operation over all problems, the lockstep V-cycle as a CUDA
    graph (FP64, or FP32 with FP64 defects), lockstep GMRES (left, or right
    in the flexible form) with restarts."""

    def __init__(self, params_list, stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.params = list(params_list)
        arr = (Params * len(self.params))(*self.params)
        h = ctypes.c_void_p()
        _check(load().bh_batch_create(arr, len(self.params), ctypes.c_void_p(stream.cuda_stream),
                                      ctypes.byref(h)))
        self._h = h

    def sizes(self):
        """Unknowns of each problem's finest level, in the batch's order."""
        return [(p.degree * 2 ** p.level - 1) ** p.dim for p in self.params]

    def close(self):
        if getattr(self, "_h", None) is not None:
            _check(load().bh_batch_destroy(self._h))
            self._h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_tile(self, degree, patches_per_block):
        """bh_batch_set_tile: patches per block of the fused MVS launch of one degree."""
        _check(load().bh_batch_set_tile(self._h, degree, patches_per_block))

    def set_persistent(self, on=True):
        """bh_batch_set_persistent: the V-cycle as one cooperative launch (True)
        or as the captured graph (False, the default)."""
        _check(load().bh_batch_set_persistent(self._h, 1 if on else 0))

    def check_barrier_timeout(self, wait_ms=50.0):
        """bh_batch_check_barrier_timeout: the persistent kernel's bounded
        barrier wait made to run out; returns the status code (BH_ETIMEOUT)."""
        return load().bh_batch_check_barrier_timeout(self._h, float(wait_ms))

    def vcycle_time(self, reps=5):
        """bh_batch_vcycle_time: device time (ms) of one replay of the batch's V-cycle graph."""
        ms = ctypes.c_double()
        _check(load().bh_batch_vcycle_time(self._h, reps, ctypes.byref(ms)))
        return ms.value

    def _ptrs(self, vs, name):
        sizes = self.sizes()
        if len(vs) != len(sizes):
            raise ValueError("%s: one vector per problem (%d)" % (name, len(sizes)))
        arr = (ctypes.c_void_p * len(sizes))(*[_dev(v, n, name).value for v, n in zip(vs, sizes)])
        return ctypes.cast(arr, ctypes.c_void_p), arr

    def vcycle(self, bs, xs):
        """bh_batch_vcycle: xs[i] = MG_L(0, bs[i]) (Algorithm 1) for every problem,
        by the batch's captured V-cycle graph in its precision."""
        bp, keep_b = self._ptrs(bs, "b")
        xp, keep_x = self._ptrs(xs, "x")
        _check(load().bh_batch_vcycle(self._h, bp, xp))

    def smooth_colors(self, xs, bs, first_color, end_color):
        """bh_batch_smooth_colors: colors first_color .. end_color-1 of one
        colored MVS step on every problem's finest level, xs in place."""
        xp, keep_x = self._ptrs(xs, "x")
        bp, keep_b = self._ptrs(bs, "b")
        _check(load().bh_batch_smooth_colors(self._h, xp, bp, first_color, end_color))

    def launches(self):
        """bh_batch_stats: kernel and graph launches the batch has issued so far."""
        n = ctypes.c_longlong()
        _check(load().bh_batch_stats(self._h, ctypes.byref(n)))
        return n.value

    def solve_host(self, bs, xs, rtol=1e-8, maxit=200):
        """bs, xs: contiguous float64 host arrays (numpy or CPU tensors)."""
        import numpy as np
        P = len(self.params)
        arrs = []
        for a, n in zip(list(bs) + list(xs), self.sizes() * 2):
            arr = a.numpy() if hasattr(a, "numpy") else a
            if arr.dtype != np.float64 or arr.size != n or not arr.flags.c_contiguous:
                raise ValueError("host buffers must be contiguous float64 arrays of the right size")
            arrs.append(arr)
        bp = (ctypes.c_void_p * P)(*[a.ctypes.data for a in arrs[:P]])
        xp = (ctypes.c_void_p * P)(*[a.ctypes.data for a in arrs[P:]])
        it = (ctypes.c_int * P)()
        rr = (ctypes.c_double * P)()
        _check(load().bh_batch_solve_host(self._h, ctypes.cast(bp, ctypes.c_void_p),
                                          ctypes.cast(xp, ctypes.c_void_p), rtol, maxit,
                                          ctypes.cast(it, ctypes.c_void_p),
                                          ctypes.cast(rr, ctypes.c_void_p)))
        return list(it), list(rr)

    def solve(self, bs, xs, rtol=1e-8, maxit=200, raise_on_noconv=True):
        """bh_batch_solve on device tensors; returns per-problem iterations and
        true relative residuals."""
        P = len(self.params)
        sizes = self.sizes()
        bp = (ctypes.c_void_p * P)(*[_dev(b, n, "b").value for b, n in zip(bs, sizes)])
        xp = (ctypes.c_void_p * P)(*[_dev(x, n, "x").value for x, n in zip(xs, sizes)])
        it = (ctypes.c_int * P)()
        rr = (ctypes.c_double * P)()
        st = load().bh_batch_solve(self._h, ctypes.cast(bp, ctypes.c_void_p),
                                   ctypes.cast(xp, ctypes.c_void_p), rtol, maxit,
                                   ctypes.cast(it, ctypes.c_void_p), ctypes.cast(rr, ctypes.c_void_p))
        if st != BH_ENOCONV or raise_on_noconv:
            _check(st)
        return list(it), list(rr)


class Server:
    """Continuous-batching solve server (resident hierarchies, admission by
    device-memory footprint, overlapping solves on several slots)."""

    def __init__(self, **cfg):
        c = ServerConfig()
        _check(load().bh_server_default_config(ctypes.byref(c)))
        for k, v in cfg.items():
            if not hasattr(c, k):
                raise KeyError(k)
            setattr(c, k, v)
        self.config = c
        h = ctypes.c_void_p()
        _check(load().bh_server_create(ctypes.byref(c), ctypes.byref(h)))
        self._h = h
        self._keep = {}

    def submit(self, dim, degree, level, b, x, deadline=0.0):
        """b, x: contiguous float64 numpy arrays (kept alive until wait);
        deadline: seconds after which a request that has not started is
        dropped (bh_server_submit_deadline; 0: none)."""
        import numpy as np
        n = (degree * 2 ** level - 1) ** dim
        for a in (b, x):
            if not isinstance(a, np.ndarray) or a.dtype != np.float64 or a.size != n \
                    or not a.flags.c_contiguous:
                raise ValueError("b and x must be contiguous float64 arrays with %d values" % n)
        t = ctypes.c_int64()
        _check(load().bh_server_submit_deadline(self._h, dim, degree, level, b.ctypes.data,
                                                x.ctypes.data, float(deadline), ctypes.byref(t)))
        self._keep[t.value] = (b, x)
        return t.value

    def cancel(self, ticket):
        """bh_server_cancel: drop a queued request (BiharmError BH_EBUSY once it
        has started)."""
        _check(load().bh_server_cancel(self._h, ticket))

    def wait(self, ticket, timeout=-1.0):
        """bh_server_wait: the request's status, iterations, relres and latencies
        (timeout in seconds, < 0: no limit)."""
        r = ServerResult()
        _check(load().bh_server_wait(self._h, ticket, timeout, ctypes.byref(r)))
        self._keep.pop(ticket, None)
        return {"status": r.status, "iters": r.iters, "relres": r.relres,
                "latency_s": r.latency_s, "service_s": r.service_s}

    def stats(self):
        """bh_server_stats as a dict: queue, slot and memory counters (admitted,
        completed, created, evictions, reserved and budget bytes, busy time)."""
        import json
        buf = ctypes.create_string_buffer(4096)
        _check(load().bh_server_stats(self._h, buf, len(buf)))
        return json.loads(buf.value.decode())

    def close(self):
        if getattr(self, "_h", None) is not None:
            _check(load().bh_server_destroy(self._h))
            self._h = None
            self._keep.clear()

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
