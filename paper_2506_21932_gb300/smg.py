"""Python binding of the C ABI in include/smg.h (argument marshalling only).

Every numerical step runs in libsmg.so's CUDA kernels.  PyTorch supplies
device memory and streams: tensors are passed by ``data_ptr()`` and the
current CUDA stream by its handle.  If the shared library has not been built,
every call raises instead of falling back to anything else.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsmg.so")

OK, EINVAL, ENOMEM, ECUDA, EBREAKDOWN, ENOTCONV, ENAN, ETIMEOUT = range(8)
SGS, ILU0, LGS = 0, 1, 2
FW27V, PC8C, C64C, C16XY = 0, 1, 2, 3
FP64, FP32, BF16 = 0, 1, 2
PCG, FPCG, FGMRES = 0, 1, 2
LEARNED_AFTER, LEARNED_REPLACE = 0, 1
OP_SPMV, OP_RESIDUAL, OP_GS_FORWARD, OP_GS_BACKWARD, OP_GS_ZERO, OP_ILU_APPLY, OP_RESTRICT, OP_PROLONG_ADD, \
    OP_COARSE_SOLVE, OP_ILU_LOWER, OP_ILU_UPPER, OP_LGS_FORWARD, OP_LGS_BACKWARD, OP_LGS_ZERO = range(14)
ARR_A, ARR_LU, ARR_DINV, ARR_AV, ARR_AS, ARR_LUV, ARR_LS, ARR_US, ARR_DINV32 = range(9)
LOSS_ERROR, LOSS_RESIDUAL = 0, 1

_lib = None


class SmgError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__("%s failed: %s (status %d)" % (what, strerror(status), status))


class Options(ctypes.Structure):
    _fields_ = [("smoother", ctypes.c_int), ("transfer", ctypes.c_int), ("precision", ctypes.c_int),
                ("krylov", ctypes.c_int), ("restart", ctypes.c_int), ("relax_w", ctypes.c_double),
                ("max_levels", ctypes.c_int), ("spin_budget_ms", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("fuse_restrict", ctypes.c_int), ("sweep_warps", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("dims", (ctypes.c_int * 3) * 16), ("nstencil", ctypes.c_int * 16),
                ("grid_complexity", ctypes.c_double), ("operator_complexity", ctypes.c_double),
                ("vcycle_bytes", ctypes.c_double), ("vcycle_fp64_flops", ctypes.c_double),
                ("setup_ms", ctypes.c_double), ("precision", ctypes.c_int), ("smoother", ctypes.c_int),
                ("transfer", ctypes.c_int), ("block", ctypes.c_int)]


def lib():
    """Load libsmg.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libsmg.so is not built; run __graft_entry__.build() or "
                               "python paper_2506_21932_gb300/build.py")
        L = ctypes.CDLL(LIB_PATH)
        vp, ip, i, d = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_double
        L.smg_setup.argtypes = [ctypes.POINTER(vp), ip, i, ip, vp, i, ctypes.POINTER(Options), vp]
        L.smg_vcycle.argtypes = [vp, vp, vp, vp]
        L.smg_solve.argtypes = [vp, vp, vp, d, i, ip, ctypes.POINTER(d), vp]
        L.smg_stats.argtypes = [vp, ctypes.POINTER(Stats)]
        L.smg_destroy.argtypes = [vp]
        L.smg_destroy.restype = None
        L.smg_strerror.argtypes = [i]
        L.smg_strerror.restype = ctypes.c_char_p
        L.smg_level_count.argtypes = [vp]
        L.smg_level_info.argtypes = [vp, i, ip, ip, ip]
        L.smg_level_sweep_warps.argtypes = [vp, i, i]
        L.smg_level_copy.argtypes = [vp, i, i, vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t), vp]
        L.smg_level_apply.argtypes = [vp, i, i, vp, vp, vp, vp]
        L.smg_derive_chains.argtypes = [i, i, ip, i, ip, i, ip, i, ip]
        L.smg_rap_chain_count.argtypes = [i, i, ip, ip]
        L.smg_version.restype = ctypes.c_char_p
        L.smg_launch_count.restype = ctypes.c_longlong
        L.smg_selftest_wait.argtypes = [vp, i, vp]
        L.smg_set_wait_budget_ns.argtypes = [vp, ctypes.c_longlong]
        L.smg_vcycle_profile.argtypes = [vp, vp, vp, i, ip, ip, ip, ctypes.POINTER(ctypes.c_float), vp]
        L.smg_sweep_noalloc.argtypes = [i, ip, i, ip, vp, vp, vp, vp, d, i, vp]
        sz = ctypes.c_size_t
        f = ctypes.c_float
        L.smg_cnn_workspace_bytes.argtypes = [ip, ctypes.POINTER(sz)]
        L.smg_cnn_forward.argtypes = [ip, vp, vp, vp, vp, sz, vp]
        L.smg_cnn_loss_grad.argtypes = [ip, vp, vp, vp, vp, vp, vp, sz, vp]
        L.smg_cnn_adam.argtypes = [i, vp, vp, vp, vp, i, f, f, f, f, f, vp]
        L.smg_set_learned_smoother.argtypes = [vp, vp, vp, vp]
        L.smg_set_learned_mode.argtypes = [vp, ctypes.c_int]
        L.smg_learned_sample.argtypes = [vp, vp, vp, vp, vp, vp]
        L.smg_learned_loss_grad.argtypes = [vp, vp, vp, vp, i, vp, vp, vp, ctypes.c_size_t, vp]
        _lib = L
    return _lib


# ---- learned post-smoother network (FP32 tensors on the device) ------------

def cnn_param_count():
    return int(lib().smg_cnn_param_count())


def cnn_workspace(dims):
    """Allocates (through torch) the device workspace the network needs."""
    import torch
    nb = ctypes.c_size_t(0)
    rc = lib().smg_cnn_workspace_bytes(_iarr(dims), ctypes.byref(nb))
    if rc != OK:
        raise SmgError(rc, "smg_cnn_workspace_bytes")
    return torch.empty(nb.value, dtype=torch.uint8, device="cuda")


def cnn_forward(dims, theta, in2, out, ws, stream=None):
    rc = lib().smg_cnn_forward(_iarr(dims), _ptr(theta), _ptr(in2), _ptr(out), _ptr(ws), ws.numel(), _stream(stream))
    if rc != OK:
        raise SmgError(rc, "smg_cnn_forward")


def cnn_loss_grad(dims, theta, in2, target, grad, loss, ws, stream=None):
    rc = lib().smg_cnn_loss_grad(_iarr(dims), _ptr(theta), _ptr(in2), _ptr(target), _ptr(grad), _ptr(loss), _ptr(ws),
                                 ws.numel(), _stream(stream))
    if rc != OK:
        raise SmgError(rc, "smg_cnn_loss_grad")


def cnn_adam(theta, m, v, grad, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, grad_scale=1.0, stream=None):
    rc = lib().smg_cnn_adam(theta.numel(), _ptr(theta), _ptr(m), _ptr(v), _ptr(grad), step, lr, beta1, beta2, eps,
                            grad_scale, _stream(stream))
    if rc != OK:
        raise SmgError(rc, "smg_cnn_adam")


def sweep_noalloc(op, dims, offsets, M, dinv, b, u, relax_w=1.0, spin_budget_ms=0, stream=None):
    """One GS or ILU(0) sweep through smg_sweep_noalloc, the entry point that
    allocates no device memory (for callers whose device memory is owned by
    someone else).  Tensors are float64 CUDA tensors; returns the status."""
    import torch
    n = int(dims[0]) * int(dims[1]) * int(dims[2])
    for name, t, count in (("M", M, n * len(offsets)), ("dinv", dinv, n), ("b", b, n), ("u", u, n)):
        if t is None:
            continue  # passed as NULL: the library decides whether the op needs it
        if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous() or t.numel() != count:
            raise ValueError("sweep_noalloc: %s must be a contiguous float64 CUDA tensor of %d values, got %s %s "
                             "with %d values" % (name, count, t.dtype, t.device, t.numel()))
    flat = [c for o in offsets for c in o]
    return lib().smg_sweep_noalloc(op, _iarr(dims), len(offsets), _iarr(flat), _ptr(M), _ptr(dinv), _ptr(b),
                                   _ptr(u), relax_w, spin_budget_ms, _stream(stream))


def launch_count():
    """Kernels enqueued by libsmg.so since it was loaded."""
    return int(lib().smg_launch_count())


def strerror(status):
    try:
        return lib().smg_strerror(int(status)).decode()
    except RuntimeError:
        return "status %d" % status


def _iarr(vals):
    vals = [int(v) for v in vals]
    return (ctypes.c_int * max(1, len(vals)))(*vals)


def derive_chains(roff, aoff, poff, dim=3):
    """Host-only symbolic chain derivation; returns a list of (r, a, q, dJ)."""
    L = lib()
    flat = lambda offs: _iarr([c for o in offs for c in (list(o) + [0] * (3 - len(o)))])
    ro, ao, po = flat(roff), flat(aoff), flat(poff)
    n = L.smg_derive_chains(dim, len(roff), ro, len(aoff), ao, len(poff), po, 0, None)
    if n < 0:
        raise ValueError("chain derivation failed")
    buf = (ctypes.c_int * (5 * max(1, n)))()
    L.smg_derive_chains(dim, len(roff), ro, len(aoff), ao, len(poff), po, n, buf)
    return [tuple(buf[5 * t:5 * t + 4]) for t in range(n)]


def rap_chain_count(transfer, offsets):
    """Host-only: (chains, coarse mask size) of the set-up's Galerkin chain table."""
    L = lib()
    nc = ctypes.c_int(0)
    n = L.smg_rap_chain_count(transfer, len(offsets), _iarr([c for o in offsets for c in o]), ctypes.byref(nc))
    if n < 0:
        raise ValueError("no chain table for this transfer / mask")
    return n, nc.value


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


class SMG:
    """A structured-multigrid hierarchy living on the current CUDA device."""

    def __init__(self, dims, offsets, coeffs, block=1, smoother=SGS, transfer=FW27V, precision=FP64,
                 krylov=PCG, restart=30, relax_w=1.0, max_levels=0, spin_budget_ms=0, use_graph=0, fuse_restrict=0,
                 sweep_warps=0, stream=None):
        import torch
        if not (coeffs.is_cuda and coeffs.dtype == torch.float64 and coeffs.is_contiguous()):
            raise ValueError("coeffs must be a contiguous float64 CUDA tensor")
        self._lib = lib()
        self.dims = tuple(int(t) for t in dims)
        self.block = int(block)
        self.n = self.dims[0] * self.dims[1] * self.dims[2]
        self.precision = precision
        opt = Options(smoother, transfer, precision, krylov, restart, relax_w, max_levels, spin_budget_ms, use_graph,
                      fuse_restrict, sweep_warps)
        offs = [c for o in offsets for c in o]
        h = ctypes.c_void_p()
        rc = self._lib.smg_setup(ctypes.byref(h), _iarr(self.dims), len(offsets), _iarr(offs),
                                 ctypes.c_void_p(coeffs.data_ptr()), self.block, ctypes.byref(opt), _stream(stream))
        if rc != OK:
            raise SmgError(rc, "smg_setup")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self._lib.smg_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def vcycle(self, r, z, stream=None):
        rc = self._lib.smg_vcycle(self.h, _ptr(r), _ptr(z), _stream(stream))
        if rc != OK:
            raise SmgError(rc, "smg_vcycle")

    def solve(self, b, x, tol=1e-9, maxit=500, stream=None, check=True):
        it, rr = ctypes.c_int(0), ctypes.c_double(0.0)
        rc = self._lib.smg_solve(self.h, _ptr(b), _ptr(x), tol, maxit, ctypes.byref(it), ctypes.byref(rr),
                                 _stream(stream))
        if check and rc != OK:
            raise SmgError(rc, "smg_solve")
        return it.value, rr.value, rc

    def stats(self):
        s = Stats()
        rc = self._lib.smg_stats(self.h, ctypes.byref(s))
        if rc != OK:
            raise SmgError(rc, "smg_stats")
        return {"levels": s.levels, "dims": [tuple(s.dims[l]) for l in range(s.levels)],
                "nstencil": [s.nstencil[l] for l in range(s.levels)], "grid_complexity": s.grid_complexity,
                "operator_complexity": s.operator_complexity, "vcycle_bytes": s.vcycle_bytes,
                "vcycle_fp64_flops": s.vcycle_fp64_flops, "setup_ms": s.setup_ms}

    @property
    def nlevels(self):
        return self._lib.smg_level_count(self.h)

    def level_info(self, l):
        d = (ctypes.c_int * 3)()
        ns = ctypes.c_int()
        off = (ctypes.c_int * 81)()
        rc = self._lib.smg_level_info(self.h, l, d, ctypes.byref(ns), off)
        if rc != OK:
            raise SmgError(rc, "smg_level_info")
        return tuple(d), [tuple(off[3 * e:3 * e + 3]) for e in range(ns.value)]

    def level_sweep_warps(self, l, op):
        """Warps per strip of the kernel running sweep `op` on level l (0: another kernel)."""
        rc = self._lib.smg_level_sweep_warps(self.h, l, op)
        if rc < 0:
            raise SmgError(-rc, "smg_level_sweep_warps")
        return rc

    def level_array(self, l, which, stream=None):
        """Copies a level array into a new uint8 CUDA tensor and returns it."""
        import torch
        need = ctypes.c_size_t(0)
        rc = self._lib.smg_level_copy(self.h, l, which, None, 0, ctypes.byref(need), _stream(stream))
        if rc != OK:
            raise SmgError(rc, "smg_level_copy")
        out = torch.empty(need.value, dtype=torch.uint8, device="cuda")
        rc = self._lib.smg_level_copy(self.h, l, which, ctypes.c_void_p(out.data_ptr()), need.value, None,
                                      _stream(stream))
        if rc != OK:
            raise SmgError(rc, "smg_level_copy")
        return out

    def level_apply(self, l, op, x=None, b=None, y=None, stream=None):
        rc = self._lib.smg_level_apply(self.h, l, op, _ptr(x), _ptr(b), _ptr(y), _stream(stream))
        if rc != OK:
            raise SmgError(rc, "smg_level_apply")

    def set_learned_smoother(self, theta, logk, stream=None):
        """Attach (theta: FP32 [8241], logk: float64 [n]) or detach (None)."""
        self._ls = (theta, logk)  # keep the tensors alive while attached
        rc = self._lib.smg_set_learned_smoother(self.h, _ptr(theta), _ptr(logk), _stream(stream))
        if rc != OK:
            raise SmgError(rc, "smg_set_learned_smoother")

    def set_learned_mode(self, mode):
        """LEARNED_AFTER (the network after the V-cycle) or LEARNED_REPLACE
        (in place of the finest level's post-smoothing)."""
        rc = self._lib.smg_set_learned_mode(self.h, int(mode))
        if rc != OK:
            raise SmgError(rc, "smg_set_learned_mode")

    def learned_sample(self, e0, logk, in2, target, stream=None):
        """One training pair from a known error e0 (see smg_learned_sample)."""
        rc = self._lib.smg_learned_sample(self.h, _ptr(e0), _ptr(logk), _ptr(in2), _ptr(target), _stream(stream))
        if rc != OK:
            raise SmgError(rc, "smg_learned_sample")

    def learned_loss_grad(self, theta, in2, target, grad, loss, ws, kind=1, stream=None):
        """Accumulates the loss (LOSS_ERROR or LOSS_RESIDUAL) and its gradient
        for one training pair on this hierarchy's finest grid."""
        rc = self._lib.smg_learned_loss_grad(self.h, _ptr(theta), _ptr(in2), _ptr(target), int(kind), _ptr(grad),
                                             _ptr(loss), _ptr(ws), ws.numel(), _stream(stream))
        if rc != OK:
            raise SmgError(rc, "smg_learned_loss_grad")

    STAGES = {1: "pre1", 2: "pre2", 3: "residual", 4: "restrict", 5: "coarse", 6: "prolong", 7: "post_residual",
              8: "post1", 9: "post2", 10: "post_add", 11: "cast", 12: "learned", 13: "pack", 14: "unpack"}

    def vcycle_profile(self, r, z, stream=None):
        """One eager V-cycle with an event after every stage; returns a list of
        (level, stage name, device ms)."""
        cap = 512
        cnt = ctypes.c_int()
        lv, sg = (ctypes.c_int * cap)(), (ctypes.c_int * cap)()
        ms = (ctypes.c_float * cap)()
        rc = self._lib.smg_vcycle_profile(self.h, _ptr(r), _ptr(z), cap, ctypes.byref(cnt), lv, sg, ms,
                                          _stream(stream))
        if rc != OK:
            raise SmgError(rc, "smg_vcycle_profile")
        return [(lv[t], self.STAGES.get(sg[t], str(sg[t])), float(ms[t])) for t in range(min(cnt.value, cap))]

    def set_wait_budget_ns(self, budget_ns):
        """Bound of every device wait of this context, in ns (0: give up at once)."""
        rc = self._lib.smg_set_wait_budget_ns(self.h, int(budget_ns))
        if rc != OK:
            raise SmgError(rc, "smg_set_wait_budget_ns")

    def selftest_wait(self, budget_ms=20, stream=None):
        """Runs one bounded device wait that must time out; returns the status."""
        return self._lib.smg_selftest_wait(self.h, budget_ms, _stream(stream))
