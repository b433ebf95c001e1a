"""ctypes front-end of the plain C FP64 oracle (smg_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the package smoke check and
by the benchmark's CPU-baseline leg, never by the product path.  The shared
library is compiled from source with gcc on first use (or by ``build()``).
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "smg_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None

ORC_OK, ORC_EINVAL, ORC_ENOMEM, ORC_EBREAKDOWN, ORC_ENOTCONV, ORC_ENAN = 0, 1, 2, 4, 5, 6
SGS, ILU0, LGS = 0, 1, 2
FW27V, PC8C, C64C, C16XY = 0, 1, 2, 3
FP64, FP32, BF16 = 0, 1, 2


def build(force=False):
    """Compile liboracle.so (plain C, -O2, no FMA contraction).  The Galerkin
    product's independent coarse points run on OpenMP threads when the
    compiler supports it; otherwise the same source builds serially."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        base = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
        if subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True).returncode != 0:
            subprocess.check_call(base)
        os.replace(tmp, _SO)
    return _SO


def set_threads(n):
    """Threads of the oracle's parallel loops (the benchmark times it on 1)."""
    lib().orc_set_threads(int(n))


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_SO)
        _lib.orc_bf16_round.restype = ctypes.c_float
        _lib.orc_bf16_round.argtypes = [ctypes.c_double]
        _lib.orc_mg_level_array.restype = ctypes.c_long
        _lib.orc_mg_free.argtypes = [ctypes.c_void_p]
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _i3(d):
    return np.ascontiguousarray(np.asarray(d, dtype=np.int32).reshape(3))


def _offs(off):
    return np.ascontiguousarray(np.asarray(off, dtype=np.int32).reshape(-1, 3))


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def npts(d):
    return int(d[0]) * int(d[1]) * int(d[2])


def mask_validate(off):
    o = _offs(off)
    return lib().orc_mask_validate(len(o), _p(o))


def spmv(d, off, A, x, B=1):
    d, o, A, x = _i3(d), _offs(off), _f64(A), _f64(x)
    y = np.zeros(npts(d) * B)
    lib().orc_spmv(_p(d), len(o), _p(o), B, _p(A), _p(x), _p(y))
    return y


def residual(d, off, A, b, x, B=1):
    d, o, A, b, x = _i3(d), _offs(off), _f64(A), _f64(b), _f64(x)
    r = np.zeros(npts(d) * B)
    lib().orc_residual(_p(d), len(o), _p(o), B, _p(A), _p(b), _p(x), _p(r))
    return r


def diag_inverse(d, off, A, B=1):
    d, o, A = _i3(d), _offs(off), _f64(A)
    D = np.zeros(npts(d) * B * B)
    rc = lib().orc_diag_inverse(_p(d), len(o), _p(o), B, _p(A), _p(D))
    if rc:
        raise ArithmeticError("zero diagonal")
    return D


def gs_forward(d, off, A, Dinv, b, u, w=1.0, B=1):
    d, o, A, Dinv, b = _i3(d), _offs(off), _f64(A), _f64(Dinv), _f64(b)
    u = _f64(u).copy()
    lib().orc_gs_forward(_p(d), len(o), _p(o), B, _p(A), _p(Dinv), _p(b), _p(u), ctypes.c_double(w))
    return u


def gs_backward(d, off, A, Dinv, b, u, w=1.0, B=1):
    d, o, A, Dinv, b = _i3(d), _offs(off), _f64(A), _f64(Dinv), _f64(b)
    u = _f64(u).copy()
    lib().orc_gs_backward(_p(d), len(o), _p(o), B, _p(A), _p(Dinv), _p(b), _p(u), ctypes.c_double(w))
    return u


def lgs_forward(d, off, A, b, u):
    d, o, A, b = _i3(d), _offs(off), _f64(A), _f64(b)
    u = _f64(u).copy()
    lib().orc_lgs_forward(_p(d), len(o), _p(o), _p(A), _p(b), _p(u))
    return u


def lgs_backward(d, off, A, b, u):
    d, o, A, b = _i3(d), _offs(off), _f64(A), _f64(b)
    u = _f64(u).copy()
    lib().orc_lgs_backward(_p(d), len(o), _p(o), _p(A), _p(b), _p(u))
    return u


def lgs_check(d, off, A, spd_check=True):
    d, o, A = _i3(d), _offs(off), _f64(A)
    return lib().orc_lgs_check(_p(d), len(o), _p(o), _p(A), int(spd_check))


def ilu0_factor(d, off, A, spd_check=True):
    d, o, A = _i3(d), _offs(off), _f64(A)
    LU = np.zeros_like(A)
    rc = lib().orc_ilu0_factor(_p(d), len(o), _p(o), _p(A), _p(LU), int(spd_check))
    if rc:
        raise ArithmeticError("ILU(0) breakdown")
    return LU


def ilu0_apply(d, off, LU, Udinv, r):
    d, o, LU, Udinv, r = _i3(d), _offs(off), _f64(LU), _f64(Udinv), _f64(r)
    x = np.zeros_like(r)
    lib().orc_ilu0_apply(_p(d), len(o), _p(o), _p(LU), _p(Udinv), _p(r), _p(x))
    return x


def coarse_dims(d, transfer=0):
    """Coarse grid: every dimension halved (z kept by the x-y semi-coarsening, transfer 3)."""
    return [int(t) if (transfer == 3 and a == 2) else int(t) // 2 for a, t in enumerate(d)]


def restrict(transfer, fd, rf, B=1):
    fd, rf = _i3(fd), _f64(rf)
    fc = np.zeros(npts(coarse_dims(fd, transfer)) * B)
    lib().orc_restrict(transfer, _p(fd), B, _p(rf), _p(fc))
    return fc


def prolong_add(transfer, fd, ec, uf, B=1):
    fd, ec = _i3(fd), _f64(ec)
    uf = _f64(uf).copy()
    lib().orc_prolong_add(transfer, _p(fd), B, _p(ec), _p(uf))
    return uf


def rap27(transfer, fd, off, Af, B=1):
    """Brute-force Galerkin product.  Returns (Ac27 [nc,27,B,B], present[27])."""
    fd, o, Af = _i3(fd), _offs(off), _f64(Af)
    nc = npts(coarse_dims(fd, transfer))
    Ac = np.zeros(nc * 27 * B * B)
    present = np.zeros(27, dtype=np.int32)
    rc = lib().orc_rap27(transfer, _p(fd), len(o), _p(o), B, _p(Af), _p(Ac), _p(present))
    if rc:
        raise ValueError("coarse offset outside {-1,0,1}^3")
    return Ac.reshape(nc, 27, B, B), present


def rap27_at(transfer, fd, off, Af, points, B=1):
    """Brute-force Galerkin coefficients of the listed coarse points only:
    returns [len(points), 27, B, B] (all 27 offsets, lexicographic)."""
    fd, o, Af = _i3(fd), _offs(off), _f64(Af)
    pts = np.ascontiguousarray(np.asarray(points, dtype=np.int64))
    out = np.zeros(len(pts) * 27 * B * B)
    rc = lib().orc_rap27_at(transfer, _p(fd), len(o), _p(o), B, _p(Af), ctypes.c_long(len(pts)), _p(pts), _p(out))
    if rc:
        raise ValueError("coarse offset outside {-1,0,1}^3")
    return out.reshape(len(pts), 27, B, B)


def assemble_dense(d, off, A, B=1):
    d, o, A = _i3(d), _offs(off), _f64(A)
    n = npts(d) * B
    M = np.zeros((n, n))
    lib().orc_assemble_dense(_p(d), len(o), _p(o), B, _p(A), _p(M))
    return M


def bf16_round(x):
    return lib().orc_bf16_round(float(x))


def plan_levels(d, max_levels=16, transfer=0):
    d = _i3(d)
    out = np.zeros((16, 3), dtype=np.int32)
    L = lib().orc_plan_levels_t(transfer, _p(d), max_levels, _p(out))
    return [tuple(int(t) for t in out[l]) for l in range(L)]


class MG:
    """Oracle multigrid hierarchy (V(1,1)-cycle preconditioner + Krylov)."""

    def __init__(self, d, off, A, B=1, smoother=SGS, transfer=FW27V, w=1.0, precision=FP64, max_levels=16):
        d, o, A = _i3(d), _offs(off), _f64(A)
        h = ctypes.c_void_p()
        rc = lib().orc_mg_setup(ctypes.byref(h), _p(d), len(o), _p(o), B, _p(A), smoother, transfer,
                                ctypes.c_double(w), precision, max_levels)
        if rc:
            raise ValueError("oracle setup failed: %d" % rc)
        self.h, self.B, self.dims = h, B, tuple(int(t) for t in d)

    def __del__(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _lib.orc_mg_free(self.h)
            self.h = None

    @property
    def nlevels(self):
        return lib().orc_mg_nlevels(self.h)

    def level_info(self, l):
        d = np.zeros(3, dtype=np.int32)
        ns = ctypes.c_int()
        off = np.zeros((27, 3), dtype=np.int32)
        lib().orc_mg_level_info(self.h, l, _p(d), ctypes.byref(ns), _p(off))
        return tuple(int(t) for t in d), off[: ns.value].copy()

    def level_array(self, l, which):
        n = lib().orc_mg_level_array(self.h, l, which, None)
        dt = np.float64 if which <= 2 else np.float32
        out = np.zeros(n, dtype=dt)
        if n:
            lib().orc_mg_level_array(self.h, l, which, _p(out))
        return out

    def level_apply32(self, l, op, x=None, b=None, y=None):
        """One FP32 / BF16 level operation of a reduced-precision hierarchy
        (orc_mg_level_apply32): op 0 y = b - A x, 1 / 2 forward / backward
        Gauss-Seidel sweep on x (in place, returned), 3 y = ILU(0) apply of b,
        4 y = R x, 5 y += P x.  Vectors are float32; returns the output."""
        f32 = lambda a: None if a is None else np.ascontiguousarray(np.asarray(a, dtype=np.float32))
        x, b, y = f32(x), f32(b), f32(y)
        if op in (1, 2):
            x = x.copy()
        elif op == 5:
            y = y.copy()
        nul = ctypes.c_void_p()
        rc = lib().orc_mg_level_apply32(self.h, l, op, nul if x is None else _p(x), nul if b is None else _p(b),
                                        nul if y is None else _p(y))
        if rc:
            raise ValueError("level_apply32: operation %d unavailable on level %d" % (op, l))
        return x if op in (1, 2) else y

    def vcycle(self, r):
        r = _f64(r)
        z = np.zeros_like(r)
        lib().orc_mg_vcycle(self.h, _p(r), _p(z))
        return z

    def pcg(self, b, x0=None, tol=1e-9, maxit=200, flexible=False):
        b = _f64(b)
        x = np.zeros_like(b) if x0 is None else _f64(x0).copy()
        it, rr = ctypes.c_int(), ctypes.c_double()
        hist = np.zeros(maxit + 1)
        rc = lib().orc_pcg(self.h, _p(b), _p(x), ctypes.c_double(tol), maxit, int(flexible),
                           ctypes.byref(it), ctypes.byref(rr), _p(hist))
        return x, rc, it.value, rr.value, hist[: it.value + 1]

    def fgmres(self, b, x0=None, tol=1e-8, maxit=200, restart=30):
        b = _f64(b)
        x = np.zeros_like(b) if x0 is None else _f64(x0).copy()
        it, rr = ctypes.c_int(), ctypes.c_double()
        hist = np.zeros(maxit + 1)
        rc = lib().orc_fgmres(self.h, _p(b), _p(x), ctypes.c_double(tol), maxit, restart,
                              ctypes.byref(it), ctypes.byref(rr), _p(hist))
        return x, rc, it.value, rr.value, hist[: it.value + 1]
