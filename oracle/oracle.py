"""ctypes wrapper of the plain FP64 CPU oracle (msrcg_oracle.c).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg use this module to check and time the GPU library; the
library itself never imports it.  It does not import the library either.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "msrcg_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAXLEV = 16
OK, EINVAL, ENOMEM, ENOCONV, EBREAKDOWN = 0, -1, -2, -3, -4

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, no FMA contraction)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off",
                                   "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        L.or_hierarchy_dims.argtypes = [C.c_int, _ip, C.c_int, C.c_int, C.c_int, _ip]
        L.or_hierarchy_dims.restype = C.c_int
        L.or_hierarchy_dims2.argtypes = [C.c_int, _ip, _dp, C.c_int, C.c_int, C.c_int, C.c_int, _ip]
        L.or_hierarchy_dims2.restype = C.c_int
        L.or_transfer_table_pc.argtypes = [C.c_int, C.c_int, _ip, _ip, _dp]
        L.or_transfer_table_pc.restype = None
        L.or_face_trans.argtypes = [C.c_int, _ip, _dp, _dp, C.c_int, _u8p, _dp, _dp, C.c_void_p]
        L.or_face_trans.restype = None
        L.or_upscale.argtypes = [C.c_int, _ip, _ip, _dp, _dp, C.c_void_p, _dp, _dp, C.c_void_p]
        L.or_upscale.restype = None
        L.or_transfer_table.argtypes = [C.c_int, C.c_int, _ip, _ip, _dp]
        L.or_transfer_table.restype = None
        L.or_build.argtypes = [C.c_int, _ip, _dp, _dp, C.c_int, _u8p, C.c_int, C.c_int, C.c_double,
                               C.c_int, C.c_int, C.c_int, C.c_int, C.c_int]
        L.or_build.restype = C.c_void_p
        L.or_build_faces.argtypes = [C.c_int, _ip, _dp, _dp, _dp, C.c_void_p, C.c_int, C.c_int, C.c_double,
                                     C.c_int, C.c_int, C.c_int, C.c_int, C.c_int]
        L.or_build_faces.restype = C.c_void_p
        L.or_face_trans_faces.argtypes = [C.c_int, _ip, _dp, _dp, _dp, C.c_void_p, _dp, _dp, C.c_void_p]
        L.or_face_trans_faces.restype = None
        L.or_free.argtypes = [C.c_void_p]
        L.or_free.restype = None
        L.or_nlev.argtypes = [C.c_void_p]
        L.or_nlev.restype = C.c_int
        L.or_level_dims.argtypes = [C.c_void_p, C.c_int, _ip]
        L.or_level_dims.restype = None
        L.or_get_T.argtypes = [C.c_void_p, C.c_int, _dp, _dp, C.c_void_p]
        L.or_get_T.restype = None
        L.or_set_eps2.argtypes = [C.c_void_p, C.c_double]
        L.or_set_eps2.restype = None
        L.or_get_stats.argtypes = [C.c_void_p, _i64p, _i64p]
        L.or_get_stats.restype = None
        L.or_reset_stats.argtypes = [C.c_void_p]
        L.or_reset_stats.restype = None
        L.or_solve.argtypes = [C.c_void_p, _dp, C.c_double, _dp, _dp]
        L.or_solve.restype = C.c_int
        L.or_set_splitting.argtypes = [C.c_void_p, C.c_int]
        L.or_set_splitting.restype = None
        L.or_set_precond.argtypes = [C.c_void_p, C.c_int]
        L.or_set_trace.argtypes = [C.c_void_p, C.c_void_p, C.c_int64]
        L.or_set_trace.restype = None
        L.or_trace_count.argtypes = [C.c_void_p]
        L.or_trace_count.restype = C.c_int64
        L.or_set_precond.restype = None
        for name in ("or_apply_level", "or_sgs_level", "or_jacobi_level", "or_lex_level", "or_restrict_level",
                     "or_prolong_level"):
            getattr(L, name).argtypes = [C.c_void_p, C.c_int, _dp, _dp]
            getattr(L, name).restype = None
        L.or_sweep_level.argtypes = [C.c_void_p, C.c_int, C.c_int, _dp, _dp]
        L.or_sweep_level.restype = None
        L.or_precond_level.argtypes = [C.c_void_p, C.c_int, _dp, _dp]
        L.or_precond_level.restype = None
        L.or_pcg_level.argtypes = [C.c_void_p, C.c_int, _dp, _dp]
        L.or_pcg_level.restype = None
        L.or_status.argtypes = [C.c_void_p]
        L.or_status.restype = C.c_int
        L.or_lift_rhs.argtypes = [C.c_void_p, _dp, _u8p, _dp, C.c_void_p, _dp, _dp]
        L.or_lift_rhs.restype = None
        _lib = L
    return _lib


def _i3(v, dim):
    a = list(v) + [1] * (3 - len(v))
    return np.array(a[:3], np.int32)


def _d3(v, dim):
    a = list(v) + [1.0] * (3 - len(v))
    return np.array(a[:3], np.float64)


def hierarchy_dims(dim, n, s=4, maxside=None, h=None, coarsening=0):
    """Level sides; coarsening 1 aims at square cells (needs the cell sizes h)."""
    maxside = maxside or (8 if dim == 2 else 4)
    out = np.zeros(3 * MAXLEV, np.int32)
    if coarsening:
        nl = lib().or_hierarchy_dims2(dim, _i3(n, dim), _d3(h, dim), s, maxside, coarsening, MAXLEV, out)
    else:
        nl = lib().or_hierarchy_dims(dim, _i3(n, dim), s, maxside, MAXLEV, out)
    if nl < 1:
        raise ValueError("invalid grid")
    return [tuple(int(v) for v in out[3 * k:3 * k + 3]) for k in range(nl)]


def face_trans(dim, n, h, K, bc):
    n3 = list(n) + [1] * (3 - len(n))
    nx, ny, nz = n3
    K = np.ascontiguousarray(K, np.float64)
    ncomp = K.shape[0] if K.ndim == 2 else 1
    Tx = np.zeros((nx + 1) * ny * nz)
    Ty = np.zeros(nx * (ny + 1) * nz)
    Tz = np.zeros(nx * ny * (nz + 1)) if dim == 3 else None
    lib().or_face_trans(dim, _i3(n, dim), _d3(h, dim), K.reshape(-1), ncomp,
                        np.ascontiguousarray(bc, np.uint8), Tx, Ty,
                        Tz.ctypes.data if Tz is not None else None)
    return Tx, Ty, Tz


def face_trans_faces(dim, n, h, Kx, Ky, Kz=None):
    """T = (h_perp/h_par) K_face on every face (Sec. 3, face-centred K)."""
    n3 = list(n) + [1] * (3 - len(n))
    nx, ny, nz = n3
    Tx = np.zeros((nx + 1) * ny * nz)
    Ty = np.zeros(nx * (ny + 1) * nz)
    Tz = np.zeros(nx * ny * (nz + 1)) if dim == 3 else None
    Kz = np.ascontiguousarray(Kz, np.float64) if dim == 3 else None
    lib().or_face_trans_faces(dim, _i3(n, dim), _d3(h, dim), np.ascontiguousarray(Kx, np.float64),
                              np.ascontiguousarray(Ky, np.float64), Kz.ctypes.data if Kz is not None else None,
                              Tx, Ty, Tz.ctypes.data if Tz is not None else None)
    return Tx, Ty, Tz


def upscale(dim, nf, nc, Tx, Ty, Tz=None):
    f3, c3 = _i3(nf, dim), _i3(nc, dim)
    Txc = np.zeros((c3[0] + 1) * c3[1] * c3[2])
    Tyc = np.zeros(c3[0] * (c3[1] + 1) * c3[2])
    Tzc = np.zeros(c3[0] * c3[1] * (c3[2] + 1)) if dim == 3 else None
    lib().or_upscale(dim, f3, c3, np.ascontiguousarray(Tx), np.ascontiguousarray(Ty),
                     np.ascontiguousarray(Tz).ctypes.data if Tz is not None else None,
                     Txc, Tyc, Tzc.ctypes.data if Tzc is not None else None)
    return Txc, Tyc, Tzc


def transfer_table(nf, nc, interp=0):
    """1-D extension table: interp 0 = linear with zero slope at the boundary,
    1 = piecewise constant."""
    i0 = np.zeros(nf, np.int32)
    i1 = np.zeros(nf, np.int32)
    w = np.zeros(nf, np.float64)
    (lib().or_transfer_table_pc if interp else lib().or_transfer_table)(nf, nc, i0, i1, w)
    return i0, i1, w


class Hierarchy:
    """Oracle level hierarchy of one problem (Sec. 2.3 / Sec. 3)."""

    def __init__(self, prob, s=4, m=4, f=0.1, maxside=None, maxit_outer=200, maxit_inner=500, splitting=0,
                 coarsening=0, interp=0, Kfaces=None, precond=0):
        """splitting: 0 = symmetric Gauss-Seidel (red-black), 1 = modified
        Jacobi P = 2D, 2 = symmetric Gauss-Seidel in the natural order
        (Sec. 3).  coarsening: 0 = factor s on every long axis, 1 = toward
        square cells (Sec. 4.4).  interp: 0 = linear extension, 1 = piecewise
        constant (Sec. 3).  precond: 0 = recursive multi-scale (eq. 2.10),
        1 = multigrid V-step (eq. 2.9, Tatebe), 2 = polynomial (eq. 2.6 with
        W = P^-1).  Kfaces: (Kx, Ky[, Kz]) face permeabilities with
        the boundary conditions in the boundary faces' values; when given,
        they replace the problem's cell K and boundary types."""
        self.prob = prob
        self.dim = prob.dim
        maxside = maxside or (8 if prob.dim == 2 else 4)
        if Kfaces is not None:
            Kf = [np.ascontiguousarray(a, np.float64) for a in Kfaces]
            self._h = lib().or_build_faces(prob.dim, _i3(prob.n, prob.dim), _d3(prob.h, prob.dim), Kf[0], Kf[1],
                                           Kf[2].ctypes.data if prob.dim == 3 else None, s, m, f, maxside,
                                           maxit_outer, maxit_inner, coarsening, interp)
            self._keep = Kf
        else:
            K = np.ascontiguousarray(prob.K, np.float64)
            self._h = lib().or_build(prob.dim, _i3(prob.n, prob.dim), _d3(prob.h, prob.dim), K.reshape(-1),
                                     K.shape[0], np.ascontiguousarray(prob.bc, np.uint8), s, m, f, maxside,
                                     maxit_outer, maxit_inner, coarsening, interp)
        if not self._h:
            raise ValueError("oracle build failed")
        lib().or_set_splitting(self._h, int(splitting))
        lib().or_set_precond(self._h, int(precond))
        self.nlev = lib().or_nlev(self._h)
        self.dims = []
        for k in range(self.nlev):
            d = np.zeros(3, np.int32)
            lib().or_level_dims(self._h, k, d)
            self.dims.append(tuple(int(v) for v in d))

    def __del__(self):
        if getattr(self, "_h", None):
            lib().or_free(self._h)
            self._h = None

    def ncells(self, k):
        d = self.dims[k]
        return d[0] * d[1] * d[2]

    def T(self, k):
        nx, ny, nz = self.dims[k]
        Tx = np.zeros((nx + 1) * ny * nz)
        Ty = np.zeros(nx * (ny + 1) * nz)
        Tz = np.zeros(nx * ny * (nz + 1)) if self.dim == 3 else None
        lib().or_get_T(self._h, k, Tx, Ty, Tz.ctypes.data if Tz is not None else None)
        return Tx, Ty, Tz

    def lift_rhs(self, prob=None):
        """Right-hand side of the lifted system (Sec. 4.1) for this hierarchy's
        problem, or for `prob`: another problem on the same grid, permeability
        and boundary data that differs only in its source term or lifting."""
        p = self.prob if prob is None else prob
        if not p.lifted:
            return np.ascontiguousarray(p.b, np.float64).copy()
        b = np.zeros(p.N)
        f = np.ascontiguousarray(p.f, np.float64) if p.f is not None else None
        lib().or_lift_rhs(self._h, _d3(p.h, p.dim), np.ascontiguousarray(p.bc, np.uint8),
                          np.ascontiguousarray(p.gD, np.float64), f.ctypes.data if f is not None else None,
                          np.ascontiguousarray(p.pbf, np.float64), b)
        return b

    def solve(self, b, tau, trace_cap=0):
        """x and stats; with trace_cap > 0 the stats also hold the level tree
        (Fig. 2): "trace" = [(level, call, iterations, pass), ...] in the
        order the PCG calls returned, "trace_count" = all of them."""
        x = np.zeros(self.ncells(0))
        out = np.zeros(2)
        buf = np.zeros(4 * max(int(trace_cap), 1), np.int32)
        lib().or_set_trace(self._h, buf.ctypes.data if trace_cap > 0 else None, int(trace_cap))
        st = lib().or_solve(self._h, np.ascontiguousarray(b, np.float64), tau, x, out)
        it = np.zeros(MAXLEV, np.int64)
        ca = np.zeros(MAXLEV, np.int64)
        lib().or_get_stats(self._h, it, ca)
        res = {"status": st, "iters": it[:self.nlev].tolist(), "calls": ca[:self.nlev].tolist(),
               "relres_recursive": float(out[0]), "relres_true": float(out[1])}
        if trace_cap > 0:
            n = int(lib().or_trace_count(self._h))
            res["trace_count"] = n
            res["trace"] = [tuple(int(v) for v in e) for e in buf[:4 * min(n, int(trace_cap))].reshape(-1, 4)]
            lib().or_set_trace(self._h, None, 0)
        return x, res

    # ---- level-wise operators (tests) ----
    def apply(self, k, x):
        y = np.zeros(self.ncells(k))
        lib().or_apply_level(self._h, k, np.ascontiguousarray(x, np.float64), y)
        return y

    def sgs(self, k, rhs, x):
        x = np.array(x, np.float64)
        lib().or_sgs_level(self._h, k, np.ascontiguousarray(rhs, np.float64), x)
        return x

    def lex_sgs(self, k, rhs, x):
        x = np.array(x, np.float64)
        lib().or_lex_level(self._h, k, np.ascontiguousarray(rhs, np.float64), x)
        return x

    def jacobi(self, k, rhs, x):
        x = np.array(x, np.float64)
        lib().or_jacobi_level(self._h, k, np.ascontiguousarray(rhs, np.float64), x)
        return x

    def sweep(self, k, colour, rhs, x):
        x = np.array(x, np.float64)
        lib().or_sweep_level(self._h, k, colour, np.ascontiguousarray(rhs, np.float64), x)
        return x

    def restrict(self, k, rf):
        rc = np.zeros(self.ncells(k + 1))
        lib().or_restrict_level(self._h, k, np.ascontiguousarray(rf, np.float64), rc)
        return rc

    def prolong_add(self, k, xc, xf):
        xf = np.array(xf, np.float64)
        lib().or_prolong_level(self._h, k, np.ascontiguousarray(xc, np.float64), xf)
        return xf

    def set_eps2(self, eps2):
        lib().or_set_eps2(self._h, eps2)

    def precond(self, k, r):
        z = np.zeros(self.ncells(k))
        lib().or_precond_level(self._h, k, np.ascontiguousarray(r, np.float64), z)
        return z

    def pcg(self, k, b):
        x = np.zeros(self.ncells(k))
        lib().or_pcg_level(self._h, k, np.ascontiguousarray(b, np.float64), x)
        return x

    def stats(self):
        it = np.zeros(MAXLEV, np.int64)
        ca = np.zeros(MAXLEV, np.int64)
        lib().or_get_stats(self._h, it, ca)
        return it[:self.nlev].tolist(), ca[:self.nlev].tolist()

    def reset_stats(self):
        lib().or_reset_stats(self._h)

    def status(self):
        return lib().or_status(self._h)

    def dense(self, k):
        n = self.ncells(k)
        A = np.zeros((n, n))
        e = np.zeros(n)
        for j in range(n):
            e[j] = 1.0
            A[:, j] = self.apply(k, e)
            e[j] = 0.0
        return A
