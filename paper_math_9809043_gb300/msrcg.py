"""Python binding of libmsrcg (ctypes).

Argument marshalling only: every step of the solver runs in the library's
CUDA kernels.  PyTorch provides device memory and streams.  There is no CPU
fallback: the first call into the library raises ImportError if libmsrcg.so
is missing.

Reference: Lackner & Menikoff, "Multi-scale linear solvers for very large
systems derived from PDEs" (arXiv math/9809043), Sec. 2.3 (recursive
multi-scale preconditioned CG) and Sec. 3 (porous-flow discretisation).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmsrcg.so")

OK, EINVAL, ENOMEM, ENOCONV, EBREAKDOWN, ETIMEOUT, ENANINF, ECUDA = 0, -1, -2, -3, -4, -5, -6, -7
MAXLEV = 16


class Grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("h", C.c_double * 3)]


class Opts(C.Structure):
    _fields_ = [("scale", C.c_int), ("m", C.c_int), ("f", C.c_double), ("coarsest_max_side", C.c_int),
                ("precision", C.c_int), ("maxit_outer", C.c_int), ("maxit_inner", C.c_int),
                ("timeout_ns", C.c_uint64), ("inner_floor", C.c_double), ("small_cells", C.c_int),
                ("plain_sweeps", C.c_int), ("fuse_width", C.c_int), ("fuse_min_cells", C.c_int),
                ("splitting", C.c_int), ("coarsening", C.c_int), ("interp", C.c_int),
                ("stall_iters", C.c_int), ("escalate", C.c_int), ("flexible", C.c_int),
                ("precond", C.c_int), ("reserved", C.c_int * 1)]


class Stats(C.Structure):
    _fields_ = [("levels", C.c_int), ("dims", (C.c_int * 3) * MAXLEV), ("iters", C.c_int64 * MAXLEV),
                ("calls", C.c_int64 * MAXLEV), ("relres_recursive", C.c_double), ("relres_true", C.c_double),
                ("status", C.c_int), ("restarts", C.c_int), ("flexible", C.c_int), ("escalated", C.c_int)]

    def as_dict(self):
        L = self.levels
        return {"levels": L, "dims": [tuple(self.dims[k]) for k in range(L)],
                "iters": [int(self.iters[k]) for k in range(L)], "calls": [int(self.calls[k]) for k in range(L)],
                "relres_recursive": float(self.relres_recursive), "relres_true": float(self.relres_true),
                "status": int(self.status), "restarts": int(self.restarts), "flexible": int(self.flexible),
                "escalated": int(self.escalated)}


class MsrcgError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})")


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run paper_math_9809043_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        vp = C.c_void_p
        L.msrcg_default_opts.argtypes = [C.POINTER(Opts)]
        L.msrcg_build.argtypes = [C.POINTER(Grid), vp, C.c_int, vp, C.POINTER(Opts), vp, C.POINTER(vp)]
        L.msrcg_build_faces.argtypes = [C.POINTER(Grid), vp, vp, vp, C.POINTER(Opts), vp, C.POINTER(vp)]
        L.msrcg_build_laplace.argtypes = [C.POINTER(Grid), C.POINTER(C.c_double * 3), C.POINTER(C.c_uint8 * 6),
                                          C.POINTER(Opts), vp, C.POINTER(vp)]
        L.msrcg_lift_rhs.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.msrcg_solve.argtypes = [vp, vp, C.c_double, vp, C.POINTER(Stats), vp]
        L.msrcg_batch_solve.argtypes = [C.c_int, C.POINTER(vp), C.POINTER(vp), C.c_double, C.POINTER(vp),
                                        C.POINTER(Stats), vp]
        L.msrcg_level_info.argtypes = [vp, C.c_int, C.POINTER(C.c_int * 3), C.POINTER(C.c_int64),
                                       C.POINTER(C.c_int64)]
        L.msrcg_get_trans.argtypes = [vp, C.c_int, vp, vp, vp, vp]
        L.msrcg_apply.argtypes = [vp, C.c_int, vp, vp, vp]
        L.msrcg_num_levels.argtypes = [vp]
        L.msrcg_device_bytes.argtypes = [vp]
        L.msrcg_device_bytes.restype = C.c_size_t
        L.msrcg_free.argtypes = [vp]
        L.msrcg_free.restype = None
        L.msrcg_solve_static.argtypes = [C.POINTER(Grid), vp, C.c_int, vp, C.POINTER(Opts), vp, C.c_double, vp,
                                         C.POINTER(Stats), vp]
        L.msrcg_server_create.argtypes = [C.c_size_t, C.c_int, C.POINTER(Opts), C.POINTER(vp)]
        L.msrcg_server_submit.argtypes = [vp, C.POINTER(Grid), vp, C.c_int, vp, vp, C.c_double, vp,
                                          C.POINTER(C.c_int64)]
        L.msrcg_server_progress.argtypes = [vp]
        L.msrcg_server_poll.argtypes = [vp, C.c_int64, C.POINTER(Stats)]
        L.msrcg_server_drain.argtypes = [vp]
        L.msrcg_server_bytes_in_use.argtypes = [vp]
        L.msrcg_server_bytes_in_use.restype = C.c_size_t
        L.msrcg_server_destroy.argtypes = [vp]
        L.msrcg_server_destroy.restype = None
        L.msrcg_profile_kernel_count.argtypes = []
        L.msrcg_profile_kernel_name.argtypes = [C.c_int]
        L.msrcg_profile_kernel_name.restype = C.c_char_p
        L.msrcg_profile_level.argtypes = [vp, C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double), vp]
        L.msrcg_set_trace.argtypes = [vp, vp, C.c_int64]
        L.msrcg_strerror.argtypes = [C.c_int]
        L.msrcg_strerror.restype = C.c_char_p
        _lib = L
    return _lib


def strerror(code: int) -> str:
    return lib().msrcg_strerror(code).decode()


def default_opts(**kw) -> Opts:
    o = Opts()
    lib().msrcg_default_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def _dev(a, dtype, device, n=None, what="array"):
    """`a` as a contiguous device tensor of `dtype` (a copy only when needed);
    with `n`, its size is checked first: the library reads and writes
    exactly the sizes it documents through raw pointers."""
    if isinstance(a, torch.Tensor):
        t = a.to(device=device, dtype=dtype).contiguous()
    else:
        t = torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=device)
    if n is not None and t.numel() != n:
        raise ValueError(f"{what}: {t.numel()} elements, expected {n}")
    return t


def _out(t, dtype, device, n, what):
    """A caller-supplied output tensor: written in place, so it must already
    be contiguous, of `dtype`, on `device` and of `n` elements."""
    if not (isinstance(t, torch.Tensor) and t.dtype == dtype and t.device == device and t.is_contiguous()
            and t.numel() == n):
        raise ValueError(f"{what}: expected a contiguous {dtype} tensor of {n} elements on {device}")
    return t


def _device(device) -> torch.device:
    """`device` with its index (tensors report theirs: cuda:0, not cuda)."""
    d = torch.device(device)
    if d.type == "cuda" and d.index is None:
        d = torch.device("cuda", torch.cuda.current_device())
    return d


def n_boundary_faces(dim, n) -> int:
    """Entries of the boundary layout (bc, gD): x-low and x-high faces (ny nz
    each), y-low and y-high (nx nz each), z-low and z-high (nx ny each, 3D)."""
    nx, ny = int(n[0]), int(n[1])
    nz = int(n[2]) if dim == 3 else 1
    return 2 * (ny * nz + nx * nz) + (2 * nx * ny if dim == 3 else 0)


def _valid_grid(dim, n) -> bool:
    """Grids the library accepts; the binding checks array sizes only for
    those and leaves every other grid to the library's own MSRCG_EINVAL."""
    return dim in (2, 3) and len(n) >= dim and all(int(v) >= 1 for v in n[:dim])


def _check_K(Kt, dim, N):
    ncomp = Kt.numel() // max(N, 1)
    if ncomp not in (1, dim) or Kt.numel() != ncomp * N:
        raise ValueError(f"K: {Kt.numel()} elements, expected N = {N} (scalar) or dim * N = {dim * N} (diagonal)")
    return ncomp


def _hold(stream, *ts):
    """Tensors that work enqueued on `stream` reads or writes: when that is
    not the current stream, record it with the caching allocator so that
    their memory is not handed out again before that work has run."""
    if stream is None or stream == torch.cuda.current_stream(stream.device):
        return
    for t in ts:
        if t is not None:
            t.record_stream(stream)


class Hierarchy:
    """Level hierarchy of one problem, resident on the GPU (msrcg_build)."""

    def __init__(self, dim, n, h, K, bc, opts: Opts | None = None, device="cuda", stream=None):
        self.device = _device(device)
        self.dim = dim
        self.n = tuple(int(v) for v in n)
        self.N = int(np.prod(self.n))
        g = Grid()
        g.dim = dim
        for a in range(3):
            g.n[a] = self.n[a] if a < min(dim, len(self.n)) else 1
            g.h[a] = float(h[a]) if a < min(dim, len(h)) else 1.0
        Kt = _dev(K, torch.float64, self.device).reshape(-1)
        if _valid_grid(dim, self.n):
            ncomp = _check_K(Kt, dim, self.N)
            bct = _dev(bc, torch.uint8, self.device, self.n_boundary_faces(), "bc")
        else:
            ncomp = Kt.numel() // max(self.N, 1)
            bct = _dev(bc, torch.uint8, self.device)
        self.opts = opts or default_opts()
        hp = C.c_void_p()
        with torch.cuda.device(self.device):
            rc = lib().msrcg_build(C.byref(g), _ptr(Kt), ncomp, _ptr(bct), C.byref(self.opts), _stream(stream),
                                   C.byref(hp))
        if rc != OK:
            raise MsrcgError(rc, "msrcg_build")
        self._h = hp
        self.nlev = lib().msrcg_num_levels(self._h)

    def n_boundary_faces(self) -> int:
        return n_boundary_faces(self.dim, self.n)

    @classmethod
    def from_problem(cls, prob, opts: Opts | None = None, device="cuda", stream=None):
        return cls(prob.dim, prob.n, prob.h, prob.K, prob.bc, opts, device, stream)

    @classmethod
    def laplace(cls, dim, n, h, K, side_bc, opts: Opts | None = None, device="cuda", stream=None):
        """Constant-coefficient hierarchy (msrcg_build_laplace): K a scalar or
        one value per axis, side_bc six 0/1 flags (x-low, x-high, y-low,
        y-high, z-low, z-high; 1 = Dirichlet)."""
        self = cls.__new__(cls)
        self.device = _device(device)
        self.dim = dim
        self.n = tuple(int(v) for v in n)
        self.N = int(np.prod(self.n))
        g = Grid()
        g.dim = dim
        for a in range(3):
            g.n[a] = self.n[a] if a < min(dim, len(self.n)) else 1
            g.h[a] = float(h[a]) if a < min(dim, len(h)) else 1.0
        Kv = np.broadcast_to(np.asarray(K, np.float64).reshape(-1), (3,)) if np.size(K) == 1 else \
            np.asarray(list(np.asarray(K, np.float64).reshape(-1)) + [1.0] * 3)[:3]
        Ka = (C.c_double * 3)(*[float(v) for v in Kv])
        sb = list(side_bc) + [0] * 6
        Sa = (C.c_uint8 * 6)(*[int(v) for v in sb[:6]])
        self.opts = opts or default_opts()
        hp = C.c_void_p()
        with torch.cuda.device(self.device):
            rc = lib().msrcg_build_laplace(C.byref(g), C.byref(Ka), C.byref(Sa), C.byref(self.opts), _stream(stream),
                                           C.byref(hp))
        if rc != OK:
            raise MsrcgError(rc, "msrcg_build_laplace")
        self._h = hp
        self.nlev = lib().msrcg_num_levels(self._h)
        return self

    @classmethod
    def from_faces(cls, dim, n, h, Kfaces, opts: Opts | None = None, device="cuda", stream=None):
        """Hierarchy from face permeabilities (msrcg_build_faces): Kfaces =
        (Kx, Ky[, Kz]) with (nx+1) ny nz, nx (ny+1) nz[, nx ny (nz+1)] entries,
        boundary faces included (a Dirichlet face holds its K, a Neumann face 0)."""
        self = cls.__new__(cls)
        self.device = _device(device)
        self.dim = dim
        self.n = tuple(int(v) for v in n)
        self.N = int(np.prod(self.n))
        g = Grid()
        g.dim = dim
        for a in range(3):
            g.n[a] = self.n[a] if a < min(dim, len(self.n)) else 1
            g.h[a] = float(h[a]) if a < min(dim, len(h)) else 1.0
        n3 = [g.n[0], g.n[1], g.n[2]]
        sizes = [(n3[0] + 1) * n3[1] * n3[2], n3[0] * (n3[1] + 1) * n3[2], n3[0] * n3[1] * (n3[2] + 1)]
        Kt = [None, None, None]
        if _valid_grid(dim, self.n):
            if len(Kfaces) < dim:
                raise ValueError(f"Kfaces: {len(Kfaces)} arrays for a {dim}D grid")
            for a in range(dim):
                Kt[a] = _dev(Kfaces[a], torch.float64, self.device, sizes[a], f"K{'xyz'[a]}")
        else:
            for a in range(min(dim, len(Kfaces))):
                Kt[a] = _dev(Kfaces[a], torch.float64, self.device)
        self.opts = opts or default_opts()
        hp = C.c_void_p()
        with torch.cuda.device(self.device):
            rc = lib().msrcg_build_faces(C.byref(g), _ptr(Kt[0]), _ptr(Kt[1]), _ptr(Kt[2]), C.byref(self.opts),
                                         _stream(stream), C.byref(hp))
        if rc != OK:
            raise MsrcgError(rc, "msrcg_build_faces")
        self._h = hp
        self.nlev = lib().msrcg_num_levels(self._h)
        return self

    def close(self):
        if getattr(self, "_h", None):
            lib().msrcg_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def device_bytes(self) -> int:
        return int(lib().msrcg_device_bytes(self._h))

    def dims(self, k):
        d = (C.c_int * 3)()
        it, ca = C.c_int64(), C.c_int64()
        rc = lib().msrcg_level_info(self._h, k, C.byref(d), C.byref(it), C.byref(ca))
        if rc != OK:
            raise MsrcgError(rc, "msrcg_level_info")
        return tuple(d), int(it.value), int(ca.value)

    def lift_rhs(self, bc, gD, f, pbf, stream=None):
        nbf = self.n_boundary_faces()
        bct = _dev(bc, torch.uint8, self.device, nbf, "bc")
        gDt = _dev(gD, torch.float64, self.device, nbf, "gD")
        ft = _dev(f, torch.float64, self.device, self.N, "f") if f is not None else None
        pt = _dev(pbf, torch.float64, self.device, self.N, "pbf")
        b = torch.empty(self.N, dtype=torch.float64, device=self.device)
        _hold(stream, bct, gDt, ft, pt, b)
        rc = lib().msrcg_lift_rhs(self._h, _ptr(bct), _ptr(gDt), _ptr(ft), _ptr(pt), _ptr(b), _stream(stream))
        if rc != OK:
            raise MsrcgError(rc, "msrcg_lift_rhs")
        return b

    def rhs_for(self, prob, stream=None):
        """Device right-hand side of a generated problem (lifted or direct)."""
        if prob.lifted:
            return self.lift_rhs(prob.bc, prob.gD, prob.f, prob.pbf, stream)
        return _dev(prob.b, torch.float64, self.device)

    def solve(self, b, tol=1e-8, x=None, stats=True, stream=None, check=True):
        b = _dev(b, torch.float64, self.device, self.N, "b")
        if x is None:
            x = torch.empty(self.N, dtype=torch.float64, device=self.device)
        else:
            _out(x, torch.float64, self.device, self.N, "x")
        _hold(stream, b, x)
        st = Stats()
        rc = lib().msrcg_solve(self._h, _ptr(b), float(tol), _ptr(x), C.byref(st) if stats else None,
                               _stream(stream))
        if check and rc != OK:
            raise MsrcgError(rc, "msrcg_solve")
        return x, (st.as_dict() if stats else {"status": rc})

    def trans(self, k, stream=None):
        d, _, _ = self.dims(k)
        nx, ny, nz = d
        Tx = torch.empty((nx + 1) * ny * nz, dtype=torch.float64, device=self.device)
        Ty = torch.empty(nx * (ny + 1) * nz, dtype=torch.float64, device=self.device)
        Tz = torch.empty(nx * ny * (nz + 1), dtype=torch.float64, device=self.device) if self.dim == 3 else None
        _hold(stream, Tx, Ty, Tz)
        rc = lib().msrcg_get_trans(self._h, k, _ptr(Tx), _ptr(Ty), _ptr(Tz), _stream(stream))
        if rc != OK:
            raise MsrcgError(rc, "msrcg_get_trans")
        return Tx, Ty, Tz

    def set_trace(self, capacity):
        """Attach a level-tree buffer of `capacity` entries (msrcg_set_trace);
        capacity 0 detaches.  The buffer is a device tensor held here."""
        if capacity <= 0:
            rc = lib().msrcg_set_trace(self._h, None, 0)
            self._trace = None
        else:
            buf = torch.zeros(4 + 4 * int(capacity), dtype=torch.int32, device=self.device)
            rc = lib().msrcg_set_trace(self._h, _ptr(buf), int(capacity))
            self._trace = buf if rc == OK else None
        if rc != OK:
            raise MsrcgError(rc, "msrcg_set_trace")

    def trace(self):
        """The level tree of the last solve: (total entries, [(level, call,
        iterations, pass), ...]) in the order the calls returned."""
        buf = getattr(self, "_trace", None)
        if buf is None:
            return 0, []
        host = buf.cpu()
        count = int(host[:2].view(torch.int64)[0])
        n = min(count, (host.numel() - 4) // 4)
        ent = host[4:4 + 4 * n].view(-1, 4).tolist()
        return count, [tuple(e) for e in ent]

    def profile_level(self, k, reps=20, stream=None):
        """Per-kernel mean launch time (ms) and algorithmic bytes of level k's
        multi-CTA kernels, timed standalone (msrcg_profile_level)."""
        n = lib().msrcg_profile_kernel_count()
        ms = (C.c_double * n)()
        by = (C.c_double * n)()
        rc = lib().msrcg_profile_level(self._h, k, int(reps), ms, by, _stream(stream))
        if rc != OK:
            raise MsrcgError(rc, "msrcg_profile_level")
        return [{"kernel": lib().msrcg_profile_kernel_name(i).decode(), "ms": ms[i], "bytes": by[i],
                 "gbs": by[i] / (ms[i] * 1e6) if ms[i] > 0 else 0.0} for i in range(n)]

    def apply(self, k, x, stream=None):
        d, _, _ = self.dims(k)
        x = _dev(x, torch.float64, self.device, d[0] * d[1] * d[2], "x")
        y = torch.empty_like(x)
        _hold(stream, x, y)
        rc = lib().msrcg_apply(self._h, k, _ptr(x), _ptr(y), _stream(stream))
        if rc != OK:
            raise MsrcgError(rc, "msrcg_apply")
        return y


def batch_solve(hs, bs, tol=1e-8, xs=None, stream=None, check=True):
    """Solve independent problems in one persistent launch (msrcg_batch_solve)."""
    n = len(hs)
    if len(bs) != n or (xs is not None and len(xs) != n):
        raise ValueError("batch_solve: hs, bs and xs differ in length")
    if any(h.handle is None for h in hs):
        raise ValueError("batch_solve: a hierarchy has been closed")
    bs = [_dev(b, torch.float64, h.device, h.N, f"bs[{i}]") for i, (h, b) in enumerate(zip(hs, bs))]
    if xs is None:
        xs = [torch.empty(h.N, dtype=torch.float64, device=h.device) for h in hs]
    else:
        for i, (h, x) in enumerate(zip(hs, xs)):
            _out(x, torch.float64, h.device, h.N, f"xs[{i}]")
    H = (C.c_void_p * n)(*[h.handle.value for h in hs])
    B = (C.c_void_p * n)(*[b.data_ptr() for b in bs])
    X = (C.c_void_p * n)(*[x.data_ptr() for x in xs])
    st = (Stats * n)()
    rc = lib().msrcg_batch_solve(n, H, B, float(tol), X, st, _stream(stream))
    if check and rc != OK:
        raise MsrcgError(rc, "msrcg_batch_solve")
    return xs, [s.as_dict() for s in st]


STATIC_SCRATCH_BYTES = 4 << 20


def solve_static(dim, n, h, K, bc, b, tol=1e-8, x=None, opts: Opts | None = None, device="cuda", stream=None,
                 check=True):
    """Build and solve one small problem without allocating (msrcg_solve_static).

    For callers that cannot allocate device memory; the library works in a
    fixed scratch of STATIC_SCRATCH_BYTES.  Overlapping calls race."""
    device = _device(device)
    g = Grid()
    g.dim = dim
    nn = tuple(int(v) for v in n)
    for a in range(3):
        g.n[a] = nn[a] if a < min(dim, len(nn)) else 1
        g.h[a] = float(h[a]) if a < min(dim, len(h)) else 1.0
    N = int(np.prod(nn))
    Kt = _dev(K, torch.float64, device).reshape(-1)
    if _valid_grid(dim, nn):
        _check_K(Kt, dim, N)
        bct = _dev(bc, torch.uint8, device, n_boundary_faces(dim, nn), "bc")
        bt = _dev(b, torch.float64, device, N, "b")
    else:
        bct = _dev(bc, torch.uint8, device)
        bt = _dev(b, torch.float64, device)
    if x is None:
        x = torch.empty(N, dtype=torch.float64, device=device)
    else:
        _out(x, torch.float64, device, N, "x")
    st = Stats()
    o = opts or default_opts()
    rc = lib().msrcg_solve_static(C.byref(g), _ptr(Kt), Kt.numel() // max(N, 1), _ptr(bct), C.byref(o), _ptr(bt),
                                  float(tol), _ptr(x), C.byref(st), _stream(stream))
    if check and rc != OK:
        raise MsrcgError(rc, "msrcg_solve_static")
    return x, st.as_dict()
