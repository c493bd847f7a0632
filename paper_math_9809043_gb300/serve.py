"""Serving front-end: continuous batching of independent porous-flow solves.

Thin wrapper over the library's server (msrcg_server_*): requests are
admitted by device-memory budget, each keeps its level hierarchy resident
while it runs, and requests built since the last launch go to the GPU as
one batched wave on a stream of their own, overlapping earlier waves.
`replay` drives a server with a timed arrival stream and reports latency
(arrival to result on the host, including the copies and the build) and
throughput.
"""
from __future__ import annotations

import ctypes as C
import time

import numpy as np

from . import msrcg as M


class Server:
    def __init__(self, budget_bytes: int, max_waves: int = 8, opts: M.Opts | None = None):
        self.opts = opts or M.default_opts()
        h = C.c_void_p()
        rc = M.lib().msrcg_server_create(int(budget_bytes), int(max_waves), C.byref(self.opts), C.byref(h))
        if rc != M.OK:
            raise M.MsrcgError(rc, "msrcg_server_create")
        self._h = h
        self._keep = {}

    def close(self):
        if getattr(self, "_h", None):
            M.lib().msrcg_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, prob, b, tol=1e-8):
        """Queue problem `prob` (generated Problem) with right-hand side b
        (host array); returns (id, x) where x is filled when done."""
        g = M.Grid()
        g.dim = prob.dim
        for a in range(3):
            g.n[a] = prob.n[a] if a < prob.dim else 1
            g.h[a] = float(prob.h[a]) if a < prob.dim else 1.0
        K = np.ascontiguousarray(prob.K, np.float64)
        bc = np.ascontiguousarray(prob.bc, np.uint8)
        bb = np.ascontiguousarray(b, np.float64)
        ncomp = K.shape[0] if K.ndim == 2 else 1
        # the library copies exactly these sizes from the host pointers
        if ncomp not in (1, prob.dim) or K.size != ncomp * prob.N:
            raise ValueError(f"K: {K.size} elements for N = {prob.N}")
        if bc.size != M.n_boundary_faces(prob.dim, prob.n) or bb.size != prob.N:
            raise ValueError(f"bc / b: {bc.size} / {bb.size} elements, expected "
                             f"{M.n_boundary_faces(prob.dim, prob.n)} / {prob.N}")
        x = np.empty(prob.N, np.float64)
        rid = C.c_int64()
        rc = M.lib().msrcg_server_submit(self._h, C.byref(g), K.ctypes.data, ncomp,
                                         bc.ctypes.data, bb.ctypes.data, float(tol), x.ctypes.data, C.byref(rid))
        if rc != M.OK:
            raise M.MsrcgError(rc, "msrcg_server_submit")
        self._keep[rid.value] = (K, bc, bb, x)
        return rid.value, x

    def progress(self) -> int:
        n = M.lib().msrcg_server_progress(self._h)
        if n < 0:
            raise M.MsrcgError(n, "msrcg_server_progress")
        return n

    def poll(self, rid):
        """(done, stats): done once the request's x is written."""
        st = M.Stats()
        rc = M.lib().msrcg_server_poll(self._h, rid, C.byref(st))
        if rc == 0:
            return False, None
        self._keep.pop(rid, None)
        if rc < 0:
            return True, {"status": rc}
        return True, st.as_dict()

    def drain(self):
        rc = M.lib().msrcg_server_drain(self._h)
        if rc != M.OK:
            raise M.MsrcgError(rc, "msrcg_server_drain")

    def bytes_in_use(self) -> int:
        return int(M.lib().msrcg_server_bytes_in_use(self._h))


def replay(server: Server, arrivals, problems, rhs, tol=1e-8, max_seconds=None):
    """Submit request i at time arrivals[i] (seconds from start) with problem
    problems[i] and right-hand side rhs[i]; poll continuously.  Returns
    per-request latencies (s), results, stats and the makespan."""
    n = len(arrivals)
    t0 = time.perf_counter()
    sub_t = [None] * n
    done_t = [None] * n
    ids = [None] * n
    xs = [None] * n
    stats = [None] * n
    nxt = 0
    open_ids = {}
    while True:
        now = time.perf_counter() - t0
        while nxt < n and arrivals[nxt] <= now and (max_seconds is None or now < max_seconds):
            ids[nxt], xs[nxt] = server.submit(problems[nxt], rhs[nxt], tol)
            sub_t[nxt] = arrivals[nxt]
            open_ids[ids[nxt]] = nxt
            nxt += 1
        server.progress()
        for rid, i in list(open_ids.items()):
            done, st = server.poll(rid)
            if done:
                done_t[i] = time.perf_counter() - t0
                stats[i] = st
                del open_ids[rid]
        if not open_ids and (nxt >= n or (max_seconds is not None and now >= max_seconds)):
            break
        if not open_ids and nxt < n:
            time.sleep(max(0.0, min(arrivals[nxt] - (time.perf_counter() - t0), 0.001)))
    lat = [d - s for d, s in zip(done_t, sub_t) if d is not None]
    makespan = max(d for d in done_t if d is not None) if lat else 0.0
    return {"latency_s": lat, "x": xs, "stats": stats, "submitted": nxt, "makespan_s": makespan}
