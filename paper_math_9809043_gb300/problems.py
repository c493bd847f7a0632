"""Seeded synthetic porous-flow problems.

This module only draws inputs: cell permeabilities, boundary-condition masks
and values, sources, lifting fields and right-hand sides.  It holds none of
the solver's arithmetic (no transmissibilities, no operator, no transfers), so
that both the GPU library and the CPU oracle can be fed the same arrays.

Workloads follow the paper's test problems (Sec. 4: random log-normal
permeability with Dirichlet p=1 / p=0 on the x faces and no flow on the
others); the paper's own power-law fields are not available, so Gaussian
random fields and layered channel fields of the stated contrast stand in.

Array conventions
-----------------
* cells are indexed ``c = i + nx*(j + ny*k)`` (x fastest); NumPy arrays are
  shaped ``(nz, ny, nx)`` (2D: ``(ny, nx)``) in C order, which is the same
  memory order;
* ``K`` is shaped ``(ncomp, N)``: one scalar permeability (ncomp=1) or the
  diagonal of the tensor (ncomp=dim);
* ``bc`` (uint8, 1 = Dirichlet, 0 = Neumann) and ``gD`` (Dirichlet values)
  hold one entry per boundary face, in blocks x-low, x-high (ny*nz each),
  y-low, y-high (nx*nz each), z-low, z-high (nx*ny each, 3D only); inside a
  block the faces are ordered with the lower remaining axis fastest.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np


@dataclass
class Problem:
    dim: int
    n: tuple                      # cells per axis (nx, ny[, nz])
    h: tuple                      # cell sizes
    K: np.ndarray                 # (ncomp, N) float64 cell permeability
    bc: np.ndarray                # (nbf,) uint8
    gD: np.ndarray                # (nbf,) float64 Dirichlet values
    f: Optional[np.ndarray] = None    # (N,) source density, or None
    pbf: Optional[np.ndarray] = None  # (N,) lifting field, or None
    b: Optional[np.ndarray] = None    # (N,) right-hand side used directly
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return int(np.prod(self.n))

    @property
    def n3(self) -> tuple:
        return (self.n[0], self.n[1], self.n[2] if self.dim == 3 else 1)

    @property
    def h3(self) -> tuple:
        return (self.h[0], self.h[1], self.h[2] if self.dim == 3 else 1.0)

    @property
    def lifted(self) -> bool:
        return self.b is None


def n_boundary_faces(dim: int, n) -> int:
    nx, ny = n[0], n[1]
    nz = n[2] if dim == 3 else 1
    return 2 * (ny * nz + nx * nz) + (2 * nx * ny if dim == 3 else 0)


def standard_bc(dim: int, n, p_left: float = 1.0, p_right: float = 0.0):
    """Dirichlet p_left on x-low, p_right on x-high, no flow elsewhere."""
    nx, ny = n[0], n[1]
    nz = n[2] if dim == 3 else 1
    nbf = n_boundary_faces(dim, n)
    bc = np.zeros(nbf, np.uint8)
    gD = np.zeros(nbf, np.float64)
    m = ny * nz
    bc[:m] = 1
    gD[:m] = p_left
    bc[m:2 * m] = 1
    gD[m:2 * m] = p_right
    return bc, gD


def linear_lifting(dim: int, n, p_left: float = 1.0, p_right: float = 0.0):
    """A smooth field matching the standard boundary values: linear in x."""
    nx = n[0]
    xc = (np.arange(nx) + 0.5) / nx
    prof = p_left + (p_right - p_left) * xc
    shape = (n[2], n[1], nx) if dim == 3 else (n[1], nx)
    return np.broadcast_to(prof, shape).reshape(-1).astype(np.float64).copy()


def gaussian_random_field(shape, ell_cells: float, rng: np.random.Generator) -> np.ndarray:
    """Periodic Gaussian random field with Gaussian covariance exp(-r^2/ell^2).

    White noise is filtered in Fourier space by the square root of the
    covariance spectrum, exp(-ell^2 |k|^2 / 8), k in radians per cell.
    """
    w = rng.standard_normal(shape)
    W = np.fft.fftn(w)
    k2 = np.zeros(shape)
    for ax, m in enumerate(shape):
        kk = 2.0 * np.pi * np.fft.fftfreq(m)
        sh = [1] * len(shape)
        sh[ax] = m
        k2 = k2 + (kk ** 2).reshape(sh)
    g = np.real(np.fft.ifftn(W * np.exp(-(ell_cells ** 2) * k2 / 8.0)))
    return g


def power_law_field(n: int, rng: np.random.Generator, cutoff=(32.0, 4.0), angle_deg: float = 15.0,
                    big: int = 2048) -> np.ndarray:
    """Zero-mean, unit-variance Gaussian field on an n x n grid whose
    autocorrelation is the power law (1 + d^T Lambda d)^(-1/4) of the paper's
    test fields (Sec. 4), d in cells.  Lambda = Rot diag(1/c1^2, 1/c2^2) Rot^T
    with cutoff lengths (c1, c2) in cells, the long axis at `angle_deg` to x.
    The field is synthesised on a periodic big x big grid (the spectral
    density is the FFT of the covariance, negative parts clipped) and the
    lower-left n x n corner is kept, as the paper truncates its 2048^2 field
    (Sec. 4.2).  Returned shape (n, n), x fastest."""
    if n > big:
        raise ValueError("field larger than its synthesis grid")
    d = np.fft.fftfreq(big) * big  # signed periodic distances
    X, Y = np.meshgrid(d, d, indexing="xy")
    th = np.deg2rad(angle_deg)
    u = np.cos(th) * X + np.sin(th) * Y
    v = -np.sin(th) * X + np.cos(th) * Y
    cov = (1.0 + (u / cutoff[0]) ** 2 + (v / cutoff[1]) ** 2) ** -0.25
    spec = np.real(np.fft.fft2(cov))
    spec[spec < 0.0] = 0.0
    w = rng.standard_normal((big, big))
    g = np.real(np.fft.ifft2(np.fft.fft2(w) * np.sqrt(spec)))[:n, :n]
    return (g - g.mean()) / g.std()


def base_case_problem(n: int = 1001, seed: int = 1006, variance: float = 2.0) -> Problem:
    """The paper's base case (Sec. 4.1): a log-normal permeability with the
    power-law autocorrelation, variance 2 of ln K, cutoff lengths 32 x 4
    cells at 15 degrees (0.016 and 0.002 on a quarter of the unit square at
    1000 cells), on an n x n grid of square cells; p = 1 at x = 0, p = 0 at
    x = 1, no flow on the other sides, no source; lifted boundary data.  The
    paper's own field is not published: this draws a field of the same
    statistics."""
    rng = np.random.default_rng(seed)
    lnk = np.sqrt(variance) * power_law_field(n, rng)
    bc, gD = standard_bc(2, (n, n))
    return Problem(dim=2, n=(n, n), h=(0.5 / n, 0.5 / n), K=np.exp(lnk).reshape(1, -1), bc=bc, gD=gD,
                   f=None, pbf=linear_lifting(2, (n, n)), name=f"base-case-{n}",
                   meta={"seed": seed, "lnK_variance": variance, "cutoff_cells": [32, 4], "angle_deg": 15})


def rescale(g: np.ndarray, lo: float, hi: float) -> np.ndarray:
    gmin, gmax = g.min(), g.max()
    return lo + (hi - lo) * (g - gmin) / (gmax - gmin)


def uniform_logk_problem(n=(32, 32), seed=1000, half_span=1.5) -> Problem:
    """i.i.d. log10 K ~ U[-half_span, half_span]; no source; lifted BCs."""
    rng = np.random.default_rng(seed)
    dim = len(n)
    shape = tuple(reversed(n))
    logk = rng.uniform(-half_span, half_span, size=shape)
    K = (10.0 ** logk).reshape(1, -1)
    bc, gD = standard_bc(dim, n)
    return Problem(dim=dim, n=tuple(n), h=tuple(1.0 / m for m in n), K=K, bc=bc, gD=gD,
                   f=None, pbf=linear_lifting(dim, n), name=f"uniform-logk-{'x'.join(map(str, n))}",
                   meta={"seed": seed, "log10K": [-half_span, half_span]})


def grf_problem(n=(1024, 1024), seed=1001, ell=16.0, half_span=4.5, source=True) -> Problem:
    """GRF log10 K rescaled to [-half_span, half_span]; N(0,1) source; lifted BCs."""
    rng = np.random.default_rng(seed)
    dim = len(n)
    shape = tuple(reversed(n))
    logk = rescale(gaussian_random_field(shape, ell, rng), -half_span, half_span)
    K = (10.0 ** logk).reshape(1, -1)
    f = rng.standard_normal(int(np.prod(n))) if source else None
    bc, gD = standard_bc(dim, n)
    return Problem(dim=dim, n=tuple(n), h=tuple(1.0 / m for m in n), K=K, bc=bc, gD=gD,
                   f=f, pbf=linear_lifting(dim, n), name=f"grf-{'x'.join(map(str, n))}",
                   meta={"seed": seed, "ell": ell, "log10K": [-half_span, half_span]})


def grf3d_problem(side: int = 128, seed: int = 1002) -> Problem:
    """3D Gaussian random field of the 3D workload's size: log10 K with
    correlation length 8 cells rescaled to [-4.5, 4.5] (1e9 contrast), N(0,1)
    source, lifted BCs.  Stands beside the layered channel field, on which
    the method does not converge at this size (oracle and GPU alike)."""
    return grf_problem((side, side, side), seed=seed, ell=8.0, half_span=4.5)


def strip_problem(n=(2000, 500), aspect: float = 10.0, seed: int = 1005, ell: float = 16.0,
                  half_span: float = 3.3, Ly: float = 0.25) -> Problem:
    """Anisotropic cells (Sec. 4.4): a log-normal field drawn on the n_x x n_y
    cell grid (correlation length `ell` cells, log10 K in [-half_span,
    half_span]) and read with cells `aspect` times longer in x than in y; at
    2000 x 500 and 10:1 the domain is 10 x 0.25, a channel 40 times longer
    than wide, as in the paper's narrow-channel test.  N(0,1) source, lifted
    standard boundary types."""
    rng = np.random.default_rng(seed)
    nx, ny = n
    logk = rescale(gaussian_random_field((ny, nx), ell, rng), -half_span, half_span)
    hy = Ly / ny
    bc, gD = standard_bc(2, n)
    return Problem(dim=2, n=(nx, ny), h=(aspect * hy, hy), K=(10.0 ** logk).reshape(1, -1), bc=bc, gD=gD,
                   f=rng.standard_normal(nx * ny), pbf=linear_lifting(2, n), name=f"strip-{nx}x{ny}-{aspect:g}to1",
                   meta={"seed": seed, "ell": ell, "log10K": [-half_span, half_span], "aspect": aspect})


def channel_problem(n=(128, 128, 128), seed=1002, slab=4, k_lo=1e-9, k_hi=1.0,
                    max_channels=4, wmin=2, wmax=8) -> Problem:
    """Layered 3D channel field.

    z-slabs of `slab` cells are K = k_hi or k_lo by Bernoulli(0.5); inside each
    slab, 1..max_channels rectangular channels of width U{wmin..wmax} cells in
    y, the slab's z cells, and a length of U{nx/4..nx} cells along x (random
    start) carry K = k_hi.  Channels of finite length keep the field varying
    along x; with full-length channels the linear lifting would already be
    the exact solution.
    """
    rng = np.random.default_rng(seed)
    nx, ny, nz = n
    Kc = np.empty((nz, ny, nx))
    for s0 in range(0, nz, slab):
        s1 = min(nz, s0 + slab)
        Kc[s0:s1] = k_hi if rng.random() < 0.5 else k_lo
        nch = int(rng.integers(1, max_channels + 1))
        for _ in range(nch):
            w = int(rng.integers(wmin, wmax + 1))
            w = min(w, ny)
            y0 = int(rng.integers(0, ny - w + 1))
            ln = int(rng.integers(max(1, nx // 4), nx + 1))
            x0 = int(rng.integers(0, nx - ln + 1))
            Kc[s0:s1, y0:y0 + w, x0:x0 + ln] = k_hi
    bc, gD = standard_bc(3, n)
    return Problem(dim=3, n=tuple(n), h=tuple(1.0 / m for m in n), K=Kc.reshape(1, -1), bc=bc, gD=gD,
                   f=None, pbf=linear_lifting(3, n), name=f"channel-{nx}x{ny}x{nz}",
                   meta={"seed": seed, "slab": slab, "K": [k_lo, k_hi]})


BATCH_SIDES = (64, 96, 128, 192, 256, 384, 512)


def batch_problem(j: int, seed_base: int = 3000, ell=8.0, half_span=3.0) -> Problem:
    """Problem j of the uneven batch: random side, GRF log10 K in [-3, 3],
    N(0,1) right-hand side used directly (standard boundary types)."""
    rng = np.random.default_rng(seed_base + j)
    side = int(rng.choice(BATCH_SIDES))
    n = (side, side)
    logk = rescale(gaussian_random_field((side, side), ell, rng), -half_span, half_span)
    K = (10.0 ** logk).reshape(1, -1)
    b = rng.standard_normal(side * side)
    bc, gD = standard_bc(2, n)
    return Problem(dim=2, n=n, h=(1.0 / side, 1.0 / side), K=K, bc=bc, gD=gD, b=b,
                   name=f"batch-{j}-{side}", meta={"seed": seed_base + j})


def batch_problems(count: int = 256, seed_base: int = 3000):
    return [batch_problem(j, seed_base) for j in range(count)]


def config_problem(i: int, scale: Optional[int] = None) -> Problem:
    """Workloads 0..2: 32^2 uniform log K, 1024^2 GRF (1e9 contrast), 128^3
    channels.  `scale` overrides the side length (tests use smaller cases)."""
    if i == 0:
        s = scale or 32
        return uniform_logk_problem((s, s), seed=1000)
    if i == 1:
        s = scale or 1024
        return grf_problem((s, s), seed=1001, ell=16.0, half_span=4.5)
    if i == 2:
        s = scale or 128
        return channel_problem((s, s, s), seed=1002)
    raise ValueError(i)


def serving_stream(count: int = 2000, rate_hz: float = 200.0, seed: int = 4004,
                   max_side_2d: int = 1024, max_side_3d: int = 96, channel_fraction: float = 0.5):
    """Poisson arrivals of mixed 2D / 3D requests.  Returns a list of
    (arrival_time_s, spec) with spec a dict that `serving_problem` expands;
    the fields themselves are drawn lazily so the stream stays small.
    channel_fraction: share of requests with the layered channel model
    (the rest are Gaussian random fields)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, size=count))
    out = []
    for r in range(count):
        is2d = rng.random() < 0.5
        if is2d:
            side = int(np.rint(np.exp(rng.uniform(np.log(32), np.log(max_side_2d)))))
        else:
            side = int(np.rint(np.exp(rng.uniform(np.log(32), np.log(max_side_3d)))))
        kind = "channel" if rng.random() < channel_fraction else "grf"
        decades = float(rng.uniform(2.0, 9.0))
        out.append((float(t[r]), {"dim": 2 if is2d else 3, "side": side, "kind": kind,
                                  "decades": decades, "seed": seed * 10000 + r}))
    return out


def serving_problem(spec: dict) -> Problem:
    """Expand one serving request: a GRF (ell = 8 cells) or channel field with
    10^decades contrast and an N(0,1) right-hand side used directly."""
    rng = np.random.default_rng(spec["seed"])
    dim, side, dec = spec["dim"], spec["side"], spec["decades"]
    n = (side,) * dim
    shape = (side,) * dim
    if spec["kind"] == "grf":
        logk = rescale(gaussian_random_field(shape, 8.0, rng), -dec / 2, dec / 2)
    else:
        logk = np.full(shape, -dec / 2)
        ax = 0  # layers stacked along the slowest axis, channels along x
        nlay = max(1, shape[ax] // 4)
        for s in range(nlay):
            sl = slice(4 * s, min(shape[ax], 4 * s + 4))
            if rng.random() < 0.5:
                logk[sl] = dec / 2
            w = int(rng.integers(2, 9))
            w = min(w, shape[1] if dim == 3 else shape[0])
            y0 = int(rng.integers(0, (shape[1] if dim == 3 else shape[0]) - w + 1))
            nx = shape[-1]
            ln = int(rng.integers(max(1, nx // 4), nx + 1))
            x0 = int(rng.integers(0, nx - ln + 1))
            if dim == 3:
                logk[sl, y0:y0 + w, x0:x0 + ln] = dec / 2
            else:
                logk[y0:y0 + w, x0:x0 + ln] = dec / 2
    K = (10.0 ** logk).reshape(1, -1)
    b = rng.standard_normal(int(np.prod(n)))
    bc, gD = standard_bc(dim, n)
    return Problem(dim=dim, n=n, h=tuple(1.0 / side for _ in n), K=K, bc=bc, gD=gD, b=b,
                   name=f"req-{spec['seed']}", meta=dict(spec))
