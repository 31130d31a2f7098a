"""Seeded synthetic inputs shaped like the paper's flood workloads.

The paper's DEMs, hydrographs and observations (Sect. 3) are not public, so
every input here is generated from a seed.  This module holds no arithmetic of
the method itself: it only writes vertex rasters (DEM, initial depth or free
surface, discharges), per-cell Manning coefficients and boundary forcing, which
both the CUDA library and the CPU oracle then project (Eq. 8) and evolve.

Workloads:
  dam_break_circular   uniform 128 x 128, dx = 1 m, flat frictionless bed,
                       h = 2 m inside r = 10 m, 0.5 m outside, walls
  valley               fractal terrain (amplitude spectrum slope -2, i.e. power
                       spectral density |k|^-4, 30 m relief, 1 m/km
                       west-east tilt) with a carved 40 m x 3 m meandering
                       channel fed by a triangular inflow hydrograph on the
                       west edge (rapid flow; shaped like Sect. 3.1)
  urban                1 m random-walk terrain, 8 m blocks 10-40 m on a side
                       covering 25 %, 12 m roads every 100 m with n = 0.013,
                       uniform rain (slow-to-gradual flow; shaped like
                       Sect. 3.2-3.3)
  lake_at_rest         seeded rough terrain under a flat free surface, with
                       optional emerging islands (well-balancing checks)
  dam_break_strip      y-invariant 1D dam break (Ritter dry bed, Stoker wet
                       bed)
  adjoint_reach        uniform crop of the valley terrain with water in the
                       channel, a 60-knot hydrograph over 1 h, spatially
                       varying Manning n and 16 gauge cells (gradient checks)
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

WALL, OPEN = 0, 1
WEST, EAST, SOUTH, NORTH = 0, 1, 2, 3
UNIFORM, STATIC, ADAPTIVE = 0, 1, 2


@dataclass
class Problem:
    """A flood problem on a finest grid of nx = M 2^L by ny = N 2^L cells."""
    name: str
    M: int
    N: int
    L: int
    dx: float
    z_vert: np.ndarray                  # (ny+1, nx+1) DEM at cell vertices
    h_vert: np.ndarray                  # (ny+1, nx+1) depth, or free surface if is_eta
    qx_vert: np.ndarray
    qy_vert: np.ndarray
    is_eta: bool = False
    n_manning: object = 0.0             # scalar or (ny, nx)
    bc: tuple = (WALL, WALL, WALL, WALL)
    inflow_edge: int = -1
    inflow_c0: int = 0
    inflow_c1: int = -1
    inflow_t: np.ndarray = field(default_factory=lambda: np.zeros(0))
    inflow_Q: np.ndarray = field(default_factory=lambda: np.zeros(0))
    rain_rate: float = 0.0
    rain_t_end: float = 0.0
    eps: float = 1e-3
    mode: int = UNIFORM
    t_end: float = 1.0
    limiter: int = 1
    dt_max: float = 1.0
    iface_rule: int = 0                 # static grids: 0 paper rule, 1 reflux
    scheme: int = 0                     # 0 DG2, 1 FV1 (adaptive: HWFV1)
    cfl: float = 0.33                   # Courant number (DG2 0.33, FV1 0.5)

    @property
    def nx(self) -> int:
        return self.M << self.L

    @property
    def ny(self) -> int:
        return self.N << self.L

    def n_cell(self) -> np.ndarray:
        return np.ascontiguousarray(
            np.broadcast_to(np.asarray(self.n_manning, np.float64), (self.ny, self.nx)))


def _vertex_xy(nx, ny, dx):
    x = np.arange(nx + 1) * dx
    y = np.arange(ny + 1) * dx
    return np.meshgrid(x, y)          # (ny+1, nx+1), row j = y


def dam_break_circular(n: int = 128, dx: float = 1.0, radius: float = 10.0, h_in: float = 2.0,
                       h_out: float = 0.5, L: int = 7, eps: float = 0.0, mode: int = UNIFORM,
                       t_end: float = 5.0) -> Problem:
    """Circular dam break on a flat frictionless bed (centre of the domain)."""
    X, Y = _vertex_xy(n, n, dx)
    c = 0.5 * n * dx
    r = np.hypot(X - c, Y - c)
    h = np.where(r <= radius, h_in, h_out)
    zeros = np.zeros_like(h)
    M = n >> L
    return Problem("dam_break_circular", M, M, L, dx, zeros.copy(), h, zeros.copy(), zeros.copy(),
                   n_manning=0.0, eps=eps, mode=mode, t_end=t_end)


def fractal_surface(nv: int, seed: int, beta: float = 2.0) -> np.ndarray:
    """(nv, nv) Fourier-synthesised surface with power spectral density
    |k|^-beta and random phases, zero mean, unit standard deviation."""
    rng = np.random.Generator(np.random.PCG64(seed))
    kx = np.fft.fftfreq(nv)[None, :]
    ky = np.fft.fftfreq(nv)[:, None]
    k = np.hypot(kx, ky)
    k[0, 0] = 1.0
    amp = k ** (-beta / 2.0)
    amp[0, 0] = 0.0
    noise = rng.standard_normal((nv, nv)) + 1j * rng.standard_normal((nv, nv))
    s = np.real(np.fft.ifft2(noise * amp))
    s -= s.mean()
    return s / s.std()


def valley(n: int = 1024, dx: float = 10.0, seed: int = 1, L: int = 10, relief: float = 30.0,
           beta: float = 4.0, tilt_per_km: float = 1.0, channel_width: float = 40.0,
           channel_depth: float = 3.0, peak_Q: float = 400.0, t_peak: float = 1800.0,
           n_manning: float = 0.035, eps: float = 1e-3, mode: int = ADAPTIVE,
           t_end: float = 7200.0) -> Problem:
    """Fractal terrain with a carved meandering channel and a triangular inflow
    hydrograph on the west edge, entering through the channel cells."""
    nv = n + 1
    X, Y = _vertex_xy(n, n, dx)
    Lx = n * dx
    z = fractal_surface(nv, seed, beta)
    z = (z - z.min()) / (z.max() - z.min()) * relief
    z = z - tilt_per_km * 1e-3 * X                  # drains west -> east
    # channel centre line y_c(x) and a bed that never rises downstream
    yc = 0.5 * Lx + 0.15 * Lx * np.sin(2.0 * np.pi * X[0] / (0.5 * Lx))
    jc = np.clip(np.rint(yc / dx).astype(int), 0, n)
    centre = z[jc, np.arange(nv)]
    bed = np.minimum.accumulate(centre) - channel_depth
    inside = np.abs(Y - yc[None, :]) <= 0.5 * channel_width
    z = np.where(inside, np.minimum(z, bed[None, :]), z)
    # inflow cells on the west edge: cells whose centre is in the channel
    yc0 = yc[0]
    jcell = np.arange(n)
    ycell = (jcell + 0.5) * dx
    sel = np.nonzero(np.abs(ycell - yc0) <= 0.5 * channel_width)[0]
    c0, c1 = int(sel.min()), int(sel.max())
    zeros = np.zeros((nv, nv))
    M = n >> L
    return Problem("valley", M, M, L, dx, z, zeros.copy(), zeros.copy(), zeros.copy(),
                   n_manning=n_manning, inflow_edge=WEST, inflow_c0=c0, inflow_c1=c1,
                   inflow_t=np.array([0.0, t_peak, 2.0 * t_peak, max(t_end, 2.0 * t_peak) + 1.0]),
                   inflow_Q=np.array([0.0, peak_Q, 0.0, 0.0]), eps=eps, mode=mode, t_end=t_end)


def ensemble(count: int = 64, seed: int = 4, base_seed: int = 1000, sides=(256, 512, 768, 1024),
             n_range=(0.02, 0.06), q_scale=(0.5, 2.0), eps: float = 1e-3, dx: float = 10.0) -> list:
    """Batched scenarios of uneven sizes: fractal valleys (as `valley`) with
    sides drawn from `sides` (each M 2^L with M in {1, 3}), member k seeded
    base_seed + k, Manning n ~ U(n_range) and the inflow peak scaled by
    U(q_scale)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for k in range(count):
        side = int(rng.choice(sides))
        M = 3 if side % 3 == 0 else 1
        L = int(np.log2(side // M))
        nm = float(rng.uniform(*n_range))
        qs = float(rng.uniform(*q_scale))
        out.append(valley(n=side, dx=dx, seed=base_seed + k, L=L, n_manning=nm, peak_Q=400.0 * qs,
                          eps=eps))
    return out


def urban(n: int = 2048, dx: float = 2.0, seed: int = 2, L: int = 11, relief: float = 1.0,
          block_min: float = 10.0, block_max: float = 40.0, block_height: float = 8.0,
          cover: float = 0.25, road_spacing: float = 100.0, road_width: float = 12.0,
          n_road: float = 0.013, n_other: float = 0.035, rain_mm_per_h: float = 50.0,
          rain_hours: float = 1.0, eps: float = 1e-2, mode: int = STATIC,
          t_end: float = 3.0 * 3600.0) -> Problem:
    """Urban-like DEM: random-walk terrain, buildings off a road grid, rain."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nv = n + 1
    X, Y = _vertex_xy(n, n, dx)
    a = np.cumsum(rng.standard_normal(nv))
    b = np.cumsum(rng.standard_normal(nv))
    z = a[None, :] + b[:, None]
    z = (z - z.min()) / (z.max() - z.min()) * relief
    # roads on cell centres
    xc = (np.arange(n) + 0.5) * dx
    road_x = np.mod(xc, road_spacing) < road_width
    road = road_x[None, :] | road_x[:, None]
    ncell = np.where(road, n_road, n_other)
    # buildings: rectangles on non-road cells until the cover is reached
    occ = np.zeros((n, n), bool)
    target = cover * n * n
    tries = 0
    while occ.sum() < target and tries < 200000:
        tries += 1
        w = int(rng.uniform(block_min, block_max) / dx)
        h = int(rng.uniform(block_min, block_max) / dx)
        i0 = int(rng.integers(0, n - w))
        j0 = int(rng.integers(0, n - h))
        if road[j0:j0 + h, i0:i0 + w].any():
            continue
        occ[j0:j0 + h, i0:i0 + w] = True
    # raise every vertex touching a building cell
    vb = np.zeros((nv, nv), bool)
    vb[:-1, :-1] |= occ
    vb[1:, :-1] |= occ
    vb[:-1, 1:] |= occ
    vb[1:, 1:] |= occ
    z = z + np.where(vb, block_height, 0.0)
    zeros = np.zeros((nv, nv))
    M = n >> L
    return Problem("urban", M, M, L, dx, z, zeros.copy(), zeros.copy(), zeros.copy(),
                   n_manning=ncell, rain_rate=rain_mm_per_h * 1e-3 / 3600.0,
                   rain_t_end=rain_hours * 3600.0, eps=eps, mode=mode, t_end=t_end)


def lake_at_rest(n: int = 64, dx: float = 1.0, seed: int = 3, L: int = 0, eta: float = 1.5,
                 relief: float = 1.0, islands: bool = False, mode: int = UNIFORM,
                 eps: float = 1e-3, n_manning: float = 0.03) -> Problem:
    """Flat free surface over seeded rough terrain.  With islands, terrain
    pokes above the surface; vertices of cells that start dry are raised so
    that no dry cell has an interface centre below the surface (the
    piecewise-planar initial state is then exactly at rest)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nv = n + 1
    z = rng.uniform(0.0, relief, (nv, nv))
    if islands:
        X, Y = _vertex_xy(n, n, dx)
        c = 0.5 * n * dx
        bump = 2.5 * eta * np.exp(-((X - 0.3 * c) ** 2 + (Y - 0.6 * c) ** 2) / (0.05 * (n * dx) ** 2))
        bump += 2.0 * eta * np.exp(-((X - 1.4 * c) ** 2 + (Y - 1.3 * c) ** 2) / (0.03 * (n * dx) ** 2))
        z = z + bump
        for _ in range(100):
            z0 = 0.25 * (z[:-1, :-1] + z[1:, :-1] + z[:-1, 1:] + z[1:, 1:])
            dry = z0 >= eta
            vb = np.zeros((nv, nv), bool)
            vb[:-1, :-1] |= dry
            vb[1:, :-1] |= dry
            vb[:-1, 1:] |= dry
            vb[1:, 1:] |= dry
            low = vb & (z < eta + 0.05)
            if not low.any():
                break
            z = np.where(low, eta + 0.05 + 0.1 * rng.uniform(size=z.shape), z)
    e = np.full((nv, nv), eta)
    zeros = np.zeros((nv, nv))
    M = n >> L
    return Problem("lake_at_rest", M, M, L, dx, z, e, zeros.copy(), zeros.copy(), is_eta=True,
                   n_manning=n_manning, mode=mode, eps=eps)


def dam_break_strip(nx: int = 256, ny: int = 4, dx: float = 0.5, h_left: float = 1.0,
                    h_right: float = 0.0, x0_frac: float = 0.5, L: int = 0) -> Problem:
    """y-invariant dam break in a walled strip (Ritter when h_right = 0,
    Stoker otherwise)."""
    X, _ = _vertex_xy(nx, ny, dx)
    x0 = x0_frac * nx * dx
    h = np.where(X < x0, h_left, np.where(X > x0, h_right, 0.5 * (h_left + h_right)))
    zeros = np.zeros_like(h)
    M, N = nx >> L, ny >> L
    return Problem("dam_break_strip", M, N, L, dx, zeros.copy(), h, zeros.copy(), zeros.copy(),
                   n_manning=0.0, limiter=1)


def fv1(p: Problem) -> Problem:
    """The same problem solved by FV1 (Sect. 2.1.2; adaptive: HWFV1), at its
    Courant number 0.5."""
    return replace(p, scheme=1, cfl=0.5)


def acc(p: Problem) -> Problem:
    """The same problem solved by ACC (Sect. 2.1.3), at its Courant number 0.7."""
    return replace(p, scheme=2, cfl=0.7)


def sloped_channel(nx: int = 256, ny: int = 4, dx: float = 10.0, slope: float = 1e-3, q_in: float = 2.0,
                   n_manning: float = 0.03) -> Problem:
    """A y-invariant strip with a uniform bed slope falling eastward, unit
    inflow q_in (m^2/s) through the whole west edge and an open east edge."""
    X, Y = _vertex_xy(nx, ny, dx)
    z = slope * (nx * dx - X)
    zeros = np.zeros_like(z)
    Lx = nx * dx
    return Problem("sloped_channel", nx, ny, 0, dx, z, zeros.copy(), zeros.copy(), zeros.copy(),
                   n_manning=n_manning, bc=(WALL, OPEN, WALL, WALL), inflow_edge=WEST, inflow_c0=0,
                   inflow_c1=ny - 1, inflow_t=np.array([0.0, 1e9]), inflow_Q=np.array([q_in * ny * dx] * 2),
                   mode=UNIFORM, t_end=1e9)


def crop(p: Problem, i0: int, j0: int, nx: int, ny: int, L: int) -> Problem:
    """A window of a problem (finest cells [i0, i0+nx) x [j0, j0+ny)) as its own
    problem with maximum level L; the inflow segment is clipped to it."""
    sl = (slice(j0, j0 + ny + 1), slice(i0, i0 + nx + 1))
    nm = p.n_manning
    if np.ndim(nm) == 2:
        nm = np.ascontiguousarray(np.asarray(nm)[j0:j0 + ny, i0:i0 + nx])
    edge, c0, c1 = p.inflow_edge, p.inflow_c0, p.inflow_c1
    if edge in (WEST, EAST):
        on = (edge == WEST and i0 == 0) or (edge == EAST and i0 + nx == p.nx)
        c0, c1 = max(c0, j0) - j0, min(c1, j0 + ny - 1) - j0
    elif edge in (SOUTH, NORTH):
        on = (edge == SOUTH and j0 == 0) or (edge == NORTH and j0 + ny == p.ny)
        c0, c1 = max(c0, i0) - i0, min(c1, i0 + nx - 1) - i0
    else:
        on = False
    Q = p.inflow_Q
    if not on or c1 < c0:
        edge, c0, c1 = -1, 0, -1
    else:
        # keep the unit discharge: the crop carries its share of the hydrograph
        Q = Q * (c1 - c0 + 1) / (p.inflow_c1 - p.inflow_c0 + 1)
    return replace(p, name=p.name + "_crop", M=nx >> L, N=ny >> L, L=L, inflow_Q=Q,
                   z_vert=np.ascontiguousarray(p.z_vert[sl]),
                   h_vert=np.ascontiguousarray(p.h_vert[sl]),
                   qx_vert=np.ascontiguousarray(p.qx_vert[sl]),
                   qy_vert=np.ascontiguousarray(p.qy_vert[sl]),
                   n_manning=nm, inflow_edge=edge, inflow_c0=c0, inflow_c1=c1)


def adjoint_reach(n: int = 64, dx: float = 10.0, seed: int = 5, knots: int = 60, t_span: float = 3600.0,
                  n_gauges: int = 16, depth0: float = 1.0, relief: float = 10.0, q_unit: float = 1.0,
                  n_mean: float = 0.035, crop_of: int = 0) -> tuple:
    """Gradient workload: an n x n uniform grid of valley terrain with a channel
    holding about depth0 metres of flowing water over each column's lowest
    point, an open east edge, a piecewise-linear inflow hydrograph of `knots`
    seeded positive knots over t_span seconds (unit discharge around q_unit)
    and a spatially varying Manning n (n_mean +- 30 %).  The terrain is a small
    valley of its own (seed `seed`, `relief` metres, 4-cell channel), or with
    crop_of = N the n x n window at the inlet of the N x N valley (seed 1,
    30 m relief, 40 m channel).  Returns (problem, gauges), gauges an
    (n_gauges, 2) array of (j, i) cells drawn from the initially wet ones."""
    if crop_of:
        big = valley(n=crop_of, dx=dx, seed=1, L=0, mode=UNIFORM, t_end=t_span)
        mid = (big.inflow_c0 + big.inflow_c1) // 2
        j0 = int(min(max(mid - n // 2, 0), crop_of - n))
        p = crop(big, 0, j0, n, n, 0)
    else:
        p = valley(n=n, dx=dx, seed=seed, L=0, relief=relief, channel_width=4.0 * dx, channel_depth=2.0,
                   mode=UNIFORM, t_end=t_span)
    rng = np.random.Generator(np.random.PCG64(seed))
    z = p.z_vert
    # a flowing start: a rippled free surface over the channel and a seeded
    # discharge field (a derivative needs a state away from rest, where the
    # limiter's differences are all zero)
    ripple = fractal_surface(n + 1, seed + 2, 4.0)
    eta = z.min(axis=0, keepdims=True) + depth0 + 0.1 * ripple / np.abs(ripple).max()
    h = np.maximum(0.0, eta - z)
    swirl = fractal_surface(n + 1, seed + 3, 4.0)
    qx = h * (0.5 + 0.2 * swirl / np.abs(swirl).max())
    qy = h * (0.2 * ripple / np.abs(ripple).max())
    nin = p.inflow_c1 - p.inflow_c0 + 1
    t = np.linspace(0.0, t_span, knots)
    Q = q_unit * nin * dx * (0.6 + 0.8 * rng.random(knots))
    rough = fractal_surface(n + 1, seed + 1, 3.0)[:n, :n]
    nm = np.clip(n_mean * (1.0 + 0.3 * rough / max(1e-12, np.abs(rough).max())), 0.5 * n_mean, 1.5 * n_mean)
    q = replace(p, name="adjoint_reach", h_vert=h, qx_vert=qx, qy_vert=qy, n_manning=np.ascontiguousarray(nm),
                bc=(WALL, OPEN, WALL, WALL), inflow_t=t, inflow_Q=Q)
    hc = 0.25 * (h[:-1, :-1] + h[1:, :-1] + h[:-1, 1:] + h[1:, 1:])
    wet = np.argwhere(hc > 0.25 * depth0)
    pick = rng.choice(len(wet), size=min(n_gauges, len(wet)), replace=False)
    return q, np.ascontiguousarray(wet[np.sort(pick)].astype(np.int64))
