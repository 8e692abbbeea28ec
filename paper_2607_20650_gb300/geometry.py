"""Seeded synthetic inputs: solid masks, initial fields and case parameters.

This module holds no lattice-Boltzmann arithmetic; it only produces inputs
that the CUDA path and the CPU oracle both consume. Scenarios follow the
paper's benchmark families (Sec. 4: Hagen-Poiseuille, Karman street behind an
obstacle, porous medium of random solid nodes, wing at an angle of attack) at
the sizes of the workloads below.

Random numbers: splitmix64 (Steele, Lea & Flood, OOPSLA 2014), one stream
per use, seeded with ``seed ^ splitmix64(stream_id)``; doubles are
``(x >> 11) * 2**-53``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Edge-condition codes (identical numbering in the C ABI header).
PERIODIC, WALL, FREESLIP, INLET_ZOUHE, INLET_EQ, OUTFLOW_ZG, INLET_EQ_NEUMANN, OUTLET_PRESSURE = range(8)

_M64 = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15


def _mix64(z: int) -> int:
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9 & _M64
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB & _M64
    return z ^ (z >> 31)


class SplitMix64:
    """splitmix64 stream; vectorised draws with numpy uint64 arithmetic."""

    def __init__(self, seed: int, stream_id: int = 0):
        self.state = (seed ^ _mix64((stream_id * _GAMMA + _GAMMA) & _M64)) & _M64

    def u64(self, n: int) -> np.ndarray:
        with np.errstate(over="ignore"):
            k = np.arange(1, n + 1, dtype=np.uint64)
            z = np.uint64(self.state) + k * np.uint64(_GAMMA)
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            z = z ^ (z >> np.uint64(31))
        self.state = (self.state + n * _GAMMA) & _M64
        return z

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (self.u64(n) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
        return lo + (hi - lo) * u

    def integers(self, n: int, lo: int, hi_inclusive: int) -> np.ndarray:
        span = hi_inclusive - lo + 1
        return lo + np.floor(self.uniform(n) * span).astype(np.int64)


# ----------------------------------------------------------------- masks

def channel_walls(nx: int, ny: int) -> np.ndarray:
    """Solid rows y = 0 and y = ny - 1 (Hagen-Poiseuille channel)."""
    m = np.zeros((ny, nx), np.uint8)
    m[0, :] = 1
    m[-1, :] = 1
    return m


def disc(nx: int, ny: int, xc: float, yc: float, r: float, periodic: bool = False,
         out: np.ndarray | None = None) -> np.ndarray:
    """Nodes (x, y) with (x - xc)^2 + (y - yc)^2 <= r^2 set to 1."""
    m = np.zeros((ny, nx), np.uint8) if out is None else out
    x0, x1 = int(math.floor(xc - r)), int(math.ceil(xc + r))
    y0, y1 = int(math.floor(yc - r)), int(math.ceil(yc + r))
    xs = np.arange(x0, x1 + 1)
    ys = np.arange(y0, y1 + 1)
    inside = (xs[None, :] - xc) ** 2 + (ys[:, None] - yc) ** 2 <= r * r
    if periodic:
        m[np.ix_(ys % ny, xs % nx)] |= inside.astype(np.uint8)
    else:
        kx = (xs >= 0) & (xs < nx)
        ky = (ys >= 0) & (ys < ny)
        m[np.ix_(ys[ky], xs[kx])] |= inside[np.ix_(ky, kx)].astype(np.uint8)
    return m


def porous_discs(nx: int, ny: int, seed: int, rmin: float = 8.0, rmax: float = 32.0,
                 solid_fraction: float = 0.4) -> np.ndarray:
    """Random overlapping discs on a periodic domain until the solid fraction
    reaches ``solid_fraction``: centres uniform in [0,nx) x [0,ny), radii
    uniform in [rmin, rmax], minimum-image (periodic) rasterisation."""
    m = np.zeros((ny, nx), np.uint8)
    rng = SplitMix64(seed, 1)
    target = solid_fraction * nx * ny
    solid = 0
    while solid < target:
        batch = rng.uniform(3 * 256).reshape(256, 3)
        for u, v, w in batch:
            xc, yc = u * nx, v * ny
            r = rmin + (rmax - rmin) * w
            x0, x1 = int(math.floor(xc - r)), int(math.ceil(xc + r))
            y0, y1 = int(math.floor(yc - r)), int(math.ceil(yc + r))
            xs = np.arange(x0, x1 + 1)
            ys = np.arange(y0, y1 + 1)
            inside = (xs[None, :] - xc) ** 2 + (ys[:, None] - yc) ** 2 <= r * r
            ix = np.ix_(ys % ny, xs % nx)
            before = int(m[ix].sum())
            m[ix] |= inside.astype(np.uint8)
            solid += int(m[ix].sum()) - before
            if solid >= target:
                break
    return m


def square(nx: int, ny: int, xc: float, yc: float, size: int) -> np.ndarray:
    m = np.zeros((ny, nx), np.uint8)
    x0, y0 = int(round(xc - size / 2)), int(round(yc - size / 2))
    m[max(y0, 0):min(y0 + size, ny), max(x0, 0):min(x0 + size, nx)] = 1
    return m


def plate(nx: int, ny: int, xc: float, yc: float, height: int, thickness: int = 2) -> np.ndarray:
    m = np.zeros((ny, nx), np.uint8)
    x0, y0 = int(round(xc - thickness / 2)), int(round(yc - height / 2))
    m[max(y0, 0):min(y0 + height, ny), max(x0, 0):min(x0 + thickness, nx)] = 1
    return m


def naca4_outline(m: float, p: float, t: float, chord: float, n: int = 2048) -> np.ndarray:
    """Closed NACA 4-digit outline (camber m, camber position p, thickness t)
    from the standard closed-form thickness and camber-line equations, with a
    closed trailing edge (last thickness coefficient -0.1036) and cosine
    spacing; returns (2n-1, 2) points, leading edge at the origin."""
    beta = np.linspace(0.0, math.pi, n)
    xc = 0.5 * (1.0 - np.cos(beta))
    yt = 5.0 * t * (0.2969 * np.sqrt(xc) - 0.1260 * xc - 0.3516 * xc ** 2
                    + 0.2843 * xc ** 3 - 0.1036 * xc ** 4)
    fore = xc < p
    yc = np.where(fore, m / p ** 2 * (2 * p * xc - xc ** 2),
                  m / (1 - p) ** 2 * ((1 - 2 * p) + 2 * p * xc - xc ** 2))
    dyc = np.where(fore, 2 * m / p ** 2 * (p - xc), 2 * m / (1 - p) ** 2 * (p - xc))
    th = np.arctan(dyc)
    xu, yu = xc - yt * np.sin(th), yc + yt * np.cos(th)
    xl, yl = xc + yt * np.sin(th), yc - yt * np.cos(th)
    x = np.concatenate([xu[::-1], xl[1:]])
    y = np.concatenate([yu[::-1], yl[1:]])
    return np.stack([x, y], axis=1) * chord


def polygon_mask(nx: int, ny: int, poly: np.ndarray) -> np.ndarray:
    """Nodes inside a closed polygon (even-odd rule), by scanlines."""
    m = np.zeros((ny, nx), np.uint8)
    x0, y0 = poly[:, 0], poly[:, 1]
    x1, y1 = np.roll(x0, -1), np.roll(y0, -1)
    for yy in range(max(0, int(math.floor(y0.min()))), min(ny, int(math.ceil(y0.max())) + 1)):
        Y = float(yy)
        hit = ((y0 <= Y) & (y1 > Y)) | ((y1 <= Y) & (y0 > Y))
        if not hit.any():
            continue
        xs = x0[hit] + (Y - y0[hit]) * (x1[hit] - x0[hit]) / (y1[hit] - y0[hit])
        xs.sort()
        for a, b in zip(xs[0::2], xs[1::2]):
            lo = max(0, int(math.ceil(a)))
            hi = min(nx - 1, int(math.floor(b)))
            if hi >= lo:
                m[yy, lo:hi + 1] = 1
    return m


def naca_wing(nx: int, ny: int, chord: float, aoa_deg: float = 8.0,
              digits=(0.02, 0.4, 0.12), n_points: int = 2048) -> np.ndarray:
    """NACA airfoil (default 2412) with leading edge at (nx/4, ny/2), rotated
    nose-up by ``aoa_deg`` about its quarter-chord point."""
    pts = naca4_outline(*digits, chord=chord, n=n_points)
    a = -math.radians(aoa_deg)
    qc = np.array([0.25 * chord, 0.0])
    rot = np.array([[math.cos(a), -math.sin(a)], [math.sin(a), math.cos(a)]])
    pts = (pts - qc) @ rot.T + qc
    pts = pts + np.array([nx / 4.0, ny / 2.0])
    return polygon_mask(nx, ny, pts)


# ----------------------------------------------------------------- workloads

def tau_from_reynolds(u: float, length: float, re: float) -> float:
    """tau = 3 nu + 1/2 with nu = u L / Re (lattice units)."""
    return 3.0 * u * length / re + 0.5


@dataclass
class Workload:
    """One lattice case with its mask and optional initial fields."""
    name: str
    nx: int
    ny: int
    tau: float
    mask: np.ndarray
    fx: float = 0.0
    fy: float = 0.0
    ux_in: float = 0.0
    uy_in: float = 0.0
    bc_w: int = PERIODIC
    bc_e: int = PERIODIC
    bc_s: int = PERIODIC
    bc_n: int = PERIODIC
    ux0: np.ndarray | None = None
    uy0: np.ndarray | None = None
    body: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def cells(self) -> int:
        return self.nx * self.ny


def poiseuille(nx: int = 256, ny: int = 64, tau: float = 0.8, g: float = 1e-6) -> Workload:
    """Body-force-driven channel, periodic in x, solid rows 0 and ny-1."""
    return Workload("poiseuille", nx, ny, tau, channel_walls(nx, ny), fx=g,
                    meta={"H": ny - 2, "g": g}, body=channel_walls(nx, ny))


def karman(nx: int = 2048, ny: int = 512, u: float = 0.05, diameter: int = 64,
           centre=(400, 256), re: float = 200.0, seed: int = 2, perturb: float = 1e-3) -> Workload:
    """Cylinder in a channel: Zou-He inlet, zero-gradient outflow, free-slip
    top/bottom; initial u = (U, eps) with eps ~ U(-perturb, perturb)."""
    mask = disc(nx, ny, centre[0], centre[1], diameter / 2)
    rng = SplitMix64(seed, 2)
    uy0 = rng.uniform(nx * ny, -perturb, perturb).reshape(ny, nx)
    ux0 = np.full((ny, nx), u)
    ux0[mask > 0] = 0.0
    uy0[mask > 0] = 0.0
    return Workload("karman", nx, ny, tau_from_reynolds(u, diameter, re), mask,
                    ux_in=u, bc_w=INLET_ZOUHE, bc_e=OUTFLOW_ZG, bc_s=FREESLIP, bc_n=FREESLIP,
                    ux0=ux0, uy0=uy0, body=mask.copy(),
                    meta={"U": u, "L": diameter, "Re": re})


def porous(nx: int = 16384, ny: int = 8192, tau: float = 0.9, g: float = 1e-6,
           seed: int = 3) -> Workload:
    """Periodic porous medium of random discs, body force g_x."""
    return Workload("porous", nx, ny, tau, porous_discs(nx, ny, seed), fx=g,
                    meta={"seed": seed})


def wing(nx: int = 8192, ny: int = 4096, chord: int = 1024, u: float = 0.05,
         re: float = 1000.0, aoa: float = 8.0) -> Workload:
    """NACA 2412 at ``aoa`` degrees: Zou-He inlet, zero-gradient outflow,
    free-slip top/bottom, uniform initial velocity U."""
    mask = naca_wing(nx, ny, chord, aoa)
    ux0 = np.full((ny, nx), u)
    ux0[mask > 0] = 0.0
    return Workload("wing", nx, ny, tau_from_reynolds(u, chord, re), mask, ux_in=u,
                    bc_w=INLET_ZOUHE, bc_e=OUTFLOW_ZG, bc_s=FREESLIP, bc_n=FREESLIP,
                    ux0=ux0, uy0=np.zeros((ny, nx)), body=mask.copy(),
                    meta={"U": u, "L": chord, "Re": re, "aoa": aoa})


def batch_channels(ncases: int = 256, seed: int = 4, wmin: int = 64, wmax: int = 1024,
                   hmin: int = 32, hmax: int = 512) -> list[Workload]:
    """Independent channels: width/height/tau/inlet speed uniform, one obstacle
    (cylinder, square or plate of size 8-64, clamped to h/2) at (w/4, h/2);
    half-way walls top/bottom, Zou-He inlet, zero-gradient outflow."""
    rng = SplitMix64(seed, 4)
    w = rng.integers(ncases, wmin, wmax)
    h = rng.integers(ncases, hmin, hmax)
    tau = rng.uniform(ncases, 0.55, 1.5)
    uin = rng.uniform(ncases, 0.02, 0.08)
    kind = rng.integers(ncases, 0, 2)
    size = rng.integers(ncases, 8, 64)
    out = []
    for c in range(ncases):
        nx, ny = int(w[c]), int(h[c])
        s = int(min(size[c], ny // 2))
        xc, yc = nx / 4.0, ny / 2.0
        if kind[c] == 0:
            mask = disc(nx, ny, xc, yc, s / 2)
        elif kind[c] == 1:
            mask = square(nx, ny, xc, yc, s)
        else:
            mask = plate(nx, ny, xc, yc, s)
        ux0 = np.full((ny, nx), float(uin[c]))
        ux0[mask > 0] = 0.0
        out.append(Workload(f"channel{c}", nx, ny, float(tau[c]), mask, ux_in=float(uin[c]),
                            bc_w=INLET_ZOUHE, bc_e=OUTFLOW_ZG, bc_s=WALL, bc_n=WALL,
                            ux0=ux0, uy0=np.zeros((ny, nx)), body=mask.copy(),
                            meta={"kind": ["cylinder", "square", "plate"][int(kind[c])],
                                  "size": s}))
    return out


# ------------------------------------------------------------ D3Q19 inputs

def porous_spheres(nx: int, ny: int, nz: int, seed: int, rmin: float = 4.0, rmax: float = 12.0,
                   solid_fraction: float = 0.3) -> np.ndarray:
    """3-D counterpart of porous_discs: random overlapping spheres on a
    periodic box until the solid fraction is reached; mask[z, y, x]."""
    m = np.zeros((nz, ny, nx), np.uint8)
    rng = SplitMix64(seed, 5)
    target = solid_fraction * nx * ny * nz
    solid = 0
    while solid < target:
        batch = rng.uniform(4 * 256).reshape(256, 4)
        for u, v, s, w in batch:
            xc, yc, zc = u * nx, v * ny, s * nz
            r = rmin + (rmax - rmin) * w
            xs = np.arange(int(math.floor(xc - r)), int(math.ceil(xc + r)) + 1)
            ys = np.arange(int(math.floor(yc - r)), int(math.ceil(yc + r)) + 1)
            zs = np.arange(int(math.floor(zc - r)), int(math.ceil(zc + r)) + 1)
            inside = ((xs[None, None, :] - xc) ** 2 + (ys[None, :, None] - yc) ** 2
                      + (zs[:, None, None] - zc) ** 2) <= r * r
            ix = np.ix_(zs % nz, ys % ny, xs % nx)
            before = int(m[ix].sum())
            m[ix] |= inside.astype(np.uint8)
            solid += int(m[ix].sum()) - before
            if solid >= target:
                break
    return m


def ball(nx: int, ny: int, nz: int, xc: float, yc: float, zc: float, r: float) -> np.ndarray:
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx]
    return (((x - xc) ** 2 + (y - yc) ** 2 + (z - zc) ** 2) <= r * r).astype(np.uint8)
