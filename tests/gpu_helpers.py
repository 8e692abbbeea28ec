"""Shared set-up for the GPU parity tests: small seeded cases that span
several 32x8 tiles with ragged tails, built once for both the CUDA path and
the FP64 oracle from the same inputs."""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import numpy as np

import oracle as O
from paper_2607_20650_gb300 import geometry as G

LAYOUTS = ("stream", "bundle", "collision")
ALGOS = ("lptl", "nptl", "npol", "nsol")
COMBOS = list(itertools.product(LAYOUTS, ALGOS))


@dataclass
class Spec:
    name: str
    nx: int
    ny: int
    tau: float
    mask: np.ndarray
    bc: tuple
    force: tuple = (0.0, 0.0)
    u_in: tuple = (0.0, 0.0)
    rho0: np.ndarray | None = None
    rho_out: float = 1.0
    ux0: np.ndarray | None = None
    uy0: np.ndarray | None = None

    def oracle(self) -> O.Lattice:
        c = O.Case(self.nx, self.ny, self.tau, fx=self.force[0], fy=self.force[1],
                   ux_in=self.u_in[0], uy_in=self.u_in[1], bc_w=self.bc[0], bc_e=self.bc[1],
                   bc_s=self.bc[2], bc_n=self.bc[3], rho_out=self.rho_out)
        return O.Lattice(c, self.mask, rho=self.rho0, ux=self.ux0, uy=self.uy0)

    def gpu(self, **kw):
        from paper_2607_20650_gb300 import lbm
        kw.setdefault("rho_out", self.rho_out)
        lat = lbm.Lattice(self.nx, self.ny, self.tau, self.mask, force=self.force, u_in=self.u_in,
                          bc=self.bc, **kw)
        lat.init(self.rho0, self.ux0, self.uy0)
        return lat


def specs() -> dict[str, Spec]:
    out = {}
    # Channel with a cylinder: Zou-He inlet, zero-gradient outflow, free-slip walls.
    nx, ny = 61, 29
    m = G.disc(nx, ny, 15.0, 14.0, 4.5)
    r = G.SplitMix64(7, 9)
    ux0 = np.where(m.ravel() > 0, 0.0, 0.05)
    uy0 = np.where(m.ravel() > 0, 0.0, r.uniform(nx * ny, -1e-3, 1e-3))
    out["channel"] = Spec("channel", nx, ny, 0.6, m, (G.INLET_ZOUHE, G.OUTFLOW_ZG, G.FREESLIP, G.FREESLIP),
                          u_in=(0.05, 0.0), ux0=ux0, uy0=uy0)
    # Forced channel between half-way wall edges with an obstacle block.
    nx, ny = 37, 21
    m = np.zeros((ny, nx), np.uint8)
    m[6:12, 10:14] = 1
    out["walls"] = Spec("walls", nx, ny, 0.8, m, (G.PERIODIC, G.PERIODIC, G.WALL, G.WALL),
                        force=(1e-5, 0.0))
    # Periodic porous medium, forced, perturbed initial density and velocity.
    nx, ny = 67, 45
    m = G.porous_discs(nx, ny, seed=5, rmin=3, rmax=6, solid_fraction=0.35)
    r = G.SplitMix64(8, 9)
    out["porous"] = Spec("porous", nx, ny, 0.9, m, (G.PERIODIC,) * 4, force=(1e-5, 2e-6),
                         rho0=1.0 + r.uniform(nx * ny, -1e-3, 1e-3),
                         ux0=r.uniform(nx * ny, -1e-2, 1e-2), uy0=r.uniform(nx * ny, -1e-2, 1e-2))
    # Equilibrium inlet, wall east, wall south, free-slip north.
    nx, ny = 45, 23
    m = np.zeros((ny, nx), np.uint8)
    m[8:15, 20:23] = 1
    out["eq_inlet"] = Spec("eq_inlet", nx, ny, 0.7, m, (G.INLET_EQ, G.WALL, G.WALL, G.FREESLIP),
                           u_in=(0.04, 0.005), ux0=np.full(nx * ny, 0.02))
    # The paper's own pair: equilibrium inlet with Neumann density, Zou-He
    # pressure outlet; free-slip south, wall north.
    nx, ny = 58, 21
    m = G.square(nx, ny, 22.0, 9.0, 5)
    r = G.SplitMix64(14, 9)
    out["neumann_pressure"] = Spec("neumann_pressure", nx, ny, 0.75, m,
                                   (G.INLET_EQ_NEUMANN, G.OUTLET_PRESSURE, G.FREESLIP, G.WALL),
                                   u_in=(0.04, 0.0), rho0=1.0 + r.uniform(nx * ny, -1e-3, 1e-3),
                                   ux0=np.where(m.ravel() > 0, 0.0, 0.04))
    return out


def rel_linf(a, b, mask=None):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if mask is not None:
        a, b = a[..., mask], b[..., mask]
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def aa_specs() -> dict[str, Spec]:
    """Cases the AA pattern supports (every edge kind but zero-gradient
    outflow): the periodic/wall/equilibrium-inlet specs above plus a Zou-He
    channel closed by a wall at the east end, free-slip top and bottom."""
    out = {k: v for k, v in specs().items() if G.OUTFLOW_ZG not in v.bc and G.INLET_EQ_NEUMANN not in v.bc}
    nx, ny = 53, 27
    m = G.disc(nx, ny, 20.0, 13.0, 4.0)
    r = G.SplitMix64(12, 9)
    out["zouhe_wall"] = Spec("zouhe_wall", nx, ny, 0.7, m, (G.INLET_ZOUHE, G.WALL, G.FREESLIP, G.FREESLIP),
                             u_in=(0.03, 0.002), ux0=np.where(m.ravel() > 0, 0.0, 0.03),
                             uy0=np.where(m.ravel() > 0, 0.0, r.uniform(nx * ny, -1e-3, 1e-3)))
    out["zouhe_pressure"] = Spec("zouhe_pressure", nx, ny, 0.7, m,
                                 (G.INLET_ZOUHE, G.OUTLET_PRESSURE, G.WALL, G.FREESLIP), u_in=(0.03, 0.0),
                                 rho_out=0.999, ux0=np.where(m.ravel() > 0, 0.0, 0.03))
    return out
