"""Exact-rational brute force of the D2Q9I BGK update, for tiny grids.

A second, independent statement of the same method, used only to pin the
FP64 oracle: it keeps the plain populations f (not deviations), uses Python
``Fraction`` arithmetic (no rounding at all), stores nodes in a dict, and
obtains the Zou-He unknowns by solving their three defining conditions
(prescribed momentum in x and y, bounce-back of the non-equilibrium part of
the normal population) instead of using closed formulas.

Method: PortLBM Sec. 3.1, Eq. (1) (BGK), Eq. (2) (D2Q9I equilibrium,
v = sum f c), directions of Fig. 2 (c_i = (i%3-1, i//3-1)), half-way
bounce-back; Guo body force with v = sum f c + F/2.
"""
from fractions import Fraction as Fr

W = [Fr(1, 36), Fr(1, 9), Fr(1, 36), Fr(1, 9), Fr(4, 9), Fr(1, 9), Fr(1, 36), Fr(1, 9), Fr(1, 36)]
C = [(i % 3 - 1, i // 3 - 1) for i in range(9)]
PERIODIC, WALL, FREESLIP, INLET_ZOUHE, INLET_EQ, OUTFLOW_ZG, INLET_EQ_NEUMANN, OUTLET_PRESSURE = range(8)


def feq(rho, ux, uy):
    out = []
    for (cx, cy), w in zip(C, W):
        cu = cx * ux + cy * uy
        out.append(w * (rho + 3 * cu + Fr(9, 2) * cu * cu - Fr(3, 2) * (ux * ux + uy * uy)))
    return out


def index_of(cx, cy):
    return (cx + 1) + 3 * (cy + 1)


class RationalLBM:
    def __init__(self, nx, ny, tau, solid, bc, force=(0, 0), u_in=(0, 0), rho0=None, u0=None, rho_out=1):
        self.nx, self.ny = nx, ny
        self.omega = 1 / Fr(tau)
        self.solid = solid  # set of (x, y)
        self.bc = bc        # dict: 'w','e','s','n' -> code
        self.F = (Fr(force[0]), Fr(force[1]))
        self.U = (Fr(u_in[0]), Fr(u_in[1]))
        self.rho_out = Fr(rho_out)
        self.f = {}
        for y in range(ny):
            for x in range(nx):
                if (x, y) in solid:
                    self.f[(x, y)] = list(W)
                else:
                    r = Fr(1) if rho0 is None else Fr(rho0[(x, y)])
                    ux, uy = (Fr(0), Fr(0)) if u0 is None else (Fr(u0[(x, y)][0]), Fr(u0[(x, y)][1]))
                    self.f[(x, y)] = feq(r, ux, uy)
        self.moments = {}

    def incoming(self, x, y, i):
        """Value reaching (x, y) in direction i, or None if it must come from the inlet."""
        cx, cy = C[i]
        sx, sy, d = x - cx, y - cy, i
        if not 0 <= sy < self.ny:
            kind = self.bc['s'] if sy < 0 else self.bc['n']
            if kind == PERIODIC:
                sy %= self.ny
            elif kind == FREESLIP:
                # specular reflection: it left (x - cx, y) moving with (cx, -cy)
                sy, d = y, index_of(cx, -cy)
            else:
                return self.f[(x, y)][index_of(-cx, -cy)]
        if not 0 <= sx < self.nx:
            kind = self.bc['w'] if sx < 0 else self.bc['e']
            if kind == PERIODIC:
                sx %= self.nx
            elif kind == OUTFLOW_ZG:
                sx = min(max(sx, 0), self.nx - 1)
            elif kind in (INLET_ZOUHE, INLET_EQ, INLET_EQ_NEUMANN, OUTLET_PRESSURE):
                return None
            else:
                return self.f[(x, y)][index_of(-cx, -cy)]
        if (sx, sy) in self.solid:
            return self.f[(x, y)][index_of(-cx, -cy)]
        return self.f[(sx, sy)][d]

    def step(self):
        new = {}
        Fx, Fy = self.F
        om = self.omega
        for (x, y), fl in self.f.items():
            if (x, y) in self.solid:
                new[(x, y)] = fl
                continue
            g = [self.incoming(x, y, i) for i in range(9)]
            if x == 0 and self.bc['w'] == INLET_ZOUHE:
                Ux, Uy = self.U
                # unknowns a=g2, b=g5, c=g8 from:  b - b_eq = g3 - g3_eq (rho cancels),
                # sum g cx = Ux, sum g cy = Uy.
                b = g[3] + (W[5] * 3 * Ux - W[3] * 3 * (-Ux))
                # a + c = Ux + g0 + g3 + g6 - b ;  c - a = Uy + g0 + g1 - g6 - g7
                s = Ux + g[0] + g[3] + g[6] - b
                dlt = Uy + g[0] + g[1] - g[6] - g[7]
                g[2], g[5], g[8] = (s - dlt) / 2, b, (s + dlt) / 2
            elif x == 0 and self.bc['w'] == INLET_EQ:
                g = feq(Fr(1), *self.U)
            elif x == 0 and self.bc['w'] == INLET_EQ_NEUMANN:
                # density of the east neighbour in the previous state
                r_in = Fr(1) if (1, y) in self.solid else sum(self.f[(1, y)])
                g = feq(r_in, *self.U)
            if x == self.nx - 1 and self.bc['e'] == OUTLET_PRESSURE:
                # unknowns a=g0, b=g3, c=g6 from: sum g = rho_out, sum g c_y = 0,
                # b - b_eq = g5 - g5_eq (rho cancels; the equilibria differ by
                # w 6 u_x with u_x = sum g c_x).
                K = g[1] + g[2] + g[4] + g[5] + g[7] + g[8]
                ux = (g[2] + g[5] + g[8]) - (self.rho_out - K)
                b = g[5] - (W[5] * 3 * ux - W[3] * 3 * (-ux))
                s_ac = self.rho_out - K - b
                d_ca = g[1] + g[2] - g[7] - g[8]
                g[0], g[3], g[6] = (s_ac - d_ca) / 2, b, (s_ac + d_ca) / 2
            rho = sum(g)
            ux = sum(gi * c[0] for gi, c in zip(g, C)) + Fx / 2
            uy = sum(gi * c[1] for gi, c in zip(g, C)) + Fy / 2
            eq = feq(rho, ux, uy)
            out = []
            for i, ((cx, cy), w) in enumerate(zip(C, W)):
                cu = cx * ux + cy * uy
                src = (1 - om / 2) * w * ((3 * (cx - ux) + 9 * cu * cx) * Fx
                                          + (3 * (cy - uy) + 9 * cu * cy) * Fy)
                out.append(g[i] - om * (g[i] - eq[i]) + src)
            new[(x, y)] = out
            self.moments[(x, y)] = (rho, ux, uy)
        self.f = new

    def deviations(self):
        """9 x N array-like (lists) of f_i - w_i in canonical order n = y*nx + x."""
        N = self.nx * self.ny
        out = [[0.0] * N for _ in range(9)]
        for (x, y), fl in self.f.items():
            n = y * self.nx + x
            for i in range(9):
                out[i][n] = 0.0 if (x, y) in self.solid else float(fl[i] - W[i])
        return out
