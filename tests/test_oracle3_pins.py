"""Pins for the D3Q19 oracle (the 3-D extension of the method).

The strongest pin is a projection: summing the D3Q19 populations of a lattice
that is invariant along one axis over the velocity component of that axis
gives D2Q9 populations with the D2Q9 weights, and the BGK update with Guo
forcing and bounce-back commutes with that sum. So a y-invariant (or
z-invariant) D3Q19 run must reproduce the D2Q9 oracle, which is itself
pinned by exact-rational brute force."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2607_20650_gb300 import geometry as G

C3, W3 = O.directions3()


def test_direction_set():
    assert C3.shape == (19, 3)
    assert (C3[::-1] == -C3).all()                      # opposite(i) = 18 - i
    assert (C3[9] == 0).all() and W3[9] == pytest.approx(1 / 3)
    assert abs(W3.sum() - 1) < 1e-15
    q = (C3 ** 2).sum(axis=1)
    assert set(q) == {0, 1, 2}
    assert np.allclose(W3[q == 1], 1 / 18) and np.allclose(W3[q == 2], 1 / 36)


@pytest.mark.parametrize("drho,u", [(0.0, (0.0, 0.0, 0.0)), (0.02, (0.05, -0.03, 0.01)),
                                    (-0.1, (-0.1, 0.2, -0.05))])
def test_equilibrium_moments_3d(drho, u):
    h = O.equilibrium3(drho, *u)
    f = h + W3
    rho = 1 + drho
    tol = 5e-16 * (1 + abs(rho))
    assert abs(f.sum() - rho) < tol
    for a in range(3):
        assert abs((f * C3[:, a]).sum() - u[a]) < tol
        for b in range(3):
            exp = rho / 3 * (a == b) + u[a] * u[b]
            assert abs((f * C3[:, a] * C3[:, b]).sum() - exp) < tol


def test_pure_streaming_3d_is_exact_shift():
    nx, ny, nz, T = 6, 5, 4, 3
    rng = np.random.default_rng(1)
    h0 = rng.normal(0, 0.01, size=(19, nx * ny * nz))
    lat = O.Lattice3(O.Case3(nx, ny, nz, math.inf))
    lat.set_h(h0)
    lat.run(T)
    for i in range(19):
        exp = np.roll(h0[i].reshape(nz, ny, nx), (T * C3[i, 2], T * C3[i, 1], T * C3[i, 0]), axis=(0, 1, 2))
        assert np.array_equal(lat.h[i].reshape(nz, ny, nx), exp)


def test_mass_conserved_3d():
    nx, ny, nz = 10, 9, 8
    rng = np.random.default_rng(2)
    mask = (rng.random(nx * ny * nz) < 0.2).astype(np.uint8)
    lat = O.Lattice3(O.Case3(nx, ny, nz, 0.8, fx=1e-4, fz=-2e-5), mask,
                     rho=1 + 1e-2 * rng.random(nx * ny * nz), ux=1e-2 * rng.random(nx * ny * nz))
    m0 = lat.mass()
    lat.run(40)
    assert abs(lat.mass() - m0) / m0 < 1e-14


def test_mass_value_is_sum_of_rho_3d():
    """sum_i f_i^eq = rho (Eq. 2 in 3-D), so after initialisation from a given
    density field the mass is that field summed over the fluid nodes, and
    the rest state gives the fluid-node count. The fluid set is known by
    construction: a solid 3x3x3 cube with a one-node hole at its centre
    (the hole has no open pull, so it counts as solid) and a solid slab.
    Dropping the rest weight or counting solid nodes fails."""
    nx, ny, nz = 9, 8, 7
    m = np.zeros((nz, ny, nx), np.uint8)
    m[1:4, 1:4, 1:4] = 1
    m[2, 2, 2] = 0
    m[5, :, 6:8] = 1
    fluid = m == 0
    fluid[2, 2, 2] = False
    case = O.Case3(nx, ny, nz, 0.7, bc_z=O.WALL)
    assert O.Lattice3(case, m).mass() == float(fluid.sum())
    rng = np.random.default_rng(5)
    N = nx * ny * nz
    rho = 1.0 + 0.05 * (rng.random(N) - 0.5)
    u = [0.06 * (rng.random(N) - 0.5) for _ in range(3)]
    lat = O.Lattice3(case, m, rho=rho, ux=u[0], uy=u[1], uz=u[2])
    exp = math.fsum(rho[fluid.ravel()])
    assert abs(lat.mass() - exp) <= 4e-16 * exp
    h = lat.h.copy()
    h[:, ~fluid.ravel()] = rng.normal(0, 0.3, size=(19, int((~fluid).sum())))
    lat.set_h(h)
    assert abs(lat.mass() - exp) <= 4e-16 * exp


def _project(h3, nx, ny, nz, axis):
    """Sum D3Q19 populations over the velocity component along `axis` of a
    lattice invariant along that axis; returns D2Q9 h on the other two axes."""
    keep = [a for a in range(3) if a != axis]                  # (first, second) -> (x2, y2)
    h3 = h3.reshape(19, nz, ny, nx)
    slab = h3.take(0, axis=3 - axis)                            # one layer along the axis
    out = np.zeros((9,) + slab.shape[1:])
    for i in range(19):
        c2x, c2y = C3[i, keep[0]], C3[i, keep[1]]
        out[(c2x + 1) + 3 * (c2y + 1)] += slab[i]
    return out                                                  # 2-D arrays indexed [y2][x2]


@pytest.mark.parametrize("axis", [1, 2])
def test_invariant_axis_reduces_to_d2q9(axis):
    n1, n2 = 14, 9                       # the two kept axes
    rng = np.random.default_rng(axis)
    mask2 = (rng.random((n2, n1)) < 0.15).astype(np.uint8)
    rho2 = 1 + 1e-2 * rng.random((n2, n1))
    u2 = 1e-2 * rng.random((2, n2, n1))
    bc2 = O.WALL
    if axis == 2:                        # z-invariant: kept (x, y)
        nx, ny, nz = n1, n2, 2
        tile = lambda a: np.broadcast_to(a, (nz, ny, nx))
        case3 = O.Case3(nx, ny, nz, 0.7, fx=2e-4, fy=-1e-4, bc_x=O.PERIODIC, bc_y=bc2)
        uu = dict(ux=tile(u2[0]).ravel(), uy=tile(u2[1]).ravel())
    else:                                # y-invariant: kept (x, z)
        nx, ny, nz = n1, 3, n2
        tile = lambda a: np.broadcast_to(a[:, None, :], (nz, ny, nx))
        case3 = O.Case3(nx, ny, nz, 0.7, fx=2e-4, fz=-1e-4, bc_x=O.PERIODIC, bc_z=bc2)
        uu = dict(ux=tile(u2[0]).ravel(), uz=tile(u2[1]).ravel())
    lat3 = O.Lattice3(case3, tile(mask2).ravel(), rho=tile(rho2).ravel(), **uu).run(25)
    case2 = O.Case(n1, n2, 0.7, fx=2e-4, fy=-1e-4, bc_s=bc2, bc_n=bc2)
    lat2 = O.Lattice(case2, mask2, rho=rho2, ux=u2[0], uy=u2[1]).run(25)
    proj = _project(lat3.h, nx, ny, nz, axis).reshape(9, -1)
    np.testing.assert_allclose(proj, lat2.h, rtol=0, atol=5e-16)


def test_plane_poiseuille_3d_slip_closed_form():
    """Walls on the z faces, force along x: the steady profile is the
    parabola plus the BGK bounce-back slip g (16 L - 3) / (24 nu)."""
    H, tau, g = 8, 0.8, 1e-6
    nu = (tau - 0.5) / 3
    lat = O.Lattice3(O.Case3(2, 2, H, tau, fx=g, bc_z=O.WALL)).run(int(60 * H * H / nu))
    ux = lat.ux.reshape(H, 2, 2)[:, 0, 0]
    z = np.arange(H) + 0.5
    par = g / (2 * nu) * z * (H - z)
    slip = g * (16 * (tau - 0.5) ** 2 - 3) / (24 * nu)
    assert np.max(np.abs(ux - par - slip)) / par.max() < 1e-10


def test_force_balance_steady_duct_3d():
    """Momentum exchange (3-D): at steady state the force on the walls (rows
    of solid nodes on the z faces, everything periodic) equals the body force
    on the fluid, g * (number of fluid nodes), per update, split equally
    between the two walls by symmetry; the transverse components vanish."""
    H, n, g = 8, 3, 1e-5
    tau = 0.5 + math.sqrt(3.0) / 4.0
    nu = (tau - 0.5) / 3
    mask = np.zeros((H + 2, n, n), np.uint8)
    mask[0] = 1
    mask[-1] = 1
    lat = O.Lattice3(O.Case3(n, n, H + 2, tau, fx=g), mask).run(int(40 * H * H / nu))
    F = lat.force(mask)
    total = g * n * n * H
    assert abs(F[0] - total) / total < 1e-9
    assert abs(F[1]) < 1e-15 and abs(F[2]) < 1e-12
    bottom = np.zeros_like(mask)
    bottom[0] = 1
    Fb = lat.force(bottom)
    assert abs(Fb[0] - total / 2) / total < 1e-9
    assert np.all(lat.force(np.zeros_like(mask)) == 0.0)


# ---------------------------------------------------------------- inlet / outflow

def test_uniform_inflow_outflow_is_a_fixed_point_3d():
    """Equilibrium inlet (west) at U and zero-gradient outflow (east) with
    periodic y and z: the uniform state f^eq(1, U) is stationary."""
    U = (0.04, 0.01, -0.005)
    nx, ny, nz = 7, 4, 3
    N = nx * ny * nz
    case = O.Case3(nx, ny, nz, 0.8, bc_x=O.INLET_EQ, bc_xe=O.OUTFLOW_ZG, u_in=U)
    lat = O.Lattice3(case, None, ux=np.full(N, U[0]), uy=np.full(N, U[1]), uz=np.full(N, U[2]))
    h0 = lat.h.copy()
    lat.run(50)
    assert np.max(np.abs(lat.h - h0)) < 1e-16
    assert np.max(np.abs(lat.ux - U[0])) < 1e-16 and np.max(np.abs(lat.uz - U[2])) < 1e-16


def test_inlet_outflow_channel_reduces_to_d2q9():
    """A z-invariant channel with an obstacle, equilibrium inlet, zero-gradient
    outflow and walls on y, summed over c_z, is the 2-D oracle's channel with
    the same edges (the 2-D oracle is pinned by exact-rational brute force)."""
    nx, ny, nz = 16, 9, 3
    rng = np.random.default_rng(5)
    mask2 = np.zeros((ny, nx), np.uint8)
    mask2[3:6, 5:7] = 1
    u2 = np.where(mask2 > 0, 0.0, 0.03 + 5e-3 * rng.random((ny, nx)))
    v2 = np.where(mask2 > 0, 0.0, 5e-3 * rng.random((ny, nx)))
    tile = lambda a: np.broadcast_to(a, (nz, ny, nx))
    case3 = O.Case3(nx, ny, nz, 0.7, bc_x=O.INLET_EQ, bc_xe=O.OUTFLOW_ZG, bc_y=O.WALL, u_in=(0.03, 0.0, 0.0))
    lat3 = O.Lattice3(case3, tile(mask2).ravel(), ux=tile(u2).ravel(), uy=tile(v2).ravel()).run(30)
    case2 = O.Case(nx, ny, 0.7, ux_in=0.03, bc_w=O.INLET_EQ, bc_e=O.OUTFLOW_ZG, bc_s=O.WALL, bc_n=O.WALL)
    lat2 = O.Lattice(case2, mask2, ux=u2, uy=v2).run(30)
    proj = _project(lat3.h, nx, ny, nz, 2).reshape(9, -1)
    np.testing.assert_allclose(proj, lat2.h, rtol=0, atol=5e-16)


# ---------------------------------------------------------------- Zou-He faces

@pytest.mark.parametrize("axis", [1, 2])
def test_zou_he_channel_reduces_to_d2q9(axis):
    """Zou-He velocity inlet (west) and pressure outlet (east) with walls on
    the kept transverse axis and an obstacle: a lattice invariant along y
    (axis 1, inlet velocity with a z component) or z (axis 2, with a y
    component), summed over that velocity component, is the 2-D oracle's
    channel with the same edges, whose inlet and outlet are pinned by their
    defining conditions and by exact-rational brute force."""
    n1, n2, m = 18, 9, 3
    rng = np.random.default_rng(7 + axis)
    mask2 = np.zeros((n2, n1), np.uint8)
    mask2[3:6, 6:8] = 1
    u2 = np.where(mask2 > 0, 0.0, 0.03 + 5e-3 * rng.random((n2, n1)))
    v2 = np.where(mask2 > 0, 0.0, 5e-3 * (rng.random((n2, n1)) - 0.5))
    rho2 = 1.0 + 1e-3 * rng.random((n2, n1))
    U, Ut, rho_out = 0.035, 0.004, 0.9985
    if axis == 2:
        nx, ny, nz = n1, n2, m
        tile = lambda a: np.broadcast_to(a, (nz, ny, nx))
        case3 = O.Case3(nx, ny, nz, 0.7, bc_x=O.INLET_ZOUHE, bc_xe=O.OUTLET_PRESSURE, bc_y=O.WALL,
                        u_in=(U, Ut, 0.0), rho_out=rho_out)
        uu = dict(ux=tile(u2).ravel(), uy=tile(v2).ravel())
    else:
        nx, ny, nz = n1, m, n2
        tile = lambda a: np.broadcast_to(a[:, None, :], (nz, ny, nx))
        case3 = O.Case3(nx, ny, nz, 0.7, bc_x=O.INLET_ZOUHE, bc_xe=O.OUTLET_PRESSURE, bc_z=O.WALL,
                        u_in=(U, 0.0, Ut), rho_out=rho_out)
        uu = dict(ux=tile(u2).ravel(), uz=tile(v2).ravel())
    lat3 = O.Lattice3(case3, tile(mask2).ravel(), rho=tile(rho2).ravel(), **uu).run(30)
    case2 = O.Case(n1, n2, 0.7, ux_in=U, uy_in=Ut, bc_w=O.INLET_ZOUHE, bc_e=O.OUTLET_PRESSURE, bc_s=O.WALL,
                   bc_n=O.WALL, rho_out=rho_out)
    lat2 = O.Lattice(case2, mask2, rho=rho2, ux=u2, uy=v2).run(30)
    proj = _project(lat3.h, nx, ny, nz, axis).reshape(9, -1)
    np.testing.assert_allclose(proj, lat2.h, rtol=0, atol=5e-16)


def test_zou_he_faces_fix_their_moments_3d():
    """The defining conditions, on a fully 3-D state (no invariant axis):
    every inlet node's velocity after the update is U (sum_i g_i c_i = U, no
    force), every outlet node's density is rho_out and its transverse
    velocity is zero."""
    nx, ny, nz = 9, 6, 5
    N = nx * ny * nz
    rng = np.random.default_rng(11)
    U, rho_out = (0.03, -0.006, 0.004), 1.002
    case = O.Case3(nx, ny, nz, 0.65, bc_x=O.INLET_ZOUHE, bc_xe=O.OUTLET_PRESSURE, bc_y=O.WALL,
                   u_in=U, rho_out=rho_out)
    lat = O.Lattice3(case, None, rho=1 + 2e-3 * rng.random(N), ux=0.03 + 1e-2 * rng.random(N),
                     uy=1e-2 * (rng.random(N) - 0.5), uz=1e-2 * (rng.random(N) - 0.5)).run(3)
    x = np.arange(N) % nx
    inl, out = x == 0, x == nx - 1
    for comp, u in zip((lat.ux, lat.uy, lat.uz), U):
        assert np.max(np.abs(comp[inl] - u)) < 1e-16
    assert np.max(np.abs(lat.rho[out] - rho_out)) < 4e-16
    assert np.max(np.abs(lat.uy[out])) < 1e-16 and np.max(np.abs(lat.uz[out])) < 1e-16
