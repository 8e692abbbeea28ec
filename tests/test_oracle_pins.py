"""Pins for the FP64 CPU oracle, against facts that do not come from the oracle.

Each test names what fixes the expected value: an identity of Eq. (2), a
closed-form solution, an exact invariant, or an exact-rational brute force.
Together they make a dropped term, a wrong sign, weight, index or mirror in
``oracle/lbm_oracle.c`` fail at least one test.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2607_20650_gb300 import geometry as G
from tests.rational_lbm import RationalLBM, W as WR

CX, CY = O.CX, O.CY
W = np.array([float(w) for w in WR])


# ---------------------------------------------------------------- Eq. (2)

@pytest.mark.parametrize("drho,ux,uy", [(0.0, 0.0, 0.0), (0.013, 0.05, -0.02),
                                        (-0.2, -0.11, 0.07), (0.5, 0.3, 0.3)])
def test_equilibrium_moments(drho, ux, uy):
    """D2Q9I moments of Eq. (2): sum f = rho, sum f c = v, sum f c c = rho/3 I + v v."""
    h = O.equilibrium(drho, ux, uy)
    f = h + W
    rho = 1.0 + drho
    tol = 4e-16 * (1 + abs(rho))
    assert abs(f.sum() - rho) < tol
    assert abs(h.sum() - drho) < tol
    assert abs((f * CX).sum() - ux) < tol
    assert abs((f * CY).sum() - uy) < tol
    assert abs((f * CX * CX).sum() - (rho / 3 + ux * ux)) < tol
    assert abs((f * CY * CY).sum() - (rho / 3 + uy * uy)) < tol
    assert abs((f * CX * CY).sum() - ux * uy) < tol


def test_weights_and_directions():
    """Fig. 2 order: opposite(i) = 8 - i, rest at 4, weights of Eq. (2)."""
    assert (CX[::-1] == -CX).all() and (CY[::-1] == -CY).all()
    assert CX[4] == 0 and CY[4] == 0
    np.testing.assert_allclose(O.equilibrium(0.0, 0.0, 0.0), 0.0, atol=0)


# ---------------------------------------------------------------- streaming

def test_pure_streaming_is_exact_shift():
    """omega = 0 (tau = inf), F = 0, periodic: S_T is S_0 shifted by T c_i, bit for bit."""
    nx, ny, T = 13, 7, 5
    case = O.Case(nx, ny, math.inf)
    lat = O.Lattice(case)
    rng = np.random.default_rng(1)
    h0 = rng.normal(0, 0.01, size=(9, nx * ny))
    lat.set_h(h0)
    lat.run(T)
    for i in range(9):
        exp = np.roll(h0[i].reshape(ny, nx), shift=(T * CY[i], T * CX[i]), axis=(0, 1))
        assert np.array_equal(lat.h[i].reshape(ny, nx), exp), i


def test_periodic_shift_equivariance():
    """Shifting mask and state on a periodic lattice shifts the result exactly."""
    nx, ny = 12, 9
    rng = np.random.default_rng(2)
    mask = (rng.random((ny, nx)) < 0.2).astype(np.uint8)
    case = O.Case(nx, ny, 0.7, fx=1e-4, fy=-3e-5)
    a = O.Lattice(case, mask)
    h0 = rng.normal(0, 0.01, size=(9, nx * ny)) * (1 - a.solid)
    a.set_h(h0)
    a.run(4)
    dx, dy = 5, 3
    ms = np.roll(mask, (dy, dx), axis=(0, 1))
    b = O.Lattice(case, ms)
    b.set_h(np.stack([np.roll(h0[i].reshape(ny, nx), (dy, dx), axis=(0, 1)).ravel()
                      for i in range(9)]))
    b.run(4)
    for i in range(9):
        exp = np.roll(a.h[i].reshape(ny, nx), (dy, dx), axis=(0, 1))
        assert np.array_equal(b.h[i].reshape(ny, nx), exp)


# ---------------------------------------------------------------- invariants

def test_mass_conserved_porous_periodic():
    """Bounce-back + periodic + Guo force conserve mass exactly in exact arithmetic."""
    nx, ny = 64, 48
    mask = G.porous_discs(nx, ny, seed=11, rmin=3, rmax=6, solid_fraction=0.3)
    lat = O.Lattice(O.Case(nx, ny, 0.9, fx=1e-5), mask,
                    rho=1 + 0.01 * np.random.default_rng(3).random(nx * ny))
    m0 = lat.mass()
    lat.run(300)
    assert abs(lat.mass() - m0) / m0 < 1e-14


def _pocket_mask(nx, ny):
    """Mask with two solid blocks and one enclosed single-node fluid pocket.
    Returns the mask and the fluid set known by construction: every mask-0
    node except the pocket node (all eight neighbours solid: no open pull)."""
    m = np.zeros((ny, nx), np.uint8)
    m[2:5, 3:6] = 1          # 3x3 block with a hole in the middle ...
    m[3, 4] = 0              # ... the enclosed pocket
    m[6:8, 9:12] = 1         # a plain 2x3 block
    fluid = (m == 0)
    fluid[3, 4] = False
    return m, fluid


@pytest.mark.parametrize("edges", ["periodic", "walls"])
def test_mass_value_is_sum_of_rho(edges):
    """Eq. (2) gives sum_i f_i^eq = rho, so right after initialisation from a
    given density field (any velocity) the total mass is sum of that field
    over the fluid nodes; the rest state gives the fluid-node count. The
    expected values use the inputs and the hand-known fluid set only.
    Dropping the rest weight (rho = sum h) gives ~0.1 instead of ~100;
    counting solid or pocket nodes adds >= 1 per node."""
    nx, ny = 14, 10
    mask, fluid = _pocket_mask(nx, ny)
    kw = dict(bc_s=O.WALL, bc_n=O.WALL) if edges == "walls" else {}
    case = O.Case(nx, ny, 0.8, **kw)
    rest = O.Lattice(case, mask)
    assert rest.mass() == float(fluid.sum())
    rng = np.random.default_rng(21)
    rho = 1.0 + 0.05 * (rng.random(nx * ny) - 0.5)
    ux = 0.08 * (rng.random(nx * ny) - 0.5)
    uy = 0.08 * (rng.random(nx * ny) - 0.5)
    lat = O.Lattice(case, mask, rho=rho, ux=ux, uy=uy)
    exp = math.fsum(rho[fluid.ravel()])
    assert abs(lat.mass() - exp) <= 4e-16 * exp
    # Values written into solid and pocket nodes are not mass.
    h = lat.h.copy()
    h[:, ~fluid.ravel()] = rng.normal(0, 0.3, size=(9, int((~fluid).sum())))
    lat.set_h(h)
    assert abs(lat.mass() - exp) <= 4e-16 * exp


def test_isolated_fluid_node_is_solid():
    nx, ny = 7, 7
    mask = np.ones((ny, nx), np.uint8)
    mask[3, 3] = 0          # isolated: all eight neighbours solid
    mask[1, 1:3] = 0        # a pair: each has one fluid neighbour
    s = O.effective_solid(O.Case(nx, ny, 0.8), mask).reshape(ny, nx)
    assert s[3, 3] == 1 and s[1, 1] == 0 and s[1, 2] == 0


def test_wall_edge_equals_solid_rows():
    """A half-way wall edge is the same boundary as a row of solid nodes."""
    nx, ny = 10, 6
    rng = np.random.default_rng(4)
    h0 = rng.normal(0, 0.01, size=(9, nx, ny))
    a = O.Lattice(O.Case(nx, ny, 0.75, fx=2e-5, bc_s=O.WALL, bc_n=O.WALL))
    a.set_h(h0.transpose(0, 2, 1).reshape(9, -1))
    a.run(6)
    m = np.zeros((ny + 2, nx), np.uint8)
    m[0] = 1
    m[-1] = 1
    b = O.Lattice(O.Case(nx, ny + 2, 0.75, fx=2e-5), m)
    hb = np.zeros((9, ny + 2, nx))
    hb[:, 1:-1, :] = h0.transpose(0, 2, 1)
    b.set_h(hb.reshape(9, -1))
    b.run(6)
    assert np.array_equal(b.h.reshape(9, ny + 2, nx)[:, 1:-1, :], a.h.reshape(9, ny, nx))


def test_mirror_symmetry_freeslip():
    """A y-symmetric free-slip channel stays mirror-symmetric: h_i(x, y) = h_{m(i)}(x, ny-1-y)."""
    nx, ny = 20, 10
    mask = np.zeros((ny, nx), np.uint8)
    mask[3:7, 6:9] = 1
    case = O.Case(nx, ny, 0.6, ux_in=0.04, bc_w=O.INLET_ZOUHE, bc_e=O.OUTFLOW_ZG,
                  bc_s=O.FREESLIP, bc_n=O.FREESLIP)
    lat = O.Lattice(case, mask, ux=np.full(nx * ny, 0.04))
    lat.run(40)
    h = lat.h.reshape(9, ny, nx)
    mir = [(i % 3) + 3 * (2 - i // 3) for i in range(9)]
    np.testing.assert_allclose(h[mir][:, ::-1, :], h, rtol=0, atol=1e-15)


# ---------------------------------------------------------------- closed forms

def _poiseuille(tau, H, steps, nx=2, g=1e-6):
    ny = H + 2
    lat = O.Lattice(O.Case(nx, ny, tau, fx=g), G.channel_walls(nx, ny)).run(steps)
    ux = lat.field(lat.ux)[1:-1, 0]
    nu = (tau - 0.5) / 3
    y = np.arange(1, ny - 1) - 0.5          # distance from the half-way wall at y = 1/2
    return ux, g / (2 * nu) * y * (H - y), nu, lat


def test_poiseuille_magic_tau_exact():
    """For BGK with half-way bounce-back, (tau-1/2)^2 = 3/16 places the wall exactly:
    the steady discrete profile is the Navier-Stokes parabola to round-off."""
    tau = 0.5 + math.sqrt(3.0) / 4.0
    ux, ua, _, _ = _poiseuille(tau, 16, 40000)
    assert np.max(np.abs(ux - ua)) / ua.max() < 1e-11


@pytest.mark.parametrize("tau", [0.6, 0.8, 1.0, 1.4])
def test_poiseuille_slip_closed_form(tau):
    """Steady BGK Poiseuille with half-way bounce-back is the parabola plus a
    uniform slip g (16 L - 3) / (24 nu), L = (tau - 1/2)^2 (Ginzburg's magic
    parameter analysis of BGK/TRT bounce-back)."""
    H = 8
    nu = (tau - 0.5) / 3
    steps = int(60 * H * H / nu)
    ux, ua, nu, _ = _poiseuille(tau, H, steps)
    lam = (tau - 0.5) ** 2
    slip = 1e-6 * (16 * lam - 3) / (24 * nu)
    assert np.max(np.abs(ux - ua - slip)) / ua.max() < 1e-10


def startup_series(y, t, H, nu, g, terms=400):
    """Start-up of plane Poiseuille flow from rest (separation of variables)."""
    umax = g * H * H / (8 * nu)
    u = g / (2 * nu) * y * (H - y)
    for k in range(terms):
        n = 2 * k + 1
        u = u - 32 * umax / (n * math.pi) ** 3 * np.sin(n * math.pi * y / H) * \
            math.exp(-(n * math.pi) ** 2 * nu * t / H ** 2)
    return u


def test_poiseuille_256x64_startup_and_mass():
    """The 256x64, tau = 0.8, g = 1e-6 channel after 20,000 updates: relative
    L-inf error against the closed-form start-up series <= 1e-3 (the steady
    parabola is not yet reached at H^2/nu = 38,440), and mass drift <= 1e-12."""
    w = G.poiseuille()
    lat = O.Lattice(O.Case(w.nx, w.ny, w.tau, fx=w.fx), w.mask)
    m0 = lat.mass()
    lat.run(20000)
    H, nu = w.ny - 2, (w.tau - 0.5) / 3
    ux = lat.field(lat.ux)[1:-1, :]
    assert np.ptp(ux, axis=1).max() == 0.0          # invariant in x
    y = np.arange(1, w.ny - 1) - 0.5
    ua = startup_series(y, 20000 - 0.5, H, nu, w.fx)
    err = np.max(np.abs(ux[:, 0] - ua)) / np.max(np.abs(ua))
    assert err < 1e-3
    assert err > 1e-5                                # the BGK wall slip is visible
    assert abs(lat.mass() - m0) / m0 <= 1e-12


def test_freeslip_plug_flow_accelerates_uniformly():
    """Free-slip walls carry no shear: a forced channel stays a plug, and with
    Guo forcing the update-k velocity is exactly (k - 1/2) g."""
    nx, ny, g = 6, 5, 1e-4
    lat = O.Lattice(O.Case(nx, ny, 0.7, fx=g, bc_s=O.FREESLIP, bc_n=O.FREESLIP))
    for k in (1, 7, 30):
        lat.run(k - lat.steps)
        np.testing.assert_allclose(lat.ux, (k - 0.5) * g, rtol=1e-13, atol=0)
        np.testing.assert_allclose(lat.uy, 0.0, atol=1e-18)


def test_zou_he_prescribes_inlet_velocity():
    """After Zou-He reconstruction sum_i g_i c_i = U exactly (F = 0)."""
    nx, ny = 8, 6
    rng = np.random.default_rng(5)
    case = O.Case(nx, ny, 0.8, ux_in=0.07, uy_in=-0.01, bc_w=O.INLET_ZOUHE,
                  bc_e=O.OUTFLOW_ZG, bc_s=O.WALL, bc_n=O.WALL)
    lat = O.Lattice(case, ux=0.05 + 0.01 * rng.random(nx * ny), uy=0.01 * rng.random(nx * ny))
    lat.run(3)
    col = lambda a: lat.field(a)[:, 0]
    np.testing.assert_allclose(col(lat.ux), 0.07, rtol=0, atol=2e-17)
    np.testing.assert_allclose(col(lat.uy), -0.01, rtol=0, atol=2e-17)


def test_uniform_inflow_outflow_fixed_point():
    """Uniform equilibrium at the inlet velocity is a fixed point of the
    Zou-He inlet + zero-gradient outflow + free-slip channel."""
    nx, ny, U = 16, 6, 0.05
    case = O.Case(nx, ny, 0.6, ux_in=U, bc_w=O.INLET_ZOUHE, bc_e=O.OUTFLOW_ZG,
                  bc_s=O.FREESLIP, bc_n=O.FREESLIP)
    lat = O.Lattice(case, ux=np.full(nx * ny, U))
    lat.run(50)
    heq = O.equilibrium(0.0, U, 0.0)
    np.testing.assert_allclose(lat.h, np.repeat(heq[:, None], nx * ny, 1), rtol=0, atol=5e-16)
    np.testing.assert_allclose(lat.ux, U, rtol=0, atol=5e-16)


def test_force_balance_steady_poiseuille():
    """At steady state the momentum exchanged with the walls equals the body
    force on the fluid, g * (number of fluid nodes), per update."""
    tau = 0.5 + math.sqrt(3.0) / 4.0
    H, nx = 8, 4
    _, _, _, lat = _poiseuille(tau, H, 20000, nx=nx, g=1e-5)
    body = G.channel_walls(nx, H + 2)
    F = lat.force(body)
    assert abs(F[0] - 1e-5 * nx * H) / (1e-5 * nx * H) < 1e-9
    assert abs(F[1]) < 1e-15


# ---------------------------------------------------------------- brute force

def _compare_rational(nx, ny, tau, solid, bc, force=(0, 0), u_in=(0, 0), u0=None, steps=3, rho_out=1):
    from fractions import Fraction as Fr
    r = RationalLBM(nx, ny, Fr(tau), solid, bc, force=force, u_in=u_in, u0=u0, rho_out=rho_out)
    mask = np.zeros((ny, nx), np.uint8)
    for (x, y) in solid:
        mask[y, x] = 1
    case = O.Case(nx, ny, float(Fr(tau)), fx=float(force[0]), fy=float(force[1]),
                  ux_in=float(u_in[0]), uy_in=float(u_in[1]),
                  bc_w=bc['w'], bc_e=bc['e'], bc_s=bc['s'], bc_n=bc['n'], rho_out=float(Fr(rho_out)))
    ux0 = uy0 = None
    if u0 is not None:
        ux0 = np.array([float(u0[(n % nx, n // nx)][0]) for n in range(nx * ny)])
        uy0 = np.array([float(u0[(n % nx, n // nx)][1]) for n in range(nx * ny)])
    lat = O.Lattice(case, mask, ux=ux0, uy=uy0)
    for s in range(steps):
        r.step()
        lat.run(1)
        np.testing.assert_allclose(lat.h, np.array(r.deviations()), rtol=0, atol=2e-16)
        for (x, y), (rho, ux, uy) in r.moments.items():
            n = y * nx + x
            assert abs(lat.rho[n] - float(rho)) < 1e-15
            assert abs(lat.ux[n] - float(ux)) < 1e-16
            assert abs(lat.uy[n] - float(uy)) < 1e-16


def test_bruteforce_channel_zouhe_outflow_freeslip():
    from fractions import Fraction as Fr
    nx, ny = 5, 4
    u0 = {(x, y): (Fr(1, 25) + Fr(x, 400), Fr(y - 1, 300)) for x in range(nx) for y in range(ny)}
    _compare_rational(nx, ny, Fr(4, 5), {(2, 1)},
                      {'w': O.INLET_ZOUHE, 'e': O.OUTFLOW_ZG, 's': O.FREESLIP, 'n': O.FREESLIP},
                      u_in=(Fr(1, 20), Fr(1, 100)), u0=u0)


def test_bruteforce_periodic_walls_force():
    from fractions import Fraction as Fr
    nx, ny = 4, 3
    u0 = {(x, y): (Fr(x + 1, 90), Fr(-y, 70)) for x in range(nx) for y in range(ny)}
    _compare_rational(nx, ny, Fr(7, 10), {(1, 1)},
                      {'w': O.PERIODIC, 'e': O.PERIODIC, 's': O.WALL, 'n': O.WALL},
                      force=(Fr(1, 1000), Fr(-1, 3000)), u0=u0)


def test_bruteforce_equilibrium_inlet_wall_edges():
    from fractions import Fraction as Fr
    nx, ny = 5, 3
    u0 = {(x, y): (Fr(x, 150), Fr(1, 200)) for x in range(nx) for y in range(ny)}
    _compare_rational(nx, ny, Fr(3, 2), set(),
                      {'w': O.INLET_EQ, 'e': O.WALL, 's': O.WALL, 'n': O.FREESLIP},
                      u_in=(Fr(3, 100), 0), u0=u0)


def test_bruteforce_fully_periodic_obstacles():
    from fractions import Fraction as Fr
    nx, ny = 5, 4
    u0 = {(x, y): (Fr(x * y, 500), Fr(x - y, 400)) for x in range(nx) for y in range(ny)}
    _compare_rational(nx, ny, Fr(11, 20), {(0, 0), (3, 2), (4, 2)},
                      {'w': O.PERIODIC, 'e': O.PERIODIC, 's': O.PERIODIC, 'n': O.PERIODIC},
                      force=(Fr(1, 500), Fr(1, 700)), u0=u0)


def test_bruteforce_neumann_inlet_pressure_outlet():
    from fractions import Fraction as Fr
    nx, ny = 6, 4
    u0 = {(x, y): (Fr(1, 40) + Fr(x, 300), Fr(y - 2, 500)) for x in range(nx) for y in range(ny)}
    _compare_rational(nx, ny, Fr(3, 4), {(3, 2)},
                      {'w': O.INLET_EQ_NEUMANN, 'e': O.OUTLET_PRESSURE, 's': O.FREESLIP, 'n': O.WALL},
                      u_in=(Fr(1, 25), Fr(1, 200)), u0=u0, rho_out=Fr(999, 1000))


def test_pressure_outlet_prescribes_density_and_normal_flow():
    """After the Zou-He pressure reconstruction sum_i g_i = rho_out and
    sum_i g_i c_y = 0 exactly (F = 0)."""
    nx, ny = 9, 7
    rng = np.random.default_rng(6)
    case = O.Case(nx, ny, 0.7, ux_in=0.04, bc_w=O.INLET_ZOUHE, bc_e=O.OUTLET_PRESSURE,
                  bc_s=O.WALL, bc_n=O.FREESLIP, rho_out=1.002)
    lat = O.Lattice(case, ux=0.03 + 0.01 * rng.random(nx * ny), uy=0.005 * rng.random(nx * ny))
    lat.run(4)
    col = lambda a: lat.field(a)[:, -1]
    np.testing.assert_allclose(col(lat.rho), 1.002, rtol=0, atol=4e-16)
    np.testing.assert_allclose(col(lat.uy), 0.0, rtol=0, atol=4e-17)


def test_neumann_inlet_takes_previous_neighbour_density():
    """The equilibrium inlet's density at update k is the density of node
    (1, y) in the state after update k - 1 (and Eq. 2 reproduces it)."""
    nx, ny = 8, 5
    rng = np.random.default_rng(7)
    case = O.Case(nx, ny, 0.8, ux_in=0.05, bc_w=O.INLET_EQ_NEUMANN, bc_e=O.OUTLET_PRESSURE,
                  bc_s=O.FREESLIP, bc_n=O.FREESLIP)
    lat = O.Lattice(case, rho=1 + 1e-3 * rng.random(nx * ny), ux=np.full(nx * ny, 0.05))
    lat.run(3)
    prev = 1.0 + lat.h.reshape(9, ny, nx)[:, :, 1].sum(axis=0)
    lat.run(1)
    np.testing.assert_allclose(lat.field(lat.rho)[:, 0], prev, rtol=0, atol=4e-16)
    np.testing.assert_allclose(lat.field(lat.ux)[:, 0], 0.05, rtol=0, atol=2e-17)
