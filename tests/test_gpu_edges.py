"""Degenerate and extreme inputs on the GPU: tiny lattices where a node is
its own neighbour, one-node-wide strips, all-solid masks, the largest tile,
and a lattice large enough (9N >= 2^32 elements) to take the 64-bit
addressing path, each against the FP64 oracle or an invariant."""
import math

import numpy as np
import pytest

import oracle as O
from tests.gpu_helpers import ALGOS, LAYOUTS, rel_linf

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2607_20650_gb300 import build, geometry as G, lbm  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    lbm.load()


def _pair(nx, ny, tau, mask, bc, force=(0.0, 0.0), u_in=(0.0, 0.0), rho0=None, ux0=None, uy0=None, **kw):
    ref = O.Lattice(O.Case(nx, ny, tau, fx=force[0], fy=force[1], ux_in=u_in[0], uy_in=u_in[1],
                           bc_w=bc[0], bc_e=bc[1], bc_s=bc[2], bc_n=bc[3]), mask, rho=rho0, ux=ux0, uy=uy0)
    lat = lbm.Lattice(nx, ny, tau, mask, force=force, u_in=u_in, bc=bc, **kw)
    lat.init(rho0, ux0, uy0)
    return ref, lat


def test_empty_lattice_is_rejected():
    for nx, ny in [(0, 5), (5, 0), (-1, 3)]:
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_workspace_bytes(lbm.make_params(nx, ny, 0.8))
        assert e.value.status == lbm.LBM_EINVAL


@pytest.mark.parametrize("nx,ny", [(1, 1), (1, 7), (9, 1), (2, 2), (3, 1)])
@pytest.mark.parametrize("algo", ALGOS + ("aa",))
def test_tiny_periodic_lattices_match_oracle(nx, ny, algo):
    """On a 1x1 periodic lattice every pull reads the node itself; strips
    wrap onto themselves in one direction."""
    rng = np.random.default_rng(nx * 31 + ny)
    rho0 = 1 + 1e-2 * rng.random(nx * ny)
    ux0, uy0 = 1e-2 * rng.random(nx * ny), 1e-2 * rng.random(nx * ny)
    ref, lat = _pair(nx, ny, 0.7, np.zeros(nx * ny, np.uint8), (G.PERIODIC,) * 4, force=(1e-4, -2e-5),
                     rho0=rho0, ux0=ux0, uy0=uy0, algo=algo, storage="f64", tile=(4, 2))
    ref.run(12)
    lat.step(12, moments=True).sync()
    assert rel_linf(lat.populations(), ref.h) <= 1e-13
    assert rel_linf(lat.moments()[1], ref.ux) <= 1e-13
    lat.close()


@pytest.mark.parametrize("algo", ALGOS)
def test_one_row_channel_with_inlet_outflow(algo):
    """A single row between free-slip edges: every vertical pull is mirrored
    onto the row itself."""
    nx, ny = 23, 1
    ref, lat = _pair(nx, ny, 0.6, np.zeros(nx, np.uint8), (G.INLET_ZOUHE, G.OUTFLOW_ZG, G.FREESLIP, G.FREESLIP),
                     u_in=(0.04, 0.0), ux0=np.full(nx, 0.02), algo=algo, storage="f64", tile=(8, 1))
    ref.run(30)
    lat.step(30, moments=True).sync()
    assert rel_linf(lat.populations(), ref.h) <= 1e-12
    lat.close()


@pytest.mark.parametrize("algo", ALGOS + ("aa",))
def test_all_solid_lattice_stays_zero(algo):
    nx, ny = 40, 12
    lat = lbm.Lattice(nx, ny, 0.8, np.ones(nx * ny, np.uint8), force=(1e-5, 0.0), algo=algo, storage="f32")
    lat.step(10, moments=True).sync()
    assert not lat.populations().any()
    rho, ux, uy = lat.moments()
    assert (rho == 1.0).all() and not ux.any() and not uy.any()
    assert lat.mass() == 0.0
    assert lat.info()["fluid_cells"] == 0
    lat.close()


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("algo,tile", [("nptl", (512, 1)), ("npol", (32, 16)), ("nsol", (16, 32)),
                                       ("nptl", (1, 512)), ("npol", (7, 3))])
def test_largest_and_odd_tiles_on_ragged_lattice(layout, algo, tile):
    nx, ny = 131, 77
    mask = G.porous_discs(nx, ny, seed=19, rmin=3, rmax=7, solid_fraction=0.25)
    ref, lat = _pair(nx, ny, 0.85, mask, (G.PERIODIC,) * 4, force=(2e-5, 1e-5), layout=layout, algo=algo,
                     storage="f64", tile=tile)
    ref.run(25)
    lat.step(25).sync()
    assert rel_linf(lat.populations(), ref.h, ref.solid == 0) <= 1e-12
    lat.close()


def test_tile_above_limit_is_rejected():
    with pytest.raises(lbm.LbmError):
        lbm.lbm_workspace_bytes(lbm.make_params(100, 100, 0.8, algo="nptl", tile=(1024, 1)))


def test_64bit_addressing_path_on_500m_nodes():
    """32768 x 15360 = 503M nodes, FP16 shifted storage, two lattices
    (18 GB): 9N exceeds 2^32 elements, so every kernel takes the 64-bit
    offset path. Three updates from a non-uniform start; sampled nodes equal
    the FP64 oracle on 11x11 windows, and mass is conserved to FP16
    round-off."""
    nx, ny, T, R = 32768, 15360, 3, 5
    assert 9 * nx * ny >= 2 ** 32
    mask = G.porous_discs(nx, ny, seed=41, rmin=8, rmax=32, solid_fraction=0.3)
    lat = lbm.Lattice(nx, ny, 0.9, mask, force=(1e-5, 0.0), layout="stream", algo="nptl",
                      storage="f16s", tile=(64, 4))
    yy = np.arange(ny)[:, None]
    ux0 = np.broadcast_to(2e-2 * np.cos(2 * np.pi * yy / 97.0), (ny, nx)).ravel()
    lat.init(None, ux0, None)
    del ux0
    h0 = lat.populations("f32").reshape(9, ny, nx)
    m0 = lat.mass()
    lat.step(T).sync()
    h1 = lat.populations("f32").reshape(9, ny, nx)
    m1 = lat.mass()
    assert abs(m1 - m0) / m0 <= 1e-6
    rng = np.random.default_rng(3)
    checked = 0
    while checked < 24:
        cy, cx = int(rng.integers(0, ny)), int(rng.integers(0, nx))
        if cx < 2 * nx // 3 or mask[cy, cx]:     # sample the far end of the 64-bit range
            continue
        ys = np.arange(cy - R, cy + R + 1) % ny
        xs = np.arange(cx - R, cx + R + 1) % nx
        n = 2 * R + 1
        o = O.Lattice(O.Case(n, n, 0.9, fx=1e-5, bc_w=O.WALL, bc_e=O.WALL, bc_s=O.WALL, bc_n=O.WALL),
                      mask[np.ix_(ys, xs)])
        if o.solid.reshape(n, n)[R, R]:
            continue
        o.set_h(h0[:, ys][:, :, xs].astype(np.float64).reshape(9, -1))
        o.run(T)
        ref = o.h.reshape(9, n, n)[:, R, R]
        got = h1[:, cy, cx].astype(np.float64)
        # FP32 arithmetic, FP16 storage rounding (half an ulp of ~1e-2 values each update)
        assert np.max(np.abs(got - ref)) <= 3 * T * 2.0 ** -11 * max(np.max(np.abs(ref)), 1e-3)
        checked += 1
    lat.close()
