"""NSOL with each tile staged by one tensor copy (TMA) into shared memory:
FP32 storage, stream and bundle layouts, whenever nx and tile_x are multiples
of 4 and a tile's row fits one copy. The staging is the only change, so the
states and moments must equal those of the per-thread staging
(LBM_FLAG_NO_TMA) bit for bit: ragged tiles at the lattice edges, every edge
kind the one-lattice algorithms take, the widest bundle row (3 x 84 values)
and the tallest tile; lattices that do not qualify fall back."""
import numpy as np
import pytest

from paper_2607_20650_gb300 import geometry as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2607_20650_gb300 import lbm  # noqa: E402

P, W = lbm.PERIODIC, lbm.WALL


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2607_20650_gb300 import build
    build.build()
    lbm.load()


def _porous(nx, ny, seed):
    return G.porous_discs(nx, ny, seed=seed, rmin=3, rmax=7, solid_fraction=0.3)


CASES = {
    # name: nx, ny, mask, edges (w, e, s, n), extra parameters
    "porous_periodic": (124, 60, _porous(124, 60, 5), (P, P, P, P), dict(force=(1e-5, 2e-6))),
    "channel_inlet_outflow": (96, 30, G.disc(96, 30, 24.0, 15.0, 5.0), (lbm.INLET_ZOUHE, lbm.OUTFLOW_ZG, W, W),
                              dict(u_in=(0.04, 0.0))),
    "channel_eq_inlet_pressure": (72, 26, G.disc(72, 26, 20.0, 13.0, 4.0),
                                  (lbm.INLET_EQ_NEUMANN, lbm.OUTLET_PRESSURE, W, W), dict(u_in=(0.03, 0.0))),
    "walls_force": (64, 36, _porous(64, 36, 9), (W, W, W, W), dict(force=(3e-6, -1e-6))),
}


def _lattice(name, layout, tile, flags):
    nx, ny, mask, bc, extra = CASES[name]
    lat = lbm.Lattice(nx, ny, 0.7, mask, bc=bc, layout=layout, algo="nsol", storage="f32", tile=tile,
                      flags=flags, **extra)
    r = G.SplitMix64(3, 7)
    ux = r.uniform(nx * ny, -0.02, 0.02)
    uy = r.uniform(nx * ny, -0.02, 0.02)
    if mask is not None:
        ux[np.asarray(mask).reshape(-1) > 0] = 0.0
        uy[np.asarray(mask).reshape(-1) > 0] = 0.0
    lat.init(None, ux, uy)
    return lat


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("layout,tile", [("stream", (32, 8)), ("bundle", (32, 8)), ("stream", (4, 64)),
                                         ("bundle", (84, 2)), ("stream", (16, 16)), ("bundle", (8, 4))])
def test_tensor_copy_staging_is_bit_identical(name, layout, tile):
    T = 37
    a = _lattice(name, layout, tile, 0)
    b = _lattice(name, layout, tile, lbm.LBM_FLAG_NO_TMA)
    assert a.info()["aux"] == 1 and b.info()["aux"] == 0
    a.step(T, moments=True).sync()
    b.step(T, moments=True).sync()
    ha, hb = a.populations("f32"), b.populations("f32")
    assert np.array_equal(ha, hb)
    assert np.all(np.isfinite(ha))
    for u, v in zip(a.moments(), b.moments()):
        assert np.array_equal(u, v)
    a.close()
    b.close()


def test_lattices_that_do_not_qualify_stage_per_thread():
    for nx, tile, layout, storage in [(62, (32, 8), "stream", "f32"),     # nx not a multiple of 4
                                      (64, (30, 8), "stream", "f32"),     # tile_x not a multiple of 4
                                      (256, (128, 2), "bundle", "f32"),   # bundle row of 384 values
                                      (64, (32, 8), "collision", "f32"),  # collision layout
                                      (64, (32, 8), "stream", "f16s")]:   # 16-bit storage
        lat = lbm.Lattice(nx, 32, 0.8, None, bc=(P,) * 4, layout=layout, algo="nsol", storage=storage, tile=tile)
        assert lat.info()["aux"] == 0, (nx, tile, layout, storage)
        lat.step(3).sync()
        lat.close()
