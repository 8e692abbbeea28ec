"""The L2 prefetch of the FP32 two-lattice and AA kernels changes no result.

On a lattice larger than L2, states after the same updates with and without
the prefetch (LBM_FLAG_NO_PREFETCH) must be bit-identical for every kernel
that carries it, and the distance the library reports must be the one it
documents: 5/4 of the device's resident threads, in nodes (LPTL) or rows
(NPTL, AA). Kernels without it (16-bit storage, the collision layout, FP64,
NPOL) and lattices that fit in L2 report 0."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2607_20650_gb300 import geometry as G  # noqa: E402
from paper_2607_20650_gb300 import lbm  # noqa: E402

NX, NY = 2048, 2560            # 5.2M nodes: 189 MB of FP32 populations per lattice, > L2


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2607_20650_gb300 import build
    build.build()
    lbm.load()


@pytest.fixture(scope="module")
def inputs():
    rng = np.random.default_rng(11)
    mask = G.porous_discs(NX, NY, seed=5)
    ux = 0.02 + 2e-3 * rng.standard_normal(NX * NY)
    uy = 2e-3 * rng.standard_normal(NX * NY)
    return mask, ux, uy


def _resident_nodes():
    p = torch.cuda.get_device_properties(0)
    return p.multi_processor_count * p.max_threads_per_multi_processor * 5 // 4


def _run(inputs, layout, algo, storage, tile, flags, steps=6):
    mask, ux, uy = inputs
    kw = dict(tile=tile) if tile else {}
    lat = lbm.Lattice(NX, NY, 0.8, mask, force=(1e-5, 0.0), bc=(lbm.PERIODIC, lbm.PERIODIC, lbm.WALL, lbm.WALL),
                      layout=layout, algo=algo, storage=storage, flags=flags, **kw)
    lat.init(None, ux, uy)
    lat.step(steps).sync()
    info = lat.info()
    h = lat.populations(storage)
    lat.close()
    return info["prefetch_distance"], h


@pytest.mark.parametrize("layout,algo,tile", [("bundle", "nptl", (32, 4)), ("stream", "nptl", (32, 4)),
                                              ("bundle", "lptl", None), ("stream", "lptl", None),
                                              ("bundle", "aa", (128, 1)), ("stream", "aa", (64, 2))])
def test_prefetch_bit_identical_and_distance(inputs, layout, algo, tile):
    d_on, h_on = _run(inputs, layout, algo, "f32", tile, 0)
    d_off, h_off = _run(inputs, layout, algo, "f32", tile, lbm.LBM_FLAG_NO_PREFETCH)
    nodes = _resident_nodes()
    expected = nodes if algo == "lptl" else max(1, (nodes + NX // 2) // NX)
    assert d_on == expected and d_off == 0
    assert np.array_equal(h_on, h_off)
    assert np.all(np.isfinite(h_on))


@pytest.mark.parametrize("layout,algo,storage,tile", [("bundle", "nptl", "f16s", (64, 4)),
                                                      ("collision", "nptl", "f32", (64, 4)),
                                                      ("collision", "lptl", "f32", None),
                                                      ("bundle", "nptl", "f64", (128, 1)),
                                                      ("stream", "npol", "f32", (32, 8))])
def test_no_prefetch_where_it_is_compiled_out(inputs, layout, algo, storage, tile):
    mask, _, _ = inputs
    kw = dict(tile=tile) if tile else {}
    lat = lbm.Lattice(NX, NY, 0.8, mask, bc=(lbm.PERIODIC,) * 4, layout=layout, algo=algo, storage=storage, **kw)
    assert lat.info()["prefetch_distance"] == 0
    lat.close()


def test_no_prefetch_when_the_lattice_fits_in_l2():
    lat = lbm.Lattice(512, 256, 0.8, None, bc=(lbm.PERIODIC,) * 4, layout="bundle", algo="nptl", storage="f32",
                      tile=(32, 4))
    assert lat.info()["prefetch_distance"] == 0
    lat.close()
