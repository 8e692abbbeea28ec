"""The node-pair two-lattice kernel for 16-bit storage (two adjacent nodes
per thread, packed FP32 arithmetic, packed conversions and 32-bit stores)
must give the same bits as one node per thread (LBM_FLAG_NO_PAIRS) and as
the one-lattice algorithms, which never use pairs.

Lattices have an even nx (pairs need it) and span several tiles with ragged
tails; every edge kind appears, and the porous case puts fluid and solid
nodes in the same pair."""
import numpy as np
import pytest

from tests.gpu_helpers import Spec, rel_linf

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle as O  # noqa: E402
from paper_2607_20650_gb300 import geometry as G, lbm  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2607_20650_gb300 import build
    build.build()
    lbm.load()


def even_specs() -> dict[str, Spec]:
    out = {}
    nx, ny = 62, 29
    m = G.disc(nx, ny, 15.0, 14.0, 4.5)
    r = G.SplitMix64(17, 9)
    out["channel"] = Spec("channel", nx, ny, 0.6, m, (G.INLET_ZOUHE, G.OUTFLOW_ZG, G.FREESLIP, G.FREESLIP),
                          u_in=(0.05, 0.0), ux0=np.where(m.ravel() > 0, 0.0, 0.05),
                          uy0=np.where(m.ravel() > 0, 0.0, r.uniform(nx * ny, -1e-3, 1e-3)))
    nx, ny = 38, 21
    m = np.zeros((ny, nx), np.uint8)
    m[6:12, 11:14] = 1            # odd start and width: mixed pairs on both sides
    out["walls"] = Spec("walls", nx, ny, 0.8, m, (G.PERIODIC, G.PERIODIC, G.WALL, G.WALL), force=(1e-5, 0.0))
    nx, ny = 70, 45
    m = G.porous_discs(nx, ny, seed=15, rmin=3, rmax=6, solid_fraction=0.35)
    r = G.SplitMix64(18, 9)
    out["porous"] = Spec("porous", nx, ny, 0.9, m, (G.PERIODIC,) * 4, force=(1e-5, 2e-6),
                         rho0=1.0 + r.uniform(nx * ny, -1e-3, 1e-3),
                         ux0=r.uniform(nx * ny, -1e-2, 1e-2), uy0=r.uniform(nx * ny, -1e-2, 1e-2))
    nx, ny = 46, 23
    m = np.zeros((ny, nx), np.uint8)
    m[8:15, 21:24] = 1
    out["eq_inlet"] = Spec("eq_inlet", nx, ny, 0.7, m, (G.INLET_EQ, G.WALL, G.WALL, G.FREESLIP),
                           u_in=(0.04, 0.005), ux0=np.full(nx * ny, 0.02))
    nx, ny = 58, 21
    m = G.square(nx, ny, 23.0, 9.0, 5)
    r = G.SplitMix64(19, 9)
    out["neumann_pressure"] = Spec("neumann_pressure", nx, ny, 0.75, m,
                                   (G.INLET_EQ_NEUMANN, G.OUTLET_PRESSURE, G.FREESLIP, G.WALL),
                                   u_in=(0.04, 0.0), rho0=1.0 + r.uniform(nx * ny, -1e-3, 1e-3),
                                   ux0=np.where(m.ravel() > 0, 0.0, 0.04))
    return out


SPECS = even_specs()


def _run(spec, T, **kw):
    lat = spec.gpu(seed=4321, **kw)
    lat.step(T, moments=True).sync()
    out = (lat.populations("f64"), *lat.moments())
    lat.close()
    return out


@pytest.mark.parametrize("case", list(SPECS))
@pytest.mark.parametrize("storage,rounding", [("f16s", "rne"), ("f16s", "sr"), ("bf16s", "rne"),
                                              ("bf16s", "sr")])
def test_pairs_bit_identical_to_one_node_per_thread(case, storage, rounding):
    spec = SPECS[case]
    T = 33
    kw = dict(storage=storage, rounding=rounding)
    base = _run(spec, T, layout="stream", algo="npol", tile=(32, 4), **kw)
    runs = []
    for layout in ("stream", "bundle"):
        for algo, tile in (("lptl", (0, 0)), ("nptl", (64, 2)), ("nptl", (16, 4)), ("nptl", (6, 5))):
            runs.append(dict(layout=layout, algo=algo, tile=tile))
            runs.append(dict(layout=layout, algo=algo, tile=tile, flags=lbm.LBM_FLAG_NO_PAIRS))
    for r in runs:
        got = _run(spec, T, **r, **kw)
        for a, b in zip(got, base):
            assert np.array_equal(a, b), r


def test_pairs_match_oracle_within_fp16_rounding():
    """16-bit shifted storage on the pair path stays near the FP64 oracle:
    after 40 updates of the porous case the velocity error is a few FP16
    units of the ~1e-2 velocities."""
    spec = SPECS["porous"]
    T = 40
    ref = spec.oracle().run(T)
    h, rho, ux, uy = _run(spec, T, layout="bundle", algo="nptl", tile=(64, 2), storage="f16s")
    fl = ref.solid == 0
    assert rel_linf(np.stack([ux, uy]), np.stack([ref.ux, ref.uy]), fl) <= 5e-3
    assert rel_linf(rho, ref.rho, fl) <= 1e-3


def test_odd_nx_runs_one_node_per_thread():
    """A lattice with odd nx (no pairs possible) runs the one-node kernel
    and matches NPOL bit for bit."""
    nx, ny = 41, 17
    m = G.porous_discs(nx, ny, seed=3, rmin=2, rmax=4, solid_fraction=0.3)
    spec = Spec("odd", nx, ny, 0.8, m, (G.PERIODIC,) * 4, force=(1e-5, 0.0))
    a = _run(spec, 20, layout="bundle", algo="nptl", tile=(64, 2), storage="f16s")
    b = _run(spec, 20, layout="stream", algo="npol", tile=(32, 4), storage="f16s")
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    ref = O.Lattice(O.Case(nx, ny, 0.8, fx=1e-5), m).run(20)
    fl = ref.solid == 0
    assert rel_linf(np.stack([a[2], a[3]]), np.stack([ref.ux, ref.uy]), fl) <= 5e-2
