"""The AA pattern (in-place streaming, one lattice, no buffer grid): same
bits as the two-lattice pull at every precision, FP64 parity with the oracle,
exact streaming, and the documented limits (state readable after an even
number of updates; zero-gradient outflow rejected)."""
import math

import numpy as np
import pytest

from tests.gpu_helpers import LAYOUTS, aa_specs, rel_linf, specs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2607_20650_gb300 import build, lbm  # noqa: E402

SPECS = aa_specs()


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    lbm.load()


@pytest.mark.parametrize("case", list(SPECS))
@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("storage,rounding", [("f64", "rne"), ("f32", "rne"), ("f16s", "sr")])
def test_aa_equals_two_lattice_pull(case, layout, storage, rounding):
    spec = SPECS[case]
    T = 38
    aa = spec.gpu(layout=layout, algo="aa", storage=storage, rounding=rounding, seed=31, tile=(32, 4))
    ref = spec.gpu(layout="stream", algo="nptl", storage=storage, rounding=rounding, seed=31)
    aa.step(T, moments=True).sync()
    ref.step(T, moments=True).sync()
    assert np.array_equal(aa.populations(), ref.populations())
    for x, y in zip(aa.moments(), ref.moments()):
        assert np.array_equal(x, y)
    aa.close()
    ref.close()


@pytest.mark.parametrize("case", list(SPECS))
def test_aa_fp64_matches_oracle(case):
    spec = SPECS[case]
    T = 60
    ref = spec.oracle().run(T)
    lat = spec.gpu(layout="bundle", algo="aa", storage="f64")
    lat.step(T, moments=True).sync()
    fl = ref.solid == 0
    assert rel_linf(lat.populations(), ref.h, fl) <= 1e-12
    rho, ux, uy = lat.moments()
    assert rel_linf(np.stack([ux, uy]), np.stack([ref.ux, ref.uy]), fl) <= 1e-12
    assert abs(lat.mass() - ref.mass()) <= 1e-13 * ref.mass()
    lat.close()


def test_aa_state_after_odd_count_and_graphs():
    spec = SPECS["porous"]
    a = spec.gpu(algo="aa", storage="f32", tile=(32, 8))
    b = spec.gpu(algo="aa", storage="f32", tile=(32, 8), flags=lbm.LBM_FLAG_NO_GRAPH)
    a.step(131, moments=True).sync()       # two 64-update graphs and three single updates
    b.step(131, moments=True).sync()
    for x, y in zip(a.moments(), b.moments()):
        assert np.array_equal(x, y)
    with pytest.raises(lbm.LbmError) as e:
        a.populations()
    assert e.value.status == lbm.LBM_EINVAL
    a.step(1).sync()
    b.step(1).sync()
    assert np.array_equal(a.populations(), b.populations())
    a.close()
    b.close()


@pytest.mark.parametrize("layout", LAYOUTS)
def test_aa_pure_streaming_is_exact_shift(layout):
    nx, ny, T = 41, 23, 8
    rng = np.random.default_rng(5)
    h0 = rng.normal(0.0, 0.01, size=(9, nx * ny)).astype(np.float32).astype(np.float64)
    lat = lbm.Lattice(nx, ny, math.inf, None, layout=layout, algo="aa", storage="f32", tile=(32, 4))
    lat.write_populations(h0)
    lat.step(T).sync()
    h = lat.populations()
    for i in range(9):
        exp = np.roll(h0[i].reshape(ny, nx), (T * (i // 3 - 1), T * (i % 3 - 1)), axis=(0, 1)).ravel()
        assert np.array_equal(h[i], exp)
    lat.close()


def test_aa_rejects_zero_gradient_outflow():
    spec = specs()["channel"]
    with pytest.raises(lbm.LbmError) as e:
        spec.gpu(algo="aa", storage="f32")
    assert e.value.status == lbm.LBM_EUNSUPPORTED
