"""Host read-back of the moments through the C ABI.

lbm_read_moments takes one of four routes: FP64 moments are copied as they
are; FP32 moments are widened to FP64 either by the device straight into a
page-locked destination, or on the host for a pageable one: through an
unpinned buffer for a field of up to 64 MB, through two page-locked staging
chunks of 64 MB beyond that. Every route must give the device's moments
exactly (widening FP32 to FP64 is exact), including a lattice whose fields
span several staging chunks with a ragged tail, and a call that asks for one
field only."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2607_20650_gb300 import lbm  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2607_20650_gb300 import build
    build.build()
    lbm.load()


def _pinned(N):
    return [torch.empty(N, dtype=torch.float64, pin_memory=True).numpy() for _ in range(3)]


# 96 x 40: one partial chunk; 6144 x 5600 = 34,406,400 values per field:
# two full chunks of 16,777,216 FP32 values and a tail of 851,968.
@pytest.mark.parametrize("nx,ny", [(96, 40), (6144, 5600)])
@pytest.mark.parametrize("storage", ["f32", "f16s", "f64"])
def test_read_moments_routes_agree(storage, nx, ny):
    N = nx * ny
    rng = np.random.default_rng(7)
    mask = np.zeros((ny, nx), np.uint8)
    mask[ny // 3: ny // 3 + ny // 8, nx // 4: nx // 4 + nx // 16] = 1
    ux0 = 0.02 + 1e-3 * rng.standard_normal(N)
    uy0 = 1e-3 * rng.standard_normal(N)
    lat = lbm.Lattice(nx, ny, 0.8, mask, force=(1e-5, 0.0), bc=(lbm.PERIODIC,) * 4,
                      layout="bundle", algo="nptl", storage=storage)
    lat.init(None, ux0, uy0)
    lat.step(3, moments=True).sync()
    pageable = lat.moments()
    pinned = lat.moments(out=_pinned(N))
    comp = torch.float64 if storage == "f64" else torch.float32
    dev = [torch.empty(N, dtype=comp, device="cuda") for _ in range(3)] if storage != "f64" else None
    if dev is not None:
        lbm.lbm_moments_device(lat.h, *dev)
        lat.sync()
        ref = [d.cpu().numpy().astype(np.float64) for d in dev]
    else:
        ref = pageable
    for k in range(3):
        assert np.array_equal(pageable[k], ref[k]), f"pageable field {k}"
        assert np.array_equal(pinned[k], ref[k]), f"page-locked field {k}"
    assert np.any(pinned[1] != 0.0) and np.all(np.isfinite(pinned[1]))
    # one field only, the others NULL
    ux = np.empty(N)
    assert lbm.load().lbm_read_moments(lat.h, None, ux.ctypes.data, None) == 0
    assert np.array_equal(ux, ref[1])
    lat.close()


def test_read_moments_rejects_bad_out():
    lat = lbm.Lattice(64, 16, 0.8, np.zeros((16, 64), np.uint8), bc=(lbm.PERIODIC,) * 4,
                      layout="stream", algo="lptl", storage="f32")
    with pytest.raises(ValueError):
        lat.moments(out=[np.empty(64 * 16, np.float32)] * 3)
    with pytest.raises(ValueError):
        lat.moments(out=[np.empty(10)] * 3)
    lat.close()
