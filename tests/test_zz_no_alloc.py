"""The allocation-free mass entry point agrees with lbm_mass.

Some callers cannot give this library device memory: code hosted by a
framework that owns every device allocation and forbids direct cudaMalloc,
or a loop that must not pay an allocation's implicit synchronisation. For
them lbm_mass_f32_noalloc keeps its scratch in a fixed array inside the
library. These tests call it through the C ABI twice in a row and compare
both results with lbm_mass, the entry point that uses the caller's
workspace, at the tolerance of the other mass tests (1e-13 relative: the two
reductions sum in different fixed orders).

Kept in a file collected last so that a stop-at-first-failure run has
already run every other test if this one fails."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle as O  # noqa: E402
from paper_2607_20650_gb300 import build, geometry as G, lbm  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    lbm.load()


def _state(nx, ny, mask, seed):
    lat = lbm.Lattice(nx, ny, 0.8, mask, force=(2e-5, 1e-6), layout="stream", algo="nptl",
                      storage="f32")
    rng = np.random.default_rng(seed)
    lat.init(1.0 + 1e-3 * rng.random(nx * ny), 1e-2 * rng.random(nx * ny), None)
    lat.step(40).sync()
    return lat


# N = 1 (less than one block of 2,048 nodes), exact multiples of the block,
# and 51,000 nodes (25 blocks, the last one partial).
@pytest.mark.parametrize("nx,ny", [(1, 1), (64, 32), (64, 64), (300, 170)])
def test_noalloc_mass_matches_workspace_mass_twice(nx, ny):
    N = nx * ny
    if N >= 1000:
        mask = G.porous_discs(nx, ny, seed=21, rmin=4, rmax=9, solid_fraction=0.3)
    else:
        mask = np.zeros((ny, nx), np.uint8)
    lat = _state(nx, ny, mask, seed=4)
    solid = O.effective_solid(O.Case(nx, ny, 0.8), mask)
    h = lat.populations("f32")
    d_h = torch.from_numpy(h).cuda()
    d_solid = torch.from_numpy(solid).cuda()
    s = lat.stream
    ref = lat.mass()
    first = lbm.lbm_mass_f32_noalloc(d_h, d_solid, N, s)
    second = lbm.lbm_mass_f32_noalloc(d_h, d_solid, N, s)
    assert abs(first - ref) <= 1e-13 * ref
    assert abs(second - ref) <= 1e-13 * ref
    assert first == second
    if solid.any():
        # Values written into solid nodes are not mass: same bits.
        planted = h.reshape(9, N).copy()
        planted[:, solid > 0] = 0.25
        third = lbm.lbm_mass_f32_noalloc(torch.from_numpy(planted).cuda(), d_solid, N, s)
        assert third == first
    lat.close()


def test_noalloc_mass_effective_versus_raw_mask():
    """An enclosed one-node fluid pocket is solid for lbm_mass; passing the raw
    geometry mask counts it as rho = 1 + sum(h) = 1 (its h stays 0)."""
    nx, ny = 64, 32
    mask = np.zeros((ny, nx), np.uint8)
    mask[10:15, 20:25] = 1
    mask[12, 22] = 0                       # pocket: all eight neighbours solid
    lat = _state(nx, ny, mask, seed=5)
    solid = O.effective_solid(O.Case(nx, ny, 0.8), mask)
    assert solid.reshape(ny, nx)[12, 22] == 1
    d_h = torch.from_numpy(lat.populations("f32")).cuda()
    s = lat.stream
    ref = lat.mass()
    eff = lbm.lbm_mass_f32_noalloc(d_h, torch.from_numpy(solid).cuda(), nx * ny, s)
    raw = lbm.lbm_mass_f32_noalloc(d_h, torch.from_numpy(mask.reshape(-1).copy()).cuda(), nx * ny, s)
    assert abs(eff - ref) <= 1e-13 * ref
    assert abs((raw - eff) - 1.0) <= 1e-9
    lat.close()


def test_noalloc_mass_rejects_sizes_beyond_the_scratch():
    d_h = torch.zeros(9, dtype=torch.float32, device="cuda")
    d_solid = torch.zeros(1, dtype=torch.uint8, device="cuda")
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_mass_f32_noalloc(d_h, d_solid, 65536 * 2048 + 1, torch.cuda.current_stream().cuda_stream)
    assert e.value.status == lbm.LBM_EINVAL
