"""The allocation-free mass entry point (for callers that cannot allocate
device memory: hosts whose framework owns all device allocations, or loops
that must not pay an allocation's synchronisation) agrees with lbm_mass.

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


def test_noalloc_mass_matches_workspace_mass_twice():
    build.build()
    lbm.load()
    nx, ny = 300, 170
    mask = G.porous_discs(nx, ny, seed=21, rmin=4, rmax=9, solid_fraction=0.3)
    lat = lbm.Lattice(nx, ny, 0.8, mask, force=(2e-5, 1e-6), layout="stream", algo="nptl",
                      storage="f32")
    rng = np.random.default_rng(4)
    lat.init(1.0 + 1e-3 * rng.random(nx * ny), 1e-2 * rng.random(nx * ny), None)
    lat.step(40).sync()
    solid = O.effective_solid(O.Case(nx, ny, 0.8), mask)
    d_h = torch.from_numpy(lat.populations("f32")).cuda()
    d_solid = torch.from_numpy(solid).cuda()
    s = lat.stream
    ref = lat.mass()
    first = lbm.lbm_mass_f32_noalloc(d_h, d_solid, lat.N, s)
    second = lbm.lbm_mass_f32_noalloc(d_h, d_solid, lat.N, s)
    assert abs(first - ref) <= 1e-13 * ref
    assert abs(second - ref) <= 1e-13 * ref
    assert first == second
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_mass_f32_noalloc(d_h, d_solid, 65536 * 2048 + 1, s)
    assert e.value.status == lbm.LBM_EINVAL
    lat.close()
