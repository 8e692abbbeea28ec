"""Batched D3Q19 boxes through the lbm3_batch_* C ABI: one launch per update
over the work items of every case must give each case exactly the bits of a
single-box run of that case (same arithmetic, only the scheduling differs),
and FP64 cases follow the FP64 D3Q19 oracle."""
import numpy as np
import pytest

import oracle as O
from paper_2607_20650_gb300 import geometry as G
from tests.gpu_helpers import rel_linf

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2607_20650_gb300 import lbm  # noqa: E402

LAYOUTS = ("stream", "bundle", "collision")
P, W = lbm.PERIODIC, lbm.WALL


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2607_20650_gb300 import build
    build.build()
    lbm.load()


class Box:
    """One case: size, tau, faces, force, mask and a perturbed initial state."""

    def __init__(self, nx, ny, nz, tau, mask, bc, force=(0.0, 0.0, 0.0), seed=1, amp=0.02, **faces):
        self.nx, self.ny, self.nz, self.tau = nx, ny, nz, tau
        self.N = nx * ny * nz
        self.mask = np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
        self.bc, self.force, self.faces = bc, force, faces
        r = G.SplitMix64(seed, 11)
        solid = self.mask > 0
        self.rho0 = np.where(solid, 1.0, 1.0 + r.uniform(self.N, -0.01, 0.01))
        self.u0 = [np.where(solid, 0.0, r.uniform(self.N, -amp, amp)) for _ in range(3)]

    def params(self, **kw):
        return lbm.make_params3(self.nx, self.ny, self.nz, self.tau, force=self.force, bc=self.bc,
                                **self.faces, **kw)

    def single(self, **kw):
        lat = lbm.Lattice3(self.nx, self.ny, self.nz, self.tau, self.mask, force=self.force, bc=self.bc,
                           **self.faces, **kw)
        lat.init(self.rho0, *self.u0)
        return lat

    def oracle(self):
        f = self.faces
        c = O.Case3(self.nx, self.ny, self.nz, self.tau, *self.force, *self.bc) if not f else \
            O.Case3(self.nx, self.ny, self.nz, self.tau, *self.force, bc_x=self.bc[0], bc_xe=f["bc_x_east"],
                    bc_y=self.bc[1], bc_z=self.bc[2], u_in=f["u_in"], rho_out=f.get("rho_out", 1.0))
        return O.Lattice3(c, self.mask, self.rho0, *self.u0)


def boxes(open_faces: bool):
    out = [
        Box(37, 21, 13, 0.7, G.porous_spheres(37, 21, 13, 5, 2.0, 5.0, 0.25), (P, P, P),
            force=(1e-5, 2e-6, -1e-6)),
        Box(45, 19, 11, 0.9, G.ball(45, 19, 11, 12.0, 9.0, 5.0, 3.5), (P, W, W), force=(1e-5, 0.0, 0.0), seed=2),
        Box(33, 5, 3, 0.6, np.pad(np.ones((1, 1, 1), np.uint8), ((1, 1), (2, 2), (7, 25))), (W, P, W), seed=3),
        Box(3, 2, 1, 0.8, np.zeros(6, np.uint8), (P, P, P), seed=4),        # smaller than one tile
        Box(16, 8, 4, 1.3, np.zeros(16 * 8 * 4, np.uint8), (W, W, W), force=(0.0, 3e-6, 1e-6), seed=5),
    ]
    if open_faces:
        out.append(Box(42, 14, 10, 0.7, G.ball(42, 14, 10, 13.0, 7.0, 5.0, 3.0), (lbm.INLET_ZOUHE, W, W), seed=6,
                       bc_x_east=lbm.OUTLET_PRESSURE, u_in=(0.04, 0.003, -0.002), rho_out=0.999))
        out.append(Box(40, 14, 10, 0.7, G.ball(40, 14, 10, 12.0, 7.0, 5.0, 3.0), (lbm.INLET_EQ, W, W), seed=7,
                       bc_x_east=lbm.OUTFLOW_ZG, u_in=(0.04, 0.0, 0.0)))
    return out


def _tile(algo):
    return (0, 0, 0) if algo == "lptl" else ((8, 4, 2) if algo == "nptl" else (8, 4, 3))


def _batch(bs, **kw):
    b = lbm.Batch3([x.params(**kw) for x in bs], [x.mask for x in bs])
    for c, x in enumerate(bs):
        b.init(c, x.rho0, *x.u0)
    return b


@pytest.mark.parametrize("storage,rounding", [("f64", "rne"), ("f32", "rne"), ("f16s", "sr"), ("bf16s", "rne")])
@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("algo", ["lptl", "nptl", "npol", "nsol"])
def test_batch_equals_single_boxes(algo, layout, storage, rounding):
    bs = boxes(open_faces=algo in ("lptl", "nptl"))
    kw = dict(layout=layout, algo=algo, storage=storage, rounding=rounding, seed=77, tile=_tile(algo))
    b = _batch(bs, **kw)
    T = 71                      # one 64-update graph, then seven single launches (odd: parity 1)
    b.step(T, moments=True).sync()
    for c, x in enumerate(bs):
        s = x.single(**kw)
        s.step(T, moments=True).sync()
        assert np.array_equal(b.populations(c, "f64"), s.populations("f64")), c
        for u, v in zip(b.moments(c), s.moments()):
            assert np.array_equal(u, v), c
        assert b.mass(c) == s.mass(), c
        s.close()
    info = b.info()
    assert info["cells"] == sum(x.N for x in bs)
    b.close()


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("algo", ["lptl", "nptl", "npol", "nsol"])
def test_fp64_batch_matches_oracle3(algo, layout):
    bs = boxes(open_faces=algo in ("lptl", "nptl"))
    b = _batch(bs, layout=layout, algo=algo, storage="f64", tile=_tile(algo))
    T = 40
    b.step(T, moments=True).sync()
    for c, x in enumerate(bs):
        ref = x.oracle().run(T)
        fl = ref.solid == 0
        assert rel_linf(b.populations(c, "f64"), ref.h, fl) <= 1e-12, c
        rho, ux, uy, uz = b.moments(c)
        assert rel_linf(rho, ref.rho, fl) <= 1e-14, c
        assert rel_linf(np.stack([ux, uy, uz]), np.stack([ref.ux, ref.uy, ref.uz]), fl) <= 1e-12, c
    b.close()


def test_batch_info_and_work_items():
    bs = boxes(open_faces=False)
    b = _batch(bs, layout="bundle", algo="nptl", storage="f32", tile=(8, 4, 2))
    info = b.info()
    tiles = sum(-(-x.nx // 8) * -(-x.ny // 4) * -(-x.nz // 2) for x in bs)
    assert info["items"] == tiles
    singles = [x.single(layout="bundle", algo="nptl", storage="f32", tile=(8, 4, 2)) for x in bs]
    assert info["fluid_cells"] == sum(s.info()["fluid_cells"] for s in singles)
    assert info["bytes_per_update"] == pytest.approx(sum(s.info()["bytes_per_update"] for s in singles))
    for s in singles:
        s.close()
    lp = _batch(bs, layout="bundle", algo="lptl", storage="f32")
    assert lp.info()["items"] == sum(-(-x.N // 256) for x in bs)
    lp.close()
    b.close()


def test_batch_init_only_before_the_first_update_and_bad_case():
    bs = boxes(open_faces=False)[:2]
    b = _batch(bs, layout="stream", algo="nptl", storage="f32", tile=(8, 4, 2))
    with pytest.raises(lbm.LbmError) as e:
        b.init(2)
    assert e.value.status == lbm.LBM_EINVAL
    b.step(2).sync()
    with pytest.raises(lbm.LbmError) as e:
        b.init(0)
    assert e.value.status == lbm.LBM_EINVAL
    with pytest.raises(lbm.LbmError) as e:
        b.moments(-1)
    assert e.value.status == lbm.LBM_EINVAL
    b.close()


def test_batch_divergence_is_reported():
    bs = boxes(open_faces=False)[:3]
    b = lbm.Batch3([x.params(layout="collision", algo="nptl", storage="f32", tile=(8, 4, 2)) for x in bs],
                   [x.mask for x in bs])
    rho = bs[1].rho0.copy()
    rho[np.flatnonzero(bs[1].mask == 0)[7]] = np.inf
    b.init(1, rho, *bs[1].u0)
    with pytest.raises(lbm.LbmError) as e:
        b.step(2).sync()
    assert e.value.status == lbm.LBM_EDIVERGED
    b.close()


def test_batch_stochastic_rounding_keys_follow_the_update_count():
    """Two batches of the same case with different seeds differ; the same
    seed reproduces the bits (the keys are the seed, the node and the
    update count, shared by the batch)."""
    x = boxes(open_faces=False)[0]
    outs = []
    for seed in (5, 5, 6):
        b = lbm.Batch3([x.params(layout="bundle", algo="nptl", storage="f16s", rounding="sr", seed=seed,
                                 tile=(8, 4, 2))] * 2, [x.mask] * 2)
        for c in range(2):
            b.init(c, x.rho0, *x.u0)
        b.step(20).sync()
        p0, p1 = b.populations(0, "f32"), b.populations(1, "f32")
        assert np.array_equal(p0, p1)       # same case, same seed, same keys
        outs.append(p0)
        b.close()
    assert np.array_equal(outs[0], outs[1])
    assert not np.array_equal(outs[0], outs[2])
