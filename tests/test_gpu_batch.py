"""Batched ensembles: one persistent launch per update over all cases must
give, for every case, exactly the bits of a single-lattice run of that case
(same arithmetic, only the scheduling differs)."""
import numpy as np
import pytest

from tests.gpu_helpers import COMBOS

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2607_20650_gb300 import build, geometry as G, lbm  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    lbm.load()


def _cases(n, seed=9):
    return G.batch_channels(ncases=n, seed=seed, wmin=20, wmax=140, hmin=9, hmax=70)


def _params(w, storage="f32", rounding="rne", **kw):
    return lbm.make_params(w.nx, w.ny, w.tau, u_in=(w.ux_in, 0.0), bc=(w.bc_w, w.bc_e, w.bc_s, w.bc_n),
                           storage=storage, rounding=rounding, seed=77, **kw)


@pytest.mark.parametrize("storage,rounding", [("f32", "rne"), ("f16s", "sr"), ("f64", "rne")])
def test_batch_equals_single_runs_for_every_combination(storage, rounding):
    ws = _cases(len(COMBOS) + 3)
    params = []
    for k, w in enumerate(ws):
        layout, algo = COMBOS[k % len(COMBOS)]
        tile = (0, 0) if algo == "lptl" else [(32, 8), (64, 4), (16, 16), (32, 2)][k % 4]
        params.append(_params(w, storage, rounding, layout=layout, algo=algo, tile=tile))
    b = lbm.Batch(params, [w.mask for w in ws], plan=False)
    for c, w in enumerate(ws):
        b.init(c, None, w.ux0, w.uy0)
    T = 137                    # one 100-update graph plus a remainder
    b.step(T, moments=True).sync()
    for c, w in enumerate(ws):
        single = lbm.Lattice(w.nx, w.ny, w.tau, w.mask, u_in=(w.ux_in, 0.0),
                             bc=(w.bc_w, w.bc_e, w.bc_s, w.bc_n), layout="stream", algo="nptl",
                             storage=storage, rounding=rounding, seed=77)
        single.init(None, w.ux0, w.uy0)
        single.step(T, moments=True).sync()
        assert np.array_equal(b.populations(c), single.populations()), c
        for x, y in zip(b.moments(c), single.moments()):
            assert np.array_equal(x, y), c
        single.close()
    info = b.info()
    assert info["tiles"] > len(ws) and info["grid"] >= 1
    b.close()


def test_autotuned_batch_equals_single_runs():
    ws = _cases(10, seed=13)
    probe = lbm.make_params(512, 256, 0.8, storage="f32")
    mask = G.porous_discs(512, 256, seed=3, rmin=8, rmax=16)
    nbytes = lbm.lbm_tune_workspace_bytes(probe)
    wsp = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    tuning = lbm.lbm_tune(probe, mask, wsp, nbytes, lbm.current_stream())
    assert tuning.valid == 1
    ns = np.array([[tuning.ns_per_cell[l][a] for a in range(4)] for l in range(3)])
    assert (ns > 0).all() and np.isfinite(ns).all()
    params = [_params(w, layout=lbm.LBM_AUTO, algo=lbm.LBM_AUTO) for w in ws]
    b = lbm.Batch(params, [w.mask for w in ws], tuning=tuning)
    for c, w in enumerate(ws):
        b.init(c, None, w.ux0, w.uy0)
    b.step(60).sync()
    for c, w in enumerate(ws):
        single = lbm.Lattice(w.nx, w.ny, w.tau, w.mask, u_in=(w.ux_in, 0.0),
                             bc=(w.bc_w, w.bc_e, w.bc_s, w.bc_n), storage="f32")
        single.init(None, w.ux0, w.uy0)
        single.step(60).sync()
        assert np.array_equal(b.populations(c), single.populations()), c
        single.close()
    with pytest.raises(lbm.LbmError):
        b.init(0)
    b.close()
