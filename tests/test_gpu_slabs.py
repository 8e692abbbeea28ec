"""The x-slab decomposition on the GPU, through the C ABI's face exchange
(lbm_face_pack / lbm_face_unpack): slabs held by one process exchange on the
device, slabs held by two processes (gloo ranks sharing this GPU, their
kernels never waiting on one another) exchange through page-locked host
memory. Either way the slabs' interiors equal the undivided lattice bit for
bit: every algorithm the exchange takes (LPTL, NPTL, NPOL, NSOL), every
layout and storage type, the edge kinds of the one-lattice and two-lattice
paths, ragged tiles; the undivided lattice itself is held to the FP64 oracle
by the parity tests."""
import os
import socket
import tempfile

import numpy as np
import pytest

from paper_2607_20650_gb300 import geometry as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2607_20650_gb300 import lbm  # noqa: E402
from paper_2607_20650_gb300 import slabs as S  # noqa: E402

P, W = lbm.PERIODIC, lbm.WALL


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2607_20650_gb300 import build
    build.build()
    lbm.load()


def _porous(nx, ny, seed):
    return G.porous_discs(nx, ny, seed=seed, rmin=3, rmax=6, solid_fraction=0.3)


CASES = {
    # name: nx, ny, mask, edges (w, e, s, n), extra parameters
    "porous_periodic": (90, 40, _porous(90, 40, 5), (P, P, P, P), dict(force=(1e-5, 2e-6))),
    "zou_he_outflow": (96, 30, G.disc(96, 30, 33.0, 15.0, 5.0), (lbm.INLET_ZOUHE, lbm.OUTFLOW_ZG, W, W),
                       dict(u_in=(0.04, 0.0))),
    "neumann_pressure": (72, 26, G.disc(72, 26, 24.0, 13.0, 4.0), (lbm.INLET_EQ_NEUMANN, lbm.OUTLET_PRESSURE, W, W),
                         dict(u_in=(0.03, 0.0), rho_out=0.995)),
    "walls_force": (64, 36, _porous(64, 36, 9), (W, W, W, W), dict(force=(3e-6, -1e-6))),
}


def _fields(nx, ny, mask):
    r = G.SplitMix64(3, 7)
    rho = 1.0 + r.uniform(nx * ny, -0.01, 0.01)
    ux = r.uniform(nx * ny, -0.02, 0.02)
    uy = r.uniform(nx * ny, -0.02, 0.02)
    solid = np.asarray(mask).reshape(-1) > 0
    ux[solid] = 0.0
    uy[solid] = 0.0
    return rho, ux, uy


def _reference(name, T, **kw):
    nx, ny, mask, bc, extra = CASES[name]
    lat = lbm.Lattice(nx, ny, 0.7, mask, bc=bc, **extra, **kw)
    lat.init(*_fields(nx, ny, mask))
    lat.step(T, moments=True).sync()
    out = lat.populations("f64"), lat.moments()
    lat.close()
    return out


def _check_equal(dec, ref, owned=None):
    pops, mom = ref
    got_p, got_m = dec.populations("f64"), dec.moments()
    nx, ny = dec.nx, dec.ny
    cols = np.zeros(nx, bool)
    for s in (dec.owned if owned is None else owned):
        cols[dec.slabs[s].x0:dec.slabs[s].x1] = True
    a, b = got_p.reshape(9, ny, nx)[:, :, cols], pops.reshape(9, ny, nx)[:, :, cols]
    assert np.array_equal(a, b)
    for u, v in zip(got_m, mom):
        assert np.array_equal(u.reshape(ny, nx)[:, cols], v.reshape(ny, nx)[:, cols])
    assert np.all(np.isfinite(a))


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("algo,layout,tile", [("lptl", "stream", (0, 0)), ("nptl", "bundle", (0, 0)),
                                              ("nptl", "collision", (16, 4)), ("npol", "stream", (8, 4)),
                                              ("npol", "bundle", (16, 8)), ("nsol", "bundle", (8, 4)),
                                              ("nsol", "stream", (32, 8)), ("nsol", "collision", (8, 8))])
@pytest.mark.parametrize("parts", [2, 3])
def test_slabs_equal_the_undivided_lattice_fp32(name, algo, layout, tile, parts):
    T = 33
    kw = dict(algo=algo, layout=layout, storage="f32", tile=tile)
    ref = _reference(name, T, **kw)
    nx, ny, mask, bc, extra = CASES[name]
    dec = S.Decomposition(nx, ny, 0.7, mask, parts=parts, bc=bc, **extra, **kw)
    dec.init(*_fields(nx, ny, mask))
    dec.step(T, moments=True).sync()
    _check_equal(dec, ref)
    dec.close()


@pytest.mark.parametrize("storage", ["f64", "f16s", "bf16s"])
@pytest.mark.parametrize("algo,layout", [("nptl", "stream"), ("lptl", "bundle"), ("npol", "collision"),
                                         ("nsol", "bundle")])
def test_slabs_equal_the_undivided_lattice_other_storage(storage, algo, layout):
    T = 29
    for name in ("porous_periodic", "zou_he_outflow"):
        kw = dict(algo=algo, layout=layout, storage=storage)
        ref = _reference(name, T, **kw)
        nx, ny, mask, bc, extra = CASES[name]
        dec = S.Decomposition(nx, ny, 0.7, mask, parts=4, bc=bc, align=1, **extra, **kw)
        dec.init(*_fields(nx, ny, mask))
        dec.step(T, moments=True).sync()
        _check_equal(dec, ref)
        dec.close()


def test_one_slab_is_the_lattice():
    T = 20
    name = "porous_periodic"
    ref = _reference(name, T)
    nx, ny, mask, bc, extra = CASES[name]
    dec = S.Decomposition(nx, ny, 0.7, mask, parts=1, bc=bc, **extra)
    assert dec.msgs == []
    dec.init(*_fields(nx, ny, mask))
    dec.step(T, moments=True).sync()
    _check_equal(dec, ref)
    dec.close()


def test_stochastic_rounding_slabs_draw_their_own_keys():
    """With stochastic rounding each slab keys its draws on its own node
    index: the state differs from the undivided lattice's in the last bits
    only, and stays as close to it as two runs with different seeds."""
    T = 40
    name = "porous_periodic"
    nx, ny, mask, bc, extra = CASES[name]
    kw = dict(algo="nptl", layout="bundle", storage="f16s", rounding="sr", seed=5)
    ref_p, ref_m = _reference(name, T, **kw)
    other_p, _ = _reference(name, T, **dict(kw, seed=6))
    dec = S.Decomposition(nx, ny, 0.7, mask, parts=3, bc=bc, **extra, **kw)
    dec.init(*_fields(nx, ny, mask))
    dec.step(T, moments=True).sync()
    p = dec.populations("f64")
    assert np.all(np.isfinite(p))
    assert not np.array_equal(p, ref_p)
    assert np.abs(p - ref_p).max() <= 2.0 * np.abs(other_p - ref_p).max() + 1e-12
    assert np.abs(dec.moments()[0] - ref_m[0]).max() < 2e-3
    dec.close()


@pytest.mark.parametrize("algo,layout,storage", [("nptl", "bundle", "f32"), ("npol", "stream", "f16s"),
                                                  ("nsol", "collision", "f64")])
def test_many_slabs_exchange_in_several_launches(algo, layout, storage):
    """Nine slabs of a periodic lattice: 18 messages per update, more than
    one launch of the one-launch exchange takes."""
    T = 17
    name = "porous_periodic"
    kw = dict(algo=algo, layout=layout, storage=storage, tile=(8, 4))
    ref = _reference(name, T, **kw)
    nx, ny, mask, bc, extra = CASES[name]
    dec = S.Decomposition(nx, ny, 0.7, mask, parts=9, bc=bc, align=4, **extra, **kw)
    assert len(dec.msgs) == 18
    dec.init(*_fields(nx, ny, mask))
    dec.step(T, moments=True).sync()
    _check_equal(dec, ref)
    dec.close()


def test_one_launch_exchange_equals_pack_then_unpack():
    nx, ny = 40, 12
    for storage, layout, algo in [("f32", "stream", "nptl"), ("bf16s", "bundle", "nsol")]:
        lats = []
        for seed in range(4):
            lat = lbm.Lattice(nx, ny, 0.8, None, storage=storage, layout=layout, algo=algo, force=(1e-4 * seed, 0.0))
            lat.init(*_fields(nx, ny, np.zeros(nx * ny)))
            lat.step(2 + seed).sync()
            lats.append(lat)
        a0, a1, b0, b1 = lats
        b0.write_populations(a0.populations("f64"))
        b1.write_populations(a1.populations("f64"))
        assert np.array_equal(b0.populations("f64"), a0.populations("f64"))
        before = a1.populations("f64")
        msgs = [(5, 0, 1), (nx - 2, nx - 1, -1), (17, 3, 1)]
        lbm.lbm_face_exchange([a0.h] * 3, [m[0] for m in msgs], [a1.h] * 3, [m[1] for m in msgs],
                              [m[2] for m in msgs], a0.stream)
        assert not np.array_equal(a1.populations("f64"), before)
        buf = torch.zeros(3 * ny * S.ELEM_BYTES[storage], dtype=torch.uint8, device="cuda")
        for xs, xd, sense in msgs:
            b0.face_pack(xs, sense, buf)
            b1.face_unpack(xd, sense, buf)
        for lat in lats:
            lat.sync()
        assert np.array_equal(a1.populations("f64"), b1.populations("f64"))
        for lat in lats:
            lat.close()


def test_face_exchange_rejects_bad_arguments():
    nx, ny = 32, 16
    buf = torch.zeros(3 * ny * 4, dtype=torch.uint8, device="cuda")
    lat = lbm.Lattice(nx, ny, 0.8, None, algo="nptl")
    lat.init()
    for x, sense in [(-1, 1), (nx, 1), (3, 0), (3, 2)]:
        with pytest.raises(lbm.LbmError) as e:
            lat.face_pack(x, sense, buf)
        assert e.value.status == lbm.LBM_EINVAL
        with pytest.raises(lbm.LbmError):
            lat.face_unpack(x, sense, buf)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_face_pack(lat.h, 3, 1, None)
    lat.close()
    other = lbm.Lattice(nx, ny, 0.8, None, algo="nptl")
    other_ny = lbm.Lattice(nx, ny + 2, 0.8, None, algo="nptl")
    other_st = lbm.Lattice(nx, ny, 0.8, None, algo="nptl", storage="f16s")
    for dst in (other_ny, other_st):
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_face_exchange([other.h], [3], [dst.h], [0], [1], other.stream)
        assert e.value.status == lbm.LBM_EINVAL
    with pytest.raises(lbm.LbmError):
        lbm.lbm_face_exchange([other.h] * 65, [3] * 65, [other.h] * 65, [0] * 65, [1] * 65, other.stream)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_face_exchange([other.h], [nx], [other.h], [0], [1], other.stream)
    lbm.lbm_face_exchange([], [], [], [], [], other.stream)
    for x in (other, other_ny, other_st):
        x.close()
    aa = lbm.Lattice(nx, ny, 0.8, None, algo="aa")
    aa.init()
    with pytest.raises(lbm.LbmError) as e:
        aa.face_pack(3, 1, buf)
    assert e.value.status == lbm.LBM_EINVAL
    aa.close()
    with pytest.raises(ValueError):
        S.Decomposition(nx, ny, 0.8, None, parts=2, algo="aa")


def test_face_pack_then_unpack_moves_the_stored_bits():
    """Pack of column x equals the three stored values read back in
    canonical order; unpack into another lattice writes exactly them."""
    nx, ny = 24, 10
    for storage, layout, algo in [("f32", "bundle", "nptl"), ("f16s", "collision", "nsol"), ("f64", "stream", "npol")]:
        a = lbm.Lattice(nx, ny, 0.8, None, storage=storage, layout=layout, algo=algo)
        a.init(*_fields(nx, ny, np.zeros(nx * ny)))
        a.step(3).sync()
        b = lbm.Lattice(nx, ny, 0.8, None, storage=storage, layout=layout, algo=algo)
        b.init()
        b.step(3).sync()
        elem = S.ELEM_BYTES[storage]
        sent = {}
        for x, sense in [(0, 1), (nx - 1, -1), (7, 1), (7, -1)]:
            buf = torch.zeros(3 * ny * elem, dtype=torch.uint8, device="cuda")
            a.face_pack(x, sense, buf)
            b.face_unpack(x, sense, buf)
            sent[(x, sense)] = buf
        a.sync()
        b.sync()
        pa = a.populations("f64").reshape(9, ny, nx)
        pb = b.populations("f64").reshape(9, ny, nx)
        as_type = {"f64": torch.float64, "f32": torch.float32, "f16s": torch.float16, "bf16s": torch.bfloat16}
        for (x, sense), buf in sent.items():
            dirs = [3 * k + sense + 1 for k in range(3)]
            # the message holds directions SE, E, NE (or SW, W, NW) of column x, y-major
            msg = buf.view(as_type[storage]).double().cpu().numpy().reshape(3, ny)
            assert np.array_equal(msg, pa[dirs, :, x])
            assert np.array_equal(pa[dirs, :, x], pb[dirs, :, x])
        a.close()
        b.close()


# ---------------------------------------------------------------- two processes

def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, port, name, parts, kw, T, outdir):
    import datetime

    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=parts, timeout=datetime.timedelta(seconds=120))
    try:
        torch.cuda.set_device(0)
        lbm.load()
        nx, ny, mask, bc, extra = CASES[name]
        dec = S.Decomposition(nx, ny, 0.7, mask, parts=parts, owned=[rank], bc=bc, **extra, **kw)
        dec.init(*_fields(nx, ny, mask))
        dec.step(T, moments=True).sync()
        rho, ux, uy = dec.moments()
        np.savez(os.path.join(outdir, f"r{rank}.npz"), p=dec.populations("f64"), rho=rho, ux=ux, uy=uy)
        dec.close()
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name,parts,kw", [("porous_periodic", 2, dict(algo="nptl", layout="bundle")),
                                           ("zou_he_outflow", 2, dict(algo="nsol", layout="stream")),
                                           ("neumann_pressure", 3, dict(algo="lptl", layout="collision",
                                                                        storage="f16s"))])
def test_slabs_on_separate_processes_exchange_through_host_memory(name, parts, kw):
    import torch.multiprocessing as mp
    T = 21
    ref = _reference(name, T, **kw)
    ctx = mp.get_context("spawn")
    port = _free_port()
    with tempfile.TemporaryDirectory() as d:
        procs = [ctx.Process(target=_rank, args=(r, port, name, parts, kw, T, d)) for r in range(parts)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(300)
        for p in procs:
            if p.is_alive():
                p.terminate()
                p.join(30)
        assert all(p.exitcode == 0 for p in procs)
        nx, ny, _, bc, _ = CASES[name]
        sl = S.split(nx, parts, bc[0] == P and bc[1] == P)
        pops, mom = ref
        for r in range(parts):
            z = np.load(os.path.join(d, f"r{r}.npz"))
            c = slice(sl[r].x0, sl[r].x1)
            assert np.array_equal(z["p"].reshape(9, ny, nx)[:, :, c], pops.reshape(9, ny, nx)[:, :, c])
            for k, key in enumerate(("rho", "ux", "uy")):
                assert np.array_equal(z[key].reshape(ny, nx)[:, c], mom[k].reshape(ny, nx)[:, c])


# ---------------------------------------------------------------- D3Q19 boxes

CASES3 = {
    # name: nx, ny, nz, mask, (bc_x, bc_y, bc_z), extra parameters
    "spheres_periodic": (40, 12, 10, G.porous_spheres(40, 12, 10, 5, 1.5, 3.0, 0.25), (P, P, P),
                         dict(force=(2e-5, -4e-6, 1e-6))),
    "walls_force": (36, 10, 8, G.porous_spheres(36, 10, 8, 7, 1.5, 2.5, 0.2), (W, P, W),
                    dict(force=(1e-5, 0.0, 3e-6))),
    "zou_he_pressure": (44, 10, 8, G.ball(44, 10, 8, 15.0, 5.0, 4.0, 2.5), (lbm.INLET_ZOUHE, W, W),
                        dict(bc_x_east=lbm.OUTLET_PRESSURE, u_in=(0.04, 0.0, 0.0), rho_out=0.997)),
    "eq_outflow": (40, 10, 8, G.ball(40, 10, 8, 21.0, 5.0, 4.0, 2.0), (lbm.INLET_EQ, P, W),
                   dict(bc_x_east=lbm.OUTFLOW_ZG, u_in=(0.03, 0.0, 0.0))),
}


def _fields3(nx, ny, nz, mask):
    r = G.SplitMix64(11, 2)
    n = nx * ny * nz
    rho = 1.0 + r.uniform(n, -0.01, 0.01)
    u = [r.uniform(n, -0.02, 0.02) for _ in range(3)]
    for a in u:
        a[np.asarray(mask).reshape(-1) > 0] = 0.0
    return (rho, *u)


def _reference3(name, T, **kw):
    nx, ny, nz, mask, bc, extra = CASES3[name]
    lat = lbm.Lattice3(nx, ny, nz, 0.75, mask, bc=bc, **extra, **kw)
    lat.init(*_fields3(nx, ny, nz, mask))
    lat.step(T, moments=True).sync()
    out = lat.populations("f64"), lat.moments()
    lat.close()
    return out


def _run3(name, T, parts, align, **kw):
    nx, ny, nz, mask, bc, extra = CASES3[name]
    dec = S.Decomposition(nx, ny, 0.75, mask, nz=nz, parts=parts, bc=bc, align=align, **extra, **kw)
    dec.init(*_fields3(nx, ny, nz, mask))
    dec.step(T, moments=True).sync()
    p, m = dec.populations("f64"), dec.moments()
    dec.close()
    return p, m


def _equal3(got, ref):
    assert np.array_equal(got[0], ref[0])
    assert len(got[1]) == 4
    for u, v in zip(got[1], ref[1]):
        assert np.array_equal(u, v)
    assert np.all(np.isfinite(got[0]))


OPEN3 = ("zou_he_pressure", "eq_outflow")   # inlet and outlet faces: LPTL / NPTL only
ALGOS3 = [("lptl", "bundle", (0, 0, 0)), ("nptl", "stream", (16, 2, 2)), ("nptl", "collision", (0, 0, 0)),
          ("npol", "stream", (8, 4, 2)), ("npol", "bundle", (4, 4, 4)), ("nsol", "bundle", (8, 4, 2)),
          ("nsol", "collision", (4, 4, 4))]
RUNS3 = [(name,) + a for name in CASES3 for a in ALGOS3 if not (name in OPEN3 and a[0] in ("npol", "nsol"))]


@pytest.mark.parametrize("name,algo,layout,tile", RUNS3)
@pytest.mark.parametrize("parts,align", [(2, 32), (3, 1)])
def test_d3q19_slabs_equal_the_undivided_box_fp32(name, algo, layout, tile, parts, align):
    T = 21
    kw = dict(algo=algo, layout=layout, storage="f32", tile=tile)
    _equal3(_run3(name, T, parts, align, **kw), _reference3(name, T, **kw))


@pytest.mark.parametrize("storage", ["f64", "f16s", "bf16s"])
@pytest.mark.parametrize("algo,layout", [("nptl", "bundle"), ("lptl", "stream"), ("nsol", "stream")])
def test_d3q19_slabs_equal_the_undivided_box_other_storage(storage, algo, layout):
    T = 17
    for name in ("spheres_periodic", "zou_he_pressure"):
        if name in OPEN3 and algo == "nsol":
            continue
        kw = dict(algo=algo, layout=layout, storage=storage, tile=(8, 4, 2) if algo == "nsol" else (0, 0, 0))
        _equal3(_run3(name, T, 4, 1, **kw), _reference3(name, T, **kw))


def test_d3q19_face_pack_moves_the_stored_bits():
    nx, ny, nz = 12, 6, 5
    as_type = {"f64": torch.float64, "f32": torch.float32, "f16s": torch.float16, "bf16s": torch.bfloat16}
    for storage, layout, algo in [("f32", "bundle", "nptl"), ("f16s", "collision", "nsol"), ("f64", "stream", "npol"),
                                  ("bf16s", "bundle", "lptl")]:
        tile = (4, 2, 2) if algo in ("npol", "nsol") else (0, 0, 0)
        a = lbm.Lattice3(nx, ny, nz, 0.8, None, storage=storage, layout=layout, algo=algo, tile=tile)
        a.init(*_fields3(nx, ny, nz, np.zeros(nx * ny * nz)))
        a.step(3).sync()
        b = lbm.Lattice3(nx, ny, nz, 0.8, None, storage=storage, layout=layout, algo=algo, tile=tile)
        b.init()
        b.step(3).sync()
        elem = S.ELEM_BYTES[storage]
        sent = {}
        for x, sense in [(0, 1), (nx - 1, -1), (5, 1), (5, -1)]:
            buf = torch.zeros(5 * ny * nz * elem, dtype=torch.uint8, device="cuda")
            a.face_pack(x, sense, buf)
            b.face_unpack(x, sense, buf)
            sent[(x, sense)] = buf
        a.sync()
        b.sync()
        pa = a.populations("f64").reshape(19, ny * nz, nx)
        pb = b.populations("f64").reshape(19, ny * nz, nx)
        cx = [0, -1, 0, 1, 0, -1, 0, 1, -1, 0, 1, -1, 0, 1, 0, -1, 0, 1, 0]  # D3Q19 order, c_x of each direction
        for (x, sense), buf in sent.items():
            dirs = [i for i in range(19) if cx[i] == sense]
            msg = buf.view(as_type[storage]).double().cpu().numpy().reshape(5, ny * nz)
            assert np.array_equal(msg, pa[dirs, :, x])
            assert np.array_equal(pa[dirs, :, x], pb[dirs, :, x])
        a.close()
        b.close()
    aa = lbm.Lattice3(nx, ny, nz, 0.8, None, algo="aa")
    aa.init()
    buf = torch.zeros(5 * ny * nz * 4, dtype=torch.uint8, device="cuda")
    with pytest.raises(lbm.LbmError) as e:
        aa.face_pack(3, 1, buf)
    assert e.value.status == lbm.LBM_EINVAL
    aa.close()
