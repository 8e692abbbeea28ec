"""The x-slab decomposition on the CPU: the split and its message plan, the
plan run on the FP64 oracle (slabs updated one at a time, the face messages
copied between them) against the undivided oracle lattice bit for bit, and
the rank-to-rank transport of the messages over gloo process groups of two
and three ranks."""
import os
import socket

import numpy as np
import pytest

import oracle as O
from paper_2607_20650_gb300 import geometry as G
from paper_2607_20650_gb300 import slabs as S


# ---------------------------------------------------------------- the plan

@pytest.mark.parametrize("align", [1, 8, 32])
@pytest.mark.parametrize("nx,parts,periodic", [(10, 1, True), (10, 1, False), (11, 2, True), (11, 2, False),
                                               (17, 3, True), (17, 3, False), (8, 4, True), (40, 5, False)])
def test_split_covers_the_columns_and_every_ghost_gets_one_message(nx, parts, periodic, align):
    sl = S.split(nx, parts, periodic, align)
    assert [s.x0 for s in sl] == [0] + [s.x1 for s in sl[:-1]] and sl[-1].x1 == nx
    widths = [s.width for s in sl]
    assert min(widths) >= 2 and max(widths) - min(widths) <= 1
    msgs = S.messages(sl, periodic)
    got = {}
    for src, xs, dst, xd, sense in msgs:
        a, b = sl[src], sl[dst]
        assert a.interior.start <= xs < a.interior.stop           # sent from an interior column
        assert not (b.interior.start <= xd < b.interior.stop)     # into a ghost column
        col_a = a.columns(nx)[xs - a.pw]
        col_b = b.columns(nx)[xd - b.pw]
        assert col_a == col_b                                     # both stand for the same column
        assert sense == (S.EAST_GOING if xd == b.first - 1 else S.WEST_GOING)
        got[(dst, xd)] = got.get((dst, xd), 0) + 1
    ghosts = {(s.index, s.first - 1) for s in sl if s.gw} | {(s.index, s.first + s.width) for s in sl if s.ge}
    assert got == {g: 1 for g in ghosts}
    for s in sl:
        # padding only beyond a ghost column, and rows a multiple of align
        assert s.pw == 0 or s.gw
        assert s.pe == 0 or s.ge
        assert parts == 1 or s.nx % align == 0
        if not s.gw:
            assert s.first == 0
        if not s.ge:
            assert s.nx == s.first + s.width
    if parts == 1:
        assert msgs == [] and sl[0].nx == nx


def test_split_rejects_slabs_narrower_than_two_columns():
    with pytest.raises(ValueError):
        S.split(7, 4, False)
    with pytest.raises(ValueError):
        S.split(5, 0, True)


def test_layout_offsets_are_affine_in_the_node_index():
    """The face kernels address population slot i of node n as
    base(i) + n * stride in all three layouts (Fig. 2)."""
    from paper_2607_20650_gb300 import build, lbm
    build.build()
    for N in (6, 35):
        for name in ("stream", "bundle", "collision"):
            stride = lbm.lbm_layout_index(name, N, 1, 0) - lbm.lbm_layout_index(name, N, 0, 0)
            for i in range(9):
                base = lbm.lbm_layout_index(name, N, 0, i)
                assert [lbm.lbm_layout_index(name, N, n, i) for n in range(N)] == \
                    [base + n * stride for n in range(N)], (name, i)


def test_decomposition_rejects_what_it_cannot_split_before_any_device_work():
    pytest.importorskip("torch")
    with pytest.raises(ValueError):
        S.Decomposition(32, 8, 0.8, None, parts=2, algo="aa")            # two forms of the state
    with pytest.raises(ValueError):
        S.Decomposition(32, 8, 0.8, None, parts=17)                      # slabs narrower than 2 columns
    with pytest.raises(ValueError):
        S.Decomposition(12, 8, 0.8, None, nz=4, parts=7, bc=(O.PERIODIC,) * 3)


def test_ghost_faces_of_3d_slabs():
    """A slab without ghosts keeps the box's x faces; ghost faces of periodic
    or walled boxes become walls; inlet / outlet boxes keep their kinds."""
    one = S.split(12, 1, True)[0]
    assert S.edges3(one, (O.PERIODIC, O.WALL, O.PERIODIC), O.OUTFLOW_ZG)[:3] == (O.PERIODIC, O.WALL, O.PERIODIC)
    for sl in S.split(12, 3, True, 4):
        assert S.edges3(sl, (O.PERIODIC, O.PERIODIC, O.WALL), O.OUTFLOW_ZG)[:3] == (O.WALL, O.PERIODIC, O.WALL)
    for sl in S.split(12, 3, False):
        assert S.edges3(sl, (O.INLET_ZOUHE, O.WALL, O.WALL), O.OUTLET_PRESSURE) == \
            (O.INLET_ZOUHE, O.WALL, O.WALL, O.OUTLET_PRESSURE)


# ---------------------------------------------------------------- the plan on the oracle

P, W = O.PERIODIC, O.WALL


def _case(name):
    nx, ny = 30, 16
    if name == "porous_periodic":
        return nx, ny, G.porous_discs(nx, ny, seed=4, rmin=2, rmax=4, solid_fraction=0.3), (P, P, P, P), \
            dict(fx=2e-5, fy=-5e-6)
    if name == "zou_he_outflow":
        return nx, ny, G.disc(nx, ny, 15.0, 8.0, 3.5), (O.INLET_ZOUHE, O.OUTFLOW_ZG, W, W), dict(ux_in=0.04)
    if name == "neumann_pressure":
        return nx, ny, G.disc(nx, ny, 11.0, 7.0, 3.0), (O.INLET_EQ_NEUMANN, O.OUTLET_PRESSURE, W, W), \
            dict(ux_in=0.03, rho_out=0.995)
    return nx, ny, G.porous_discs(nx, ny, seed=8, rmin=2, rmax=3, solid_fraction=0.25), (W, W, W, W), \
        dict(fx=1e-5, fy=3e-6)


def _fields(nx, ny, mask):
    r = G.SplitMix64(21, 3)
    rho = 1.0 + np.asarray(r.uniform(nx * ny, -0.01, 0.01))
    ux = np.asarray(r.uniform(nx * ny, -0.03, 0.03))
    uy = np.asarray(r.uniform(nx * ny, -0.03, 0.03))
    solid = np.asarray(mask).reshape(-1) > 0
    ux[solid] = 0.0
    uy[solid] = 0.0
    return rho, ux, uy


@pytest.mark.parametrize("name,parts,align", [("porous_periodic", 2, 1), ("porous_periodic", 3, 8),
                                              ("zou_he_outflow", 3, 1), ("zou_he_outflow", 2, 16),
                                              ("neumann_pressure", 2, 1), ("neumann_pressure", 3, 8),
                                              ("walls_force", 4, 1), ("walls_force", 3, 32)])
def test_slab_plan_on_the_oracle_is_bit_identical(name, parts, align):
    """Slabs with the split's ghost and padding columns, masks and edges, each
    updated by the oracle and given the plan's face messages after every
    update, hold exactly the undivided lattice's state and moments."""
    nx, ny, mask, bc, extra = _case(name)
    T = 25
    periodic = bc[0] == P and bc[1] == P
    rho, ux, uy = _fields(nx, ny, mask)
    full = O.Lattice(O.Case(nx, ny, 0.8, bc_w=bc[0], bc_e=bc[1], bc_s=bc[2], bc_n=bc[3], **extra),
                     mask, rho, ux, uy).run(T)
    sl = S.split(nx, parts, periodic, align)
    lats = []
    for s in sl:
        e = s.edges(bc)
        case = O.Case(s.nx, ny, 0.8, bc_w=e[0], bc_e=e[1], bc_s=e[2], bc_n=e[3], **extra)
        lats.append(O.Lattice(case, s.local(mask, nx, 1), *[s.local(a, nx, 0.0) for a in (rho, ux, uy)]))
    msgs = S.messages(sl, periodic)
    for _ in range(T):
        for lat in lats:
            lat.run(1)
        for src, xs, dst, xd, sense in msgs:
            dirs = [3 * k + sense + 1 for k in range(3)]
            a = lats[src].h.reshape(9, ny, sl[src].nx)
            b = lats[dst].h.reshape(9, ny, sl[dst].nx)
            b[dirs, :, xd] = a[dirs, :, xs]
    fh = full.h.reshape(9, ny, nx)
    for s, lat in zip(sl, lats):
        assert np.array_equal(lat.h.reshape(9, ny, s.nx)[:, :, s.interior], fh[:, :, s.x0:s.x1]), s
        for a, b in ((lat.rho, full.rho), (lat.ux, full.ux), (lat.uy, full.uy)):
            assert np.array_equal(a.reshape(ny, s.nx)[:, s.interior], b.reshape(ny, nx)[:, s.x0:s.x1])
    assert np.all(np.isfinite(full.h)) and np.abs(full.ux).max() > 1e-4


# ---------------------------------------------------------------- the plan on the 3-D oracle

def _case3(name):
    nx, ny, nz = 20, 8, 6
    if name == "spheres_periodic":
        return nx, ny, nz, G.porous_spheres(nx, ny, nz, 5, 1.5, 2.5, 0.25), (P, P, P), dict(fx=2e-5, fy=-4e-6), {}
    if name == "walls_force":
        return nx, ny, nz, G.porous_spheres(nx, ny, nz, 7, 1.5, 2.5, 0.2), (W, P, W), dict(fx=1e-5, fz=3e-6), {}
    if name == "zou_he_pressure":
        return nx, ny, nz, G.ball(nx, ny, nz, 9.0, 4.0, 3.0, 2.2), (O.INLET_ZOUHE, W, W), {}, \
            dict(bc_xe=O.OUTLET_PRESSURE, u_in=(0.04, 0.0, 0.0), rho_out=0.997)
    return nx, ny, nz, G.ball(nx, ny, nz, 11.0, 4.0, 3.0, 2.0), (O.INLET_EQ, P, W), {}, \
        dict(bc_xe=O.OUTFLOW_ZG, u_in=(0.03, 0.0, 0.0))


@pytest.mark.parametrize("name,parts,align", [("spheres_periodic", 2, 1), ("spheres_periodic", 3, 8),
                                              ("walls_force", 3, 1), ("zou_he_pressure", 2, 8),
                                              ("zou_he_pressure", 3, 1), ("eq_outflow", 2, 1)])
def test_slab_plan_on_the_3d_oracle_is_bit_identical(name, parts, align):
    """D3Q19 boxes split into x-slabs with the plan's ghost planes, masks and
    x faces, each updated by the 3-D oracle and given the five crossing
    populations per face node after every update, equal the undivided box."""
    nx, ny, nz, mask, bc, force, xface = _case3(name)
    T = 18
    rows = ny * nz
    r = G.SplitMix64(9, 4)
    rho = 1.0 + r.uniform(nx * rows, -0.01, 0.01)
    u = [r.uniform(nx * rows, -0.02, 0.02) for _ in range(3)]
    for a in u:
        a[np.asarray(mask).reshape(-1) > 0] = 0.0
    full = O.Lattice3(O.Case3(nx, ny, nz, 0.8, bc_x=bc[0], bc_y=bc[1], bc_z=bc[2], **force, **xface),
                      mask, rho, *u).run(T)
    periodic = bc[0] == P
    sl = S.split(nx, parts, periodic, align)
    c, _ = O.directions3()
    lats = []
    for s in sl:
        bx, by, bz, bxe = S.edges3(s, bc, xface.get("bc_xe", O.OUTFLOW_ZG))
        extra = dict(xface, bc_xe=bxe) if bx in (O.INLET_EQ, O.INLET_ZOUHE) else {}
        case = O.Case3(s.nx, ny, nz, 0.8, bc_x=bx, bc_y=by, bc_z=bz, **force, **extra)
        lats.append(O.Lattice3(case, s.local(mask, nx, 1), *[s.local(a, nx, 0.0) for a in (rho, *u)]))
    for _ in range(T):
        for lat in lats:
            lat.run(1)
        for src, xs, dst, xd, sense in S.messages(sl, periodic):
            dirs = [i for i in range(19) if c[i, 0] == sense]
            assert len(dirs) == 5
            a = lats[src].h.reshape(19, rows, sl[src].nx)
            b = lats[dst].h.reshape(19, rows, sl[dst].nx)
            b[dirs, :, xd] = a[dirs, :, xs]
    fh = full.h.reshape(19, rows, nx)
    for s, lat in zip(sl, lats):
        assert np.array_equal(lat.h.reshape(19, rows, s.nx)[:, :, s.interior], fh[:, :, s.x0:s.x1]), s
        for a, b in ((lat.rho, full.rho), (lat.ux, full.ux), (lat.uz, full.uz)):
            assert np.array_equal(a.reshape(rows, s.nx)[:, s.interior], b.reshape(rows, nx)[:, s.x0:s.x1])
    assert np.all(np.isfinite(full.h)) and np.abs(full.ux).max() > 1e-4


# ---------------------------------------------------------------- the transport

def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _payload(k, nbytes):
    return np.frombuffer(np.random.default_rng(1000 + k).bytes(nbytes), np.uint8).copy()


def _rank(rank, world, port, periodic, q):
    import datetime

    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=120))
    try:
        nbytes = 3 * 24 * 4
        msgs = S.messages(S.split(6 * world, world, periodic), periodic)
        sends, recvs, want = [], [], {}
        for k, (src, _, dst, _, sense) in enumerate(msgs):
            if src == rank and dst != rank:
                sends.append((dst, sense, torch.from_numpy(_payload(k, nbytes))))
            if dst == rank and src != rank:
                t = torch.zeros(nbytes, dtype=torch.uint8)
                recvs.append((src, sense, t))
                want[k] = t
        for _ in range(3):  # repeated exchanges reuse the same tags
            S.exchange_host(sends, recvs)
        ok = all(np.array_equal(t.numpy(), _payload(k, nbytes)) for k, t in want.items())
        q.put((rank, ok, len(recvs)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,periodic", [(2, True), (2, False), (3, True), (3, False)])
def test_face_messages_cross_gloo_ranks(world, periodic):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, periodic, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
    for p in procs:
        if p.is_alive():
            p.terminate()
            p.join(30)
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(q.get(timeout=5) for _ in range(world))
    assert all(ok for _, ok, _ in res)
    # ghosts per rank: two on a periodic lattice, one at the ends of an open one
    assert [n for _, _, n in res] == ([2] * world if periodic else [1] + [2] * (world - 2) + [1])
