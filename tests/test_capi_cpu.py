"""CPU checks of the C ABI: the library loads, exports every function that
include/*.h declares, and the host copy of each layout's index map is the
bijection Fig. 2 (Sec. 3.2) draws. No compute call needs a GPU here."""
import glob
import os
import re

import numpy as np
import pytest

from paper_2607_20650_gb300 import build, lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return lbm.load()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*[\s\*]+(lbm3?_[A-Za-z0-9_]+)\s*\(",
                             text, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_abi():
    names = declared_functions()
    for core in ("lbm_create", "lbm_step", "lbm_read_moments", "lbm_force", "lbm_mass",
                 "lbm_batch_create", "lbm_batch_step", "lbm3_create", "lbm3_step", "lbm3_mass"):
        assert core in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(declared_functions()) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(declared_functions()) <= set(lbm.SIGNATURES)


def test_layout_maps_match_fig1_and_are_bijections(lib):
    for nx, ny in [(1, 1), (3, 2), (7, 5)]:
        N = nx * ny
        for name in ("stream", "bundle", "collision"):
            offs = np.array([[lbm.lbm_layout_index(name, N, n, i) for n in range(N)] for i in range(9)])
            assert sorted(offs.ravel().tolist()) == list(range(9 * N)), name
            n = np.arange(N)
            for i in range(9):
                if name == "stream":
                    exp = i * N + n                        # SoA: one array per direction
                elif name == "collision":
                    exp = 9 * n + i                        # AoS: the nine values of a node together
                else:
                    exp = (i // 3) * 3 * N + 3 * n + i % 3  # SoAoS: bundles {SW,S,SE},{W,0,E},{NW,N,NE}
                assert (offs[i] == exp).all()
    assert lbm.lbm_layout_index("stream", 4, 4, 0) == -1
    assert lbm.lbm_layout_index("stream", 4, 0, 9) == -1


def test_bad_params_are_rejected_without_gpu(lib):
    p = lbm.make_params(16, 8, 0.4)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_workspace_bytes(p)
    assert e.value.status == lbm.LBM_EINVAL
    p = lbm.make_params(16, 8, 0.8, bc=(lbm.PERIODIC, lbm.WALL, lbm.PERIODIC, lbm.PERIODIC))
    with pytest.raises(lbm.LbmError):
        lbm.lbm_workspace_bytes(p)
    p = lbm.make_params(16, 8, 0.8, bc=(lbm.INLET_ZOUHE, lbm.INLET_ZOUHE, lbm.WALL, lbm.WALL))
    with pytest.raises(lbm.LbmError):
        lbm.lbm_workspace_bytes(p)
    p = lbm.make_params(16, 8, 0.8, tile=(64, 16), algo="npol")
    with pytest.raises(lbm.LbmError):
        lbm.lbm_workspace_bytes(p)


def test_workspace_sizes(lib):
    N = 100 * 60
    two = lbm.lbm_workspace_bytes(lbm.make_params(100, 60, 0.8, algo="nptl", storage="f32"))
    one = lbm.lbm_workspace_bytes(lbm.make_params(100, 60, 0.8, algo="npol", storage="f32"))
    half = lbm.lbm_workspace_bytes(lbm.make_params(100, 60, 0.8, algo="nptl", storage="f16s"))
    assert two >= 2 * 9 * N * 4 + N + 12 * N
    assert one < two - 9 * N * 4 + 9 * N * 4 // 2     # one lattice + a buffer grid well below a lattice
    assert half < two


def test_batch_planner_resolves_every_case(lib):
    from paper_2607_20650_gb300 import geometry as G
    cases = G.batch_channels(ncases=24, seed=4)
    ps = [lbm.make_params(w.nx, w.ny, w.tau, u_in=(w.ux_in, 0.0), bc=(w.bc_w, w.bc_e, w.bc_s, w.bc_n),
                          layout=lbm.LBM_AUTO, algo=lbm.LBM_AUTO, storage="f32") for w in cases]
    planned = lbm.lbm_batch_plan(ps)
    for w, p in zip(cases, planned):
        assert p.layout in (0, 1, 2) and p.algo in (0, 1, 2, 3)
        if p.algo != 0:
            assert 1 <= p.tile_x * p.tile_y <= 256
            # no shape in the candidate set pads this case less at the same cost class
            pad = -(-w.nx // p.tile_x) * -(-w.ny // p.tile_y) * 256 - w.nx * w.ny
            assert pad < 256 * (-(-w.nx // 32) + -(-w.ny // 8))
    # the built-in model prefers the bundle two-lattice pull (measured fastest)
    assert sum(p.layout == 1 for p in planned) == len(planned)
    fixed = [lbm.make_params(100, 40, 0.8, layout="stream", algo="npol", tile=(32, 8))]
    assert lbm.lbm_batch_plan(fixed)[0].algo == 2
    total = lbm.lbm_batch_workspace_bytes(planned)
    assert total > sum(lbm.lbm_workspace_bytes(p) for p in planned) - 1


def test_batch_rejects_unresolved_or_mixed(lib):
    a = lbm.make_params(64, 32, 0.8, layout=lbm.LBM_AUTO, algo="nptl")
    with pytest.raises(lbm.LbmError):
        lbm.lbm_batch_workspace_bytes([a])
    b = lbm.make_params(64, 32, 0.8, storage="f32")
    c = lbm.make_params(64, 32, 0.8, storage="f16s")
    with pytest.raises(lbm.LbmError):
        lbm.lbm_batch_workspace_bytes([b, c])
    d = lbm.make_params(64, 32, 0.8, algo="npol", tile=(32, 16))
    with pytest.raises(lbm.LbmError):
        lbm.lbm_batch_workspace_bytes([d])


def test_aa_rejects_outflow_without_gpu(lib):
    p = lbm.make_params(64, 32, 0.8, algo="aa", bc=(lbm.INLET_ZOUHE, lbm.OUTFLOW_ZG, lbm.WALL, lbm.WALL))
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_workspace_bytes(p)
    assert e.value.status == lbm.LBM_EUNSUPPORTED
    one = lbm.lbm_workspace_bytes(lbm.make_params(100, 60, 0.8, algo="aa"))
    two = lbm.lbm_workspace_bytes(lbm.make_params(100, 60, 0.8, algo="nptl"))
    assert one < two - 9 * 100 * 60 * 4 + 4096          # one lattice, no buffer grid


def test_d3q19_layout_maps_are_bijections_grouped_by_source_row(lib):
    """Bundle layout in 3-D: the directions that pull from one source row
    (equal c_y and c_z, derived here from the oracle's velocity table) are
    stored side by side per node, groups in direction order."""
    from oracle import directions3
    c, _ = directions3()
    for nx, ny, nz in [(1, 1, 1), (3, 2, 2), (5, 3, 4)]:
        N = nx * ny * nz
        n = np.arange(N)
        groups = {}
        for i in range(19):
            groups.setdefault((int(c[i, 1]), int(c[i, 2])), []).append(i)
        first = {i: g[0] for g in groups.values() for i in g}
        size = {i: len(g) for g in groups.values() for i in g}
        for name in ("stream", "bundle", "collision"):
            offs = np.array([[lbm.lbm3_layout_index(name, N, k, i) for k in range(N)] for i in range(19)])
            assert sorted(offs.ravel().tolist()) == list(range(19 * N)), name
            for i in range(19):
                if name == "stream":
                    exp = i * N + n
                elif name == "collision":
                    exp = 19 * n + i
                else:
                    exp = first[i] * N + size[i] * n + (i - first[i])
                assert (offs[i] == exp).all(), (name, i)
    assert lbm.lbm3_layout_index("bundle", 4, 0, 19) == -1


def test_d3q19_params_checked_without_gpu(lib):
    ok = lbm.lbm3_workspace_bytes(lbm.make_params3(16, 8, 4, 0.8, storage="f32"))
    assert ok >= 2 * 19 * 16 * 8 * 4 * 4
    assert lbm.lbm3_workspace_bytes(lbm.make_params3(16, 8, 4, 0.8, algo="nsol", tile=(8, 4, 2))) >= \
        19 * 16 * 8 * 4 * 4
    zh = (lbm.INLET_ZOUHE, lbm.WALL, lbm.PERIODIC)
    for bad in (dict(tau=0.5), dict(bc=(lbm.FREESLIP, lbm.PERIODIC, lbm.PERIODIC)),
                dict(algo="nsol", bc=zh, bc_x_east=lbm.OUTLET_PRESSURE), dict(tile=(32, 8, 4)),
                dict(bc=zh, bc_x_east=lbm.OUTLET_PRESSURE, rho_out=-1.0),
                dict(bc=zh, bc_x_east=lbm.INLET_ZOUHE)):
        kw = dict(tau=0.8)
        kw.update(bad)
        tau = kw.pop("tau")
        with pytest.raises(lbm.LbmError):
            lbm.lbm3_workspace_bytes(lbm.make_params3(16, 8, 4, tau, **kw))


def test_batch_planner_prefers_one_shared_pair(lib):
    """With a measured-style cost table under which a few small cases would
    pick another pair on their own, the plan still gives every case one
    layout and algorithm (the specialised batch kernel), unless a fixed case
    makes a shared pair impossible."""
    from paper_2607_20650_gb300 import geometry as G
    t = lbm.lbm_tuning()
    table = [[0.01849, 0.0173, 0.03252, 0.03291], [0.02043, 0.01809, 0.03251, 0.03486],
             [0.04423, 0.02434, 0.04927, 0.05439]]
    for l in range(3):
        for a in range(4):
            t.ns_per_cell[l][a] = table[l][a]
    t.ns_per_tile = 2.0
    t.valid = 1
    cases = G.batch_channels(ncases=64, seed=4)
    ps = [lbm.make_params(w.nx, w.ny, w.tau, u_in=(w.ux_in, 0.0), bc=(w.bc_w, w.bc_e, w.bc_s, w.bc_n),
                          layout=lbm.LBM_AUTO, algo=lbm.LBM_AUTO, storage="f32") for w in cases]
    planned = lbm.lbm_batch_plan(ps, t)
    assert len({(p.layout, p.algo) for p in planned}) == 1
    # one case pinned to NSOL: the others follow it only if that stays within the penalty
    pinned = [lbm.make_params(300, 100, 0.8, layout="collision", algo="nsol", tile=(32, 8))]
    mixed = lbm.lbm_batch_plan(pinned + ps[:8], t)
    assert (mixed[0].layout, mixed[0].algo) == (2, 3)
    assert all(p.layout in (0, 1, 2) and p.algo in (0, 1, 2, 3) for p in mixed)


def test_tune_workspace_covers_every_candidate(lib):
    probe = lbm.make_params(512, 256, 0.8, storage="f32")
    need = lbm.lbm_tune_workspace_bytes(probe)
    one = lbm.lbm_workspace_bytes(lbm.make_params(512, 256, 0.8, storage="f32", layout="collision",
                                                  algo="lptl"))
    assert need >= 8 * one


def test_d3q19_aa_is_one_lattice_and_needs_offset_tables(lib):
    two = lbm.lbm3_workspace_bytes(lbm.make_params3(32, 16, 8, 0.8, algo="nptl", storage="f32"))
    one = lbm.lbm3_workspace_bytes(lbm.make_params3(32, 16, 8, 0.8, algo="aa", storage="f32"))
    assert one <= two - 19 * 32 * 16 * 8 * 4 + 256
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm3_workspace_bytes(lbm.make_params3(32, 16, 8, 0.8, algo="aa",
                                                  flags=lbm.LBM_FLAG_WIDE_OFFSETS))
    assert e.value.status == lbm.LBM_EUNSUPPORTED


def test_d3q19_npol_is_one_lattice_plus_buffer_grid(lib):
    nx, ny, nz = 64, 32, 16
    two = lbm.lbm3_workspace_bytes(lbm.make_params3(nx, ny, nz, 0.8, algo="nptl", storage="f32"))
    one = lbm.lbm3_workspace_bytes(lbm.make_params3(nx, ny, nz, 0.8, algo="npol", storage="f32",
                                                    tile=(16, 4, 4)))
    # tiles 16x4x4: faces 16 + 64 + 64 nodes, 10 values per face node per parity
    tiles = (nx // 16) * (ny // 4) * (nz // 4)
    grid = 2 * tiles * 10 * (4 * 4 + 16 * 4 + 16 * 4) * 4
    assert two - 19 * nx * ny * nz * 4 + grid - 1024 <= one <= two - 19 * nx * ny * nz * 4 + grid + 1024


def test_d3q19_inlet_outflow_params(lib):
    ok = lbm.make_params3(32, 8, 8, 0.8, bc=(lbm.INLET_EQ, lbm.WALL, lbm.WALL), bc_x_east=lbm.OUTFLOW_ZG,
                          u_in=(0.05, 0.0, 0.0))
    assert lbm.lbm3_workspace_bytes(ok) > 0
    for bad in (dict(bc=(lbm.INLET_EQ, lbm.WALL, lbm.WALL), bc_x_east=lbm.PERIODIC),
                dict(bc=(lbm.WALL, lbm.INLET_EQ, lbm.WALL)),
                dict(bc=(lbm.FREESLIP, lbm.WALL, lbm.WALL))):
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm3_workspace_bytes(lbm.make_params3(32, 8, 8, 0.8, **bad))
        assert e.value.status == lbm.LBM_EINVAL
    for algo in ("aa", "npol"):
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm3_workspace_bytes(lbm.make_params3(32, 8, 8, 0.8, algo=algo,
                                                      bc=(lbm.OUTFLOW_ZG, lbm.WALL, lbm.WALL)))
        assert e.value.status == lbm.LBM_EUNSUPPORTED


def test_d3q19_batch_plan_checked_without_gpu(lib):
    a = lbm.make_params3(24, 16, 8, 0.8, algo="nptl", storage="f32", tile=(8, 4, 2))
    b = lbm.make_params3(40, 8, 12, 0.7, algo="nptl", storage="f32", tile=(8, 4, 2), force=(1e-6, 0, 0))
    total = lbm.lbm3_batch_workspace_bytes([a, b])
    assert total >= lbm.lbm3_workspace_bytes(a) + lbm.lbm3_workspace_bytes(b)
    # one record per case and one (case, item) pair per tile on top of the boxes
    assert total <= lbm.lbm3_workspace_bytes(a) + lbm.lbm3_workspace_bytes(b) + 64 * 1024
    for algo in ("lptl", "npol", "nsol"):
        assert lbm.lbm3_batch_workspace_bytes([lbm.make_params3(24, 16, 8, 0.8, algo=algo, tile=(8, 4, 2))]) > 0
    bad = [
        ([a, lbm.make_params3(24, 16, 8, 0.8, algo="nptl", storage="f16s", tile=(8, 4, 2))], lbm.LBM_EINVAL),
        ([a, lbm.make_params3(24, 16, 8, 0.8, algo="nptl", storage="f32", tile=(8, 2, 4))], lbm.LBM_EINVAL),
        ([a, lbm.make_params3(24, 16, 8, 0.8, algo="lptl", storage="f32")], lbm.LBM_EINVAL),
        ([a, lbm.make_params3(24, 16, 8, 0.8, algo="nptl", storage="f32", layout="bundle",
                              tile=(8, 4, 2))], lbm.LBM_EINVAL),
        ([lbm.make_params3(24, 16, 8, 0.8, algo="aa", tile=(8, 4, 2))], lbm.LBM_EUNSUPPORTED),
        ([lbm.make_params3(24, 16, 8, 0.8, algo="nptl", tile=(8, 4, 2), flags=lbm.LBM_FLAG_WIDE_OFFSETS)],
         lbm.LBM_EUNSUPPORTED),
        ([], lbm.LBM_EINVAL),
    ]
    for params, status in bad:
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm3_batch_workspace_bytes(params)
        assert e.value.status == status


def test_flag_constants_match_header():
    """Every LBM_FLAG_* of include/lbm.h has the same value in the binding."""
    import re
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    flags = dict(re.findall(r"#define (LBM_FLAG_\w+) (0x[0-9a-fA-F]+)u", text))
    assert {"LBM_FLAG_NO_GRAPH", "LBM_FLAG_NO_PREFETCH", "LBM_FLAG_WIDE_OFFSETS"} <= set(flags)
    for name, value in flags.items():
        assert getattr(lbm, name) == int(value, 16), name


# ---------------------------------------------------------------- host mask generator

def test_c_mask_generator_matches_the_python_input_generator(lib):
    """The C ABI's host mask generator and the package's Python input
    generator draw the same splitmix64 streams and apply the same
    double-precision tests, so the seeded masks agree bit for bit."""
    from paper_2607_20650_gb300 import geometry as G
    for nx, ny, seed in ((300, 170, 21), (512, 256, 3), (97, 61, 5)):
        assert np.array_equal(lbm.lbm_mask_porous_discs(nx, ny, seed, 4.0, 9.0, 0.3),
                              G.porous_discs(nx, ny, seed, rmin=4, rmax=9, solid_fraction=0.3))
    assert np.array_equal(lbm.lbm_mask_porous_discs(1024, 512, 3), G.porous_discs(1024, 512, 3))
    assert np.array_equal(lbm.lbm_mask_channel_walls(256, 64), G.channel_walls(256, 64))
    for periodic in (False, True):
        assert np.array_equal(lbm.lbm_mask_disc(96, 40, 3.5, 20.0, 6.5, periodic),
                              G.disc(96, 40, 3.5, 20.0, 6.5, periodic=periodic))
    assert np.array_equal(lbm.lbm3_mask_porous_spheres(40, 36, 30, 3, 2.0, 5.0, 0.25),
                          G.porous_spheres(40, 36, 30, 3, 2.0, 5.0, 0.25))
    # the wing: transcendental functions of two libraries may differ in the
    # last place, which can move a node lying on the outline
    c = lbm.lbm_mask_naca4(2048, 1024, 256.0)
    p = G.naca_wing(2048, 1024, 256.0)
    assert int(p.sum()) > 0.06 * 256 * 256 * 0.12 and np.count_nonzero(c != p) <= 4


def test_c_mask_generator_rejects_bad_arguments(lib):
    for call in (lambda: lbm.lbm_mask_porous_discs(0, 8, 1), lambda: lbm.lbm_mask_porous_discs(8, 8, 1, 5.0, 4.0),
                 lambda: lbm.lbm_mask_porous_discs(8, 8, 1, 1.0, 2.0, 1.0),
                 lambda: lbm.lbm_mask_naca4(64, 32, -1.0), lambda: lbm.lbm3_mask_porous_spheres(4, 4, 0, 1)):
        with pytest.raises(lbm.LbmError) as e:
            call()
        assert e.value.status == lbm.LBM_EINVAL


def test_face_exchange_argument_errors_need_no_gpu(lib):
    """The face calls check their arguments before any device work (include/lbm.h)."""
    import ctypes
    for fn in (lib.lbm_face_pack, lib.lbm_face_unpack, lib.lbm3_face_pack, lib.lbm3_face_unpack):
        assert fn(None, 0, 1, None) == lbm.LBM_EINVAL
    one = (ctypes.c_int32 * 1)(0)
    for fn in (lib.lbm_face_exchange, lib.lbm3_face_exchange):
        assert fn(0, None, None, None, None, None, None) == lbm.LBM_OK        # nothing to exchange
        assert fn(-1, None, None, None, None, None, None) == lbm.LBM_EINVAL
        assert fn(65, None, None, None, None, None, None) == lbm.LBM_EINVAL  # more than 64 messages
        assert fn(1, None, one, None, one, one, None) == lbm.LBM_EINVAL      # NULL lattice arrays
        hs = (ctypes.c_void_p * 1)(None)
        assert fn(1, hs, one, hs, one, one, None) == lbm.LBM_EINVAL          # NULL lattices
