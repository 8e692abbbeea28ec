"""D3Q19 lattices (the 3-D extension of Sec. 6) through the lbm3_* C ABI,
against the FP64 D3Q19 oracle.

Bars:
  * FP64 GPU vs FP64 oracle: relative L-inf <= 1e-12 on populations and
    velocities, 1e-14 on density (rounding order only).
  * Every layout x algorithm x tile shape: bit-identical at equal storage.
  * omega = 0: bit-exact cyclic shift by T c_i.
  * A z-invariant D3Q19 flow summed over c_z is the D2Q9 update: checked
    against the 2-D oracle.
  * Full size (4.6 M nodes, FP32): sampled nodes against the oracle run on
    their 3x3x3 neighbourhood, which determines one update exactly.
"""
import math

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
ALGOS = ("lptl", "nptl")
P, W = lbm.PERIODIC, lbm.WALL


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2607_20650_gb300 import build
    build.build()
    lbm.load()


class Spec3:
    def __init__(self, nx, ny, nz, tau, mask, bc, force=(0.0, 0.0, 0.0), seed=1, amp=0.02):
        self.nx, self.ny, self.nz, self.tau = nx, ny, nz, tau
        self.mask = np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
        self.bc, self.force = bc, force
        N = nx * ny * nz
        r = G.SplitMix64(seed, 11)
        solid = self.mask > 0
        self.rho0 = np.where(solid, 1.0, 1.0 + r.uniform(N, -0.01, 0.01))
        self.u0 = [np.where(solid, 0.0, r.uniform(N, -amp, amp)) for _ in range(3)]

    def oracle(self):
        c = O.Case3(self.nx, self.ny, self.nz, self.tau, *self.force, *self.bc)
        return O.Lattice3(c, self.mask, self.rho0, *self.u0)

    def gpu(self, **kw):
        lat = lbm.Lattice3(self.nx, self.ny, self.nz, self.tau, self.mask, force=self.force,
                           bc=self.bc, **kw)
        lat.init(self.rho0, *self.u0)
        return lat


def specs():
    out = {}
    nx, ny, nz = 37, 21, 13
    out["porous"] = Spec3(nx, ny, nz, 0.7, G.porous_spheres(nx, ny, nz, 5, 2.0, 5.0, 0.25), (P, P, P),
                          force=(1e-5, 2e-6, -1e-6))
    nx, ny, nz = 45, 19, 11
    out["duct"] = Spec3(nx, ny, nz, 0.9, G.ball(nx, ny, nz, 12.0, 9.0, 5.0, 3.5), (P, W, W),
                        force=(1e-5, 0.0, 0.0), seed=2)
    nx, ny, nz = 33, 5, 3
    m = np.zeros((nz, ny, nx), np.uint8)
    m[1, 2, 7] = 1
    out["ragged"] = Spec3(nx, ny, nz, 0.6, m, (W, P, W), seed=3)
    return out


SPECS = specs()


@pytest.mark.parametrize("case", list(SPECS))
@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("algo", ALGOS + ("nptl_wide", "npol", "npol_wide", "nsol", "nsol_spanx"))
def test_fp64_matches_oracle3(case, layout, algo):
    spec = SPECS[case]
    T = 40
    ref = spec.oracle().run(T)
    flags = lbm.LBM_FLAG_WIDE_OFFSETS if algo.endswith("_wide") else 0
    # nsol_spanx: one tile spans the whole x axis (64 >= nx), so periodic x
    # pulls wrap inside the tile
    tile = (64, 2, 3) if algo == "nsol_spanx" else ((8, 4, 3) if algo.startswith(("npol", "nsol")) else (0, 0, 0))
    lat = spec.gpu(layout=layout, algo=algo.split("_")[0], storage="f64", flags=flags, tile=tile)
    lat.step(T, moments=True).sync()
    h = lat.populations("f64")
    rho, ux, uy, uz = lat.moments()
    fl = ref.solid == 0
    assert rel_linf(h, ref.h, fl) <= 1e-12
    assert rel_linf(rho, ref.rho, fl) <= 1e-14
    assert rel_linf(np.stack([ux, uy, uz]), np.stack([ref.ux, ref.uy, ref.uz]), fl) <= 1e-12
    assert np.all(h[:, ~fl] == 0.0)
    assert np.all(rho[~fl] == 1.0) and np.all(ux[~fl] == 0.0) and np.all(uz[~fl] == 0.0)
    assert abs(lat.mass() - np.sum(1.0 + ref.h[:, fl].sum(axis=0))) <= 1e-13 * fl.sum()
    info = lat.info()
    assert info["fluid_cells"] == int(fl.sum()) and info["steps"] == T
    lat.close()


@pytest.mark.parametrize("storage,rounding", [("f64", "rne"), ("f32", "rne"), ("f16s", "rne"),
                                              ("f16s", "sr"), ("bf16s", "rne"), ("bf16s", "sr")])
def test_all_layouts_algorithms_and_tiles_bit_identical(storage, rounding):
    spec = SPECS["porous"]
    T = 70   # one graph of 64 updates plus single launches
    base = None
    for layout in LAYOUTS:
        for algo, tile, flags in (("lptl", (0, 0, 0), 0), ("nptl", (32, 4, 2), 0), ("nptl", (8, 8, 8), 0),
                                  ("nptl", (16, 2, 1), 0), ("lptl", (0, 0, 0), lbm.LBM_FLAG_WIDE_OFFSETS),
                                  ("nptl", (128, 1, 1), lbm.LBM_FLAG_WIDE_OFFSETS),
                                  ("npol", (8, 4, 2), 0), ("npol", (16, 2, 3), 0), ("npol", (64, 1, 1), 0),
                                  ("nsol", (8, 4, 2), 0), ("nsol", (16, 2, 3), 0), ("nsol", (64, 1, 1), 0),
                                  ("nsol", (4, 21, 2), 0)):
            lat = spec.gpu(layout=layout, algo=algo, tile=tile, storage=storage, rounding=rounding,
                           seed=99, flags=flags)
            lat.step(T, moments=True).sync()
            got = (lat.populations("f64"), *lat.moments())
            lat.close()
            if base is None:
                base = got
            else:
                for a, b in zip(got, base):
                    assert np.array_equal(a, b, equal_nan=False), (layout, algo, tile, flags)


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("algo", ALGOS + ("npol", "nsol"))
@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_pure_streaming_is_bit_exact_shift3(layout, algo, storage):
    nx, ny, nz, T = 23, 9, 7, 5
    N = nx * ny * nz
    rng = np.random.default_rng(4)
    h0 = rng.normal(0.0, 0.01, size=(19, N))
    if storage == "f32":
        h0 = h0.astype(np.float32).astype(np.float64)
    lat = lbm.Lattice3(nx, ny, nz, math.inf, None, layout=layout, algo=algo, storage=storage,
                       tile=(8, 4, 2))
    lat.write_populations(h0)
    lat.step(T).sync()
    h = lat.populations("f64")
    c, _ = O.directions3()
    for i in range(19):
        exp = np.roll(h0[i].reshape(nz, ny, nx), (T * c[i, 2], T * c[i, 1], T * c[i, 0]),
                      axis=(0, 1, 2)).ravel()
        assert np.array_equal(h[i], exp), i
    lat.close()


def test_fp32_close_to_oracle3():
    """FP32 arithmetic and storage after 200 updates: relative L-inf error on
    rho and v below 1e-5, the bar the 2-D path meets."""
    spec = SPECS["duct"]
    T = 200
    ref = spec.oracle().run(T)
    lat = spec.gpu(layout="bundle", algo="nptl", storage="f32")
    lat.step(T, moments=True).sync()
    rho, ux, uy, uz = lat.moments()
    fl = ref.solid == 0
    assert rel_linf(rho, ref.rho, fl) <= 1e-5
    assert rel_linf(np.stack([ux, uy, uz]), np.stack([ref.ux, ref.uy, ref.uz]), fl) <= 1e-5
    lat.close()


def test_z_invariant_flow_projects_to_d2q9_oracle():
    """Summing a z-invariant D3Q19 state over c_z gives D2Q9 populations with
    the D2Q9 weights (4/9, 1/9, 1/36), and one D3Q19 update of the state is
    one D2Q9 update of the sum: checked against the 2-D oracle."""
    nx, ny, nz, T = 29, 17, 4, 30
    m2 = G.disc(nx, ny, 10.0, 8.0, 3.0)
    r = G.SplitMix64(8, 3)
    ux0 = np.where(m2.ravel() > 0, 0.0, r.uniform(nx * ny, -0.02, 0.02))
    uy0 = np.where(m2.ravel() > 0, 0.0, r.uniform(nx * ny, -0.02, 0.02))
    force = (2e-5, -1e-5)
    ref = O.Lattice(O.Case(nx, ny, 0.8, fx=force[0], fy=force[1], bc_w=P, bc_e=P, bc_s=W, bc_n=W),
                    m2, ux=ux0, uy=uy0).run(T)
    m3 = np.broadcast_to(m2.reshape(1, ny, nx), (nz, ny, nx)).copy()
    lat = lbm.Lattice3(nx, ny, nz, 0.8, m3, force=(*force, 0.0), bc=(P, W, P), storage="f64",
                       layout="bundle", algo="nptl")
    lat.init(None, np.tile(ux0, nz), np.tile(uy0, nz), None)
    lat.step(T, moments=True).sync()
    h3 = lat.populations("f64").reshape(19, nz, ny * nx)
    c, _ = O.directions3()
    h2 = np.zeros((9, ny * nx))
    for i in range(19):
        j = (c[i, 1] + 1) * 3 + (c[i, 0] + 1)   # D2Q9 index of (c_x, c_y)
        h2[j] += h3[i, 0]
    assert np.all(h3 == h3[:, :1])                # stays z-invariant, bit for bit
    fl = ref.solid == 0
    assert rel_linf(h2, ref.h, fl) <= 1e-12
    rho, ux, uy, uz = lat.moments()
    assert rel_linf(ux[: nx * ny], ref.ux, fl) <= 1e-12
    # v_z sums the c_z = +1 values minus the c_z = -1 ones in direction order:
    # equal pairs cancel only up to the rounding of the partial sums
    assert np.max(np.abs(uz)) <= 1e-14 * np.max(np.abs(ux))
    lat.close()


def _effective_solid(mask3, bc):
    """Solid mask plus fluid nodes whose 18 pulls all bounce (any size; numpy)."""
    c, _ = O.directions3()
    solid = mask3 > 0
    nz, ny, nx = mask3.shape
    open_ = np.zeros_like(solid)
    for i in range(19):
        if i == 9:
            continue
        src = np.roll(solid, (c[i, 2], c[i, 1], c[i, 0]), axis=(0, 1, 2))  # solid[r - c_i]
        ok = ~src
        for a, (ext, shape_axis) in enumerate(((nx, 2), (ny, 1), (nz, 0))):
            if bc[a] == W and c[i, a] != 0:
                edge = [slice(None)] * 3
                edge[shape_axis] = 0 if c[i, a] > 0 else ext - 1
                ok[tuple(edge)] = False
        open_ |= ok
    return solid | ~open_


def test_full_size_sampled_nodes_match_oracle_neighbourhood():
    """4.6 M-node porous box, FP32 bundle NPTL: after 3 updates, one further
    update of sampled nodes equals the oracle's update of their 3x3x3
    neighbourhood (decoded FP32 state, effective solid flags of the whole
    lattice) within FP32 rounding; NPTL, LPTL and the collision layout agree
    bit for bit at this size."""
    nx, ny, nz = 192, 160, 150
    N = nx * ny * nz
    mask = G.porous_spheres(nx, ny, nz, 7, 3.0, 9.0, 0.3)
    bc = (P, P, W)
    force = (1e-5, 0.0, 0.0)
    kw = dict(force=force, bc=bc, storage="f32")
    lat = lbm.Lattice3(nx, ny, nz, 0.8, mask, layout="bundle", algo="nptl", **kw)
    r = G.SplitMix64(12, 1)
    u0 = [np.where(mask.ravel() > 0, 0.0, r.uniform(N, -0.03, 0.03)) for _ in range(3)]
    lat.init(None, *u0).step(3).sync()
    h3 = lat.populations("f64")
    lat.step(1, moments=True).sync()
    h4 = lat.populations("f64")
    other = {}
    for layout, algo in (("bundle", "lptl"), ("collision", "nptl"), ("stream", "nptl")):
        o = lbm.Lattice3(nx, ny, nz, 0.8, mask, layout=layout, algo=algo, **kw)
        o.init(None, *u0).step(4).sync()
        other[(layout, algo)] = o.populations("f32")
        o.close()
    for key, v in other.items():
        assert np.array_equal(v.astype(np.float64), h4), key
    eff = _effective_solid(mask, bc)
    rs = G.SplitMix64(13, 2)
    xs, ys, zs = rs.integers(64, 0, nx - 1), rs.integers(64, 0, ny - 1), rs.integers(64, 0, nz - 1)
    checked = 0
    for x, y, z in zip(xs, ys, zs):
        x, y, z = int(x), int(y), int(z)
        if eff[z, y, x]:
            continue
        zi = [(z + d) for d in (-1, 0, 1)]
        if any(q < 0 or q >= nz for q in zi):
            continue   # the oracle box would wrap a wall axis: sample interior planes only
        yi = [(y + d) % ny for d in (-1, 0, 1)]
        xi = [(x + d) % nx for d in (-1, 0, 1)]
        sub_m = eff[np.ix_(zi, yi, xi)].astype(np.uint8)
        idx = (np.array(zi)[:, None, None] * ny + np.array(yi)[None, :, None]) * nx + np.array(xi)[None, None, :]
        sub_h = h3[:, idx.ravel()]
        ref = O.Lattice3(O.Case3(3, 3, 3, 0.8, *force, P, P, P), sub_m)
        ref.set_h(sub_h)
        ref.run(1)
        n = (z * ny + y) * nx + x
        got, exp = h4[:, n], ref.h[:, 13]
        assert np.max(np.abs(got - exp)) <= 2e-6 * max(np.max(np.abs(exp)), 1e-3), (x, y, z)
        checked += 1
    assert checked >= 20
    lat.close()


def test_graphs_match_single_launches3():
    spec = SPECS["duct"]
    a = spec.gpu(layout="stream", algo="nptl", storage="f32")
    b = spec.gpu(layout="stream", algo="nptl", storage="f32", flags=lbm.LBM_FLAG_NO_GRAPH)
    a.step(130).step(3, moments=True).sync()
    b.step(133, moments=True).sync()
    assert np.array_equal(a.populations("f32"), b.populations("f32"))
    assert all(np.array_equal(u, v) for u, v in zip(a.moments(), b.moments()))
    a.close()
    b.close()


def test_divergence_is_reported3():
    spec = SPECS["ragged"]
    lat = lbm.Lattice3(spec.nx, spec.ny, spec.nz, 0.51, spec.mask, bc=spec.bc, storage="f32",
                       layout="collision", algo="lptl")
    h = np.zeros((19, spec.nx * spec.ny * spec.nz))
    h[3, 5] = np.inf
    lat.write_populations(h)
    with pytest.raises(lbm.LbmError) as e:
        lat.step(2).sync()
    assert e.value.status == lbm.LBM_EDIVERGED
    lat.write_populations(np.zeros_like(h))   # the report cleared the flag; the lattice stays usable
    lat.step(1).sync()
    lat.close()


@pytest.mark.parametrize("storage", ["f32", "f64"])
def test_momentum_conserved_over_long_runs3(storage):
    """As in 2-D: a sheared uniform flow in a periodic box keeps its total
    momentum up to rounding noise over 10,000 updates (a momentum source
    from rounded FP32 weights would move it by ~1.5e-4)."""
    nx, ny, nz, T = 32, 64, 8, 10000
    N = nx * ny * nz
    y = (np.arange(N) // nx) % ny
    ux = 0.05 + 0.02 * np.sin(2 * np.pi * y / ny)
    lat = lbm.Lattice3(nx, ny, nz, 0.65, None, layout="bundle", algo="nptl", storage=storage)
    lat.init(None, ux, None, None)
    c, _ = O.directions3()
    cx = c[:, 0].astype(np.float64)
    p0 = float(np.sum(cx[:, None] * lat.populations("f64")))
    lat.step(T).sync()
    p1 = float(np.sum(cx[:, None] * lat.populations("f64")))
    assert abs(p1 - p0) <= (1e-5 if storage == "f32" else 1e-10) * abs(p0)
    lat.close()


# ---------------------------------------------------------------- AA pattern

@pytest.mark.parametrize("case", list(SPECS))
@pytest.mark.parametrize("layout", LAYOUTS)
def test_aa_fp64_matches_oracle3(case, layout):
    spec = SPECS[case]
    T = 40
    ref = spec.oracle().run(T)
    lat = spec.gpu(layout=layout, algo="aa", storage="f64", tile=(16, 4, 2))
    lat.step(T, moments=True).sync()
    h = lat.populations("f64")
    rho, ux, uy, uz = lat.moments()
    fl = ref.solid == 0
    assert rel_linf(h, ref.h, fl) <= 1e-12
    assert rel_linf(np.stack([ux, uy, uz]), np.stack([ref.ux, ref.uy, ref.uz]), fl) <= 1e-12
    assert np.all(h[:, ~fl] == 0.0)
    lat.close()


@pytest.mark.parametrize("storage,rounding", [("f32", "rne"), ("f16s", "sr"), ("bf16s", "rne")])
def test_aa_bit_identical_to_two_lattice(storage, rounding):
    """After an even number of updates the AA array is the canonical state:
    equal, bit for bit, to the two-lattice NPTL result; the moments of an odd
    update (the pushing phase) are equal too."""
    for case in ("porous", "duct", "ragged"):
        spec = SPECS[case]
        for T in (70, 37):
            runs = {}
            for algo, tile in (("nptl", (32, 4, 2)), ("aa", (32, 4, 2)), ("aa", (128, 1, 1))):
                lat = spec.gpu(layout="bundle", algo=algo, tile=tile, storage=storage, rounding=rounding,
                               seed=5)
                lat.step(T, moments=True).sync()
                mom = lat.moments()
                pops = lat.populations("f64") if T % 2 == 0 else None
                runs[(algo, tile)] = (mom, pops)
                lat.close()
            base = runs[("nptl", (32, 4, 2))]
            for key, (mom, pops) in runs.items():
                assert all(np.array_equal(a, b) for a, b in zip(mom, base[0])), (case, T, key)
                if pops is not None:
                    assert np.array_equal(pops, base[1]), (case, T, key)


def test_aa_state_access_after_even_updates_only():
    spec = SPECS["duct"]
    lat = spec.gpu(layout="stream", algo="aa", storage="f32")
    lat.step(3).sync()
    with pytest.raises(lbm.LbmError) as e:
        lat.populations()
    assert e.value.status == lbm.LBM_EINVAL
    with pytest.raises(lbm.LbmError):
        lat.mass()
    lat.step(1).sync()
    assert lat.populations().shape == (19, spec.nx * spec.ny * spec.nz)
    assert np.isfinite(lat.mass())
    lat.close()


@pytest.mark.parametrize("layout", LAYOUTS)
def test_aa_pure_streaming_is_bit_exact_shift3(layout):
    nx, ny, nz, T = 23, 9, 7, 6
    N = nx * ny * nz
    rng = np.random.default_rng(5)
    h0 = rng.normal(0.0, 0.01, size=(19, N))
    lat = lbm.Lattice3(nx, ny, nz, math.inf, None, layout=layout, algo="aa", storage="f64",
                       tile=(8, 4, 2))
    lat.write_populations(h0)
    lat.step(T).sync()
    h = lat.populations("f64")
    c, _ = O.directions3()
    for i in range(19):
        exp = np.roll(h0[i].reshape(nz, ny, nx), (T * c[i, 2], T * c[i, 1], T * c[i, 0]),
                      axis=(0, 1, 2)).ravel()
        assert np.array_equal(h[i], exp), i
    lat.close()


@pytest.mark.parametrize("case", ["porous", "duct"])
@pytest.mark.parametrize("layout,algo", [("stream", "nptl"), ("bundle", "lptl"), ("collision", "nptl"),
                                         ("bundle", "aa"), ("stream", "npol")])
def test_force_matches_oracle3(case, layout, algo):
    """FP64 momentum-exchange force on the solid mask (and on a body given as
    a device mask) against the D3Q19 oracle after 40 updates. The force is a
    sum over some 10^3-10^4 body links of terms 2 c_i f_i with f_i ~ w_i
    ~ 0.06 that cancel to ~1e-2: summed in two orders (block tree on the GPU,
    sequential in the oracle), the results may differ by ~eps * 0.1 * links
    ~ 1e-13 absolute, so the bar is 1e-11 relative to the largest component."""
    spec = SPECS[case]
    T = 40
    ref = spec.oracle().run(T)
    lat = spec.gpu(layout=layout, algo=algo, storage="f64", tile=(16, 4, 2))
    lat.step(T).sync()
    body = torch.from_numpy(spec.mask.astype(np.uint8)).cuda()
    f_gpu = lat.force(body)
    f_ref = ref.force(spec.mask)
    assert np.max(np.abs(f_gpu - f_ref)) <= 1e-11 * max(np.max(np.abs(f_ref)), 1e-14)
    f_all = lat.force(None)
    f_ref_all = ref.force(ref.solid)
    assert np.max(np.abs(f_all - f_ref_all)) <= 1e-11 * max(np.max(np.abs(f_ref_all)), 1e-14)
    lat.close()


def _effective_solid_at(mask3, bc, nodes):
    """Effective solidity (mask, or all 18 pulls bouncing) of the given
    (z, y, x) nodes only."""
    c, _ = O.directions3()
    nz, ny, nx = mask3.shape
    ext = (nx, ny, nz)
    out = []
    for (z, y, x) in nodes:
        if mask3[z, y, x]:
            out.append(True)
            continue
        open_ = False
        for i in range(19):
            if i == 9:
                continue
            s = [x - c[i, 0], y - c[i, 1], z - c[i, 2]]
            ok = True
            for a in range(3):
                if s[a] < 0 or s[a] >= ext[a]:
                    if bc[a] != P:
                        ok = False
                    s[a] %= ext[a]
            if ok and not mask3[s[2], s[1], s[0]]:
                open_ = True
                break
        out.append(not open_)
    return np.array(out)


def test_wide_addressing_path_at_136m_nodes():
    """520 x 512 x 512 (136M nodes, 19 N > 2^31: 64-bit addressing), FP16
    storage, stream layout: one update of sampled nodes equals the oracle's
    update of their 3x3x3 neighbourhood taken from the stored state (decoded
    exactly from the device), within one FP16 ulp."""
    nx, ny, nz = 520, 512, 512
    N = nx * ny * nz
    xs, ys, zs = np.arange(nx), np.arange(ny), np.arange(nz)
    mask = (((xs[None, None, :] // 13 + ys[None, :, None] // 11 + zs[:, None, None] // 7) % 9) == 0)
    mask = mask.astype(np.uint8)
    bc = (P, P, W)
    lat = lbm.Lattice3(nx, ny, nz, 0.8, mask, force=(1e-5, 0.0, 0.0), bc=bc, storage="f16s",
                       layout="stream", algo="nptl", tile=(128, 1, 1))
    assert lat.info()["wide_addressing"]
    ux = np.broadcast_to(0.03 * np.sin(2 * np.pi * ys / ny)[None, :, None], (nz, ny, nx)).ravel()
    uz = np.broadcast_to(0.01 * np.cos(2 * np.pi * xs / nx)[None, None, :], (nz, ny, nx)).ravel()
    lat.init(None, np.where(mask.ravel() > 0, 0.0, ux), None, np.where(mask.ravel() > 0, 0.0, uz))
    del ux, uz
    # samples: interior in z (the oracle box must not wrap the wall axis)
    rs = G.SplitMix64(17, 3)
    cand = list(zip(rs.integers(48, 1, nz - 2), rs.integers(48, 0, ny - 1), rs.integers(48, 0, nx - 1)))
    idx = []
    boxes = []
    for (z, y, x) in cand:
        z, y, x = int(z), int(y), int(x)
        zi = [z - 1, z, z + 1]
        yi = [(y + d) % ny for d in (-1, 0, 1)]
        xi = [(x + d) % nx for d in (-1, 0, 1)]
        nodes = [(a, b, c) for a in zi for b in yi for c in xi]
        eff = _effective_solid_at(mask, bc, nodes)
        if eff[13]:
            continue
        boxes.append(((z, y, x), nodes, eff))
        idx.extend((a * ny + b) * nx + c for (a, b, c) in nodes)
    assert len(boxes) >= 20
    idx = torch.tensor(idx, dtype=torch.int64, device="cuda")
    slot = torch.arange(19, device="cuda")[:, None] * N          # stream layout: i N + n
    lattice_bytes = 19 * N * 2
    second = (lattice_bytes + 255) // 256 * 256                   # lattice 1 follows lattice 0

    def stored(which):
        torch.cuda.synchronize()
        raw = lat.workspace[which * second: which * second + lattice_bytes].view(torch.float16)
        return raw[(slot + idx[None, :]).reshape(-1)].reshape(19, -1).double().cpu().numpy()

    lat.step(1).sync()
    h1 = stored(1)          # after an odd number of updates the state is in lattice 1
    lat.step(1).sync()
    h2 = stored(0)
    lat.close()
    for k, ((z, y, x), nodes, eff) in enumerate(boxes):
        cols = slice(27 * k, 27 * k + 27)
        ref = O.Lattice3(O.Case3(3, 3, 3, 0.8, 1e-5, 0.0, 0.0, P, P, P), eff.astype(np.uint8).reshape(3, 3, 3))
        ref.set_h(h1[:, cols])
        ref.run(1)
        got, exp = h2[:, cols][:, 13], ref.h[:, 13]
        assert np.all(np.abs(got - exp) <= 2.0 ** -10 * np.abs(exp) + 1e-7), (x, y, z)


# ---------------------------------------------------------------- degenerate inputs

@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 1, 7), (5, 1, 1), (2, 3, 2), (1, 4, 3)])
@pytest.mark.parametrize("algo", ["lptl", "nptl", "aa", "npol"])
def test_tiny_periodic_boxes_match_oracle3(shape, algo):
    """Boxes where a node is its own neighbour (extent 1) or its neighbour on
    both sides (extent 2), fully periodic, with a force and random velocities."""
    nx, ny, nz = shape
    N = nx * ny * nz
    r = G.SplitMix64(31, nx * 100 + ny * 10 + nz)
    u = [r.uniform(N, -0.02, 0.02) for _ in range(3)]
    rho = 1.0 + r.uniform(N, -0.01, 0.01)
    case = O.Case3(nx, ny, nz, 0.7, 2e-5, -1e-5, 3e-6, P, P, P)
    ref = O.Lattice3(case, None, rho, *u).run(12)
    lat = lbm.Lattice3(nx, ny, nz, 0.7, None, force=(2e-5, -1e-5, 3e-6), algo=algo, storage="f64",
                       tile=(8, 4, 2))
    lat.init(rho, *u).step(12, moments=True).sync()
    assert rel_linf(lat.populations("f64"), ref.h) <= 1e-12
    lat.close()


@pytest.mark.parametrize("algo", ["lptl", "nptl", "aa", "npol"])
def test_all_solid_and_walled_strip3(algo):
    """An all-solid box stays zero with no fluid nodes; a one-node-wide strip
    between walls on two axes (every transverse pull bounces) matches the
    oracle."""
    m = np.ones((4, 5, 6), np.uint8)
    lat = lbm.Lattice3(6, 5, 4, 0.8, m, algo=algo, storage="f32", tile=(8, 4, 2))
    lat.step(6).sync()
    assert lat.info()["fluid_cells"] == 0
    assert np.all(lat.populations() == 0.0) and lat.mass() == 0.0
    lat.close()
    nx, ny, nz = 9, 1, 1
    case = O.Case3(nx, ny, nz, 0.8, 1e-5, 0.0, 0.0, P, W, W)
    ref = O.Lattice3(case, None).run(10)
    lat = lbm.Lattice3(nx, ny, nz, 0.8, None, force=(1e-5, 0.0, 0.0), bc=(P, W, W), algo=algo,
                       storage="f64", tile=(8, 4, 2))
    lat.step(10).sync()
    assert rel_linf(lat.populations("f64"), ref.h) <= 1e-12
    lat.close()


@pytest.mark.parametrize("tile", [(8, 8, 8), (512, 1, 1), (1, 1, 64), (7, 5, 3)])
def test_largest_and_odd_tiles3(tile):
    spec = SPECS["porous"]
    base = spec.gpu(layout="bundle", algo="lptl", storage="f32")
    base.step(20, moments=True).sync()
    ref = base.populations("f32")
    base.close()
    for algo in ("nptl", "aa", "npol"):
        lat = spec.gpu(layout="bundle", algo=algo, storage="f32", tile=tile)
        lat.step(20, moments=True).sync()
        assert np.array_equal(lat.populations("f32"), ref), (algo, tile)
        lat.close()


def test_bad_shapes_rejected3():
    for shape in [(0, 4, 4), (4, -1, 4), (4, 4, 0)]:
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm3_workspace_bytes(lbm.make_params3(*shape, 0.8))
        assert e.value.status == lbm.LBM_EINVAL
    with pytest.raises(lbm.LbmError):
        lbm.lbm3_workspace_bytes(lbm.make_params3(8, 8, 8, 0.8, tile=(8, 8, 9)))


# ---------------------------------------------------------------- inlet / outflow

def _channel3(**kw):
    """Channel 40 x 14 x 10 with a ball: equilibrium inlet U = 0.04 (west),
    zero-gradient outflow (east), walls on y and z, initial u = U."""
    nx, ny, nz = 40, 14, 10
    mask = G.ball(nx, ny, nz, 12.0, 7.0, 5.0, 3.0).ravel()
    r = G.SplitMix64(41, 1)
    ux = np.where(mask > 0, 0.0, 0.04)
    uy = np.where(mask > 0, 0.0, r.uniform(nx * ny * nz, -1e-3, 1e-3))
    case = O.Case3(nx, ny, nz, 0.7, bc_x=lbm.INLET_EQ, bc_xe=lbm.OUTFLOW_ZG, bc_y=W, bc_z=W,
                   u_in=(0.04, 0.0, 0.0))
    ref = O.Lattice3(case, mask, None, ux, uy, None)
    lat = lbm.Lattice3(nx, ny, nz, 0.7, mask, bc=(lbm.INLET_EQ, W, W), bc_x_east=lbm.OUTFLOW_ZG,
                       u_in=(0.04, 0.0, 0.0), **kw)
    lat.init(None, ux, uy, None)
    return ref, lat, mask


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("algo", ["lptl", "nptl", "nptl_wide"])
def test_inlet_outflow_channel_fp64_matches_oracle3(layout, algo):
    T = 60
    flags = lbm.LBM_FLAG_WIDE_OFFSETS if algo.endswith("_wide") else 0
    ref, lat, mask = _channel3(layout=layout, algo=algo.split("_")[0], storage="f64", flags=flags,
                               tile=(16, 4, 2))
    ref.run(T)
    lat.step(T, moments=True).sync()
    fl = ref.solid == 0
    assert rel_linf(lat.populations("f64"), ref.h, fl) <= 1e-12
    rho, ux, uy, uz = lat.moments()
    assert rel_linf(np.stack([ux, uy, uz]), np.stack([ref.ux, ref.uy, ref.uz]), fl) <= 1e-12
    body = torch.from_numpy(mask.astype(np.uint8)).cuda()
    f_gpu, f_ref = lat.force(body), ref.force(mask)
    assert np.max(np.abs(f_gpu - f_ref)) <= 1e-11 * np.max(np.abs(f_ref))
    lat.close()


@pytest.mark.parametrize("storage,rounding", [("f32", "rne"), ("f16s", "sr")])
def test_inlet_outflow_channel_bit_identical(storage, rounding):
    base = None
    for layout in LAYOUTS:
        for algo, tile in (("lptl", (0, 0, 0)), ("nptl", (16, 4, 2)), ("nptl", (128, 1, 1))):
            _, lat, _ = _channel3(layout=layout, algo=algo, tile=tile, storage=storage, rounding=rounding,
                                  seed=3)
            lat.step(70, moments=True).sync()
            got = (lat.populations("f64"), *lat.moments())
            lat.close()
            if base is None:
                base = got
            else:
                assert all(np.array_equal(a, b) for a, b in zip(got, base)), (layout, algo, tile)


def test_inlet_outflow_channel_fp32_close_to_oracle3():
    ref, lat, _ = _channel3(layout="bundle", algo="nptl", storage="f32")
    ref.run(200)
    lat.step(200, moments=True).sync()
    fl = ref.solid == 0
    rho, ux, uy, uz = lat.moments()
    assert rel_linf(rho, ref.rho, fl) <= 1e-5
    assert rel_linf(np.stack([ux, uy, uz]), np.stack([ref.ux, ref.uy, ref.uz]), fl) <= 1e-5
    lat.close()


def test_outflow_on_both_x_faces_matches_oracle3():
    nx, ny, nz, T = 20, 6, 5, 30
    N = nx * ny * nz
    r = G.SplitMix64(43, 2)
    ux = r.uniform(N, 0.0, 0.03)
    case = O.Case3(nx, ny, nz, 0.8, fx=1e-5, bc_x=lbm.OUTFLOW_ZG, bc_y=P, bc_z=W)
    ref = O.Lattice3(case, None, None, ux, None, None).run(T)
    lat = lbm.Lattice3(nx, ny, nz, 0.8, None, force=(1e-5, 0.0, 0.0), bc=(lbm.OUTFLOW_ZG, P, W),
                       storage="f64", tile=(8, 4, 2))
    lat.init(None, ux, None, None).step(T).sync()
    assert rel_linf(lat.populations("f64"), ref.h) <= 1e-12
    lat.close()


# ---------------------------------------------------------------- Zou-He faces

def _zou_he3(**kw):
    """Channel 42 x 14 x 10 with a ball: Zou-He velocity inlet
    U = (0.04, 0.003, -0.002) (west), Zou-He pressure outlet rho = 0.999
    (east), walls on y and z, perturbed initial velocity."""
    nx, ny, nz = 42, 14, 10
    N = nx * ny * nz
    mask = G.ball(nx, ny, nz, 13.0, 7.0, 5.0, 3.0).ravel()
    r = G.SplitMix64(47, 1)
    ux = np.where(mask > 0, 0.0, 0.04)
    uy = np.where(mask > 0, 0.0, r.uniform(N, -1e-3, 1e-3))
    uz = np.where(mask > 0, 0.0, r.uniform(N, -1e-3, 1e-3))
    U, rho_out = (0.04, 0.003, -0.002), 0.999
    case = O.Case3(nx, ny, nz, 0.7, bc_x=lbm.INLET_ZOUHE, bc_xe=lbm.OUTLET_PRESSURE, bc_y=W, bc_z=W,
                   u_in=U, rho_out=rho_out)
    ref = O.Lattice3(case, mask, None, ux, uy, uz)
    lat = lbm.Lattice3(nx, ny, nz, 0.7, mask, bc=(lbm.INLET_ZOUHE, W, W), bc_x_east=lbm.OUTLET_PRESSURE,
                       u_in=U, rho_out=rho_out, **kw)
    lat.init(None, ux, uy, uz)
    return ref, lat, mask


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("algo", ["lptl", "nptl", "nptl_wide"])
def test_zou_he_channel_fp64_matches_oracle3(layout, algo):
    T = 60
    flags = lbm.LBM_FLAG_WIDE_OFFSETS if algo.endswith("_wide") else 0
    ref, lat, mask = _zou_he3(layout=layout, algo=algo.split("_")[0], storage="f64", flags=flags,
                              tile=(16, 4, 2))
    ref.run(T)
    lat.step(T, moments=True).sync()
    fl = ref.solid == 0
    assert rel_linf(lat.populations("f64"), ref.h, fl) <= 1e-12
    rho, ux, uy, uz = lat.moments()
    assert rel_linf(rho, ref.rho, fl) <= 1e-14
    assert rel_linf(np.stack([ux, uy, uz]), np.stack([ref.ux, ref.uy, ref.uz]), fl) <= 1e-12
    x = np.arange(lat.N) % 42
    # the faces' defining conditions hold on the GPU too
    assert np.max(np.abs(ux[(x == 0) & fl] - 0.04)) < 1e-15
    assert np.max(np.abs(rho[(x == 41) & fl] - 0.999)) < 1e-15
    body = torch.from_numpy(mask.astype(np.uint8)).cuda()
    f_gpu, f_ref = lat.force(body), ref.force(mask)
    assert np.max(np.abs(f_gpu - f_ref)) <= 1e-11 * np.max(np.abs(f_ref))
    lat.close()


@pytest.mark.parametrize("storage,rounding", [("f32", "rne"), ("f16s", "sr"), ("bf16s", "rne")])
def test_zou_he_channel_bit_identical3(storage, rounding):
    base = None
    for layout in LAYOUTS:
        for algo, tile in (("lptl", (0, 0, 0)), ("nptl", (16, 4, 2)), ("nptl", (128, 1, 1))):
            _, lat, _ = _zou_he3(layout=layout, algo=algo, tile=tile, storage=storage, rounding=rounding,
                                 seed=5)
            lat.step(70, moments=True).sync()
            got = (lat.populations("f64"), *lat.moments())
            lat.close()
            if base is None:
                base = got
            else:
                assert all(np.array_equal(a, b) for a, b in zip(got, base)), (layout, algo, tile)


def test_zou_he_channel_fp32_close_to_oracle3():
    ref, lat, _ = _zou_he3(layout="bundle", algo="nptl", storage="f32")
    ref.run(200)
    lat.step(200, moments=True).sync()
    fl = ref.solid == 0
    rho, ux, uy, uz = lat.moments()
    assert rel_linf(rho, ref.rho, fl) <= 1e-5
    assert rel_linf(np.stack([ux, uy, uz]), np.stack([ref.ux, ref.uy, ref.uz]), fl) <= 1e-5
    lat.close()


def test_open_faces_rejected_for_one_lattice_algorithms3():
    for algo in ("npol", "nsol", "aa"):
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm3_workspace_bytes(lbm.make_params3(16, 8, 8, 0.8, bc=(lbm.INLET_ZOUHE, W, W), algo=algo,
                                                      bc_x_east=lbm.OUTLET_PRESSURE))
        assert e.value.status == lbm.LBM_EUNSUPPORTED
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm3_workspace_bytes(lbm.make_params3(16, 8, 8, 0.8, bc=(lbm.INLET_ZOUHE, W, W),
                                                  bc_x_east=lbm.OUTLET_PRESSURE, rho_out=0.0))
    assert e.value.status == lbm.LBM_EINVAL


def test_nsol_mass_and_force_match_oracle3():
    spec = SPECS["duct"]
    T = 30
    ref = spec.oracle().run(T)
    lat = spec.gpu(layout="bundle", algo="nsol", storage="f64", tile=(8, 4, 3))
    lat.step(T).sync()
    fl = ref.solid == 0
    assert abs(lat.mass() - ref.mass()) <= 1e-13 * ref.mass()
    body = torch.from_numpy(spec.mask.astype(np.uint8)).cuda()
    f_gpu, f_ref = lat.force(body), ref.force(spec.mask)
    assert np.max(np.abs(f_gpu - f_ref)) <= 1e-11 * np.max(np.abs(f_ref))
    lat.close()


def _even_specs():
    out = {}
    nx, ny, nz = 36, 21, 13
    out["porous"] = Spec3(nx, ny, nz, 0.7, G.porous_spheres(nx, ny, nz, 5, 2.0, 5.0, 0.25), (P, P, P),
                          force=(1e-5, 2e-6, -1e-6))
    nx, ny, nz = 44, 19, 11
    out["duct"] = Spec3(nx, ny, nz, 0.9, G.ball(nx, ny, nz, 12.0, 9.0, 5.0, 3.5), (P, W, W),
                        force=(1e-5, 0.0, 0.0), seed=2)
    nx, ny, nz = 34, 5, 3
    m = np.zeros((nz, ny, nx), np.uint8)
    m[1, 2, 7] = 1
    m[1, 2, 8] = 1
    out["ragged"] = Spec3(nx, ny, nz, 0.6, m, (W, P, W), seed=3)
    return out


EVEN = _even_specs()


@pytest.mark.parametrize("case", list(EVEN))
@pytest.mark.parametrize("layout", ["bundle", "stream"])
@pytest.mark.parametrize("storage,rounding", [("f16s", "rne"), ("f16s", "sr"), ("bf16s", "rne"), ("bf16s", "sr")])
@pytest.mark.parametrize("algo,tile", [("lptl", (0, 0, 0)), ("nptl", (8, 4, 2)), ("nptl", (16, 2, 3))])
def test_node_pairs_bit_identical3(case, layout, storage, rounding, algo, tile):
    """D3Q19 with 16-bit storage: two x-adjacent nodes per thread with the
    collision on packed FP32 pairs give the bits of one node per thread
    (LBM_FLAG_NO_PAIRS), states and moments, on odd and even tiles, ragged
    edges, walls and solid pairs."""
    spec = EVEN[case]
    kw = dict(layout=layout, algo=algo, storage=storage, rounding=rounding, seed=13, tile=tile)
    a = spec.gpu(**kw)
    b = spec.gpu(flags=lbm.LBM_FLAG_NO_PAIRS, **kw)
    assert a.info()["node_pairs"] and not b.info()["node_pairs"]
    a.step(29, moments=True).sync()
    b.step(29, moments=True).sync()
    assert np.array_equal(a.populations("f32"), b.populations("f32"))
    assert all(np.array_equal(u, v) for u, v in zip(a.moments(), b.moments()))
    a.close()
    b.close()


@pytest.mark.parametrize("algo", ["lptl", "nptl"])
def test_node_pairs_with_inlet_outlet_faces3(algo):
    """Pairs on the Zou-He channel (inlet, pressure outlet, walls; nx = 42):
    bit-identical to one node per thread, FP16 with stochastic rounding."""
    kw = dict(layout="bundle", algo=algo, storage="f16s", rounding="sr", seed=3, tile=(8, 2, 2))
    _, a, _ = _zou_he3(**kw)
    _, b, _ = _zou_he3(flags=lbm.LBM_FLAG_NO_PAIRS, **kw)
    assert a.info()["node_pairs"]
    a.step(40, moments=True).sync()
    b.step(40, moments=True).sync()
    assert np.array_equal(a.populations("f32"), b.populations("f32"))
    a.close()
    b.close()
