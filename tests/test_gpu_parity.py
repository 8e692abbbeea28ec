"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Bars (from the method and the arithmetic):
  * FP64 GPU vs FP64 oracle: relative L-inf <= 1e-12 on populations and
    moments (two FP64 implementations that differ only in rounding order;
    a few ulps per update over <= 100 updates).
  * All 3 layouts x 4 algorithms: bit-identical states and moments at equal
    storage precision (the update is the same arithmetic; only the memory
    traffic differs), including the stochastically rounded 16-bit stores.
  * Pure streaming (omega = 0): bit-exact cyclic shift.
"""
import math

import numpy as np
import pytest

from tests.gpu_helpers import ALGOS, COMBOS, LAYOUTS, Spec, rel_linf, specs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2607_20650_gb300 import lbm  # noqa: E402

SPECS = specs()


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2607_20650_gb300 import build
    build.build()
    lbm.load()


def _fluid(spec, ref):
    return ref.solid == 0


@pytest.mark.parametrize("case", list(SPECS))
@pytest.mark.parametrize("layout,algo", COMBOS)
def test_fp64_matches_oracle(case, layout, algo):
    spec = SPECS[case]
    T = 60
    ref = spec.oracle().run(T)
    lat = spec.gpu(layout=layout, algo=algo, storage="f64", tile=(32, 8))
    lat.step(T, moments=True).sync()
    h = lat.populations("f64")
    rho, ux, uy = lat.moments()
    fl = _fluid(spec, ref)
    assert rel_linf(h, ref.h, fl) <= 1e-12
    assert rel_linf(rho, ref.rho, fl) <= 1e-14
    assert rel_linf(np.stack([ux, uy]), np.stack([ref.ux, ref.uy]), fl) <= 1e-12
    assert np.all(h[:, ~fl] == 0.0)
    assert np.all(rho[~fl] == 1.0) and np.all(ux[~fl] == 0.0)
    lat.close()


STORAGE_CASES = [("f64", "rne"), ("f32", "rne"), ("f16s", "rne"), ("f16s", "sr"),
                 ("bf16s", "rne"), ("bf16s", "sr")]


@pytest.mark.parametrize("case", ["channel", "porous", "walls", "neumann_pressure"])
@pytest.mark.parametrize("storage,rounding", STORAGE_CASES)
def test_all_layouts_and_algorithms_bit_identical(case, storage, rounding):
    spec = SPECS[case]
    T = 37
    results = {}
    runs = [(layout, algo, 0) for layout, algo in COMBOS]
    runs += [(layout, "nptl", lbm.LBM_FLAG_TWO_NODES_PER_THREAD) for layout in LAYOUTS]
    for layout, algo, flags in runs:
        tile = (32, 4) if algo in ("npol", "nsol") else (64, 2)
        lat = spec.gpu(layout=layout, algo=algo, storage=storage, rounding=rounding, seed=1234,
                       tile=tile, flags=flags)
        lat.step(T, moments=True).sync()
        results[(layout, algo, flags)] = (lat.populations("f64"), *lat.moments())
        lat.close()
    base = results[("stream", "lptl", 0)]
    for key, r in results.items():
        for a, b in zip(r, base):
            assert np.array_equal(a, b), key


@pytest.mark.parametrize("layout,algo", COMBOS)
@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_pure_streaming_is_bit_exact_shift(layout, algo, storage):
    nx, ny, T = 45, 19, 7
    rng = np.random.default_rng(3)
    h0 = rng.normal(0.0, 0.01, size=(9, nx * ny))
    if storage == "f32":
        h0 = h0.astype(np.float32).astype(np.float64)
    lat = lbm.Lattice(nx, ny, math.inf, None, layout=layout, algo=algo, storage=storage,
                      tile=(32, 4))
    lat.write_populations(h0)
    lat.step(T).sync()
    h = lat.populations("f64")
    cx = np.array([i % 3 - 1 for i in range(9)])
    cy = np.array([i // 3 - 1 for i in range(9)])
    for i in range(9):
        exp = np.roll(h0[i].reshape(ny, nx), (T * cy[i], T * cx[i]), axis=(0, 1)).ravel()
        assert np.array_equal(h[i], exp), i
    lat.close()


@pytest.mark.parametrize("case", list(SPECS))
def test_fp32_close_to_oracle(case):
    """FP32 arithmetic with shifted FP32 storage after 200 updates: relative
    L-inf error on rho and v below 1e-5."""
    spec = SPECS[case]
    T = 200
    ref = spec.oracle().run(T)
    lat = spec.gpu(layout="stream", algo="nptl", storage="f32")
    lat.step(T, moments=True).sync()
    rho, ux, uy = lat.moments()
    fl = ref.solid == 0
    assert rel_linf(rho, ref.rho, fl) <= 1e-5
    assert rel_linf(np.stack([ux, uy]), np.stack([ref.ux, ref.uy]), fl) <= 1e-5
    lat.close()


@pytest.mark.parametrize("case", ["porous", "walls", "channel"])
@pytest.mark.parametrize("algo", ["nptl", "nsol"])
def test_mass_and_force_match_oracle(case, algo):
    spec = SPECS[case]
    T = 50
    ref = spec.oracle().run(T)
    lat = spec.gpu(layout="bundle", algo=algo, storage="f64")
    lat.step(T).sync()
    m_gpu, m_ref = lat.mass(), ref.mass()
    assert abs(m_gpu - m_ref) <= 1e-13 * m_ref
    body = torch.from_numpy(spec.mask.reshape(-1).astype(np.uint8)).cuda()
    f_gpu = lat.force(body)
    f_ref = ref.force(spec.mask)
    assert np.max(np.abs(f_gpu - f_ref)) <= 1e-12 * max(np.max(np.abs(f_ref)), 1e-12)
    lat.close()


def test_graphs_match_single_launches():
    spec = SPECS["channel"]
    a = spec.gpu(layout="stream", algo="npol", storage="f32")
    b = spec.gpu(layout="stream", algo="npol", storage="f32", flags=lbm.LBM_FLAG_NO_GRAPH)
    a.step(150, moments=True).sync()
    b.step(150, moments=True).sync()
    assert np.array_equal(a.populations(), b.populations())
    for x, y in zip(a.moments(), b.moments()):
        assert np.array_equal(x, y)
    a.close()
    b.close()


@pytest.mark.parametrize("algo", ALGOS)
def test_checkpoint_resume_is_bit_exact(algo):
    spec = SPECS["porous"]
    a = spec.gpu(layout="collision", algo=algo, storage="f32")
    a.step(30).sync()
    snap = a.populations("f32")
    a.step(20, moments=True).sync()
    b = spec.gpu(layout="stream", algo=algo, storage="f32")
    b.write_populations(snap)
    b.step(20, moments=True).sync()
    assert np.array_equal(a.populations(), b.populations())
    a.close()
    b.close()


def test_moments_device_matches_host():
    spec = SPECS["channel"]
    lat = spec.gpu(storage="f32")
    lat.step(10, moments=True).sync()
    r, u, v = [torch.empty(lat.N, dtype=torch.float32, device="cuda") for _ in range(3)]
    lbm.lbm_moments_device(lat.h, r, u, v)
    torch.cuda.synchronize()
    host = lat.moments()
    for d, hst in zip((r, u, v), host):
        assert np.array_equal(d.cpu().numpy().astype(np.float64), hst)
    lat.close()


def test_divergence_is_reported_not_trapped():
    spec = SPECS["walls"]
    lat = spec.gpu(storage="f32")
    h = lat.populations("f64")
    h[3, spec.nx * 10 + 5] = np.nan
    lat.write_populations(h)
    lat.step(2)
    with pytest.raises(lbm.LbmError) as e:
        lat.sync()
    assert e.value.status == lbm.LBM_EDIVERGED
    lat.sync()          # flag cleared after it was reported
    lat.close()


def test_bounded_wait_times_out_then_completes():
    """2,000 ungraphed updates of an 8.4M-node lattice queue about 100 ms of
    GPU work; a zero timeout right after enqueueing must report LBM_ETIMEOUT
    (the queue holds at most ~1,000 launches, so at least half of it is
    still pending), and a long one must then complete."""
    lat = lbm.Lattice(4096, 2048, 0.8, None, storage="f32", flags=lbm.LBM_FLAG_NO_GRAPH)
    lat.step(2000)
    s = lbm.lbm_wait(lat.h, 0.0)
    assert s == lbm.LBM_ETIMEOUT
    assert lbm.lbm_wait(lat.h, 120.0) == lbm.LBM_OK
    lat.close()


def _bf16_rne(x32: np.ndarray) -> np.ndarray:
    """Round-to-nearest-even FP32 -> BF16 (upper 16 bits), textbook bias trick."""
    b = x32.view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16).astype(np.uint32) << 16
    return r.astype(np.uint32).view(np.float32)


def test_codec_round_to_nearest_even_matches_numpy():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(0, 1e-3, 40000), rng.normal(0, 1.0, 40000),
                        rng.uniform(-7e-8, 7e-8, 20000)]).astype(np.float32)
    d_in = torch.from_numpy(x).cuda()
    out = torch.empty(x.size, dtype=torch.int16, device="cuda")
    back = torch.empty_like(d_in)
    s = lbm.current_stream()
    lbm.lbm_quantize("f16s", "rne", 0, 0, d_in, out, back, x.size, s)
    torch.cuda.synchronize()
    assert np.array_equal(back.cpu().numpy(), x.astype(np.float16).astype(np.float32))
    lbm.lbm_quantize("bf16s", "rne", 0, 0, d_in, out, back, x.size, s)
    torch.cuda.synchronize()
    assert np.array_equal(back.cpu().numpy(), _bf16_rne(x))


@pytest.mark.parametrize("storage", ["f16s", "bf16s"])
def test_codec_stochastic_rounding_is_unbiased_and_keyed(storage):
    """Each value rounds to one of its two 16-bit neighbours, away from zero
    with probability (|x| - |lo|) / ulp (below 2^-14, FP16's, cut to 13 bits:
    at most 2^-13 low): checked for values in the FP16 normal range, in its
    subnormal range (2.5e-5 < 2^-14, 9.1e-8 just above 2^-24, 3.7e-8 below
    it), negative ones and a large one. The draws depend on the keys only (same update index, same
    bits; another index, other draws), and the decisions of different
    directions of one node are uncorrelated."""
    K = 9 * 200000
    s = lbm.current_stream()
    for val in (np.float32(1.0e-3 + 3.3e-7), np.float32(-2.5e-5 - 1.3e-9), np.float32(0.3 + 1.1e-7),
                np.float32(-7.1e-2 - 2.9e-9), np.float32(9.1e-8), np.float32(-3.7e-8)):
        x = np.full(K, val, dtype=np.float32)
        d_in = torch.from_numpy(x).cuda()
        out = torch.empty(K, dtype=torch.int16, device="cuda")
        b1, b2, b3 = (torch.empty_like(d_in) for _ in range(3))
        lbm.lbm_quantize(storage, "sr", 42, 5, d_in, out, b1, K, s)
        lbm.lbm_quantize(storage, "sr", 42, 5, d_in, out, b2, K, s)
        lbm.lbm_quantize(storage, "sr", 42, 6, d_in, out, b3, K, s)
        torch.cuda.synchronize()
        v1, v2, v3 = (b.cpu().numpy().astype(np.float64) for b in (b1, b2, b3))
        assert np.array_equal(v1, v2)                    # same keys, same bits
        assert not np.array_equal(v1, v3)                # another update index, other draws
        vals = np.unique(v1)
        assert len(vals) == 2, (val, vals)               # only the two neighbours
        near, far = (vals[1], vals[0]) if val < 0 else (vals[0], vals[1])
        assert abs(near) < abs(float(val)) < abs(far)
        p = (abs(float(val)) - abs(near)) / (abs(far) - abs(near))
        up = (v1 == far)
        frac = np.mean(up)
        assert abs(frac - p) < 5 * math.sqrt(p * (1 - p) / K) + 2 ** -13, (val, frac, p)
        # directions of one node (k = 9 n + i): decisions of i and i + 1 uncorrelated
        d = up.reshape(-1, 9).astype(np.float64)
        for i in range(8):
            c = np.corrcoef(d[:, i], d[:, i + 1])[0, 1]
            assert abs(c) < 5 / math.sqrt(d.shape[0]), (val, i, c)


def _u32(v):
    return np.asarray(v, dtype=np.uint64) & np.uint64(0xFFFFFFFF)


def _mix32(x):
    """lowbias32 (C. Wellons' hash-prospector): the keys' finaliser."""
    x = _u32(x)
    x ^= x >> np.uint64(16)
    x = _u32(x * np.uint64(0x7FEB352D))
    x ^= x >> np.uint64(15)
    x = _u32(x * np.uint64(0x846CA68B))
    x ^= x >> np.uint64(16)
    return x


def _draws(seed, t, count):
    """Random word of element k = 9 n + i at update t: the node's hashed key
    with the direction folded in (the keys of LBM_ROUND_SR)."""
    sk = _mix32(np.uint64(seed & 0xFFFFFFFF) ^ _mix32(np.uint64(seed >> 32) ^ _mix32(np.uint64(t))))
    k = np.arange(count, dtype=np.uint64)
    nk = _mix32((k // np.uint64(9)) ^ sk)
    i = k % np.uint64(9)
    return _u32((nk ^ _u32(i * np.uint64(0x9E3779B9))) * np.uint64(0x85EBCA6B))


@pytest.mark.parametrize("storage", ["f16s", "bf16s"])
def test_codec_stochastic_rounding_matches_its_definition(storage):
    """Bit-level check of the stochastic codec against its definition, on a
    spread of magnitudes (FP16 normal and subnormal ranges, below 2^-24, BF16
    over the FP32 range) and both signs: with ulp the 16-bit spacing at x and
    lo = x truncated toward zero to a multiple of it, the value rounds away
    from zero exactly when floor(frac 2^m) + (r >> (32 - m)) >= 2^m, frac =
    (|x| - |lo|) / ulp, m = 13 (FP16) or 16 (BF16), r the element's random
    word."""
    K = 9 * 120000
    rng = np.random.default_rng(11)
    e = rng.integers(-34, 6, K) if storage == "f16s" else rng.integers(-120, 120, K)
    x = (rng.uniform(1.0, 2.0, K) * np.exp2(e.astype(np.float64)) * rng.choice([-1.0, 1.0], K)).astype(np.float32)
    s = lbm.current_stream()
    d_in = torch.from_numpy(x).cuda()
    out = torch.empty(K, dtype=torch.int16, device="cuda")
    back = torch.empty_like(d_in)
    seed, t = 0x1234567890ABCDEF, 77
    lbm.lbm_quantize(storage, "sr", seed, t, d_in, out, back, K, s)
    torch.cuda.synchronize()
    got = back.cpu().numpy().astype(np.float64)
    r = _draws(seed, t, K)
    xa = np.abs(x.astype(np.float64))
    if storage == "f16s":
        m = 13
        ex = np.floor(np.log2(np.maximum(xa, 2.0 ** -40)))
        ulp = np.where(xa >= 2.0 ** -14, np.exp2(ex - 10), 2.0 ** -24)
    else:
        m = 16
        ulp = np.exp2(np.floor(np.log2(xa)) - 7)
    lo = np.floor(xa / ulp) * ulp
    frac = (xa - lo) / ulp
    dm = np.floor(frac * 2.0 ** m)
    away = dm + (r >> np.uint64(32 - m)).astype(np.float64) >= 2.0 ** m
    want = np.sign(x) * (lo + np.where(away, ulp, 0.0))
    bad = np.flatnonzero(got != want)
    assert bad.size == 0, [(float(x[k]), got[k], want[k]) for k in bad[:5]]
    assert 0.2 < away.mean() < 0.8     # both outcomes exercised


def test_neumann_inlet_rejected_for_aa_and_thin_one_lattice_tiles():
    spec = SPECS["neumann_pressure"]
    with pytest.raises(lbm.LbmError) as e:
        spec.gpu(algo="aa", storage="f32")
    assert e.value.status == lbm.LBM_EUNSUPPORTED
    with pytest.raises(lbm.LbmError):
        spec.gpu(algo="npol", storage="f32", tile=(1, 64))


@pytest.mark.parametrize("storage", ["f32", "f64"])
def test_momentum_conserved_over_long_runs(storage):
    """Periodic box, no force, u_x = U0 + U1 sin(2 pi y / ny): BGK conserves
    total momentum exactly, so after 20,000 updates the stored state's
    sum_n sum_i c_i h_i may differ from the initial one by rounding noise
    only. A systematic source of omega * delta * u per node and update
    (delta ~ 1e-8, the error of rounded FP32 weights in sum_i w_i c_i c_i)
    would move it by ~3e-4; the bar is 1e-5 (FP32) and 1e-10 (FP64, where
    the rounded weights' delta ~1e-16 still gives omega delta T ~ 1e-11)."""
    nx, ny, T = 64, 256, 20000
    y = np.arange(ny)[:, None] * np.ones((1, nx))
    ux = 0.05 + 0.02 * np.sin(2 * np.pi * y / ny)
    lat = lbm.Lattice(nx, ny, 0.65, None, layout="bundle", algo="nptl", storage=storage)
    lat.init(None, ux.ravel(), np.zeros(nx * ny))
    cx = np.array([i % 3 - 1 for i in range(9)], dtype=np.float64)
    p0 = float(np.sum(cx[:, None] * lat.populations("f64")))
    lat.step(T).sync()
    p1 = float(np.sum(cx[:, None] * lat.populations("f64")))
    assert abs(p1 - p0) <= (1e-5 if storage == "f32" else 1e-10) * abs(p0)
    lat.close()
