#!/usr/bin/env python3
"""Throughput of the D2Q9I BGK stream-and-collide update on one GB300.

Workload (default): the large porous medium, 16384 x 8192 nodes (134M),
seeded random overlapping discs (radii 8-32, solid fraction 0.4), periodic
in x and y, body force g_x = 1e-6, tau = 0.9. One step = one lattice
update (pull, bounce-back, moments, BGK + Guo collision, store) of the whole
lattice, FP32 storage and arithmetic, bundle layout (SoAoS), NPTL (2-D tiles
of 32 x 4 nodes, two lattices): the fastest two-lattice combination measured
on this workload. MLUPS counts every node (solid ones included), as the paper does.

Also reported: the same update with FP16/BF16 shifted storage, the one-lattice
NPOL, NSOL and AA variants, the batched ensemble of 256 channels against 256
sequential single-case runs, the D3Q19 extension (a 384^3 sphere packing in
every layout and algorithm, and a batch of 128 boxes against sequential
runs), the headline lattice split into 2 and 4 x-slabs exchanging their
faces after every update (slabs), the FP64 CPU oracle on a bounded sample (cpu_baseline), and an
end-to-end number through the C ABI with host buffers (e2e).

Prints ONE JSON line. ``--impl reference`` times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

def workload(nx: int = 16384, ny: int = 8192) -> str:
    return (f"porous {nx}x{ny} ({nx * ny / 1e6:.0f}M nodes), discs r 8-32 phi 0.4 seed 3, periodic, "
            f"g_x 1e-6, tau 0.9")


WORKLOAD = workload()
METRIC = "D2Q9 BGK MLUPS (FP32 two-lattice, 134M-node porous medium)"
PROFILE = os.path.join(ROOT, "profiles", "k_two_lattice_f32_bundle_nptl_porous16384x8192.md")
KERNEL_SOURCES = ["paper_2607_20650_gb300/csrc/lbm_kernels.cuh",
                  "paper_2607_20650_gb300/csrc/lbm_device.cuh"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nx", type=int, default=16384)
    ap.add_argument("--ny", type=int, default=8192)
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--tile", default="")
    ap.add_argument("--layout", default="bundle", choices=["stream", "bundle", "collision"])
    ap.add_argument("--algo", default="nptl", choices=["lptl", "nptl", "npol", "nsol", "aa"],
                    help="D3Q19 (--lattice d3q19): lptl, nptl, npol, nsol or aa")
    ap.add_argument("--storage", default="f32", choices=["f32", "f16s", "bf16s", "f64"])
    ap.add_argument("--rounding", default="rne", choices=["rne", "sr"])
    ap.add_argument("--flags", type=lambda v: int(v, 0), default=0, help="lbm_params.flags (LBM_FLAG_*)")
    ap.add_argument("--lattice", default="d2q9", choices=["d2q9", "d3q19"],
                    help="d3q19: time only the 3-D extension on an n3^3 sphere packing")
    ap.add_argument("--n3", type=int, default=384)
    ap.add_argument("--geo3", default="porous", choices=["porous", "fluid"])
    ap.add_argument("--batch-only", action="store_true",
                    help="time only the 256-channel batched ensemble (profiling)")
    ap.add_argument("--batch3-only", action="store_true",
                    help="time only the batch of 512 D3Q19 boxes (profiling)")
    ap.add_argument("--ref-seconds", type=float, default=120.0,
                    help="--impl reference: CPU seconds for the warm-up and timed steps together")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_sha() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """dram bytes per launch from the committed ncu summary, if the kernel
    sources still hash to what was profiled."""
    try:
        text = open(PROFILE).read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    s = re.search(r"kernel_source_sha:\s*([0-9a-f]+)", text)
    if not m or not s or s.group(1) != kernel_sha():
        return None
    return float(m.group(1))


class Clocks:
    """nvidia-smi samples (200 ms) while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", gpu_id, f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.tmp, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.tmp.flush()
        rows = [r.split(",") for r in open(self.tmp.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.tmp.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for name, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def smi_id(torch, local: int) -> str:
    """nvidia-smi id (UUID) of the CUDA device the process uses."""
    props = torch.cuda.get_device_properties(local)
    gpu_id = str(getattr(props, "uuid", local))
    if gpu_id and not gpu_id.startswith("GPU-") and "-" in gpu_id:
        gpu_id = "GPU-" + gpu_id
    return gpu_id


def max_over_ranks(value: float, device: str) -> float:
    """Largest value over all ranks of the default process group (the timed
    region's length: the job is as slow as its slowest replica)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def kernel_name(args, tile=(32, 4)) -> str:
    """The update kernel as ncu lists it (layout as its enum value: stream 0,
    bundle 1, collision 2)."""
    t = {"f32": "float", "f64": "double", "f16s": "__half", "bf16s": "__nv_bfloat16"}[args.storage]
    lay = {"stream": 0, "bundle": 1, "collision": 2}[args.layout]
    pairs = (args.storage in ("f16s", "bf16s") and args.layout == "bundle" and args.nx % 2 == 0
             and not (getattr(args, "flags", 0) & 0x20))
    if args.algo == "lptl":
        return f"k_two_lattice_pair<{t}, {lay}, true>" if pairs else f"k_two_lattice<{t}, {lay}, true>"
    if args.algo == "nptl":
        if pairs and tile[0] % 2 == 0:
            return f"k_two_lattice_pair<{t}, {lay}, false>"
        if args.layout == "collision" and tile[0] % 32 == 0:
            return f"k_two_lattice_aos<{t}>"
        return f"k_two_lattice<{t}, {lay}, false>"
    return {"npol": f"k_npol<{t}, {lay}>", "nsol": f"k_nsol<{t}, {lay}>",
            "aa": f"k_aa<{t}, {lay}, 0|1> (two phases)"}[args.algo]


def launches_for(k: int, graph_block: int = 64) -> int:
    """Kernels one lbm_step(k) call (no moments) enqueues: k updates, one
    counter bump per graph block and one after the directly launched
    remainder."""
    n = 0
    left = k
    while left >= graph_block:
        n += graph_block + 1
        left -= graph_block
    if left > 0:
        n += left + 1
    return n


def chunks_of(k: int, runs: int = 10) -> list[int]:
    """k updates split into up to `runs` consecutive runs (multiples of 64
    where possible, so graphs of whole blocks carry most of each run)."""
    if k < 2 * runs:
        return [k]
    base = max(64, (k // runs) // 64 * 64)
    out = []
    left = k
    while left > 0:
        c = min(base, left)
        out.append(c)
        left -= c
    if len(out) > 1 and out[-1] < base // 2:
        out[-2] += out.pop()
    return out


def time_steps(lat, k, torch, runs: int = 10):
    """k updates bracketed by CUDA events on the lattice's own stream, issued
    as consecutive runs (the paper's protocol: runs, median, min / max) with
    an event between runs; returns (total seconds, per-update ms of each run,
    run lengths)."""
    from paper_2607_20650_gb300 import lbm
    s = lat.torch_stream
    parts = chunks_of(k, runs)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(parts) + 1)]
    torch.cuda.synchronize()
    ev[0].record(s)
    for j, c in enumerate(parts):
        lbm.lbm_step(lat.h, c, False)
        ev[j + 1].record(s)
    ev[-1].synchronize()
    lbm.lbm_sync(lat.h)
    per = [ev[j].elapsed_time(ev[j + 1]) / c for j, c in enumerate(parts)]
    return ev[0].elapsed_time(ev[-1]) / 1e3, per, parts


def _oracle_rate(lat, cells: int, target_s: float) -> tuple[float, int, float]:
    t = time.perf_counter()
    lat.run(2)
    per = (time.perf_counter() - t) / 2
    k = max(2, int(target_s / per))
    t = time.perf_counter()
    lat.run(k)
    dt = time.perf_counter() - t
    return cells * k / dt / 1e6, k, dt


def cpu_sample(target_s: float = 12.0):
    """FP64 oracle on the 2048x1024 porous sub-run (same disc statistics,
    seed 33) for as many updates as fit ~target_s seconds on every host
    thread; then the same on one thread, and the Poiseuille 256x64 and
    Karman 2048x512 configurations briefly (all threads)."""
    import oracle as O
    from paper_2607_20650_gb300 import geometry as G
    nx, ny = 2048, 1024
    mask = G.porous_discs(nx, ny, seed=33)
    lat = O.Lattice(O.Case(nx, ny, 0.9, fx=1e-6), mask)
    threads = O.omp_threads()
    mlups, k, dt = _oracle_rate(lat, nx * ny, target_s)
    O.set_threads(1)
    one, k1, dt1 = _oracle_rate(lat, nx * ny, 3.0)
    O.set_threads(threads)
    pw = G.poiseuille()
    pois, _, _ = _oracle_rate(O.Lattice(O.Case(pw.nx, pw.ny, pw.tau, fx=pw.fx, bc_s=pw.bc_s, bc_n=pw.bc_n),
                                        pw.mask), pw.nx * pw.ny, 1.5)
    kw = G.karman()
    karman, _, _ = _oracle_rate(O.Lattice(O.Case(kw.nx, kw.ny, kw.tau, ux_in=kw.ux_in, bc_w=kw.bc_w,
                                                 bc_e=kw.bc_e, bc_s=kw.bc_s, bc_n=kw.bc_n),
                                          kw.mask, ux=kw.ux0, uy=kw.uy0), kw.nx * kw.ny, 2.0)
    return {"value": mlups, "unit": "MLUPS", "cores": threads, "kind": "oracle",
            "sample": f"porous 2048x1024 (seed 33, same statistics), {k} FP64 updates, "
                      f"{dt:.1f} s, OpenMP threads {threads}",
            "one_core_MLUPS": one, "one_core_sample": f"{k1} updates, {dt1:.1f} s",
            "poiseuille_256x64_MLUPS": pois, "karman_2048x512_MLUPS": karman}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    steps, warm = args.steps, args.warmup
    import oracle as O
    from paper_2607_20650_gb300 import geometry as G
    nx, ny = 2048, 1024
    mask = G.porous_discs(nx, ny, seed=33)
    lat = O.Lattice(O.Case(nx, ny, 0.9, fx=1e-6), mask)
    # Bounded sample per step: updates of the 2M-node sub-run; keep the whole
    # run within a few minutes.
    t = time.perf_counter()
    lat.run(1)
    per = time.perf_counter() - t
    k_per_step = max(1, int(args.ref_seconds / max(steps + warm, 1) / per))
    for _ in range(warm):
        lat.run(k_per_step)
    t = time.perf_counter()
    for _ in range(steps):
        lat.run(k_per_step)
    dt = time.perf_counter() - t
    mlups = nx * ny * k_per_step * steps / dt / 1e6
    sample = (f"FP64 oracle, porous 2048x1024 sub-run (seed 33, same statistics as the 16384x8192 "
              f"workload), {k_per_step} updates per step")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": mlups, "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": steps, "warmup": warm,
        "ms_per_step": dt / steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload(2048, 1024).replace("seed 3", "seed 33"), "sample": sample,
                   "stands_in_for": WORKLOAD},
        "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": O.omp_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_ours(args):
    import torch
    world, rank, local = dist_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2607_20650_gb300 import build, geometry as G, lbm
    build.build()
    lbm.load()
    nx, ny = args.nx, args.ny
    tile = tuple(int(v) for v in args.tile.split("x")) if args.tile else (32, 4)
    mask = G.porous_discs(nx, ny, seed=3)
    kw = dict(force=(1e-6, 0.0), bc=(lbm.PERIODIC,) * 4, layout=args.layout, algo=args.algo,
              storage=args.storage, rounding=args.rounding, seed=7, tile=tile, flags=args.flags)
    stream = torch.cuda.Stream()
    lat = lbm.Lattice(nx, ny, 0.9, mask, stream=stream, **kw)
    info = lat.info()
    lat.step(args.warmup).sync()

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    barrier()
    clk = Clocks(smi_id(torch, local))
    dt, per_run, parts = time_steps(lat, args.steps, torch)
    clocks = clk.stop()
    barrier()
    if dist is not None:
        dt = max_over_ranks(dt, "cuda")
    cells = nx * ny
    mlups = cells * args.steps * world / dt / 1e6
    per_launch = dt / args.steps
    hbm, peak_kind = peaks()
    achieved = info["bytes_per_update"] / per_launch / 1e9
    traffic = profiled_traffic() if (args.layout, args.algo, args.storage, nx, ny, tile) == \
        ("bundle", "nptl", "f32", 16384, 8192, (32, 4)) else None
    result = {
        "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_launch * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"f32": "f32", "f64": "f64", "f16s": "f16 storage, f32 arithmetic",
                  "bf16s": "bf16 storage, f32 arithmetic"}[args.storage],
        "data": "synthetic",
        "config": {"workload": workload(nx, ny), "layout": args.layout, "algo": args.algo,
                   "tile": f"{info['tile_x']}x{info['tile_y']}", "storage": f"{args.storage} shifted",
                   "fluid_nodes": info["fluid_cells"], "nodes": cells,
                   "l2": "inputs larger than L2 (two 4.8 GB lattices)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "gpu_launches": sum(launches_for(c) for c in parts),
        "runs": {"updates": parts, "ms_per_update_median": statistics.median(per_run),
                 "ms_per_update_min": min(per_run), "ms_per_update_max": max(per_run)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": traffic, "peak_kind": peak_kind,
                     "algorithmic_bytes_per_launch": info["bytes_per_update"],
                     "kernel": kernel_name(args, tile)},
        "clocks": clocks,
        "mlups_fluid": info["fluid_cells"] * args.steps * world / dt / 1e6,
    }
    lat.close()
    del lat
    torch.cuda.empty_cache()

    if not args.no_variants:
        result["variants"] = variants(args, mask, torch, world)
        result["slabs"] = slab_split(args, mask, torch, tile)
        result["batched"] = batched(args, torch)
        result["d3q19"] = d3q19(args, torch)
        result["batched_d3q19"] = batched3(args, torch)
    result["e2e"] = e2e(args, mask, torch, world)
    if rank == 0 and not args.no_cpu and world == 1:
        result["cpu_baseline"] = cpu_sample()
    if rank == 0:
        print(json.dumps(result))
    if dist is not None:
        dist.destroy_process_group()


def variants(args, mask, torch, world):
    from paper_2607_20650_gb300 import lbm
    nx, ny = args.nx, args.ny
    k = min(args.steps, 400)
    out = {}
    hbm, _ = peaks()
    for name, kw in [("f32_bundle_nptl_128x1_allfluid", dict(storage="f32", layout="bundle", tile=(128, 1),
                                                            geo="fluid")),
                     ("f64_bundle_nptl_128x1_allfluid", dict(storage="f64", layout="bundle", tile=(128, 1),
                                                             geo="fluid")),
                     ("f32_stream_nptl_32x4", dict(storage="f32", tile=(32, 4))),
                     ("f32_stream_lptl", dict(storage="f32", algo="lptl")),
                     ("f32_collision_nptl_64x4", dict(storage="f32", layout="collision", tile=(64, 4))),
                     ("f32_stream_npol_32x8", dict(storage="f32", algo="npol", tile=(32, 8))),
                     ("f32_bundle_npol_64x4", dict(storage="f32", algo="npol", layout="bundle", tile=(64, 4))),
                     ("f32_bundle_nsol_64x4", dict(storage="f32", algo="nsol", layout="bundle", tile=(64, 4))),
                     ("f32_bundle_nsol_64x4_no_tma", dict(storage="f32", algo="nsol", layout="bundle", tile=(64, 4),
                                                          flags=0x40)),
                     ("f32_bundle_aa_64x2", dict(storage="f32", algo="aa", layout="bundle", tile=(64, 2))),
                     ("f16s_rne_bundle_nptl_32x8", dict(storage="f16s", layout="bundle", tile=(32, 8))),
                     ("f16s_rne_bundle_nptl_32x8_one_node_per_thread",
                      dict(storage="f16s", layout="bundle", tile=(32, 8), flags=0x20)),
                     ("bf16s_rne_bundle_nptl_32x8", dict(storage="bf16s", layout="bundle", tile=(32, 8))),
                     ("f16s_sr_bundle_nptl_32x8", dict(storage="f16s", layout="bundle", tile=(32, 8),
                                                       rounding="sr", seed=7)),
                     ("bf16s_sr_bundle_nptl_32x8", dict(storage="bf16s", layout="bundle", tile=(32, 8),
                                                        rounding="sr", seed=7)),
                     ("f16s_rne_stream_npol_32x8", dict(storage="f16s", algo="npol", tile=(32, 8))),
                     ("bf16s_rne_stream_npol_32x8", dict(storage="bf16s", algo="npol", tile=(32, 8)))]:
        kw = dict(kw)
        kw.setdefault("layout", "stream")
        geo = kw.pop("geo", "porous")
        m = mask if geo == "porous" else np.zeros_like(mask)
        lat = lbm.Lattice(nx, ny, 0.9, m, stream=torch.cuda.Stream(), force=(1e-6, 0.0),
                          bc=(lbm.PERIODIC,) * 4, **kw)
        info = lat.info()
        lat.step(args.warmup).sync()
        dt, per_run, _ = time_steps(lat, k, torch, runs=4)
        out[name] = {"MLUPS": nx * ny * k / dt / 1e6, "ms_per_step": dt / k * 1e3,
                     "ms_per_step_min_max": [min(per_run), max(per_run)],
                     "GBps_algorithmic": info["bytes_per_update"] / (dt / k) / 1e9,
                     "frac_of_measured_hbm": info["bytes_per_update"] / (dt / k) / 1e9 / hbm,
                     "bytes_per_update": info["bytes_per_update"],
                     "workspace_GB": info["workspace_bytes"] / 1e9, "steps": k}
        lat.close()
        del lat
        torch.cuda.empty_cache()
    return out


def slab_split(args, mask, torch, tile):
    """The headline lattice split into 2 and 4 x-slabs on this GPU, the
    crossing populations of every face exchanged on the device after every
    update (the domain split of a multi-GPU run with its transport inside one
    process): the cost of the split against the undivided lattice."""
    from paper_2607_20650_gb300 import lbm
    from paper_2607_20650_gb300 import slabs as S
    nx, ny = args.nx, args.ny
    k = min(args.steps, 200)
    out = {}
    for parts in (2, 4):
        dec = S.Decomposition(nx, ny, 0.9, mask, parts=parts, force=(1e-6, 0.0), bc=(lbm.PERIODIC,) * 4,
                              layout="bundle", algo="nptl", storage="f32", tile=tile)
        dec.init()
        dec.step(args.warmup).sync()
        s = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s)
        dec.step(k)
        e1.record(s)
        e1.synchronize()
        dec.sync()
        dt = e0.elapsed_time(e1) / 1e3
        out[f"f32_bundle_nptl_{tile[0]}x{tile[1]}_{parts}_slabs"] = {
            "MLUPS": nx * ny * k / dt / 1e6, "ms_per_step": dt / k * 1e3, "steps": k,
            "slab_columns": [sl.nx for sl in dec.slabs], "messages_per_update": len(dec.msgs),
            "bytes_per_message": 3 * ny * 4,
            # per slab: the update kernel and the update-counter bump; one exchange launch per 16 messages
            "launches_per_update": 2 * parts + -(-len(dec.msgs) // 16)}
        dec.close()
        del dec
        torch.cuda.empty_cache()
    return out


def run_d3q19(args):
    """One JSON line for the 3-D extension alone (profiling and sweeps):
    n3^3 periodic sphere packing or all-fluid box, --layout/--algo/--storage,
    --tile as AxBxC (default 128x1x1)."""
    import torch
    from paper_2607_20650_gb300 import build, geometry as G, lbm
    build.build()
    lbm.load()
    n = args.n3
    N = n ** 3
    tile = tuple(int(v) for v in args.tile.split("x")) if args.tile else (128, 1, 1)
    mask = G.porous_spheres(n, n, n, 3, 4.0, 12.0, 0.3)
    if args.geo3 == "fluid":
        mask = np.zeros_like(mask)
    stream = torch.cuda.Stream()
    lat = lbm.Lattice3(n, n, n, 0.8, mask, stream=stream, force=(1e-6, 0.0, 0.0), layout=args.layout,
                       algo=args.algo, storage=args.storage, tile=tile)
    info = lat.info()
    lat.step(args.warmup).sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    clk = Clocks(smi_id(torch, torch.cuda.current_device()))
    e0.record(stream)
    lbm.lbm3_step(lat.h, args.steps, False)
    e1.record(stream)
    e1.synchronize()
    clocks = clk.stop()
    lat.sync()
    dt = e0.elapsed_time(e1) / 1e3
    hbm, peak_kind = peaks()
    achieved = info["bytes_per_update"] / (dt / args.steps) / 1e9
    print(json.dumps({
        "metric": "D3Q19 BGK MLUPS", "value": N * args.steps / dt / 1e6, "unit": "MLUPS", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.storage,
        "data": "synthetic",
        "config": {"workload": f"{n}^3 {args.geo3} box (spheres r 4-12, phi 0.3, seed 3), periodic, "
                               f"g_x 1e-6, tau 0.8", "layout": args.layout, "algo": args.algo,
                   "tile": "x".join(map(str, tile)), "fluid_nodes": info["fluid_cells"]},
        "gpu_launches": launches_for(args.steps),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": None, "peak_kind": peak_kind,
                     "algorithmic_bytes_per_launch": info["bytes_per_update"]},
        "clocks": clocks}))
    lat.close()


def d3q19(args, torch):
    """The 3-D extension: a 384^3 periodic box of random overlapping spheres
    (radii 4-12, solid fraction 0.3, seed 3; tau 0.8, g_x = 1e-6) and the
    same box all fluid, through the lbm3_* C ABI. Algorithmic bytes per
    update: fluid nodes x 2 x 19 x sizeof(storage) + 4 link bytes per node."""
    from paper_2607_20650_gb300 import geometry as G, lbm
    n = 384
    N = n ** 3
    k = max(20, min(args.steps, 200))
    porous = G.porous_spheres(n, n, n, 3, 4.0, 12.0, 0.3)
    hbm, _ = peaks()
    out = {"workload": f"{n}^3 periodic box, spheres r 4-12, solid fraction {porous.mean():.3f}"}
    for name, geo, kw in [("f32_bundle_nptl_128x1x1_porous", "porous", dict(storage="f32", layout="bundle")),
                          ("f32_bundle_nptl_128x1x1_allfluid", "fluid", dict(storage="f32", layout="bundle")),
                          ("f32_stream_nptl_128x1x1_porous", "porous", dict(storage="f32", layout="stream")),
                          ("f32_collision_nptl_128x1x1_porous", "porous", dict(storage="f32", layout="collision")),
                          ("f16s_rne_bundle_nptl_128x1x1_porous", "porous", dict(storage="f16s", layout="bundle")),
                          ("f16s_rne_stream_nptl_128x1x1_porous", "porous", dict(storage="f16s", layout="stream")),
                          ("f16s_rne_bundle_lptl_porous", "porous", dict(storage="f16s", layout="bundle", algo="lptl",
                                                                         tile=(0, 0, 0))),
                          ("f32_bundle_aa_128x1x1_porous", "porous", dict(storage="f32", layout="bundle", algo="aa")),
                          ("f32_stream_npol_8x8x8_porous", "porous", dict(storage="f32", layout="stream", algo="npol",
                                                                         tile=(8, 8, 8))),
                          ("f32_bundle_nsol_8x8x8_porous", "porous", dict(storage="f32", layout="bundle", algo="nsol",
                                                                         tile=(8, 8, 8))),
                          ("f32_stream_nsol_8x8x8_porous", "porous", dict(storage="f32", layout="stream", algo="nsol",
                                                                         tile=(8, 8, 8)))]:
        m = porous if geo == "porous" else np.zeros_like(porous)
        stream = torch.cuda.Stream()
        kw = dict(kw)
        kw.setdefault("algo", "nptl")
        kw.setdefault("tile", (128, 1, 1))
        lat = lbm.Lattice3(n, n, n, 0.8, m, stream=stream, force=(1e-6, 0.0, 0.0), **kw)
        info = lat.info()
        lat.step(args.warmup).sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        lbm.lbm3_step(lat.h, k, False)
        e1.record(stream)
        e1.synchronize()
        lat.sync()
        dt = e0.elapsed_time(e1) / 1e3
        gbs = info["bytes_per_update"] / (dt / k) / 1e9
        out[name] = {"MLUPS": N * k / dt / 1e6, "ms_per_step": dt / k * 1e3, "GBps_algorithmic": gbs,
                     "frac_of_measured_hbm": gbs / hbm, "bytes_per_update": info["bytes_per_update"],
                     "fluid_nodes": info["fluid_cells"], "steps": k}
        lat.close()
        del lat
        torch.cuda.empty_cache()
    return out


def batched(args, torch):
    """256 independent channels (seeded widths 64-1024, heights 32-512, tau in
    [0.55, 1.5], one obstacle each, Zou-He inlet, zero-gradient outflow, FP32):
    one persistent launch per update (graphs of 100 updates, layout /
    algorithm / tile per case from the autotuner) against the same 256 cases
    run one after another as single lattices (each lbm_step(K), graphs of 64)."""
    from paper_2607_20650_gb300 import geometry as G, lbm
    ws = G.batch_channels(256, seed=4)
    probe_w = G.batch_channels(1, seed=99, wmin=1024, wmax=1024, hmin=512, hmax=512)[0]
    bc = lambda w: (w.bc_w, w.bc_e, w.bc_s, w.bc_n)
    probe = lbm.make_params(probe_w.nx, probe_w.ny, probe_w.tau, u_in=(probe_w.ux_in, 0.0), bc=bc(probe_w),
                            storage="f32")
    pb = lbm.lbm_tune_workspace_bytes(probe)
    stream = torch.cuda.Stream()
    pws = torch.empty(pb, dtype=torch.uint8, device="cuda")
    tuning = lbm.lbm_tune(probe, probe_w.mask, pws, pb, stream.cuda_stream)
    del pws
    params = [lbm.make_params(w.nx, w.ny, w.tau, u_in=(w.ux_in, 0.0), bc=bc(w), storage="f32",
                              layout=lbm.LBM_AUTO, algo=lbm.LBM_AUTO) for w in ws]
    b = lbm.Batch(params, [w.mask for w in ws], stream=stream, tuning=tuning)
    for c, w in enumerate(ws):
        b.init(c, None, w.ux0, w.uy0)
    cells = sum(w.cells for w in ws)
    k = max(100, min(args.steps, 1000) // 100 * 100)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b.step(100).sync()
    torch.cuda.synchronize()
    e0.record(stream)
    b.step(k)
    e1.record(stream)
    e1.synchronize()
    b.sync()
    t_batch = e0.elapsed_time(e1) / 1e3
    info = b.info()
    chosen = {}
    for p in b.params:
        key = f"{['stream', 'bundle', 'collision'][p.layout]}/{['lptl', 'nptl', 'npol', 'nsol'][p.algo]}"
        chosen[key] = chosen.get(key, 0) + 1
    b.close()
    del b
    singles = []
    for w, p in zip(ws, [lbm.lbm_batch_plan([q], tuning)[0] for q in params]):
        lat = lbm.Lattice(w.nx, w.ny, w.tau, w.mask, stream=stream, u_in=(w.ux_in, 0.0), bc=bc(w),
                          storage="f32", layout=p.layout, algo=p.algo,
                          tile=(p.tile_x, p.tile_y))
        lat.init(None, w.ux0, w.uy0)
        singles.append(lat)
    for lat in singles:
        lbm.lbm_step(lat.h, 100, False)
    torch.cuda.synchronize()
    e0.record(stream)
    for lat in singles:
        lbm.lbm_step(lat.h, k, False)
    e1.record(stream)
    e1.synchronize()
    t_seq = e0.elapsed_time(e1) / 1e3
    for lat in singles:
        lat.close()
    del singles
    torch.cuda.empty_cache()
    return {"cases": len(ws), "nodes": cells, "steps": k,
            "batched_MLUPS": cells * k / t_batch / 1e6, "sequential_MLUPS": cells * k / t_seq / 1e6,
            "speedup": t_seq / t_batch, "tiles": info["tiles"], "grid": info["grid"],
            "chosen": chosen,
            "tuned_ns_per_node": [[round(tuning.ns_per_cell[l][a], 5) for a in range(4)] for l in range(3)]}


def batched3(args, torch, ncases: int = 512, edges=(12, 48), algo: str = "lptl", tile=(0, 0, 0)):
    """512 independent D3Q19 boxes (seeded edges 12-48 per axis, random
    sphere packings r 2-5 of solid fraction 0.2, periodic, tau in
    [0.6, 1.2], g_x = 1e-6, FP32 bundle layout, LPTL): one launch per update
    over the work items of every box (graphs of 64 updates) against the same
    boxes run one after another as single boxes (each lbm3_step(K), graphs
    of 64)."""
    from paper_2607_20650_gb300 import geometry as G, lbm
    r = G.SplitMix64(21, 3)
    dims = r.integers(3 * ncases, edges[0], edges[1]).reshape(ncases, 3)
    taus = r.uniform(ncases, 0.6, 1.2)
    kw = dict(storage="f32", layout="bundle", algo=algo, tile=tuple(tile), force=(1e-6, 0.0, 0.0))
    masks = [G.porous_spheres(int(nx), int(ny), int(nz), 100 + c, 2.0, 5.0, 0.2) for c, (nx, ny, nz) in enumerate(dims)]
    params = [lbm.make_params3(int(nx), int(ny), int(nz), float(t), **kw) for (nx, ny, nz), t in zip(dims, taus)]
    stream = torch.cuda.Stream()
    b = lbm.Batch3(params, masks, stream=stream)
    info = b.info()
    k = 128
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b.step(64).sync()
    torch.cuda.synchronize()
    e0.record(stream)
    b.step(k)
    e1.record(stream)
    e1.synchronize()
    b.sync()
    t_batch = e0.elapsed_time(e1) / 1e3
    b.close()
    del b
    singles = []
    for (nx, ny, nz), t, m in zip(dims, taus, masks):
        singles.append(lbm.Lattice3(int(nx), int(ny), int(nz), float(t), m, stream=stream, **kw))
    for lat in singles:
        lbm.lbm3_step(lat.h, 64, False)
    torch.cuda.synchronize()
    e0.record(stream)
    for lat in singles:
        lbm.lbm3_step(lat.h, k, False)
    e1.record(stream)
    e1.synchronize()
    t_seq = e0.elapsed_time(e1) / 1e3
    for lat in singles:
        lat.close()
    del singles
    torch.cuda.empty_cache()
    hbm, _ = peaks()
    gbs = info["bytes_per_update"] * k / t_batch / 1e9
    return {"cases": ncases, "edges": list(edges), "algo": algo, "tile": list(tile),
            "nodes": info["cells"], "fluid_nodes": info["fluid_cells"], "steps": k,
            "work_items": info["items"], "batched_MLUPS": info["cells"] * k / t_batch / 1e6,
            "sequential_MLUPS": info["cells"] * k / t_seq / 1e6, "speedup": t_seq / t_batch,
            "GBps_algorithmic": gbs, "frac_of_measured_hbm": gbs / hbm}


def e2e(args, mask, torch, world=1):
    """Through the C ABI with page-locked host buffers: create (mask H2D),
    init, K updates, moments D2H (three FP64 arrays), all inside the timed
    region. With several ranks (replicas) the ranks start together and the
    job's time is the slowest rank's."""
    from paper_2607_20650_gb300 import lbm
    nx, ny = args.nx, args.ny
    N = nx * ny
    k = args.steps
    p = lbm.make_params(nx, ny, 0.9, force=(1e-6, 0.0), bc=(lbm.PERIODIC,) * 4,
                        layout=args.layout, algo="nptl", storage="f32", tile=(32, 4))
    nbytes = lbm.lbm_workspace_bytes(p)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    # inputs and outputs in page-locked host memory (the moments are widened
    # to FP64 on the device and written over the CPU-GPU link)
    host_mask = torch.empty(N, dtype=torch.uint8, pin_memory=True).numpy()
    host_mask[:] = mask.reshape(-1)
    rho, ux, uy = (torch.empty(N, dtype=torch.float64, pin_memory=True).numpy() for _ in range(3))
    stream = torch.cuda.Stream().cuda_stream
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    t = time.perf_counter()
    h = lbm.lbm_create(p, host_mask, ws, nbytes, stream)       # synchronous
    t1 = time.perf_counter()
    lbm.lbm_step(h, k, True)
    lbm.lbm_sync(h)
    t2 = time.perf_counter()
    lib = lbm.load()
    st = lib.lbm_read_moments(h, rho.ctypes.data, ux.ctypes.data, uy.ctypes.data)
    dt = time.perf_counter() - t
    parts = {"create_and_init_ms": (t1 - t) * 1e3, "updates_ms": (t2 - t1) * 1e3,
             "read_moments_ms": (t + dt - t2) * 1e3}
    lbm.lbm_destroy(h)
    assert st == 0
    del ws
    torch.cuda.empty_cache()
    if world > 1:
        dt = max_over_ranks(dt, "cuda")
    return {"value": N * k * world / dt / 1e6, "unit": "MLUPS", "h2d_bytes_per_step": N * world / k,
            "d2h_bytes_per_step": 3 * 8 * N * world / k, "steps": k, "replicas": world,
            "host_buffers": "page-locked", "parts": parts,
            "region": "lbm_create(host mask) + init + K updates + lbm_read_moments(host f64)"}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.lattice == "d3q19":
        run_d3q19(args)
    elif args.batch_only:
        import torch
        from paper_2607_20650_gb300 import build, lbm
        build.build()
        lbm.load()
        b = batched(args, torch)
        print(json.dumps({"metric": "batched D2Q9 BGK MLUPS (256 channels)", "value": b["batched_MLUPS"],
                          "unit": "MLUPS", "n_gpus": 1, "steps": b["steps"], "higher_is_better": True,
                          "config": {"workload": "256 seeded channels, 37.1M nodes, FP32"}, "batched": b}))
    elif args.batch3_only:
        import torch
        from paper_2607_20650_gb300 import build, lbm
        build.build()
        lbm.load()
        b = batched3(args, torch)
        print(json.dumps({"metric": "batched D3Q19 BGK MLUPS (512 boxes)", "value": b["batched_MLUPS"],
                          "unit": "MLUPS", "n_gpus": 1, "steps": b["steps"], "higher_is_better": True,
                          "config": {"workload": "512 seeded boxes of 12-48 nodes per edge, 13.8M nodes, FP32"},
                          "batched_d3q19": b}))
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
