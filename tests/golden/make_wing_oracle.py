"""Writes wing_coarse_oracle.json: lift and drag of the 2x coarsened wing flow
computed by the FP64 CPU oracle alone.

Workload: NACA 2412 at 8 degrees, chord 512 on 4096 x 2048, Zou-He inlet
U = 0.05, Re = 1000, zero-gradient outflow, free-slip top and bottom,
initial velocity U on fluid nodes; 25,000 updates (the convective time of
50,000 updates at chord 1024). C_D = 2 F_x / (U^2 c), C_L = 2 F_y / (U^2 c)
from the oracle's momentum-exchange force, sampled every 250 updates over the
last 5,000: the final values and the averages of those 20 samples.

Only the oracle and the seeded input generators run here; no value comes from
the CUDA path. Run from the repository root:
    python tests/golden/make_wing_oracle.py
(about 20 minutes on 8 host cores)."""
import json
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.abspath(os.path.join(os.path.dirname(__file__), "..", "..")))

import oracle as O  # noqa: E402
from paper_2607_20650_gb300 import geometry as G  # noqa: E402

TOTAL, EVERY, WINDOW = 25000, 250, 5000


def main(out_path: str) -> None:
    w = G.wing(nx=4096, ny=2048, chord=512)
    case = O.Case(w.nx, w.ny, w.tau, ux_in=w.ux_in, bc_w=w.bc_w, bc_e=w.bc_e, bc_s=w.bc_s, bc_n=w.bc_n)
    lat = O.Lattice(case, w.mask, ux=w.ux0, uy=w.uy0)
    q = 0.5 * w.meta["U"] ** 2 * w.meta["L"]
    samples = []
    t0 = time.time()
    done = 0
    while done < TOTAL:
        k = min(EVERY, TOTAL - done)
        lat.run(k)
        done += k
        if done > TOTAL - WINDOW:
            F = lat.force(w.body)
            samples.append([float(F[0] / q), float(F[1] / q)])
    s = np.array(samples)
    rec = {
        "workload": "NACA 2412, 8 deg, chord 512, 4096x2048, U 0.05, Re 1000, tau %.17g" % w.tau,
        "updates": TOTAL, "sample_every": EVERY, "window": WINDOW, "samples": len(samples),
        "cd_cl_end": s[-1].tolist(), "cd_cl_avg": s.mean(axis=0).tolist(),
        "oracle_threads": O.omp_threads(), "seconds": round(time.time() - t0, 1),
        "made_by": "tests/golden/make_wing_oracle.py (FP64 CPU oracle only)",
    }
    with open(out_path, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main(os.path.join(os.path.dirname(os.path.abspath(__file__)), "wing_coarse_oracle.json"))
