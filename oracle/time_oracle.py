"""Time the FP64 oracle on the host cores, single-threaded and on all cores.

Test infrastructure, like the rest of oracle/: this script only measures how
fast the plain CPU reference steps the benchmark workloads, as the CPU
baseline of the measurements.  MLUPS = cells x steps / wall seconds, after
one untimed warm-up step, for

  * the 128 x 256 film (ratio 10), 1000 steps on all cores and 200 steps on
    one core;
  * the 2048 x 4096 film: a band of the bottom 256 rows (2048 x 256, the film
    and the interface) for 3 steps;
  * the 256 x 256 x 512 3D film: a slab of the bottom 64 layers (256 x 256 x
    64) for 2 steps;
  * the 512 x 512 evaporating droplet's gradient (oracle.adjoint, reverse mode
    through the FP64 step, recomputing 10-step segments to bound memory): one
    100-step segment on all cores, 10 steps on one core; MLUPS counts the
    forward steps of the segment (each taken forward and back).

The per-cell work of a step does not depend on the grid size, so a band or a
slab gives the per-step throughput of the whole grid; it keeps the run within
a few minutes and within host memory.

    python oracle/time_oracle.py [--quick] [--adjoint-only]   # prints one JSON object
"""
import json
import os
import platform
import sys
import time

import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import model as M  # noqa: E402


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or "unknown"


def mlups(w, steps):
    P, G = M.Params.from_dict(w.params), M.Grid(w.n, w.periodic)
    st = M.init_state(w.phi0, w.T0, P, G, p0=w.p0)
    st = M.step(st, P, G)                     # warm-up
    t0 = time.perf_counter()
    for _ in range(steps):
        st = M.step(st, P, G)
    dt = time.perf_counter() - t0
    return w.cells * steps / dt / 1e6, dt


def adjoint_mlups(w, steps):
    """MLUPS of the oracle's gradient over `steps` forward steps (forward and
    reverse), the target being the initial phase field shifted by 2 cells."""
    import numpy as np
    from oracle import adjoint as A
    target = np.roll(w.phi0, 2, axis=1)
    t0 = time.perf_counter()
    # 10-step segments bound the memory of the reverse pass (each segment's
    # forward runs twice), as for the oracle's long reference gradients
    A.gradients(w.phi0, w.T0, w.params, M.Grid(w.n, w.periodic), steps, target, segment=10)
    dt = time.perf_counter() - t0
    return w.cells * steps / dt / 1e6, dt


def main(quick=False, adjoint_only=False):
    cores = os.cpu_count() or 1
    cases = [
        ("c1_film_128x256", W.c1_parity, 1000, 200),
        ("c2_film_2048x4096 (band 2048x256)",
         lambda: W.film_boiling_2d(2048, 256, modes=8, seed=1, y0=64.0, paper=True, phi_wall=(1.0, 0.0)), 3, 1),
        ("c3_film_256x256x512 (slab 256x256x64)",
         lambda: W.film_boiling_3d(256, 256, 64, modes=4, seed=2, z0=32.0, paper=True, phi_wall=(1.0, 0.0)),
         2, 1),
    ]
    cases.append(("c4_droplet_512x512 gradient (100-step segment)", lambda: W.c4_droplet(), 100, 10))
    if adjoint_only:
        cases = cases[-1:]
    if quick:
        cases = [(n, mk, max(1, a // 100), max(1, b // 100)) for n, mk, a, b in cases]
    out = {"cpu": cpu_model(), "nproc": cores, "torch_threads_all": cores, "results": []}
    for name, make, steps_all, steps_one in cases:
        w = make()
        run = adjoint_mlups if "gradient" in name else mlups
        torch.set_num_threads(cores)
        v_all, t_all = run(w, steps_all)
        torch.set_num_threads(1)
        v_one, t_one = run(w, steps_one)
        out["results"].append({"workload": name, "cells": w.cells,
                               "all_cores": {"MLUPS": v_all, "steps": steps_all, "seconds": t_all},
                               "one_core": {"MLUPS": v_one, "steps": steps_one, "seconds": t_one}})
        print(json.dumps(out["results"][-1]), file=sys.stderr, flush=True)
    torch.set_num_threads(cores)
    print(json.dumps(out))


if __name__ == "__main__":
    main(quick="--quick" in sys.argv, adjoint_only="--adjoint-only" in sys.argv)
