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
    64) for 2 steps.

The per-cell work of a step does not depend on the grid size, so a band or a
slab gives the per-step throughput of the whole grid; it keeps the run within
a few minutes and within host memory.

    python oracle/time_oracle.py [--quick]   # prints one JSON object
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


def main(quick=False):
    cores = os.cpu_count() or 1
    cases = [
        ("c1_film_128x256", W.c1_parity, 1000, 200),
        ("c2_film_2048x4096 (band 2048x256)",
         lambda: W.film_boiling_2d(2048, 256, modes=8, seed=1, y0=64.0, paper=True, phi_wall=(1.0, 0.0)), 3, 1),
        ("c3_film_256x256x512 (slab 256x256x64)",
         lambda: W.film_boiling_3d(256, 256, 64, modes=4, seed=2, z0=32.0, paper=True, phi_wall=(1.0, 0.0)),
         2, 1),
    ]
    if quick:
        cases = [(n, mk, max(1, a // 100), max(1, b // 100)) for n, mk, a, b in cases]
    out = {"cpu": cpu_model(), "nproc": cores, "torch_threads_all": cores, "results": []}
    for name, make, steps_all, steps_one in cases:
        w = make()
        torch.set_num_threads(cores)
        v_all, t_all = mlups(w, steps_all)
        torch.set_num_threads(1)
        v_one, t_one = mlups(w, steps_one)
        out["results"].append({"workload": name, "cells": w.cells,
                               "all_cores": {"MLUPS": v_all, "steps": steps_all, "seconds": t_all},
                               "one_core": {"MLUPS": v_one, "steps": steps_one, "seconds": t_one}})
        print(json.dumps(out["results"][-1]), file=sys.stderr, flush=True)
    torch.set_num_threads(cores)
    print(json.dumps(out))


if __name__ == "__main__":
    main(quick="--quick" in sys.argv)
