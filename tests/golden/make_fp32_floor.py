"""Write tests/golden/c1_fp32_floor.json: the rounding floor of the method in
FP32 arithmetic on the 128 x 256 film-boiling parity case after 1000 steps.

The oracle's own step (oracle/model.py) is run twice from the same seeded
initial state, once in float64 and once with every tensor in float32; the
max-abs differences of phi, T, u and p are what FP32 arithmetic alone costs
on this trajectory, independent of any GPU code.  Only oracle/ and the input
generators are used.

    python tests/golden/make_fp32_floor.py
"""
import json
import os
import sys

import torch

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import model as M  # noqa: E402


def main(steps=1000):
    w = W.c1_parity()
    P, G = M.Params.from_dict(w.params), M.Grid(w.n, w.periodic)
    st64 = M.init_state(w.phi0, w.T0, P, G, p0=w.p0)
    st32 = {k: v.float() for k, v in st64.items()}
    for _ in range(steps):
        st64 = M.step(st64, P, G)
        st32 = M.step(st32, P, G)
    a, b = M.fields(st64, P, G), M.fields(st32, P, G)
    out = {k: float((a[k] - b[k].double()).abs().max()) for k in ("phi", "T", "p")}
    out["u"] = max(float((x - y.double()).abs().max()) for x, y in zip(a["u"], b["u"]))
    out.update(steps=steps, workload=w.name, note="max-abs difference of the oracle run in float32 vs float64")
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c1_fp32_floor.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(out)


if __name__ == "__main__":
    main()
