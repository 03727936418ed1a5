"""Helpers shared by the GPU parity tests: run a workload through the C ABI
and through the FP64 oracle from the same seeded inputs, and compare."""
import numpy as np
import torch

from oracle import model as M


def oracle_fields(w, steps, state=False):
    P, G = M.Params.from_dict(w.params), M.Grid(w.n, w.periodic)
    st = M.init_state(w.phi0, w.T0, P, G, p0=w.p0)
    st = M.run(st, P, G, steps)
    F = M.fields(st, P, G)
    out = dict(phi=F["phi"].numpy(), T=F["T"].numpy(), p=F["p"].numpy(),
               u=[u.numpy() for u in F["u"]])
    if state:
        out["state"] = st
        out["reductions"] = M.reductions(st, P, G)
    return out


def gpu_solver(w, storage="fp32", **kw):
    from paper_2003_06342_b300 import Solver
    s = Solver(w.n, w.periodic, w.params, storage=storage, **kw)
    s.init(w.phi0, w.T0, p0=w.p0)
    return s


def gpu_fields(s):
    F = s.fields()
    torch.cuda.synchronize()
    return dict(phi=F["phi"].double().cpu().numpy(), T=F["T"].double().cpu().numpy(),
                p=F["p"].double().cpu().numpy(), u=[u.double().cpu().numpy() for u in F["u"]])


def max_errors(a, b):
    err = {k: float(np.abs(a[k] - b[k]).max()) for k in ("phi", "T", "p")}
    err["u"] = max(float(np.abs(x - y).max()) for x, y in zip(a["u"], b["u"]))
    return err
