"""A slab of the decomposition stepped by the FP64 oracle (CPU), for testing
the decomposition's host logic (partition, ghost exchange, the point-to-point
pairing over gloo) without a GPU.  It offers the interface the drivers in
paper_2003_06342_b300.slabs expect: step, pack, unpack, halo, width."""
import numpy as np
import torch

from oracle import model as M
from paper_2003_06342_b300.slabs import slab_columns

KEYS = ("f", "g", "s", "phi_prev", "q_prev")


class OracleSlab:
    def __init__(self, w, lo, hi, halo):
        self.lo, self.hi, self.halo, self.width = lo, hi, halo, hi - lo
        cols = slab_columns(lo, hi, halo, w.n[0])
        n = (self.width + 2 * halo,) + tuple(w.n[1:])
        self.P, self.G = M.Params.from_dict(w.params), M.Grid(n, w.periodic)
        take = lambda a: None if a is None else np.ascontiguousarray(np.take(a, cols, axis=-1))
        self.st = M.init_state(take(w.phi0), take(w.T0), self.P, self.G, p0=take(w.p0))

    def step(self, n=1):
        self.st = M.run(self.st, self.P, self.G, n)

    def pack(self, x0, ncols):
        return torch.cat([self.st[k][..., x0:x0 + ncols].reshape(-1) for k in KEYS])

    def unpack(self, x0, ncols, buf):
        off = 0
        for k in KEYS:
            part = self.st[k][..., x0:x0 + ncols]
            n = part.numel()
            self.st[k][..., x0:x0 + ncols] = buf[off:off + n].reshape(part.shape)
            off += n

    def owned_state(self):
        sl = slice(self.halo, self.halo + self.width)
        return {k: self.st[k][..., sl].clone() for k in KEYS}


def undivided_state(w, steps):
    P, G = M.Params.from_dict(w.params), M.Grid(w.n, w.periodic)
    return M.run(M.init_state(w.phi0, w.T0, P, G, p0=w.p0), P, G, steps)
