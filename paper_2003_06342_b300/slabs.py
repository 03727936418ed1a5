"""Slab domain decomposition along the periodic x axis with ghost-column
exchange: the paper's multi-GPU scheme (implementation section: the domain is
split into sub-domains along one axis, one per GPU, and neighbouring
sub-domains trade ghost layers every time step).

Each sub-domain (a "slab") owns columns [lo, hi) of the global grid and is
stepped by the ordinary single-grid kernels on a grid of width
(hi - lo) + 2 h: its owned columns plus h ghost columns on each side, with
the slab's own x axis periodic (a wrap there only ever reaches ghost
columns).  After every step each slab receives its neighbours' h outermost
owned columns into its ghosts (the whole stored state of those columns:
populations, phi^{n-1} and the lagged source).  The owned columns then evolve
exactly as in the undivided grid, bit for bit:

  * a cell's update reads its own populations and phi on a ring of radius 1
    (central gradient) or 2 (biased gradient), and phi of a cell needs only
    that cell's g populations and lagged source;
  * so the innermost ghost column (x = lo - 1) updates correctly when the
    h = 2 (or 3) columns beyond it hold the true state, and it is the only
    ghost column that pushes populations into the owned region; the outer
    ghost columns compute garbage that never reaches an owned cell and is
    overwritten by the next exchange.

The exchange moves 2 h columns of the full state per slab and step, more
than the populations that actually cross a cut (3 of 9 per set in 2D); the
wider halo keeps the step kernels unchanged.

Two transports move the column blocks: `LocalSlabs` keeps every slab in
this process (device-to-device copies on one GPU, the emulated
multi-domain run), `DistSlab` keeps one slab per rank and trades blocks with
torch.distributed point-to-point sends (gloo for CPU tensors, NCCL for CUDA
tensors).  A slab is any object with `step(n)`, `pack(x0, ncols)` (a tensor)
and `unpack(x0, ncols, buf)`; `SolverSlab` is the CUDA one.
"""
import numpy as np
import torch

from .solver import Solver


def halo_width(params):
    """Ghost columns a slab needs on each side: 2 for the central gradient, 3
    for the second-order biased one (its stencil reaches two cells)."""
    gs = params.get("grad_scheme", "central")
    biased = gs in ("biased2", 1)
    return 3 if biased else 2


def partition(nx, nslabs, halo):
    """Owned column ranges [(lo, hi), ...] of nslabs slabs covering [0, nx),
    as equal as possible (the first nx % nslabs slabs one column wider)."""
    if nslabs < 1:
        raise ValueError("need at least one slab")
    base, extra = divmod(nx, nslabs)
    if base < halo:
        raise ValueError(f"{nslabs} slabs of a {nx}-wide grid are narrower than the halo ({halo})")
    out, lo = [], 0
    for k in range(nslabs):
        hi = lo + base + (1 if k < extra else 0)
        out.append((lo, hi))
        lo = hi
    return out


def slab_columns(lo, hi, halo, nx):
    """Global x index of every column of a slab's grid, ghosts included
    (wrapped over the periodic axis)."""
    return np.arange(lo - halo, hi + halo) % nx


def _take_x(a, cols):
    return None if a is None else np.ascontiguousarray(np.take(np.asarray(a), cols, axis=-1))


class SolverSlab:
    """One slab stepped by the CUDA library (a Solver on the slab's grid)."""

    def __init__(self, n, periodic, params, lo, hi, halo, storage="fp32", device="cuda", stream=None):
        if not periodic[0]:
            raise ValueError("slabs split the x axis, which must be periodic")
        self.lo, self.hi, self.halo = lo, hi, halo
        self.width = hi - lo
        self.nx_global = n[0]
        self.cols = slab_columns(lo, hi, halo, n[0])
        sub = (self.width + 2 * halo,) + tuple(n[1:])
        self.solver = Solver(sub, periodic, params, storage=storage, device=device, stream=stream)

    def init(self, phi0, T0, u0=None, p0=None):
        u = None if u0 is None else [_take_x(ua, self.cols) for ua in u0]
        self.solver.init(_take_x(phi0, self.cols), _take_x(T0, self.cols), u0=u, p0=_take_x(p0, self.cols))
        return self

    def step(self, n=1):
        self.solver.step(n)

    def pack(self, x0, ncols):
        return self.solver.pack_columns(x0, ncols)

    def unpack(self, x0, ncols, buf):
        self.solver.unpack_columns(x0, ncols, buf)

    def fields(self):
        """Fields of the owned columns (dict of CUDA tensors, x last)."""
        F = self.solver.fields()
        sl = slice(self.halo, self.halo + self.width)
        return dict(phi=F["phi"][..., sl], T=F["T"][..., sl], p=F["p"][..., sl],
                    u=[u[..., sl] for u in F["u"]])


class LocalSlabs:
    """Every slab in this process; the exchange is a pack on one slab and an
    unpack on its neighbour (device-to-device on one GPU)."""

    def __init__(self, slabs):
        self.slabs = list(slabs)
        self.steps = 0

    def exchange(self):
        S = self.slabs
        m = len(S)
        # pack everything first: a slab's owned columns and its ghosts are
        # disjoint, so the order against the unpacks does not matter, but
        # packing first keeps the blocks of one exchange from one time level
        left = [s.pack(s.halo, s.halo) for s in S]             # to the left neighbour
        right = [s.pack(s.width, s.halo) for s in S]           # to the right neighbour
        for k, s in enumerate(S):
            s.unpack(0, s.halo, right[(k - 1) % m])
            s.unpack(s.width + s.halo, s.halo, left[(k + 1) % m])

    def start(self):
        """Fill every ghost column from its owner (call once after init)."""
        self.exchange()
        return self

    def step(self, n=1):
        for _ in range(n):
            for s in self.slabs:
                s.step(1)
            self.exchange()
            self.steps += 1
        return self

    def fields(self):
        """The undivided fields (owned columns of every slab, in x order)."""
        parts = [s.fields() for s in self.slabs]
        cat = lambda xs: torch.cat(xs, dim=-1)
        return dict(phi=cat([p["phi"] for p in parts]), T=cat([p["T"] for p in parts]),
                    p=cat([p["p"] for p in parts]),
                    u=[cat([p["u"][a] for p in parts]) for a in range(len(parts[0]["u"]))])


class DistSlab:
    """This rank's slab of a decomposition over a torch.distributed group:
    rank r owns slab r, its neighbours are ranks r - 1 and r + 1 (mod the
    world size).  Each exchange posts two sends and two receives; the send
    to the left neighbour carries tag 0 and the one to the right tag 1, and
    both are posted before the receives in the same order on every rank, so
    the blocks also match where a transport ignores tags and pairs messages
    in posting order (NCCL), including a world of two where both neighbours
    are the same rank."""

    def __init__(self, slab, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.slab = slab
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.steps = 0

    def _peer(self, r):
        return self.dist.get_global_rank(self.group, r) if self.group is not None else r

    def exchange(self):
        s = self.slab
        h = s.halo
        to_left = s.pack(h, h)
        to_right = s.pack(s.width, h)
        if self.world == 1:
            s.unpack(0, h, to_right)
            s.unpack(s.width + h, h, to_left)
            return
        left, right = self._peer((self.rank - 1) % self.world), self._peer((self.rank + 1) % self.world)
        from_right = torch.empty_like(to_left)
        from_left = torch.empty_like(to_right)
        if to_left.is_cuda:
            torch.cuda.current_stream(to_left.device).synchronize()
        d = self.dist
        reqs = [d.isend(to_left, left, group=self.group, tag=0),
                d.isend(to_right, right, group=self.group, tag=1),
                d.irecv(from_right, right, group=self.group, tag=0),
                d.irecv(from_left, left, group=self.group, tag=1)]
        for r in reqs:
            r.wait()
        s.unpack(0, h, from_left)
        s.unpack(s.width + h, h, from_right)

    def start(self):
        self.exchange()
        return self

    def step(self, n=1):
        for _ in range(n):
            self.slab.step(1)
            self.exchange()
            self.steps += 1
        return self
