"""Slab domain decomposition (the paper's multi-GPU scheme) on CPU: the
partition, and the ghost-column exchange of the drivers in
paper_2003_06342_b300.slabs with every slab stepped by the FP64 oracle, in
one process (LocalSlabs) and on two and three gloo ranks (DistSlab).  The
owned columns must evolve bit for bit as in the undivided grid."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import workloads as W
from paper_2003_06342_b300.slabs import DistSlab, LocalSlabs, halo_width, partition, slab_columns

from _oracle_slab import KEYS, OracleSlab, undivided_state


def _film(nx=40, ny=18, **extra):
    w = W.film_boiling_2d(nx, ny, rho_ratio=10.0, y0=6.0, amplitude=1.5, phi_wall=(1.0, 0.0))
    w.params.update(**extra)
    return w


def test_partition_and_columns():
    assert partition(10, 3, 2) == [(0, 4), (4, 7), (7, 10)]
    assert partition(8, 1, 2) == [(0, 8)]
    with pytest.raises(ValueError):
        partition(5, 3, 2)                    # a slab narrower than the halo
    assert list(slab_columns(0, 4, 2, 10)) == [8, 9, 0, 1, 2, 3, 4, 5]
    assert halo_width({"grad_scheme": "biased2"}) == 3 and halo_width({}) == 2


def _assemble(slabs, shape_like):
    owned = [s.owned_state() for s in slabs]
    return {k: torch.cat([o[k] for o in owned], dim=-1) for k in KEYS}


@pytest.mark.parametrize("nslabs,extra", [(2, {}), (3, {}), (4, {"grad_scheme": "biased2"}),
                                          (3, {"collision": "trt", "trt_magic": (0.1875, 0.25, 0.25)})])
def test_local_slabs_bit_identical(nslabs, extra):
    w = _film(**extra)
    steps = 12
    h = halo_width(w.params)
    slabs = [OracleSlab(w, lo, hi, h) for lo, hi in partition(w.n[0], nslabs, h)]
    LocalSlabs(slabs).start().step(steps)
    got = _assemble(slabs, None)
    ref = undivided_state(w, steps)
    for k in KEYS:
        assert torch.equal(got[k], ref[k]), k


def test_ghost_exchange_is_needed():
    """Without the exchange the slab edges drift from the undivided run (the
    test above is not passing trivially)."""
    w = _film()
    h = halo_width(w.params)
    slabs = [OracleSlab(w, lo, hi, h) for lo, hi in partition(w.n[0], 2, h)]
    for s in slabs:
        s.step(6)
    got = _assemble(slabs, None)
    ref = undivided_state(w, 6)
    assert not torch.equal(got["g"], ref["g"])


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, steps, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = _film(nx=36)
        h = halo_width(w.params)
        lo, hi = partition(w.n[0], world, h)[rank]
        d = DistSlab(OracleSlab(w, lo, hi, h)).start().step(steps)
        out[rank] = {k: v.numpy() for k, v in d.slab.owned_state().items()}
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_bit_identical(world):
    steps = 8
    out = mp.get_context("spawn").Manager().dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), steps, out), nprocs=world,
                       start_method="spawn")
    ref = undivided_state(_film(nx=36), steps)
    for k in KEYS:
        got = np.concatenate([out[r][k] for r in range(world)], axis=-1)
        assert np.array_equal(got, ref[k].numpy()), k
