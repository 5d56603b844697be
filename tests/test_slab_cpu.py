"""z-slab decomposition of one periodic box (the multi-GPU path) on the CPU.

The product's plane bookkeeping (SlabLayout), halo exchange and timestep
agreement (SlabExchange over torch.distributed with gloo, 2 and 4 ranks) move
the slabs' halos; each rank steps its slab box with the FP64 oracle at the
box's cell size along z.  The own planes gathered from all ranks must equal
the whole box stepped by the oracle, bit for bit, after every step."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_1004_1680_gb300 import initial_conditions as ic
from paper_1004_1680_gb300 import slab

G = 5.0 / 3.0
DIMS = (24, 20, 64)
STEPS = 3


def _state():
    return ic.turbulence(DIMS, seed=11, dtype=torch.float64, kmin=1.0, kmax=4.0)


def test_layout_bookkeeping_and_local_exchange():
    """Cutting the slabs and exchanging their halos in one process gives every
    slab box exactly the box's planes (own and halo); own planes tile the box."""
    st = _state()
    world = 4
    lays = [slab.SlabLayout(DIMS, world, r) for r in range(world)]
    assert all(L.local_dims == (24, 20, 16 + 32) for L in lays)
    own = torch.cat([L.own_planes(L.cut(st)) for L in lays], dim=1)
    assert torch.equal(own, st)
    locs = [L.cut(st) for L in lays]
    for x in locs:                       # spoil the halos, then refill them
        x[:, :16] = -1.0
        x[:, -16:] = -1.0
    getters = [lambda z, n, x=x: x[:, z:z + n].clone() for x in locs]

    def setter(x):
        def s(z, t):
            x[:, z:z + t.shape[1]] = t
        return s
    slab.exchange_local(lays, getters, [setter(x) for x in locs])
    for L, x in zip(lays, locs):
        assert torch.equal(x, L.cut(st))
    with pytest.raises(ValueError):
        slab.SlabLayout(DIMS, 8, 0)      # 8 planes per slab < 16 halo planes


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        oracle.build()
        oracle.set_threads(2)
        oracle.set_resolution(0, 0, DIMS[2])      # the box's h along z
        L = slab.SlabLayout(DIMS, world, rank)
        local = L.cut(_state()).numpy().copy()
        ex = slab.SlabExchange(L)
        t = torch.from_numpy(local)

        def get(z, n):
            return t[:, z:z + n].clone()

        def put(z, planes):
            t[:, z:z + planes.shape[1]] = planes
        for s in range(STEPS):
            ex.exchange(get, put)
            dt = ex.agree_dt(oracle.cfl_dt(local, G, 0.7))
            oracle.step(local, dt, G)
            own = torch.from_numpy(np.ascontiguousarray(L.own_planes(t).numpy()))
            parts = [torch.empty_like(own) for _ in range(world)] if rank == 0 else None
            dist.gather(own, parts, dst=0)
            if rank == 0:
                np.save(os.path.join(out_dir, f"step{s}.npy"), torch.cat(parts, dim=1).numpy())
                np.save(os.path.join(out_dir, f"dt{s}.npy"), np.array([dt]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_gloo_slabs_reproduce_the_whole_box(tmp_path, world, oracle_lib):
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn")
    whole = _state().numpy().copy()
    for s in range(STEPS):
        dt = oracle_lib.cfl_dt(whole, G, 0.7)
        oracle_lib.step(whole, dt, G)
        assert np.load(tmp_path / f"dt{s}.npy")[0] == dt
        assert np.array_equal(np.load(tmp_path / f"step{s}.npy"), whole), s
