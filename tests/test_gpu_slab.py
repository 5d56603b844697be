"""z-slab decomposition on the GPU: slab boxes (own planes plus 16 halo
planes at each end, the box's cell size along z, CFL rate over own planes)
exchanged through mhd_copy_planes and stepped by the library give the own
planes of the whole box's step bit for bit, with the same timestep."""
import pytest
import torch

from paper_1004_1680_gb300 import initial_conditions as ic
from paper_1004_1680_gb300 import slab

pytestmark = pytest.mark.gpu

DIMS = (24, 20, 64)


# (24, 20, 64): register-load sweeps; (32, 32, 64): every y and z sweep of
# the whole box and of the slab boxes (16 own + 32 halo planes or more) is
# TMA-staged, so both sides take the same arithmetic
@pytest.mark.parametrize("dims", [DIMS, (32, 32, 64)])
@pytest.mark.parametrize("world", [1, 2, 4])
def test_gpu_slabs_reproduce_the_whole_box(world, dims):
    from paper_1004_1680_gb300 import mhd
    DIMS = dims
    st = ic.turbulence(DIMS, seed=12, dtype=torch.float64, kmin=1.0, kmax=4.0).to(torch.float32).cuda()
    whole = mhd.Box(*DIMS)
    whole.set_state(st)
    lays = [slab.SlabLayout(DIMS, world, r) for r in range(world)]
    boxes = [slab.make_box(L) for L in lays]
    for L, b in zip(lays, boxes):
        b.set_state(L.cut(st))
    getters = [lambda z, n, b=b: b.get_planes(z, n) for b in boxes]
    setters = [lambda z, t, b=b: b.set_planes(z, t) for b in boxes]
    for _ in range(3):
        slab.exchange_local(lays, getters, setters)
        dt = min(b.cfl_dt(0.7) for b in boxes)
        assert dt == whole.cfl_dt(0.7)
        for b in boxes:
            b.step(dt)
        whole.step(dt)
        own = torch.cat([L.own_planes(b.get_state()) for L, b in zip(lays, boxes)], dim=1)
        assert torch.equal(own, whole.get_state())
    for b in boxes:
        b.close()
    whole.close()


def test_planes_round_trip_and_bounds():
    from paper_1004_1680_gb300 import mhd
    st = ic.turbulence((16, 8, 12), seed=1, dtype=torch.float32).cuda()
    b = mhd.Box(16, 8, 12)
    b.set_state(st)
    assert torch.equal(b.get_planes(3, 4), st[:, 3:7])
    b.set_planes(0, st[:, 8:12].contiguous())
    got = b.get_state()
    assert torch.equal(got[:, :4], st[:, 8:12]) and torch.equal(got[:, 4:], st[:, 4:])
    with pytest.raises(mhd.MHDError):
        b.get_planes(10, 4)
    with pytest.raises(mhd.MHDError):
        b.set_interior(2, 5, 5)
    b.close()
