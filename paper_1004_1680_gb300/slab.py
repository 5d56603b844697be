"""One periodic box sharded over ranks as slabs along z (one rank per GPU).

The paper evolves one box on one processor and names running across nodes
as future work (Section VI).  A box of nz planes splits into `world` slabs of
nz/world planes.  Each rank's slab box holds its own planes plus `halo` planes
at each end, copies of the neighbouring slabs' planes (periodic along z):

    local plane  0 .. H-1            halo: the planes below (rank - 1)
                 H .. H+L-1          own planes z0 .. z0+L-1 of the box
                 H+L .. L+2H-1       halo: the planes above (rank + 1)

with L = nz/world, z0 = rank*L, H = halo.  A full step of the Section II.B
schedule reaches 14 cells along any axis (fluid stencil 3 cells per sweep,
one pencil across per magnetic sweep), so with H >= 14 one exchange per
step makes the own planes of the slab step exactly the box's step: before
each step every rank sends its lowest H own planes down and its highest H
own planes up and receives both halos; the timestep is the minimum of the
ranks' CFL timesteps (each over its own cells), which is the box's.  The slab
box keeps the box's cell size along z (cells per unit length nz).

SlabLayout does the plane bookkeeping; SlabExchange moves the halos over
torch.distributed (NCCL for CUDA tensors, gloo for CPU tensors) and agrees
on the timestep; exchange_local does the same for several slabs held by
one process.  The stepping itself is the caller's (an mhd.Box per slab).
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

HALO = 16  # >= 14, the reach of one full step


@dataclass(frozen=True)
class SlabLayout:
    """Planes of rank `rank`'s slab of a periodic (nx, ny, nz) box cut into
    `world` slabs along z, with `halo` halo planes at each end."""
    dims: tuple
    world: int
    rank: int
    halo: int = HALO

    def __post_init__(self):
        nx, ny, nz = self.dims
        if self.world < 1 or not 0 <= self.rank < self.world:
            raise ValueError("need 0 <= rank < world")
        if nz % self.world:
            raise ValueError("nz must be a multiple of the number of slabs")
        if nz // self.world < self.halo:
            raise ValueError("each slab needs at least `halo` own planes")

    @property
    def own(self) -> int:
        """Own planes per slab, L."""
        return self.dims[2] // self.world

    @property
    def z0(self) -> int:
        """First own plane in the box."""
        return self.rank * self.own

    @property
    def local_dims(self) -> tuple:
        """(nx, ny, L + 2H): the slab box."""
        return (self.dims[0], self.dims[1], self.own + 2 * self.halo)

    @property
    def prev(self) -> int:
        return (self.rank - 1) % self.world

    @property
    def next(self) -> int:
        return (self.rank + 1) % self.world

    def box_planes(self) -> torch.Tensor:
        """Box plane index of every local plane (periodic)."""
        return (torch.arange(self.own + 2 * self.halo) + self.z0 - self.halo) % self.dims[2]

    def cut(self, state: torch.Tensor) -> torch.Tensor:
        """The slab box (own and halo planes) of a whole-box state (8, nz, ny, nx)."""
        return state[:, self.box_planes()].contiguous()

    def own_planes(self, local: torch.Tensor) -> torch.Tensor:
        """The own planes of a slab-box state (8, L + 2H, ny, nx)."""
        return local[:, self.halo:self.halo + self.own]

    # local plane ranges of the exchange: (first plane, count)
    def send_down(self):
        """Lowest H own planes: the halo above the previous slab."""
        return self.halo, self.halo

    def send_up(self):
        """Highest H own planes: the halo below the next slab."""
        return self.own, self.halo

    def halo_below(self):
        return 0, self.halo

    def halo_above(self):
        return self.halo + self.own, self.halo


class SlabExchange:
    """Halo exchange and timestep agreement of one rank over a
    torch.distributed process group (the default group unless given)."""

    TAG_DOWN, TAG_UP = 0, 1

    def __init__(self, layout: SlabLayout, group=None):
        self.L = layout
        self.group = group

    def exchange(self, get_planes, set_planes):
        """get_planes(z, n) -> (8, n, ny, nx) tensor of local planes z..z+n-1;
        set_planes(z, tensor) writes them.  Sends this rank's lowest and
        highest H own planes to the previous and next rank and fills both
        halos from them."""
        import torch.distributed as dist
        L = self.L
        down = get_planes(*L.send_down())
        up = get_planes(*L.send_up())
        if L.world == 1:  # the box is periodic: a single slab is its own neighbour
            set_planes(L.halo_above()[0], down)
            set_planes(L.halo_below()[0], up)
            return
        above = torch.empty_like(down)
        below = torch.empty_like(up)
        # per peer the operations are matched in order (NCCL) or by tag (gloo):
        # a rank's first receive from `next` is next's downward send, its
        # second from `prev` is prev's upward send
        ops = [dist.P2POp(dist.isend, down, L.prev, self.group, self.TAG_DOWN),
               dist.P2POp(dist.isend, up, L.next, self.group, self.TAG_UP),
               dist.P2POp(dist.irecv, above, L.next, self.group, self.TAG_DOWN),
               dist.P2POp(dist.irecv, below, L.prev, self.group, self.TAG_UP)]
        for r in dist.batch_isend_irecv(ops):
            r.wait()
        set_planes(L.halo_above()[0], above)
        set_planes(L.halo_below()[0], below)

    def agree_dt(self, dt_local: float, device="cpu") -> float:
        """The box's CFL timestep: the smallest of the ranks' (each computed
        over its own cells; dt = 2 cfl / rate is monotone in the rate)."""
        if self.L.world == 1:
            return float(dt_local)
        import torch.distributed as dist
        t = torch.tensor([float(dt_local)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MIN, group=self.group)
        return float(t.item())


def exchange_local(layouts, getters, setters):
    """The halo exchange of several slabs held by one process (slab r has
    layouts[r], getters[r], setters[r]): every slab's halos from its
    neighbours' own planes."""
    sent = [(g(*L.send_down()), g(*L.send_up())) for L, g in zip(layouts, getters)]
    for L, s in zip(layouts, setters):
        s(L.halo_above()[0], sent[L.next][0])
        s(L.halo_below()[0], sent[L.prev][1])


def make_box(layout: SlabLayout, gamma: float = 5.0 / 3.0, stream=None):
    """An mhd.Box for the slab: the slab box's cells, the box's cell size
    along z, and the CFL rate over the own planes only."""
    from . import mhd
    nx, ny, nzl = layout.local_dims
    box = mhd.Box(nx, ny, nzl, gamma=gamma, stream=stream)
    box.set_resolution(0.0, 0.0, float(layout.dims[2]))
    box.set_interior(2, layout.halo, layout.halo + layout.own)
    return box
