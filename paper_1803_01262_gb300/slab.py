"""Z-slab domain decomposition of one periodic box over several ranks.

The explicit step of Section 2.2 reads, for the update of plane k, the planes
k-2 .. k+2 of phi (the normals of planes k+-1 need their z neighbours) and the
w faces of planes k-1 and k.  So a box of nz planes splits along z into one
slab per rank: rank r owns planes [z_begin, z_end) and keeps them in a local
array of (z_end - z_begin) + 4 planes -- two halo planes below, the owned
planes, two halo planes above.  Each step

1. fills the four halo planes from the neighbouring ranks (periodic in the
   rank index: rank 0's lower halo is the last rank's two top planes), and
2. updates the owned planes, local planes [2, 2 + owned), with
   ``cdi_step_planes`` -- no periodic wrap is taken inside a slab, so every
   owned plane sees exactly the values the single-domain step sees and the
   glued result is the single-domain step's bit for bit;
3. combines the per-rank statistics (sum, min, max, violation counts) in rank
   order, so the result does not depend on message timing.

The face velocities are static: each rank copies its planes and halos of u, v
and w once.  The exchange plan (which local planes go to which rank and land
where) is computed once per rank; two transports carry it: ``DistTransport``
(torch.distributed point-to-point sends, NCCL between GPUs or gloo on the CPU)
and ``LocalTransport`` (several slabs of one process, device-to-device copies).
The update itself runs in the CUDA library; a different stepping function may
be given (the tests pass the FP64 oracle to check the partition and exchange
on the CPU).
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

HALO = 2  # planes of phi needed on each side (radius of the stencil along z)


def partition(nz: int, world: int):
    """Slabs [z_begin, z_end) of ``nz`` planes over ``world`` ranks: the first
    ``nz % world`` ranks get one plane more.  Every slab needs at least HALO
    planes (a halo must come from the neighbouring rank alone)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    if nz < HALO * world:
        raise ValueError(f"nz = {nz} gives slabs thinner than {HALO} planes on {world} ranks")
    base, extra = divmod(nz, world)
    out, z = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append((z, z + n))
        z += n
    return out


@dataclass(frozen=True)
class HaloMessage:
    """One halo message: local planes [src, src + HALO) of rank ``sender`` land in local
    planes [dst, dst + HALO) of rank ``receiver``; ``tag`` 0 fills the receiver's upper
    halo, 1 its lower halo."""
    sender: int
    receiver: int
    src: int
    dst: int
    tag: int


def halo_plan(rank: int, world: int, slabs):
    """(sends, recvs) of one rank: its two bottom owned planes go to the rank below
    (that rank's upper halo), its two top owned planes to the rank above (its lower
    halo).  Sends and receives are listed in the order both sides post them."""
    prev, nxt = (rank - 1) % world, (rank + 1) % world
    own = slabs[rank][1] - slabs[rank][0]
    n_prev = slabs[prev][1] - slabs[prev][0]
    sends = [HaloMessage(rank, prev, HALO, HALO + n_prev, 0),        # -> prev's upper halo
             HaloMessage(rank, nxt, own, 0, 1)]                        # -> next's lower halo
    n_next = slabs[nxt][1] - slabs[nxt][0]
    recvs = [HaloMessage(nxt, rank, HALO, HALO + own, 0),              # my upper halo
             HaloMessage(prev, rank, n_prev, 0, 1)]                    # my lower halo
    assert n_next >= HALO
    return sends, recvs


def local_slab(a, z_begin: int, z_end: int):
    """Planes z_begin - HALO .. z_end + HALO - 1 of a full (nz, ny, nx) array, periodic in z
    (a copy)."""
    nz = a.shape[0]
    idx = torch.arange(z_begin - HALO, z_end + HALO, device=a.device) % nz
    return a.index_select(0, idx).contiguous()


class DistTransport:
    """Halo messages between ranks of a torch.distributed process group."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)

    def exchange(self, domains):
        (d,) = domains
        dist = self.dist
        if self.world == 1:
            LocalTransport().exchange(domains)
            return
        ops = []
        for m in d.sends:
            ops.append(dist.P2POp(dist.isend, d.phi[m.src:m.src + HALO].contiguous(), m.receiver, self.group,
                                  tag=m.tag))
        bufs = []
        for m in d.recvs:
            buf = d.phi[m.dst:m.dst + HALO]   # contiguous: whole planes of a contiguous array
            bufs.append(buf)
            ops.append(dist.P2POp(dist.irecv, buf, m.sender, self.group, tag=m.tag))
        for req in dist.batch_isend_irecv(ops):
            req.wait()

    def gather_stats(self, domains):
        (d,) = domains
        dist = self.dist
        mine = torch.tensor(d.last_stats_vector(), dtype=torch.float64, device=d.phi.device)
        out = [torch.empty_like(mine) for _ in range(self.world)]
        dist.all_gather(out, mine, group=self.group)
        return [o.cpu().tolist() for o in out]


class LocalTransport:
    """All slabs in one process: halo messages are plane copies between their arrays."""

    def exchange(self, domains):
        # every message reads owned planes and writes halo planes, so the order is free
        for d in domains:
            for m in d.sends:
                dst = domains[m.receiver] if len(domains) > 1 else d
                dst.phi[m.dst:m.dst + HALO].copy_(d.phi[m.src:m.src + HALO])

    def gather_stats(self, domains):
        return [d.last_stats_vector() for d in domains]


def combine_stats(vectors, dV):
    """Rank-ordered combination of per-slab [sum, min, max, n_strict, n_tol] vectors."""
    s = 0.0
    mn, mx = float("inf"), float("-inf")
    ns = nt = 0
    for v in vectors:
        s += v[0]
        mn = min(mn, v[1])
        mx = max(mx, v[2])
        ns += int(v[3])
        nt += int(v[4])
    return dict(mass=dV * s, sum=s, min=mn, max=mx, n_strict=ns, n_tol=nt)


class SlabDomain:
    """One rank's slab of an (nz, ny, nx) periodic box.

    ``phi``, ``u``, ``v``, ``w`` are the FULL arrays (any device; only this rank's planes
    and halos are copied); ``stepper`` is None for the CUDA library (``cdi.Grid`` of the
    padded slab, ``cdi_step_planes``) or a function
    ``stepper(phi_padded, u, v, w, vel_scale) -> new phi_padded`` whose owned planes
    [HALO, HALO + owned) are used."""

    def __init__(self, rank, world, phi, u, v, w, dx, stepper=None, slabs=None):
        self.rank, self.world = rank, world
        nz, ny, nx = phi.shape
        self.shape_full = (nz, ny, nx)
        self.slabs = slabs or partition(nz, world)
        self.z_begin, self.z_end = self.slabs[rank]
        self.owned = self.z_end - self.z_begin
        self.sends, self.recvs = halo_plan(rank, world, self.slabs)
        self.dx = dx
        self.phi = local_slab(phi, self.z_begin, self.z_end)
        self.u, self.v, self.w = (local_slab(x, self.z_begin, self.z_end) for x in (u, v, w))
        self.stepper = stepper
        self._stats = None
        if stepper is None:
            from . import cdi
            self.grid = cdi.Grid(nx, ny, self.owned + 2 * HALO, dx, phi.dtype)
            # U of Eq. 24 over the slab (its own planes and halos); the caller may set a
            # global one with set_umax
            self.grid.set_velocity(self.u, self.v, self.w)
            self.other = torch.empty_like(self.phi)
        else:
            self.grid = None

    def owned_view(self):
        return self.phi[HALO:HALO + self.owned]

    def step(self, dt, eps, gamma, vel_scale=1.0):
        """Update the owned planes (halos must be current); the halos of the new state are
        stale until the next exchange."""
        if self.stepper is None:
            self.grid.step_planes(self.phi, self.other, HALO, HALO + self.owned, dt, eps, gamma, vel_scale)
            self.phi, self.other = self.other, self.phi
            self._stats = None
        else:
            new = self.stepper(self.phi, self.u, self.v, self.w, vel_scale)
            self.phi = self.phi.clone()
            self.phi[HALO:HALO + self.owned] = new[HALO:HALO + self.owned]
            self._stats = new[HALO:HALO + self.owned]

    def last_stats_vector(self):
        """[sum, min, max, n_strict, n_tol] of the owned planes after the last step."""
        if self.stepper is None:
            st = self.grid.stats()
            return [st["sum"], st["min"], st["max"], float(st["n_strict"]), float(st["n_tol"])]
        p = self._stats.double()
        tol = torch.finfo(self._stats.dtype).eps
        return [float(p.sum()), float(p.min()), float(p.max()), float(((p < 0) | (p > 1)).sum()),
                float(((p < -tol) | (p > 1 + tol)).sum())]


class SlabRun:
    """Steps a decomposed box: exchange halos, update every local slab, combine statistics.

    ``domains``: the SlabDomain(s) of this process (one per rank under torch.distributed,
    all of them with a LocalTransport)."""

    def __init__(self, domains, transport):
        self.domains = list(domains)
        self.transport = transport
        nz, ny, nx = self.domains[0].shape_full
        self.Df = (nx > 1) + (ny > 1) + (nz > 1)
        self.dV = self.domains[0].dx ** self.Df

    def step(self, dt, eps, gamma, vel_scale=1.0):
        self.transport.exchange(self.domains)
        for d in self.domains:
            d.step(dt, eps, gamma, vel_scale)

    def stats(self):
        """Statistics of the whole box after the last step (rank order)."""
        return combine_stats(self.transport.gather_stats(self.domains), self.dV)

    def gather_local(self):
        """The owned planes of this process's slabs glued in z order (LocalTransport: the
        whole box)."""
        return torch.cat([d.owned_view() for d in self.domains], dim=0)
