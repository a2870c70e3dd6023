"""Slab decomposition of one simulation domain across ranks, host side: the
halo exchange and the migration of one iteration (the aura update of the
thesis's distributed engine, without its serialization or delta encoding).

The domain is cut into equal slabs along z; rank r owns the agents whose
center lies in [edges[r], edges[r + 1]) (the outermost slabs are open).
Before an iteration every rank sends the agents within `width` of a slab
face to the neighbour across that face; `width` at least the largest
diameter puts every interaction partner of an owned agent (Eq 4.1 needs a
distance below r_i + r_j) on the owner's rank.  Each rank then steps its
owned agents together with the received ones (in the library: as ghosts,
read-only neighbours), keeps the owned agents' results, and sends the
agents that left its slab to their new owner.

Messages are arrays of rows (ID, x, y, z, diameter) in float64 (IDs below
2^53 are exact), exchanged with torch.distributed point-to-point calls
(gloo on the CPU; the same calls move CUDA tensors under NCCL).  The pack,
unpack, halo and migration rules are plain functions, testable without any
process group.
"""
from __future__ import annotations

import numpy as np

ROW = 5  # id, x, y, z, diameter


class Slabs:
    """Equal slabs along z between z_lo and z_hi for `world` ranks."""

    def __init__(self, z_lo: float, z_hi: float, world: int):
        if world < 1 or not z_hi > z_lo:
            raise ValueError("need world >= 1 and z_hi > z_lo")
        self.world = world
        self.edges = np.linspace(z_lo, z_hi, world + 1)

    @property
    def width(self) -> float:
        return float(self.edges[1] - self.edges[0])

    def owner(self, z) -> np.ndarray:
        """Rank owning each z (open outermost slabs)."""
        return np.searchsorted(self.edges[1:-1], np.asarray(z, dtype=np.float64), side="right")


def pack(ids, xyz, d) -> np.ndarray:
    """Rows (id, x, y, z, d), float64."""
    ids = np.asarray(ids, dtype=np.int64)
    if ids.size and int(ids.max()) >= 2 ** 53:
        raise ValueError("IDs must stay below 2^53")
    out = np.empty((ids.shape[0], ROW))
    out[:, 0] = ids
    out[:, 1:4] = xyz
    out[:, 4] = d
    return out


def unpack(rows):
    """(ids, xyz, d) of packed rows."""
    rows = np.asarray(rows, dtype=np.float64).reshape(-1, ROW)
    return rows[:, 0].astype(np.int64), rows[:, 1:4].copy(), rows[:, 4].copy()


def halo_masks(z, slabs: Slabs, rank: int, width: float):
    """Owned agents to send down (within width above the lower face) and up
    (within width below the upper face); empty at the domain's ends."""
    z = np.asarray(z, dtype=np.float64)
    down = np.zeros(z.shape, bool)
    up = np.zeros(z.shape, bool)
    if rank > 0:
        down = z < slabs.edges[rank] + width
    if rank < slabs.world - 1:
        up = z >= slabs.edges[rank + 1] - width
    return down, up


def merge_by_id(ids, xyz, d):
    """The agents in ascending ID order (the order of every sum over
    neighbours in the plain definition)."""
    order = np.argsort(ids, kind="stable")
    return ids[order], xyz[order], d[order]


def _swap(dist, rows_down, rows_up, rank, world):
    """Send rows_down to rank - 1 and rows_up to rank + 1; return what the
    neighbours sent (from below, from above).  Counts go first."""
    import torch
    reqs = []
    keep = []  # buffers of the sends in flight
    got = {}
    cnt_in = {}
    for peer, rows in ((rank - 1, rows_down), (rank + 1, rows_up)):
        if 0 <= peer < world:
            keep.append(torch.tensor([rows.shape[0]], dtype=torch.int64))
            reqs.append(dist.isend(keep[-1], peer))
            cnt_in[peer] = torch.zeros(1, dtype=torch.int64)
            reqs.append(dist.irecv(cnt_in[peer], peer))
    for r in reqs:
        r.wait()
    reqs = []
    for peer, rows in ((rank - 1, rows_down), (rank + 1, rows_up)):
        if 0 <= peer < world:
            if rows.shape[0]:
                keep.append(torch.from_numpy(np.ascontiguousarray(rows)))
                reqs.append(dist.isend(keep[-1], peer))
            n = int(cnt_in[peer].item())
            got[peer] = torch.zeros((n, ROW), dtype=torch.float64)
            if n:
                reqs.append(dist.irecv(got[peer], peer))
    for r in reqs:
        r.wait()
    below = got[rank - 1].numpy() if rank - 1 in got else np.zeros((0, ROW))
    above = got[rank + 1].numpy() if rank + 1 in got else np.zeros((0, ROW))
    return below, above


class SlabDomain:
    """This rank's owned agents and one iteration with halo exchange and
    migration.  `engine(xyz, d, ghost)` steps a set of agents (in ascending
    ID order; ghost marks the halo agents, which the engine may leave in
    place) by one iteration and returns their new positions."""

    def __init__(self, slabs: Slabs, rank: int, ids, xyz, d):
        self.slabs, self.rank = slabs, rank
        mine = slabs.owner(np.asarray(xyz)[:, 2]) == rank
        self.ids = np.asarray(ids, dtype=np.int64)[mine]
        self.xyz = np.asarray(xyz, dtype=np.float64)[mine]
        self.d = np.asarray(d, dtype=np.float64)[mine]

    def largest_diameter(self) -> float:
        return float(self.d.max()) if self.d.size else 0.0

    def halo_width(self, dist) -> float:
        """The largest diameter over all ranks."""
        import torch
        t = torch.tensor([self.largest_diameter()], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def halo_rows(self, width: float):
        """Rows of the owned agents within `width` of the lower and the upper
        slab face (to send to rank - 1 and rank + 1)."""
        if self.slabs.world > 1 and self.slabs.width < width:
            raise ValueError("slabs narrower than the halo width")
        down, up = halo_masks(self.xyz[:, 2], self.slabs, self.rank, width)
        return (pack(self.ids[down], self.xyz[down], self.d[down]),
                pack(self.ids[up], self.xyz[up], self.d[up]))

    def advance(self, below, above, engine):
        """Step the owned agents with the halo rows received from below and
        above, keep the owned results, and return the rows of the agents
        that left the slab (to rank - 1, to rank + 1) and the halo size."""
        rank = self.rank
        hi_ids, hi_xyz, hi_d = unpack(np.concatenate([below, above]))
        ids = np.concatenate([self.ids, hi_ids])
        xyz = np.concatenate([self.xyz, hi_xyz])
        d = np.concatenate([self.d, hi_d])
        owned = np.concatenate([np.ones(self.ids.shape[0], bool), np.zeros(hi_ids.shape[0], bool)])
        order = np.argsort(ids, kind="stable")
        new_xyz = np.asarray(engine(xyz[order], d[order], ~owned[order]), dtype=np.float64)
        back = np.empty_like(order)
        back[order] = np.arange(order.shape[0])
        self.xyz = new_xyz[back[owned]]
        dest = self.slabs.owner(self.xyz[:, 2])
        if np.any(np.abs(dest - rank) > 1):
            raise ValueError("an agent crossed more than one slab in one iteration")
        self._stay = dest == rank
        go_down, go_up = dest == rank - 1, dest == rank + 1
        return (pack(self.ids[go_down], self.xyz[go_down], self.d[go_down]),
                pack(self.ids[go_up], self.xyz[go_up], self.d[go_up]), int(hi_ids.shape[0]))

    def absorb(self, below, above) -> int:
        """Drop the agents that left and take in the ones that arrived (rows
        from below and above); the agents stay in ascending ID order."""
        stay = self._stay
        in_ids, in_xyz, in_d = unpack(np.concatenate([below, above]))
        self.ids = np.concatenate([self.ids[stay], in_ids])
        self.xyz = np.concatenate([self.xyz[stay], in_xyz])
        self.d = np.concatenate([self.d[stay], in_d])
        self.ids, self.xyz, self.d = merge_by_id(self.ids, self.xyz, self.d)
        return int((~stay).sum())

    def step(self, dist, engine) -> dict:
        """One iteration over a process group; returns the number of halo
        agents received and of owned agents that migrated out."""
        width = self.halo_width(dist)
        below, above = _swap(dist, *self.halo_rows(width), self.rank, self.slabs.world)
        mig_down, mig_up, n_halo = self.advance(below, above, engine)
        below, above = _swap(dist, mig_down, mig_up, self.rank, self.slabs.world)
        return {"halo_in": n_halo, "migrated_out": self.absorb(below, above)}


def step_local(domains, engine) -> list:
    """One iteration of every rank's domain in this process: the exchange of
    SlabDomain.step, with the messages handed over directly instead of
    through a process group (a single GPU stepping every slab)."""
    world = len(domains)
    none = np.zeros((0, ROW))
    width = max(dom.largest_diameter() for dom in domains)

    def swap(out):
        return [(out[r - 1][1] if r > 0 else none, out[r + 1][0] if r < world - 1 else none) for r in range(world)]

    got = swap([dom.halo_rows(width) for dom in domains])
    adv = [dom.advance(below, above, engine) for dom, (below, above) in zip(domains, got)]
    got = swap([(a[0], a[1]) for a in adv])
    return [{"halo_in": a[2], "migrated_out": dom.absorb(below, above)}
            for dom, a, (below, above) in zip(domains, adv, got)]


class LibraryEngine:
    """Steps a rank's agents with the library: the owned agents move, the
    halo agents are ghosts (bdm_set_ghosts), so only the owned agents'
    results are the rank's.  `params` is a workloads.SimParams."""

    def __init__(self, params, capacity: int):
        from . import binding
        self.ctx = binding.Context(binding.make_params(params), int(capacity))

    def __call__(self, xyz, d, ghost):
        self.ctx.set_agents(0, xyz, d)
        self.ctx.set_ghosts(0, ghost)
        self.ctx.step(1)
        return self.ctx.get_agents(0)[0]
