"""x-slab decomposition of one lattice: host-side planning and the two
exchanges of an iteration (records, halos).

The step is a radius-2 stencil (Section 3: 4th-order first, second and mixed
differences reach two sites along each axis) and the arrest rule (Section 3)
compares the static energy of the whole lattice with the previous
iteration's.  A lattice is therefore cut along x, its slowest axis, into slabs
of whole interior planes.  Each slab is a lattice of its own: its p interior
planes plus two ghost planes on each side, which hold the neighbour's two
nearest interior planes (or, at the whole lattice's boundary, the two vacuum
layers).  One iteration of every slab is

1. ``skyrme_slab_step``: the slab's step up to the arrest decision, leaving an
   8-double record of its sums;
2. an all-gather of the records, in slab order;
3. ``skyrme_slab_finish``: the decision over the whole lattice (identical in
   every slab, since every slab sums the same records in the same order) and
   the arrest fix-up;
4. the halo exchange of the new field.

Slabs may live on several ranks (:class:`DistExchange`, torch.distributed:
NCCL between GPUs, gloo between CPU processes) or in one process
(:class:`LocalExchange`).  The exchanges only move data; every number of the
flow is computed by the library's kernels.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Sequence, Tuple

from . import Lattice, State, load_field, slab_finish, slab_step

GHOST = 2  # ghost planes per side: the stencil radius


@dataclass(frozen=True)
class SlabPlan:
    """Interior x-planes 2 .. n0 - 3 of an n0-plane lattice cut into
    ``nslabs`` contiguous slabs of as equal size as possible."""
    n0: int
    nslabs: int

    def __post_init__(self):
        interior = self.n0 - 2 * GHOST
        if self.nslabs < 1 or interior < GHOST * self.nslabs:
            # a slab's two boundary planes must both be its own interior planes
            raise ValueError(f"{self.n0} planes cannot be cut into {self.nslabs} slabs "
                             f"of at least {GHOST} interior planes")

    def ranges(self) -> List[Tuple[int, int]]:
        """(first global interior plane, number of planes) of every slab."""
        interior = self.n0 - 2 * GHOST
        base, extra = divmod(interior, self.nslabs)
        out, start = [], GHOST
        for i in range(self.nslabs):
            p = base + (1 if i < extra else 0)
            out.append((start, p))
            start += p
        return out

    def planes(self, i: int) -> int:
        return self.ranges()[i][1]

    def local_n0(self, i: int) -> int:
        return self.planes(i) + 2 * GHOST

    def global_span(self, i: int) -> Tuple[int, int]:
        """Global planes [lo, hi) held by slab i, ghosts included."""
        a, p = self.ranges()[i]
        return a - GHOST, a + p + GHOST

    def local_lattice(self, lat: Lattice, i: int) -> Lattice:
        n = list(int(v) for v in lat.n)
        n[0] = self.local_n0(i)
        return Lattice(n, lat.h, lat.m, lat.precision, lat.m_y, lat.m_z, lat.m_w, lat.c6)

    def extract(self, field, i: int):
        """Slab i's planes (ghosts included) of a whole-lattice field."""
        lo, hi = self.global_span(i)
        return field[lo:hi]

    def interior(self, local_field, i: int):
        """The slab's own interior planes of a slab field."""
        return local_field[GHOST:GHOST + self.planes(i)]

    def halo_pairs(self, i: int):
        """The halo exchange of slab i: (neighbour, planes sent, ghost planes
        received), as local plane slices of the slab's field."""
        p = self.planes(i)
        pairs = []
        if i > 0:
            pairs.append((i - 1, slice(GHOST, 2 * GHOST), slice(0, GHOST)))
        if i < self.nslabs - 1:
            pairs.append((i + 1, slice(p, p + GHOST), slice(p + GHOST, p + 2 * GHOST)))
        return pairs


class DistExchange:
    """The exchanges between ranks, one slab per rank (slab index = rank),
    with torch.distributed: NCCL for device tensors, gloo for CPU ones."""

    def __init__(self, plan: SlabPlan, rank: int, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.plan, self.rank, self.group = plan, rank, group
        if dist.get_world_size(group) != plan.nslabs:
            raise ValueError("one slab per rank: world size must equal the slab count")

    def gather(self, record, records):
        """records[j] <- record of rank j, for every j (slab order)."""
        self.dist.all_gather(list(records.unbind(0)), record, group=self.group)

    def exchange(self, field):
        """Ghost planes of this rank's field <- the neighbours' nearest
        interior planes.  Sent and received slices are whole x-planes, so they
        are contiguous views of the field: nothing is packed."""
        dist = self.dist
        ops = []
        for peer, send, recv in self.plan.halo_pairs(self.rank):
            ops.append(dist.P2POp(dist.isend, field[send], peer, self.group))
            ops.append(dist.P2POp(dist.irecv, field[recv], peer, self.group))
        if ops:
            for w in dist.batch_isend_irecv(ops):
                w.wait()


class LocalExchange:
    """The same exchanges for slabs held in one process (device copies)."""

    def __init__(self, plan: SlabPlan):
        self.plan = plan

    def gather_all(self, recs: Sequence, records):
        for j, r in enumerate(recs):
            records[j].copy_(r)

    def exchange_all(self, fields: Sequence):
        for i, f in enumerate(fields):
            for peer, _, recv in self.plan.halo_pairs(i):
                # peer's planes that face slab i
                for q, send, _ in self.plan.halo_pairs(peer):
                    if q == i:
                        f[recv].copy_(fields[peer][send])


class SlabState:
    """One slab's lattice, device state and record buffers."""

    def __init__(self, lat: Lattice, plan: SlabPlan, i: int, device="cuda"):
        import torch
        self.plan, self.index = plan, i
        self.lat = plan.local_lattice(lat, i)
        self.st = State(self.lat, device)
        self.record = torch.zeros(8, dtype=torch.float64, device=self.st.device)
        self.records = torch.zeros((plan.nslabs, 8), dtype=torch.float64, device=self.st.device)
        self.k = 0  # iterations since the load: the current buffer is k mod 2

    def load(self, whole_field):
        """Start from the slab's planes of a whole-lattice field (the ghost
        planes are refreshed by the first halo exchange)."""
        load_field(self.lat, self.st, self.plan.extract(whole_field, self.index))
        self.k = 0

    def field(self):
        return self.st.phi[self.k & 1]

    def step(self, dt: float, mode: int):
        slab_step(self.lat, dt, mode, self.st, self.record)

    def finish(self, dt: float, mode: int):
        slab_finish(self.lat, dt, mode, self.st, self.records)
        self.k += 1


class DistSlabFlow:
    """This rank's slab of a lattice flowed across ranks (one slab per rank)."""

    def __init__(self, lat: Lattice, rank: int, world: int, device="cuda", group=None):
        self.plan = SlabPlan(int(lat.n[0]), world)
        self.slab = SlabState(lat, self.plan, rank, device)
        self.comm = DistExchange(self.plan, rank, group)

    def load(self, whole_field):
        self.slab.load(whole_field)
        self.comm.exchange(self.slab.field())

    def flow(self, dt: float, nsteps: int, mode: int):
        s = self.slab
        for _ in range(nsteps):
            s.step(dt, mode)
            self.comm.gather(s.record, s.records)
            s.finish(dt, mode)
            self.comm.exchange(s.field())

    def report(self) -> dict:
        return self.slab.st.report()


class LocalSlabFlow:
    """All slabs of a lattice in one process, on one device."""

    def __init__(self, lat: Lattice, nslabs: int, device="cuda"):
        self.plan = SlabPlan(int(lat.n[0]), nslabs)
        self.slabs = [SlabState(lat, self.plan, i, device) for i in range(nslabs)]
        self.comm = LocalExchange(self.plan)

    def load(self, whole_field):
        for s in self.slabs:
            s.load(whole_field)
        self.comm.exchange_all([s.field() for s in self.slabs])

    def flow(self, dt: float, nsteps: int, mode: int):
        for _ in range(nsteps):
            for s in self.slabs:
                s.step(dt, mode)
            for s in self.slabs:
                self.comm.gather_all([t.record for t in self.slabs], s.records)
            for s in self.slabs:
                s.finish(dt, mode)
            self.comm.exchange_all([s.field() for s in self.slabs])

    def whole_field(self, out):
        """Assemble the slabs' interior planes into a whole-lattice tensor
        (whose outer layers the caller provides)."""
        for s in self.slabs:
            a, p = self.plan.ranges()[s.index]
            out[a:a + p].copy_(self.plan.interior(s.field(), s.index))
        return out

    def report(self) -> dict:
        return self.slabs[0].st.report()
