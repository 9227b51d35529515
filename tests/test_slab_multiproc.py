"""The x-slab decomposition's multi-rank logic on CPU ranks (gloo, world
size 2), with the oracle doing each slab's arithmetic.

Each rank holds one slab of a 26 x 20 x 22 lattice (its interior planes plus
two ghost planes per side).  Every iteration it computes its slab's forces and
sums with the oracle, all-gathers the 8-double records in slab order
(DistExchange.gather), applies the arrest rule of Section 3 to the whole
lattice's energy, updates its interior sites and exchanges halos
(DistExchange.exchange).  After 30 iterations the assembled field must equal
the oracle's whole-lattice flow, and every rank must have reached the same
decisions and energies.  The library's own planner and exchanges are what is
tested; the GPU kernels' slab mode is tested on a GPU
(tests/test_gpu_slab.py)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

N = (26, 20, 22)
H, M, DT, STEPS = 0.25, 1.0, 0.0125, 30


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _seed():
    import oracle
    # off-centre B=1 so that the two slabs carry different energy
    phi = oracle.rational_map_field(N, H, 1, 1.0, X=(0.6, -0.3, 0.2))
    return oracle.apply_vacuum_boundary(np.ascontiguousarray(phi))


def _worker(rank, ws, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    import oracle
    from paper_2604_25876_gb300.slab import DistExchange, SlabPlan

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    plan = SlabPlan(N[0], ws)
    comm = DistExchange(plan, rank)
    phi = torch.from_numpy(np.ascontiguousarray(plan.extract(_seed(), rank)))
    v = torch.zeros_like(phi)
    # the ghost planes the exchange must fill start out wrong on purpose
    p = plan.planes(rank)
    for _, _, recv in plan.halo_pairs(rank):
        phi[recv] = 0.0
    comm.exchange(phi)
    record = torch.zeros(8, dtype=torch.float64)
    records = torch.zeros((ws, 8), dtype=torch.float64)
    E_prev, energies, arrests = float("inf"), [], 0
    inner = (slice(2, 2 + p), slice(2, N[1] - 2), slice(2, N[2] - 2))
    for _ in range(STEPS):
        _, F, d = oracle.forces(phi.numpy(), H, M)
        F = torch.from_numpy(F)
        f2 = (F[inner] ** 2).sum(-1)
        record.copy_(torch.tensor([d[inner][..., 0].sum(), d[inner][..., 1].sum(),
                                   d[inner][..., 2].sum(), d[inner][..., 3].sum(),
                                   float(f2.sum()), float(f2.max()), float(f2.numel()), 0.0],
                                  dtype=torch.float64))
        comm.gather(record, records)
        tot = records.sum(0)
        E = H ** 3 * float(tot[0] + tot[1] + tot[2])
        arrested = E > E_prev
        arrests += int(arrested)
        E_prev = E
        energies.append(E)
        if arrested:
            v.zero_()
        v[inner] += DT * F[inner]
        t = phi[inner] + DT * v[inner]
        phi[inner] = t / t.norm(dim=-1, keepdim=True)
        comm.exchange(phi)
    pieces = [None] * ws
    dist.all_gather_object(pieces, (rank, plan.interior(phi, rank).numpy().copy()))
    out.put((rank, energies, arrests, pieces))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_slab_flow_matches_whole_lattice_oracle():
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    st = oracle.new_state(_seed())
    reps = oracle.flow(st, H, M, DT, STEPS, reports=True)
    ref_E = [r["E"] for r in reps]
    ref_arrests = sum(r["arrested"] for r in reps)
    assert 0 < ref_arrests < STEPS  # the run exercises both branches of the rule
    from paper_2604_25876_gb300.slab import SlabPlan
    plan = SlabPlan(N[0], 2)
    for rank, energies, arrests, pieces in res:
        # every rank reached the whole lattice's energies and decisions
        np.testing.assert_allclose(energies, ref_E, rtol=1e-13)
        assert arrests == ref_arrests
        whole = _seed()
        for r, piece in sorted(pieces, key=lambda t: t[0]):
            a, p = plan.ranges()[r]
            whole[a:a + p] = piece
        np.testing.assert_allclose(whole, st.phi, rtol=0, atol=1e-13)


def test_plan_covers_every_interior_plane_once():
    from paper_2604_25876_gb300.slab import SlabPlan
    for n0, k in [(26, 2), (37, 3), (12, 4), (520, 7)]:
        plan = SlabPlan(n0, k)
        r = plan.ranges()
        assert r[0][0] == 2 and sum(p for _, p in r) == n0 - 4
        assert all(r[i][0] + r[i][1] == r[i + 1][0] for i in range(k - 1))
        assert max(p for _, p in r) - min(p for _, p in r) <= 1
        for i in range(k):
            lo, hi = plan.global_span(i)
            assert hi - lo == plan.local_n0(i)
            for peer, send, recv in plan.halo_pairs(i):
                # the planes a neighbour sends are exactly slab i's ghost planes
                s2 = [s for q2, s, _ in plan.halo_pairs(peer) if q2 == i][0]
                a_peer = plan.ranges()[peer][0]
                sent = range(a_peer - 2 + s2.start, a_peer - 2 + s2.stop)
                ghost = range(lo + recv.start, lo + recv.stop)
                assert list(sent) == list(ghost)
    with pytest.raises(ValueError):
        SlabPlan(9, 3)  # 5 interior planes: a slab of 1 plane cannot feed a 2-plane halo
