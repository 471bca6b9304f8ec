"""One problem over several ranks (paper_2507_01770_gb300.shard), host logic
with two gloo ranks on the CPU: the snapshot of the first phase is dealt out
round-robin, every rank resumes its share in rounds with the incumbent
exchanged between rounds, and the merged enclosure is [min GLB, min GUB]
with the regions whose LB is not above the global GUB.  The solver is a
stand-in (no GPU), so the test checks the plumbing, the exchange and the
merge."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class _FakeResult:
    def __init__(self, lo, hi, flo, gub, gens):
        self.box_lo, self.box_hi, self.box_flo = lo, hi, flo
        self.fmin_lo = float(flo.min()) if len(flo) else np.inf
        self.fmin_hi, self.generations, self.status = gub, gens, 0


class _FakeSolver:
    """First phase: 10 regions of a 3-D box with LB = q / 10, GUB 0.55.
    Resume: the first round stops on its generation limit with a
    rank-dependent incumbent (0.5, 0.25); the second records the incumbent
    it was given and keeps the regions with LB not above it."""

    def __init__(self, rank, max_gen):
        self.rank, self.max_gen, self.calls, self.given, self.seen = rank, max_gen, 0, [], []
        self.regions = None

    def solve(self, raise_on_error=True):
        return _FakeResult(None, None, np.zeros(0), 0.55, self.max_gen)

    def snapshot(self):
        import paper_2507_01770_gb300 as gb
        if self.regions is not None:     # after a round: the shard's regions, its own incumbent
            lo, hi, flo = self.regions
            return gb.Snapshot(3, 3, lo, hi, flo, np.zeros(len(flo), np.int32), [0.5, 0.25][self.rank], 9)
        q = np.arange(10, dtype=np.float64)
        lo = np.stack([q, q, q], axis=1)
        return gb.Snapshot(3, 3, lo, lo + 0.5, q / 10, np.zeros(10, np.int32), 0.55, self.max_gen)

    def resume(self, snap, raise_on_error=True):
        self.calls += 1
        self.given.append(snap.gub)
        self.seen.append([round(float(v), 6) for v in snap.flo])
        self.regions = (snap.lo, snap.hi, snap.flo)
        if self.calls == 1:
            r = _FakeResult(snap.lo, snap.hi, snap.flo, [0.5, 0.25][self.rank], 3)
            r.status = 4                  # generation limit of the round
            return r
        keep = ~(snap.flo > snap.gub)
        return _FakeResult(snap.lo[keep], snap.hi[keep], snap.flo[keep], snap.gub, 4 + self.rank)

    def close(self):
        pass


def _rank(rank, world, port, out, rebalance=False):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    from paper_2507_01770_gb300 import shard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    made = []

    def make(g):
        made.append(_FakeSolver(rank, g))
        return made[-1]

    res = shard.sharded_solve(make, 5, dist, rank, world, round_generations=3, rebalance=rebalance)
    out.put((rank, res.fmin_lo, res.fmin_hi, res.box_flo.tolist(), res.generations, made[-1].given,
             made[-1].seen))
    dist.destroy_process_group()


@pytest.mark.parametrize("rebalance", [False, True])
def test_sharded_solve_two_gloo_ranks(rebalance):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q, rebalance)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, glb, gub, flo, gens, given, seen in got:
        # round 2 regions: the rank's own, or (rebalanced) the pooled lists
        # [0 .2 .4 .6 .8 | .1 .3 .5 .7 .9] dealt out again
        own = [[0.0, 0.2, 0.4, 0.6, 0.8], [0.1, 0.3, 0.5, 0.7, 0.9]][rank]
        dealt = [[0.0, 0.4, 0.8, 0.3, 0.7], [0.2, 0.6, 0.1, 0.5, 0.9]][rank]
        assert seen == [own, dealt if rebalance else own]
        # round 1 starts from the split's incumbent 0.55; after it the ranks
        # exchange 0.5 and 0.25, so round 2 of every rank runs with 0.25 and
        # keeps its regions with LB <= 0.25: rank 0 {0, 0.2}, rank 1 {0.1}
        assert given == [0.55, 0.25]
        assert gub == 0.25
        assert sorted(flo) == [0.0, 0.1, 0.2]
        assert glb == 0.0
        assert sorted(gens) == [3 + 4, 3 + 5]


def test_split_and_merge_without_ranks():
    import paper_2507_01770_gb300 as gb
    from paper_2507_01770_gb300 import shard
    q = np.arange(7, dtype=np.float64)
    lo = np.stack([q, -q], axis=1)
    snap = gb.Snapshot(2, 2, lo, lo + 1, q, np.arange(7, dtype=np.int32) % 2, 3.5, 4)
    parts = shard.split_snapshot(snap, 3)
    assert [list(p.flo) for p in parts] == [[0, 3, 6], [1, 4], [2, 5]]
    assert all(p.gub == 3.5 and p.generations == 4 and p.n == 2 for p in parts)
    assert np.array_equal(np.concatenate([p.lo for p in parts])[np.argsort(np.concatenate([p.flo for p in parts]))],
                          lo)
    m = shard.merge_results([(0.0, 2.0, lo[:3], lo[:3] + 1, q[:3], 1, 0), (1.0, 1.5, lo[3:], lo[3:] + 1, q[3:], 2, 0)],
                            2)
    assert m.fmin_hi == 1.5 and m.fmin_lo == 0.0 and list(m.box_flo) == [0.0, 1.0]


def test_split_with_more_ranks_than_regions_and_merge_of_empty_parts():
    import paper_2507_01770_gb300 as gb
    from paper_2507_01770_gb300 import shard
    lo = np.array([[0.0, 1.0], [2.0, 3.0]])
    snap = gb.Snapshot(2, 2, lo, lo + 1, np.array([0.5, 0.25]), np.array([0, 1], np.int32), 1.0, 2)
    parts = shard.split_snapshot(snap, 4)
    assert [len(p.flo) for p in parts] == [1, 1, 0, 0]
    assert parts[2].lo.shape == (0, 2) and parts[3].gub == 1.0
    m = shard.merge_results([(np.inf, 1.0, None, None, np.zeros(0), 0, 0),
                             (0.25, 0.75, lo[1:], lo[1:] + 1, np.array([0.25]), 3, 0)], 2)
    assert m.fmin_hi == 0.75 and m.fmin_lo == 0.25 and len(m.box_flo) == 1
    c = shard._concat([parts[0], parts[1], parts[2]])
    assert list(c.flo) == [0.5, 0.25] and c.gub == 1.0
    with pytest.raises(ValueError):
        shard.split_snapshot(snap, 0)


class _FailingSolver(_FakeSolver):
    """As _FakeSolver, but rank 1's first resume fails (GB_E_CUDA): its
    result holds no regions and reads status 6."""

    def resume(self, snap, raise_on_error=True):
        if self.rank == 1:
            self.calls += 1
            self.given.append(snap.gub)
            self.seen.append([round(float(v), 6) for v in snap.flo])
            r = _FakeResult(None, None, np.zeros(0), 0.0, 0)
            r.fmin_lo = r.fmin_hi = 0.0     # what a zeroed result holds: not a bound of anything
            r.status = 6
            return r
        return super().resume(snap, raise_on_error)


def _rank_failing(rank, world, port, out, rebalance):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    from paper_2507_01770_gb300 import shard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    res = shard.sharded_solve(lambda g: _FailingSolver(rank, g), 5, dist, rank, world, round_generations=3,
                              rebalance=rebalance)
    out.put((rank, res.fmin_lo, res.fmin_hi, sorted(res.box_flo.tolist()), res.statuses))
    dist.destroy_process_group()


@pytest.mark.parametrize("rebalance", [False, True])
def test_failed_resume_keeps_its_regions_in_the_merge(rebalance):
    # rank 1's resume fails: its zeroed result (GUB 0, no regions) must not
    # enter the merge.  It keeps the regions it was given (LB .1 .3 .5 .7 .9)
    # with the split's incumbent 0.55; rank 0 runs round 1 (GUB 0.5) and
    # round 2 with the exchanged 0.5 (regions 0 .2 .4).  Merge: GUB 0.5, the
    # regions with LB <= 0.5 from both ranks, GLB 0, statuses report 6.
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_failing, args=(r, 2, port, q, rebalance)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, glb, gub, flo, statuses in got:
        assert gub == 0.5 and glb == 0.0
        assert flo == [0.0, 0.1, 0.2, 0.3, 0.4, 0.5]
        assert 6 in statuses and 0 in statuses
