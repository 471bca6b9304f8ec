"""Checkpoint and resume of the region list (gb_snapshot_take /
gb_solve_resume): a solve stopped after k generations and resumed from its
snapshot runs the same generations as the uninterrupted solve, generation
by generation, and ends with the same enclosure and regions (the pool order,
lower bounds, cycling words and incumbent are the whole state of section
3.1's loop; the cached sums are recomputed bit for bit)."""
import numpy as np
import pytest

import oracle as O
import synthetic as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2507_01770_gb300 as gb  # noqa: E402

TRACE = ("parents", "children", "kept32", "kept", "pool", "gub")


def _solve(p, **opts):
    s = gb.Solver(p, **opts)
    r = s.solve(raise_on_error=False)
    return s, r


def _check_continuation(p, k, opts, resume_opts=None):
    full_s, full = _solve(p, **opts)
    full_s.close()
    part_s, part = _solve(p, max_generations=k, **opts)
    assert part.status == gb.GB_E_LIMIT and part.generations == k
    snap = part_s.snapshot()
    part_s.close()
    assert snap.generations == k and snap.n == p.n and len(snap.flo) == part.trace["pool"][-1]
    res_s = gb.Solver(p, **dict(opts, **(resume_opts or {})))
    rest = res_s.resume(snap)
    res_s.close()
    assert rest.status == full.status
    assert k + rest.generations == full.generations
    for key in TRACE:
        joined = np.concatenate([part.trace[key], rest.trace[key]])
        assert np.array_equal(joined, full.trace[key]), key
    assert rest.fmin_lo == full.fmin_lo and rest.fmin_hi == full.fmin_hi
    assert np.array_equal(rest.box_lo, full.box_lo) and np.array_equal(rest.box_hi, full.box_hi)
    assert np.array_equal(rest.box_flo, full.box_flo)
    return full, part, rest


@pytest.mark.parametrize("fp32", [0, 1])
@pytest.mark.parametrize("k", [1, 7])
def test_resume_continues_the_solve(fp32, k):
    p = S.chain(n=12, seed=3, block=6)
    opts = dict(block=6, split_m=2, split_d=3, max_children=8 * 8, fp32_prefilter=fp32, gens_per_sync=1)
    full, part, rest = _check_continuation(p, k, opts)
    # and the joined run is the oracle's uninterrupted run
    o = O.Oracle(p, block=6).solve(tol_f=p.tol_f, split_m=2, split_d=3, fp32=bool(fp32), max_parents=8)
    assert np.array_equal(np.concatenate([part.trace["gub"], rest.trace["gub"]]), o.trace["gub"])
    assert rest.fmin_lo == o.glb and rest.fmin_hi == o.gub


def test_resume_in_paper_mode_with_graphs():
    p = S.paper_levy(n=10, block=5)
    opts = dict(block=5, split_m=4, split_d=5, max_children=1024, tol_x=1e-4, tol_f=0.0, samples=10, mono_all=1)
    _check_continuation(p, 5, opts)
    _check_continuation(p, 5, dict(opts, gens_per_sync=4))


def test_records_pool_snapshot_resumes_on_dense_rows():
    # a block-record pool (n >= 128) is snapshotted as plain boxes; resumed
    # on dense rows it continues identically (the layouts hold the same doubles)
    p = S.chain(n=160, seed=1)
    opts = dict(block=10, split_m=2, split_d=5, max_children=4 * 32)
    full_s, full = _solve(p, **opts)
    assert full.pool_mode == 2
    full_s.close()
    part_s, part = _solve(p, max_generations=40, **opts)
    snap = part_s.snapshot()
    part_s.close()
    res_s = gb.Solver(p, pool_mode=1, **opts)
    rest = res_s.resume(snap)
    res_s.close()
    assert 40 + rest.generations == full.generations
    for key in TRACE:
        assert np.array_equal(np.concatenate([part.trace[key], rest.trace[key]]), full.trace[key]), key
    assert rest.fmin_lo == full.fmin_lo and rest.fmin_hi == full.fmin_hi
    # a resume into the record pool itself is refused (dense rows only)
    rec = gb.Solver(p, **opts)
    with pytest.raises(gb.GbError) as e:
        rec.resume(snap)
    assert e.value.status == gb.GB_E_INVALID
    rec.close()


def test_capacity_stop_then_resume_in_a_larger_pool():
    p = S.chain(n=10, seed=2, block=5)
    opts = dict(block=5, split_m=2, split_d=5, max_children=64 * 32)
    small_s, small = _solve(p, max_boxes=300, **opts)
    assert small.status == gb.GB_E_CAPACITY
    snap = small_s.snapshot()
    small_s.close()
    big_s = gb.Solver(p, **opts)
    rest = big_s.resume(snap)
    big_s.close()
    assert rest.status == gb.GB_OK
    assert rest.fmin_lo <= 0.0 <= rest.fmin_hi and rest.fmin_hi - rest.fmin_lo <= p.tol_f
    assert np.any(np.all((rest.box_lo <= p.s) & (p.s <= rest.box_hi), axis=1))


def test_malformed_snapshots_are_refused():
    p = S.chain(n=8, seed=4, block=4)
    s = gb.Solver(p, block=4, split_m=2, split_d=2, max_children=64)
    with pytest.raises(gb.GbError) as e:          # no solve yet
        s.snapshot()
    assert e.value.status == gb.GB_E_INVALID
    s.solve()
    r = gb.Solver(p, block=4, split_m=2, split_d=2, max_children=64, max_generations=3)
    r.solve(raise_on_error=False)
    snap = r.snapshot()
    r.close()
    assert len(snap.flo) > 0
    bad = [dict(lo=snap.hi + 1.0), dict(cyc=snap.cyc + 100), dict(n=7)]
    for change in bad:
        b = gb.Snapshot(**{**snap.__dict__, **change})
        with pytest.raises(gb.GbError) as e:
            s.resume(b)
        assert e.value.status == gb.GB_E_INVALID, change
    s.close()


class _ThreadDist:
    """broadcast_object_list / all_gather_object / all_reduce (MIN) /
    all_gather between threads (one per rank, all on this GPU: the ranks
    share nothing but these host calls)."""

    def __init__(self, world):
        import threading
        self.world, self.bar, self.local = world, threading.Barrier(world), threading.local()
        self.slots, self.shared = [None] * world, None

    def broadcast_object_list(self, lst, src=0):
        if self.local.rank == src:
            self.shared = lst[0]
        self.bar.wait()
        lst[0] = self.shared
        self.bar.wait()

    def all_gather_object(self, out, obj):
        self.slots[self.local.rank] = obj
        self.bar.wait()
        out[:] = list(self.slots)
        self.bar.wait()

    class ReduceOp:
        MIN = "min"

    def all_reduce(self, t, op=None):
        self.slots[self.local.rank] = t.clone()
        self.bar.wait()
        r = self.slots[0].clone()
        for x in self.slots[1:]:
            r = torch.minimum(r, x)
        self.bar.wait()
        t.copy_(r)

    def all_gather(self, out, t):
        self.slots[self.local.rank] = t.clone()
        self.bar.wait()
        for o, x in zip(out, self.slots):
            o.copy_(x)
        self.bar.wait()


@pytest.mark.parametrize("rebalance", [False, True])
@pytest.mark.parametrize("world", [2, 3])
def test_sharded_solve_ranks_as_threads(world, rebalance):
    # shard.sharded_solve with its ranks as threads on this GPU: rounds of
    # generations with the incumbent exchanged between them; the merged
    # enclosure is rigorous and within tol_f, covers the planted minimiser
    # and overlaps the single-rank solve's
    import threading
    from paper_2507_01770_gb300 import shard
    p = S.chain(n=12, seed=3, block=6)
    opts = dict(block=6, split_m=2, split_d=3, max_children=8 * 8)
    D = _ThreadDist(world)
    res, errs = [None] * world, []

    def run(rank):
        try:
            D.local.rank = rank
            res[rank] = shard.sharded_solve(lambda g: gb.Solver(p, max_generations=g, **opts), 6, D, rank, world,
                                            round_generations=16, rebalance=rebalance)
        except Exception as e:   # noqa: BLE001 - reported below
            errs.append(e)
            D.bar.abort()

    th = [threading.Thread(target=run, args=(r,)) for r in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=300)
    assert not errs, errs
    m = res[0]
    assert all(r.fmin_lo == m.fmin_lo and r.fmin_hi == m.fmin_hi for r in res)
    assert all(st == gb.GB_OK for st in m.statuses)
    assert m.fmin_lo <= 0.0 <= m.fmin_hi and m.fmin_hi - m.fmin_lo <= p.tol_f
    assert np.any(np.all((m.box_lo <= p.s) & (p.s <= m.box_hi), axis=1))
    full_s, full = _solve(p, **opts)
    full_s.close()
    assert max(full.fmin_lo, m.fmin_lo) <= min(full.fmin_hi, m.fmin_hi)
