"""One problem over several GPUs: the region list is split between ranks.

The branch and bound of section 3.1 keeps a list of regions; regions are
independent, so after a first phase on one rank the list can be dealt out
(the paper's outlook to GPU clusters, sections 3.2 and 5).  Each rank
continues its share with ``gb_solve_resume`` on its own GPU in rounds of a
fixed number of generations; between rounds the ranks exchange their
incumbents (a min over the ranks' GUBs: one all-reduce of a 16-byte tensor,
the one exchange of the path).  The global enclosure is [min GLB, min GUB]
over the ranks (every rank's regions end with LB >= its GUB - tol_f >= the
global GUB - tol_f, so the width stays within tol_f), and the output regions
are those with LB <= the global GUB.  Optional rebalancing moves region
lists between ranks as structure-of-arrays tensors (an all-gather: device to
device under NCCL).

Only host-side logic lives here: splitting a snapshot, merging results and
the collectives that carry them (any ``torch.distributed`` backend).  The
search itself runs in the CUDA library through ``Solver.resume``.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import Snapshot


def split_snapshot(snap: Snapshot, world: int) -> list[Snapshot]:
    """Deal the regions of a snapshot to `world` shards round-robin in pool
    order (rank r gets regions r, r + world, ...; each shard keeps the pool
    order of its regions, the incumbent and the generation count)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    out = []
    for r in range(world):
        idx = np.arange(r, len(snap.flo), world)
        out.append(Snapshot(snap.n, snap.block, snap.lo[idx].copy(), snap.hi[idx].copy(),
                            snap.flo[idx].copy(), snap.cyc[idx].copy(), snap.gub, snap.generations))
    return out


@dataclass
class ShardedResult:
    fmin_lo: float
    fmin_hi: float
    box_lo: np.ndarray
    box_hi: np.ndarray
    box_flo: np.ndarray
    generations: list          # per rank, after the split
    statuses: list


def merge_results(parts, n: int) -> ShardedResult:
    """parts: per rank (fmin_lo, fmin_hi, box_lo, box_hi, box_flo, generations,
    status).  The enclosure is [min GLB, min GUB]; a region is kept if its LB
    is not above the global GUB."""
    glb = min(p[0] for p in parts)
    gub = min(p[1] for p in parts)
    los, his, flos = [], [], []
    for p in parts:
        if p[2] is None or len(p[4]) == 0:
            continue
        keep = ~(np.asarray(p[4]) > gub)
        los.append(np.asarray(p[2]).reshape(-1, n)[keep])
        his.append(np.asarray(p[3]).reshape(-1, n)[keep])
        flos.append(np.asarray(p[4])[keep])
    if los:
        lo, hi, flo = np.concatenate(los), np.concatenate(his), np.concatenate(flos)
    else:
        lo, hi, flo = np.zeros((0, n)), np.zeros((0, n)), np.zeros(0)
    if len(flo):   # the lowest LB among the kept regions (the rank of the global GUB keeps some)
        glb = float(flo.min())
    return ShardedResult(glb, gub, lo, hi, flo, [p[5] for p in parts], [p[6] for p in parts])


def _pack(snap: Snapshot):
    return dict(n=snap.n, block=snap.block, lo=snap.lo, hi=snap.hi, flo=snap.flo, cyc=snap.cyc, gub=snap.gub,
                generations=snap.generations)


def _concat(snaps: list[Snapshot]) -> Snapshot:
    """The regions of several snapshots in rank order (incumbent: the lowest)."""
    n, blk = snaps[0].n, snaps[0].block
    lo = np.concatenate([x.lo.reshape(-1, n) for x in snaps])
    hi = np.concatenate([x.hi.reshape(-1, n) for x in snaps])
    flo = np.concatenate([x.flo for x in snaps])
    cyc = np.concatenate([x.cyc for x in snaps]).astype(np.int32)
    return Snapshot(n, blk, lo, hi, flo, cyc, min(x.gub for x in snaps), max(x.generations for x in snaps))


def _exchange(dist, gub: float, done: bool, device) -> tuple[float, bool]:
    """The one exchange of a round: the minimum of the ranks' incumbents and
    whether every rank is done, as one all-reduce (MIN) of a 16-byte tensor
    [GUB, -1 if this rank still has active regions else 0] on `device` (a
    CUDA device under NCCL, the CPU under gloo)."""
    import torch
    t = torch.tensor([gub, 0.0 if done else -1.0], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MIN)
    v = t.cpu().tolist()
    return float(v[0]), v[1] == 0.0


def _gather_lists(dist, snap: Snapshot | None, n: int, block: int, world: int, device) -> list[Snapshot]:
    """Every rank's region list (None: the rank has none to give), gathered
    on every rank in rank order as tensors: the counts first (one all-gather
    of 8 bytes per rank), then the structure-of-arrays slices (lo, hi: count
    x n; LB; cycling word) padded to the largest count."""
    import torch
    c = 0 if snap is None else len(snap.flo)
    cnt = torch.tensor([c], dtype=torch.int64, device=device)
    counts = [torch.zeros(1, dtype=torch.int64, device=device) for _ in range(world)]
    dist.all_gather(counts, cnt)
    counts = [int(x.item()) for x in counts]
    cmax = max(counts)
    if cmax == 0:
        return []
    # rows: lo (n) | hi (n) | LB | cycling word | GUB | generations (the integers are exact in a double)
    rows = torch.zeros((cmax, 2 * n + 4), dtype=torch.float64, device=device)
    if c:
        rows[:c, :n] = torch.from_numpy(np.ascontiguousarray(snap.lo, dtype=np.float64).reshape(c, n))
        rows[:c, n:2 * n] = torch.from_numpy(np.ascontiguousarray(snap.hi, dtype=np.float64).reshape(c, n))
        rows[:c, 2 * n] = torch.from_numpy(np.ascontiguousarray(snap.flo, dtype=np.float64))
        rows[:c, 2 * n + 1] = torch.from_numpy(np.asarray(snap.cyc, dtype=np.int64).astype(np.float64))
        rows[:c, 2 * n + 2] = float(snap.gub)
        rows[:c, 2 * n + 3] = float(snap.generations)
    got = [torch.empty_like(rows) for _ in range(world)]
    dist.all_gather(got, rows)
    out = []
    for k, g in zip(counts, got):
        if k == 0:
            continue
        a = g[:k].cpu().numpy()
        out.append(Snapshot(n, block, a[:, :n].copy(), a[:, n:2 * n].copy(), a[:, 2 * n].copy(),
                            a[:, 2 * n + 1].astype(np.int64).astype(np.int32), float(a[0, 2 * n + 2]),
                            int(a[0, 2 * n + 3])))
    return out


def sharded_solve(make_solver, first_generations: int, dist, rank: int, world: int,
                  round_generations: int = 64, rebalance: bool = False, device="cpu") -> ShardedResult:
    """Solve one problem on `world` ranks (one GPU each).

    make_solver(max_generations) -> an object with ``solve(raise_on_error)``,
    ``snapshot()``, ``resume(snapshot, raise_on_error)`` and ``close()``
    (``Solver`` of this package).  Rank 0 runs the first `first_generations`
    generations and snapshots the pool; the shards go to the ranks
    (broadcast).  Then, in rounds, every rank resumes its own region list for
    up to `round_generations` generations and snapshots it again, and the
    ranks exchange their incumbents (the minimum over the ranks becomes every
    rank's incumbent: any upper bound of the global minimum is a valid
    cut-off for every region); with `rebalance` the ranks' region lists are
    also pooled and dealt out again after every round.  The rounds end when
    no rank has an active region.  The results are gathered on every rank
    and merged.  `dist` is ``torch.distributed`` with an initialised process
    group; `device` holds the exchanged tensors (the rank's CUDA device under
    NCCL, "cpu" under gloo).

    A resume that fails (a status other than OK, CAPACITY or LIMIT) ends that
    rank's work: its result holds no regions, so the rank keeps the regions
    it gave to that resume, unrefined, with their lower bounds, and reports
    the failed status.  The merged enclosure then still covers every region
    nobody ruled out (it is rigorous, only wider than tol_f)."""
    payload = [None]
    if rank == 0:
        s = make_solver(first_generations)
        s.solve(raise_on_error=False)
        snap = s.snapshot()
        s.close()
        payload = [dict(shards=[_pack(x) for x in split_snapshot(snap, world)])]
    dist.broadcast_object_list(payload, src=0)
    snap = Snapshot(**payload[0]["shards"][rank])
    n, block = snap.n, snap.block
    solver = make_solver(round_generations)
    finished = []   # results of the region lists this rank has run to the end (or given up on)
    gens = 0
    while True:
        done = True
        if len(snap.flo):
            r = solver.resume(snap, raise_on_error=False)
            gens += r.generations
            if r.status == _LIMIT:
                done = False
                snap = solver.snapshot()
            else:
                if r.status in _RIGOROUS:
                    finished.append((r.fmin_lo, r.fmin_hi, r.box_lo, r.box_hi, r.box_flo, gens, r.status))
                    gub_left = float(r.fmin_hi)
                else:   # failed: the regions it was given stay unresolved
                    finished.append((float(np.min(snap.flo)), float(snap.gub), snap.lo, snap.hi, snap.flo, gens,
                                     r.status))
                    gub_left = float(snap.gub)
                snap = Snapshot(n, block, np.zeros((0, n)), np.zeros((0, n)), np.zeros(0),
                                np.zeros(0, np.int32), gub_left, snap.generations)
        gub, all_done = _exchange(dist, float(snap.gub), done, device)
        if all_done:
            break
        if rebalance:   # pool the unfinished lists and deal them out again
            live = _gather_lists(dist, None if done else snap, n, block, world, device)
            if live:
                snap = split_snapshot(_concat(live), world)[rank]
        snap = Snapshot(snap.n, snap.block, snap.lo, snap.hi, snap.flo, snap.cyc, min(snap.gub, gub),
                        snap.generations)
    solver.close()
    mine = finished or [(np.inf, snap.gub, None, None, np.zeros(0), gens, 0)]
    parts = [None] * world
    dist.all_gather_object(parts, mine)
    return merge_results([q for p in parts for q in p], n)


_LIMIT = 4                 # GB_E_LIMIT: the round's generation limit, regions still active
_RIGOROUS = (0, 3)         # GB_OK, GB_E_CAPACITY: the result's regions and enclosure are valid
