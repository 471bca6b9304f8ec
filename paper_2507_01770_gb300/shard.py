"""One problem over several GPUs: the region list is split between ranks.

The branch and bound of section 3.1 keeps a list of regions; regions are
independent, so after a first phase on one rank the list can be dealt out
(the paper's outlook to GPU clusters, sections 3.2 and 5).  Each rank
continues its share with ``gb_solve_resume`` on its own GPU in rounds of a
fixed number of generations; between rounds the ranks exchange their
incumbents (a min over the ranks' GUBs, 8 bytes each: the one exchange of
the path).  The global enclosure is [min GLB, min GUB] over the ranks
(every rank's regions end with LB >= its GUB - tol_f >= the global GUB -
tol_f, so the width stays within tol_f), and the output regions are those
with LB <= the global GUB.

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


def sharded_solve(make_solver, first_generations: int, dist, rank: int, world: int,
                  round_generations: int = 64, rebalance: bool = False) -> ShardedResult:
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
    and merged.  `dist` is ``torch.distributed`` (or any object with
    ``broadcast_object_list`` and ``all_gather_object``) with an initialised
    process group."""
    payload = [None]
    if rank == 0:
        s = make_solver(first_generations)
        s.solve(raise_on_error=False)
        snap = s.snapshot()
        s.close()
        payload = [dict(shards=[_pack(x) for x in split_snapshot(snap, world)])]
    dist.broadcast_object_list(payload, src=0)
    snap = Snapshot(**payload[0]["shards"][rank])
    n = snap.n
    solver = make_solver(round_generations)
    finished = []   # results of the region lists this rank has run to the end
    gens = 0
    while True:
        done = True
        if len(snap.flo):
            r = solver.resume(snap, raise_on_error=False)
            gens += r.generations
            done = r.status != _LIMIT
            if done:
                finished.append((r.fmin_lo, r.fmin_hi, r.box_lo, r.box_hi, r.box_flo, gens, r.status))
                snap = Snapshot(n, snap.block, np.zeros((0, n)), np.zeros((0, n)), np.zeros(0),
                                np.zeros(0, np.int32), float(r.fmin_hi), snap.generations)
            else:
                snap = solver.snapshot()
        # the incumbent exchange: a min over the ranks' GUBs (and whether all are done)
        views = [None] * world
        dist.all_gather_object(views, (float(snap.gub), done))
        gub = min(v[0] for v in views)
        if all(v[1] for v in views):
            break
        if rebalance:   # pool the unfinished lists and deal them out again
            lists = [None] * world
            dist.all_gather_object(lists, None if done else _pack(snap))
            live = [Snapshot(**x) for x in lists if x is not None]
            snap = split_snapshot(_concat(live), world)[rank]
        snap = Snapshot(snap.n, snap.block, snap.lo, snap.hi, snap.flo, snap.cyc, min(snap.gub, gub),
                        snap.generations)
    solver.close()
    mine = finished or [(np.inf, snap.gub, None, None, np.zeros(0), gens, 0)]
    parts = [None] * world
    dist.all_gather_object(parts, mine)
    return merge_results([q for p in parts for q in p], n)


_LIMIT = 4   # GB_E_LIMIT: the round's generation limit, regions still active
