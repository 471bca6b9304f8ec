"""One problem over several GPUs: the region list is split between ranks.

The branch and bound of section 3.1 keeps a list of regions; regions are
independent, so after a first phase on one rank the list can be dealt out
(the paper's outlook to GPU clusters, sections 3.2 and 5).  Each rank
continues its share with ``gb_solve_resume`` on its own GPU, starting from
the incumbent of the split; the global enclosure is [min GLB, min GUB] over
the ranks (every rank's regions end with LB >= its GUB - tol_f >= the
global GUB - tol_f, so the width stays within tol_f), and the output
regions are those with LB <= the global GUB.  Ranks do not exchange the
incumbent during their phase (no collective on the data path).

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


def sharded_solve(make_solver, first_generations: int, dist, rank: int, world: int) -> ShardedResult:
    """Solve one problem on `world` ranks (one GPU each).

    make_solver(max_generations) -> an object with ``solve(raise_on_error)``,
    ``snapshot()``, ``resume(snapshot)`` and ``close()`` (``Solver`` of this
    package).  Rank 0 runs the first `first_generations` generations and
    snapshots the pool; the shards go to the ranks (broadcast), each resumes
    its own; the results are gathered on every rank and merged.  `dist` is
    ``torch.distributed`` with an initialised process group."""
    payload = [None]
    if rank == 0:
        s = make_solver(first_generations)
        s.solve(raise_on_error=False)
        snap = s.snapshot()
        s.close()
        payload = [dict(shards=[_pack(x) for x in split_snapshot(snap, world)])]
    dist.broadcast_object_list(payload, src=0)
    mine = payload[0]["shards"][rank]
    snap = Snapshot(**mine)
    if len(snap.flo) == 0:
        part = (np.inf, snap.gub, None, None, np.zeros(0), 0, 0)
    else:
        s = make_solver(0)
        r = s.resume(snap, raise_on_error=False)
        s.close()
        part = (r.fmin_lo, r.fmin_hi, r.box_lo, r.box_hi, r.box_flo, r.generations, r.status)
    parts = [None] * world
    dist.all_gather_object(parts, part)
    return merge_results(parts, snap.n)
