"""Pins of the oracle's branch and bound (section 3.1, variable cycling of
section 3.2) against what the paper and the mathematics fix:

* the paper's own iteration and region counts (Table 2, Tables S2-S10),
  reproduced per cycling block in paper mode;
* the planted minimum (closed form min f = 0 at s) and the enclosure width;
* a separable problem against its 1-D sub-problems solved separately;
* brute force on a grid for n <= 3;
* the output regions always cover the planted minimiser, also when the solve
  stops early on a capacity or generation limit.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
import synthetic as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_iterations.txt")


def _golden_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if line:
            fam, n, it, reg = line.split()
            rows.append((fam, int(n), int(it), int(reg)))
    return rows


def _covers(res, x):
    inside = np.all((res.box_lo <= x) & (x <= res.box_hi), axis=1)
    return bool(inside.any())


PAPER_FAMILIES = ["paper_rastrigin", "paper_breiman", "paper_ackley", "paper_belegundu", "paper_fu",
                  "paper_levy", "paper_salomon", "paper_griewank", "paper_styblinski", "paper_zabinsky"]


def _fstar(p):
    return p.meta.get("fstar", -0.1 * p.n if p.family == "paper_breiman" else 0.0)   # SI Appendix A


@pytest.mark.parametrize("fam", PAPER_FAMILIES)
def test_paper_mode_iteration_counts(fam):
    rows = [r for r in _golden_rows() if r[0] == fam]
    per_block = {r[2] * 10 // r[1] for r in rows}
    assert len(per_block) == 1            # the paper's rows scale as n/10
    per_block = per_block.pop()
    for n, B in ((5, 5), (10, 5)):
        p = S.make(fam, n=n, block=B)
        res = O.Oracle(p, block=B).solve(tol_f=0.0, tol_x=1e-4, split_m=4, split_d=B,
                                         max_parents=1)
        assert res.status == O.ST_OK
        assert res.generations == (n // B) * per_block
        assert len(res.box_flo) == 1 == rows[0][3]
        assert np.all(res.box_hi - res.box_lo < 1e-4)
        assert res.glb <= _fstar(p) <= res.gub
        assert _covers(res, p.s)


@pytest.mark.parametrize("fam", PAPER_FAMILIES)
def test_full_paper_procedure_iteration_counts(fam):
    # the paper's procedure in full: 10 diagonal samples per region and the
    # first-order test on every coordinate (section 3.1, section 4), besides
    # the 4-way split of a block, one region per iteration and tol_x = 1e-4
    rows = [r for r in _golden_rows() if r[0] == fam]
    per_block = rows[0][2] * 10 // rows[0][1]
    for n, B in ((5, 5), (10, 5)):
        p = S.make(fam, n=n, block=B)
        res = O.Oracle(p, block=B).solve(tol_f=0.0, tol_x=1e-4, split_m=4, split_d=B, max_parents=1,
                                         samples=10, mono_all=True)
        assert res.status == O.ST_OK
        assert res.generations == (n // B) * per_block
        assert len(res.box_flo) == 1 == rows[0][3]
        assert res.glb <= _fstar(p) <= res.gub
        assert _covers(res, p.s)


@pytest.mark.parametrize("fam", PAPER_FAMILIES + ["paper_rosenbrock"])
@pytest.mark.parametrize("n", [2, 3])
def test_paper_functions_enclose_their_printed_minimum(fam, n):
    # SI Appendix A / D print each function's minimiser and minimum value
    p = S.make(fam, n=n)
    res = O.Oracle(p, block=n).solve(tol_f=1e-6, split_m=2, split_d=n, max_parents=16)
    assert res.status == O.ST_OK
    assert res.glb <= _fstar(p) <= res.gub and res.gub - res.glb <= 1e-6
    assert _covers(res, p.s)


def _diag_quadratic(n, s):
    """f(x) = sum_i (x_i - s_i)^2 on [0, 11]^n (closed form: min 0 at s)."""
    g = S.Dag()
    ts = g.table(np.asarray(s, dtype=np.float64))
    y = g.sub(g.ivar(0), g.icoef(ts))
    f = g.isum(g.sqr(y), 0, n, 1)
    return S.Problem("quad", n, g.nodes(), f, g.tables, np.zeros(n), np.full(n, 11.0), 1e-9, n,
                     np.asarray(s, dtype=np.float64), 0)


def test_discontinuous_paper_procedure():
    # SI Appendix F: the minimum -1 sits on the cube D of side 1e-6 around
    # 1.5.  Under the paper's procedure the region holding D is kept (its
    # F_lo is -1) and narrowed to tol_x; no diagonal sample lands in D, so
    # the GUB stays at the Levy minimum 0 and Levy's minimiser keeps a second
    # region (Table S14 prints one region: the reading differs there)
    p = S.paper_discontinuous(n=5, block=5)
    res = O.Oracle(p, block=5).solve(tol_f=0.0, tol_x=1e-4, split_m=4, split_d=5, max_parents=1,
                                     samples=10, mono_all=True)
    assert res.status == O.ST_OK
    assert res.glb == -1.0 and res.glb <= -1.0 <= res.gub
    assert _covers(res, np.full(5, 1.5)) and _covers(res, np.ones(5))
    assert len(res.box_flo) == 2
    assert np.all(res.box_hi - res.box_lo < 1e-4)


def test_diagonal_samples_hit_a_minimiser_on_the_diagonal():
    # the interior diagonal points of [0, 11]^n at j / 11 are (j, ..., j)
    # exactly; with the minimiser at (5, ..., 5) the root's samples already
    # give GUB = f(s) = 0, while the midpoint (5.5, ...) gives n / 4
    n = 3
    p = _diag_quadratic(n, [5.0] * n)
    o = O.Oracle(p, block=n)
    paper = o.solve(tol_f=1e-9, split_m=2, split_d=n, samples=10, max_gen=1)
    mid = o.solve(tol_f=1e-9, split_m=2, split_d=n, samples=0, max_gen=1)
    # the root's samples close the enclosure at once: no region is active
    assert paper.status == O.ST_OK and paper.generations == 0 and paper.mids == 10
    assert paper.gub == 0.0 and paper.glb == 0.0
    assert mid.trace["gub"][0] > 0.0
    # off the diagonal the samples only give an upper bound above the minimum
    q = _diag_quadratic(n, [5.0, 3.0, 5.0])
    r = O.Oracle(q, block=n).solve(tol_f=1e-9, split_m=2, split_d=n, samples=10, max_gen=1)
    assert r.trace["gub"][0] > 0.0


def test_mono_all_discards_at_least_as_much():
    # testing every coordinate can only rule out more regions than testing
    # the active block: same enclosure, never more boxes
    p = S.chain(n=8, seed=3)
    o = O.Oracle(p, block=4)
    a = o.solve(split_m=2, split_d=4, max_parents=4)
    b = o.solve(split_m=2, split_d=4, max_parents=4, mono_all=True)
    assert a.status == b.status == O.ST_OK
    assert b.glb <= 0.0 <= b.gub and b.gub - b.glb <= p.tol_f
    assert b.evals64 <= a.evals64 * 2


CASES = [("sep_cos", dict(n=2), dict(split_m=2, split_d=1)),
         ("sep_cos", dict(n=3, tol_f=1e-6), dict(split_m=4, split_d=3)),
         ("chain", dict(n=6, block=3), dict(split_m=2, split_d=3)),
         ("chain", dict(n=10, block=5), dict(split_m=2, split_d=5, max_parents=8)),
         ("ackley", dict(n=3), dict(split_m=2, split_d=3)),
         ("mixed", dict(n=6, block=3), dict(split_m=2, split_d=3)),
         ("prod_poly", dict(n=6, block=3), dict(split_m=2, split_d=3, max_parents=16))]


@pytest.mark.parametrize("fp32", [False, True])
@pytest.mark.parametrize("fam,kw,opt", CASES)
def test_planted_minimum_enclosed(fam, kw, opt, fp32):
    p = S.make(fam, seed=2, **kw)
    res = O.Oracle(p).solve(fp32=fp32, **opt)
    assert res.status == O.ST_OK
    assert res.glb <= 0.0 <= res.gub
    assert res.gub - res.glb <= p.tol_f
    assert _covers(res, p.s)
    assert np.all(res.box_flo <= res.gub)


def test_separable_reduction():
    p = S.sep_cos(n=2, seed=5, tol_f=1e-9)
    res = O.Oracle(p).solve(split_m=2, split_d=1)
    a, b, s = p.tables
    lo_sum = hi_sum = 0.0
    for j in range(2):
        g = S.Dag()
        ta, tb, ts = g.table(a[j:j + 1]), g.table(b[j:j + 1]), g.table(s[j:j + 1])
        y = g.sub(g.ivar(0), g.icoef(ts))
        term = g.add(g.mul(g.icoef(ta), g.sqr(y)),
                     g.mul(g.icoef(tb), g.sub(g.const(1.0), g.cos(g.mul(g.scale(g.pi(), 2.0), y)))))
        root = g.isum(term, 0, 1, 1)
        q = S.Problem("1d", 1, g.nodes(), root, g.tables,
                      p.l[j:j + 1], p.u[j:j + 1], 1e-9, 1, s[j:j + 1], 0)
        r1 = O.Oracle(q).solve(split_m=2, split_d=1)
        assert r1.glb <= 0.0 <= r1.gub
        lo_sum += r1.glb
        hi_sum += r1.gub
    # both enclose the same minimum 0: the intervals must overlap
    assert max(lo_sum, res.glb) <= min(hi_sum, res.gub) + 1e-15


@pytest.mark.parametrize("fam,kw", [("sep_cos", dict(n=2)), ("chain", dict(n=3, block=3)),
                                     ("ackley", dict(n=2)), ("paper_breiman", dict(n=2)),
                                     ("paper_griewank", dict(n=2)), ("paper_styblinski", dict(n=2)),
                                     ("paper_zabinsky", dict(n=2)), ("prod_poly", dict(n=3, block=3))])
def test_brute_force_grid(fam, kw):
    import itertools
    import mp_ref
    p = S.make(fam, **kw) if fam.startswith("paper") else S.make(fam, seed=3, **kw)
    res = O.Oracle(p).solve(tol_f=1e-6, split_m=2, split_d=p.block)
    G = 41 if p.n == 2 else 17
    axes = [np.linspace(p.l[j], p.u[j], G) for j in range(p.n)]
    pts = list(itertools.product(*axes)) + [tuple(p.s)]
    vals = [float(mp_ref.point_value(p, x, dps=30)) for x in pts]
    k = int(np.argmin(vals))
    assert min(vals) >= res.glb                 # GLB is a lower bound of f
    fstar = p.meta.get("fstar", -0.1 * p.n) if fam.startswith("paper") else 0.0
    assert res.glb <= fstar <= res.gub
    # every point with f below the final GUB lies in some output region
    for x, v in zip(pts, vals):
        if v < res.gub:
            assert _covers(res, np.array(x)), (x, v)
    assert vals[k] >= res.glb


def test_determinism():
    p = S.chain(n=8, seed=7, block=4)
    a = O.Oracle(p).solve(split_m=2, split_d=2, max_parents=16)
    b = O.Oracle(p).solve(split_m=2, split_d=2, max_parents=16)
    assert a.glb == b.glb and a.gub == b.gub and a.generations == b.generations
    assert np.array_equal(a.box_lo, b.box_lo) and np.array_equal(a.box_hi, b.box_hi)
    assert np.array_equal(a.trace["gub"], b.trace["gub"])


def test_capacity_and_limit_keep_a_valid_enclosure():
    p = S.chain(n=8, seed=1, block=4)
    r = O.Oracle(p).solve(split_m=2, split_d=4, cap=40)
    assert r.status == O.ST_CAPACITY
    assert r.glb <= 0.0 <= r.gub and _covers(r, p.s)
    r = O.Oracle(p).solve(split_m=2, split_d=1, max_gen=5)
    assert r.status == O.ST_LIMIT and r.generations == 5
    assert r.glb <= 0.0 <= r.gub and _covers(r, p.s)


def test_bad_options_rejected():
    p = S.chain(n=4)
    assert O.Oracle(p).solve(split_m=3).status == O.ST_INVALID
    assert O.Oracle(p).solve(split_d=0).status == O.ST_INVALID


@pytest.mark.parametrize("fp32", [False, True])
def test_threaded_oracle_equals_single_thread(oracle_mod, fp32):
    # the per-child passes on several threads write per-child slots and take
    # an exact minimum: the run must be the same as on one thread
    p = S.ackley(n=12, seed=3, block=6) if fp32 else S.chain(n=12, seed=5, block=6)
    o = oracle_mod.Oracle(p, block=6)
    a = o.solve(split_m=2, split_d=3, max_parents=8, fp32=fp32, threads=1)
    b = o.solve(split_m=2, split_d=3, max_parents=8, fp32=fp32, threads=5)
    assert a.status == b.status and a.generations == b.generations
    for k in a.trace:
        assert np.array_equal(a.trace[k], b.trace[k]), k
    assert a.glb == b.glb and a.gub == b.gub and a.mids == b.mids and a.evals64 == b.evals64
    assert np.array_equal(a.box_lo, b.box_lo) and np.array_equal(a.box_flo, b.box_flo)
