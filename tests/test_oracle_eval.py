"""Pins of the oracle's box evaluation: F(X), the interval partials and the
first-order test (section 3.1), against references that do not share its code.

* the reduction tree against exact rational arithmetic with directed rounding;
* F(X) for polynomial objectives bit-for-bit against mpmath's 53-bit interval
  arithmetic in the same grouping and order;
* containment (the rigour claim of section 2.1): for sampled points p in X,
  f(p) computed at 60 digits lies in F(X) and each partial at p in G(X)_j;
* the closed form: every family has f(s) = 0 at its planted point.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

pytest.importorskip("mpmath")
import mpmath  # noqa: E402

import oracle as O  # noqa: E402
import synthetic as S  # noqa: E402
import mp_ref  # noqa: E402


def _rd(fr: Fraction) -> float:
    x = float(fr)
    if Fraction(x) > fr:
        x = math.nextafter(x, -math.inf)
    return x


def _ru(fr: Fraction) -> float:
    x = float(fr)
    if Fraction(x) < fr:
        x = math.nextafter(x, math.inf)
    return x


def _exact_tree(lo, hi):
    a = [(float(l), float(h)) for l, h in zip(lo, hi)]
    m = len(a)
    s = 1
    while s < m:
        for i in range(0, m - s, 2 * s):
            a[i] = (_rd(Fraction(a[i][0]) + Fraction(a[i + s][0])),
                    _ru(Fraction(a[i][1]) + Fraction(a[i + s][1])))
        s *= 2
    return a[0] if m else (0.0, 0.0)


def test_tree_sum_matches_exact_rational_rounding():
    rng = np.random.default_rng(3)
    for m in list(range(1, 40)) + [63, 64, 65, 100]:
        mag = 10.0 ** rng.uniform(-8, 8, m)
        lo = rng.uniform(-1, 1, m) * mag
        hi = lo + np.abs(rng.uniform(0, 1, m)) * mag
        assert O.tree_sum(lo, hi) == _exact_tree(lo, hi)


def _exact_mul(a, b):
    ps = [Fraction(x) * Fraction(y) for x in a for y in b]
    return (_rd(min(ps)), _ru(max(ps)))


def _exact_prod_tree(lo, hi):
    a = [(float(l), float(h)) for l, h in zip(lo, hi)]
    m = len(a)
    s = 1
    while s < m:
        for i in range(0, m - s, 2 * s):
            a[i] = _exact_mul(a[i], a[i + s])
        s *= 2
    return a[0] if m else (1.0, 1.0)


def _random_intervals(rng, m):
    mag = 2.0 ** rng.integers(-20, 20, m)
    lo = rng.uniform(-1, 1, m) * mag
    hi = lo + np.abs(rng.uniform(0, 1, m)) * mag
    return lo, hi


def test_tree_prod_matches_exact_rational_rounding():
    # the IPROD reduction: the pairwise tree of tree_sum with products, each
    # node the optimal outward rounding of the exact interval product
    rng = np.random.default_rng(4)
    for m in list(range(0, 20)) + [31, 32, 33, 50]:
        lo, hi = _random_intervals(rng, m)
        assert O.tree_prod(lo, hi) == _exact_prod_tree(lo, hi)


def test_tree_prod_adjoint_closed_form_on_exact_points():
    # d/dx_i prod_j x_j = prod_{j != i} x_j: with signed powers of two every
    # product is exact, so the reverse sweep must give it exactly (a wrong
    # partner, a skipped level or the item's own value fails here)
    rng = np.random.default_rng(5)
    for m in (1, 2, 3, 5, 7, 8, 13, 16, 21):
        x = rng.choice([-1.0, 1.0], m) * 2.0 ** rng.integers(-6, 6, m)
        seed = (0.75, 0.75)
        adj = O.tree_prod_adjoint(x, x, seed)
        for i in range(m):
            want = 0.75 * float(np.prod(np.delete(x, i)))
            assert adj[i, 0] == want == adj[i, 1], (m, i)


def test_tree_prod_adjoint_encloses_partial_products():
    # for interval items the adjoint of item i must enclose prod_{j != i} x_j
    # at every point of the box (exact rational check at sampled points)
    rng = np.random.default_rng(6)
    for m in (2, 3, 6, 9, 17):
        lo, hi = _random_intervals(rng, m)
        adj = O.tree_prod_adjoint(lo, hi)
        for _ in range(20):
            t = rng.uniform(0, 1, m)
            t[rng.integers(0, m)] = rng.integers(0, 2)
            x = [Fraction(float(a)) + (Fraction(float(b)) - Fraction(float(a))) * Fraction(float(u))
                 for a, b, u in zip(lo, hi, t)]
            for i in range(m):
                pr = Fraction(1)
                for j in range(m):
                    if j != i:
                        pr *= x[j]
                assert Fraction(adj[i, 0]) <= pr <= Fraction(adj[i, 1])


def test_tree_sum_is_not_sequential():
    # 1 + 3 * 2^-53: sequential rounding down keeps 1, the pairwise tree
    # first adds the two small terms exactly
    lo = np.array([1.0, 2.0**-53, 2.0**-53, 2.0**-53])
    got = O.tree_sum(lo, lo)
    seq = 1.0
    for v in lo[1:]:
        seq = _rd(Fraction(seq) + Fraction(v))
    assert got == _exact_tree(lo, lo)
    assert got[0] != seq


def _poly_product_problem(n):
    """1 + prod_i (1 + a_i (x_i - x_{i+1})^2) - prod_i (x_i - c_i): polynomial IPROD templates."""
    rng = np.random.default_rng(n)
    g = S.Dag()
    ta = g.table(rng.uniform(0.5, 2.0, n))
    tc = g.table(rng.uniform(-1.0, 1.0, n))
    t1 = g.add(g.const(1.0), g.mul(g.icoef(ta), g.sqr(g.sub(g.ivar(0), g.ivar(1)))))
    t2 = g.sub(g.ivar(0), g.icoef(tc))
    f = g.sub(g.add(g.const(1.0), g.iprod(t1, 0, n - 1, 1)), g.iprod(t2, 0, n, 1))
    return S.Problem("poly_prod", n, g.nodes(), f, g.tables, np.full(n, -2.0), np.full(n, 3.0),
                     1e-6, 3, np.zeros(n), 0)


@pytest.mark.parametrize("n,B", [(3, 3), (7, 3), (12, 5), (21, 4)])
def test_polynomial_product_F_bit_exact_vs_mpmath(n, B):
    p = _poly_product_problem(n)
    o = O.Oracle(p, block=B)
    lo, hi = S.random_boxes(p, 30, seed=n + 7)
    for k in range(len(lo)):
        F, _, _, _ = o.eval_box(lo[k], hi[k])
        assert tuple(F) == mp_ref.iv53_value(p, lo[k], hi[k], B)


def test_polynomial_product_partials_contain_derivative():
    p = _poly_product_problem(8)
    B = 3
    o = O.Oracle(p, block=B)
    rng = np.random.default_rng(9)
    lo, hi = S.random_boxes(p, 10, seed=19, min_width=1e-4)
    for k in range(len(lo)):
        blk = k % 3
        F, _, G, _ = o.eval_box(lo[k], hi[k], blk=blk)
        for x in _sample_points(rng, lo[k], hi[k], 3):
            assert F[0] <= mp_ref.point_value(p, x) <= F[1]
            for t in range(min(B, p.n - blk * B)):
                gx = mp_ref.point_grad(p, x, blk * B + t)
                assert G[t, 0] <= gx + mpmath.mpf(1e-30) and gx - mpmath.mpf(1e-30) <= G[t, 1]


@pytest.mark.parametrize("n,B", [(2, 2), (5, 3), (7, 3), (12, 5), (20, 10), (33, 10)])
def test_polynomial_F_bit_exact_vs_mpmath(n, B):
    p = S.chain(n=n, seed=n)
    o = O.Oracle(p, block=B)
    lo, hi = S.random_boxes(p, 40, seed=n + 100, around_s=0.5)
    for k in range(len(lo)):
        F, _, _, _ = o.eval_box(lo[k], hi[k])
        assert tuple(F) == mp_ref.iv53_value(p, lo[k], hi[k], B)


def test_polynomial_F_bit_exact_custom_dag():
    # outer VAR leaves, a stride-2 sum, scaling and negation
    g = S.Dag()
    y = g.sub(g.ivar(0), g.ivar(1))
    t = g.mul(g.icoef(g.table(np.linspace(0.5, 3.0, 9))), g.sqr(y))
    s_even = g.isum(t, 0, 8, 2)
    f = g.add(g.sub(s_even, g.scale(g.var(3), -1.5)), g.neg(g.mul(g.var(0), g.var(8))))
    p = S.Problem("custom", 9, g.nodes(), f, g.tables, np.full(9, -2.0), np.full(9, 3.0),
                  1e-6, 3, np.zeros(9), 0)
    o = O.Oracle(p)
    lo, hi = S.random_boxes(p, 60, seed=5)
    for k in range(len(lo)):
        F, _, _, _ = o.eval_box(lo[k], hi[k])
        assert tuple(F) == mp_ref.iv53_value(p, lo[k], hi[k], 3)


def _sample_points(rng, lo, hi, count):
    t = rng.uniform(0, 1, (count, len(lo)))
    t[0] = 0.0
    t[1] = 1.0
    return lo + t * (hi - lo)


CASES = [("sep_cos", dict(n=3)), ("chain", dict(n=6)), ("ackley", dict(n=4)),
         ("mixed", dict(n=7)), ("paper_rastrigin", dict(n=3)), ("paper_breiman", dict(n=3)),
         ("paper_griewank", dict(n=5)), ("paper_styblinski", dict(n=4)), ("paper_zabinsky", dict(n=5)),
         ("prod_poly", dict(n=6)), ("paper_discontinuous", dict(n=4))]


@pytest.mark.parametrize("f32", [False, True])
@pytest.mark.parametrize("fam,kw", CASES)
def test_containment_of_f_and_partials(fam, kw, f32):
    p = S.make(fam, **kw)
    B = max(1, min(p.n, 3))
    o = O.Oracle(p, block=B)
    rng = np.random.default_rng(17)
    lo, hi = S.random_boxes(p, 12, seed=23, min_width=1e-5, around_s=0.4)
    nb = (p.n + B - 1) // B
    for k in range(len(lo)):
        blk = k % nb
        F, Fm, G, _ = o.eval_box(lo[k], hi[k], blk=blk, f32=f32)
        for x in _sample_points(rng, lo[k], hi[k], 4):
            fx = mp_ref.point_value(p, x)
            assert F[0] <= fx <= F[1], (fam, k, F, fx)
            for t in range(min(B, p.n - blk * B)):
                j = blk * B + t
                if fam == "ackley":
                    r = math.sqrt(sum((x[q] - p.s[q]) ** 2 for q in range(p.n)))
                    if r < 1e-6:
                        continue           # derivative undefined at the minimiser
                gx = mp_ref.point_grad(p, x, j)
                assert G[t, 0] <= gx + mpmath.mpf(1e-30) and gx - mpmath.mpf(1e-30) <= G[t, 1], \
                    (fam, k, j, G[t], gx)
        # the midpoint sample is a point enclosure of f at RN(0.5 lo + 0.5 hi)
        mid = 0.5 * lo[k] + 0.5 * hi[k]
        fm = mp_ref.point_value(p, mid)
        assert Fm[0] <= fm <= Fm[1]


def _disc_and_levy(n, B):
    return S.paper_discontinuous(n=n, block=B), S.paper_levy(n=n, block=B)


def test_discontinuous_equals_levy_off_the_cube():
    # Eq. S24: f = L away from the cube D.  Boxes that miss D in some
    # coordinate give the Levy F and the Levy partials bit for bit (the
    # indicator is exactly [0, 0] there and its adjoints vanish)
    n, B = 7, 3
    p, lev = _disc_and_levy(n, B)
    a, b = p.meta["cube"]
    od, ol = O.Oracle(p, block=B), O.Oracle(lev, block=B)
    lo, hi = S.random_boxes(p, 60, seed=31, around_s=0.2)
    k = 0
    for j in range(len(lo)):
        x0, x1 = lo[j].copy(), hi[j].copy()
        q = j % n                         # make coordinate q miss D
        if j % 2:
            x0[q], x1[q] = b + 1e-3, b + 0.5
        else:
            x0[q], x1[q] = a - 0.5, a - 1e-9
        for blk in range((n + B - 1) // B):
            F, Fm, G, M = od.eval_box(x0, x1, blk=blk)
            F2, Fm2, G2, M2 = ol.eval_box(x0, x1, blk=blk)
            assert tuple(F) == tuple(F2) and tuple(Fm) == tuple(Fm2)
            assert np.array_equal(G, G2) and M == M2
            k += 1
    assert k > 0


def test_discontinuous_on_and_across_the_cube():
    n, B = 4, 4
    p, lev = _disc_and_levy(n, B)
    a, b = p.meta["cube"]
    o = O.Oracle(p, block=B)
    # a box inside D: the constant -1, and every partial holds 0
    inner_lo = np.full(n, a + (b - a) / 4)
    inner_hi = np.full(n, b - (b - a) / 4)
    F, _, G, M = o.eval_box(inner_lo, inner_hi, blk=0)
    assert tuple(F) == (-1.0, -1.0)
    assert np.all(G[:, 0] <= 0.0) and np.all(G[:, 1] >= 0.0) and M == 0
    # a box across the boundary of D in every coordinate: F holds -1 and the
    # Levy values of its points off D; the partials are unbounded (no
    # first-order discard of a box that may hold the minimum)
    lo, hi = np.full(n, 1.4), np.full(n, 1.5)
    F, _, G, M = o.eval_box(lo, hi, blk=0)
    FL, _, _, _ = O.Oracle(lev, block=B).eval_box(lo, hi, blk=0)
    assert F[0] <= -1.0 <= F[1] and F[1] >= FL[1] and F[0] <= FL[0]
    assert np.all(np.isinf(G)) and M == 0
    # the GUB sample at a point of D is -1, off D the Levy value
    import mp_ref
    assert mp_ref.point_value(p, np.full(n, 1.5)) == -1
    assert abs(mp_ref.point_value(p, np.full(n, 1.0))) < 1e-50    # Levy's minimum 0 (sin(pi) at 60 digits)


@pytest.mark.parametrize("fam,kw", CASES[:4])
def test_planted_point_encloses_zero_tightly(fam, kw):
    p = S.make(fam, **kw)
    o = O.Oracle(p)
    F, Fm, _, _ = o.eval_box(p.s, p.s)
    assert F[0] <= 0.0 <= F[1]
    assert F[1] - F[0] < 1e-12
    assert mp_ref.point_value(p, p.s) == 0


def test_point_box_partials_are_tight():
    p = S.chain(n=8, seed=4)
    o = O.Oracle(p, block=4)
    rng = np.random.default_rng(9)
    for _ in range(20):
        x = rng.uniform(-1, 2, 8)
        for blk in (0, 1):
            _, _, G, _ = o.eval_box(x, x, blk=blk)
            for t in range(4):
                g = float(mp_ref.point_grad(p, x, blk * 4 + t))
                assert G[t, 0] <= g <= G[t, 1]
                assert G[t, 1] - G[t, 0] <= 1e-10 * max(1.0, abs(g))


def test_monotonicity_rules_out_far_boxes_and_keeps_edges():
    p = S.sep_cos(n=2, seed=1)
    o = O.Oracle(p, block=2)
    s = p.s
    # a thin box right of s_0 in coordinate 0 (derivative > 0 there), s_1 inside
    lo = np.array([s[0] + 1e-3, s[1] - 1e-4])
    hi = np.array([s[0] + 1.1e-3, s[1] + 1e-4])
    _, _, G, mono = o.eval_box(lo, hi, blk=0)
    assert G[0, 0] > 0 and mono == 1
    # the same box containing s in both coordinates is kept
    lo2 = np.array([s[0] - 1e-4, s[1] - 1e-4])
    hi2 = np.array([s[0] + 1e-4, s[1] + 1e-4])
    assert o.eval_box(lo2, hi2, blk=0)[3] == 0
    # a box whose lower face lies on l is exempt when DLB > 0 (edge of the domain)
    g = S.Dag()
    f = g.isum(g.sqr(g.ivar(0)), 0, 1, 1)      # f = x^2 on [1, 3]
    q = S.Problem("edge", 1, g.nodes(), f, g.tables, np.array([1.0]), np.array([3.0]),
                  1e-6, 1, np.array([1.0]), 0)
    oq = O.Oracle(q)
    assert oq.eval_box(np.array([1.0]), np.array([1.5]), blk=0)[3] == 0
    assert oq.eval_box(np.array([1.5]), np.array([2.0]), blk=0)[3] == 1


def test_invalid_problems_are_rejected():
    p = S.chain(n=4)
    bad = p.nodes.copy()
    bad[2]["a"] = 7                          # SUB node referring forward
    q = S.Problem("bad", 4, bad, p.root, p.tables, p.l, p.u, 1e-6, 2, p.s, 0)
    with pytest.raises(ValueError):
        O.Oracle(q)
    q2 = S.Problem("bad", 4, p.nodes, p.root, p.tables, p.l, p.l, 1e-6, 2, p.s, 0)
    with pytest.raises(ValueError):
        O.Oracle(q2)                         # l < u violated


def test_product_special_cases():
    # the empty product is 1; a one-term product is the term; a product of
    # point factors is their exact product when it is representable
    g = S.Dag()
    x = g.ivar(0)
    empty = g.iprod(g.add(x, g.const(1.0)), 2, 2, 1)
    one = g.iprod(g.sqr(x), 1, 2, 1)
    f = g.add(g.scale(empty, 3.0), one)
    p = S.Problem("prod_special", 3, g.nodes(), f, g.tables, np.full(3, -2.0), np.full(3, 2.0), 1e-6, 3,
                  np.zeros(3), 0)
    o = O.Oracle(p, block=3)
    F, _, G, _ = o.eval_box(np.array([0.0, 0.5, 0.0]), np.array([0.0, 0.5, 0.0]), blk=0)
    assert tuple(F) == (3.25, 3.25)
    assert tuple(G[1]) == (1.0, 1.0) and tuple(G[0]) == (0.0, 0.0)
    g2 = S.Dag()
    t = g2.iprod(g2.scale(g2.ivar(0), 2.0), 0, 4, 1)
    p2 = S.Problem("prod_points", 4, g2.nodes(), t, g2.tables, np.full(4, -4.0), np.full(4, 4.0), 1e-6, 4,
                   np.zeros(4), 0)
    pts = np.array([0.5, -1.5, 3.0, 0.25])
    F2, _, G2, _ = O.Oracle(p2, block=4).eval_box(pts, pts, blk=0)
    assert tuple(F2) == (float(np.prod(2 * pts)),) * 2
    for j in range(4):   # d/dx_j prod_i 2 x_i = 2 prod_{i != j} 2 x_i, exact here
        want = 2.0 * float(np.prod(np.delete(2 * pts, j)))
        assert tuple(G2[j]) == (want, want)


def test_nested_reductions_rejected():
    g = S.Dag()
    inner = g.iprod(g.ivar(0), 0, 2, 1)
    f = g.isum(g.add(g.ivar(0), inner), 0, 2, 1)
    p = S.Problem("nested", 2, g.nodes(), f, g.tables, np.zeros(2), np.ones(2), 1e-6, 2, np.zeros(2), 0)
    with pytest.raises(Exception):
        O.Oracle(p, block=2)
