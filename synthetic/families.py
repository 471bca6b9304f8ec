"""Seeded synthetic minimisation problems with a planted global minimum.

Every family is a sum of non-negative terms that vanish at a seeded point s,
so min f = 0 is attained at x = s (the closed form that pins the solvers).
Coefficients are drawn as FP64 from numpy's PCG64 generator; nothing here
performs interval arithmetic or any step of the branch-and-bound method.

Families (shapes follow the paper's benchmark families of SI Appendix A and D,
shifted so the minimiser is planted):

* ``sep_cos``  (C0): sum_i a_i (x_i-s_i)^2 + b_i (1 - cos(2 pi (x_i-s_i)))
                     a~U[0.5,2], b~U[5,15], s~U[-2,2], box [-5.12,5.12]^n
* ``chain``    (C1): sum_{i<n-1} alpha_i ((x_{i+1}-s_{i+1}) - (x_i-s_i)^2)^2
                                 + beta_i (x_i-s_i)^2
                     alpha~U[50,150], beta~U[0.5,2], s~U[-1,2], box [-5,10]^n
* ``ackley``   (C2): -20 exp(-0.2 sqrt(mean((x-s)^2))) - exp(mean(cos(2 pi (x-s))))
                     + 20 + e + sum_i gamma_i (x_i-s_i)^2
                     gamma~U[0,0.01], s~U[-3,3], box [-32.768,32.768]^n
* ``mixed``    (C3): sep_cos terms on even i (s~U[-2,2]) and chain terms on odd
                     i (s~U[-1,2]; the alpha part only when i+1<n),
                     box [-5.12,5.12]^n
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .dag import Dag


@dataclass
class Problem:
    family: str
    n: int
    nodes: np.ndarray
    root: int
    tables: list
    l: np.ndarray
    u: np.ndarray
    tol_f: float
    block: int
    s: np.ndarray
    seed: int
    meta: dict = field(default_factory=dict)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _shifted(g: Dag, s_tab: int, off: int = 0) -> int:
    """Template node for y = x[i+off] - s[i+off]."""
    return g.sub(g.ivar(off), g.icoef(s_tab, off))


def sep_cos(n: int = 2, seed: int = 0, tol_f: float = 1e-8, block: int | None = None) -> Problem:
    r = _rng(seed)
    a = r.uniform(0.5, 2.0, n)
    b = r.uniform(5.0, 15.0, n)
    s = r.uniform(-2.0, 2.0, n)
    g = Dag()
    ta, tb, ts = g.table(a), g.table(b), g.table(s)
    y = _shifted(g, ts)
    quad = g.mul(g.icoef(ta), g.sqr(y))
    two_pi = g.scale(g.pi(), 2.0)
    osc = g.mul(g.icoef(tb), g.sub(g.const(1.0), g.cos(g.mul(two_pi, y))))
    term = g.add(quad, osc)
    root = g.isum(term, 0, n, 1)
    return Problem("sep_cos", n, g.nodes(), root, g.tables,
                   np.full(n, -5.12), np.full(n, 5.12), tol_f,
                   block if block else min(n, 10), s, seed)


def chain(n: int = 100, seed: int = 0, tol_f: float = 1e-6, block: int | None = None) -> Problem:
    if n < 2:
        raise ValueError("chain needs n >= 2")
    r = _rng(seed)
    alpha = r.uniform(50.0, 150.0, n)
    beta = r.uniform(0.5, 2.0, n)
    s = r.uniform(-1.0, 2.0, n)
    g = Dag()
    tal, tbe, ts = g.table(alpha), g.table(beta), g.table(s)
    y0 = _shifted(g, ts, 0)
    y1 = _shifted(g, ts, 1)
    sq0 = g.sqr(y0)
    t_alpha = g.mul(g.icoef(tal), g.sqr(g.sub(y1, sq0)))
    t_beta = g.mul(g.icoef(tbe), g.sqr(y0))
    root = g.isum(g.add(t_alpha, t_beta), 0, n - 1, 1)
    return Problem("chain", n, g.nodes(), root, g.tables,
                   np.full(n, -5.0), np.full(n, 10.0), tol_f,
                   block if block else min(n, 10), s, seed)


def ackley(n: int = 1000, seed: int = 0, tol_f: float = 1e-6, block: int | None = None) -> Problem:
    r = _rng(seed)
    gamma = r.uniform(0.0, 0.01, n)
    s = r.uniform(-3.0, 3.0, n)
    g = Dag()
    tg, ts = g.table(gamma), g.table(s)
    # template 1: (x_i - s_i)^2
    t1 = g.sqr(_shifted(g, ts))
    s1 = g.isum(t1, 0, n, 1)
    # template 2: cos(2 pi (x_i - s_i))
    two_pi = g.scale(g.pi(), 2.0)
    t2 = g.cos(g.mul(two_pi, _shifted(g, ts)))
    s2 = g.isum(t2, 0, n, 1)
    # template 3: gamma_i (x_i - s_i)^2
    t3 = g.mul(g.icoef(tg), g.sqr(_shifted(g, ts)))
    s3 = g.isum(t3, 0, n, 1)
    nn = g.const(float(n))
    a_part = g.scale(g.exp(g.scale(g.sqrt(g.div(s1, nn)), -0.2)), -20.0)
    c_part = g.neg(g.exp(g.div(s2, nn)))
    f = g.add(g.add(g.add(a_part, c_part), g.add(g.const(20.0), g.euler())), s3)
    return Problem("ackley", n, g.nodes(), f, g.tables,
                   np.full(n, -32.768), np.full(n, 32.768), tol_f,
                   block if block else min(n, 10), s, seed)


def mixed(n: int = 10000, seed: int = 0, tol_f: float = 1e-6, block: int | None = None) -> Problem:
    if n < 2:
        raise ValueError("mixed needs n >= 2")
    r = _rng(seed)
    even = np.arange(n) % 2 == 0
    a = np.where(even, r.uniform(0.5, 2.0, n), 0.0)
    b = np.where(even, r.uniform(5.0, 15.0, n), 0.0)
    alpha = np.where(~even, r.uniform(50.0, 150.0, n), 0.0)
    beta = np.where(~even, r.uniform(0.5, 2.0, n), 0.0)
    s = np.where(even, r.uniform(-2.0, 2.0, n), r.uniform(-1.0, 2.0, n))
    g = Dag()
    ta, tb, tal, tbe, ts = (g.table(a), g.table(b), g.table(alpha),
                            g.table(beta), g.table(s))
    # even i: separable cosine term
    y = _shifted(g, ts)
    two_pi = g.scale(g.pi(), 2.0)
    t_even = g.add(g.mul(g.icoef(ta), g.sqr(y)),
                   g.mul(g.icoef(tb), g.sub(g.const(1.0), g.cos(g.mul(two_pi, y)))))
    s_even = g.isum(t_even, 0, n, 2)
    # odd i with i+1 < n: chain term
    y0 = _shifted(g, ts, 0)
    y1 = _shifted(g, ts, 1)
    sq0 = g.sqr(y0)
    t_odd = g.add(g.mul(g.icoef(tal), g.sqr(g.sub(y1, sq0))),
                  g.mul(g.icoef(tbe), g.sqr(y0)))
    last_odd = n - 1 if (n - 1) % 2 == 1 else n - 2
    end_full = last_odd if last_odd + 1 >= n else last_odd + 2
    f = s_even
    if end_full > 1:
        f = g.add(f, g.isum(t_odd, 1, end_full, 2))
    if last_odd + 1 >= n:  # odd index n-1 has no successor: beta term only
        t_tail = g.mul(g.icoef(tbe), g.sqr(_shifted(g, ts)))
        f = g.add(f, g.isum(t_tail, last_odd, last_odd + 1, 1))
    return Problem("mixed", n, g.nodes(), f, g.tables,
                   np.full(n, -5.12), np.full(n, 5.12), tol_f,
                   block if block else min(n, 100), s, seed)


def prod_poly(n: int = 8, seed: int = 0, tol_f: float = 1e-6, block: int | None = None) -> Problem:
    """A polynomial objective with a coupled product (products over an index
    set, no transcendentals, so every interval operation is exact up to its
    directed rounding):
    sum_i (x_i - c_i)^2 + prod_{i<n-1} (1 + a_i ((x_i - c_i) - (x_{i+1} - c_{i+1}))^2) - 1,
    a_i ~ U[0.5, 2], c_i ~ U[-1, 1], box [-2, 3]^n; min 0 at x = c (every factor >= 1)."""
    if n < 2:
        raise ValueError("prod_poly needs n >= 2")
    r = _rng(seed)
    a = r.uniform(0.5, 2.0, n)
    c = r.uniform(-1.0, 1.0, n)
    g = Dag()
    ta, tc = g.table(a), g.table(c)
    d0 = g.sub(g.ivar(0), g.icoef(tc))
    s1 = g.isum(g.sqr(d0), 0, n, 1)
    d1 = g.sub(g.sub(g.ivar(0), g.icoef(tc)), g.sub(g.ivar(1), g.icoef(tc, 1)))
    p1 = g.iprod(g.add(g.const(1.0), g.mul(g.icoef(ta), g.sqr(d1))), 0, n - 1, 1)
    f = g.sub(g.add(s1, p1), g.const(1.0))
    return Problem("prod_poly", n, g.nodes(), f, g.tables, np.full(n, -2.0), np.full(n, 3.0), tol_f,
                   block if block else min(n, 10), c.copy(), seed)


FAMILIES = {"sep_cos": sep_cos, "chain": chain, "ackley": ackley, "mixed": mixed, "prod_poly": prod_poly}


def make(family: str, **kw) -> Problem:
    return FAMILIES[family](**kw)


def random_boxes(p: Problem, count: int, seed: int, min_width: float = 1e-6,
                 max_frac: float = 1.0, around_s: float = 0.0) -> tuple[np.ndarray, np.ndarray]:
    """Seeded random sub-boxes of [l, u] (count x n, row-major).

    Each coordinate interval has a log-uniform width between ``min_width`` and
    ``max_frac`` of the domain width.  With ``around_s`` > 0 a fraction of the
    boxes is placed so that it contains the planted point s.
    """
    r = _rng(seed)
    n = p.n
    span = p.u - p.l
    lw = r.uniform(np.log(min_width), np.log(max_frac), (count, n))
    w = np.minimum(np.exp(lw) * span, span)
    lo = p.l + r.uniform(0.0, 1.0, (count, n)) * (span - w)
    if around_s > 0.0:
        pick = r.uniform(0.0, 1.0, count) < around_s
        shift = r.uniform(0.0, 1.0, (count, n)) * w
        lo_s = np.clip(p.s - shift, p.l, p.u - w)
        lo = np.where(pick[:, None], lo_s, lo)
    hi = np.minimum(lo + w, p.u)
    lo = np.maximum(lo, p.l)
    return np.ascontiguousarray(lo), np.ascontiguousarray(hi)


def serving_stream(count: int = 512, seed: int = 0, rate: float = 20.0,
                   n_min: int = 2, n_max: int = 2000, tol_f: float = 1e-6):
    """Poisson request stream: (arrival time s, Problem) pairs.

    n is log-uniform on [n_min, n_max]; the family is uniform over
    sep_cos / chain / ackley; every request draws fresh coefficients.
    """
    r = _rng(seed)
    gaps = r.exponential(1.0 / rate, count)
    t = np.cumsum(gaps)
    out = []
    fams = ["sep_cos", "chain", "ackley"]
    for k in range(count):
        n = int(round(np.exp(r.uniform(np.log(n_min), np.log(n_max)))))
        fam = fams[int(r.integers(0, 3))]
        sub_seed = int(r.integers(0, 2**31 - 1))
        if fam == "chain":
            n = max(n, 2)
        out.append((float(t[k]), make(fam, n=n, seed=sub_seed, tol_f=tol_f)))
    return out


# ---------------------------------------------------------------------------
# Benchmark functions printed in the paper (SI Appendix A), unshifted.
def paper_rastrigin(n: int = 10, tol_f: float = 0.0, block: int | None = None) -> Problem:
    """Eq. S14-S15: 10n + sum_i (x_i^2 - 10 cos(2 pi x_i)), -5.5 <= x_i <= 6."""
    g = Dag()
    x = g.ivar(0)
    two_pi = g.scale(g.pi(), 2.0)
    term = g.sub(g.sqr(x), g.scale(g.cos(g.mul(two_pi, x)), 10.0))
    root = g.add(g.const(10.0 * n), g.isum(term, 0, n, 1))
    return Problem("paper_rastrigin", n, g.nodes(), root, g.tables,
                   np.full(n, -5.5), np.full(n, 6.0), tol_f,
                   block if block else min(n, 10), np.zeros(n), 0)


def paper_breiman(n: int = 10, tol_f: float = 0.0, block: int | None = None) -> Problem:
    """Eq. S5-S6: -0.1 sum_i cos(5 pi x_i) + sum_i x_i^2, -1 <= x_i <= 2."""
    g = Dag()
    x = g.ivar(0)
    five_pi = g.scale(g.pi(), 5.0)
    term = g.sub(g.sqr(x), g.scale(g.cos(g.mul(five_pi, x)), 0.1))
    root = g.isum(term, 0, n, 1)
    return Problem("paper_breiman", n, g.nodes(), root, g.tables,
                   np.full(n, -1.0), np.full(n, 2.0), tol_f,
                   block if block else min(n, 10), np.zeros(n), 0)


def paper_ackley(n: int = 10, tol_f: float = 0.0, block: int | None = None) -> Problem:
    """Eq. S1-S2 as printed: -20 exp(-0.02 sqrt(mean x_i^2)) - exp(mean cos(2 pi x_i)) + 20 + e,
    -35 <= x_i <= 40; min 0 at x = 0."""
    g = Dag()
    x = g.ivar(0)
    s1 = g.isum(g.sqr(x), 0, n, 1)
    s2 = g.isum(g.cos(g.mul(g.scale(g.pi(), 2.0), x)), 0, n, 1)
    nn = g.const(float(n))
    a_part = g.scale(g.exp(g.scale(g.sqrt(g.div(s1, nn)), -0.02)), -20.0)
    c_part = g.neg(g.exp(g.div(s2, nn)))
    f = g.add(g.add(a_part, c_part), g.add(g.const(20.0), g.euler()))
    return Problem("paper_ackley", n, g.nodes(), f, g.tables, np.full(n, -35.0), np.full(n, 40.0), tol_f,
                   block if block else min(n, 10), np.zeros(n), 0, meta=dict(fstar=0.0))


def paper_belegundu(n: int = 10, tol_f: float = 0.0, block: int | None = None) -> Problem:
    """Eq. S3-S4: 0.1 sum (x_i - 5)^2 - cos(5 sqrt(sum (x_i - 5)^2)), -10 <= x_i <= 11; min -1 at x = 5."""
    g = Dag()
    d = g.sub(g.ivar(0), g.const(5.0))
    s1 = g.isum(g.sqr(d), 0, n, 1)
    f = g.sub(g.scale(s1, 0.1), g.cos(g.scale(g.sqrt(s1), 5.0)))
    return Problem("paper_belegundu", n, g.nodes(), f, g.tables, np.full(n, -10.0), np.full(n, 11.0), tol_f,
                   block if block else min(n, 10), np.full(n, 5.0), 0, meta=dict(fstar=-1.0))


def paper_fu(n: int = 10, tol_f: float = 0.0, block: int | None = None) -> Problem:
    """Eq. S7-S8: 1 + sum [8 sin^2(7 (x_i - 0.9)^2) + 6 sin^2(14 (x_i - 0.9)^2) + (x_i - 0.9)^2],
    -10 <= x_i <= 10; min 1 at x = 0.9."""
    g = Dag()
    q = g.sqr(g.sub(g.ivar(0), g.const(0.9)))
    term = g.add(g.add(g.scale(g.sqr(g.sin(g.scale(q, 7.0))), 8.0), g.scale(g.sqr(g.sin(g.scale(q, 14.0))), 6.0)),
                 q)
    f = g.add(g.const(1.0), g.isum(term, 0, n, 1))
    return Problem("paper_fu", n, g.nodes(), f, g.tables, np.full(n, -10.0), np.full(n, 10.0), tol_f,
                   block if block else min(n, 10), np.full(n, 0.9), 0, meta=dict(fstar=1.0))


def paper_levy(n: int = 10, tol_f: float = 0.0, block: int | None = None) -> Problem:
    """Eq. S11-S13 with y_i = 1 + 0.25 (x_i - 1) (so y_i - 1 = 0.25 (x_i - 1)):
    (pi / n) {10 sin^2(pi y_1) + (y_n - 1)^2 + sum_{i<n} (y_i - 1)^2 (1 + 10 sin^2(pi y_{i+1}))},
    -10 <= x_i <= 10; min 0 at x = 1."""
    if n < 2:
        raise ValueError("paper_levy needs n >= 2")
    g = Dag()

    def y(node):          # y = 1 + 0.25 (x - 1)
        return g.add(g.const(1.0), g.scale(g.sub(node, g.const(1.0)), 0.25))

    def ym1_sq(node):     # (y - 1)^2 = (0.25 (x - 1))^2
        return g.sqr(g.scale(g.sub(node, g.const(1.0)), 0.25))

    def sin2_pi(node):    # sin^2(pi y)
        return g.sqr(g.sin(g.mul(g.pi(), y(node))))

    term = g.mul(ym1_sq(g.ivar(0)), g.add(g.const(1.0), g.scale(sin2_pi(g.ivar(1)), 10.0)))
    inner = g.add(g.add(g.scale(sin2_pi(g.var(0)), 10.0), ym1_sq(g.var(n - 1))), g.isum(term, 0, n - 1, 1))
    f = g.div(g.mul(g.pi(), inner), g.const(float(n)))
    return Problem("paper_levy", n, g.nodes(), f, g.tables, np.full(n, -10.0), np.full(n, 10.0), tol_f,
                   block if block else min(n, 10), np.ones(n), 0, meta=dict(fstar=0.0))


def paper_salomon(n: int = 10, tol_f: float = 0.0, block: int | None = None) -> Problem:
    """Eq. S16-S17: 1 - cos(2 pi sqrt(sum x_i^2)) + 0.1 sqrt(sum x_i^2), -100 <= x_i <= 110; min 0 at x = 0."""
    g = Dag()
    r = g.sqrt(g.isum(g.sqr(g.ivar(0)), 0, n, 1))
    f = g.add(g.sub(g.const(1.0), g.cos(g.mul(g.scale(g.pi(), 2.0), r))), g.scale(r, 0.1))
    return Problem("paper_salomon", n, g.nodes(), f, g.tables, np.full(n, -100.0), np.full(n, 110.0), tol_f,
                   block if block else min(n, 10), np.zeros(n), 0, meta=dict(fstar=0.0))


def paper_rosenbrock(n: int = 10, tol_f: float = 0.0, block: int | None = None) -> Problem:
    """Eq. S22-S23: sum_{i<n} [100 (x_i^2 - x_{i+1})^2 + (x_i - 1)^2], -30 <= x_i <= 30; min 0 at x = 1."""
    if n < 2:
        raise ValueError("paper_rosenbrock needs n >= 2")
    g = Dag()
    term = g.add(g.scale(g.sqr(g.sub(g.sqr(g.ivar(0)), g.ivar(1))), 100.0), g.sqr(g.sub(g.ivar(0), g.const(1.0))))
    f = g.isum(term, 0, n - 1, 1)
    return Problem("paper_rosenbrock", n, g.nodes(), f, g.tables, np.full(n, -30.0), np.full(n, 30.0), tol_f,
                   block if block else min(n, 10), np.ones(n), 0, meta=dict(fstar=0.0))


def paper_griewank(n: int = 10, tol_f: float = 0.0, block: int | None = None) -> Problem:
    """Eq. S9-S10: 1 + sum_i x_i^2 / 4000 - prod_i cos(x_i / sqrt(i)) (i = 1..n), -100 <= x_i <= 110;
    min 0 at x = 0.  sqrt(i) is the interval square root of the exact integer i (table 0)."""
    g = Dag()
    x = g.ivar(0)
    idx = g.table(np.arange(1, n + 1, dtype=np.float64))
    s1 = g.isum(g.div(g.sqr(x), g.const(4000.0)), 0, n, 1)
    p1 = g.iprod(g.cos(g.div(x, g.sqrt(g.icoef(idx)))), 0, n, 1)
    f = g.sub(g.add(g.const(1.0), s1), p1)
    return Problem("paper_griewank", n, g.nodes(), f, g.tables, np.full(n, -100.0), np.full(n, 110.0), tol_f,
                   block if block else min(n, 10), np.zeros(n), 0, meta=dict(fstar=0.0))


def paper_styblinski(n: int = 10, tol_f: float = 0.0, block: int | None = None) -> Problem:
    """Eq. S18-S19: (1 / (2n)) sum_i x_i^2 - 4n prod_i cos(x_i), -10 <= x_i <= 11; min -4n at x = 0."""
    g = Dag()
    x = g.ivar(0)
    s1 = g.div(g.isum(g.sqr(x), 0, n, 1), g.const(2.0 * n))
    p1 = g.iprod(g.cos(x), 0, n, 1)
    f = g.sub(s1, g.scale(p1, 4.0 * n))
    return Problem("paper_styblinski", n, g.nodes(), f, g.tables, np.full(n, -10.0), np.full(n, 11.0), tol_f,
                   block if block else min(n, 10), np.zeros(n), 0, meta=dict(fstar=-4.0 * n))


def paper_zabinsky(n: int = 10, tol_f: float = 0.0, block: int | None = None) -> Problem:
    """Eq. S20-S21: -2.5 prod_i sin(x_i - pi/6) - prod_i sin(5 (x_i - pi/6)), 0 <= x_i <= pi;
    min -3.5 at x = 2 pi / 3.  The upper bound is the double nearest pi (just below it)."""
    g = Dag()
    d = g.sub(g.ivar(0), g.div(g.pi(), g.const(6.0)))
    p1 = g.iprod(g.sin(d), 0, n, 1)
    p2 = g.iprod(g.sin(g.scale(d, 5.0)), 0, n, 1)
    f = g.sub(g.scale(p1, -2.5), p2)
    return Problem("paper_zabinsky", n, g.nodes(), f, g.tables, np.zeros(n), np.full(n, np.pi), tol_f,
                   block if block else min(n, 10), np.full(n, 2.0 * np.pi / 3.0), 0, meta=dict(fstar=-3.5))


def paper_discontinuous(n: int = 10, tol_f: float = 0.0, block: int | None = None) -> Problem:
    """Eq. S24-S27: -1 on the small cube D = [1.5 - eps/2, 1.5 + eps/2]^n (eps = 1e-6; S24 prints
    1.5 - eps/2 on both sides, read as the cube centred on 1.5), the Levy function L elsewhere,
    -10 <= x_i <= 10; min -1 on D.  Written as (1 - I) L - I with the indicator
    I = prod_i H(x_i - a) H(b - x_i) of D (H the unit step; a, b the doubles nearest 1.5 -/+ eps/2)."""
    lev = paper_levy(n=n, tol_f=tol_f, block=block)
    g = Dag()
    g._nodes = [tuple(r) for r in lev.nodes.tolist()]
    g.tables = list(lev.tables)
    eps = 1e-6
    a, b = 1.5 - eps / 2, 1.5 + eps / 2
    x = g.ivar(0)
    ind = g.iprod(g.mul(g.step(g.sub(x, g.const(a))), g.step(g.sub(g.const(b), x))), 0, n, 1)
    f = g.sub(g.mul(g.sub(g.const(1.0), ind), int(lev.root)), ind)
    return Problem("paper_discontinuous", n, g.nodes(), f, g.tables, lev.l, lev.u, tol_f,
                   lev.block, np.full(n, 1.5), 0, meta=dict(fstar=-1.0, cube=(a, b)))


FAMILIES.update(paper_discontinuous=paper_discontinuous)
FAMILIES.update(paper_griewank=paper_griewank, paper_styblinski=paper_styblinski, paper_zabinsky=paper_zabinsky)
FAMILIES.update(paper_rastrigin=paper_rastrigin, paper_breiman=paper_breiman, paper_ackley=paper_ackley,
                paper_belegundu=paper_belegundu, paper_fu=paper_fu, paper_levy=paper_levy,
                paper_salomon=paper_salomon, paper_rosenbrock=paper_rosenbrock)
