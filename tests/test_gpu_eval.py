"""Per-box parity of the CUDA evaluation with the CPU oracle (runs on a GPU).

For objectives built from +, -, x, square and scaling the FP64 and FP32
results must be bit-identical: F(X), the FP64 midpoint sample, every interval
partial of the tested block, and the first-order verdict.  With sin, cos and
exp both sides widen library results by their own documented error bounds,
so the endpoints must agree within the deviation bound the oracle computes
for each result (the library difference propagated through the evaluation).
"""
import numpy as np
import pytest

import oracle as O
import synthetic as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2507_01770_gb300 as gb  # noqa: E402


def _gpu_eval(solver, lo, hi, blk, fp32):
    dlo = torch.from_numpy(lo).cuda()
    dhi = torch.from_numpy(hi).cuda()
    F, Fm, G, mono = solver.eval_boxes(dlo, dhi, blk, fp32)
    torch.cuda.synchronize()
    return F.cpu().numpy(), Fm.cpu().numpy(), G.cpu().numpy(), mono.cpu().numpy()


def _oracle_eval(orc, lo, hi, blk, fp32):
    F, Fm, G, M = [], [], [], []
    for k in range(len(lo)):
        f, fm, g, m = orc.eval_box(lo[k], hi[k], blk=blk, f32=fp32)
        F.append(f); Fm.append(fm); G.append(g); M.append(m)
    return np.array(F), np.array(Fm), np.array(G), np.array(M)


POLY = [("chain", dict(n=33, seed=3), 10), ("chain", dict(n=12, seed=4), 5),
        ("chain", dict(n=2, seed=5), 2), ("chain", dict(n=100, seed=0), 10),
        ("prod_poly", dict(n=12, seed=1), 5), ("prod_poly", dict(n=37, seed=2), 10)]


@pytest.mark.parametrize("fp32", [False, True])
@pytest.mark.parametrize("fam,kw,B", POLY)
def test_polynomial_bit_exact(fam, kw, B, fp32):
    p = S.make(fam, **kw)
    solver = gb.Solver(p, block=B)
    orc = O.Oracle(p, block=B)
    nb = (p.n + B - 1) // B
    count = 160 if p.n <= 40 else 40
    lo, hi = S.random_boxes(p, count, seed=11, around_s=0.5)
    for blk in sorted({0, nb // 2, nb - 1}):
        gF, gFm, gG, gM = _gpu_eval(solver, lo, hi, blk, fp32)
        oF, oFm, oG, oM = _oracle_eval(orc, lo, hi, blk, fp32)
        w = min(B, p.n - blk * B)
        assert np.array_equal(gF, oF), (blk, np.argwhere(gF != oF)[:5])
        assert np.array_equal(gFm, oFm)
        assert np.array_equal(gG[:, :w], oG[:, :w]), (blk, np.argwhere(gG[:, :w] != oG[:, :w])[:5])
        assert np.array_equal(gM, oM)
    solver.close()


def test_signed_product_bit_exact():
    # products whose factors straddle zero and change sign (every case of
    # the interval product), two products and a sum, offsets 0 and 1
    n = 11
    rng = np.random.default_rng(8)
    g = S.Dag()
    tc = g.table(rng.uniform(-1.0, 1.0, n))
    t1 = g.sub(g.ivar(0), g.icoef(tc))
    t2 = g.add(g.const(0.5), g.mul(g.ivar(0), g.ivar(1)))
    f = g.add(g.sub(g.iprod(t1, 0, n, 1), g.scale(g.iprod(t2, 0, n - 1, 2), 0.75)),
              g.isum(g.sqr(g.ivar(0)), 0, n, 1))
    p = S.Problem("signed_prod", n, g.nodes(), f, g.tables, np.full(n, -2.0), np.full(n, 2.0),
                  1e-6, 4, np.zeros(n), 0)
    solver = gb.Solver(p, block=4)
    orc = O.Oracle(p, block=4)
    lo, hi = S.random_boxes(p, 200, seed=6)
    for fp32 in (False, True):
        for blk in range(3):
            gF, gFm, gG, gM = _gpu_eval(solver, lo, hi, blk, fp32)
            oF, oFm, oG, oM = _oracle_eval(orc, lo, hi, blk, fp32)
            w = min(4, n - blk * 4)
            assert np.array_equal(gF, oF) and np.array_equal(gFm, oFm)
            assert np.array_equal(gG[:, :w], oG[:, :w]) and np.array_equal(gM, oM)
    solver.close()


def _step_poly(n, seed):
    """sum_i (x_i - c_i)^2 + 0.5 H(x_i - c_i)(x_i - c_i) - 0.25 prod_i H(x_i - c_i + 0.3) H(c_i + 0.3 - x_i):
    unit steps in a sum template, a product of steps and a kink at c."""
    rng = np.random.default_rng(seed)
    g = S.Dag()
    tc = g.table(rng.uniform(-1.0, 1.0, n))
    d = g.sub(g.ivar(0), g.icoef(tc))
    s1 = g.isum(g.add(g.sqr(d), g.scale(g.mul(g.step(d), d), 0.5)), 0, n, 1)
    ind = g.iprod(g.mul(g.step(g.add(d, g.const(0.3))), g.step(g.sub(g.const(0.3), d))), 0, n, 1)
    f = g.sub(s1, g.scale(ind, 0.25))
    return S.Problem("step_poly", n, g.nodes(), f, g.tables, np.full(n, -2.0), np.full(n, 2.0),
                     1e-6, 4, np.zeros(n), 0)


def test_step_bit_exact():
    # the unit step forward (exact, or [0, 1] across the jump) and its
    # reverse step (0, or unbounded across the jump) bit for bit
    p = _step_poly(10, 3)
    solver = gb.Solver(p, block=4)
    orc = O.Oracle(p, block=4)
    lo, hi = S.random_boxes(p, 300, seed=4)
    for fp32 in (False, True):
        for blk in range(3):
            gF, gFm, gG, gM = _gpu_eval(solver, lo, hi, blk, fp32)
            oF, oFm, oG, oM = _oracle_eval(orc, lo, hi, blk, fp32)
            w = min(4, 10 - blk * 4)
            assert np.array_equal(gF, oF) and np.array_equal(gFm, oFm)
            assert np.array_equal(gG[:, :w], oG[:, :w]) and np.array_equal(gM, oM)
            assert np.isinf(oG[:, :w]).any()          # some boxes hold a jump
    solver.close()


def test_product_special_cases_bit_exact():
    # an empty product (1), a one-term product and products of points
    g = S.Dag()
    x = g.ivar(0)
    empty = g.iprod(g.add(x, g.const(1.0)), 2, 2, 1)
    one = g.iprod(g.sqr(x), 1, 2, 1)
    allp = g.iprod(g.scale(x, 2.0), 0, 5, 1)
    f = g.add(g.add(g.scale(empty, 3.0), one), allp)
    p = S.Problem("prod_special", 5, g.nodes(), f, g.tables, np.full(5, -2.0), np.full(5, 2.0), 1e-6, 3,
                  np.zeros(5), 0)
    solver = gb.Solver(p, block=3)
    orc = O.Oracle(p, block=3)
    lo, hi = S.random_boxes(p, 100, seed=9)
    lo[:10] = hi[:10]                      # point boxes
    for fp32 in (False, True):
        for blk in range(2):
            gF, gFm, gG, gM = _gpu_eval(solver, lo, hi, blk, fp32)
            oF, oFm, oG, oM = _oracle_eval(orc, lo, hi, blk, fp32)
            w = min(3, 5 - blk * 3)
            assert np.array_equal(gF, oF) and np.array_equal(gFm, oFm)
            assert np.array_equal(gG[:, :w], oG[:, :w]) and np.array_equal(gM, oM)
    solver.close()


def test_custom_dag_bit_exact():
    g = S.Dag()
    y = g.sub(g.ivar(0), g.ivar(1))
    t = g.mul(g.icoef(g.table(np.linspace(0.5, 3.0, 9))), g.sqr(y))
    s_even = g.isum(t, 0, 8, 2)
    f = g.add(g.sub(s_even, g.scale(g.var(3), -1.5)), g.neg(g.mul(g.var(0), g.var(8))))
    p = S.Problem("custom", 9, g.nodes(), f, g.tables, np.full(9, -2.0), np.full(9, 3.0),
                  1e-6, 3, np.zeros(9), 0)
    solver = gb.Solver(p, block=3)
    orc = O.Oracle(p, block=3)
    lo, hi = S.random_boxes(p, 200, seed=5)
    for fp32 in (False, True):
        for blk in range(3):
            gF, gFm, gG, gM = _gpu_eval(solver, lo, hi, blk, fp32)
            oF, oFm, oG, oM = _oracle_eval(orc, lo, hi, blk, fp32)
            assert np.array_equal(gF, oF) and np.array_equal(gFm, oFm)
            assert np.array_equal(gG, oG) and np.array_equal(gM, oM)


TRANS = [("sep_cos", dict(n=2, seed=1), 2), ("sep_cos", dict(n=25, seed=2), 10),
         ("ackley", dict(n=10, seed=3), 5), ("ackley", dict(n=1000, seed=0), 10),
         ("mixed", dict(n=21, seed=4), 10), ("paper_rastrigin", dict(n=7), 7),
         ("paper_breiman", dict(n=5), 5), ("paper_griewank", dict(n=13), 5),
         ("paper_styblinski", dict(n=6), 3), ("paper_zabinsky", dict(n=9), 9),
         ("paper_discontinuous", dict(n=6), 3)]


def _oracle_dev(orc, lo, hi, blk, fp32):
    out = [[] for _ in range(6)]
    for k in range(len(lo)):
        for a, v in zip(out, orc.eval_box_dev(lo[k], hi[k], blk=blk, f32=fp32)):
            a.append(v)
    return [np.array(a) for a in out]


@pytest.mark.parametrize("fp32", [False, True])
@pytest.mark.parametrize("fam,kw,B", TRANS)
def test_transcendental_within_deviation_bound(fam, kw, B, fp32):
    """Both sides run the same directed operations in the same order; only
    the library values of exp, sin and cos differ (each within its
    documented error, widened by its own count of ulps).  The oracle
    propagates that difference through the rest of the evaluation and the
    reverse sweep (its deviation bound): every endpoint of F, of the
    midpoint sample and of every finite partial must lie within it, and a
    first-order verdict may differ only where a tested partial lies within
    its bound of 0."""
    p = S.make(fam, **kw)
    solver = gb.Solver(p, block=B)
    orc = O.Oracle(p, block=B)
    nb = (p.n + B - 1) // B
    count = 120 if p.n <= 100 else 12
    lo, hi = S.random_boxes(p, count, seed=13, min_width=1e-7, around_s=0.5)
    for blk in sorted({0, nb - 1}):
        gF, gFm, gG, gM = _gpu_eval(solver, lo, hi, blk, fp32)
        oF, dF, oFm, dFm, oG, dG = _oracle_dev(orc, lo, hi, blk, fp32)
        assert np.any(dF > 0)                      # the family has transcendental terms
        assert np.all(np.abs(gF - oF) <= dF[:, None]), np.max(np.abs(gF - oF) - dF[:, None])
        assert np.all(np.abs(gFm - oFm) <= dFm[:, None]), np.max(np.abs(gFm - oFm) - dFm[:, None])
        w = min(B, p.n - blk * B)
        fin = np.isfinite(oG[:, :w])
        assert np.array_equal(fin, np.isfinite(gG[:, :w]))
        gap = np.where(fin, np.abs(gG[:, :w] - oG[:, :w]), 0.0)
        tol = dG[:, :w, None]
        assert np.all(gap <= tol), np.max(gap - tol)
        _, _, _, oM = _oracle_eval(orc, lo, hi, blk, fp32)
        for k in np.nonzero(gM != oM)[0]:
            near0 = np.minimum(np.abs(oG[k, :w, 0]), np.abs(oG[k, :w, 1])) <= dG[k, :w]
            assert near0.any(), (k, oG[k, :w], gG[k, :w])
    solver.close()


def test_point_boxes_enclose_planted_zero():
    for fam, kw in (("sep_cos", dict(n=3)), ("chain", dict(n=7)), ("ackley", dict(n=5)),
                    ("mixed", dict(n=6))):
        p = S.make(fam, **kw)
        solver = gb.Solver(p)
        lo = p.s[None, :].copy()
        F, Fm, _, _ = _gpu_eval(solver, lo, lo.copy(), -1, False)
        assert F[0, 0] <= 0.0 <= F[0, 1] and Fm[0, 0] <= 0.0 <= Fm[0, 1]
        solver.close()
