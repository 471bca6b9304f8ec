"""GPU containment (section 2.1: an outward-rounded interval extension
encloses the range of the function over the box).

* The GPU's interval exp, sin, cos and sqrt, in FP64 and in FP32 directed
  rounding, contain mpmath's tight interval range (200-bit interval
  arithmetic) on random intervals, on intervals whose interior holds an
  extremum (k pi for cos, pi/2 + k pi for sin, on both sides of the
  inclusion decision), on intervals that end at the double nearest such a
  point, and on point intervals.  Each endpoint also lies within the
  oracle's deviation bound of the oracle's endpoint.
* For boxes of the n = 2 cosine family, the n = 1000 exp/sqrt/cos family and
  the n = 10,000 mixed family, f at seeded points of each box (60-digit
  mpmath value) lies in the GPU's F(X), and the partials of the tested block
  at those points (60-digit numerical derivatives) lie in the GPU's interval
  partials, in both precisions.
"""
import math

import numpy as np
import pytest

import oracle as O
import synthetic as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)
mpmath = pytest.importorskip("mpmath")

import paper_2507_01770_gb300 as gb  # noqa: E402
import mp_ref  # noqa: E402


def _unary(op, lo, hi):
    g = S.Dag()
    x = g.var(0)
    f = {"exp": g.exp, "sin": g.sin, "cos": g.cos, "sqrt": g.sqrt}[op](x)
    return S.Problem(op, 1, g.nodes(), f, g.tables, np.array([lo]), np.array([hi]), 1e-6, 1, np.zeros(1), 0)


def _gpu(solver, lo, hi, blk, fp32):
    F, Fm, G, M = solver.eval_boxes(torch.from_numpy(np.ascontiguousarray(lo)).cuda(),
                                    torch.from_numpy(np.ascontiguousarray(hi)).cuda(), blk, fp32)
    torch.cuda.synchronize()
    return F.cpu().numpy(), G.cpu().numpy()


def _intervals(op, rng):
    """Random intervals plus intervals around the extrema of sin / cos."""
    dom = {"exp": (-60.0, 60.0), "sqrt": (0.0, 1e4)}.get(op, (-40.0, 40.0))
    w = np.exp(rng.uniform(np.log(1e-13), np.log(8.0), 300))
    a = rng.uniform(dom[0], dom[1] - 8.0, 300)
    ivs = [(x, x + y) for x, y in zip(a, w)]
    ivs += [(x, x) for x in rng.uniform(dom[0], dom[1], 40)]            # point intervals
    if op in ("sin", "cos"):
        for k in range(-12, 13):
            c = k * math.pi + (math.pi / 2 if op == "sin" else 0.0)
            cd = float(c)
            for e1, e2 in ((1e-12, 1e-12), (1e-7, 3e-7), (0.1, 0.05), (2.0, 1.0)):
                ivs.append((cd - e1, cd + e2))
            ivs += [(cd, cd + 0.1), (cd - 0.1, cd), (np.nextafter(cd, np.inf), cd + 1e-3),
                    (cd - 1e-3, np.nextafter(cd, -np.inf))]
    return [(max(x, dom[0]), min(y, dom[1])) for x, y in ivs]


def _ulp(x, fp32):
    return float(np.spacing(np.float32(abs(x)))) if fp32 else math.ulp(abs(x))


@pytest.mark.parametrize("fp32", [False, True])
@pytest.mark.parametrize("op", ["exp", "sin", "cos", "sqrt"])
def test_elementary_functions_contain_the_tight_range(op, fp32):
    rng = np.random.default_rng({"exp": 1, "sin": 2, "cos": 3, "sqrt": 4}[op])
    ivs = _intervals(op, rng)
    dom = {"exp": (-60.0, 60.0), "sqrt": (0.0, 1e4)}.get(op, (-40.0, 40.0))
    p = _unary(op, *dom)
    solver = gb.Solver(p, block=1)
    orc = O.Oracle(p, block=1)
    lo = np.array([[x] for x, _ in ivs])
    hi = np.array([[y] for _, y in ivs])
    F, _ = _gpu(solver, lo, hi, -1, fp32)
    mpmath.iv.prec = 200
    fn = {"exp": mpmath.iv.exp, "sin": mpmath.iv.sin, "cos": mpmath.iv.cos, "sqrt": mpmath.iv.sqrt}[op]
    for k, (x, y) in enumerate(ivs):
        r = fn(mpmath.iv.mpf([x, y]))
        tight_lo, tight_hi = mpmath.mpf(r.a), mpmath.mpf(r.b)
        slack = mpmath.mpf(2) ** -150 * (1 + abs(tight_lo) + abs(tight_hi))
        assert mpmath.mpf(float(F[k, 0])) <= tight_lo + slack, (op, fp32, x, y, F[k], r)
        assert mpmath.mpf(float(F[k, 1])) >= tight_hi - slack, (op, fp32, x, y, F[k], r)
        oF, dF, _, _, _, _ = orc.eval_box_dev(lo[k], hi[k], f32=fp32)
        assert abs(F[k, 0] - oF[0]) <= dF and abs(F[k, 1] - oF[1]) <= dF, (op, fp32, x, y, F[k], oF, dF)
    solver.close()


def _points(rng, lo, hi, count):
    """Seeded points of the box: its midpoint, a corner and uniform draws."""
    pts = [0.5 * lo + 0.5 * hi, lo.copy()]
    while len(pts) < count:
        pts.append(lo + rng.uniform(0.0, 1.0, lo.shape) * (hi - lo))
    return [np.minimum(np.maximum(q, lo), hi) for q in pts]


@pytest.mark.parametrize("fam,n,nbox,npts,ncoord", [("sep_cos", 2, 24, 8, 2), ("ackley", 1000, 3, 8, 2),
                                                    ("mixed", 10000, 1, 3, 2)])
def test_f_and_partials_at_points_lie_in_the_gpu_enclosures(fam, n, nbox, npts, ncoord):
    p = S.make(fam, n=n, seed=0)
    B = p.block
    solver = gb.Solver(p, block=B)
    rng = np.random.default_rng(n)
    lo, hi = S.random_boxes(p, nbox, seed=n + 1, min_width=1e-8, max_frac=0.05, around_s=0.5)
    nb = (n + B - 1) // B
    blk = int(rng.integers(0, nb))
    w = min(B, n - blk * B)
    coords = sorted(rng.choice(w, size=min(ncoord, w), replace=False).tolist())
    enc = [_gpu(solver, lo, hi, blk, fp32) for fp32 in (False, True)]
    solver.close()
    for k in range(nbox):
        for x in _points(rng, lo[k], hi[k], npts):
            fx = mp_ref.point_value(p, x, dps=60)
            dx = {t: mp_ref.point_grad(p, x, blk * B + t, dps=60) for t in coords}
            for F, G in enc:
                assert mpmath.mpf(float(F[k, 0])) <= fx <= mpmath.mpf(float(F[k, 1])), (k, F[k], fx)
                for t in coords:
                    assert mpmath.mpf(float(G[k, t, 0])) <= dx[t] <= mpmath.mpf(float(G[k, t, 1])), (k, t, G[k, t],
                                                                                                      dx[t])
