"""Pins of the oracle's interval arithmetic (section 2.1, Eqs. 3-6).

The oracle's endpoint results are compared with mpmath's interval type, whose
endpoints are rounded outward optimally at the working precision (53 bits for
FP64, 24 for FP32): the paper's "optimal outward rounding".  For +, -, x,
square, sqrt and scaling the results must be bit-identical; division follows
Eq. 6 (multiplication by the outward reciprocal).  Transcendentals must
enclose a tight multiprecision range and stay within a few ulps of it.
"""
import math
import zlib

import numpy as np
import pytest

mpmath = pytest.importorskip("mpmath")
from mpmath import iv, mp  # noqa: E402

import oracle as O  # noqa: E402


def _rand_intervals(rng, count, f32=False):
    """Sign-mixed, zero-straddling and one-sided intervals over many scales."""
    mag = 10.0 ** rng.uniform(-6, 6, (count, 2))
    sign = rng.choice([-1.0, 1.0], (count, 2))
    v = mag * sign
    kind = rng.integers(0, 4, count)
    v[kind == 1, 0] = 0.0                         # touches zero
    v[kind == 2, 1] = v[kind == 2, 0] * (1 + 1e-12)   # very narrow
    if f32:
        v = v.astype(np.float32).astype(np.float64)
    lo = np.minimum(v[:, 0], v[:, 1])
    hi = np.maximum(v[:, 0], v[:, 1])
    return lo, hi


def _mp(lo, hi):
    return iv.mpf([float(lo), float(hi)])


def _ends(x):
    return float(x.a), float(x.b)


@pytest.mark.parametrize("f32", [False, True])
@pytest.mark.parametrize("op", ["ADD", "SUB", "MUL", "SQR", "NEG", "SQRT", "SCALE"])
def test_exact_ops_match_mpmath(op, f32):
    rng = np.random.default_rng(zlib.crc32(f"{op}{f32}".encode()))
    iv.prec = 24 if f32 else 53
    lo1, hi1 = _rand_intervals(rng, 3000, f32)
    lo2, hi2 = _rand_intervals(rng, 3000, f32)
    scales = rng.uniform(-50, 50, 3000)
    if f32:
        scales = scales.astype(np.float32).astype(np.float64)
    for k in range(3000):
        x = (lo1[k], hi1[k])
        y = (lo2[k], hi2[k])
        if op == "SQRT":
            x = (abs(lo1[k]), abs(lo1[k]) + abs(hi1[k]))
            if f32:
                x = tuple(float(np.float32(v)) for v in x)
        got = O.iv_op(op, x, y, c=scales[k], f32=f32)
        X, Y = _mp(*x), _mp(*y)
        ref = {"ADD": lambda: X + Y, "SUB": lambda: X - Y, "MUL": lambda: X * Y,
               "SQR": lambda: X ** 2, "NEG": lambda: -X, "SQRT": lambda: iv.sqrt(X),
               "SCALE": lambda: X * iv.mpf(float(scales[k]))}[op]()
        assert got == _ends(ref), (op, f32, x, y, got, _ends(ref))


@pytest.mark.parametrize("f32", [False, True])
def test_div_is_eq6_product_with_reciprocal(f32):
    rng = np.random.default_rng(7)
    iv.prec = 24 if f32 else 53
    lo1, hi1 = _rand_intervals(rng, 2000, f32)
    lo2, hi2 = _rand_intervals(rng, 2000, f32)
    for k in range(2000):
        x = (lo1[k], hi1[k])
        y = (lo2[k], hi2[k])
        got = O.iv_op("DIV", x, y, f32=f32)
        X, Y = _mp(*x), _mp(*y)
        if y[0] <= 0.0 <= y[1]:
            assert got == (-math.inf, math.inf) or (x == (0.0, 0.0) and got == (0.0, 0.0))
            continue
        rec = iv.mpf(1) / Y
        assert got == _ends(X * rec)
        # and the quotient set is enclosed
        with mp.workprec(200):
            q = [mpmath.mpf(a) / mpmath.mpf(b) for a in x for b in y]
        assert got[0] <= min(q) and got[1] >= max(q)


@pytest.mark.parametrize("f32", [False, True])
def test_unit_step_is_the_image_of_the_interval(f32):
    # H(y) = 1 for y >= 0 and 0 for y < 0; the interval image of [a, b] is
    # {H(y) : a <= y <= b}, enclosed by [0, 1] exactly when it holds both values
    cases = {(0.0, 0.0): (1.0, 1.0), (-0.0, 2.0): (1.0, 1.0), (1e-300, 1.0): (1.0, 1.0),
             (-1e-300, -1e-300): (0.0, 0.0), (-3.0, -1.0): (0.0, 0.0), (-1.0, 0.0): (0.0, 1.0),
             (-1e-300, 1e-300): (0.0, 1.0), (-math.inf, math.inf): (0.0, 1.0)}
    for x, want in cases.items():
        assert O.iv_op("STEP", x, f32=f32) == want, x
    rng = np.random.default_rng(12)
    lo, hi = _rand_intervals(rng, 2000, f32)
    for a, b in zip(lo, hi):
        img = {1.0 if y >= 0 else 0.0 for y in (a, b, 0.0) if a <= y <= b}
        assert O.iv_op("STEP", (a, b), f32=f32) == (min(img), max(img))


def test_closed_interval_zero_times_infinity():
    assert O.iv_op("MUL", (0.0, 0.0), (-math.inf, math.inf)) == (0.0, 0.0)
    assert O.iv_op("MUL", (0.0, 2.0), (1.0, math.inf)) == (0.0, math.inf)
    assert O.iv_op("MUL", (-1.0, 0.0), (1.0, math.inf)) == (-math.inf, 0.0)
    assert O.iv_op("DIV", (1.0, 2.0), (-1.0, 1.0)) == (-math.inf, math.inf)


@pytest.mark.parametrize("f32", [False, True])
def test_pi_and_e_are_adjacent_enclosures(f32):
    with mp.workdps(50):
        for name, val in (("PI", +mp.pi), ("EULER", +mp.e)):
            lo, hi = O.iv_op(name, (0.0, 0.0), f32=f32)
            assert mpmath.mpf(lo) < val < mpmath.mpf(hi)
            nxt = (float(np.nextafter(np.float32(lo), np.float32(np.inf))) if f32
                   else math.nextafter(lo, math.inf))
            assert hi == nxt


def _ulp(x, f32):
    x = abs(x)
    if f32:
        return float(np.spacing(np.float32(x)))
    return math.ulp(x)


def _trig_range(fn, a, b):
    """Tight range of sin/cos over [a, b] at 120 bits (critical points found
    from the multiprecision value of pi)."""
    with mp.workprec(120):
        A, Bv = mpmath.mpf(a), mpmath.mpf(b)
        vals = [fn(A), fn(Bv)]
        shift = mpmath.mpf(0) if fn is mpmath.cos else mp.pi / 2
        k0 = int(mpmath.ceil((A - shift) / mp.pi))
        k1 = int(mpmath.floor((Bv - shift) / mp.pi))
        for k in range(k0, min(k1, k0 + 4) + 1):
            vals.append(fn(shift + k * mp.pi))
        return min(vals), max(vals)


@pytest.mark.parametrize("f32", [False, True])
@pytest.mark.parametrize("name", ["EXP", "SIN", "COS"])
def test_transcendentals_enclose_and_are_tight(name, f32):
    rng = np.random.default_rng(11 + len(name) + int(f32))
    K = 6  # allowed excess width, in ulps of the endpoint, per side
    for _ in range(2500):
        c = rng.uniform(-40, 40) if name != "EXP" else rng.uniform(-30, 30)
        w = 10.0 ** rng.uniform(-12, 1)
        a, b = c - w, c + w * rng.uniform(0, 1)
        if rng.uniform() < 0.2:       # land exactly around a critical point
            kpi = round(c / math.pi) * math.pi + (0 if name != "SIN" else math.pi / 2)
            a, b = kpi - w, kpi + w
        if f32:
            a = float(np.float32(a))
            b = float(np.float32(b))
            if b < a:
                a, b = b, a
        got = O.iv_op(name, (a, b), f32=f32)
        if name == "EXP":
            with mp.workprec(120):
                lo, hi = mpmath.exp(mpmath.mpf(a)), mpmath.exp(mpmath.mpf(b))
        else:
            lo, hi = _trig_range(mpmath.sin if name == "SIN" else mpmath.cos, a, b)
        assert mpmath.mpf(got[0]) <= lo and mpmath.mpf(got[1]) >= hi, (name, a, b, got, lo, hi)
        assert got[0] >= float(lo) - K * _ulp(float(lo), f32) - (1e-300 if not f32 else 1e-38)
        assert got[1] <= float(hi) + K * _ulp(float(hi), f32) + (1e-300 if not f32 else 1e-38)


def test_trig_wide_argument_is_full_range():
    assert O.iv_op("COS", (0.0, 7.0)) == (-1.0, 1.0)
    assert O.iv_op("SIN", (-4.0, 4.0)) == (-1.0, 1.0)
    lo, hi = O.iv_op("COS", (3.0, 3.3))      # contains pi: minimum -1 reached
    assert lo == -1.0 and hi < -0.98
    lo, hi = O.iv_op("SIN", (1.5, 1.6))      # contains pi/2: maximum 1 reached
    assert hi == 1.0 and lo > 0.99


# ---------------------------------------------------------------------------
# A million operand pairs against exact arithmetic by error-free
# transformations (independent of mpmath and of the oracle): for a + b,
# Knuth's TwoSum gives s = RN(a + b) and the exact error e = a + b - s; for
# a * b, Dekker's splitting gives p = RN(a * b) and e = a * b - p (exact while
# nothing overflows or underflows).  The value rounded down is s when e >= 0,
# else the double below s; rounded up, s when e <= 0, else the double above.
_SPLIT = 134217729.0   # 2^27 + 1


def _two_sum(a, b):
    s = a + b
    bp = s - a
    ap = s - bp
    return s, (a - ap) + (b - bp)


def _split(a):
    c = _SPLIT * a
    hi = c - (c - a)
    return hi, a - hi


def _two_prod(a, b):
    p = a * b
    ah, al = _split(a)
    bh, bl = _split(b)
    return p, ((ah * bh - p) + ah * bl + al * bh) + al * bl


def _rd(v, e):
    return np.where(e < 0, np.nextafter(v, -np.inf), v)


def _ru(v, e):
    return np.where(e > 0, np.nextafter(v, np.inf), v)


def _million(rng):
    count = 1_000_000
    mag = 2.0 ** rng.uniform(-20, 20, (count, 2))
    v = mag * rng.choice([-1.0, 1.0], (count, 2))
    kind = rng.integers(0, 4, count)
    v[kind == 1, 0] = 0.0
    v[kind == 2, 1] = v[kind == 2, 0] * (1 + 2.0 ** -40)
    return np.minimum(v[:, 0], v[:, 1]), np.maximum(v[:, 0], v[:, 1])


@pytest.mark.parametrize("op", ["ADD", "SUB", "MUL", "SQR", "NEG", "SCALE"])
def test_a_million_operations_exact_by_error_free_transformations(op):
    rng = np.random.default_rng(zlib.crc32(op.encode()) + 1)
    a, b = _million(rng)
    c, d = _million(rng)
    k = rng.uniform(-50, 50, len(a))
    got = O.iv_op_batch(op, a, b, c, d, k)
    if op in ("ADD", "SUB"):
        y_lo, y_hi = (c, d) if op == "ADD" else (-d, -c)
        s1, e1 = _two_sum(a, y_lo)
        s2, e2 = _two_sum(b, y_hi)
        want = np.stack([_rd(s1, e1), _ru(s2, e2)], axis=1)
    elif op == "NEG":
        want = np.stack([-b, -a], axis=1)
    elif op in ("MUL", "SCALE"):
        ys = [c, d] if op == "MUL" else [k, k]
        los, his = [], []
        for x in (a, b):
            for y in ys:
                p, e = _two_prod(x, y)
                los.append(_rd(p, e))
                his.append(_ru(p, e))
        want = np.stack([np.min(los, axis=0), np.max(his, axis=0)], axis=1)
    else:   # SQR: [0, max] across zero, else the ordered squares
        pa, ea = _two_prod(a, a)
        pb, eb = _two_prod(b, b)
        lo = np.where(a >= 0, _rd(pa, ea), np.where(b <= 0, _rd(pb, eb), 0.0))
        hi = np.where(a >= 0, _ru(pb, eb), np.where(b <= 0, _ru(pa, ea), np.maximum(_ru(pa, ea), _ru(pb, eb))))
        want = np.stack([lo, hi], axis=1)
    bad = np.nonzero(got != want)
    assert bad[0].size == 0, (op, bad[0][:3], got[bad[0][:3]], want[bad[0][:3]])
