"""Multiprecision references for pinning the oracle (tests only, CPU only).

* ``point_value``  evaluates the objective's node array at a point with
  mpmath at high precision (the real-number value f(x)).
* ``point_grad``   its partial derivative by mpmath's high-precision
  numerical differentiation.
* ``iv53_value``   evaluates the node array with mpmath's interval type at a
  53-bit working precision, whose endpoint operations are optimally rounded
  outward, in the fixed term grouping and pairwise reduction order that the
  method's reading prescribes.  It supports the polynomial operators only.
"""
from __future__ import annotations

import mpmath
from mpmath import iv, mp

from synthetic import dag as D

_BIN = {D.OP_ADD, D.OP_SUB, D.OP_MUL, D.OP_DIV}


def _isum_indices(node):
    return list(range(int(node["b"]), int(node["c"]), int(node["d"])))


def point_value(p, x, dps: int = 60):
    """f(x) with mpmath at ``dps`` digits; x is a sequence of floats."""
    with mp.workdps(dps):
        return _point_value_mp(p, [mpmath.mpf(float(v)) for v in x])


def point_grad(p, x, j: int, dps: int = 60):
    """d f / d x_j at x (high-precision numerical differentiation)."""
    x = [float(v) for v in x]
    with mp.workdps(dps):
        def fj(t):
            y = list(x)
            xs = [mpmath.mpf(v) for v in y]
            xs[j] = t
            return _point_value_mp(p, xs)
        return mpmath.diff(fj, mpmath.mpf(x[j]))


def _point_value_mp(p, xs):
    nodes = p.nodes
    memo = {}

    def ev(v, i):
        key = (v, i)
        if key in memo:
            return memo[key]
        q = nodes[v]
        op = int(q["op"])
        a, b = int(q["a"]), int(q["b"])
        if op == D.OP_CONST:
            r = mpmath.mpf(float(q["v"]))
        elif op == D.OP_PI:
            r = +mp.pi
        elif op == D.OP_EULER:
            r = +mp.e
        elif op == D.OP_VAR:
            r = xs[a]
        elif op == D.OP_IDX_VAR:
            r = xs[i + b]
        elif op == D.OP_IDX_COEF:
            r = mpmath.mpf(float(p.tables[a][i + b]))
        elif op == D.OP_ADD:
            r = ev(a, i) + ev(b, i)
        elif op == D.OP_SUB:
            r = ev(a, i) - ev(b, i)
        elif op == D.OP_MUL:
            r = ev(a, i) * ev(b, i)
        elif op == D.OP_DIV:
            r = ev(a, i) / ev(b, i)
        elif op == D.OP_NEG:
            r = -ev(a, i)
        elif op == D.OP_SQR:
            r = ev(a, i) ** 2
        elif op == D.OP_SQRT:
            r = mpmath.sqrt(ev(a, i))
        elif op == D.OP_EXP:
            r = mpmath.exp(ev(a, i))
        elif op == D.OP_SIN:
            r = mpmath.sin(ev(a, i))
        elif op == D.OP_COS:
            r = mpmath.cos(ev(a, i))
        elif op == D.OP_SCALE:
            r = ev(a, i) * mpmath.mpf(float(q["v"]))
        elif op == D.OP_STEP:
            r = mpmath.mpf(1) if ev(a, i) >= 0 else mpmath.mpf(0)
        elif op == D.OP_ISUM:
            r = mpmath.fsum(ev(a, k) for k in _isum_indices(q))
        elif op == D.OP_IPROD:
            r = mpmath.fprod(ev(a, k) for k in _isum_indices(q))
        else:
            raise ValueError(op)
        memo[key] = r
        return r

    return ev(int(p.root), -1)


# -------------------------------------------------------------------------
def _tree(vals, prod: bool = False):
    """Pairwise reduction in index order (level s: a[i] = a[i] op a[i+s])."""
    a = list(vals)
    m = len(a)
    if m == 0:
        return iv.mpf(1 if prod else 0)
    s = 1
    while s < m:
        for i in range(0, m - s, 2 * s):
            a[i] = a[i] * a[i + s] if prod else a[i] + a[i + s]
        s *= 2
    return a[0]


def _template_offsets(p, root):
    nodes = p.nodes
    seen, stack, offs = set(), [root], []
    while stack:
        v = stack.pop()
        if v in seen:
            continue
        seen.add(v)
        q = nodes[v]
        op = int(q["op"])
        if op == D.OP_IDX_VAR:
            offs.append(int(q["b"]))
        if op in _BIN:
            stack += [int(q["a"]), int(q["b"])]
        elif op in (D.OP_NEG, D.OP_SQR, D.OP_SQRT, D.OP_EXP, D.OP_SIN, D.OP_COS, D.OP_SCALE, D.OP_STEP):
            stack.append(int(q["a"]))
    return offs


def iv53_value(p, lo, hi, B: int):
    """Interval F over the box with mpmath iv at 53 bits, grouped tree order."""
    iv.prec = 53
    nodes = p.nodes
    X = [iv.mpf([float(a), float(b)]) for a, b in zip(lo, hi)]

    def ev(v, i, memo):
        if (v, i) in memo:
            return memo[(v, i)]
        q = nodes[v]
        op = int(q["op"])
        a, b = int(q["a"]), int(q["b"])
        if op == D.OP_CONST:
            r = iv.mpf(float(q["v"]))
        elif op == D.OP_VAR:
            r = X[a]
        elif op == D.OP_IDX_VAR:
            r = X[i + b]
        elif op == D.OP_IDX_COEF:
            r = iv.mpf(float(p.tables[a][i + b]))
        elif op == D.OP_ADD:
            r = ev(a, i, memo) + ev(b, i, memo)
        elif op == D.OP_SUB:
            r = ev(a, i, memo) - ev(b, i, memo)
        elif op == D.OP_MUL:
            r = ev(a, i, memo) * ev(b, i, memo)
        elif op == D.OP_NEG:
            r = -ev(a, i, memo)
        elif op == D.OP_SQR:
            r = ev(a, i, memo) ** 2
        elif op == D.OP_SCALE:
            r = ev(a, i, memo) * iv.mpf(float(q["v"]))
        elif op in (D.OP_ISUM, D.OP_IPROD):
            prod = op == D.OP_IPROD
            offs = _template_offsets(p, a)
            idx = _isum_indices(q)
            terms = [ev(a, k, {}) for k in idx]
            if not offs:
                return _tree(terms, prod)
            keys = [((k + min(offs)) // B, (k + max(offs)) // B) for k in idx]
            groups, start = [], 0
            for t in range(1, len(idx) + 1):
                if t == len(idx) or keys[t] != keys[start]:
                    groups.append(_tree(terms[start:t], prod))
                    start = t
            r = _tree(groups, prod)
        else:
            raise ValueError(f"unsupported op {op} in iv53_value")
        memo[(v, i)] = r
        return r

    r = ev(int(p.root), -1, {})
    return float(r.a), float(r.b)
