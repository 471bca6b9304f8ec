"""Expression-DAG input format shared by the CUDA library and the CPU oracle.

This module holds the *problem description* only: how an objective f and its
coefficient tables are written down as a flat node array.  It contains none of
the interval arithmetic or branch-and-bound steps of the method (those live,
independently, in the CUDA library and in ``oracle/``).

Node layout (32 bytes, little endian, matches ``gb_node`` in include/gb.h):

    int32 op   operator code (OP_* below)
    int32 a    first operand node | VAR coordinate | IDX_COEF table | ISUM / IPROD template root
    int32 b    second operand node | IDX_VAR / IDX_COEF index offset | ISUM / IPROD first index
    int32 c    ISUM / IPROD end index (exclusive)
    int32 d    ISUM / IPROD index step (> 0)
    int32 pad  zero
    f64   v    CONST value | SCALE factor

Nodes are topologically ordered: every operand index is smaller than the node's
own index.  An ISUM node sums a *template* sub-DAG over an index set
{b, b+d, ...} < c; inside the template IDX_VAR(off) stands for x[i+off] and
IDX_COEF(t, off) for table t at i+off.  An IPROD node is the product of its
template over the index set, laid out like ISUM.  The objective of Eq. 1 is the node
given as ``root``; the simple bounds of Eq. 2 are passed beside it.
"""
from __future__ import annotations

import numpy as np

OP_CONST = 0
OP_PI = 1
OP_EULER = 2
OP_VAR = 3
OP_IDX_VAR = 4
OP_IDX_COEF = 5
OP_ADD = 6
OP_SUB = 7
OP_MUL = 8
OP_DIV = 9
OP_NEG = 10
OP_SQR = 11
OP_SQRT = 12
OP_EXP = 13
OP_SIN = 14
OP_COS = 15
OP_SCALE = 16
OP_ISUM = 17
OP_IPROD = 18
OP_STEP = 19

OP_NAMES = {
    OP_CONST: "CONST", OP_PI: "PI", OP_EULER: "EULER", OP_VAR: "VAR",
    OP_IDX_VAR: "IDX_VAR", OP_IDX_COEF: "IDX_COEF", OP_ADD: "ADD", OP_SUB: "SUB",
    OP_MUL: "MUL", OP_DIV: "DIV", OP_NEG: "NEG", OP_SQR: "SQR", OP_SQRT: "SQRT",
    OP_EXP: "EXP", OP_SIN: "SIN", OP_COS: "COS", OP_SCALE: "SCALE", OP_ISUM: "ISUM",
    OP_IPROD: "IPROD", OP_STEP: "STEP",
}

NODE_DTYPE = np.dtype([
    ("op", "<i4"), ("a", "<i4"), ("b", "<i4"), ("c", "<i4"),
    ("d", "<i4"), ("pad", "<i4"), ("v", "<f8"),
])
assert NODE_DTYPE.itemsize == 32


class Dag:
    """Incremental builder of a node array; methods return node indices."""

    def __init__(self) -> None:
        self._nodes: list[tuple] = []
        self.tables: list[np.ndarray] = []

    # -- leaves -----------------------------------------------------------
    def _push(self, op, a=0, b=0, c=0, d=0, v=0.0) -> int:
        self._nodes.append((op, a, b, c, d, 0, float(v)))
        return len(self._nodes) - 1

    def const(self, v: float) -> int:
        return self._push(OP_CONST, v=v)

    def pi(self) -> int:
        return self._push(OP_PI)

    def euler(self) -> int:
        return self._push(OP_EULER)

    def var(self, j: int) -> int:
        return self._push(OP_VAR, a=j)

    def ivar(self, off: int = 0) -> int:
        return self._push(OP_IDX_VAR, b=off)

    def table(self, values) -> int:
        self.tables.append(np.ascontiguousarray(values, dtype=np.float64))
        return len(self.tables) - 1

    def icoef(self, table: int, off: int = 0) -> int:
        return self._push(OP_IDX_COEF, a=table, b=off)

    # -- operators --------------------------------------------------------
    def add(self, x, y):
        return self._push(OP_ADD, a=x, b=y)

    def sub(self, x, y):
        return self._push(OP_SUB, a=x, b=y)

    def mul(self, x, y):
        return self._push(OP_MUL, a=x, b=y)

    def div(self, x, y):
        return self._push(OP_DIV, a=x, b=y)

    def neg(self, x):
        return self._push(OP_NEG, a=x)

    def sqr(self, x):
        return self._push(OP_SQR, a=x)

    def sqrt(self, x):
        return self._push(OP_SQRT, a=x)

    def exp(self, x):
        return self._push(OP_EXP, a=x)

    def sin(self, x):
        return self._push(OP_SIN, a=x)

    def cos(self, x):
        return self._push(OP_COS, a=x)

    def step(self, x):
        """Unit step: 1 where x >= 0, else 0."""
        return self._push(OP_STEP, a=x)

    def scale(self, x, v: float):
        return self._push(OP_SCALE, a=x, v=v)

    def isum(self, template_root: int, first: int, end: int, step: int = 1):
        return self._push(OP_ISUM, a=template_root, b=first, c=end, d=step)

    def iprod(self, template_root: int, first: int, end: int, step: int = 1):
        return self._push(OP_IPROD, a=template_root, b=first, c=end, d=step)

    # -- output -----------------------------------------------------------
    def nodes(self) -> np.ndarray:
        return np.array(self._nodes, dtype=NODE_DTYPE)

    def __len__(self) -> int:
        return len(self._nodes)
