"""Seeded synthetic inputs: the objective-DAG format and the planted-minimum families.

This package is the one module both the CUDA library's tests and the CPU
oracle's tests draw inputs from.  It holds no interval arithmetic and no step
of the minimisation method.
"""
from .dag import Dag, NODE_DTYPE, OP_NAMES  # noqa: F401
from . import dag  # noqa: F401
from .families import (Problem, make, sep_cos, chain, ackley, mixed, prod_poly,  # noqa: F401
                       paper_rastrigin, paper_breiman, paper_ackley, paper_belegundu, paper_fu, paper_levy,
                       paper_salomon, paper_rosenbrock, paper_griewank, paper_styblinski, paper_zabinsky,
                       paper_discontinuous,
                       random_boxes, serving_stream, FAMILIES)
