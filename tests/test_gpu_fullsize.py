"""Parity at the sizes the benchmark runs (GPU).

* The chain workload in the benchmark's exact configuration -- n = 100, blocks
  of 10, the 10 block coordinates cut into 4 pieces each (4^10 = 1,048,576
  children of one box per generation), the default child kernel (term tables,
  one child per thread, 20-bit child indices) -- for two generations: every
  generation, the GUB sequence and the pool left behind bit-identical to the
  oracle's (Eqs. 7-11 partition, section 3.1 loop, section 3.2 cycling).
* A polynomial n = 10,000 chain on the block-record pool with blocks of 100
  and the FP32 prefilter (the fused FP32-then-FP64 warp-per-child kernel):
  three generations bit-identical to the oracle.
* The n = 1000 exp/sqrt/cos family and the n = 10,000 mixed family solved to
  the end in the benchmark's configuration: the enclosure contains the
  planted minimum 0 with width <= 1e-6, the planted minimiser lies in an
  output box, and sampled output boxes re-evaluated by the oracle give the
  lower bound the pool holds, within the oracle's deviation bound.
The oracle runs its per-child passes on every host core (the result does not
depend on the thread count).
"""
import os

import numpy as np
import pytest

import oracle as O
import synthetic as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2507_01770_gb300 as gb  # noqa: E402

THREADS = max(1, os.cpu_count() or 1)


def _covers(lo, hi, x):
    return bool(np.any(np.all((lo <= x) & (x <= hi), axis=1)))


def _assert_identical(g, o):
    assert g.status == o.status
    assert g.generations == o.generations
    for k in ("parents", "children", "kept32", "kept", "pool"):
        assert np.array_equal(g.trace[k], o.trace[k]), (k, g.trace[k], o.trace[k])
    assert np.array_equal(g.trace["gub"], o.trace["gub"])
    assert g.fmin_lo == o.glb and g.fmin_hi == o.gub
    assert g.n_boxes == len(o.box_flo)
    assert np.array_equal(g.box_flo, o.box_flo)
    assert np.array_equal(g.box_lo, o.box_lo) and np.array_equal(g.box_hi, o.box_hi)


def test_chain100_bench_configuration_two_generations_bit_exact():
    p = S.chain(n=100, seed=0)
    s = gb.Solver(p, block=10, split_m=4, split_d=10, max_children=1 << 20, max_generations=2,
                  pool_bytes=16 << 30)
    g = s.solve(raise_on_error=False)
    s.close()
    assert g.status == gb.GB_E_LIMIT and g.generations == 2
    assert list(g.trace["children"]) == [1 << 20, 1 << 20]
    o = O.Oracle(p, block=10).solve(split_m=4, split_d=10, max_parents=1, max_gen=2, threads=THREADS)
    _assert_identical(g, o)
    assert g.n_boxes > 1000           # the pool holds the survivors of both generations
    assert g.box_evals_fp64 == o.evals64 and g.mid_evals == o.mids


def test_chain10k_block_records_fp32_warp_kernel_bit_exact():
    p = S.chain(n=10000, seed=1, block=100)
    s = gb.Solver(p, block=100, split_m=2, split_d=10, max_children=1 << 10, fp32_prefilter=1,
                  max_generations=3)
    g = s.solve(raise_on_error=False)
    s.close()
    assert g.pool_mode == 2           # block records (n >= 128, a child replaces 2 of 100 blocks)
    assert g.status == gb.GB_E_LIMIT and g.generations == 3
    o = O.Oracle(p, block=100).solve(split_m=2, split_d=10, max_parents=1, max_gen=3, fp32=True,
                                     threads=THREADS)
    _assert_identical(g, o)
    assert g.box_evals_fp32 == o.evals32 and g.box_evals_fp64 == o.evals64


@pytest.mark.parametrize("fam,n,B,pool_gb", [("ackley", 1000, 10, 32), ("mixed", 10000, 100, 64)])
def test_full_solve_at_benchmark_configuration(fam, n, B, pool_gb):
    p = S.make(fam, n=n, seed=0)
    s = gb.Solver(p, block=B, split_m=2, split_d=10, max_children=1 << 10, fp32_prefilter=1, gens_per_sync=16,
                  pool_bytes=pool_gb << 30)
    r = s.solve()
    s.close()
    assert r.status == 0
    assert r.fmin_lo <= 0.0 <= r.fmin_hi and r.fmin_hi - r.fmin_lo <= 1e-6
    assert _covers(r.box_lo, r.box_hi, p.s)
    assert r.box_evals_fp32 > r.box_evals_fp64 > 0
    orc = O.Oracle(p, block=B)
    pick = np.unique(np.linspace(0, r.n_boxes - 1, min(r.n_boxes, 12)).astype(int))
    for k in pick:
        F, dF, _, _, _, _ = orc.eval_box_dev(r.box_lo[k], r.box_hi[k])
        assert abs(F[0] - r.box_flo[k]) <= dF, (k, F[0], r.box_flo[k], dF)
        assert F[0] - dF <= r.fmin_hi
