"""Block-record box storage (pool_mode 2) on the GPU.

A box stored as a row of per-block record ids, with records shared between a
box and its children, holds exactly the coordinates and cached group sums of
the dense row it replaces, so every search must run identically in both
modes: the same trace, enclosure and boxes bit for bit, with the FP32
prefilter on and off, through the interpreter and the term tables, with
per-generation state reads and with graph replays.  Small pools force the
record collector to run; a record-mode run is also checked directly against
the oracle, and the n = 10,000 mixed workload (records chosen automatically)
against a dense run over its first generations.
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


def _solve(p, device_only=False, **opts):
    s = gb.Solver(p, **opts)
    r = s.solve(device_only=device_only, raise_on_error=False)
    s.close()
    return r


def _same(a, b):
    assert a.status == b.status
    assert a.generations == b.generations
    for k in ("parents", "children", "kept32", "kept", "pool"):
        assert np.array_equal(a.trace[k], b.trace[k]), k
    assert np.array_equal(a.trace["gub"], b.trace["gub"])
    assert a.fmin_lo == b.fmin_lo and a.fmin_hi == b.fmin_hi
    assert a.n_boxes == b.n_boxes
    if a.box_lo is not None or b.box_lo is not None:
        assert np.array_equal(a.box_lo, b.box_lo) and np.array_equal(a.box_hi, b.box_hi)
        assert np.array_equal(a.box_flo, b.box_flo)
    assert a.box_evals_fp64 == b.box_evals_fp64 and a.box_evals_fp32 == b.box_evals_fp32


CASES = [
    ("chain", S.chain(n=40, seed=3), dict(block=5, split_m=2, split_d=5, max_children=16 * 32)),
    ("chain_ragged", S.chain(n=23, seed=4), dict(block=5, split_m=2, split_d=3, max_children=64 * 8)),
    ("ackley", S.ackley(n=24, seed=5), dict(block=6, split_m=2, split_d=6, max_children=8 * 64)),
    ("mixed", S.mixed(n=30, seed=6), dict(block=6, split_m=2, split_d=6, max_children=8 * 64)),
    ("sep_cos", S.sep_cos(n=2, seed=7), dict(block=1, split_m=4, split_d=1, max_children=1 << 10)),
]


@pytest.mark.parametrize("name,p,o", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("fp32", [0, 1])
@pytest.mark.parametrize("eval_mode", [1, 3, 4])
def test_records_identical_to_dense(name, p, o, fp32, eval_mode):
    o = dict(o, fp32_prefilter=fp32, eval_mode=eval_mode, max_generations=3000)
    d = _solve(p, pool_mode=1, **o)
    r = _solve(p, pool_mode=2, **o)
    assert d.pool_mode == 1 and r.pool_mode == 2
    _same(d, r)


@pytest.mark.parametrize("G", [4])
def test_records_identical_under_graph_replays(G):
    p = S.chain(n=40, seed=8)
    o = dict(block=5, split_m=2, split_d=5, max_children=16 * 32, fp32_prefilter=1, max_generations=3000)
    d = _solve(p, pool_mode=1, **o)
    r = _solve(p, pool_mode=2, gens_per_sync=G, **o)
    _same(d, r)


def test_collector_runs_and_keeps_results_identical():
    p = S.chain(n=40, seed=9)
    o = dict(block=5, split_m=2, split_d=5, max_children=16 * 32, max_generations=3000)
    ref = _solve(p, pool_mode=1, **o)
    assert ref.status == 0
    created = 2 * int(ref.trace["kept"].sum()) + 8      # nrec = 2 records per child, 8 for the root
    # record stores smaller than the records the run creates: the collector
    # must run; a store too small for the live records ends the run with
    # GB_E_CAPACITY (still a rigorous enclosure), any other run is identical
    collected = 0
    for frac in (0.9, 0.75, 0.6, 0.5):
        r = _solve(p, pool_mode=2, max_records=int(frac * created), **o)
        if r.status == gb.GB_E_CAPACITY:
            assert r.fmin_lo <= 0.0 <= r.fmin_hi
            continue
        _same(ref, r)
        assert r.record_gcs > 0
        collected += 1
    assert collected > 0


def test_records_capacity_overflow_matches_dense():
    p = S.chain(n=40, seed=10)
    o = dict(block=5, split_m=2, split_d=5, max_children=16 * 32, max_generations=3000)
    d = _solve(p, pool_mode=1, max_boxes=600, **o)
    r = _solve(p, pool_mode=2, max_boxes=600, **o)
    assert d.status == gb.GB_E_CAPACITY
    _same(d, r)


def test_records_run_equals_oracle():
    p = S.chain(n=20, seed=11)
    B, m, dd, K = 5, 2, 5, 8
    r = _solve(p, pool_mode=2, block=B, split_m=m, split_d=dd, max_children=K * m ** dd)
    o = O.Oracle(p, block=B).solve(tol_f=p.tol_f, tol_x=0.0, split_m=m, split_d=dd, fp32=False,
                                   max_parents=K, max_gen=10 ** 9, cap=1 << 40)
    assert r.pool_mode == 2
    assert r.status == o.status and r.generations == o.generations
    for k in ("parents", "children", "kept", "pool"):
        assert np.array_equal(r.trace[k], o.trace[k]), k
    assert np.array_equal(r.trace["gub"], o.trace["gub"])
    assert r.fmin_lo == o.glb and r.fmin_hi == o.gub
    assert np.array_equal(r.box_lo, o.box_lo) and np.array_equal(r.box_hi, o.box_hi)


def test_tol_x_final_boxes_identical():
    # boxes narrower than tol_x in every coordinate become final: the record
    # path tracks this with per-record width flags
    p = S.chain(n=12, seed=12)
    o = dict(block=4, split_m=2, split_d=4, max_children=16 * 16, tol_x=1e-3, tol_f=1e-12,
             max_generations=2000)
    d = _solve(p, pool_mode=1, **o)
    r = _solve(p, pool_mode=2, **o)
    _same(d, r)


def test_full_size_mixed_records_auto_equals_dense_prefix():
    p = S.mixed(n=10000, seed=0)
    o = dict(block=100, split_m=2, split_d=6, max_children=4 * 64, fp32_prefilter=1, max_generations=12,
             max_boxes=4096)
    r = _solve(p, device_only=True, **o)
    assert r.pool_mode == 2 and r.status == gb.GB_E_LIMIT
    d = _solve(p, device_only=True, pool_mode=1, **o)
    assert d.pool_mode == 1
    _same(d, r)
