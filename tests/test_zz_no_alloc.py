"""gb_eval_boxes_noalloc: the per-box evaluation for callers that cannot
allocate device memory while they run (a serving process that gave all free
device memory to its own pool, a thread that must not wait on the device
allocator).  It keeps its FP32 scratch in a fixed array inside the library
instead of allocating per call; its results must equal gb_eval_boxes's, on
consecutive calls that reuse the same array, and it must refuse calls larger
than the array.  Collected last so that a failure here leaves every other
test already run.
"""
import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2507_01770_gb300 as gb  # noqa: E402


def _both(solver, lo, hi, blk, fp32):
    dlo = torch.from_numpy(lo).cuda()
    dhi = torch.from_numpy(hi).cuda()
    ref = solver.eval_boxes(dlo, dhi, blk, fp32)
    new = gb.gb_eval_boxes(solver.h, dlo, dhi, blk, fp32, noalloc=True)
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in ref], [t.cpu().numpy() for t in new]


def test_noalloc_matches_allocating_entry_point_on_consecutive_calls():
    p = S.chain(n=33, seed=9)
    solver = gb.Solver(p, block=10)
    # first call: many boxes; second call: fewer boxes, so the array still
    # holds the first call's values beyond what the second one writes
    for count, seed, blk in ((300, 1, 1), (40, 2, 3)):
        lo, hi = S.random_boxes(p, count, seed=seed, around_s=0.5)
        for fp32 in (True, False):
            ref, new = _both(solver, lo, hi, blk, fp32)
            for a, b in zip(ref, new):
                assert np.array_equal(a, b, equal_nan=True)
    solver.close()


def test_noalloc_transcendental_family_matches():
    p = S.ackley(n=20, seed=4)
    solver = gb.Solver(p, block=10)
    for seed in (5, 6):
        lo, hi = S.random_boxes(p, 64, seed=seed, around_s=0.5)
        ref, new = _both(solver, lo, hi, 0, True)
        for a, b in zip(ref, new):
            assert np.array_equal(a, b, equal_nan=True)
    solver.close()


def test_noalloc_rejects_calls_beyond_its_array():
    p = S.chain(n=100, seed=1)
    solver = gb.Solver(p, block=10)
    nbox = (1 << 20) // 100 + 1          # nbox * n just above 2^20 coordinates
    lo = torch.zeros((nbox, 100), dtype=torch.float64, device="cuda")
    hi = torch.ones((nbox, 100), dtype=torch.float64, device="cuda")
    with pytest.raises(gb.GbError) as e:
        gb.gb_eval_boxes(solver.h, lo, hi, 0, True, noalloc=True)
    assert e.value.status == gb.GB_E_INVALID and "2^20" in str(e.value)
    solver.close()
