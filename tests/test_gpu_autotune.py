"""The autotuner of the batching layer on the GPU: it returns one of its
candidate settings (fan-out, parents per generation, child-kernel shape),
and a solve with that setting is a valid solve of the same problem (the
enclosure contains the planted minimum and meets the width)."""
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2507_01770_gb300 as gb  # noqa: E402


@pytest.mark.parametrize("p", [S.chain(n=12, seed=1), S.sep_cos(n=2, seed=2), S.ackley(n=8, seed=3)],
                         ids=["chain12", "sep_cos2", "ackley8"])
def test_autotune_returns_a_valid_candidate(p):
    base = gb.gb_default_options(pool_bytes=1 << 28, fp32_prefilter=1 if p.family == "ackley" else 0)
    best, ms = gb.gb_autotune(p, budget_ms=5000.0, base=base)
    assert ms > 0.0
    B = min(p.n, 10)
    assert best.block == B and best.split_m in (2, 4) and best.split_d in (B, (B + 1) // 2)
    fan = best.split_m ** best.split_d
    assert best.max_children in (fan, 4 * fan) and best.eval_mode in (3, 4)
    assert best.fp32_prefilter == base.fp32_prefilter and best.pool_bytes == base.pool_bytes
    s = gb.Solver(p, **{f: getattr(best, f) for f, _ in gb.gb_options._fields_})
    r = s.solve()
    s.close()
    assert r.status == 0
    assert r.fmin_lo <= 0.0 <= r.fmin_hi and r.fmin_hi - r.fmin_lo <= p.tol_f
