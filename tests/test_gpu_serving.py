"""Serving (continuous batching) on the GPU: a mix of requests of different
families and dimensions submitted together runs concurrently, and every
request's result is the same as when it is solved alone (enclosure, boxes and
per-generation trace bit for bit: each search depends only on its own state),
with and without the fused child evaluation over the requests."""
import time

import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2507_01770_gb300 as gb  # noqa: E402


def _mix():
    reqs = []
    for k in range(4):
        reqs.append((S.sep_cos(n=2, seed=10 + k), dict(block=2, split_m=2, split_d=1, max_children=1 << 12)))
        reqs.append((S.chain(n=12 + 4 * k, seed=20 + k),
                     dict(block=6, split_m=2, split_d=6, max_children=16 * 64)))
        reqs.append((S.ackley(n=6 + 2 * k, seed=30 + k),
                     dict(block=min(10, 6 + 2 * k), split_m=2, split_d=min(10, 6 + 2 * k),
                          max_children=4 << 10, fp32_prefilter=1)))
    return reqs


def _wait(srv, ids, timeout=300.0):
    out, t0 = {}, time.time()
    while len(out) < len(ids):
        for rid in ids:
            if rid in out:
                continue
            r = srv.poll(rid)
            if r is not None:
                out[rid] = r
        assert time.time() - t0 < timeout, "serving did not finish"
        time.sleep(0.002)
    return out


def _fusable_mix():
    # every request on the term-table FP32-then-FP64 kernel: all in one fused launch per step
    reqs = []
    for k in range(6):
        reqs.append((S.chain(n=10 + 5 * k, seed=40 + k),
                     dict(block=5, split_m=2, split_d=5, max_children=4 * 32, fp32_prefilter=1)))
        reqs.append((S.ackley(n=8 + 4 * k, seed=50 + k),
                     dict(block=8, split_m=2, split_d=8, max_children=2 << 8, fp32_prefilter=1)))
        reqs.append((S.sep_cos(n=4 + k, seed=60 + k),
                     dict(block=4, split_m=4, split_d=2, max_children=4 * 16, fp32_prefilter=1)))
    return reqs


@pytest.mark.parametrize("fused", [True, False])
@pytest.mark.parametrize("mix", ["mixed", "fusable"])
def test_results_identical_alone_and_in_the_mix(fused, mix):
    reqs = _mix() if mix == "mixed" else _fusable_mix()
    alone = []
    for p, o in reqs:
        s = gb.Solver(p, pool_bytes=1 << 28, **o)
        alone.append(s.solve())
        s.close()
    srv = gb.Server(pool_budget_bytes=8 << 30, device=0, max_active=6 if mix == "mixed" else 12, fused=fused)
    ids = []
    for p, o in reqs:
        opts = gb.gb_default_options(pool_bytes=1 << 28, **o)
        ids.append(srv.submit(p, opts))
    got = _wait(srv, ids)
    srv.close()
    for (p, _), a, rid in zip(reqs, alone, ids):
        b = got[rid]
        assert b.status == a.status == 0
        assert b.fmin_lo == a.fmin_lo and b.fmin_hi == a.fmin_hi
        assert b.fmin_lo <= 0.0 <= b.fmin_hi and b.fmin_hi - b.fmin_lo <= p.tol_f
        assert np.array_equal(b.box_lo, a.box_lo) and np.array_equal(b.box_hi, a.box_hi)
        assert np.array_equal(b.trace["gub"], a.trace["gub"])
        assert b.generations == a.generations
        assert b.latency_ms >= b.queue_ms >= 0.0


def test_admission_waits_for_memory():
    # budget for one request at a time: all still complete, one after another
    srv = gb.Server(pool_budget_bytes=1 << 28, device=0, max_active=8)
    ids = [srv.submit(S.chain(n=10, seed=k), gb.gb_default_options(pool_bytes=1 << 28, block=5, split_d=5,
                                                                    max_children=1 << 10))
           for k in range(5)]
    got = _wait(srv, ids)
    srv.close()
    lat = sorted(got[i].latency_ms for i in ids)
    assert all(got[i].status == 0 for i in ids)
    # later requests queued behind earlier ones
    assert max(got[i].queue_ms for i in ids) > 0.0
    assert lat[-1] > lat[0]


def test_poll_errors_and_invalid_request():
    srv = gb.Server(pool_budget_bytes=1 << 28, device=0, max_active=2)
    with pytest.raises(gb.GbError) as e:
        srv.poll(12345)
    assert e.value.status == gb.GB_E_INVALID
    p = S.chain(n=6)
    bad = S.Problem("bad", 6, p.nodes, p.root, p.tables, p.u, p.l, 1e-6, 3, p.s, 0)  # l > u
    rid = srv.submit(bad, gb.gb_default_options(pool_bytes=1 << 26))
    t0 = time.time()
    with pytest.raises(gb.GbError) as e:
        while srv.poll(rid) is None:
            assert time.time() - t0 < 30
            time.sleep(0.001)
    assert e.value.status == gb.GB_E_INVALID
    srv.close()
