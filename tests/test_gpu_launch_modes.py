"""The launch mechanics do not change a solve (GPU).

A generation's kernels can be launched with programmatic dependent launch
(GB_PDL=1: a kernel may start while its predecessor finishes, and waits for
it before touching its results), a single-parent generation runs the
parent's tables on a second stream beside the pool partition, and a solve
replays several generations from one CUDA graph.  None of this may change
what the search computes (section 3.1 loop): the same solve with the early
start turned on (in a child process, as the switch is read once per
process) and off, and with one generation per host synchronisation (no
graphs), must give the same trace, enclosure and output boxes bit for bit.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# A mixed problem on the block-record pool (FP32 prefilter, warp-per-child
# kernel with term tables, one parent per generation) and a chain problem on
# dense rows (one child per thread), both for a bounded number of generations.
CHILD = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
import numpy as np
import paper_2507_01770_gb300 as gb
import synthetic as S
out = {}
for name, p, kw in [
    ("mixed", S.mixed(n=2000, seed=3), dict(block=100, split_m=2, split_d=10, max_children=1 << 10,
                                            fp32_prefilter=1, max_generations=300)),
    ("chain", S.chain(n=100, seed=1), dict(block=10, split_m=4, split_d=10, max_children=1 << 20,
                                           max_generations=20)),
]:
    for gps in (16, 1):
        s = gb.Solver(p, gens_per_sync=gps, pool_bytes=8 << 30, **kw)
        r = s.solve(raise_on_error=False)
        s.close()
        out[f"{name}-{gps}"] = dict(
            status=int(r.status), generations=int(r.generations), lo=r.fmin_lo.hex(), hi=r.fmin_hi.hex(),
            trace={k: np.asarray(r.trace[k]).tolist() for k in ("parents", "children", "kept32", "kept", "pool")},
            gub=[float(x).hex() for x in r.trace["gub"]],
            box_flo=[] if r.box_flo is None else [float(x).hex() for x in r.box_flo],
            box_lo="" if r.box_lo is None else r.box_lo.tobytes().hex(),
            box_hi="" if r.box_hi is None else r.box_hi.tobytes().hex())
print(json.dumps(out))
"""


def _run(pdl):
    env = dict(os.environ)
    env.pop("GB_PDL", None)
    if pdl:
        env["GB_PDL"] = "1"
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], capture_output=True, text=True, env=env, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_early_start_streams_and_graphs_do_not_change_the_solve():
    a = _run(pdl=False)
    b = _run(pdl=True)
    assert a.keys() == b.keys()
    for k in a:
        assert a[k] == b[k], k
    for name in ("mixed", "chain"):
        assert a[f"{name}-16"] == a[f"{name}-1"], name
        assert a[f"{name}-16"]["generations"] > 0
        assert len(a[f"{name}-16"]["gub"]) == a[f"{name}-16"]["generations"]
