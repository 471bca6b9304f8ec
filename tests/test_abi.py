"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/gb.h declares; the objective format agrees between the header,
the input generator and the oracle; validation errors need no GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2507_01770_gb300 as gb
import synthetic as S
from synthetic import dag as D

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gb.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(gb_[a-z_0-9]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    L = gb.load()
    names = _declared()
    assert names, "no declarations parsed"
    for name in names:
        assert hasattr(L, name), name
    assert set(names) == set(gb.EXPORTS)


def test_opcodes_agree_across_header_generator_and_oracle():
    import oracle
    txt = open(HEADER).read()
    hdr = {m.group(1): int(m.group(2)) for m in re.finditer(r"GB_OP_([A-Z_]+)\s*=\s*(\d+)", txt)}
    gen = {name: code for code, name in D.OP_NAMES.items()}
    assert hdr == gen == oracle.OP
    assert D.NODE_DTYPE.itemsize == 32


def test_struct_layouts_match_header(tmp_path):
    import subprocess
    src = tmp_path / "sizes.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "gb.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(gb_node), sizeof(gb_options),'
                   ' sizeof(gb_gen_stat), sizeof(gb_result), offsetof(gb_result, trace), sizeof(gb_snapshot),'
                   ' offsetof(gb_snapshot, generations)); return 0;}\n')
    exe = tmp_path / "sizes"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    assert got == [D.NODE_DTYPE.itemsize, ctypes.sizeof(gb.gb_options), ctypes.sizeof(gb.gb_gen_stat),
                   ctypes.sizeof(gb.gb_result), gb.gb_result.trace.offset, ctypes.sizeof(gb.gb_snapshot),
                   gb.gb_snapshot.generations.offset]


def test_invalid_problems_rejected_without_gpu():
    p = S.chain(n=6)
    bad = p.nodes.copy()
    bad[2]["a"] = 9
    with pytest.raises(gb.GbError) as e:
        gb.gb_create_problem(bad, p.root, p.tables, p.n, p.l, p.u, 1e-6)
    assert e.value.status == gb.GB_E_INVALID
    with pytest.raises(gb.GbError) as e:
        gb.gb_create_problem(p.nodes, p.root, p.tables, p.n, p.u, p.l, 1e-6)
    assert e.value.status == gb.GB_E_INVALID
    with pytest.raises(gb.GbError) as e:   # diagonal samples run in the interpreter only
        gb.gb_create_problem(p.nodes, p.root, p.tables, p.n, p.l, p.u, 1e-6,
                             gb.gb_default_options(samples=10, eval_mode=2))
    assert e.value.status == gb.GB_E_INVALID
    with pytest.raises(gb.GbError) as e:
        gb.gb_create_problem(p.nodes, p.root, p.tables, p.n, p.l, p.u, 1e-6, gb.gb_default_options(samples=65))
    assert e.value.status == gb.GB_E_INVALID
    with pytest.raises(gb.GbError) as e:   # split_m must be 2 or 4
        gb.gb_create_problem(p.nodes, p.root, p.tables, p.n, p.l, p.u, 1e-6,
                             gb.gb_default_options(split_m=3))
    assert e.value.status == gb.GB_E_INVALID
    q = S.paper_griewank(n=4)
    with pytest.raises(gb.GbError) as e:   # products run on the interpreter only
        gb.gb_create_problem(q.nodes, q.root, q.tables, q.n, q.l, q.u, 1e-6, gb.gb_default_options(eval_mode=3))
    assert e.value.status == gb.GB_E_INVALID and "IPROD" in str(e.value)
    g = S.Dag()
    t = g.iprod(g.ivar(0), 0, 2, 1)
    f = g.isum(g.mul(g.ivar(0), g.const(2.0)), 0, 2, 1)
    g2 = S.Dag()
    inner = g2.iprod(g2.ivar(0), 0, 2, 1)
    bad_t = g2.isum(g2.add(g2.ivar(0), inner), 0, 2, 1)   # IPROD inside a sum template
    with pytest.raises(gb.GbError) as e:
        gb.gb_create_problem(g2.nodes(), bad_t, [], 2, [0.0, 0.0], [1.0, 1.0], 1e-6)
    assert e.value.status == gb.GB_E_INVALID
    del t, f
    g = S.Dag()
    f = g.add(g.ivar(0), g.const(1.0))      # IDX_VAR outside a sum
    with pytest.raises(gb.GbError) as e:
        gb.gb_create_problem(g.nodes(), f, [], 1, [0.0], [1.0], 1e-6)
    assert e.value.status == gb.GB_E_INVALID
    assert "outside a sum" in str(e.value)


def test_autotune_rejects_invalid_problems_without_gpu():
    p = S.chain(n=6)
    bad = S.Problem("bad", 6, p.nodes, p.root, p.tables, p.u, p.l, 1e-6, 3, p.s, 0)   # l > u
    with pytest.raises(gb.GbError) as e:
        gb.gb_autotune(bad, budget_ms=10.0)
    assert e.value.status == gb.GB_E_INVALID


def test_checkpoint_and_server_calls_reject_null_without_gpu():
    import ctypes
    L = gb.load()
    snap = gb.gb_snapshot()
    res = gb.gb_result()
    assert L.gb_snapshot_take(None, ctypes.byref(snap)) == gb.GB_E_INVALID
    assert L.gb_solve_resume(None, ctypes.byref(snap), ctypes.byref(res)) == gb.GB_E_INVALID
    assert L.gb_server_set_fused(None, 1) == gb.GB_E_INVALID
    L.gb_free_snapshot(ctypes.byref(snap))          # a zeroed snapshot is released safely
    L.gb_free_result(ctypes.byref(res))


def test_status_strings():
    assert gb.gb_status_str(gb.GB_OK) == "ok"
    assert gb.gb_status_str(gb.GB_E_CAPACITY) == "box pool capacity reached"


def test_no_cpu_fallback_without_device():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    p = S.chain(n=4)
    with pytest.raises(gb.GbError) as e:
        gb.gb_create_problem(p.nodes, p.root, p.tables, p.n, p.l, p.u, 1e-6)
    assert e.value.status == gb.GB_E_CUDA
