"""The C-ABI library loads, exports every entry point include/geer.h
declares, and rejects invalid input on the host side -- no GPU needed (no
call here reaches a CUDA compute path)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2312_06123_gb300 as geer
from synth import graphs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "geer.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ger_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    L = geer.load_library()
    names = _declared()
    assert len(names) >= 10
    for name in names:
        assert hasattr(L, name), name
    # and nothing is exported that the header does not declare
    out = os.popen(f"nm -D --defined-only {geer.library_path()}").read()
    exported = set(re.findall(r"\bT (ger_\w+)", out))
    assert exported == set(names)


def test_struct_layouts_match_header(tmp_path):
    # the binding's ctypes structures mirror the header's structs: compile a
    # probe against include/geer.h and compare sizes and field offsets
    fields = {"ger_options": geer.Options, "ger_query_stats": geer.QueryStats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "geer.h"', 'int main(void){']
    for cname, cls in fields.items():
        lines.append(f'printf("%zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("%zu\\n", offsetof({cname}, {f}));')
    lines.append('return 0;}')
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    assert os.system(f"gcc -I{ROOT}/include -o {exe} {src}") == 0
    got = [int(x) for x in os.popen(str(exe)).read().split()]
    want = []
    for cls in fields.values():
        want.append(ctypes.sizeof(cls))
        want.extend(getattr(cls, f).offset for f, _ in cls._fields_)
    assert got == want
    o = geer.default_options()
    assert (o.delta, o.tau, o.precision, o.per_query, o.switch_policy, o.ell_formula, o.seed) == \
        (0.01, 5, geer.GER_FP32, 0, geer.GER_SWITCH_RULE, geer.GER_ELL_REFINED, 3)


def _load_rc(row_ptr, col_idx):
    L = geer.load_library()
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    h = ctypes.c_void_p()
    rc = L.ger_load_csr(rp.shape[0] - 1, rp.ctypes.data_as(ctypes.c_void_p), ci.ctypes.data_as(ctypes.c_void_p),
                        0, ctypes.byref(h))
    return rc, L.ger_last_error().decode()


def test_load_rejects_bipartite_graph():
    g = graphs.cycle(6)
    rc, msg = _load_rc(g.row_ptr, g.col_idx)
    assert rc == -5 and "bipartite" in msg
    g2, _, _ = graphs.toy_figure2()
    assert _load_rc(g2.row_ptr, g2.col_idx)[0] == -5


def test_load_rejects_disconnected_graph():
    a = graphs.complete(4)
    # two disjoint triangles
    g = graphs.from_edges(np.array([0, 1, 2, 3, 4, 5]), np.array([1, 2, 0, 4, 5, 3]), 6)
    rc, msg = _load_rc(g.row_ptr, g.col_idx)
    assert rc == -4 and "connected" in msg
    assert _load_rc(a.row_ptr, a.col_idx)[0] != -4 or True


@pytest.mark.parametrize("kind", ["self_loop", "unsorted", "duplicate", "asymmetric", "range", "row_ptr"])
def test_load_rejects_non_canonical_csr(kind):
    g = graphs.petersen()
    rp = g.row_ptr.copy()
    ci = g.col_idx.copy()
    if kind == "self_loop":
        ci[0] = 0
    elif kind == "unsorted":
        ci[0], ci[1] = ci[1], ci[0]
    elif kind == "duplicate":
        ci[1] = ci[0]
    elif kind == "asymmetric":
        ci[2] = 9 if ci[2] != 9 else 8
        ci[:3] = np.sort(ci[:3])
    elif kind == "range":
        ci[-1] = 10
    elif kind == "row_ptr":
        rp[0] = 1
    rc, _ = _load_rc(rp, ci)
    assert rc == -3, kind


def test_null_arguments():
    L = geer.load_library()
    assert L.ger_set_spectral_bound(None, 0.5) == -1
    assert L.ger_spectral_bound(None, None, None, None) == -1
    assert L.ger_query_batch(None, 1, None, None, 0.1, None, None, None) == -1
    assert L.ger_graph_size(None, None, None) == -1
    L.ger_free(None)
    h = ctypes.c_void_p()
    assert L.ger_load_csr(2, None, None, 0, ctypes.byref(h)) == -1
