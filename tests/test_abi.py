"""The C-ABI library builds, loads and exports every symbol include/mm.h
declares; the ctypes structures match the C layout.  No compute calls (this
runs without a GPU)."""
import ctypes
import os
import re
import subprocess
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1506_04383_gb300 import build, mm
    build.build()
    return mm.load()


def declared_symbols():
    hdr = open(os.path.join(ROOT, "include", "mm.h")).read()
    return sorted(set(re.findall(r"^\s*(?:mm_status|void|const char\*)\s+(mm_\w+)\(", hdr, re.M)))


def test_header_and_binding_agree():
    from paper_1506_04383_gb300 import mm
    assert declared_symbols() == sorted(mm.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r" T (mm_\w+)", out))
    assert set(declared_symbols()) <= exported


def test_status_strings_and_defaults(lib):
    # host-only calls: no device work
    from paper_1506_04383_gb300 import mm
    assert lib.mm_status_string(0) == b"ok"
    assert lib.mm_status_string(2) == b"graph not connected"
    p = mm.default_params()
    assert p.struct_version == mm.MM_PARAMS_VERSION
    assert (p.f, p.b, p.alpha0, p.alpha_factor, p.alpha_min) == (20.0, 2.0, 1.0, 0.3, 0.008)
    assert p.iters_per_alpha == 2 and p.eps_final == pytest.approx(1e-4)


def test_struct_layout_matches_c(tmp_path):
    from paper_1506_04383_gb300 import mm
    src = tmp_path / "layout.c"
    src.write_text(textwrap.dedent("""
        #include <stdio.h>
        #include <stddef.h>
        #include "mm.h"
        int main(void) {
          printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(mm_params), offsetof(mm_params, alpha0),
                 offsetof(mm_params, seed), offsetof(mm_params, traverse_warps),
                 sizeof(mm_graph), offsetof(mm_graph, graph_ptr));
          printf("%zu %zu %zu %zu\\n", sizeof(mm_layout_stats),
                 offsetof(mm_layout_stats, level_sweeps), offsetof(mm_layout_stats, final_stress),
                 offsetof(mm_layout_stats, level_rel_change));
          printf("%zu %zu %zu %zu %zu\\n", sizeof(mm_prolong_sample),
                 offsetof(mm_prolong_sample, n_coarse), offsetof(mm_prolong_sample, seed),
                 offsetof(mm_prolong_sample, level), offsetof(mm_prolong_sample, x_target));
          printf("%zu %zu %zu\\n", offsetof(mm_params, learned_prolong),
                 offsetof(mm_params, approx_levels), offsetof(mm_params, exact_max_n));
          return 0;
        }
    """))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    a, b, c, d = subprocess.run([str(exe)], capture_output=True,
                                text=True).stdout.split("\n")[:4]
    P, G, S = mm.Params, mm.Graph, mm.LayoutStats
    assert [int(t) for t in a.split()] == [ctypes.sizeof(P), P.alpha0.offset, P.seed.offset,
                                           P.traverse_warps.offset, ctypes.sizeof(G),
                                           G.graph_ptr.offset]
    assert [int(t) for t in b.split()] == [ctypes.sizeof(S), S.level_sweeps.offset,
                                           S.final_stress.offset, S.level_rel_change.offset]
    Q = mm.ProlongSample
    assert [int(t) for t in c.split()] == [ctypes.sizeof(Q), Q.n_coarse.offset, Q.seed.offset,
                                           Q.level.offset, Q.x_target.offset]
    assert [int(t) for t in d.split()] == [P.learned_prolong.offset, P.approx_levels.offset,
                                           P.exact_max_n.offset]


def test_product_path_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_1506_04383_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "mm_oracle" not in text, f


@pytest.mark.parametrize("field,value,status", [
    ("struct_version", 0, 1), ("k", 3, 7), ("theta", -0.5, 1), ("coarsest_n", 0, 1),
    ("alpha_factor", 1.5, 1), ("max_levels", 0, 1), ("leaf_size", 65, 1),
    ("approx_levels", -1, 1), ("approx_levels", 1000, 1), ("exact_max_n", -1, 1)])
def test_parameters_are_checked_before_any_device_work(lib, field, value, status):
    # host-only: the parameter check runs before the graph or the device is
    # touched, so a descriptor without buffers is enough
    import ctypes
    from paper_1506_04383_gb300 import mm
    g = mm.Graph(n=4, nnz=0, row_ptr=None, col=None, edge_len=None, num_graphs=1,
                 graph_ptr=None)
    p = mm.default_params()
    setattr(p, field, value)
    out = ctypes.c_void_p()
    st = lib.mm_build_hierarchy(ctypes.byref(g), ctypes.byref(p), None, ctypes.byref(out))
    assert st == status, lib.mm_last_error()
    assert out.value is None
    assert lib.mm_last_error() != b""


def test_null_graph_buffers_are_refused_on_the_host(lib):
    import ctypes
    from paper_1506_04383_gb300 import mm
    g = mm.Graph(n=4, nnz=6, row_ptr=None, col=None, edge_len=None, num_graphs=1,
                 graph_ptr=None)
    p = mm.default_params()
    out = ctypes.c_void_p()
    st = lib.mm_build_hierarchy(ctypes.byref(g), ctypes.byref(p), None, ctypes.byref(out))
    assert st == 1 and b"graph" in lib.mm_last_error()
