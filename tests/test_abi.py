"""The C-ABI library builds, loads and exports every symbol include/gcb.h
declares; argument checks answer without a GPU; the Python mirror of the
structs matches the C layout.  CPU only (no kernel is launched)."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gcb.h")


@pytest.fixture(scope="module")
def G():
    from paper_2007_14401_gb300 import build
    build.build()
    from paper_2007_14401_gb300 import gcb
    return gcb


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(gcb_[a-z0-9_]+)\s*\(", txt)))


def test_exports_every_declared_symbol(G):
    lib = G.lib()
    names = declared_functions()
    assert "gcb_push_sr" in names and len(names) >= 9
    for nm in names:
        assert hasattr(lib, nm), nm
    assert sorted(G.EXPORTS) == names
    out = subprocess.run(["nm", "-D", "--defined-only", G._build.LIB], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r" T (gcb_\w+)", out))
    assert set(names) <= exported


def test_struct_layout_matches_header(G, tmp_path):
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "gcb.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu\\n",'
                   'sizeof(gcb_grid), offsetof(gcb_grid, rec), sizeof(gcb_particles),'
                   'offsetof(gcb_particles, flags), sizeof(gcb_params),'
                   'offsetof(gcb_params, gca_tol), sizeof(gcb_stats),'
                   'offsetof(gcb_stats, sum_ekin)); return 0;}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = list(map(int, subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()))
    want = [C.sizeof(G.GcbGrid), G.GcbGrid.rec.offset, C.sizeof(G.GcbParticles),
            G.GcbParticles.flags.offset, C.sizeof(G.GcbParams), G.GcbParams.gca_tol.offset,
            C.sizeof(G.GcbStats), G.GcbStats.sum_ekin.offset]
    assert got == want


def test_strides_and_status_strings(G):
    lib = G.lib()
    assert lib.gcb_grid_stride(2, G.F32, 1) == 12
    assert lib.gcb_grid_stride(2, G.F32, 0) == 8
    assert lib.gcb_grid_stride(3, G.F32, 1) == 16
    assert lib.gcb_grid_stride(2, G.F64, 1) == 12
    assert lib.gcb_grid_stride(3, G.F64, 1) == 16
    assert lib.gcb_grid_stride(3, G.F64, 0) == 6
    assert lib.gcb_grid_stride(4, G.F32, 0) == 0
    assert lib.gcb_status_string(1) == b"GCB_EINVAL"
    assert lib.gcb_version() >= 100


def test_argument_errors_without_gpu(G):
    lib = G.lib()
    st = G.GcbStats()
    rc = lib.gcb_push_sr(None, None, None, 1, None, None, 0, C.byref(st))
    assert rc == 1 and b"grid" in lib.gcb_last_error()
    g = G.GcbGrid(2, G.F32, (C.c_int64 * 3)(16, 16, 1), (C.c_double * 3)(1, 1, 1), 1,
                  lib.gcb_grid_stride(2, G.F32, 1), 4096)
    prm = G.make_params(dict(dt=0.45, qm=(-1.0,)))
    p = G.GcbParticles()
    p.n, p.ndim = 10, 3
    rc = lib.gcb_push_sr(C.byref(p), C.byref(g), C.byref(prm), 1, None, None, 0, None)
    assert rc == 1 and b"ndim" in lib.gcb_last_error()
    g.stride = 7
    rc = lib.gcb_push_sr(C.byref(p), C.byref(g), C.byref(prm), 1, None, None, 0, None)
    assert rc == 1 and b"stride" in lib.gcb_last_error()
    assert lib.gcb_pos_split(-1, None, None, None, None) == 1
