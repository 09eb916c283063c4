"""The C-ABI library builds, loads and exports every symbol include/gcb.h
declares; argument checks answer without a GPU; the Python mirror of the
structs matches the C layout.  CPU only (no kernel is launched)."""
import ctypes as C
import os
import re
import subprocess
import sys

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
    """Every descriptor the binding passes by pointer has the header's size
    and field offsets (compiled with the host C compiler)."""
    fields = [("gcb_grid", "rec", G.GcbGrid), ("gcb_grid", "stride", G.GcbGrid),
              ("gcb_particles", "flags", G.GcbParticles), ("gcb_particles", "pid", G.GcbParticles),
              ("gcb_params", "gca_tol", G.GcbParams), ("gcb_params", "step_index", G.GcbParams),
              ("gcb_params", "fuse_steps", G.GcbParams), ("gcb_params", "drift_frame", G.GcbParams),
              ("gcb_params", "gyro_phase", G.GcbParams), ("gcb_params", "mirror", G.GcbParams),
              ("gcb_stats", "sum_ekin", G.GcbStats), ("gcb_stats", "n_exited", G.GcbStats),
              ("gcb_grid_ks", "dl", G.GcbGridKs), ("gcb_ks_params", "r_out", G.GcbKsParams),
              ("gcb_ks_params", "kick_basis", G.GcbKsParams),
              ("gcb_current", "q", G.GcbCurrent), ("gcb_current", "w", G.GcbCurrent),
              ("gcb_current", "J", G.GcbCurrent),
              ("gcb_deposit_stats", "n_atomics", G.GcbDepositStats)]
    lines = "".join(f'printf("%zu %zu\\n", sizeof({t}), offsetof({t}, {f}));\n'
                    for t, f, _ in fields)
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "gcb.h"\n'
                   "int main(void){\n" + lines + "return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = [tuple(map(int, ln.split()))
           for ln in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split("\n")
           if ln.strip()]
    want = [(C.sizeof(cls), getattr(cls, f).offset) for _, f, cls in fields]
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
    # the deposition refuses a missing current before anything else
    rc = lib.gcb_push_deposit_sr(C.byref(p), C.byref(g), C.byref(prm), None, 1, None, None, 0,
                                 None, None)
    assert rc == 1 and b"current" in lib.gcb_last_error()
    cap = re.search(r"#define GCB_DEPOSIT_MAX_CELLS (\d+)", open(HEADER).read())
    assert int(cap.group(1)) == G.DEPOSIT_MAX_CELLS
    # Kerr-Schild: an unknown kick basis is refused before any launch
    gk = G.GcbGrid(2, G.F32, (C.c_int64 * 3)(16, 17, 1), (C.c_double * 3)(0.1, 3.141592653589793 / 16, 1), 0,
                   lib.gcb_grid_stride(2, G.F32, 0), 4096)
    ks = G.GcbGridKs(gk, 0.3, 4096)
    for basis, want in ((2, 1), (-1, 1)):
        rc = lib.gcb_ks_cell_size(C.byref(ks), C.byref(G.GcbKsParams(0.9, 1.5, 50.0, basis)),
                                  C.c_void_p(4096), None)
        assert rc == want and b"kick_basis" in lib.gcb_last_error()


def test_binding_fails_loudly_without_the_library():
    """No CPU fallback: importing the binding with the CUDA library absent raises."""
    code = ("import sys; sys.path.insert(0, %r)\n"
            "import paper_2007_14401_gb300.build as b\n"
            "b.LIB = b.LIB + '.absent'\n"
            "try:\n"
            "    import paper_2007_14401_gb300.gcb\n"
            "except RuntimeError as e:\n"
            "    print('raised:', e); sys.exit(0)\n"
            "sys.exit(3)\n") % ROOT
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "is not built" in r.stdout, r.stdout + r.stderr


def test_peak_library_exports_its_declared_symbol():
    """include/gcb_peak.h's entry points are exported by libgcb_peak.so (the
    benchmark's FMA-rate and atomic-rate measurements), and answer invalid
    arguments without a GPU."""
    from paper_2007_14401_gb300 import build
    path = build.build_peak()
    txt = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "gcb_peak.h")).read(),
                 flags=re.S)
    names = sorted(set(re.findall(r"\b(gcb_[a-z0-9_]+)\s*\(", txt)))
    assert names == ["gcb_peak_fma", "gcb_peak_red"]
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True,
                         text=True).stdout
    assert set(names) <= set(re.findall(r" T (gcb_\w+)", out))
    lib = C.CDLL(path)
    lib.gcb_peak_fma.argtypes = [C.c_int, C.c_int, C.c_void_p, C.POINTER(C.c_double)]
    v = C.c_double(0.0)
    assert lib.gcb_peak_fma(7, 10, None, C.byref(v)) == 1
    assert lib.gcb_peak_fma(0, 0, None, C.byref(v)) == 1
    assert lib.gcb_peak_fma(0, 10, None, None) == 1
    lib.gcb_peak_red.argtypes = [C.c_int, C.c_int, C.c_int, C.c_void_p, C.POINTER(C.c_double)]
    assert lib.gcb_peak_red(2, 0, 10, None, C.byref(v)) == 1
    assert lib.gcb_peak_red(0, 2, 10, None, C.byref(v)) == 1
    assert lib.gcb_peak_red(0, 0, 0, None, C.byref(v)) == 1
    assert lib.gcb_peak_red(1, 1, 10, None, None) == 1
