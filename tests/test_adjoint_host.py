"""Host-side pieces of the adjoint: the mode split of the reconnection
workload's fields and the checkpoint workspace sizing (no GPU needed)."""
import ctypes as C

import numpy as np

from paper_2007_14401_gb300 import inputs


def test_mode_split_reproduces_workload_fields():
    kw = dict(nx=64, ny=32, delta=2.0, n_modes=6, max_mode=3, n_particles=16, seed=5)
    base, pats, amps, st, prm = inputs.reconnection_2d_modes(**kw)
    f, st2, prm2 = inputs.reconnection_2d(**kw)
    c = inputs.combine_fields(base, pats, amps)
    for key in ("E", "B", "dB"):
        for a, b in zip(c[key], f[key]):
            np.testing.assert_allclose(a, b, rtol=0, atol=1e-14)
    assert prm["qm"] == prm2["qm"]
    np.testing.assert_array_equal(st["u"], st2["u"])
    # a second amplitude vector: the split is linear, not just exact at amps
    a2 = np.linspace(-0.05, 0.05, len(amps))
    f2, _, _ = inputs.reconnection_2d(**kw, mode_amps=a2)
    c2 = inputs.combine_fields(base, pats, a2)
    for key in ("E", "B", "dB"):
        for a, b in zip(c2[key], f2[key]):
            np.testing.assert_allclose(a, b, rtol=0, atol=1e-14)


def test_adjoint_workspace_bytes():
    from paper_2007_14401_gb300 import gcb
    lib = gcb.lib()

    def ws(n, steps, ck, pos_mode=gcb.POS_F64, mom=gcb.F64, prm=None):
        p = gcb.GcbParticles()
        p.n, p.ndim, p.pos_mode, p.mom_dtype = n, 2, pos_mode, mom
        g = gcb.GcbGrid()
        g.ndim = 2
        g.n = (C.c_int64 * 3)(64, 32, 1)
        g.dx = (C.c_double * 3)(1.0, 1.0, 1.0)
        return lib.gcb_adjoint_workspace_bytes(C.byref(p), C.byref(g),
                                               C.byref(prm) if prm is not None else None,
                                               steps, ck)

    # one state set of n = 1024 FP64 particles: 2 x + 3 u + 2 dxp (8 B) + flags
    S = 7 * 8 * 1024 + 1024
    base = ws(1024, 16, 16)
    assert base == 256 + (1 + 15 + 2) * S
    assert ws(1024, 256, 16) == 256 + (16 + 15 + 2) * S
    assert ws(1024, 257, 16) == 256 + (17 + 15 + 2) * S
    assert ws(1024, 10, 1) == 256 + (10 + 0 + 2) * S
    assert ws(1024, 0, 16) == 0 and ws(1024, 16, 0) == 0
    # mixed: FP32 pairs (hi, lo) and FP32 momenta
    Sm = 2 * 4 * 1024 * 2 + 5 * 4 * 1024 + 1024
    assert ws(1024, 16, 4, gcb.POS_F32PAIR, gcb.F32) == 256 + (4 + 3 + 2) * Sm
    # sorting at the checkpoints adds the sort's scratch, one int32
    # permutation per checkpoint, two orders, 7 adjoint copies and an id copy
    srt = gcb.make_params(dict(dt=1.0, qm=(-1.0,)), sort_every=4, sort_tile=(1, 1))
    extra = ws(1024, 16, 4, prm=srt) - ws(1024, 16, 4)
    assert extra > (4 + 2) * 4 * 1024 + 7 * 8 * 1024 + 8 * 1024
    assert ws(1024, 16, 4, prm=gcb.make_params(dict(dt=1.0, qm=(-1.0,)))) == ws(1024, 16, 4)
