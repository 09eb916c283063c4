"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake (a dropped term, a wrong sign, a transposed
index, a misplaced factor) in a copy of the oracle's C source, compiles it on
the CPU and runs the pin suite against it in a subprocess: the suite has to
fail.  The planted copy lives in a temporary directory; the real oracle is
never modified.

Not listed: dropping the projection in d_i b_j = (d_i B_j - b_j b.d_i B)/B.
Every use of grad b in the flat-space equations is dotted with v_E or
crossed with b, and both annihilate the component along b that the
projection removes, so that change leaves every result unchanged.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "gcb_oracle.c")
HDR = os.path.join(ROOT, "oracle", "gcb_oracle.h")

MUTANTS = [
    ("vE_sign", "P->vE[k] = c * ExB[k] / B2;", "P->vE[k] = -c * ExB[k] / B2;"),
    ("db_transposed", "P->db[i][j] = (P->dB[i][j] - P->b[j] * bdB) / P->Bmag;",
     "P->db[i][j] = (P->dB[j][i] - P->b[j] * bdB) / P->Bmag;"),
    ("bgb_transposed", "P->bgb[j] = P->b[0] * P->db[0][j] + P->b[1] * P->db[1][j] +",
     "P->bgb[j] = P->b[0] * P->db[j][0] + P->b[1] * P->db[j][1] +"),
    ("gamma_kappa_dropped",
     "return P->kappa * sqrt(1.0 + (upar * upar + perp_sq(P, p, mu, uperp)) / c2);",
     "return sqrt(1.0 + (upar * upar + perp_sq(P, p, mu, uperp)) / c2);"),
    ("vc_kappa_squared", "double pref = p->c * P->kappa * P->kappa / (qm * P->Bmag);",
     "double pref = p->c * P->kappa / (qm * P->Bmag);"),
    ("vc_charge_sign", "double pref = p->c * P->kappa * P->kappa / (qm * P->Bmag);",
     "double pref = p->c * P->kappa * P->kappa / (fabs(qm) * P->Bmag);"),
    ("rho_c_power", "double rho = p->c * p->c * Gam / (Q * Bmag);",
     "double rho = p->c * Gam / (Q * Bmag);"),
    ("boris_gamma_dropped", "t[k] = h * B[k] / (c * gm);", "t[k] = h * B[k] / c;"),
    ("gather_weights_swapped", "w[d] = od ? t[d] : 1.0 - t[d];",
     "w[d] = od ? 1.0 - t[d] : t[d];"),
    ("upar_curv_accel_dropped",
     "+ qm * dt * P->Epar + 0.5 * dt * G0 * g;", "+ qm * dt * P->Epar;"),
    ("upar_Epar_dropped",
     "+ qm * dt * P->Epar + 0.5 * dt * G0 * g;", "+ 0.5 * dt * G0 * g;"),
    ("k3_D_dropped", "double k3 = upr * upr + (c2 + perp_sq(P, p, mu, uperp)) * D * D;",
     "double k3 = upr * upr + (c2 + perp_sq(P, p, mu, uperp));"),
    ("upar_new_sign", "*upar_new = (upr + 0.5 * dt * G1 * g) / D;",
     "*upar_new = (upr - 0.5 * dt * G1 * g) / D;"),
    ("zero_curv_Epar_sign", "*upar_new = upar + qm * dt * P->Epar;",
     "*upar_new = upar - qm * dt * P->Epar;"),
    ("decompose_point_sign", "Rh[k] = xn[k] - 0.5 * dxp[k];", "Rh[k] = xn[k] + 0.5 * dxp[k];"),
    ("reconstruct_at_end", "Rp[k] = 0.5 * (Rk[k] + xn[k]);", "Rp[k] = Rk[k];"),
    ("fixed_point_explicit", "xn[k] + 0.5 * p->dt * (Vn[k] + Vk[k])",
     "xn[k] + p->dt * Vn[k]"),
]


def _build_mutant(tmp, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, old
    with open(os.path.join(tmp, "gcb_oracle.c"), "w") as fh:
        fh.write(src.replace(old, new))
    shutil.copy(HDR, os.path.join(tmp, "gcb_oracle.h"))
    lib = os.path.join(tmp, "libmut.so")
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", lib,
                    os.path.join(tmp, "gcb_oracle.c"), "-lm"], check=True)
    return lib


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(name, old, new, tmp_path):
    lib = _build_mutant(str(tmp_path), old, new)
    env = dict(os.environ, GCB_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1, f"pins did not catch mutant {name}:\n{r.stdout[-2000:]}"
