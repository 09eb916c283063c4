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
SRC_KS = os.path.join(ROOT, "oracle", "gcb_oracle_ks.c")
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
     "+ qm * dt * P->Epar + 0.5 * dt * G0 * g + fm;", "+ qm * dt * P->Epar + fm;"),
    ("upar_Epar_dropped",
     "+ qm * dt * P->Epar + 0.5 * dt * G0 * g + fm;", "+ 0.5 * dt * G0 * g + fm;"),
    ("k3_D_dropped", "double k3 = upr * upr + (c2 + perp_sq(P, p, mu, uperp)) * D * D;",
     "double k3 = upr * upr + (c2 + perp_sq(P, p, mu, uperp));"),
    ("upar_new_sign", "*upar_new = (upr + 0.5 * dt * G1 * g) / D;",
     "*upar_new = (upr - 0.5 * dt * G1 * g) / D;"),
    ("zero_curv_Epar_sign", "*upar_new = upar + qm * dt * P->Epar + fm;",
     "*upar_new = upar - qm * dt * P->Epar + fm;"),
    ("decompose_point_sign", "Rh[k] = xn[k] - 0.5 * dxp[k];", "Rh[k] = xn[k] + 0.5 * dxp[k];"),
    ("reconstruct_at_end", "Rp[k] = 0.5 * (Rk[k] + xn[k]);", "Rp[k] = Rk[k];"),
    ("fixed_point_explicit", "xn[k] + 0.5 * p->dt * (Vn[k] + Vk[k])",
     "xn[k] + p->dt * Vn[k]"),
]


# mistakes in the covariant (Kerr-Schild) oracle
MUTANTS_KS = [
    ("ks_lapse", "m->alpha = ddiv(dc(1.0), dsqrt(onez));", "m->alpha = ddiv(dc(1.0), onez);"),
    ("ks_shift", "m->beta[0] = ddiv(z, onez);", "m->beta[0] = ddiv(z, dadd(onez, onez));"),
    ("ks_grphi_sign", "m->gdn[0][2] = m->gdn[2][0] = dscale(dmul(onez, s2), -a);",
     "m->gdn[0][2] = m->gdn[2][0] = dscale(dmul(onez, s2), a);"),
    ("geodesic_lapse_sign", "G[i] = -Gam * M->dalpha[i] + ub - M->alpha * uu / (2.0 * Gam);",
     "G[i] = Gam * M->dalpha[i] + ub - M->alpha * uu / (2.0 * Gam);"),
    ("geodesic_half", "G[i] = -Gam * M->dalpha[i] + ub - M->alpha * uu / (2.0 * Gam);",
     "G[i] = -Gam * M->dalpha[i] + ub - M->alpha * uu / Gam;"),
    ("velocity_shift_sign", "V[i] = M->alpha * s / Gam - M->beta[i];",
     "V[i] = M->alpha * s / Gam + M->beta[i];"),
    ("half_kick_full_dt", "ks_kick(a, x[0], x[1], D, B, qm, 0.5 * dt * alpha, basis, u);",
     "ks_kick(a, x[0], x[1], D, B, qm, dt * alpha, basis, u);"),
    ("global_kick_sqrtg_dropped",
     "c[i] += M->sqrtg * levi_civita(i, j, k) * a_up[j] * b_up[k];",
     "c[i] += levi_civita(i, j, k) * a_up[j] * b_up[k];"),
    ("global_kick_cross_not_raised", "cross_covariant(M, um_up, t, x);",
     "cross_covariant(M, um, t, x);"),
    ("global_kick_t2_euclidean", "double t2 = t[0] * t_dn[0] + t[1] * t_dn[1] + t[2] * t_dn[2];",
     "double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];"),
    ("global_kick_D_not_lowered", "for (int k = 0; k < 3; ++k) um[k] = u[k] + h * Dd[k];",
     "for (int k = 0; k < 3; ++k) um[k] = u[k] + h * D[k];"),
    ("global_kick_handedness", "return 0.5 * (double)((i - j) * (j - k) * (k - i));",
     "return -0.5 * (double)((i - j) * (j - k) * (k - i));"),
    ("frame_transposed", "for (int i = 0; i < 3; ++i) uh[a] += L[i][a] * u[i];",
     "for (int i = 0; i < 3; ++i) uh[a] += L[a][i] * u[i];"),
    ("gca_drift_dropped", "for (int j = 0; j < 3; ++j) s += Fb.M.gup[i][j] * (ub * Fb.bdn[j] / Gam + Fb.vE[j]);",
     "for (int j = 0; j < 3; ++j) s += Fb.M.gup[i][j] * (ub * Fb.bdn[j] / Gam);"),
    ("drift_sign", "F->vE[2] = sg * (D[0] * B[1] - D[1] * B[0]) / B2;",
     "F->vE[2] = sg * (D[1] * B[0] - D[0] * B[1]) / B2;"),
    ("cell_size_not_rooted", "dl[(long)j * (f->nr - 1) + i] = sqrt(area);",
     "dl[(long)j * (f->nr - 1) + i] = area;"),
    ("imr_not_midpoint", "for (int k = 0; k < 3; ++k) { xb[k] = 0.5 * (xk[k] + x[k]); ub[k] = 0.5 * (wk[k] + up[k]); }",
     "for (int k = 0; k < 3; ++k) { xb[k] = xk[k]; ub[k] = wk[k]; }"),
]


# mistakes in the oracle's exact drift frame (Sec. 2.2), run against its own pins
MUTANTS_BT = [
    ("bt_vE_half", "out[k] = 2.0 * c * ExB[k] / (S * (1.0 + sq));",
     "out[k] = c * ExB[k] / (S * (1.0 + sq));"),
    ("bt_Bprime_sign", "double Bp = sqrt(0.5 * (B2 - E2 + S * sq));",
     "double Bp = sqrt(0.5 * (B2 + E2 + S * sq));"),
    ("bt_Psi_sign", "double Psi = 2.0 * Ep * B2 / (Bp * S * (1.0 + sq));",
     "double Psi = -2.0 * Ep * B2 / (Bp * S * (1.0 + sq));"),
    ("bt_eta_unrooted", "double eta = 1.0 / (Bm * sqrt(Psi * Psi * Ep2 / B2 + 1.0));",
     "double eta = 1.0 / (Bm * (Psi * Psi * Ep2 / B2 + 1.0));"),
    ("bt_bstar_unused", "for (int k = 0; k < 3; ++k) { P->vE[k] = bt[k]; P->b[k] = bt[3 + k]; }",
     "for (int k = 0; k < 3; ++k) { P->vE[k] = bt[k]; }"),
    ("bt_kappa_simplified", "P->kappa = bt[6];", "P->kappa = P->kappa;"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS_BT, ids=[c[0] for c in MUTANTS_BT])
def test_frame_pins_catch_planted_mistake(name, old, new, tmp_path):
    lib = _build_mutant(str(tmp_path), SRC, old, new)
    env = dict(os.environ, GCB_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_frame_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1, f"pins did not catch mutant {name}:\n{r.stdout[-2000:]}"


# mistakes in the evolved gyration phase, run against its own pins
MUTANTS_PHASE = [
    ("phase_sign", "double phi = -qm * P->Bmag * p->dt / (p->c * P->kappa * G);",
     "double phi = qm * P->Bmag * p->dt / (p->c * P->kappa * G);"),
    ("phase_kappa_dropped", "double phi = -qm * P->Bmag * p->dt / (p->c * P->kappa * G);",
     "double phi = -qm * P->Bmag * p->dt / (p->c * G);"),
    ("phase_gamma_dropped", "double phi = -qm * P->Bmag * p->dt / (p->c * P->kappa * G);",
     "double phi = -qm * P->Bmag * p->dt / (p->c * P->kappa);"),
    ("phase_axis_reversed", "cross3(P->b, bpg, bxd);", "cross3(bpg, P->b, bxd);"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS_PHASE, ids=[c[0] for c in MUTANTS_PHASE])
def test_phase_pins_catch_planted_mistake(name, old, new, tmp_path):
    lib = _build_mutant(str(tmp_path), SRC, old, new)
    env = dict(os.environ, GCB_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_phase_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1, f"pins did not catch mutant {name}:\n{r.stdout[-2000:]}"


# mistakes in the oracle's current deposition and in the step velocity it uses
MUTANTS_DEP = [
    ("dep_midpoint_only", "double avg = (g[0] + 4.0 * g[1] + g[2]) / 6.0;",
     "double avg = g[1];"),
    ("dep_face_time_sign", "t[nt++] = (m - s0[a]) / ds[a];", "t[nt++] = (s0[a] - m) / ds[a];"),
    ("dep_cell_at_piece_start", "cell[a] = (long)floor(s0[a] + ds[a] * 0.5 * (ta + tb));",
     "cell[a] = (long)floor(s0[a] + ds[a] * ta);"),
    ("dep_piece_duration_dropped",
     "double pref = a < nd ? Qw * disp[a] * tau / (dt * V) : Qw * vz * tau / V;",
     "double pref = a < nd ? Qw * disp[a] / (dt * V) : Qw * vz * tau / V;"),
    ("dep_vz_over_dt",
     "double pref = a < nd ? Qw * disp[a] * tau / (dt * V) : Qw * vz * tau / V;",
     "double pref = a < nd ? Qw * disp[a] * tau / (dt * V) : Qw * vz * tau / (dt * V);"),
    ("dep_corner_offset", "for (int r = 0; r < no; ++r) idx[oth[r]] += (o >> r) & 1;",
     "for (int r = 0; r < no; ++r) idx[oth[r]] += o & 1;"),
    ("dep_path_from_new_x", "for (int k = 0; k < 3; ++k) { q[k] = x0[k]; q[3 + k] = k < nd ? di[k] : 0.0; }",
     "for (int k = 0; k < 3; ++k) { q[k] = xi[k]; q[3 + k] = k < nd ? di[k] : 0.0; }"),
    ("dep_species_charge", "double Qw = dep->q[(flags[i] >> 6) & 3] * (dep->w ? dep->w[i] : 1.0);",
     "double Qw = dep->q[0] * (dep->w ? dep->w[i] : 1.0);"),
    ("dep_weight_dropped", "double Qw = dep->q[(flags[i] >> 6) & 3] * (dep->w ? dep->w[i] : 1.0);",
     "double Qw = dep->q[(flags[i] >> 6) & 3];"),
    ("vstep_gca_last_iterate", "for (int k = 0; k < 3; ++k) d->vstep[k] = 0.5 * (Vn[k] + Vk[k]);",
     "for (int k = 0; k < 3; ++k) d->vstep[k] = Vk[k];"),
    ("vstep_boris_gamma_dropped", "for (int d = 0; d < 3; ++d) v[d] = u[d] / g;",
     "for (int d = 0; d < 3; ++d) v[d] = u[d];"),
    ("dep_frozen_deposits", "if (q[7] < 0.0) continue;   /* frozen: no step, no current */",
     "/* frozen particles not skipped */"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS_DEP, ids=[c[0] for c in MUTANTS_DEP])
def test_deposit_pins_catch_planted_mistake(name, old, new, tmp_path):
    lib = _build_mutant(str(tmp_path), SRC, old, new)
    env = dict(os.environ, GCB_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_deposit_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1, f"pins did not catch mutant {name}:\n{r.stdout[-2000:]}"


# mistakes in the mirror terms (option mirror)
MUTANTS_MIRROR = [
    ("mirror_drift_sign", "for (int k = 0; k < 3; ++k) vg[k] = pref * bxa[k];",
     "for (int k = 0; k < 3; ++k) vg[k] = -pref * bxa[k];"),
    ("mirror_drift_kappa_dropped",
     "for (int k = 0; k < 3; ++k) a[k] = mu / Gam * P->gB[k] / P->kappa;",
     "for (int k = 0; k < 3; ++k) a[k] = mu / Gam * P->gB[k];"),
    ("mirror_drift_gamma_dropped",
     "for (int k = 0; k < 3; ++k) a[k] = mu / Gam * P->gB[k] / P->kappa;",
     "for (int k = 0; k < 3; ++k) a[k] = mu * P->gB[k] / P->kappa;"),
    ("mirror_force_sign", "return -mu / G0 * dot3(P->b, P->gB) / P->kappa;",
     "return mu / G0 * dot3(P->b, P->gB) / P->kappa;"),
    ("mirror_force_gamma_dropped", "return -mu / G0 * dot3(P->b, P->gB) / P->kappa;",
     "return -mu * dot3(P->b, P->gB) / P->kappa;"),
    ("mirror_force_not_in_flat_scheme", "*upar_new = upar + qm * dt * P->Epar + fm;",
     "*upar_new = upar + qm * dt * P->Epar;"),
    ("mirror_gradB_is_gradBz", "P->gB[i] = bdB;", "P->gB[i] = P->dB[i][2] + P->dB[i][0];"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS_MIRROR, ids=[c[0] for c in MUTANTS_MIRROR])
def test_mirror_pins_catch_planted_mistake(name, old, new, tmp_path):
    lib = _build_mutant(str(tmp_path), SRC, old, new)
    env = dict(os.environ, GCB_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_mirror_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1, f"pins did not catch mutant {name}:\n{r.stdout[-2000:]}"


# mistakes in the dual-number gradient oracle: its arithmetic on derivatives
# and the seeding of the directions
SRC_GRAD = os.path.join(ROOT, "oracle", "gcb_oracle_grad.cpp")
MUTANTS_GRAD = [
    ("dual_sqrt_half", "r.d[k] = a.d[k] / (2.0 * s);", "r.d[k] = a.d[k] / s;"),
    ("dual_quotient_sign", "r.d[k] = (a.d[k] - q * b.d[k]) / b.v;",
     "r.d[k] = (a.d[k] + q * b.d[k]) / b.v;"),
    ("dual_product_term", "r.d[k] = a.d[k] * b.v + a.v * b.d[k];", "r.d[k] = a.d[k] * b.v;"),
    ("mode_seed_dropped", "FN.d[m] = pm[m];", "FN.d[m] = 0.0;"),
    ("momentum_seed_index", "ui[k].d[DU0 + k] = 1.0;", "ui[k].d[DU0] = 1.0;"),
    ("weights_position_free", "t[d] = s - fl;", "t[d] = Dual(val(s) - fl);"),
]


def _build_grad_mutant(tmp, old, new):
    text = open(SRC_GRAD).read()
    assert text.count(old) == 1, old
    with open(os.path.join(tmp, "gcb_oracle_grad.cpp"), "w") as fh:
        fh.write(text.replace(old, new))
    shutil.copy(HDR, os.path.join(tmp, "gcb_oracle.h"))
    lib = os.path.join(tmp, "libmutgrad.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-o", lib,
                    os.path.join(tmp, "gcb_oracle_grad.cpp"), "-lm"], check=True)
    return lib


@pytest.mark.parametrize("name,old,new", MUTANTS_GRAD, ids=[c[0] for c in MUTANTS_GRAD])
def test_grad_pins_catch_planted_mistake(name, old, new, tmp_path):
    lib = _build_grad_mutant(str(tmp_path), old, new)
    env = dict(os.environ, GCB_ORACLE_GRAD_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_grad_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1, f"pins did not catch mutant {name}:\n{r.stdout[-2000:]}"


def _build_mutant(tmp, src_path, old, new):
    names = {SRC: "gcb_oracle.c", SRC_KS: "gcb_oracle_ks.c"}
    for path, name in names.items():
        text = open(path).read()
        if path == src_path:
            assert text.count(old) == 1, old
            text = text.replace(old, new)
        with open(os.path.join(tmp, name), "w") as fh:
            fh.write(text)
    shutil.copy(HDR, os.path.join(tmp, "gcb_oracle.h"))
    lib = os.path.join(tmp, "libmut.so")
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", lib,
                    os.path.join(tmp, "gcb_oracle.c"), os.path.join(tmp, "gcb_oracle_ks.c"),
                    "-lm"], check=True)
    return lib


CASES = [(n, SRC, o, w) for n, o, w in MUTANTS] + [(n, SRC_KS, o, w) for n, o, w in MUTANTS_KS]


@pytest.mark.parametrize("name,src,old,new", CASES, ids=[c[0] for c in CASES])
def test_pins_catch_planted_mistake(name, src, old, new, tmp_path):
    lib = _build_mutant(str(tmp_path), src, old, new)
    env = dict(os.environ, GCB_ORACLE_LIB=lib)
    pins = "test_oracle_pins.py" if src == SRC else "test_oracle_ks_pins.py"
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", pins)],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1, f"pins did not catch mutant {name}:\n{r.stdout[-2000:]}"
