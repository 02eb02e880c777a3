"""The oracle's pins catch plausible mistakes (CPU, no GPU).

Each mutant is a copy of the oracle with one planted mistake of the kind a restatement of Secs. 2-3 could make: a
dropped term, a wrong sign, a transposed component, a wrong index or weight.  Mutants of oracle/molc_oracle.cpp
are compiled on their own and the pin suites (tests/test_oracle_pins.py, tests/test_golden_single_ray.py) run
against them in a subprocess (MOLC_ORACLE_LIB); mutants of its running error bound run against the bound's pins
(tests/test_error_bound.py); mutants of oracle/__init__.py (the closure and grey averages) run the pin suites
from a copied tree.  Each must fail at least one pin.  Control copies with no mistake, built and
run the same ways, must pass them all, so a failure is the mistake's and not the harness's.
"""
import os
import platform
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "molc_oracle.cpp")
PINS = ["tests/test_oracle_pins.py", "tests/test_golden_single_ray.py"]

# name -> (exact text in the oracle, the mistaken text)
MUTANTS = {
    # Eq. 11: the backward-Euler source without its time term I^{n-1}/(c dt)
    "source_without_time_term": ("const R Q = kap_i * B_i + inv_cdt * Iprev;", "const R Q = kap_i * B_i;"),
    # Eq. 11: kappa~ without 1/(c dt)
    "kappa_tilde_without_time_term": ("const R kt = kap_i + inv_cdt;", "const R kt = kap_i;"),
    # Eq. 13: the optical thickness multiplied by sin(zeta) instead of divided
    "tau_times_sin_zeta": ("const R tau = kt * r.len[s] / sinz;", "const R tau = kt * r.len[s] * sinz;"),
    # Eq. 12: the weights of the segment average swapped
    "alpha_swapped": ("const R Ibar = alpha * I + (R(1) - alpha) * Iout;",
                      "const R Ibar = (R(1) - alpha) * I + alpha * Iout;"),
    # Eq. 15: F_x accumulated with the y component of Omega
    "Fx_with_Omega_y": ("a[MOM_FX * ncell + i] += wA * Ox * Ibar;", "a[MOM_FX * ncell + i] += wA * Oy * Ibar;"),
    # Eq. 15: N_xy accumulated with Omega_x Omega_x
    "Nxy_with_Omega_x_squared": ("a[MOM_NXY * ncell + i] += wA * Ox * Oy * Ibar;",
                                 "a[MOM_NXY * ncell + i] += wA * Ox * Ox * Ibar;"),
    # Eq. 14: the segment area without the characteristic's width
    "area_without_width": ("ray.area.push_back((b - a) * width);", "ray.area.push_back((b - a));"),
    # boundary condition: the incoming intensity of every characteristic read from the first edge
    "boundary_from_one_edge": ("R I = bnd[r.entry * G + gsel];", "R I = bnd[gsel];"),
    # the in-plane direction with the sign of its y component flipped
    "Omega_y_sign": ("const R Ox = sinz * d.dx, Oy = sinz * d.dy;", "const R Ox = sinz * d.dx, Oy = -sinz * d.dy;"),
    # Eq. 14 with MOLC_AREA_RENORM's reading: the per-(cell, pair) renormalisation of the areas skipped
    "renormalisation_skipped": ("if (g.renorm) {", "if (false && g.renorm) {"),
    # Eq. 12: 1 - e^-tau written as e^tau - 1
    "one_minus_e_sign": ("const R one_m_e = -Fn<R>::expm1(-tau);", "const R one_m_e = Fn<R>::expm1(tau);"),
    # the zz component of the Eddington tensor with mu once instead of squared
    "Nzz_mu_once": ("a[MOM_NZZ * ncell + i] += wA * mu * mu * Ibar;", "a[MOM_NZZ * ncell + i] += wA * mu * Ibar;"),
    # Eq. 16: the face sums take the intensity leaving the segment instead of the one entering at its upwind face
    "face_downstream_intensity": ("fa[MOM_D * nf + f] += ww * I;", "fa[MOM_D * nf + f] += ww * Iout;"),
    # Eq. 16: the face F_x with the y component of Omega
    "face_Fx_with_Omega_y": ("fa[MOM_FX * nf + f] += ww * Ox * I;", "fa[MOM_FX * nf + f] += ww * Oy * I;"),
    # Sec. 3 grid: the uniform layout's characteristics at the band edges instead of their centres
    "offsets_not_centred": ("t.push_back(tmin + ((double)k + 0.5) * wk);", "t.push_back(tmin + (double)k * wk);"),
    # Sec. 3 grid: the paper layout's bands split into one more piece at a time instead of halved
    "bands_not_halved": ("while (gap / (double)pieces > g.spacing) pieces *= 2;",
                         "while (gap / (double)pieces > g.spacing) pieces += 1;"),
    # Eq. 11: 1/(c dt) with c left out
    "time_term_without_c": ("const R inv_cdt = R(1) / (R(c) * R(dt));", "const R inv_cdt = R(1) / R(dt);"),
    # Eq. 13: alpha with the sign of its second term flipped
    "alpha_sign": ("const R alpha = R(1) / tau - e / one_m_e;", "const R alpha = R(1) / tau + e / one_m_e;"),
    # Eq. 12: the source term Q not divided by kappa~
    "source_not_over_kappa_tilde": ("const R Iout = I * e + (Q / kt) * one_m_e;",
                                    "const R Iout = I * e + Q * one_m_e;"),
    # boundary condition: a characteristic entering through a vertical edge given the opposite edge's intensity
    "entry_edge_x_swapped": ("ray.entry = xedge ? (dx > R(0) ? EDGE_L : EDGE_R)",
                             "ray.entry = xedge ? (dx > R(0) ? EDGE_R : EDGE_L)"),
    # Eq. 11: a previous state given as deviations from B used without adding B back
    "previous_deviation_without_B": ("const R Iprev = I_prev ? (prev_dev ? B_i + R(I_prev[seg * Gsub + gi])",
                                     "const R Iprev = I_prev ? (prev_dev ? R(I_prev[seg * Gsub + gi])"),
    # Eq. 13: sin(zeta) from mu instead of mu^2
    "sin_zeta_mu_not_squared": ("const R sinz = Fn<R>::sqrt(R(1) - mu * mu);",
                                "const R sinz = Fn<R>::sqrt(R(1) - mu);"),
    # Eq. 11: the stored I^{n-1} the outgoing intensity instead of the segment average
    "state_stores_outgoing_intensity": (
        "if (I_new) I_new[seg * Gsub + gi] = store_dev ? (double)(Ibar - B_i) : (double)Ibar;",
        "if (I_new) I_new[seg * Gsub + gi] = store_dev ? (double)(Iout - B_i) : (double)Iout;"),
    # Eq. 15: the cell volume formed with the x side twice (wrong for cells that are not square)
    "cell_volume_x_side_twice": ("const R V = R(g->lx / g->nx) * R(g->ly / g->ny);",
                                 "const R V = R(g->lx / g->nx) * R(g->lx / g->nx);"),
    # Eq. 15: N_yy accumulated with Omega_x Omega_y
    "Nyy_with_Omega_x": ("a[MOM_NYY * ncell + i] += wA * Oy * Oy * Ibar;",
                         "a[MOM_NYY * ncell + i] += wA * Ox * Oy * Ibar;"),
    # Sec. 2: E without its factor 1/c
    "E_without_1_over_c": ("const R scale = q == MOM_D ? R(1) / (R(c) * V) : R(1) / V;",
                           "const R scale = R(1) / V;"),
    # Eq. 14 with MOLC_AREA_RENORM's reading: the renormalisation factor inverted
    "renormalisation_inverted": ("r.area[s] = r.area[s] * (V / sum[r.cell[s]]);",
                                 "r.area[s] = r.area[s] * (sum[r.cell[s]] / V);"),
    # Sec. 3 grid: the uniform layout's widths from n + 1 bands for n characteristics
    "uniform_width_n_plus_1": ("double wk = Lp / (double)n;", "double wk = Lp / (double)(n + 1);"),
    # boundary condition: a characteristic entering through a horizontal edge given the opposite edge's intensity
    "entry_edge_y_swapped": ("(dy > R(0) ? EDGE_B : EDGE_T);", "(dy > R(0) ? EDGE_T : EDGE_B);"),
    # Eq. 11: the emission kappa B formed with the previous intensity instead of B
    "emission_with_previous_intensity": ("const R Q = kap_i * B_i + inv_cdt * Iprev;",
                                         "const R Q = kap_i * Iprev + inv_cdt * Iprev;"),
    # Eq. 16: the face averages over the other side's length
    "face_length_swapped": ("const R len = f < nxf ? hy : hx;", "const R len = f < nxf ? hx : hy;"),
    # Eq. 16: N_xy of the faces with Omega_x^2
    "face_Nxy_with_Omega_x_squared": ("fa[MOM_NXY * nf + f] += ww * Ox * Oy * I;",
                                      "fa[MOM_NXY * nf + f] += ww * Ox * Ox * I;"),
    # Sec. 3 grid: cell index i = ix ny + iy instead of iy nx + ix
    "cell_index_transposed": ("ray.cell.push_back((int)(iy * g.nx + ix));",
                              "ray.cell.push_back((int)(ix * g.ny + iy));"),
    # Sec. 3 grid: a segment given to the cell of its start instead of the cell holding it
    "segment_cell_at_its_start": ("R m = R(0.5) * (a + b);", "R m = a;"),
    # Sec. 3 grid: the uniform layout's count rounded down (bands wider than the spacing)
    "uniform_count_rounded_down": ("long n = (long)std::ceil(Lp / g.spacing - 1e-9);",
                                   "long n = (long)std::floor(Lp / g.spacing);"),
    # Sec. 3 grid: the paper layout's vertices projected on the wrong normal
    "paper_projection_sign": ("auto proj = [&](double x, double y) { return -dy * x + dx * y; };",
                              "auto proj = [&](double x, double y) { return dy * x + dx * y; };"),
    # Sec. 3 grid: coincident vertex projections not merged (zero-width characteristics)
    "paper_projections_not_merged": ("if (u.empty() || x - u.back() > merge) u.push_back(x);", "u.push_back(x);"),
    # Eq. 16: a crossing in x given the face on the lower side of the step
    "upwind_x_face_lower_index": (
        "f = px != ix ? iy * (g.nx + 1) + std::max(px, ix) : nxf + std::max(py, iy) * g.nx + ix;",
        "f = px != ix ? iy * (g.nx + 1) + std::min(px, ix) : nxf + std::max(py, iy) * g.nx + ix;"),
    # Eq. 16: characteristics entering through the right edge given the left edge's faces
    "entry_face_right_as_left": ("ray.entry == EDGE_R ? iy * (g.nx + 1) + g.nx", "ray.entry == EDGE_R ? iy * (g.nx + 1)"),
}

# mistakes in the oracle's running error bound (oracle_errmodel) that make the bound too small, run against
# its pins (tests/test_error_bound.py: emulations of the paths' arithmetic must stay within it)
PINS_ERR = ["tests/test_error_bound.py"]
ERR_MUTANTS = {
    # the error a segment average inherits from the intensity entering the segment left out
    "bar_without_carried_error": ("b.bar = E1 * eps_in + (1 - E1) * eps_d", "b.bar = (1 - E1) * eps_d"),
    # the entering intensity's error not transmitted to the outgoing one (thin segments)
    "out_without_incoming_error": ("const double out_thin = e * eps_in + om * eps_d",
                                   "const double out_thin = om * eps_d"),
    # the stored state's error not carried into the next step's source
    "state_error_not_carried": (
        "? u * (3 * std::fabs(dstate * rr) + 5 * std::fabs((Br - Bc) * rr) + std::fabs(dd)) + rr * eps_state",
        "? u * (3 * std::fabs(dstate * rr) + 5 * std::fabs((Br - Bc) * rr) + std::fabs(dd))"),
    # the error of the hardware 2^x approximation left out of e^-tau
    "ex2_error_ignored": ("const double rh = 3.5 * u * tau + em.e_exp;", "const double rh = 3.5 * u * tau;"),
    # the entering intensity's error not transmitted to the outgoing one (thick segments)
    "thick_out_without_incoming_error": ("const double out_thick = e * eps_in + om * eps_d",
                                         "const double out_thick = om * eps_d"),
    # the roundings of the FP32 moment sums left out of the cell bound
    "summation_term_dropped": ("ob[i] = (E + ksum * em->u * D + 8 * u64 * (D + P)) * scale;",
                               "ob[i] = (E + 8 * u64 * (D + P)) * scale;"),
    # the roundings of the FP32 cell table (the stored deviation and the B_ref step) left out of d
    "table_roundings_dropped": (
        "? u * (3 * std::fabs(dstate * rr) + 5 * std::fabs((Br - Bc) * rr) + std::fabs(dd)) + rr * eps_state",
        "? u * std::fabs(dd) + rr * eps_state"),
}

# the same for the oracle's Python part (oracle/__init__.py): name -> (exact text, the mistaken text)
PY_MUTANTS = {
    # Eq. 7: f_xy = N_xy / E, without c
    "closure_without_c": ("fxy = np.asarray(Nxy) / cE", "fxy = np.asarray(Nxy) / np.asarray(E)"),
    # Eq. 8 with u = f: the groups' factors averaged without the E weights
    "grey_eddington_unweighted": ("out.append(np.where(se > 0, (f * E).sum(0) / np.where(se > 0, se, 1.0), 0.0))",
                                  "out.append(np.where(se > 0, f.sum(0) / E.shape[0], 0.0))"),
    # Eq. 9: K_R weighted by the signed flux instead of |F|
    "KR_signed_flux": ("kE, kB, kx, ky = avg(E), avg(B), avg(np.abs(Fx)), avg(np.abs(Fy))",
                       "kE, kB, kx, ky = avg(E), avg(B), avg(Fx), avg(Fy)"),
    # Eq. 9: <kappa>_B weighted by E
    "kappa_B_weighted_by_E": ("kE, kB, kx, ky = avg(E), avg(B), avg(np.abs(Fx)), avg(np.abs(Fy))",
                              "kE, kB, kx, ky = avg(E), avg(E), avg(np.abs(Fx)), avg(np.abs(Fy))"),
    # Eq. 9: eta_x formed with K_R's y component
    "eta_x_with_KRy": ("ex = np.where(se > 0, ((kappa - kx) * Fx).sum(0) / safe, 0.0)",
                       "ex = np.where(se > 0, ((kappa - ky) * Fx).sum(0) / safe, 0.0)"),
    # Eq. 9: eta_x divided by the sum of B instead of the sum of E
    "eta_x_over_B": ("ex = np.where(se > 0, ((kappa - kx) * Fx).sum(0) / safe, 0.0)",
                     "ex = np.where(se > 0, ((kappa - kx) * Fx).sum(0) / np.where(B.sum(0) > 0, B.sum(0), 1.0), 0.0)"),
    # Eq. 9: K_R's y component weighted by |F_x|
    "KRy_with_Fx": ("kE, kB, kx, ky = avg(E), avg(B), avg(np.abs(Fx)), avg(np.abs(Fy))",
                    "kE, kB, kx, ky = avg(E), avg(B), avg(np.abs(Fx)), avg(np.abs(Fx))"),
    # Eq. 7: f_yy formed from N_xx
    "closure_fyy_from_Nxx": ("fyy = np.asarray(Nyy) / cE", "fyy = np.asarray(Nxx) / cE"),
}


def _compile(src_text, out_dir, name):
    cpp = os.path.join(out_dir, name + ".cpp")
    so = os.path.join(out_dir, name + ".so")
    with open(cpp, "w") as f:
        f.write(src_text)
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-pthread", "-o", so, cpp]
    if platform.machine() in ("x86_64", "AMD64"):
        cmd.append("-lquadmath")
    subprocess.run(cmd, check=True, capture_output=True)
    return so


def _run_pins(so, root=ROOT, suites=PINS):
    env = dict(os.environ, MOLC_ORACLE_LIB=so)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *suites], cwd=root,
                       env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-2000:]


def _py_tree(py_text, out_dir, name):
    """A copy of what the pin suites import (tests/, synth/, the oracle package) with this oracle/__init__.py."""
    root = os.path.join(out_dir, name)
    ignore = shutil.ignore_patterns("__pycache__", "_build")
    for sub in ("tests", "synth"):
        shutil.copytree(os.path.join(ROOT, sub), os.path.join(root, sub), ignore=ignore)
    os.makedirs(os.path.join(root, "oracle"))
    shutil.copy(SRC, os.path.join(root, "oracle"))
    with open(os.path.join(root, "oracle", "__init__.py"), "w") as f:
        f.write(py_text)
    return root


@pytest.mark.timeout(900)
def test_every_planted_mistake_fails_a_pin(tmp_path):
    src = open(SRC).read()
    variants = {"control": src}
    suites = {"control": PINS + PINS_ERR}
    for table, pins in ((MUTANTS, PINS), (ERR_MUTANTS, PINS_ERR)):
        for name, (old, new) in table.items():
            assert src.count(old) == 1, name       # the text to mutate is where the pins expect it, once
            variants[name] = src.replace(old, new)
            suites[name] = pins
    workers = max(1, min(len(variants), os.cpu_count() or 1))
    with ThreadPoolExecutor(workers) as ex:
        libs = dict(zip(variants, ex.map(lambda kv: _compile(kv[1], str(tmp_path), kv[0]), variants.items())))
        results = dict(zip(libs, ex.map(lambda n: _run_pins(libs[n], suites=suites[n]), libs)))
        # the Python mutants run against the control's library from trees of their own
        py_src = open(os.path.join(ROOT, "oracle", "__init__.py")).read()
        trees = {}
        for name, (old, new) in PY_MUTANTS.items():
            assert py_src.count(old) == 1, name
            trees[name] = _py_tree(py_src.replace(old, new), str(tmp_path), name)
        trees["py_control"] = _py_tree(py_src, str(tmp_path), "py_control")
        results.update(zip(trees, ex.map(lambda r: _run_pins(libs["control"], r), trees.values())))
    for control in ("control", "py_control"):
        rc, out = results.pop(control)
        assert rc == 0, f"the unmutated oracle ({control}) must pass the pins:\n" + out
    survivors = [name for name, (rc, _) in results.items() if rc == 0]
    assert not survivors, f"mistakes no pin catches: {survivors}"
    # the pins failed (exit 1), they did not error out (exit 2+: collection or internal errors)
    assert all(rc == 1 for rc, _ in results.values()), {n: r[0] for n, r in results.items()}
