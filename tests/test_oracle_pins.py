"""Pins for the oracle against closed forms, invariants, exact geometry and brute force (no GPU).

Each test is chosen so that a plausible slip in the oracle (a dropped term in Q, a wrong sign in alpha, a
swapped Omega component, a wrong area or a wrong entry edge) fails at least one of them.
"""
import math

import numpy as np
import pytest

import bruteforce as bf
import oracle
import synth


def make_geom(nx, ny, lx, ly, quad, spacing, layout=0, renorm=1):
    return oracle.Geometry(nx, ny, lx, ly, quad.mu, quad.cos_phi, quad.sin_phi, quad.w, spacing, layout, renorm)


def homogeneous(G, ncell, kap, Bv):
    return np.tile(np.asarray(kap, float)[:, None], (1, ncell)), np.tile(np.asarray(Bv, float)[:, None], (1, ncell))


# ------------------------------------------------------------------------------------------------------------
# 1. Equilibrium: homogeneous medium, I^{n-1} = B and every edge driven at B  =>  Ibar = B everywhere,
#    E = 4 pi B / c, F = 0, f = diag(1/3, 1/3, 1/3).  Exact: I_in = Q/kappa~ gives I_out = I_in (Eq. 12).
# ------------------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("layout", [0, 1])
def test_equilibrium_closed_form(layout):
    q = synth.product_quadrature(2, 8)
    geom = make_geom(4, 3, 2.0, 1.5, q, 0.2, layout=layout)
    G = 3
    kap = [0.3, 7.0, 2.0e4]
    Bv = [1.0, 0.25, 3.0e-3]
    kappa, B = homogeneous(G, geom.ncell, kap, Bv)
    bnd = np.tile(np.asarray(Bv)[None, :], (4, 1))
    c, dt = 29.98, 2e-3
    r = oracle.sweep(geom, kappa, B, c, dt, bnd, precision="quad")
    assert np.max(np.abs(r["I"] / np.tile(Bv, (r["I"].shape[0], 1)) - 1)) < 1e-15
    for g in range(G):
        cE = c * r["E"][g]
        assert np.max(np.abs(cE / (4 * math.pi * Bv[g]) - 1)) < 1e-14
        assert np.max(np.abs(r["Fx"][g]) / cE) < 1e-14 and np.max(np.abs(r["Fy"][g]) / cE) < 1e-14
        for k in ("Nxx", "Nyy", "Nzz"):
            assert np.max(np.abs(r[k][g] / cE - 1 / 3)) < 1e-14
        assert np.max(np.abs(r["Nxy"][g]) / cE) < 1e-14


# ------------------------------------------------------------------------------------------------------------
# 2. Time term: homogeneous medium with a uniform previous intensity J != B and every edge driven at
#    S = (kappa B + J/(c dt)) / kappa~  =>  Ibar = S on every segment (the backward-Euler source of Eq. 11).
# ------------------------------------------------------------------------------------------------------------
def test_time_term_closed_form():
    q = synth.product_quadrature(3, 12)
    geom = make_geom(5, 5, 1.0, 1.0, q, 0.05)
    kap, Bv, J = np.array([0.5, 40.0]), np.array([2.0, 0.1]), np.array([7.0, 3.0])
    c, dt = 1.0, 0.25
    kt = kap + 1 / (c * dt)
    S = (kap * Bv + J / (c * dt)) / kt
    kappa, B = homogeneous(2, geom.ncell, kap, Bv)
    _, ns = oracle.counts(geom)
    I_prev = np.tile(J, (ns, 1))
    bnd = np.tile(S[None, :], (4, 1))
    r = oracle.sweep(geom, kappa, B, c, dt, bnd, I_prev=I_prev, precision="quad")
    assert np.max(np.abs(r["I"] / S[None, :] - 1)) < 1e-15
    assert np.max(np.abs(c * r["E"] / (4 * math.pi * S[:, None]) - 1)) < 1e-14


# ------------------------------------------------------------------------------------------------------------
# 3. Track geometry against independent re-derivation: offsets from the written rule, lengths by clipping the
#    line against every cell box, entry edges, and (paper layout) A = l w equal to the exact band-cell area.
# ------------------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("layout", [0, 1])
@pytest.mark.parametrize("nx,ny,lx,ly,sp", [(3, 3, 3.0, 3.0, 0.45), (5, 4, 2.5, 1.0, 0.13), (2, 1, 1.0, 0.7, 0.3),
                                             (2, 2, 2.0, 2.0, 0.04)])   # bands halved several times
def test_tracks_match_brute_force(layout, nx, ny, lx, ly, sp):
    q = synth.product_quadrature(1, 12)
    geom = make_geom(nx, ny, lx, ly, q, sp, layout=layout, renorm=0)
    tr = oracle.tracks(geom, "quad")
    hx, hy = lx / nx, ly / ny
    for m in range(q.n):
        c, s = bf.unit(q.cos_phi[m], q.sin_phi[m])
        ts, ws = (bf.uniform_offsets(lx, ly, c, s, sp) if layout == 0 else bf.paper_offsets(nx, ny, lx, ly, c, s, sp))
        r0, r1 = tr["dir_ray_off"][m], tr["dir_ray_off"][m + 1]
        assert r1 - r0 == len(ts)
        for k in range(len(ts)):
            ri = r0 + k
            segs, edge = bf.ray_segments(nx, ny, lx, ly, c, s, ts[k])
            a, b = tr["ray_seg_off"][ri], tr["ray_seg_off"][ri + 1]
            assert tr["width"][ri] == pytest.approx(ws[k], rel=1e-13)
            assert tr["entry"][ri] == edge
            assert list(tr["cell"][a:b]) == [q_[0] for q_ in segs]
            assert np.allclose(tr["len"][a:b], [q_[1] for q_ in segs], rtol=1e-12, atol=1e-13 * max(hx, hy))
            if layout == 1:
                for cell, A in zip(tr["cell"][a:b], tr["area"][a:b]):
                    ix, iy = cell % nx, cell // nx
                    exact = bf.band_cell_area(ts[k], ws[k], c, s, ix * hx, (ix + 1) * hx, iy * hy, (iy + 1) * hy)
                    assert A == pytest.approx(exact, rel=1e-11, abs=1e-14)
        if layout == 1:
            # the bands tile the domain and contain no vertex: per cell and direction, sum A = V exactly
            tot = np.zeros(nx * ny)
            a, b = tr["ray_seg_off"][r0], tr["ray_seg_off"][r1]
            np.add.at(tot, tr["cell"][a:b], tr["area"][a:b])
            assert np.max(np.abs(tot / (hx * hy) - 1)) < 1e-13


def test_renormalised_areas_sum_to_cell_volume():
    q = synth.product_quadrature(1, 16)
    geom = make_geom(8, 8, 6.0, 6.0, q, 6.0 / 8 / 2)
    tr = oracle.tracks(geom, "quad")
    V = (6.0 / 8) ** 2
    for m in range(q.n):
        a, b = tr["ray_seg_off"][tr["dir_ray_off"][m]], tr["ray_seg_off"][tr["dir_ray_off"][m + 1]]
        tot = np.zeros(64)
        np.add.at(tot, tr["cell"][a:b], tr["area"][a:b])
        assert np.max(np.abs(tot / V - 1)) < 1e-14


# ------------------------------------------------------------------------------------------------------------
# 4. Brute force on tiny grids: independent geometry + RK4 integration of dI/ds + kappa~ I = Q per segment,
#    cell moments assembled here from the brute-force segment averages.
# ------------------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("nx,ny,naz,npol", [(1, 1, 4, 1), (2, 1, 4, 2), (2, 2, 8, 1), (2, 2, 4, 2)])
def test_brute_force_tiny_grids(nx, ny, naz, npol):
    rng = np.random.default_rng(nx * 100 + ny * 10 + naz + npol)
    lx, ly, sp = 1.0, 0.8, 0.35
    q = synth.product_quadrature(npol, naz)
    geom = make_geom(nx, ny, lx, ly, q, sp)
    G, ncell = 2, nx * ny
    kappa = rng.uniform(0.2, 3.0, (G, ncell))
    B = rng.uniform(0.1, 1.0, (G, ncell))
    bnd = rng.uniform(0.0, 2.0, (4, G))
    c, dt = 1.0, 0.5
    _, ns = oracle.counts(geom)
    I_prev = rng.uniform(0.0, 1.5, (ns, G))
    r = oracle.sweep(geom, kappa, B, c, dt, bnd, I_prev=I_prev, precision="quad", want_exit=True)
    hx, hy = lx / nx, ly / ny
    V = hx * hy
    mom = {k: np.zeros((G, ncell)) for k in ("D", "Fx", "Fy", "Nxx", "Nxy", "Nyy")}
    seg = 0
    ray = 0
    for m in range(q.n):
        cphi, sphi = bf.unit(q.cos_phi[m], q.sin_phi[m])
        sinz = math.sqrt(1 - q.mu[m] ** 2)
        Ox, Oy = sinz * cphi, sinz * sphi
        ts, ws = bf.uniform_offsets(lx, ly, cphi, sphi, sp)
        rays = [bf.ray_segments(nx, ny, lx, ly, cphi, sphi, t) for t in ts]
        asum = np.zeros(ncell)
        for (segs, _), w in zip(rays, ws):
            for cell, L, _u in segs:
                asum[cell] += L * w
        for (segs, edge), w in zip(rays, ws):
            I = bnd[edge].copy()
            for cell, L, _u in segs:
                A = L * w * V / asum[cell]
                for g in range(G):
                    kt = kappa[g, cell] + 1 / (c * dt)
                    Q = kappa[g, cell] * B[g, cell] + I_prev[seg, g] / (c * dt)
                    Iout, Ibar = bf.rk4_segment(I[g], Q, kt, L / sinz)
                    assert r["I"][seg, g] == pytest.approx(Ibar, rel=1e-9)
                    wA = q.w[m] * A
                    mom["D"][g, cell] += wA * Ibar
                    mom["Fx"][g, cell] += wA * Ox * Ibar
                    mom["Fy"][g, cell] += wA * Oy * Ibar
                    mom["Nxx"][g, cell] += wA * Ox * Ox * Ibar
                    mom["Nxy"][g, cell] += wA * Ox * Oy * Ibar
                    mom["Nyy"][g, cell] += wA * Oy * Oy * Ibar
                    I[g] = Iout
                seg += 1
            assert np.allclose(r["I_exit"][ray], I, rtol=1e-9)
            ray += 1
    assert np.allclose(r["E"], mom["D"] / (c * V), rtol=1e-9)
    scale = np.abs(mom["D"]) / V
    for k in ("Fx", "Fy", "Nxx", "Nxy", "Nyy"):
        assert np.all(np.abs(r[k] - mom[k] / V) <= 1e-9 * scale)


# ------------------------------------------------------------------------------------------------------------
# 5. Per-ray discrete balance: I_in - I_out + sum_s (Q - kappa~ Ibar) l / sin(zeta) = 0 for every
#    characteristic, direction and group; the identity holds only if Ibar is the exact segment average.
# ------------------------------------------------------------------------------------------------------------
def test_per_ray_balance_and_global_balance():
    wl = synth.WORKLOADS["fc16_g4_d32"]
    d = wl.inputs(seed=1)
    geom = oracle.Geometry.from_workload(wl)
    tr = oracle.tracks(geom, "quad")
    r = oracle.sweep(geom, d["kappa"], d["B"], d["c"], d["dt"], d["bnd"], precision="quad", want_exit=True)
    q = d["quad"]
    inv = 1 / (d["c"] * d["dt"])
    G = d["kappa"].shape[0]
    worst = 0.0
    lhs_glob = np.zeros(G)
    rhs_glob = np.zeros(G)
    for m in range(q.n):
        sinz = math.sqrt(1 - q.mu[m] ** 2)
        for ri in range(tr["dir_ray_off"][m], tr["dir_ray_off"][m + 1]):
            a, b = tr["ray_seg_off"][ri], tr["ray_seg_off"][ri + 1]
            cells = tr["cell"][a:b]
            L = tr["len"][a:b] / sinz
            kt = d["kappa"][:, cells] + inv
            Q = d["kappa"][:, cells] * d["B"][:, cells] + inv * d["B"][:, cells]
            Ib = r["I"][a:b].T
            I_in = d["bnd"][tr["entry"][ri]]
            I_out = r["I_exit"][ri]
            terms = np.abs(I_in) + np.abs(I_out) + (np.abs(Q * L) + np.abs(kt * Ib * L)).sum(axis=1)
            res = I_in - I_out + ((Q - kt * Ib) * L).sum(axis=1)
            ok = terms > 0
            assert np.all(res[~ok] == 0)
            if ok.any():
                worst = max(worst, float(np.max(np.abs(res[ok]) / terms[ok])))
            lhs_glob += q.w[m] * sinz * tr["width"][ri] * (I_in - I_out)
    assert worst < 1e-13
    # Global balance: weighted net inflow = sum over cells of (absorption - source), both from the moments.
    # With renormalised areas the cell sums use A, so compare against the moments assembled from the tracks.
    for m in range(q.n):
        sinz = math.sqrt(1 - q.mu[m] ** 2)
        a, b = tr["ray_seg_off"][tr["dir_ray_off"][m]], tr["ray_seg_off"][tr["dir_ray_off"][m + 1]]
        cells = tr["cell"][a:b]
        wl_ = tr["len"][a:b] * np.repeat(tr["width"][tr["dir_ray_off"][m]:tr["dir_ray_off"][m + 1]],
                                         np.diff(tr["ray_seg_off"][tr["dir_ray_off"][m]:tr["dir_ray_off"][m + 1] + 1]))
        kt = d["kappa"][:, cells] + inv
        Q = d["kappa"][:, cells] * d["B"][:, cells] + inv * d["B"][:, cells]
        rhs_glob += q.w[m] * ((kt * r["I"][a:b].T - Q) * wl_).sum(axis=1)
    assert np.allclose(lhs_glob, rhs_glob, rtol=1e-12)


# ------------------------------------------------------------------------------------------------------------
# 6. Symmetry: rotating the problem by 90 degrees (left-driven -> bottom-driven) rotates (E, F, N); reflecting
#    y -> -y flips F_y and N_xy.  The quadrature maps onto itself exactly; the characteristic grid is defined by
#    double evaluation of the offsets, so it maps onto itself only to double rounding (~1e-16 L shifts of the
#    lines), which bounds the agreement (1e-13 of c E).
# ------------------------------------------------------------------------------------------------------------
def _rot_cells(a, n):
    # field [.., iy*n+ix] of the original -> field of the problem rotated by +90 deg about the centre:
    # (x, y) -> (L - y, x), i.e. new (ix', iy') = (n-1-iy, ix)
    a = a.reshape(a.shape[:-1] + (n, n))
    out = np.empty_like(a)
    for iy in range(n):
        for ix in range(n):
            out[..., ix, n - 1 - iy] = a[..., iy, ix]
    return out.reshape(a.shape[:-2] + (n * n,))


def test_rotation_and_reflection_symmetry():
    wl = synth.Workload("sym", 8, 8, 6.0, 3, 0.01, 10.0, 2, 8, 2, 1)
    d = wl.inputs(seed=5)
    geom = oracle.Geometry.from_workload(wl)
    base = oracle.sweep(geom, d["kappa"], d["B"], d["c"], d["dt"], d["bnd"], precision="quad", want_I=False)
    n = wl.nx
    # rotation: left edge -> bottom edge
    bnd_r = np.zeros_like(d["bnd"])
    bnd_r[synth.EDGE_BOTTOM] = d["bnd"][synth.EDGE_LEFT]
    rot = oracle.sweep(geom, _rot_cells(d["kappa"], n), _rot_cells(d["B"], n), d["c"], d["dt"], bnd_r,
                       precision="quad", want_I=False)
    cE = _rot_cells(d["c"] * base["E"], n)
    # under (x,y) -> (-y,x): E -> E, (Fx,Fy) -> (-Fy, Fx), Nxx <-> Nyy, Nxy -> -Nxy
    exp = {"E": base["E"], "Fx": -base["Fy"], "Fy": base["Fx"], "Nxx": base["Nyy"], "Nyy": base["Nxx"],
           "Nxy": -base["Nxy"]}
    for k, v in exp.items():
        assert np.max(np.abs(rot[k] - _rot_cells(v, n)) / cE) < 1e-13, k
    for k, ak in (("Fx", "absFy"), ("Fy", "absFx"), ("Nxy", "absNxy")):   # signed moments, to their own scale
        scale = _rot_cells(base[ak], n)
        ok = scale > 0
        assert np.max(np.abs(rot[k] - _rot_cells(exp[k], n))[ok] / scale[ok]) < 1e-10, k
    # reflection y -> -y: the left-driven problem maps onto itself
    refl = lambda a: a.reshape(a.shape[:-1] + (n, n))[..., ::-1, :].reshape(a.shape)
    ref = oracle.sweep(geom, refl(d["kappa"]), refl(d["B"]), d["c"], d["dt"], d["bnd"], precision="quad",
                       want_I=False)
    cE = refl(d["c"] * base["E"])
    for k, sgn in (("E", 1), ("Fx", 1), ("Fy", -1), ("Nxx", 1), ("Nyy", 1), ("Nxy", -1)):
        assert np.max(np.abs(ref[k] - sgn * refl(base[k])) / cE) < 1e-13, k


# ------------------------------------------------------------------------------------------------------------
# 7. Closure trace: N_xx + N_yy + N_zz = c E (Omega is a unit vector), so f_zz = 1 - f_xx - f_yy.
# ------------------------------------------------------------------------------------------------------------
def test_closure_trace_and_bounds():
    wl = synth.WORKLOADS["fc16_g4_d32"]
    d = wl.inputs(seed=2)
    geom = oracle.Geometry.from_workload(wl)
    r = oracle.sweep(geom, d["kappa"], d["B"], d["c"], d["dt"], d["bnd"], precision="quad", want_I=False)
    cE = d["c"] * r["E"]
    assert np.max(np.abs((r["Nxx"] + r["Nyy"] + r["Nzz"]) / cE - 1)) < 1e-14
    fxx, fxy, fyy = oracle.closure(r["E"], r["Nxx"], r["Nxy"], r["Nyy"], d["c"])
    assert np.all((fxx >= 0) & (fxx <= 1) & (fyy >= 0) & (fyy <= 1) & (np.abs(fxy) <= 0.5))
    # f_zz = 1 - f_xx - f_yy is the zz factor of the separately summed N_zz (Omega_x^2 + Omega_y^2 + mu^2 = 1), in
    # cells where the field is far from isotropic in the plane as well as elsewhere
    assert np.max(np.abs(1 - fxx - fyy - r["Nzz"] / cE)) < 1e-14
    assert np.max(np.abs(fxx - fyy)) > 1e-3
    # the tensor is symmetric positive semidefinite: f_xx f_yy >= f_xy^2
    assert np.all(fxx * fyy - fxy * fxy >= -1e-14)


# ------------------------------------------------------------------------------------------------------------
# 8. Precision and bookkeeping: double agrees with binary128 to rounding on E; results do not depend on the
#    thread count; a group subset reproduces the corresponding slice; I^{n-1} = None means I^{n-1} = B.
# ------------------------------------------------------------------------------------------------------------
def test_double_vs_quad_and_bookkeeping():
    wl = synth.WORKLOADS["fc16_g4_d32"]
    d = wl.inputs(seed=0)
    geom = oracle.Geometry.from_workload(wl)
    rq = oracle.sweep(geom, d["kappa"], d["B"], d["c"], d["dt"], d["bnd"], precision="quad")
    rd1 = oracle.sweep(geom, d["kappa"], d["B"], d["c"], d["dt"], d["bnd"], precision="double", threads=1)
    rd8 = oracle.sweep(geom, d["kappa"], d["B"], d["c"], d["dt"], d["bnd"], precision="double", threads=8)
    for k in oracle.MOMENTS:
        assert np.array_equal(rd1[k], rd8[k])
    assert np.max(np.abs(rd1["E"] / rq["E"] - 1)) < 1e-12
    cE = d["c"] * rq["E"]
    for k in ("Fx", "Fy", "Nxy"):
        # the literal double sums lose ~1e-16 c E on signed moments (the reason the GPU paths sum deviations)
        assert np.max(np.abs(rd1[k] - rq[k]) / cE) < 1e-12
    sub = oracle.sweep(geom, d["kappa"], d["B"], d["c"], d["dt"], d["bnd"], groups=[2], precision="double")
    assert np.array_equal(sub["E"][0], rd1["E"][2]) and np.array_equal(sub["I"][:, 0], rd1["I"][:, 2])
    _, ns = oracle.counts(geom)
    tr = oracle.tracks(geom, "double")
    I_prev = d["B"].T[tr["cell"]]
    assert I_prev.shape == (ns, 4)
    rp = oracle.sweep(geom, d["kappa"], d["B"], d["c"], d["dt"], d["bnd"], I_prev=I_prev, precision="double")
    assert np.array_equal(rp["E"], rd1["E"])


def test_previous_state_as_deviations_is_the_same_state():
    """I^{n-1} of Eq. 11 carried as deviations from B of each segment's cell (the form the GPU paths store) is the
    same previous state as its segment averages: the stored deviations of a step are its averages minus B of the
    cell, and a second step, with B changed, gives the same moments from either form."""
    wl = synth.WORKLOADS["fc16_g4_d32"]
    d = wl.inputs(seed=0)
    geom = oracle.Geometry.from_workload(wl)
    cell = oracle.tracks(geom, "double")["cell"]
    args = (d["kappa"], d["B"], d["c"], d["dt"], d["bnd"])
    r1 = oracle.sweep(geom, *args, precision="quad")
    r1d = oracle.sweep(geom, *args, precision="quad", I_as_deviation=True)
    Bseg = d["B"].T[cell]
    scale = np.max(np.abs(r1["I"]))
    assert np.max(np.abs(r1d["I"] - (r1["I"] - Bseg))) < 1e-15 * scale
    B2 = d["B"] * np.linspace(0.5, 1.5, d["B"].shape[1])       # the temperature moved: B differs per cell
    args2 = (d["kappa"], B2, d["c"], d["dt"], d["bnd"])
    dev2 = r1["I"] - B2.T[cell]                                # the same averages, referred to this step's B
    ra = oracle.sweep(geom, *args2, I_prev=r1["I"], precision="quad")
    rd = oracle.sweep(geom, *args2, I_prev=dev2, I_prev_is_deviation=True, precision="quad")
    cE = d["c"] * ra["E"]
    for k in ("E", "Fx", "Fy", "Nxx", "Nxy", "Nyy"):
        ref = cE if k in ("Fx", "Fy", "Nxy") else np.abs(ra[k])
        assert np.max(np.abs(rd[k] - ra[k]) / ref) < 1e-13, k


def test_multistep_relaxes_towards_steady_state():
    # With fixed material and boundary the backward-Euler steps approach the steady solution: the change
    # between steps shrinks geometrically (factor <= 1/(1 + c dt kappa_min)).
    wl = synth.Workload("ms", 8, 8, 6.0, 2, 0.1, 10.0, 2, 8, 2, 1)
    d = wl.inputs(seed=0)
    geom = oracle.Geometry.from_workload(wl)
    I = None
    prev_E = None
    deltas = []
    for _ in range(4):
        r = oracle.sweep(geom, d["kappa"], d["B"], d["c"], d["dt"], d["bnd"], I_prev=I, precision="double")
        I = r["I"]
        if prev_E is not None:
            deltas.append(np.max(np.abs(r["E"] - prev_E)))
        prev_E = r["E"]
    kmin = d["kappa"].min()
    rate = 1 / (1 + d["c"] * d["dt"] * kmin)
    for a, b in zip(deltas[:-1], deltas[1:]):
        assert b <= a * rate * 1.0000001 + 1e-300


def test_grey_coefficients_special_cases():
    """Eqs. 8-9: one group, or an opacity the same in every group, gives every average = that opacity and
    eta = 0; a single nonzero flux group picks that group's opacity for K_R."""
    rng = np.random.default_rng(5)
    G, n = 5, 7
    E = rng.uniform(0.1, 1.0, (G, n))
    Fx, Fy = rng.uniform(-1, 1, (G, n)), rng.uniform(-1, 1, (G, n))
    B = rng.uniform(0.1, 1.0, (G, n))
    k1 = np.tile(rng.uniform(1, 5, (1, n)), (G, 1))
    r = oracle.grey_coefficients(E, Fx, Fy, k1, B)
    for name in ("kappa_E", "kappa_B", "KRx", "KRy"):
        assert np.allclose(r[name], k1[0], rtol=1e-15), name
    assert np.max(np.abs(r["eta_x"])) < 1e-15 * np.max(k1) * np.max(np.abs(Fx)) / E.sum(0).min() * G
    kg = rng.uniform(1, 5, (G, n))
    Fx1 = np.zeros((G, n))
    Fx1[2] = rng.uniform(0.5, 1.0, n)
    r = oracle.grey_coefficients(E, Fx1, Fy, kg, B)
    # (kappa |F| / |F| may differ from kappa by an ulp, and eta by that ulp times |F| / sum E)
    assert np.allclose(r["KRx"], kg[2], rtol=2e-16, atol=0)
    assert np.all(np.abs(r["eta_x"]) <= 4e-16 * kg[2] * Fx1[2] / E.sum(0))
    r1 = oracle.grey_coefficients(E[:1], Fx[:1], Fy[:1], kg[:1], B[:1])
    assert np.allclose(r1["kappa_E"], kg[0], rtol=2e-16, atol=0)
    assert np.all(np.abs(r1["eta_y"]) <= 4e-16 * kg[0] * np.abs(Fy[0]) / E[0])


def test_grey_coefficients_hand_worked():
    """Eqs. 8-9 on one cell with three groups whose B, E and flux spectra differ (worked by hand): kappa = (2, 5, 7),
    B only in group 0, E only in group 1, F_x = (1, 0, -3), F_y = (0, -2, 0).  <kappa>_B = 2, <kappa>_E = 5;
    K_Rx = (2 * 1 + 7 * 3) / 4 = 5.75, K_Ry = 5; eta_x = (2 * 1 - 7 * 3 - 5.75 * (1 - 3)) / 4 = -1.875, eta_y = 0.
    Every weight tells the averages apart, so one taken with another group's weights fails here."""
    col = lambda *v: np.array(v, dtype=np.float64)[:, None]
    r = oracle.grey_coefficients(col(0, 4, 0), col(1, 0, -3), col(0, -2, 0), col(2, 5, 7), col(1, 0, 0))
    want = dict(kappa_B=2.0, kappa_E=5.0, KRx=5.75, KRy=5.0, eta_x=-1.875, eta_y=0.0)
    for k, v in want.items():
        assert r[k][0] == v, (k, r[k][0], v)


def test_grey_eddington_average_special_cases():
    """Eq. 8 with u = f: factors equal in every group average to that factor; E in one group picks that
    group's factor; a hand-worked two-group cell; zero E gives 0."""
    rng = np.random.default_rng(11)
    G, n, c = 4, 6, 29.98
    E = rng.uniform(0.1, 1.0, (G, n))
    f0 = rng.uniform(0.1, 0.5, (3, n))
    N = [np.tile(f0[i], (G, 1)) * c * E for i in range(3)]
    for got, want in zip(oracle.grey_eddington(E, *N, c), f0):
        assert np.allclose(got, want, rtol=4e-16, atol=0)
    E1 = np.zeros((G, n))
    E1[1] = E[1]
    fg = rng.uniform(-0.3, 0.5, (3, G, n))
    N1 = [fg[i] * c * E1 for i in range(3)]
    for i, got in enumerate(oracle.grey_eddington(E1, *N1, c)):
        assert np.allclose(got, fg[i][1], rtol=4e-16, atol=0)
    # two groups, E = (1, 3), f_xx = (0.2, 0.4): <f_xx>_E = (0.2 + 1.2) / 4 = 0.35
    E2 = np.array([[1.0], [3.0]])
    fxx, _, _ = oracle.grey_eddington(E2, np.array([[0.2], [0.4]]) * c * E2, np.zeros((2, 1)), np.zeros((2, 1)), c)
    assert abs(fxx[0] - 0.35) < 1e-15
    assert all(np.all(x == 0) for x in oracle.grey_eddington(np.zeros((G, n)), *N, c))


def _face_geometry(nx, ny):
    nxf = (nx + 1) * ny

    def cells_of(f):
        """(kind, index along the normal, index across): x-face (i, j) or y-face (i, j)."""
        if f < nxf:
            return "x", f % (nx + 1), f // (nx + 1)
        f -= nxf
        return "y", f % nx, f // nx
    return nxf, cells_of


@pytest.mark.parametrize("layout", [0, 1])
def test_upwind_faces_are_the_faces_segments_enter_through(layout):
    """Eq. 16 needs the upwind face of every segment: for the first segment the boundary face of the entry edge,
    otherwise a face of the entered cell that the previous cell touches, on the side the characteristic comes
    from (checked here from the cells and the direction, independently of how the oracle numbers them)."""
    nx, ny = 5, 4
    q = synth.product_quadrature(2, 16)
    geom = oracle.Geometry(nx, ny, 2.5, 1.6, q.mu, q.cos_phi, q.sin_phi, q.w, 0.17, layout, 1 - layout)
    t = oracle.tracks(geom, "double")
    nxf, cells_of = _face_geometry(nx, ny)
    for m in range(q.mu.size):
        dx, dy = q.cos_phi[m], q.sin_phi[m]
        for r in range(t["dir_ray_off"][m], t["dir_ray_off"][m + 1]):
            s0, s1 = t["ray_seg_off"][r], t["ray_seg_off"][r + 1]
            for s in range(s0, s1):
                ix, iy = t["cell"][s] % nx, t["cell"][s] // nx
                kind, a, b = cells_of(t["face"][s])
                if kind == "x":
                    assert b == iy and a == (ix if dx > 0 else ix + 1)
                else:
                    assert a == ix and b == (iy if dy > 0 else iy + 1)
                if s == s0:
                    e = t["entry"][r]
                    normal = a if kind == "x" else b
                    assert (kind, normal) == {0: ("x", 0), 1: ("x", nx), 2: ("y", 0), 3: ("y", ny)}[e]
                else:
                    px, py = t["cell"][s - 1] % nx, t["cell"][s - 1] // nx
                    assert abs(px - ix) <= 1 and abs(py - iy) <= 1 and (px, py) != (ix, iy)
                    if kind == "x":
                        assert px != ix        # crossed a vertical line
                    else:
                        assert px == ix and py != iy


def test_face_moments_equilibrium_closed_form():
    """Homogeneous medium in equilibrium (I = B everywhere), paper layout: the characteristics of direction m
    that cross an interior x-face have widths summing to |face| |d_x| exactly (bands never straddle a vertex),
    so E_f = (B/c) sum_m omega_m |d_x|, N_f = B sum_m omega_m |d_x| Omega Omega, F_f = 0 (Eq. 16 numerators);
    likewise with |d_y| on y-faces."""
    nx, ny = 4, 3
    q = synth.product_quadrature(2, 16)
    geom = oracle.Geometry(nx, ny, 2.0, 1.2, q.mu, q.cos_phi, q.sin_phi, q.w, 0.13, 1, 0)
    G = 2
    Bv = np.array([1.0, 3e-4])
    kap = np.array([0.7, 40.0])
    B = np.repeat(Bv[:, None], nx * ny, 1)
    kappa = np.repeat(kap[:, None], nx * ny, 1)
    bnd = np.repeat(Bv[None, :], 4, 0)
    c = 2.0
    r = oracle.sweep(geom, kappa, B, c, 0.5, bnd, precision="quad", want_I=False, want_faces=True)
    sz = np.sqrt(1 - q.mu ** 2)
    Ox, Oy = sz * q.cos_phi, sz * q.sin_phi
    nxf = (nx + 1) * ny
    xint = [j * (nx + 1) + i for j in range(ny) for i in range(1, nx)]
    yint = [nxf + j * nx + i for j in range(1, ny) for i in range(nx)]
    for faces, wdir in ((xint, np.abs(q.cos_phi)), (yint, np.abs(q.sin_phi))):
        ww = q.w * wdir
        exp = {"face_E": ww.sum() / c, "face_Fx": 0.0, "face_Fy": 0.0, "face_Nxx": (ww * Ox * Ox).sum(),
               "face_Nxy": (ww * Ox * Oy).sum(), "face_Nyy": (ww * Oy * Oy).sum()}
        for k, e in exp.items():
            for g in range(G):
                got = r[k][g, faces] / Bv[g]
                assert np.max(np.abs(got - e)) <= 1e-13 * ww.sum(), (k, g)


@pytest.mark.parametrize("nx,ny,naz,npol", [(2, 1, 4, 2), (2, 2, 8, 1), (3, 2, 8, 2)])
def test_face_moments_brute_force(nx, ny, naz, npol):
    """Eq. 16 away from equilibrium: every characteristic walked with the brute-force geometry and RK4 transport;
    the intensity entering each segment is added, with weight omega w Omega..Omega, to the face it enters through
    (the entry point's grid line: x first, so a vertex counts on the x-face), then averaged over the face length
    (E also divided by c).  Catches a face sum that takes another intensity or another component."""
    rng = np.random.default_rng(7 * nx + 5 * ny + naz + npol)
    lx, ly, sp = 1.0, 0.8, 0.35
    q = synth.product_quadrature(npol, naz)
    geom = make_geom(nx, ny, lx, ly, q, sp)
    G, ncell = 2, nx * ny
    kappa = rng.uniform(0.2, 3.0, (G, ncell))
    B = rng.uniform(0.1, 1.0, (G, ncell))
    bnd = rng.uniform(0.0, 2.0, (4, G))
    c, dt = 1.5, 0.5
    r = oracle.sweep(geom, kappa, B, c, dt, bnd, precision="quad", want_I=False, want_faces=True)
    hx, hy = lx / nx, ly / ny
    nxf = (nx + 1) * ny
    nf = nxf + nx * (ny + 1)
    acc = np.zeros((6, G, nf))
    tol = 1e-9 * max(lx, ly)
    for m in range(q.n):
        cphi, sphi = bf.unit(q.cos_phi[m], q.sin_phi[m])
        sinz = math.sqrt(1 - q.mu[m] ** 2)
        Om = (1.0, sinz * cphi, sinz * sphi)
        fac = (1.0, Om[1], Om[2], Om[1] * Om[1], Om[1] * Om[2], Om[2] * Om[2])
        ts, ws = bf.uniform_offsets(lx, ly, cphi, sphi, sp)
        for t, w in zip(ts, ws):
            segs, edge = bf.ray_segments(nx, ny, lx, ly, cphi, sphi, t)
            I = bnd[edge].copy()
            for cell, L, u in segs:
                px, py = -t * sphi + u * cphi, t * cphi + u * sphi
                ix, iy = cell % nx, cell // nx
                xi = round(px / hx)
                if abs(px - xi * hx) < tol:
                    f = iy * (nx + 1) + xi                       # x-face (line xi, row iy)
                else:
                    f = nxf + round(py / hy) * nx + ix           # y-face (line, column ix)
                for k in range(6):
                    acc[k, :, f] += q.w[m] * w * fac[k] * I
                for g in range(G):
                    kt = kappa[g, cell] + 1 / (c * dt)
                    Q = kappa[g, cell] * B[g, cell] + B[g, cell] / (c * dt)   # I^{n-1} = B
                    I[g], _ = bf.rk4_segment(I[g], Q, kt, L / sinz)
    flen = np.where(np.arange(nf) < nxf, hy, hx)
    names = ("face_E", "face_Fx", "face_Fy", "face_Nxx", "face_Nxy", "face_Nyy")
    scale = np.abs(acc[0]) / flen
    for k, name in enumerate(names):
        want = acc[k] / flen / (c if k == 0 else 1.0)
        got = r[name]
        if k == 0:
            assert np.allclose(got, want, rtol=1e-9, atol=0), name
        else:
            assert np.all(np.abs(got - want) <= 1e-9 * scale + 1e-300), name
