"""Pin of the oracle against a hand-worked characteristic (tests/golden/single_ray_3x3.txt, Eqs. 12-13).

The fixture gives one characteristic's cells and in-plane lengths, worked out by hand on a 3 x 3 grid.  The
oracle's characteristic grid must reproduce them, and with B = 0 and I^{n-1} = 0 (so Q = 0) its sweep must give
the pure attenuation: exit intensity I_in exp(-sum_s tau_s) and segment averages I_in,s (1 - e^-tau_s) / tau_s,
tau_s = kappa~ l_s / sin zeta.
"""
import math
import os

import numpy as np

import oracle
import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def load_fixture():
    rows = [ln.split() for ln in open(os.path.join(HERE, "golden", "single_ray_3x3.txt"))
            if ln.strip() and not ln.startswith("#")]
    direction, ray, edge = (int(x) for x in rows[0])
    cells = [int(r[0]) for r in rows[1:]]
    lens = [float(r[1]) * math.sqrt(2.0) for r in rows[1:]]
    return direction, ray, edge, cells, lens


def test_oracle_reproduces_the_hand_worked_characteristic():
    direction, ray, edge, cells, lens = load_fixture()
    q = synth.product_quadrature(1, 4)
    assert abs(q.mu[0] - 0.5) < 1e-15
    geom = oracle.Geometry(3, 3, 3.0, 3.0, q.mu, q.cos_phi, q.sin_phi, q.w, 3.0 * math.sqrt(2.0) / 4.0, 0, 1)
    tr = oracle.tracks(geom, "double")
    r_global = tr["dir_ray_off"][direction] + ray
    s0, s1 = tr["ray_seg_off"][r_global], tr["ray_seg_off"][r_global + 1]
    assert tr["entry"][r_global] == edge
    assert tr["cell"][s0:s1].tolist() == cells
    assert np.allclose(tr["len"][s0:s1], lens, rtol=0, atol=1e-14)

    # pure attenuation along it: kappa per cell, no emission, no previous-step intensity, I_in = 1 on its edge
    G = 1
    kappa = (0.3 + 0.7 * np.arange(9, dtype=float))[None, :]
    B = np.zeros((G, 9))
    bnd = np.zeros((4, G))
    bnd[edge] = 1.0
    c, dt = 29.98, 1.0e15
    res = oracle.sweep(geom, kappa, B, c, dt, bnd, precision="quad", want_exit=True)
    sinz = math.sqrt(3.0) / 2.0
    kt = kappa[0] + 1.0 / (c * dt)
    I = 1.0
    for k, (cell, ln) in enumerate(zip(cells, lens)):
        tau = kt[cell] * ln / sinz
        assert math.isclose(res["I"][s0 + k, 0], I * (-math.expm1(-tau)) / tau, rel_tol=1e-13)
        I *= math.exp(-tau)
    assert math.isclose(res["I_exit"][r_global][0], I, rel_tol=1e-13)
    tau_sum = sum(kt[cell] * ln for cell, ln in zip(cells, lens)) / sinz
    assert math.isclose(I, math.exp(-tau_sum), rel_tol=1e-13)
