"""Pins for the seeded input generator (Planck groups, opacity, quadrature, temperature fields)."""
import math

import numpy as np
import pytest

import synth


def test_planck_groups_sum_to_total():
    # Summed over groups spanning [0, inf) the group Planck intensities give a c T^4 / (4 pi) exactly.
    T = np.array([1e-3, 3e-3, 0.05, 0.3, 1.0, 3.0])
    edges = np.concatenate([[0.0], synth.group_edges(17, 0.001, 100.0), [np.inf]])
    tot = sum(synth.planck_group(T, edges[g], edges[g + 1]) for g in range(len(edges) - 1))
    ref = synth.A_RAD * synth.C_LIGHT * T ** 4 / (4 * math.pi)
    assert np.max(np.abs(tot / ref - 1)) < 1e-14


def test_planck_groups_match_adaptive_quadrature():
    quad = pytest.importorskip("scipy.integrate").quad

    def f(x):
        return x ** 3 * math.exp(-x) / -math.expm1(-x)

    e = synth.group_edges(17, 0.001, 100.0)
    worst = 0.0
    for g in range(17):
        for t in (0.001, 0.003, 0.05, 0.3, 1.0, 3.0):
            a, b = e[g] / t, e[g + 1] / t
            if a > 600:
                continue
            ref = quad(f, a, b, epsabs=0, epsrel=1e-13, limit=400)[0]
            got = synth.planck_fraction_between(np.array([a]), np.array([b]))[0]
            worst = max(worst, abs(got - ref) / ref)
    assert worst < 1e-13


def test_opacity_limits():
    nu = 2.0
    # thin limit nu/T -> 0: kappa -> 27/nu^2 / T ; thick limit: 27/nu^3
    assert synth.opacity(np.array([1e6]), nu)[0] == pytest.approx(27.0 / nu ** 2 / 1e6, rel=1e-6)
    assert synth.opacity(np.array([1e-3]), nu)[0] == pytest.approx(27.0 / nu ** 3, rel=1e-15)


@pytest.mark.parametrize("npol,naz", [(1, 4), (2, 16), (3, 24), (4, 32), (8, 64)])
def test_product_quadrature(npol, naz):
    q = synth.product_quadrature(npol, naz)
    sinz2 = 1 - q.mu ** 2
    assert q.n == npol * naz
    assert abs(q.w.sum() / (4 * math.pi) - 1) < 1e-15
    # odd moments vanish exactly; the set is symmetric under the four reflections and 90-degree rotation
    assert (q.w * q.cos_phi).sum() == pytest.approx(0.0, abs=1e-15)
    S = set(zip(q.cos_phi[:naz], q.sin_phi[:naz]))
    for c, s in zip(q.cos_phi[:naz], q.sin_phi[:naz]):
        assert (-c, -s) in S and (-s, c) in S and (c, -s) in S
    phi = np.arctan2(q.sin_phi[:naz], q.cos_phi[:naz]) % (2 * math.pi)
    assert np.allclose(phi, (np.arange(naz) + 0.5) * 2 * math.pi / naz, atol=1e-14)
    x, W = np.polynomial.legendre.leggauss(npol)
    assert np.allclose(q.mu[::naz], 0.5 * (x + 1), atol=0)
    if npol >= 2:
        # Gauss-Legendre with >= 2 nodes integrates sin^2(zeta) exactly; Chebyshev integrates cos^2(phi)
        assert (q.w * sinz2 * q.cos_phi ** 2).sum() == pytest.approx(4 * math.pi / 3, rel=1e-14)
        assert (q.w * sinz2 * q.cos_phi * q.sin_phi).sum() == pytest.approx(0.0, abs=1e-15)


def test_temperature_field_seeded():
    a = synth.temperature_front(32, 32, 6.0, seed=3)
    b = synth.temperature_front(32, 32, 6.0, seed=3)
    c = synth.temperature_front(32, 32, 6.0, seed=4)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert a.shape == (32, 32)
    assert a.min() >= synth.T_COLD * 0.95 - 1e-15 and a.max() <= synth.T_HOT * 1.05 + 1e-15
    # hot behind the front on the left, cold ahead of it
    assert a[:, 0].mean() > 0.9 and a[:, -1].mean() < 0.01
    three = synth.temperature_front(64, 64, 6.0, seed=0, n_fronts=3)
    assert three.max() > 0.9 and three.min() < 0.01


def test_workload_shapes():
    wl = synth.WORKLOADS["fc16_g4_d32"]
    d = wl.inputs(0)
    assert d["kappa"].shape == (4, 256) and d["B"].shape == (4, 256) and d["bnd"].shape == (4, 4)
    assert np.all(d["kappa"] > 0) and np.all(d["B"] >= 0)
    assert np.all(d["bnd"][1:] == 0) and np.all(d["bnd"][0] > 0)
    assert wl.quadrature().n == 32
    assert len(synth.batch_instances(64)) == 64
