"""Host FP64 energy balance between sweeps (the multistep coupling; CPU)."""
import math

import numpy as np

import synth
from paper_2305_11998_gb300 import meb


def test_equilibrium_is_a_fixed_point():
    edges = synth.group_edges(17, 0.001, 100.0)
    T = np.array([0.001, 0.05, 0.3, 1.0])
    _, B = synth.material(T, edges)
    E = 4.0 * math.pi * B / synth.C_LIGHT         # radiation in equilibrium with the material
    Tn, _ = meb.advance(T, E, edges, synth.C_LIGHT, 2e-3)
    assert np.max(np.abs(Tn / T - 1)) < 1e-12


def test_residual_vanishes_and_heating_is_monotone():
    edges = synth.group_edges(17, 0.001, 100.0)
    rng = np.random.default_rng(0)
    T_old = np.exp(rng.uniform(np.log(1e-3), 0.0, 50))
    Trad = T_old * np.exp(rng.uniform(-1.0, 1.0, 50))   # a radiation field at another temperature
    _, Brad = synth.material(Trad, edges)
    E = 4.0 * math.pi * Brad / synth.C_LIGHT
    c, dt = synth.C_LIGHT, 2e-3
    T, it = meb.advance(T_old, E, edges, c, dt)
    assert it < 100
    kappa, B = synth.material(T, edges)
    lhs = meb.C_V * (T - T_old) / dt
    rhs = np.sum(kappa * (c * E - 4.0 * math.pi * B), axis=0)
    scale = meb.C_V * T / dt + np.sum(kappa * (c * E + 4.0 * math.pi * B), axis=0)
    assert np.max(np.abs(lhs - rhs) / scale) < 1e-12
    # hotter radiation heats, colder radiation cools, and never past the radiation temperature
    hot = Trad > T_old
    assert np.all(T[hot] >= T_old[hot]) and np.all(T[~hot] <= T_old[~hot])
    assert np.all(T[hot] <= Trad[hot] * (1 + 1e-12)) and np.all(T[~hot] >= Trad[~hot] * (1 - 1e-12))
