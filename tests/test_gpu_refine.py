"""GPU: multistep runs with the temperature advanced between sweeps (reduced refinement stress).

A cold medium driven at 1 keV from the left edge; T is advanced after every FP64 sweep by the host energy
balance; FP32 and FP64 sweeps on two ray spacings then step through that same T sequence, and the FP32 moments
are held to the FP32 targets against the FP64 ones at every step.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_refinement_multistep_fp32_against_fp64():
    import paper_2305_11998_gb300 as molc
    from paper_2305_11998_gb300 import multistep
    wl = synth.Workload("refine_small", 24, 24, 6.0, 6, 0.001, 100.0, 2, 16, 2, 4, cold_start=True)
    T0 = wl.temperature()
    P = molc.Plan.from_workload(wl)
    Ts = multistep.temperature_sequence(P, wl, T0, steps=wl.steps)
    # the driven edge heats the material, the far side stays near the cold start
    T = Ts[-1].reshape(wl.ny, wl.nx)
    assert T[:, 0].min() > 1.5 * synth.T_COLD and T[:, -1].max() < T[:, 0].min()
    for div in (2, 4):
        Q = molc.Plan.from_workload(wl, spacing=wl.h / div)
        m64 = multistep.run_sequence(Q, wl, Ts, "fp64")
        m32 = multistep.run_sequence(Q, wl, Ts, "fp32")
        for a, b in zip(m32, m64):
            err = multistep.precision_errors(a, b, wl.c)
            assert err["E"] <= 2e-5, (div, err)
            assert max(err["Fx/cE"], err["Fy/cE"], err["Nxy/cE"]) <= 2e-5, (div, err)
            assert max(err["fxx"], err["fxy"], err["fyy"]) <= 1e-6, (div, err)
        assert Q.device_status() == 0
