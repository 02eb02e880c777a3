"""GPU: multistep runs with the temperature advanced between sweeps (reduced refinement stress).

A cold medium driven at 1 keV from the left edge; T is advanced after every FP64 sweep by the host energy
balance; FP32 and FP64 sweeps on two ray spacings then step through that same T sequence.  Both precisions are
held to their targets against the binary128 oracle stepping through the same sequence (the parity gate of
tests/parity.py), and the FP32 moments against the FP64 ones at every step.
"""
import numpy as np
import pytest

import oracle
import parity
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


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_refinement_steps_against_binary128(prec):
    """The same cold start and temperature sequence (the refinement stress's physics at 24^2, 6 groups, h/2),
    each step of the GPU path against the binary128 oracle fed the same kappa and B.  B changes between steps:
    the oracle's carried deviations are re-referenced to the new B in double (that rounding joins the state
    bound), and the path's stored deviations refer to the previous step's B (the error model's B_ref)."""
    import paper_2305_11998_gb300 as molc
    from paper_2305_11998_gb300 import multistep
    wl = synth.Workload("refine_small", 24, 24, 6.0, 6, 0.001, 100.0, 2, 16, 2, 4, cold_start=True)
    edges = wl.edges()
    P = molc.Plan.from_workload(wl)
    Ts = multistep.temperature_sequence(P, wl, wl.temperature(), steps=wl.steps)
    got = multistep.run_sequence(P, wl, Ts, prec)
    assert P.device_status() == 0
    P.close()
    geom = oracle.Geometry.from_workload(wl)
    cells = oracle.tracks(geom, "double")["cell"]
    bnd = synth.boundary_left_hot(edges)
    dev = err = B_prev = None
    for n in range(1, len(Ts)):
        kappa, B = synth.material(Ts[n - 1], edges)
        if dev is not None:
            jump = (B_prev - B)[:, cells].T
            dev = dev + jump
            err = err + 2 * parity.U64 * (np.abs(dev) + np.abs(jump))
        d = dict(kappa=kappa, B=B, bnd=bnd, c=wl.c, dt=wl.dt)
        r = parity.reference(geom, d, prec, wl.n_polar, I_prev=dev, I_err=err, want_I=True,
                             Bref=B if B_prev is None else B_prev)
        parity.compare(got[n - 1], r, prec, wl.c)
        dev, err, B_prev = r["I"], r["I_err"], B
